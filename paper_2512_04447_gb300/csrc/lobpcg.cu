// LOBPCG block iteration (the paper's eigensolver; Knyazev's method with the
// Rayleigh-Ritz of Eq. 1), FP64, device-resident.  Per iteration:
//   R = HX - X Theta and residual norms; soft locking of converged bands;
//   W = TPA(R) (Teter-Payne-Allan, the residual formed on the fly in the
//   first FFT pass); W <- W - X <X|W>; HW = H W; column normalisation;
//   Gram matrices of [X W P] (Hermitian, upper tiles only);
//   Cholesky with dropping + two TRSMs + eigensolve + back-substitution;
//   Ritz rotation P <- [W P] C_WP, X <- X C_X + P (and HX, HP alike).
// The host reads back one small vector per iteration (residual norms) plus
// the kept-column count of the Cholesky.
#include <cmath>
#include <algorithm>

#include "rsdft_internal.h"

namespace rsdft {

constexpr int RTHREADS = 256;

__device__ __forceinline__ double block_sum2(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        sh[32] = s;
    }
    __syncthreads();
    return sh[32];
}

// res[b] = ||hx_b - theta_b x_b|| (dV metric); vexp[b] = <x_b|V|x_b>
__global__ void __launch_bounds__(RTHREADS)
k_resid(const double2 *__restrict__ hx, const double2 *__restrict__ x, const double *__restrict__ theta,
        const double *__restrict__ v, long long n, double dV, double *res, double *vexp) {
    __shared__ double sh[33];
    const int b = blockIdx.x;
    const double th = theta[b];
    const double2 *h = hx + (size_t)b * n, *xx = x + (size_t)b * n;
    double s = 0.0, sv = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        const double2 a = h[i], c = xx[i];
        const double rx = a.x - th * c.x, ry = a.y - th * c.y;
        s += rx * rx + ry * ry;
        sv += v[i] * (c.x * c.x + c.y * c.y);
    }
    s = block_sum2(s, sh);
    sv = block_sum2(sv, sh);
    if (threadIdx.x == 0) {
        res[b] = sqrt(s * dV);
        vexp[b] = sv * dV;
    }
}

// t_b = <x_b|T|x_b> = theta_b - <x_b|V|x_b> - sum_aj E_aj |<beta_aj|x_b>|^2, for the
// active bands (compact index j).
__global__ void k_tkin(const double *__restrict__ theta, const double *__restrict__ vexp,
                       const double2 *__restrict__ p, ProjTables pt, const int *__restrict__ act,
                       int na, double *tkin) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= na) return;
    const int b = act[j];
    const int np = pt.natom * pt.nproj;
    double nl = 0.0;
    for (int q = 0; q < np; ++q) {
        const double2 c = p[(size_t)b * np + q];
        nl += pt.e_kb[q] * (c.x * c.x + c.y * c.y);
    }
    tkin[j] = theta[b] - vexp[b] - nl;
}

__global__ void __launch_bounds__(RTHREADS)
k_rownorm(const double2 *__restrict__ a, long long n, double dV, double *out) {
    __shared__ double sh[33];
    const int b = blockIdx.x;
    const double2 *r = a + (size_t)b * n;
    double s = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) s += r[i].x * r[i].x + r[i].y * r[i].y;
    s = block_sum2(s, sh);
    if (threadIdx.x == 0) out[b] = sqrt(s * dV);
}

// a[b] /= nrm[b] and (optionally) a2[b] /= nrm[b]
__global__ void k_scale_rows(double2 *a, double2 *a2, long long n, const double *__restrict__ nrm) {
    const int b = blockIdx.y;
    const double s = 1.0 / nrm[b];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double2 &x = a[(size_t)b * n + i];
        x.x *= s;
        x.y *= s;
        if (a2) {
            double2 &y = a2[(size_t)b * n + i];
            y.x *= s;
            y.y *= s;
        }
    }
}

// dst[j] = src[act[j]] (and dst2/src2 alike)
__global__ void k_gather_rows(const double2 *__restrict__ src, const double2 *__restrict__ src2,
                              const int *__restrict__ act, long long n, double2 *__restrict__ dst,
                              double2 *__restrict__ dst2) {
    const int j = blockIdx.y;
    const int b = act[j];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        dst[(size_t)j * n + i] = src[(size_t)b * n + i];
        dst2[(size_t)j * n + i] = src2[(size_t)b * n + i];
    }
}

// w[j] = hx[act[j]] - theta[act[j]] x[act[j]]
__global__ void k_residual_rows(const double2 *__restrict__ hx, const double2 *__restrict__ x,
                                const double *__restrict__ theta, const int *__restrict__ act,
                                long long n, double2 *__restrict__ w) {
    const int j = blockIdx.y;
    const int b = act[j];
    const double th = theta[b];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double2 h = hx[(size_t)b * n + i], c = x[(size_t)b * n + i];
        w[(size_t)j * n + i] = make_double2(h.x - th * c.x, h.y - th * c.y);
    }
}

rsdft_status colnorms(rsdft_ctx *ctx, const double2 *a, int nb, double *out, cudaStream_t st) {
    if (nb <= 0) return RSDFT_OK;
    k_rownorm<<<nb, RTHREADS, 0, st>>>(a, ctx->n, ctx->dV, out);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_rownorm");
    return RSDFT_OK;
}

static rsdft_status scale_rows(rsdft_ctx *ctx, double2 *a, double2 *a2, int nb, const double *nrm,
                               cudaStream_t st) {
    if (nb <= 0) return RSDFT_OK;
    dim3 g(std::min(cdiv(ctx->n, 256), 1024), nb);
    k_scale_rows<<<g, 256, 0, st>>>(a, a2, ctx->n, nrm);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_scale_rows");
    return RSDFT_OK;
}

// Per-phase CUDA-event timing of one iteration.
struct PhaseEvents {
    cudaEvent_t ev[7] = {};
    bool pending = false;
    rsdft_status init(rsdft_ctx *ctx) {
        for (auto &e : ev) RS_CUDA(ctx, cudaEventCreate(&e));
        return RSDFT_OK;
    }
    void destroy() {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
    }
    void collect(rsdft_lobpcg_stats *s) {
        if (!pending || !s) return;
        float t[6];
        for (int i = 0; i < 6; ++i) {
            t[i] = 0.f;
            cudaEventElapsedTime(&t[i], ev[i], ev[i + 1]);
        }
        s->ms_precond += t[0];
        s->ms_hpsi += t[1];
        s->ms_other += t[2];
        s->ms_gram += t[3];
        s->ms_dense += t[4];
        s->ms_rotate += t[5];
        pending = false;
    }
};

static rsdft_status lobpcg64(rsdft_ctx *ctx, double2 *x_user, int m, const rsdft_lobpcg_opts &o,
                             double *eig_host, double *res_host, rsdft_lobpcg_stats *stats,
                             cudaStream_t st) {
    RS_TRY(ensure_workspace(ctx, m));
    Workspace &w = ctx->ws;
    const long long n = ctx->n;
    const double dV = ctx->dV;
    const int nconv = (o.nconv <= 0 || o.nconv > m) ? m : o.nconv;
    double2 *X = w.X, *HX = w.HX, *Xn = w.Xn, *HXn = w.HXn;
    double *hres = w.hbuf;                    // [m]
    int *hact = reinterpret_cast<int *>(w.hbuf + m);   // [m]
    RS_CUDA(ctx, cudaMemcpyAsync(X, x_user, (size_t)m * n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    RS_TRY(apply_h64(ctx, X, HX, m, st));
    // initial Rayleigh-Ritz on span(X)
    {
        RowBlocks Y{{X, nullptr, nullptr}, {m, 0, 0}};
        RowBlocks HY{{HX, nullptr, nullptr}, {m, 0, 0}};
        RS_TRY(gram(ctx, Y, Y, w.GS, m, true, dV, st));
        RS_TRY(gram(ctx, Y, HY, w.GH, m, true, dV, st));
        int nd = 0;
        RS_TRY(rayleigh_ritz(ctx, w.GH, w.GS, m, m, o.pivot_tol, w.theta, w.Cfull, &nd, st));
        RS_TRY(rotate(ctx, Y, w.Cfull, m, m, nullptr, 1, Xn, nullptr, st));
        RS_TRY(rotate(ctx, HY, w.Cfull, m, m, nullptr, 1, HXn, nullptr, st));
        std::swap(X, Xn);
        std::swap(HX, HXn);
    }
    PhaseEvents pe;
    if (stats) RS_TRY(pe.init(ctx));
    bool haveP = false;
    int it = 0, dropped = 0;
    bool converged = false;
    rsdft_status result = RSDFT_OK;
    for (;;) {
        k_resid<<<m, RTHREADS, 0, st>>>(HX, X, w.theta, ctx->v, n, dV, w.res, w.vexp);
        count_launch(ctx);
        RS_LAUNCHED(ctx, "k_resid");
        RS_CUDA(ctx, cudaMemcpyAsync(hres, w.res, m * sizeof(double), cudaMemcpyDeviceToHost, st));
        RS_CUDA(ctx, cudaStreamSynchronize(st));
        pe.collect(stats);
        double rmax = 0.0;
        bool bad = false;
        for (int b = 0; b < m; ++b) {
            if (!std::isfinite(hres[b])) bad = true;
            if (b < nconv) rmax = std::max(rmax, hres[b]);
        }
        if (bad) { result = fail(ctx, RSDFT_E_NUMERIC, "non-finite residual at iteration %d", it); break; }
        converged = rmax <= o.tol;
        if (converged || it >= o.maxit) break;
        int na = 0;
        for (int b = 0; b < m; ++b)
            if (hres[b] > o.lock_tol) hact[na++] = b;
        if (na == 0) break;
        RS_CUDA(ctx, cudaMemcpyAsync(w.act, hact, na * sizeof(int), cudaMemcpyHostToDevice, st));
        if (stats) RS_CUDA(ctx, cudaEventRecord(pe.ev[0], st));
        // ---- preconditioned residuals W (compact over the active bands)
        RS_TRY(project(ctx, X, w.proj, m, st));
        k_tkin<<<cdiv(na, 128), 128, 0, st>>>(w.theta, w.vexp, w.proj, ctx->pt, w.act, na, w.tkin);
        count_launch(ctx);
        RS_LAUNCHED(ctx, "k_tkin");
        if (o.precond == RSDFT_PRECOND_TPA) {
            RS_TRY(fft_xy_forward(ctx, Src::Residual, HX, X, w.theta, w.act, nullptr, w.T1, na, st));
            RS_TRY(fft_z_mid(ctx, Mid::Tpa, w.T1, w.tkin, na, st));
            RS_TRY(fft_xy_inverse(ctx, w.T1, nullptr, nullptr, w.W, nullptr, na, st));
        } else {
            dim3 g(std::min(cdiv(n, 256), 1024), na);
            k_residual_rows<<<g, 256, 0, st>>>(HX, X, w.theta, w.act, n, w.W);
            count_launch(ctx);
            RS_LAUNCHED(ctx, "k_residual_rows");
        }
        // W <- W - X <X|W>
        {
            RowBlocks YX{{X, nullptr, nullptr}, {m, 0, 0}};
            RowBlocks YW{{w.W, nullptr, nullptr}, {na, 0, 0}};
            RS_TRY(gram(ctx, YX, YW, w.C, na, false, dV, st));
            RS_TRY(rotate(ctx, YX, w.C, na, na, w.W, -1, w.W, nullptr, st));
        }
        if (stats) RS_CUDA(ctx, cudaEventRecord(pe.ev[1], st));
        RS_TRY(apply_h64(ctx, w.W, w.HW, na, st));
        if (stats) RS_CUDA(ctx, cudaEventRecord(pe.ev[2], st));
        RS_TRY(colnorms(ctx, w.W, na, w.nrm, st));
        RS_TRY(scale_rows(ctx, w.W, w.HW, na, w.nrm, st));
        int np_ = 0;
        if (haveP) {
            dim3 g(std::min(cdiv(n, 256), 1024), na);
            k_gather_rows<<<g, 256, 0, st>>>(w.P, w.HP, w.act, n, w.Pn, w.HPn);
            count_launch(ctx);
            RS_LAUNCHED(ctx, "k_gather_rows");
            RS_TRY(colnorms(ctx, w.Pn, na, w.nrm, st));
            RS_TRY(scale_rows(ctx, w.Pn, w.HPn, na, w.nrm, st));
            np_ = na;
        }
        if (stats) RS_CUDA(ctx, cudaEventRecord(pe.ev[3], st));
        const int k = m + na + np_;
        RowBlocks Y{{X, w.W, w.Pn}, {m, na, np_}};
        RowBlocks HY{{HX, w.HW, w.HPn}, {m, na, np_}};
        RS_TRY(gram(ctx, Y, Y, w.GS, k, true, dV, st));
        RS_TRY(gram(ctx, Y, HY, w.GH, k, true, dV, st));
        if (stats) RS_CUDA(ctx, cudaEventRecord(pe.ev[4], st));
        int nd = 0;
        RS_TRY(rayleigh_ritz(ctx, w.GH, w.GS, k, m, o.pivot_tol, w.lam, w.Cfull, &nd, st));
        dropped += nd;
        if (stats) RS_CUDA(ctx, cudaEventRecord(pe.ev[5], st));
        RS_TRY(rotate(ctx, Y, w.Cfull, m, m, nullptr, 1, Xn, w.P, st));
        RS_TRY(rotate(ctx, HY, w.Cfull, m, m, nullptr, 1, HXn, w.HP, st));
        if (stats) {
            RS_CUDA(ctx, cudaEventRecord(pe.ev[6], st));
            pe.pending = true;
        }
        RS_CUDA(ctx, cudaMemcpyAsync(w.theta, w.lam, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
        std::swap(X, Xn);
        std::swap(HX, HXn);
        haveP = true;
        ++it;
    }
    if (stats) {
        RS_CUDA(ctx, cudaStreamSynchronize(st));
        pe.collect(stats);
        pe.destroy();
        stats->iterations = it;
        stats->converged = converged ? 1 : 0;
        stats->dropped = dropped;
    }
    // keep the workspace pointers consistent with the swaps
    w.X = X; w.Xn = Xn; w.HX = HX; w.HXn = HXn;
    RS_CUDA(ctx, cudaMemcpyAsync(x_user, X, (size_t)m * n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    if (eig_host) RS_CUDA(ctx, cudaMemcpyAsync(eig_host, w.theta, m * sizeof(double), cudaMemcpyDeviceToHost, st));
    RS_CUDA(ctx, cudaStreamSynchronize(st));
    if (res_host) memcpy(res_host, hres, m * sizeof(double));
    if (result != RSDFT_OK) return result;
    return converged || o.tol <= 0.0 ? RSDFT_OK : RSDFT_E_NOT_CONVERGED;
}

rsdft_status lobpcg_run(rsdft_ctx *ctx, double2 *x, int m, const rsdft_lobpcg_opts &o,
                        double *eig_host, double *res_host, rsdft_lobpcg_stats *stats,
                        cudaStream_t st) {
    return lobpcg64(ctx, x, m, o, eig_host, res_host, stats, st);
}

}  // namespace rsdft

using namespace rsdft;

extern "C" {

void rsdft_lobpcg_default_opts(rsdft_lobpcg_opts *o) {
    if (!o) return;
    o->maxit = 100;
    o->tol = 1e-6;
    o->nconv = 0;
    o->precond = RSDFT_PRECOND_TPA;
    o->precision = RSDFT_FP64;
    o->lock_tol = 1e-10;
    o->pivot_tol = 1e-8;
}

rsdft_status rsdft_lobpcg(rsdft_ctx *ctx, void *x_dev, int nband, const rsdft_lobpcg_opts *opts,
                          double *eig_host, double *resnorm_host, rsdft_lobpcg_stats *stats,
                          void *stream) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (!x_dev || nband <= 0 || 3LL * nband > ctx->n)
        return fail(ctx, RSDFT_E_INVALID, "need x and 0 < nband <= n/3");
    rsdft_lobpcg_opts o;
    rsdft_lobpcg_default_opts(&o);
    if (opts) o = *opts;
    if (o.maxit < 0 || !(o.tol >= 0.0) || !(o.pivot_tol >= 0.0) || !(o.lock_tol >= 0.0))
        return fail(ctx, RSDFT_E_INVALID, "bad LOBPCG options");
    if (o.precision != RSDFT_FP64) return fail(ctx, RSDFT_E_INVALID, "only RSDFT_FP64 is available");
    if (o.precond != RSDFT_PRECOND_TPA && o.precond != RSDFT_PRECOND_NONE)
        return fail(ctx, RSDFT_E_INVALID, "unknown preconditioner");
    if (stats) *stats = rsdft_lobpcg_stats{};
    return lobpcg_run(ctx, (double2 *)x_dev, nband, o, eig_host, resnorm_host, stats, as_stream(stream));
}

}  // extern "C"
