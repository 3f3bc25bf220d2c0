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
#include <algorithm>
#include <atomic>
#include <thread>
#include <cmath>
#include <type_traits>

#include "rsdft_internal.h"

namespace rsdft {

constexpr int RTHREADS = 256;
// FP32 data path: Gram entries carry ~1e-7 relative error, and the generalised
// eigenproblem divides the G_H error by the smallest G_S eigenvalue it keeps;
// a 1e-3 pivot floor bounds that amplification, and bands at the FP32 residual
// floor are soft-locked.
constexpr double PIVOT_TOL_FP32 = 1e-3;
constexpr double LOCK_TOL_FP32 = 1e-6;
// HP is carried by the rotation, not recomputed: its FP32 rounding is of the
// order eps32 |HW| |C|, so after normalising a direction p of norm |p| the
// relative error of H p grows like eps32 / |p|.  Near convergence |p| falls to
// the residual level and the magnified error produces spurious low Ritz
// values; P columns with |p| <= 1e-4 therefore leave the basis in the FP32
// phase (the FP64 phase keeps every P column).  On the 24^3 diamond cell an
// FP32 run diverged with a 3e-6 threshold and stayed at 5e-8 Ha with 1e-5; 1e-4
// keeps a factor 10 of margin while leaving unconverged bands their P.
constexpr double P_DROP_FP32 = 1e-4;
// Lowest residual the refinement with FP32 corrections is asked for; tighter
// tolerances are finished by FP64 iterations (asked for 1e-10, it ran 288
// iterations on an SCF step of the 64^3 cell and diverged; the FP64-accurate
// products of its couplings on the FP32 pipe carry ~2^-46 relative errors,
// which over gaps of 1e-3 Ha reach the 1e-9 Ha residual level).  And at most
// REFINE32_MAXIT of its iterations before the FP64 iteration takes over.
constexpr double REFINE32_FLOOR = 1e-7;
constexpr int REFINE32_MAXIT = 30;

__device__ __forceinline__ double block_sum2(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double s = lane < nw ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) sh[32] = s;
    }
    __syncthreads();
    return sh[32];
}

// Row reductions over slices: grid (S, rows), each CTA sums one slice of one row
// into part[row][S]; a small kernel finishes the sums.  FP64 blocks accumulate in
// FP64; FP32 blocks (mixed form) form each term in FP32, add runs of 32 terms in
// FP32 and the run sums in FP64 (relative error ~1e-6 on the norm), which keeps
// the FP64 pipe out of the inner loop.
// (slice lengths are even, so that FP32 rows of even n split into 16-byte pairs)
__device__ __forceinline__ void slice_of(long long n, int S, int s, long long &i0, long long &i1) {
    const long long c = ((n + S - 1) / S + 1) & ~1LL;
    i0 = (long long)s * c;
    i1 = i0 + c < n ? i0 + c : n;
}

// part[b][s] = (sum |hx_b - theta_b x_b|^2, sum V |x_b|^2) over slice s
template <typename V>
__global__ void __launch_bounds__(RTHREADS)
k_resid_part(const V *__restrict__ hx, const V *__restrict__ x, const double *__restrict__ theta,
             const double *__restrict__ v64, const float *__restrict__ v32, long long n, int S,
             double2 *__restrict__ part) {
    __shared__ double sh[33];
    const int s_ = blockIdx.x, b = blockIdx.y;
    long long i0, i1;
    slice_of(n, S, s_, i0, i1);
    const V *h = hx + (size_t)b * n, *xx = x + (size_t)b * n;
    double s = 0.0, sv = 0.0;
    if constexpr (std::is_same<V, float2>::value) {
        const float th = (float)theta[b];
        if ((n & 1) == 0) {
            // pairs of points as 16-byte loads, 16 pairs per thread in flight, each
            // run of 32 terms summed in FP32 and the runs in FP64
            const float4 *h4 = reinterpret_cast<const float4 *>(h), *x4 = reinterpret_cast<const float4 *>(xx);
            const float2 *v2 = reinterpret_cast<const float2 *>(v32);
            const long long j0 = i0 >> 1, j1 = i1 >> 1;
            for (long long jb = j0 + threadIdx.x; jb < j1; jb += 16LL * blockDim.x) {
                float a32 = 0.0f, v32s = 0.0f;
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const long long j = jb + (long long)u * blockDim.x;
                    if (j < j1) {
                        const float4 a = h4[j], c = x4[j];
                        const float2 vv = v2[j];
                        const float rx = a.x - th * c.x, ry = a.y - th * c.y;
                        const float rz = a.z - th * c.z, rw = a.w - th * c.w;
                        a32 += rx * rx + ry * ry + rz * rz + rw * rw;
                        v32s += vv.x * (c.x * c.x + c.y * c.y) + vv.y * (c.z * c.z + c.w * c.w);
                    }
                }
                s += a32;
                sv += v32s;
            }
        } else {
            float a32 = 0.0f, v32s = 0.0f;
            int cnt = 0;
            for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
                const float2 a = h[i], c = xx[i];
                const float rx = a.x - th * c.x, ry = a.y - th * c.y;
                a32 += rx * rx + ry * ry;
                v32s += v32[i] * (c.x * c.x + c.y * c.y);
                if (++cnt == 32) {
                    s += a32;
                    sv += v32s;
                    a32 = v32s = 0.0f;
                    cnt = 0;
                }
            }
            s += a32;
            sv += v32s;
        }
    } else {
        const double th = theta[b];
        for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            const V a = h[i], c = xx[i];
            const double rx = a.x - th * c.x, ry = a.y - th * c.y;
            s += rx * rx + ry * ry;
            sv += v64[i] * (c.x * c.x + c.y * c.y);
        }
    }
    s = block_sum2(s, sh);
    sv = block_sum2(sv, sh);
    if (threadIdx.x == 0) part[(size_t)b * S + s_] = make_double2(s, sv);
}

// res[b] = ||hx_b - theta_b x_b|| (dV metric); vexp[b] = <x_b|V|x_b>
__global__ void k_resid_fin(const double2 *__restrict__ part, int S, int m, double dV, double *res,
                            double *vexp) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= m) return;
    double s = 0.0, sv = 0.0;
    for (int q = 0; q < S; ++q) {
        s += part[(size_t)b * S + q].x;
        sv += part[(size_t)b * S + q].y;
    }
    res[b] = sqrt(s * dV);
    vexp[b] = sv * dV;
}

// part[b][s] = sum |a_b|^2 over slice s
template <typename V>
__global__ void __launch_bounds__(RTHREADS)
k_rownorm_part(const V *__restrict__ a, long long n, int S, double *__restrict__ part) {
    __shared__ double sh[33];
    const int s_ = blockIdx.x, b = blockIdx.y;
    long long i0, i1;
    slice_of(n, S, s_, i0, i1);
    const V *r = a + (size_t)b * n;
    double s = 0.0;
    if constexpr (std::is_same<V, float2>::value) {
        if ((n & 1) == 0) {   // as in k_resid_part
            const float4 *r4 = reinterpret_cast<const float4 *>(r);
            const long long j0 = i0 >> 1, j1 = i1 >> 1;
            for (long long jb = j0 + threadIdx.x; jb < j1; jb += 16LL * blockDim.x) {
                float a32 = 0.0f;
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const long long j = jb + (long long)u * blockDim.x;
                    if (j < j1) {
                        const float4 v = r4[j];
                        a32 += v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w;
                    }
                }
                s += a32;
            }
        } else {
            float a32 = 0.0f;
            int cnt = 0;
            for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
                const float2 v = r[i];
                a32 += v.x * v.x + v.y * v.y;
                if (++cnt == 32) {
                    s += a32;
                    a32 = 0.0f;
                    cnt = 0;
                }
            }
            s += a32;
        }
    } else {
        for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
            const double x = r[i].x, y = r[i].y;
            s += x * x + y * y;
        }
    }
    s = block_sum2(s, sh);
    if (threadIdx.x == 0) part[(size_t)b * S + s_] = s;
}

__global__ void k_rownorm_fin(const double *__restrict__ part, int S, int rows, double dV, double *out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= rows) return;
    double s = 0.0;
    for (int q = 0; q < S; ++q) s += part[(size_t)b * S + q];
    out[b] = sqrt(s * dV);
}

// slices per row: about 8 CTAs per SM in total, slices of at least 4096 points
static int row_slices(const rsdft_ctx *ctx, int rows) {
    const int want = cdiv(8 * ctx->num_sms, std::max(rows, 1));
    const int most = (int)std::max(1LL, ctx->n / 4096);
    return std::max(1, std::min(std::min(want, most), 64));
}

template <typename V>
static rsdft_status resid_norms(rsdft_ctx *ctx, const V *hx, const V *x, int m, cudaStream_t st) {
    Workspace &w = ctx->ws;
    const int S = row_slices(ctx, m);
    double2 *part = w.gram_part;   // free between Gram calls
    k_resid_part<V><<<dim3(S, m), RTHREADS, 0, st>>>(hx, x, w.theta, ctx->v, ctx->v32, ctx->n, S, part);
    k_resid_fin<<<cdiv(m, 128), 128, 0, st>>>(part, S, m, ctx->dV, w.res, w.vexp);
    count_launch(ctx, 2);
    RS_LAUNCHED(ctx, "k_resid");
    return RSDFT_OK;
}

template <typename V>
static rsdft_status row_norms(rsdft_ctx *ctx, const V *a, int rows, double *out, cudaStream_t st) {
    if (rows <= 0) return RSDFT_OK;
    const int S = row_slices(ctx, rows);
    double *part = reinterpret_cast<double *>(ctx->ws.gram_part);
    k_rownorm_part<V><<<dim3(S, rows), RTHREADS, 0, st>>>(a, ctx->n, S, part);
    k_rownorm_fin<<<cdiv(rows, 128), 128, 0, st>>>(part, S, rows, ctx->dV, out);
    count_launch(ctx, 2);
    RS_LAUNCHED(ctx, "k_rownorm");
    return RSDFT_OK;
}

// t_b = <x_b|T|x_b> = theta_b - <x_b|V|x_b> - sum_aj E_aj |<beta_aj|x_b>|^2, for the
// active bands (compact index j).
template <typename V>
__global__ void k_tkin(const double *__restrict__ theta, const double *__restrict__ vexp,
                       const V *__restrict__ p, ProjTables pt, const int *__restrict__ act,
                       int na, double *tkin) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= na) return;
    const int b = act[j];
    const int np = pt.natom * pt.nproj;
    double nl = 0.0;
    for (int q = 0; q < np; ++q) {
        const V c = p[(size_t)b * np + q];
        nl += pt.e_kb[q] * ((double)c.x * c.x + (double)c.y * c.y);
    }
    tkin[j] = theta[b] - vexp[b] - nl;
}

// a[b] /= nrm[b] and (optionally) a2[b] /= nrm[b]
template <typename V>
__global__ void k_scale_rows(V *a, V *a2, long long n, const double *__restrict__ nrm) {
    using T = decltype(V{}.x);
    const int b = blockIdx.y;
    // one reciprocal per thread: FP32 for FP32 rows (an FP64 division costs
    // ~640 cycles per warp here), FP64 for FP64 rows
    T s;
    if constexpr (std::is_same<T, float>::value) s = 1.0f / (float)nrm[b];
    else s = 1.0 / nrm[b];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        V &x = a[(size_t)b * n + i];
        x.x *= s;
        x.y *= s;
        if (a2) {
            V &y = a2[(size_t)b * n + i];
            y.x *= s;
            y.y *= s;
        }
    }
}

// dst[j] = src[act[j]] (and dst2/src2 alike)
template <typename V>
__global__ void k_gather_rows(const V *__restrict__ src, const V *__restrict__ src2,
                              const int *__restrict__ act, long long n, V *__restrict__ dst,
                              V *__restrict__ dst2) {
    const int j = blockIdx.y;
    const int b = act[j];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        dst[(size_t)j * n + i] = src[(size_t)b * n + i];
        dst2[(size_t)j * n + i] = src2[(size_t)b * n + i];
    }
}

// w[j] = hx[act[j]] - theta[act[j]] x[act[j]]
template <typename V>
__global__ void k_residual_rows(const V *__restrict__ hx, const V *__restrict__ x,
                                const double *__restrict__ theta, const int *__restrict__ act,
                                long long n, V *__restrict__ w) {
    using T = decltype(V{}.x);
    const int j = blockIdx.y;
    const int b = act[j];
    const T th = (T)theta[b];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const V h = hx[(size_t)b * n + i], c = x[(size_t)b * n + i];
        V o;
        o.x = h.x - th * c.x;
        o.y = h.y - th * c.y;
        w[(size_t)j * n + i] = o;
    }
}

template <typename A, typename B>
__global__ void k_convert(const A *__restrict__ in, long long cnt, B *__restrict__ out) {
    using T = decltype(B{}.x);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (long long)gridDim.x * blockDim.x) {
        B o;
        o.x = (T)in[i].x;
        o.y = (T)in[i].y;
        out[i] = o;
    }
}

// theta_b = Re<x_b|hx_b> / <x_b|x_b> (FP64): slice partials, then one thread per band
__global__ void __launch_bounds__(RTHREADS)
k_rq_part(const double2 *__restrict__ hx, const double2 *__restrict__ x, long long n, int S,
          double2 *__restrict__ part) {
    __shared__ double sh[33];
    const int s_ = blockIdx.x, b = blockIdx.y;
    long long i0, i1;
    slice_of(n, S, s_, i0, i1);
    const double2 *h = hx + (size_t)b * n, *xx = x + (size_t)b * n;
    double s = 0.0, q = 0.0;
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const double2 a = h[i], c = xx[i];
        s = fma(c.x, a.x, fma(c.y, a.y, s));
        q = fma(c.x, c.x, fma(c.y, c.y, q));
    }
    s = block_sum2(s, sh);
    q = block_sum2(q, sh);
    if (threadIdx.x == 0) part[(size_t)b * S + s_] = make_double2(s, q);
}

__global__ void k_rq_fin(const double2 *__restrict__ part, int S, int m, double *theta) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= m) return;
    double s = 0.0, q = 0.0;
    for (int j = 0; j < S; ++j) {
        s += part[(size_t)b * S + j].x;
        q += part[(size_t)b * S + j].y;
    }
    theta[b] = s / q;
}

// g[m + j][i] = conj(g[i][m + j]) for i < m, j < nwp, in both matrices (ld k)
__global__ void k_mirror_block(double2 *gs, double2 *gh, int k, int m, int nwp) {
    const int i = blockIdx.x * 32 + threadIdx.x;
    for (int j = blockIdx.y * 32 + threadIdx.y; j < min(nwp, (int)(blockIdx.y + 1) * 32); j += blockDim.y) {
        if (i >= m) continue;
        const double2 a = gs[(size_t)i * k + m + j], b = gh[(size_t)i * k + m + j];
        gs[(size_t)(m + j) * k + i] = make_double2(a.x, -a.y);
        gh[(size_t)(m + j) * k + i] = make_double2(b.x, -b.y);
    }
}

// The m x m leading blocks of gs and gh (ld k) made Hermitian: the upper
// triangle mirrored into the lower one, real diagonal.
__global__ void k_herm_block(double2 *gs, double2 *gh, int k, int m) {
    const int i = blockIdx.x * 32 + threadIdx.x;
    for (int j = blockIdx.y * 32 + threadIdx.y; j < min(m, (int)(blockIdx.y + 1) * 32); j += blockDim.y) {
        if (i >= m || j > i) continue;
        if (j == i) {
            gs[(size_t)i * k + i].y = 0.0;
            gh[(size_t)i * k + i].y = 0.0;
            continue;
        }
        const double2 a = gs[(size_t)j * k + i], b = gh[(size_t)j * k + i];
        gs[(size_t)i * k + j] = make_double2(a.x, -a.y);
        gh[(size_t)i * k + j] = make_double2(b.x, -b.y);
    }
}

// out += in, FP32 values added to an FP64 block
__global__ void k_add_f32(double2 *out, const float2 *__restrict__ in, long long cnt) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (long long)gridDim.x * blockDim.x) {
        const float2 a = in[i];
        double2 o = out[i];
        o.x += (double)a.x;
        o.y += (double)a.y;
        out[i] = o;
    }
}

// Precision dispatch of the building blocks.
template <typename V> struct Ops;
template <> struct Ops<double2> {
    static rsdft_status apply_h(rsdft_ctx *c, const double2 *x, double2 *h, int nb, cudaStream_t st) {
        return apply_h64(c, x, h, nb, st);
    }
    static rsdft_status project(rsdft_ctx *c, const double2 *x, double2 *p, int nb, cudaStream_t st) {
        return rsdft::project(c, x, p, nb, st);
    }
    static rsdft_status tpa(rsdft_ctx *c, const double2 *hx, const double2 *x, const double *th,
                            const int *act, const double *tk, double2 *t1, double2 *w, int na,
                            cudaStream_t st) {
        RS_TRY(fft_xy_forward(c, Src::Residual, hx, x, th, act, nullptr, t1, na, st));
        RS_TRY(fft_z_mid(c, Mid::Tpa, t1, tk, na, st));
        return fft_xy_inverse(c, t1, nullptr, nullptr, w, nullptr, na, st);
    }
    static rsdft_status gram(rsdft_ctx *c, const RowBlocks &A, const RowBlocks &B, double2 *g, int ldg,
                             bool herm, double sc, cudaStream_t st) {
        return rsdft::gram(c, A, B, g, ldg, herm, sc, st);
    }
    static rsdft_status rotate(rsdft_ctx *c, const RowBlocks &Y, const double2 *cf, int ldc, int m,
                               const double2 *base, int sign, double2 *o0, double2 *o1, cudaStream_t st) {
        return rsdft::rotate(c, Y, cf, ldc, m, base, sign, o0, o1, st);
    }
};
template <> struct Ops<float2> {
    static rsdft_status apply_h(rsdft_ctx *c, const float2 *x, float2 *h, int nb, cudaStream_t st) {
        return apply_h32(c, x, h, nb, st);
    }
    static rsdft_status project(rsdft_ctx *c, const float2 *x, float2 *p, int nb, cudaStream_t st) {
        return project32(c, x, p, nb, st);
    }
    static rsdft_status tpa(rsdft_ctx *c, const float2 *hx, const float2 *x, const double *th,
                            const int *act, const double *tk, float2 *t1, float2 *w, int na,
                            cudaStream_t st) {
        RS_TRY(fft_xy_forward32(c, Src::Residual, hx, x, th, act, t1, na, st));
        RS_TRY(fft_z_mid32(c, Mid::Tpa, t1, tk, na, st));
        return fft_xy_inverse32(c, t1, nullptr, nullptr, w, na, st);
    }
    static rsdft_status gram(rsdft_ctx *c, const RowBlocksT<float2> &A, const RowBlocksT<float2> &B,
                             double2 *g, int ldg, bool herm, double sc, cudaStream_t st) {
        return gram32(c, A, B, g, ldg, herm, sc, st);
    }
    static rsdft_status rotate(rsdft_ctx *c, const RowBlocksT<float2> &Y, const double2 *cf, int ldc,
                               int m, const float2 *base, int sign, float2 *o0, float2 *o1,
                               cudaStream_t st) {
        return rotate32(c, Y, cf, ldc, m, base, sign, o0, o1, st);
    }
};

rsdft_status colnorms(rsdft_ctx *ctx, const double2 *a, int nb, double *out, cudaStream_t st) {
    if (nb <= 0) return RSDFT_OK;
    return row_norms<double2>(ctx, a, nb, out, st);
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

// G_S = <Y|Y> and G_H = <Y|HY> (Hermitian, ld k): CUDA-core kernels, or for FP32
// blocks with tc set, one tensor-core launch for both.
template <typename V>
static rsdft_status gram_pair(rsdft_ctx *ctx, const RowBlocksT<V> &Y, const RowBlocksT<V> &HY,
                              double2 *gs, double2 *gh, int k, bool tc, cudaStream_t st) {
    if constexpr (std::is_same<V, float2>::value) {
        if (tc) return gram_tc_sh(ctx, Y, HY, gs, gh, k, st);
    }
    RS_TRY(Ops<V>::gram(ctx, Y, Y, gs, k, true, ctx->dV, st));
    return Ops<V>::gram(ctx, Y, HY, gh, k, true, ctx->dV, st);
}

// the double-float cluster tridiagonalisation in the subspace eigensolves
static bool dense_df(const rsdft_lobpcg_opts &o) {
    return o.dense == RSDFT_DENSE_DF || (o.dense == RSDFT_DENSE_AUTO && o.precision == RSDFT_MIXED);
}

struct RunState {
    int iterations = 0;
    int dropped = 0;
    bool converged = false;   // max residual over nconv <= stop_tol
    bool haveP = false;       // P and HP hold the last iteration's directions
};

// One LOBPCG run in precision V on the workspace.  x_in / x_out: [m][n] V.
// Stops when the max residual over the first nconv bands is <= stop_tol, after
// maxit iterations, when every band is soft-locked, or (stagnation = true)
// when the max residual fell by less than 10% in each of 3 iterations.
template <typename V>
static rsdft_status lobpcg_t(rsdft_ctx *ctx, const V *x_in, V *x_out, int m,
                             const rsdft_lobpcg_opts &o, double stop_tol, int maxit, bool stagnation,
                             RunState &rs, double *hres, rsdft_lobpcg_stats *stats, cudaStream_t st) {
    using Blocks = RowBlocksT<V>;
    Workspace &w = ctx->ws;
    const long long n = ctx->n;
    const double dV = ctx->dV;
    const int nconv = (o.nconv <= 0 || o.nconv > m) ? m : o.nconv;
    V *X = (V *)w.X, *HX = (V *)w.HX, *Xn = (V *)w.Xn, *HXn = (V *)w.HXn;
    V *W = (V *)w.W, *HW = (V *)w.HW, *P = (V *)w.P, *HP = (V *)w.HP;
    V *Pn = (V *)w.Pn, *HPn = (V *)w.HPn, *T1 = (V *)w.T1;
    V *proj = (V *)w.proj;
    int *hact = reinterpret_cast<int *>(w.hbuf + m);
    double *hpn = w.hbuf + 2 * m;                         // |P_b| (FP32 phase)
    int *hactp = reinterpret_cast<int *>(w.hbuf + 3 * m);  // P columns kept
    int *actp = w.act + m;
    const bool fp32 = sizeof(V) == sizeof(float2);
    const bool tc = fp32 && o.tensor_cores >= 1;       // Gram matrices on tcgen05
    const bool tc_rot = fp32 && o.tensor_cores >= 2;   // and the Ritz rotations
    const double pivot_tol = fp32 ? std::max(o.pivot_tol, PIVOT_TOL_FP32) : o.pivot_tol;
    const double lock_tol = fp32 ? std::max(o.lock_tol, LOCK_TOL_FP32) : o.lock_tol;
    const double p_drop = fp32 ? P_DROP_FP32 : 0.0;
    if ((const void *)x_in != (const void *)X)
        RS_CUDA(ctx, cudaMemcpyAsync(X, x_in, (size_t)m * n * sizeof(V), cudaMemcpyDeviceToDevice, st));
    RS_TRY(Ops<V>::apply_h(ctx, X, HX, m, st));
    {
        Blocks Y{{X, nullptr, nullptr}, {m, 0, 0}};
        Blocks HY{{HX, nullptr, nullptr}, {m, 0, 0}};
        RS_TRY(gram_pair(ctx, Y, HY, w.GS, w.GH, m, tc, st));
        int nd = 0;
        RS_TRY(rayleigh_ritz(ctx, w.GH, w.GS, m, m, pivot_tol, w.theta, w.Cfull, &nd, st, dense_df(o)));
        bool rotated = false;
        if constexpr (std::is_same<V, float2>::value) {
            if (tc_rot && rotate_tc_fits(m + 1, m)) {   // X-only rotation from the Gram's split rows
                RS_TRY(rotate_tc_split(ctx, 0, m, w.Cfull, m, m, Xn, nullptr, st));
                RS_TRY(rotate_tc_split(ctx, 1, m, w.Cfull, m, m, HXn, nullptr, st));
                rotated = true;
            }
        }
        if (!rotated) {
            RS_TRY(Ops<V>::rotate(ctx, Y, w.Cfull, m, m, nullptr, 1, Xn, nullptr, st));
            RS_TRY(Ops<V>::rotate(ctx, HY, w.Cfull, m, m, nullptr, 1, HXn, nullptr, st));
        }
        std::swap(X, Xn);
        std::swap(HX, HXn);
    }
    PhaseEvents pe;
    if (stats) RS_TRY(pe.init(ctx));
    bool haveP = false;
    int it = 0, slow = 0;
    double prev = -1.0, best = -1.0;
    rsdft_status result = RSDFT_OK;
    for (;;) {
        RS_TRY(resid_norms<V>(ctx, HX, X, m, st));
        RS_CUDA(ctx, cudaMemcpyAsync(hres, w.res, m * sizeof(double), cudaMemcpyDeviceToHost, st));
        if (haveP && p_drop > 0.0) {
            RS_TRY(row_norms<V>(ctx, P, m, w.nrm, st));
            RS_CUDA(ctx, cudaMemcpyAsync(hpn, w.nrm, m * sizeof(double), cudaMemcpyDeviceToHost, st));
        }
        RS_CUDA(ctx, cudaStreamSynchronize(st));
        pe.collect(stats);
        double rmax = 0.0;
        bool bad = false;
        for (int b = 0; b < m; ++b) {
            if (!std::isfinite(hres[b])) bad = true;
            if (b < nconv) rmax = std::max(rmax, hres[b]);
        }
        if (bad) { result = fail(ctx, RSDFT_E_NUMERIC, "non-finite residual at iteration %d", it); break; }
        rs.converged = rmax <= stop_tol;
        if (rs.converged || it >= maxit) break;
        if (stagnation && prev > 0.0) {
            slow = rmax > 0.9 * prev ? slow + 1 : 0;
            if (slow >= 3) break;
        }
        // FP64, below 1e-6: a max residual above twice its best so far restarts the
        // iteration without P.  Near convergence P and W become nearly dependent; the Cholesky
        // keeps columns down to the pivot floor, and the error of K = L^-1 G_H L^-H
        // grows as 1 / floor along them.  Iterations of the mixed form's FP64 finish
        // that went on with P grew the residual by ~4x per iteration from 4e-9 to
        // 1e5 Ha on the 64^3 cell.
        if (!fp32 && haveP && best > 0.0 && best < 1e-6 && rmax > 2.0 * best) haveP = false;
        best = best > 0.0 ? std::min(best, rmax) : rmax;
        prev = rmax;
        int na = 0;
        for (int b = 0; b < m; ++b)
            if (hres[b] > lock_tol) hact[na++] = b;
        if (na == 0) break;
        int np_ = 0;
        if (haveP) {
            for (int j = 0; j < na; ++j)
                if (p_drop <= 0.0 || hpn[hact[j]] > p_drop) hactp[np_++] = hact[j];
        }
        RS_CUDA(ctx, cudaMemcpyAsync(w.act, hact, na * sizeof(int), cudaMemcpyHostToDevice, st));
        if (np_ > 0)
            RS_CUDA(ctx, cudaMemcpyAsync(actp, hactp, np_ * sizeof(int), cudaMemcpyHostToDevice, st));
        if (stats) RS_CUDA(ctx, cudaEventRecord(pe.ev[0], st));
        // ---- preconditioned residuals W (compact over the active bands)
        const dim3 rowgrid(std::min(cdiv(n, 256), 1024), na);
        const dim3 scalegrid(std::max(1, std::min(cdiv(n, 256 * 8), 256)), na);   // >= 8 points per thread
        if (o.precond == RSDFT_PRECOND_TPA || o.precond == RSDFT_PRECOND_LEARNED) {
            RS_TRY(Ops<V>::project(ctx, X, proj, m, st));
            k_tkin<V><<<cdiv(na, 128), 128, 0, st>>>(w.theta, w.vexp, proj, ctx->pt, w.act, na, w.tkin);
            count_launch(ctx);
            RS_LAUNCHED(ctx, "k_tkin");
            RS_TRY(Ops<V>::tpa(ctx, HX, X, w.theta, w.act, w.tkin, T1, W, na, st));
            if (o.precond == RSDFT_PRECOND_LEARNED && (o.learned_iters <= 0 || rs.iterations + it < o.learned_iters)) {
                // W += s_b NN(R_b / s_b); the TPA's FFT scratch holds the residuals
                k_residual_rows<V><<<rowgrid, 256, 0, st>>>(HX, X, w.theta, w.act, n, T1);
                count_launch(ctx);
                RS_LAUNCHED(ctx, "k_residual_rows");
                RS_TRY(learned_correction<V>(ctx, T1, na, W, st));
            }
        } else {
            k_residual_rows<V><<<rowgrid, 256, 0, st>>>(HX, X, w.theta, w.act, n, W);
            count_launch(ctx);
            RS_LAUNCHED(ctx, "k_residual_rows");
        }
        // W <- W - X <X|W>
        {
            Blocks YX{{X, nullptr, nullptr}, {m, 0, 0}};
            Blocks YW{{W, nullptr, nullptr}, {na, 0, 0}};
            bool done = false;
            if constexpr (std::is_same<V, float2>::value) {
                if (tc) RS_TRY(gram_tc(ctx, YX, YW, w.C, na, st));
                else RS_TRY(Ops<V>::gram(ctx, YX, YW, w.C, na, false, dV, st));
                if (tc_rot && rotate_tc_fits(m + na, na)) {
                    // the X split rows of the Gram above are still in the workspace
                    RS_TRY(rotate_tc_ortho(ctx, m, na, w.C, W, st));
                    done = true;
                }
            } else {
                RS_TRY(Ops<V>::gram(ctx, YX, YW, w.C, na, false, dV, st));
            }
            if (!done) RS_TRY(Ops<V>::rotate(ctx, YX, w.C, na, na, W, -1, W, nullptr, st));
        }
        if (stats) RS_CUDA(ctx, cudaEventRecord(pe.ev[1], st));
        RS_TRY(Ops<V>::apply_h(ctx, W, HW, na, st));
        if (stats) RS_CUDA(ctx, cudaEventRecord(pe.ev[2], st));
        RS_TRY(row_norms<V>(ctx, W, na, w.nrm, st));
        k_scale_rows<V><<<scalegrid, 256, 0, st>>>(W, HW, n, w.nrm);
        count_launch(ctx);
        RS_LAUNCHED(ctx, "normalise W");
        if (np_ > 0) {
            const dim3 pgrid(rowgrid.x, np_);
            k_gather_rows<V><<<pgrid, 256, 0, st>>>(P, HP, actp, n, Pn, HPn);
            RS_TRY(row_norms<V>(ctx, Pn, np_, w.nrm, st));
            k_scale_rows<V><<<dim3(scalegrid.x, np_), 256, 0, st>>>(Pn, HPn, n, w.nrm);
            count_launch(ctx, 2);
            RS_LAUNCHED(ctx, "normalise P");
        }
        if (stats) RS_CUDA(ctx, cudaEventRecord(pe.ev[3], st));
        const int k = m + na + np_;
        Blocks Y{{X, W, Pn}, {m, na, np_}};
        Blocks HY{{HX, HW, HPn}, {m, na, np_}};
        RS_TRY(gram_pair(ctx, Y, HY, w.GS, w.GH, k, tc, st));
        if (stats) RS_CUDA(ctx, cudaEventRecord(pe.ev[4], st));
        int nd = 0;
        RS_TRY(rayleigh_ritz(ctx, w.GH, w.GS, k, m, pivot_tol, w.lam, w.Cfull, &nd, st, dense_df(o)));
        rs.dropped += nd;
        if (stats) RS_CUDA(ctx, cudaEventRecord(pe.ev[5], st));
        bool rotated = false;
        if constexpr (std::is_same<V, float2>::value) {
            // the split-BF16 rows of Y and HY are still in the workspace from the Gram
            if (tc_rot && rotate_tc_fits(k, m)) {
                RS_TRY(rotate_tc_split(ctx, 0, k, w.Cfull, m, m, Xn, P, st));
                RS_TRY(rotate_tc_split(ctx, 1, k, w.Cfull, m, m, HXn, HP, st));
                rotated = true;
            }
        }
        if (!rotated) {
            RS_TRY(Ops<V>::rotate(ctx, Y, w.Cfull, m, m, nullptr, 1, Xn, P, st));
            RS_TRY(Ops<V>::rotate(ctx, HY, w.Cfull, m, m, nullptr, 1, HXn, HP, st));
        }
        if (stats) {
            RS_CUDA(ctx, cudaEventRecord(pe.ev[6], st));
            pe.pending = true;
        }
        RS_CUDA(ctx, cudaMemcpyAsync(w.theta, w.lam, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
        std::swap(X, Xn);
        std::swap(HX, HXn);
        haveP = true;
        rs.haveP = true;
        ++it;
    }
    if (stats) {
        RS_CUDA(ctx, cudaStreamSynchronize(st));
        pe.collect(stats);
        pe.destroy();
    }
    rs.iterations += it;
    // keep the workspace pointers consistent with the swaps
    w.X = (double2 *)X; w.Xn = (double2 *)Xn; w.HX = (double2 *)HX; w.HXn = (double2 *)HXn;
    if ((void *)x_out != (void *)X)
        RS_CUDA(ctx, cudaMemcpyAsync(x_out, X, (size_t)m * n * sizeof(V), cudaMemcpyDeviceToDevice, st));
    return result;
}

// FP64 refinement of the mixed form with FP32 corrections.  X and HX are FP64:
// the residuals and their norms, the X-X blocks of G_S and G_H, the blocks that
// couple X to the corrections, and the X part of the Ritz rotation are formed
// to FP64 accuracy (the Grams and rotations on the FP32 pipe with error-free
// products and compensated sums, gemm_df.cu).  The corrections W = TPA(R), HW = H W and the directions P, HP are FP32,
// and only the Gram blocks among them run on the FP32 path (split-BF16 tensor
// cores when tensor_cores >= 1):
//  - an error e in a coupling block would move the Ritz vectors by O(e / gap)
//    whatever the residual, a floor at the FP32 level; so the couplings are
//    FP64, G_S[X][W] = <X|W> and G_H[X][W] = <HX|W> from the FP64 X, HX and the
//    stored FP32 rows (H Hermitian), which keeps them consistent with the W
//    that the rotation uses whatever the rounding of HW;
//  - an error e in a block among W and P moves the Ritz vectors by
//    O(e |C_WP| / gap), and the coefficients C_WP fall with the residual;
//  - R is formed in FP64 before it is rounded, so W keeps FP32 relative accuracy
//    however small the residual is;
//  - HP = H P is recomputed from the normalised P every iteration (carried by
//    the rotation, its FP32 rounding would be relative to |p|, which falls with
//    the residual), so no P column needs to leave the basis;
//  - the FP64 residual norms certify the tolerance.
// P and HP of the FP32 phase (carryP) seed the first iteration.  Three
// iterations each gaining less than 10% set *stalled, and the caller continues
// with the all-FP64 iteration.
static rsdft_status lobpcg_refine(rsdft_ctx *ctx, double2 *x, int m, const rsdft_lobpcg_opts &o, double stop_tol,
                                  int maxit, bool carryP, RunState &rs, double *hres, rsdft_lobpcg_stats *stats,
                                  bool *stalled, cudaStream_t st) {
    using B32 = RowBlocksT<float2>;
    Workspace &w = ctx->ws;
    const long long n = ctx->n;
    const double dV = ctx->dV;
    const int nconv = (o.nconv <= 0 || o.nconv > m) ? m : o.nconv;
    double2 *X = w.X, *HX = w.HX, *Xn = w.Xn, *HXn = w.HXn;
    float2 *W = (float2 *)w.W, *HW = (float2 *)w.HW, *P = (float2 *)w.P, *HP = (float2 *)w.HP;
    float2 *Pn = (float2 *)w.Pn, *HPn = (float2 *)w.HPn, *T1 = (float2 *)w.T1;
    float2 *Xs = w.Xs;
    // lo parts of X and the pairs of HX in the unused halves of the FP64-sized
    // buffers that hold FP32 rows here (T1: FFT scratch of at most m bands;
    // Pn, HPn: at most m P columns)
    const size_t mn = (size_t)m * ctx->n;
    float2 *Xl = (float2 *)w.T1 + mn, *HXh = (float2 *)w.Pn + mn, *HXl = (float2 *)w.HPn + mn;
    float2 *proj = (float2 *)w.proj;
    int *hact = reinterpret_cast<int *>(w.hbuf + m);
    int *hactp = reinterpret_cast<int *>(w.hbuf + 3 * m);
    int *actp = w.act + m;
    const bool tc = o.tensor_cores >= 1;
    const bool tc_rot = o.tensor_cores >= 2;
    const double pivot_tol = std::max(o.pivot_tol, PIVOT_TOL_FP32);
    const double lock_tol = o.lock_tol;
    if ((const void *)x != (const void *)X)
        RS_CUDA(ctx, cudaMemcpyAsync(X, x, (size_t)m * n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    RS_TRY(apply_h64(ctx, X, HX, m, st));
    {   // Rayleigh quotients of the (FP32-orthonormal) start
        const int S = row_slices(ctx, m);
        k_rq_part<<<dim3(S, m), RTHREADS, 0, st>>>(HX, X, n, S, w.gram_part);
        k_rq_fin<<<cdiv(m, 128), 128, 0, st>>>(w.gram_part, S, m, w.theta);
        count_launch(ctx, 2);
        RS_LAUNCHED(ctx, "k_rq");
    }
    const long long cntm = (long long)m * n;
    const int cgrid = std::min(cdiv(cntm, 256), 4096);
    PhaseEvents pe;
    if (stats) RS_TRY(pe.init(ctx));
    bool haveP = carryP;
    int it = 0, slow = 0;
    double prev = -1.0, best = -1.0;
    *stalled = false;
    rsdft_status result = RSDFT_OK;
    for (;;) {
        RS_TRY(resid_norms<double2>(ctx, HX, X, m, st));
        RS_CUDA(ctx, cudaMemcpyAsync(hres, w.res, m * sizeof(double), cudaMemcpyDeviceToHost, st));
        RS_CUDA(ctx, cudaStreamSynchronize(st));
        pe.collect(stats);
        double rmax = 0.0;
        bool bad = false;
        for (int b = 0; b < m; ++b) {
            if (!std::isfinite(hres[b])) bad = true;
            if (b < nconv) rmax = std::max(rmax, hres[b]);
        }
        if (bad) { result = fail(ctx, RSDFT_E_NUMERIC, "non-finite residual at refinement iteration %d", it); break; }
        rs.converged = rmax <= stop_tol;
        if (rs.converged || it >= maxit) break;
        // three iterations each gaining less than 10%, or a residual ten times its
        // best so far: hand over to the FP64 iteration
        if (prev > 0.0) {
            slow = rmax > 0.9 * prev ? slow + 1 : 0;
            if (slow >= 3 || rmax > 10.0 * best) { *stalled = true; break; }
        }
        prev = rmax;
        best = best > 0.0 ? std::min(best, rmax) : rmax;
        int na = 0;
        for (int b = 0; b < m; ++b)
            if (hres[b] > lock_tol) hact[na++] = b;
        if (na == 0) break;
        int np_ = 0;
        if (haveP)
            for (int j = 0; j < na; ++j) hactp[np_++] = hact[j];
        RS_CUDA(ctx, cudaMemcpyAsync(w.act, hact, na * sizeof(int), cudaMemcpyHostToDevice, st));
        if (np_ > 0) RS_CUDA(ctx, cudaMemcpyAsync(actp, hactp, np_ * sizeof(int), cudaMemcpyHostToDevice, st));
        if (stats) RS_CUDA(ctx, cudaEventRecord(pe.ev[0], st));
        const dim3 rowgrid(std::min(cdiv(n, 256), 1024), na);
        const dim3 scalegrid(std::max(1, std::min(cdiv(n, 256 * 8), 256)), na);
        // X and HX as FP32 hi/lo pairs: the hi part of X is its FP32 copy (for the
        // TPA T_b and the W orthogonalisation); the pairs feed the FP64-accurate
        // Grams and rotations on the FP32 pipe (gemm_df.cu)
        RS_TRY(split_df(ctx, X, cntm, Xs, Xl, st));
        RS_TRY(split_df(ctx, HX, cntm, HXh, HXl, st));
        // R = HX - X Theta of the active bands in FP64 (into Xn, free until the
        // rotation), rounded to FP32 into W
        k_residual_rows<double2><<<rowgrid, 256, 0, st>>>(HX, X, w.theta, w.act, n, Xn);
        k_convert<double2, float2><<<std::min(cdiv((long long)na * n, 256), 4096), 256, 0, st>>>(
            Xn, (long long)na * n, W);
        count_launch(ctx, 2);
        RS_LAUNCHED(ctx, "refine residual");
        if (o.precond == RSDFT_PRECOND_TPA || o.precond == RSDFT_PRECOND_LEARNED) {
            RS_TRY(project32(ctx, Xs, proj, m, st));
            k_tkin<float2><<<cdiv(na, 128), 128, 0, st>>>(w.theta, w.vexp, proj, ctx->pt, w.act, na, w.tkin);
            count_launch(ctx);
            RS_LAUNCHED(ctx, "k_tkin");
            if (o.precond == RSDFT_PRECOND_LEARNED &&
                (o.learned_iters <= 0 || rs.iterations + it < o.learned_iters)) {
                // the network correction reads the residual rows, kept in T1
                RS_CUDA(ctx, cudaMemcpyAsync(T1, W, (size_t)na * n * sizeof(float2), cudaMemcpyDeviceToDevice, st));
                RS_TRY(fft_xy_forward32(ctx, Src::Plain, W, nullptr, nullptr, nullptr, Pn, na, st));
                RS_TRY(fft_z_mid32(ctx, Mid::Tpa, Pn, w.tkin, na, st));
                RS_TRY(fft_xy_inverse32(ctx, Pn, nullptr, nullptr, W, na, st));
                RS_TRY(learned_correction<float2>(ctx, T1, na, W, st));
            } else {
                RS_TRY(fft_xy_forward32(ctx, Src::Plain, W, nullptr, nullptr, nullptr, T1, na, st));
                RS_TRY(fft_z_mid32(ctx, Mid::Tpa, T1, w.tkin, na, st));
                RS_TRY(fft_xy_inverse32(ctx, T1, nullptr, nullptr, W, na, st));
            }
        }
        // W <- W - X <X|W> (FP32)
        {
            B32 YX{{Xs, nullptr, nullptr}, {m, 0, 0}};
            B32 YW{{W, nullptr, nullptr}, {na, 0, 0}};
            bool done = false;
            if (tc) RS_TRY(gram_tc(ctx, YX, YW, w.C, na, st));
            else RS_TRY(gram32(ctx, YX, YW, w.C, na, false, dV, st));
            if (tc_rot && rotate_tc_fits(m + na, na)) {
                RS_TRY(rotate_tc_ortho(ctx, m, na, w.C, W, st));
                done = true;
            }
            if (!done) RS_TRY(rotate32(ctx, YX, w.C, na, na, W, -1, W, nullptr, st));
        }
        if (stats) RS_CUDA(ctx, cudaEventRecord(pe.ev[1], st));
        RS_TRY(apply_h32(ctx, W, HW, na, st));
        RS_TRY(row_norms<float2>(ctx, W, na, w.nrm, st));
        k_scale_rows<float2><<<scalegrid, 256, 0, st>>>(W, HW, n, w.nrm);
        count_launch(ctx);
        RS_LAUNCHED(ctx, "normalise W");
        if (np_ > 0) {
            const dim3 pgrid(rowgrid.x, np_);
            k_gather_rows<float2><<<pgrid, 256, 0, st>>>(P, HP, actp, n, Pn, HPn);
            RS_TRY(row_norms<float2>(ctx, Pn, np_, w.nrm, st));
            k_scale_rows<float2><<<dim3(scalegrid.x, np_), 256, 0, st>>>(Pn, nullptr, n, w.nrm);
            count_launch(ctx, 2);
            RS_LAUNCHED(ctx, "normalise P");
            RS_TRY(apply_h32(ctx, Pn, HPn, np_, st));
        }
        if (stats) RS_CUDA(ctx, cudaEventRecord(pe.ev[2], st));
        if (stats) RS_CUDA(ctx, cudaEventRecord(pe.ev[3], st));
        const int k = m + na + np_;
        const int nwp = na + np_;
        // Gram blocks: [W P]-[W P] on the FP32 path; X-X and the X-[W P]
        // couplings in FP64 (the latter from FP64 X and HX against the FP32 rows,
        // G_H[X][W] = <HX|W>, consistent with the stored W whatever the rounding of HW)
        {
            B32 Y{{W, Pn, nullptr}, {na, np_, 0}};
            B32 HY{{HW, HPn, nullptr}, {na, np_, 0}};
            // FP32 CUDA cores even with tensor_cores set: the split-BF16 error
            // (1e-5 of max |G|) in these blocks, divided by small gaps of the
            // projected problem, slowed the refinement below 1e-8
            RS_TRY(gram_pair<float2>(ctx, Y, HY, w.GS + (size_t)m * k + m, w.GH + (size_t)m * k + m, k, false, st));
            const B32 none{{nullptr, nullptr, nullptr}, {0, 0, 0}};
            const B32 bx{{Xs, nullptr, nullptr}, {m, 0, 0}}, bxl{{Xl, nullptr, nullptr}, {m, 0, 0}};
            const B32 bhx{{HXh, nullptr, nullptr}, {m, 0, 0}}, bhxl{{HXl, nullptr, nullptr}, {m, 0, 0}};
            RS_TRY(gram_df(ctx, Xs, Xl, m, bx, bxl, w.GS, k, dV, st));
            RS_TRY(gram_df(ctx, Xs, Xl, m, bhx, bhxl, w.GH, k, dV, st));
            RS_TRY(gram_df(ctx, Xs, Xl, m, Y, none, w.GS + m, k, dV, st));
            RS_TRY(gram_df(ctx, HXh, HXl, m, Y, none, w.GH + m, k, dV, st));
            k_herm_block<<<dim3(cdiv(m, 32), cdiv(m, 32)), dim3(32, 8), 0, st>>>(w.GS, w.GH, k, m);
            k_mirror_block<<<dim3(cdiv(m, 32), cdiv(nwp, 32)), dim3(32, 8), 0, st>>>(w.GS, w.GH, k, m, nwp);
            count_launch(ctx, 2);
            RS_LAUNCHED(ctx, "k_mirror_block");
        }
        if (stats) RS_CUDA(ctx, cudaEventRecord(pe.ev[4], st));
        int nd = 0;
        RS_TRY(rayleigh_ritz(ctx, w.GH, w.GS, k, m, pivot_tol, w.lam, w.Cfull, &nd, st, dense_df(o)));
        rs.dropped += nd;
        if (stats) RS_CUDA(ctx, cudaEventRecord(pe.ev[5], st));
        // P = [W P] C[m:], HP alike (FP32); X = X C[:m] + P, HX alike (FP64)
        {
            const double2 *cwp = w.Cfull + (size_t)m * m;
            B32 YWP{{W, Pn, nullptr}, {na, np_, 0}};
            B32 HYWP{{HW, HPn, nullptr}, {na, np_, 0}};
            RS_TRY(rotate32(ctx, YWP, cwp, m, m, nullptr, 1, P, nullptr, st));
            RS_TRY(rotate32(ctx, HYWP, cwp, m, m, nullptr, 1, HP, nullptr, st));
            RS_TRY(rotate_df(ctx, Xs, Xl, m, w.Cfull, m, m, Xn, st));
            RS_TRY(rotate_df(ctx, HXh, HXl, m, w.Cfull, m, m, HXn, st));
            k_add_f32<<<cgrid, 256, 0, st>>>(Xn, P, cntm);
            k_add_f32<<<cgrid, 256, 0, st>>>(HXn, HP, cntm);
            count_launch(ctx, 2);
            RS_LAUNCHED(ctx, "k_add_f32");
        }
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
    }
    rs.iterations += it;
    w.X = X; w.Xn = Xn; w.HX = HX; w.HXn = HXn;
    if ((void *)x != (void *)X)
        RS_CUDA(ctx, cudaMemcpyAsync(x, X, (size_t)m * n * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    return result;
}

rsdft_status lobpcg_run(rsdft_ctx *ctx, double2 *x, int m, const rsdft_lobpcg_opts &o,
                        double *eig_host, double *res_host, rsdft_lobpcg_stats *stats,
                        cudaStream_t st) {
    RS_TRY(ensure_workspace(ctx, m));
    Workspace &w = ctx->ws;
    double *hres = w.hbuf;
    RunState rs;
    int it_mixed = 0;
    const long long fallbacks0 = ctx->coop_fallbacks;
    rsdft_status r = RSDFT_OK;
    if (o.precision == RSDFT_MIXED) {
        // mixed form: FP32 data path until switch_tol (or stagnation), then FP64
        RS_TRY(refresh_v32(ctx, st));
        float2 *xs = w.Xs;
        const long long cnt = (long long)m * ctx->n;
        k_convert<double2, float2><<<std::min(cdiv(cnt, 256), 4096), 256, 0, st>>>(x, cnt, xs);
        count_launch(ctx);
        RS_LAUNCHED(ctx, "k_convert");
        const double stop = std::max(o.tol, o.switch_tol);
        r = lobpcg_t<float2>(ctx, xs, xs, m, o, stop, o.maxit, o.tol > 0.0, rs, hres, stats, st);
        if (r != RSDFT_OK) return r;
        it_mixed = rs.iterations;
        k_convert<float2, double2><<<std::min(cdiv(cnt, 256), 4096), 256, 0, st>>>(xs, cnt, x);
        count_launch(ctx);
        RS_LAUNCHED(ctx, "k_convert");
        if (o.tol > 0.0 || rs.iterations < o.maxit) {
            RunState r2;
            const int left = o.tol > 0.0 ? std::max(0, o.maxit - rs.iterations) : o.maxit - rs.iterations;
            bool stalled = false;
            if (o.refine == RSDFT_REFINE_FP32_CORRECTIONS) {
                // the FP32 blocks among the corrections bound what this refinement
                // reaches (their errors, ~eps32 |H|, enter the Ritz vectors scaled by
                // the residual over the squared gap of the projected problem): it
                // runs to REFINE32_FLOOR, the FP64 iteration finishes below
                r = lobpcg_refine(ctx, x, m, o, std::max(o.tol, REFINE32_FLOOR), std::min(left, REFINE32_MAXIT),
                                  rs.haveP, r2, hres, stats, &stalled, st);
                if (r == RSDFT_OK && !r2.converged && !stalled && r2.iterations < left) stalled = true;   // cap or lock
                if (r == RSDFT_OK && r2.converged && o.tol < REFINE32_FLOOR) stalled = true;
            } else {
                r = lobpcg_t<double2>(ctx, x, x, m, o, o.tol, left, false, r2, hres, stats, st);
            }
            if (r == RSDFT_OK && stalled) {
                RunState r3;
                r = lobpcg_t<double2>(ctx, x, x, m, o, o.tol, std::max(0, left - r2.iterations), false, r3, hres,
                                      stats, st);
                r2.iterations += r3.iterations;
                r2.dropped += r3.dropped;
                r2.converged = r3.converged;
            }
            rs.iterations += r2.iterations;
            rs.dropped += r2.dropped;
            rs.converged = r2.converged;
        }
    } else {
        r = lobpcg_t<double2>(ctx, x, x, m, o, o.tol, o.maxit, false, rs, hres, stats, st);
    }
    if (stats) {
        stats->iterations = rs.iterations;
        stats->iterations_mixed = it_mixed;
        stats->converged = rs.converged ? 1 : 0;
        stats->dropped = rs.dropped;
        stats->coop_fallbacks = (int)(ctx->coop_fallbacks - fallbacks0);
        stats->coop_last_error = stats->coop_fallbacks ? ctx->coop_last_error : 0;
    }
    if (eig_host) RS_CUDA(ctx, cudaMemcpyAsync(eig_host, w.theta, m * sizeof(double), cudaMemcpyDeviceToHost, st));
    RS_CUDA(ctx, cudaStreamSynchronize(st));
    if (res_host) memcpy(res_host, hres, m * sizeof(double));
    if (r != RSDFT_OK) return r;
    return rs.converged || o.tol <= 0.0 ? RSDFT_OK : RSDFT_E_NOT_CONVERGED;
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
    o->switch_tol = 3e-5;
    o->tensor_cores = 0;
    o->learned_iters = 0;
    o->refine = RSDFT_REFINE_FP32_CORRECTIONS;
    o->dense = RSDFT_DENSE_AUTO;
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
    if (o.maxit < 0 || !(o.tol >= 0.0) || !(o.pivot_tol >= 0.0) || !(o.lock_tol >= 0.0) ||
        !(o.switch_tol >= 0.0))
        return fail(ctx, RSDFT_E_INVALID, "bad LOBPCG options");
    if (o.precision != RSDFT_FP64 && o.precision != RSDFT_MIXED)
        return fail(ctx, RSDFT_E_INVALID, "unknown precision");
    if (o.refine != RSDFT_REFINE_FP64 && o.refine != RSDFT_REFINE_FP32_CORRECTIONS)
        return fail(ctx, RSDFT_E_INVALID, "unknown refinement mode");
    if (o.dense != RSDFT_DENSE_AUTO && o.dense != RSDFT_DENSE_FP64 && o.dense != RSDFT_DENSE_DF)
        return fail(ctx, RSDFT_E_INVALID, "unknown dense mode");
    if (o.precond != RSDFT_PRECOND_TPA && o.precond != RSDFT_PRECOND_NONE && o.precond != RSDFT_PRECOND_LEARNED)
        return fail(ctx, RSDFT_E_INVALID, "unknown preconditioner");
    if (o.precond == RSDFT_PRECOND_LEARNED && !ctx->nn.ready)
        return fail(ctx, RSDFT_E_INVALID, "learned preconditioner: no weights set");
    if (stats) *stats = rsdft_lobpcg_stats{};
    return lobpcg_run(ctx, (double2 *)x_dev, nband, o, eig_host, resnorm_host, stats, as_stream(stream));
}

rsdft_status rsdft_lobpcg_batched(rsdft_ctx *const *ctxs, int ncell, void *const *x_dev, const int *nband,
                                  const rsdft_lobpcg_opts *opts, double *const *eig_host,
                                  double *const *res_host, rsdft_lobpcg_stats *stats, int max_concurrent,
                                  int *failed_cell) {
    if (failed_cell) *failed_cell = -1;
    if (ncell < 0 || (ncell > 0 && (!ctxs || !x_dev || !nband)))
        return fail(nullptr, RSDFT_E_INVALID, "bad batch arguments");
    for (int c = 0; c < ncell; ++c)
        if (!ctxs[c]) return fail(nullptr, RSDFT_E_INVALID, "cell %d: ctx is NULL", c);
    if (ncell == 0) return RSDFT_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(nullptr, RSDFT_E_CUDA, "cudaGetDevice failed");
    // the cells' streams do not order against the caller's work: let everything
    // issued so far (e.g. the uploads of the orbital blocks) finish first
    if (cudaDeviceSynchronize() != cudaSuccess)
        return fail(nullptr, RSDFT_E_CUDA, "%s", cudaGetErrorString(cudaGetLastError()));
    const int nthr = std::max(1, std::min(ncell, max_concurrent <= 0 ? 8 : max_concurrent));
    std::vector<rsdft_status> status(ncell, RSDFT_OK);
    std::atomic<int> next{0};
    // one host thread and one stream per concurrent cell; cells are handed out
    // in order, so the cells in flight at any time are consecutive
    auto worker = [&]() {
        cudaSetDevice(dev);
        cudaStream_t st = nullptr;
        const bool have_stream = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
        for (int c; (c = next.fetch_add(1)) < ncell;) {
            if (!have_stream) {
                status[c] = fail(ctxs[c], RSDFT_E_CUDA, "could not create a stream for the batch");
                continue;
            }
            status[c] = rsdft_lobpcg(ctxs[c], x_dev[c], nband[c], opts ? &opts[c] : nullptr,
                                     eig_host ? eig_host[c] : nullptr,
                                     res_host ? res_host[c] : nullptr, stats ? &stats[c] : nullptr, st);
            if (status[c] == RSDFT_OK && cudaStreamSynchronize(st) != cudaSuccess)
                status[c] = fail(ctxs[c], RSDFT_E_CUDA, "%s", cudaGetErrorString(cudaGetLastError()));
        }
        if (have_stream) cudaStreamDestroy(st);
    };
    std::vector<std::thread> pool;
    pool.reserve(nthr);
    for (int t = 0; t < nthr; ++t) pool.emplace_back(worker);
    for (auto &t : pool) t.join();
    for (int c = 0; c < ncell; ++c) {
        if (status[c] != RSDFT_OK) {
            if (failed_cell) *failed_cell = c;
            return status[c];
        }
    }
    return RSDFT_OK;
}

}  // extern "C"
