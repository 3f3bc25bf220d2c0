// Context creation: grid, FFT plans and tables, local potential, KB projector
// tables, device workspace.  Host code plus uploads; no kernels here.
#include <cmath>
#include <cstdarg>
#include <algorithm>

#include "rsdft_internal.h"

namespace rsdft {

static thread_local std::string g_create_error;

rsdft_status fail(rsdft_ctx *ctx, rsdft_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf; else g_create_error = buf;
    return st;
}

rsdft_status cuda_check(rsdft_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation)
        return fail(ctx, RSDFT_E_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(ctx, RSDFT_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

rsdft_status dev_alloc(rsdft_ctx *ctx, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, RSDFT_E_OOM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    ctx->owned.push_back(*p);
    return RSDFT_OK;
}

template <typename T>
static rsdft_status upload(rsdft_ctx *ctx, T **dst, const T *src, size_t count) {
    RS_TRY(dev_alloc(ctx, (void **)dst, count * sizeof(T)));
    if (count) RS_CUDA(ctx, cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice));
    return RSDFT_OK;
}

// N = 2^a 3^b 5^c, 2 <= N <= MAX_N.  Radices: 8s and 4s for the power of two
// (fewer stages), then 3s, then 5s.
static bool make_axis_plan(int N, AxisPlan &p) {
    if (N < 2 || N > MAX_N) return false;
    int n = N, p2 = 0, p3 = 0, p5 = 0;
    while (n % 2 == 0) { n /= 2; ++p2; }
    while (n % 3 == 0) { n /= 3; ++p3; }
    while (n % 5 == 0) { n /= 5; ++p5; }
    if (n != 1) return false;
    std::vector<int> r;
    if (p2 % 3 == 0) { for (int i = 0; i < p2 / 3; ++i) r.push_back(8); }
    else if (p2 % 3 == 1) {
        if (p2 >= 4) { r.push_back(4); r.push_back(4); for (int i = 0; i < (p2 - 4) / 3; ++i) r.push_back(8); }
        else r.push_back(2);
    } else { r.push_back(4); for (int i = 0; i < (p2 - 2) / 3; ++i) r.push_back(8); }
    for (int i = 0; i < p3; ++i) r.push_back(3);
    for (int i = 0; i < p5; ++i) r.push_back(5);
    if ((int)r.size() > MAX_STAGES) return false;
    p.N = N;
    p.nstage = (int)r.size();
    int len = N;
    // ceil(2^32 / d): exact quotients for x < 2^16 and d < 2^16
    auto mag = [](int d) -> unsigned {
        return d <= 1 ? 0u : (unsigned)(((1ull << 32) + (unsigned long long)d - 1) / (unsigned long long)d);
    };
    p.nmag = mag(N);
    for (int s = 0; s < p.nstage; ++s) {
        p.radix[s] = r[s];
        p.len[s] = len;
        p.sub[s] = len / r[s];
        len = p.sub[s];
        p.submag[s] = mag(p.sub[s]);
        p.bfmag[s] = mag(N / r[s]);
    }
    return true;
}

// Frequency index held at a digit-reversed position after the forward stages.
static int position_to_freq(const AxisPlan &p, int pos) {
    int k = 0, w = 1;
    for (int s = 0; s < p.nstage; ++s) {
        int digit = (pos / p.sub[s]) % p.radix[s];
        k += digit * w;
        w *= p.radix[s];
    }
    return k;
}

static rsdft_status build_fft_tables(rsdft_ctx *ctx) {
    const long double two_pi = 6.283185307179586476925286766559005768L;
    for (int a = 0; a < 3; ++a) {
        AxisPlan &p = ctx->fft.ax[a];
        int N = p.N;
        std::vector<double2> tw(N);
        std::vector<float2> twf(N);
        for (int k = 0; k < N; ++k) {
            long double ang = two_pi * (long double)k / (long double)N;
            double c = (double)cosl(ang), s = -(double)sinl(ang);
            tw[k] = make_double2(c, s);
            twf[k] = make_float2((float)c, (float)s);
        }
        std::vector<double> g2(N), g1(N);
        double gunit = 2.0 * M_PI / ctx->L[a];
        for (int pos = 0; pos < N; ++pos) {
            int k = position_to_freq(p, pos);
            int ks = k < (N + 1) / 2 ? k : k - N;
            double g = gunit * ks;
            g2[pos] = g * g;
            // first derivatives: the Nyquist plane of an even axis gets 0 (for a
            // real field its derivative is imaginary, i.e. 0 in the real part)
            g1[pos] = (N % 2 == 0 && k == N / 2) ? 0.0 : g;
        }
        std::vector<float> g2f(g2.begin(), g2.end());
        double2 *d_tw; float2 *d_twf; double *d_g2; float *d_g2f; double *d_g1;
        RS_TRY(upload(ctx, &d_g1, g1.data(), N));
        ctx->fft.gpos[a] = d_g1;
        RS_TRY(upload(ctx, &d_tw, tw.data(), N));
        RS_TRY(upload(ctx, &d_twf, twf.data(), N));
        RS_TRY(upload(ctx, &d_g2, g2.data(), N));
        RS_TRY(upload(ctx, &d_g2f, g2f.data(), N));
        ctx->fft.tw64[a] = d_tw;
        ctx->fft.tw32[a] = d_twf;
        ctx->fft.g2pos[a] = d_g2;
        ctx->fft.g2pos32[a] = d_g2f;
    }
    return RSDFT_OK;
}

static inline double min_image(double d, double L) { return d - L * std::floor(d / L + 0.5); }

// Per axis: the grid indices whose minimal-image displacement from R lies
// strictly inside (-rcut, rcut), with those displacements.
static void axis_window(int N, double L, double R, double rcut, std::vector<int> &idx,
                        std::vector<double> &disp) {
    idx.clear();
    disp.clear();
    double h = L / N;
    for (int i = 0; i < N; ++i) {
        double d = min_image(i * h - R, L);
        if (std::fabs(d) < rcut) { idx.push_back(i); disp.push_back(d); }
    }
}

static rsdft_status build_projectors(rsdft_ctx *ctx, const rsdft_projectors *pj) {
    const int natom = pj->natom, nproj = pj->nproj;
    const double rc = pj->rc, rcut = pj->rcut;
    const int Nx = ctx->N[0], Ny = ctx->N[1], Nz = ctx->N[2];
    std::vector<int> a_start(natom + 1, 0), a_idx;
    std::vector<double> a_beta;
    std::vector<int> ix, iy, iz;
    std::vector<double> dx, dy, dz;
    for (int a = 0; a < natom; ++a) {
        const double *R = pj->pos + 3 * a;
        axis_window(Nx, ctx->L[0], R[0], rcut, ix, dx);
        axis_window(Ny, ctx->L[1], R[1], rcut, iy, dy);
        axis_window(Nz, ctx->L[2], R[2], rcut, iz, dz);
        size_t first = a_idx.size();
        // points in increasing linear index order (z, then y, then x)
        std::vector<int> oz(iz.size()), oy(iy.size()), ox(ix.size());
        for (size_t i = 0; i < oz.size(); ++i) oz[i] = (int)i;
        for (size_t i = 0; i < oy.size(); ++i) oy[i] = (int)i;
        for (size_t i = 0; i < ox.size(); ++i) ox[i] = (int)i;
        std::sort(oz.begin(), oz.end(), [&](int p, int q) { return iz[p] < iz[q]; });
        std::sort(oy.begin(), oy.end(), [&](int p, int q) { return iy[p] < iy[q]; });
        std::sort(ox.begin(), ox.end(), [&](int p, int q) { return ix[p] < ix[q]; });
        for (int kz : oz)
            for (int ky : oy)
                for (int kx : ox) {
                    double d2 = dx[kx] * dx[kx] + dy[ky] * dy[ky] + dz[kz] * dz[kz];
                    if (!(d2 < rcut * rcut)) continue;
                    double g = std::exp(-d2 / (2.0 * rc * rc));
                    a_idx.push_back((iz[kz] * Ny + iy[ky]) * Nx + ix[kx]);
                    a_beta.push_back(g);
                    a_beta.push_back(nproj == 4 ? dx[kx] / rc * g : 0.0);
                    a_beta.push_back(nproj == 4 ? dy[ky] / rc * g : 0.0);
                    a_beta.push_back(nproj == 4 ? dz[kz] / rc * g : 0.0);
                }
        // grid normalisation: sum beta^2 dV = 1
        for (int j = 0; j < nproj; ++j) {
            double s = 0.0;
            for (size_t e = first; e < a_idx.size(); ++e) s += a_beta[4 * e + j] * a_beta[4 * e + j];
            double c = s > 0.0 ? 1.0 / std::sqrt(s * ctx->dV) : 0.0;
            for (size_t e = first; e < a_idx.size(); ++e) a_beta[4 * e + j] *= c;
        }
        a_start[a + 1] = (int)a_idx.size();
    }
    const long long nent = (long long)a_idx.size();
    if (nent > 0x7fffffffLL) return fail(ctx, RSDFT_E_INVALID, "projector table too large");
    // point-major CSR (entries of a point ordered by atom)
    std::vector<int> rowptr(ctx->n + 1, 0), c_atom(nent);
    std::vector<double> c_beta(4 * nent);
    for (long long e = 0; e < nent; ++e) rowptr[a_idx[e] + 1]++;
    for (long long i = 0; i < ctx->n; ++i) rowptr[i + 1] += rowptr[i];
    std::vector<int> fillp(rowptr.begin(), rowptr.end() - 1);
    for (int a = 0; a < natom; ++a)
        for (int e = a_start[a]; e < a_start[a + 1]; ++e) {
            int slot = fillp[a_idx[e]]++;
            c_atom[slot] = a;
            for (int j = 0; j < 4; ++j) c_beta[4 * slot + j] = a_beta[4 * e + j];
        }
    std::vector<double> ekb(pj->e_kb, pj->e_kb + (size_t)natom * nproj);
    int *d_as, *d_ai, *d_rp, *d_ca;
    double *d_ab, *d_cb, *d_e;
    RS_TRY(upload(ctx, &d_as, a_start.data(), a_start.size()));
    RS_TRY(upload(ctx, &d_ai, a_idx.data(), a_idx.size()));
    RS_TRY(upload(ctx, &d_ab, a_beta.data(), a_beta.size()));
    RS_TRY(upload(ctx, &d_rp, rowptr.data(), rowptr.size()));
    RS_TRY(upload(ctx, &d_ca, c_atom.data(), c_atom.size()));
    RS_TRY(upload(ctx, &d_cb, c_beta.data(), c_beta.size()));
    RS_TRY(upload(ctx, &d_e, ekb.data(), ekb.size()));
    ctx->pt = ProjTables{natom, nproj, d_as, d_ai, d_ab, d_rp, d_ca, d_cb, d_e};
    std::vector<float> abf(a_beta.begin(), a_beta.end()), cbf(c_beta.begin(), c_beta.end()),
        ekf(ekb.begin(), ekb.end());
    float *d_abf, *d_cbf, *d_ef;
    RS_TRY(upload(ctx, &d_abf, abf.data(), abf.size()));
    RS_TRY(upload(ctx, &d_cbf, cbf.data(), cbf.size()));
    RS_TRY(upload(ctx, &d_ef, ekf.data(), ekf.size()));
    ctx->pt32 = ProjT<float>{natom, nproj, d_as, d_ai, d_abf, d_rp, d_ca, d_cbf, d_ef};
    ctx->nent = nent;
    return RSDFT_OK;
}

static rsdft_status check_cell_grid(const rsdft_cell *cell, const rsdft_grid *grid,
                                    rsdft_ctx *ctx, AxisPlan *plans, double *L) {
    if (!cell || !grid) return fail(ctx, RSDFT_E_INVALID, "cell and grid are required");
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (a != b && cell->a[a][b] != 0.0)
                return fail(ctx, RSDFT_E_INVALID, "only orthorhombic (diagonal) cells are supported");
    for (int a = 0; a < 3; ++a) {
        L[a] = cell->a[a][a];
        if (!(L[a] > 0.0) || !std::isfinite(L[a]))
            return fail(ctx, RSDFT_E_INVALID, "cell edge %d must be positive", a);
        if (plans && !make_axis_plan(grid->n[a], plans[a]))
            return fail(ctx, RSDFT_E_GRID_NOT_5SMOOTH,
                        "grid dimension %d = %d is not 2^a 3^b 5^c in [2, %d]", a, grid->n[a], MAX_N);
        if (!plans && (grid->n[a] < 1))
            return fail(ctx, RSDFT_E_INVALID, "grid dimension %d must be positive", a);
    }
    return RSDFT_OK;
}

rsdft_status ensure_workspace(rsdft_ctx *ctx, int nband) {
    Workspace &w = ctx->ws;
    if (nband <= w.cap_band) return RSDFT_OK;
    // free the old buffers of the workspace (they are in ctx->owned)
    auto release = [&](void *p) {
        if (!p) return;
        cudaFree(p);
        ctx->owned.erase(std::remove(ctx->owned.begin(), ctx->owned.end(), p), ctx->owned.end());
    };
    void *olds[] = {w.X, w.HX, w.W, w.HW, w.P, w.HP, w.T1, w.Xn, w.HXn, w.Pn, w.HPn, w.Xs, w.proj,
                    w.GS, w.GH, w.C, w.Cfull, w.gram_part, w.Lm, w.Km, w.Ym, w.Vh, w.Zc,
                    w.tau, w.wv, w.Tw, w.d, w.e, w.lam, w.zt, w.dscr, w.fac, w.gsync, w.drop, w.keep, w.ikeep,
                    w.theta, w.res, w.vexp, w.tkin, w.nrm, w.act};
    for (void *p : olds) release(p);
    if (w.hbuf) cudaFreeHost(w.hbuf);
    w = Workspace{};
    const size_t nb = (size_t)nband, n = (size_t)ctx->n;
    const size_t orb = nb * n * sizeof(double2);
    double2 **orbs[] = {&w.X, &w.HX, &w.W, &w.HW, &w.P, &w.HP, &w.T1, &w.Xn, &w.HXn, &w.Pn, &w.HPn};
    for (double2 **b : orbs) RS_TRY(dev_alloc(ctx, (void **)b, orb));
    RS_TRY(dev_alloc(ctx, (void **)&w.Xs, nb * n * sizeof(float2)));
    const size_t np = (size_t)std::max(1, ctx->pt.natom * ctx->pt.nproj);
    RS_TRY(dev_alloc(ctx, (void **)&w.proj, nb * np * sizeof(double2)));
    const size_t k = 3 * nb;
    const size_t kk = k * k * sizeof(double2);
    for (double2 **b : {&w.GS, &w.GH, &w.C, &w.Cfull, &w.Lm, &w.Km, &w.Ym, &w.Vh, &w.Zc})
        RS_TRY(dev_alloc(ctx, (void **)b, kk));
    w.gram_part_elems = (size_t)16 * 2 * k * k;
    RS_TRY(dev_alloc(ctx, (void **)&w.gram_part, w.gram_part_elems * sizeof(double2)));
    RS_TRY(dev_alloc(ctx, (void **)&w.tau, k * sizeof(double2)));
    // the cooperative tridiagonalisation keeps w in two buffers of up to 4 parts
    RS_TRY(dev_alloc(ctx, (void **)&w.wv, 8 * k * sizeof(double2)));
    RS_TRY(dev_alloc(ctx, (void **)&w.Tw, (k / 32 + 1) * 32 * 32 * sizeof(double2)));
    for (double **b : {&w.d, &w.e, &w.lam})
        RS_TRY(dev_alloc(ctx, (void **)b, k * sizeof(double)));
    RS_TRY(dev_alloc(ctx, (void **)&w.zt, k * k * sizeof(double)));
    RS_TRY(dev_alloc(ctx, (void **)&w.dscr, (8 * k + 64) * sizeof(double)));
    RS_TRY(dev_alloc(ctx, (void **)&w.fac, 6 * k * k * sizeof(double)));   // inverse-iteration factors
    RS_TRY(dev_alloc(ctx, (void **)&w.gsync, 64));
    for (int **b : {&w.drop, &w.keep, &w.ikeep})
        RS_TRY(dev_alloc(ctx, (void **)b, (k + 1) * sizeof(int)));
    for (double **b : {&w.theta, &w.res, &w.vexp, &w.tkin, &w.nrm})
        RS_TRY(dev_alloc(ctx, (void **)b, nb * sizeof(double)));
    RS_TRY(dev_alloc(ctx, (void **)&w.act, 2 * nb * sizeof(int)));  // active bands | P columns
    w.hbuf_elems = 8 * k + 64;
    if (cudaMallocHost((void **)&w.hbuf, w.hbuf_elems * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        w.hbuf = nullptr;
        return fail(ctx, RSDFT_E_OOM, "pinned host buffer");
    }
    w.cap_band = nband;
    w.cap_k = (int)k;
    return RSDFT_OK;
}

rsdft_status autotune_pick(rsdft_ctx *ctx, const std::string &key, int ncand, int fallback, cudaStream_t st,
                           const std::function<rsdft_status(int)> &run, int *chosen) {
    auto it = ctx->tuned.find(key);
    if (it != ctx->tuned.end() || !ctx->autotune || ncand <= 1) {
        const int c = it != ctx->tuned.end() ? it->second : fallback;
        *chosen = c;
        return run(c);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    RS_CUDA(ctx, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(ctx, RSDFT_E_CUDA, "cudaEventCreate failed");
    }
    // each candidate: one untimed run (the first launch of its instantiation and any
    // growth of the workspace it needs stay outside the timing), then the fastest of
    // two timed runs
    int best = fallback;
    float best_ms = 0.0f;
    rsdft_status r = RSDFT_OK;
    for (int c = 0; c < ncand && r == RSDFT_OK; ++c) {
        r = run(c);
        float cmin = 0.0f;
        for (int rep = 0; rep < 2 && r == RSDFT_OK; ++rep) {
            cudaEventRecord(e0, st);
            r = run(c);
            cudaEventRecord(e1, st);
            if (r != RSDFT_OK) break;
            float ms = 0.0f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                r = fail(ctx, RSDFT_E_CUDA, "%s", cudaGetErrorString(cudaGetLastError()));
                break;
            }
            if (rep == 0 || ms < cmin) cmin = ms;
        }
        if (r != RSDFT_OK) break;
        if (c == 0 || cmin < best_ms) {
            best_ms = cmin;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != RSDFT_OK) return r;
    ctx->tuned[key] = best;
    *chosen = best;
    return best == ncand - 1 ? RSDFT_OK : run(best);   // the winner's result last
}

}  // namespace rsdft

using namespace rsdft;

extern "C" rsdft_status rsdft_set_autotune(rsdft_ctx *ctx, int on) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    ctx->autotune = on != 0;
    if (!ctx->autotune) ctx->tuned.clear();
    return RSDFT_OK;
}

extern "C" {

rsdft_status rsdft_create(const rsdft_cell *cell, const rsdft_grid *grid, const double *v_loc_host,
                          const rsdft_projectors *proj, rsdft_ctx **out) {
    if (!out) return fail(nullptr, RSDFT_E_INVALID, "out is NULL");
    *out = nullptr;
    AxisPlan plans[3];
    double L[3];
    RS_TRY(check_cell_grid(cell, grid, nullptr, plans, L));
    if (!v_loc_host) return fail(nullptr, RSDFT_E_INVALID, "v_loc is NULL");
    if (proj) {
        if (proj->natom < 0 || (proj->natom > 0 && (!proj->pos || !proj->e_kb)))
            return fail(nullptr, RSDFT_E_INVALID, "projector arrays missing");
        if (proj->nproj != 1 && proj->nproj != 4)
            return fail(nullptr, RSDFT_E_INVALID, "nproj must be 1 or 4");
        if (!(proj->rc > 0.0) || !(proj->rcut > 0.0) ||
            !(proj->rcut < 0.5 * std::min(L[0], std::min(L[1], L[2]))))
            return fail(nullptr, RSDFT_E_INVALID, "need rc > 0 and 0 < rcut < min(L)/2");
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, RSDFT_E_CUDA, "no CUDA device");
    }
    rsdft_ctx *ctx = new rsdft_ctx();
    if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        ctx->num_sms = 1;
    }
    for (int a = 0; a < 3; ++a) {
        ctx->N[a] = grid->n[a];
        ctx->L[a] = L[a];
        ctx->fft.ax[a] = plans[a];
    }
    ctx->n = (long long)grid->n[0] * grid->n[1] * grid->n[2];
    ctx->dV = L[0] * L[1] * L[2] / (double)ctx->n;
    rsdft_status st = build_fft_tables(ctx);
    if (st == RSDFT_OK) st = upload(ctx, &ctx->vloc, v_loc_host, (size_t)ctx->n);
    if (st == RSDFT_OK) st = upload(ctx, &ctx->v, v_loc_host, (size_t)ctx->n);
    if (st == RSDFT_OK) st = dev_alloc(ctx, (void **)&ctx->v32, (size_t)ctx->n * sizeof(float));
    if (st == RSDFT_OK) {
        rsdft_projectors none{0, nullptr, 1, 1.0, 1.0, nullptr};
        st = build_projectors(ctx, proj ? proj : &none);
    }
    if (st != RSDFT_OK) {
        g_create_error = ctx->err;
        rsdft_destroy(ctx);
        return st;
    }
    *out = ctx;
    return RSDFT_OK;
}

void rsdft_destroy(rsdft_ctx *ctx) {
    if (!ctx) return;
    cudaDeviceSynchronize();
    for (auto &r : ctx->prof.pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : ctx->prof.pool) cudaEventDestroy(e);
    for (void *p : ctx->owned) cudaFree(p);
    if (ctx->ws.hbuf) cudaFreeHost(ctx->ws.hbuf);
    cudaGetLastError();
    delete ctx;
}

const char *rsdft_last_error(const rsdft_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

long long rsdft_projector_entries(const rsdft_ctx *ctx) { return ctx ? ctx->nent : 0; }

rsdft_status rsdft_gaussian_vloc(const rsdft_cell *cell, const rsdft_grid *grid, int natom,
                                 const double *pos_host, double Z, double sigma,
                                 double *out_host) {
    double L[3];
    RS_TRY(check_cell_grid(cell, grid, nullptr, nullptr, L));
    if (!out_host || natom < 0 || (natom > 0 && !pos_host) || !(sigma > 0.0))
        return fail(nullptr, RSDFT_E_INVALID, "bad arguments to rsdft_gaussian_vloc");
    const int Nx = grid->n[0], Ny = grid->n[1], Nz = grid->n[2];
    const size_t n = (size_t)Nx * Ny * Nz;
    for (size_t i = 0; i < n; ++i) out_host[i] = 0.0;
    std::vector<double> dx(Nx), dy(Ny), dz(Nz);
    const double inv = 1.0 / (2.0 * sigma * sigma);
    for (int a = 0; a < natom; ++a) {
        const double *R = pos_host + 3 * a;
        for (int i = 0; i < Nx; ++i) dx[i] = min_image(i * (L[0] / Nx) - R[0], L[0]);
        for (int i = 0; i < Ny; ++i) dy[i] = min_image(i * (L[1] / Ny) - R[1], L[1]);
        for (int i = 0; i < Nz; ++i) dz[i] = min_image(i * (L[2] / Nz) - R[2], L[2]);
        for (int z = 0; z < Nz; ++z)
            for (int y = 0; y < Ny; ++y) {
                double dyz = dy[y] * dy[y] + dz[z] * dz[z];
                double *row = out_host + ((size_t)z * Ny + y) * Nx;
                for (int x = 0; x < Nx; ++x) row[x] -= Z * std::exp(-(dx[x] * dx[x] + dyz) * inv);
            }
    }
    return RSDFT_OK;
}

rsdft_status rsdft_set_potential(rsdft_ctx *ctx, const double *v, int on_device, void *stream) {
    if (!ctx || !v) return fail(ctx, RSDFT_E_INVALID, "ctx and v are required");
    RS_CUDA(ctx, cudaMemcpyAsync(ctx->v, v, (size_t)ctx->n * sizeof(double),
                                 on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                 as_stream(stream)));
    if (!on_device) RS_CUDA(ctx, cudaStreamSynchronize(as_stream(stream)));
    return RSDFT_OK;
}

}  // extern "C"

namespace rsdft {

static cudaEvent_t pool_get(Profiler &p) {
    if (!p.pool.empty()) {
        cudaEvent_t e = p.pool.back();
        p.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    return e;
}

ProfScope::ProfScope(rsdft_ctx *c, int kid, double fl, double by, cudaStream_t s, int nlaunch)
    : ctx(c), st(s), id(kid), flops(fl), bytes(by) {
    ctx->launches += nlaunch;
    if (!ctx->prof.on) return;
    a = pool_get(ctx->prof);
    if (a) cudaEventRecord(a, st);
}

ProfScope::~ProfScope() {
    if (!a) return;
    cudaEvent_t b = pool_get(ctx->prof);
    if (!b) return;
    cudaEventRecord(b, st);
    ctx->prof.pending.push_back(Profiler::Rec{a, b, id, flops, bytes});
}

static void prof_drain(rsdft_ctx *ctx) {
    Profiler &p = ctx->prof;
    for (auto &r : p.pending) {
        float ms = 0.f;
        cudaEventSynchronize(r.b);
        cudaEventElapsedTime(&ms, r.a, r.b);
        p.ms[r.id] += ms;
        p.flops[r.id] += r.flops;
        p.bytes[r.id] += r.bytes;
        p.count[r.id] += 1;
        p.pool.push_back(r.a);
        p.pool.push_back(r.b);
    }
    p.pending.clear();
    cudaGetLastError();
}

}  // namespace rsdft

extern "C" {

rsdft_status rsdft_profile_enable(rsdft_ctx *ctx, int on) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    prof_drain(ctx);
    Profiler &p = ctx->prof;
    for (int i = 0; i < RSDFT_K_COUNT; ++i) { p.ms[i] = p.flops[i] = p.bytes[i] = 0.0; p.count[i] = 0; }
    p.on = on != 0;
    return RSDFT_OK;
}

rsdft_status rsdft_profile_read(rsdft_ctx *ctx, int id, double *ms, long long *launches,
                                double *flops, double *bytes) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (id < 0 || id >= RSDFT_K_COUNT) return fail(ctx, RSDFT_E_INVALID, "bad kernel id");
    prof_drain(ctx);
    const Profiler &p = ctx->prof;
    if (ms) *ms = p.ms[id];
    if (launches) *launches = p.count[id];
    if (flops) *flops = p.flops[id];
    if (bytes) *bytes = p.bytes[id];
    return RSDFT_OK;
}

long long rsdft_launch_count(const rsdft_ctx *ctx) { return ctx ? ctx->launches : 0; }

}  // extern "C"
