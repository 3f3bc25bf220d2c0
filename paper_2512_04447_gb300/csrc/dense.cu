// Dense core of the Rayleigh-Ritz step (SCF task (3), Eq. 1), FP64 complex,
// all on the device:
//   Cholesky G_S = L L^H (blocked, right-looking; a column whose pivot falls to
//   the floor is dropped), compaction to the kept columns, two triangular
//   solves K = L^-1 G_H L^-H, the lowest eigenpairs of K (Householder
//   tridiagonalisation, Sturm bisection, inverse iteration, Gram-Schmidt within
//   eigenvalue clusters, back-transformation), and C = L^-H Z.
// Matrices are row-major k x k complex128 with leading dimension ld.
#include <cfloat>
#include <cmath>

#include <mutex>

#include "dfloat.h"
#include "rsdft_internal.h"

namespace rsdft {

constexpr int NBK = 32;   // block size of the Cholesky and the triangular solves
constexpr int MAX_K_COOP = 4096;   // largest subspace for the cooperative tridiagonalisation

__device__ __forceinline__ double2 c_mul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 c_mulc(double2 a, double2 b) {  // a * conj(b)
    return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ double2 c_conj(double2 a) { return make_double2(a.x, -a.y); }
// s += a b and s -= a b as four FMAs each (an FP64 instruction costs the same
// whether or not it fuses, so complex products are written as FMA chains)
__device__ __forceinline__ void c_fma(double2 &s, double2 a, double2 b) {
    s.x = fma(a.x, b.x, fma(-a.y, b.y, s.x));
    s.y = fma(a.x, b.y, fma(a.y, b.x, s.y));
}
__device__ __forceinline__ void c_fms(double2 &s, double2 a, double2 b) {
    s.x = fma(-a.x, b.x, fma(a.y, b.y, s.x));
    s.y = fma(-a.x, b.y, fma(-a.y, b.x, s.y));
}

// 1/x in FP64 by the Newton-Raphson iteration y <- y + y (1 - x y) from an FP32
// seed: each step squares the relative error (2^-23 -> 2^-46 -> below one ulp),
// two FMA pairs instead of the long FP64 division sequence.  Arguments outside
// the FP32 range take the division.
__device__ __forceinline__ double rcp_nr(double x) {
    const float xf = (float)x;
    const float ax = fabsf(xf);
    if (!(ax > 1e-30f && ax < 1e30f)) return 1.0 / x;
    double y = (double)__frcp_rn(xf);
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}


// Block-wide sum of one double (blockDim.x a multiple of 32, <= 1024); the warp
// partials are combined by warp 0 with shuffles (a chain of dependent FP64 adds
// in one thread costs ~64 cycles per add on this part).
__device__ double block_sum(double v, double *sh) {
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

// ---- grid barrier of the cooperative kernels ----------------------------------------
// Values written by other blocks of a cooperative launch are read with
// ld.global.cg (L2, not the incoherent L1).  Every barrier wait is bounded: on
// timeout the block sets the error flag and returns, and the others see the
// flag and return.
struct GridSync {
    unsigned int count;
    unsigned int gen;
    int err;
    int pad;
};

__device__ __forceinline__ double2 ldcg2(const double2 *p) { return __ldcg(p); }

std::mutex &coop_mutex() {
    static std::mutex m;
    return m;
}

// Grid barrier on a monotonic arrival counter (zeroed before the launch): the
// e-th barrier of the launch completes when count reaches nblocks * (e + 1).
// The wait is bounded by `limit` SM cycles; a block that gives up sets the
// error flag, and blocks that see the flag stop waiting.
__device__ bool grid_sync(GridSync *g, unsigned int nblocks, long long limit, int *s_ok, unsigned int &epoch) {
    __threadfence();
    __syncthreads();
    ++epoch;
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned int *vcount = &g->count;
        volatile int *verr = &g->err;
        const unsigned int target = nblocks * epoch;
        atomicAdd(&g->count, 1u);
        const long long t0 = clock64();
        while (*vcount < target) {
            if (*verr) { ok = 0; break; }
            if (clock64() - t0 > limit) { atomicExch(&g->err, 1); ok = 0; break; }
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// ---- Cholesky with dropping -----------------------------------------------------
__global__ void k_maxdiag(const double2 *__restrict__ a, int k, int ld, double tol, double *out) {
    __shared__ double sh[33];
    double m = 0.0;
    for (int i = threadIdx.x; i < k; i += blockDim.x) m = fmax(m, a[(size_t)i * ld + i].x);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, sh[w]);
        out[0] = tol * r;
    }
}

// Cholesky of G_S, right-looking in panels of NBK columns.  Per panel kb:
//  (1) every CTA loads the nb x nb diagonal block and factors it in shared
//      memory (column c is dropped when its Schur pivot is <= the floor:
//      l_cc = 1 and L[c+1:, c] = 0);
//  (2) the rows below the block, l_i = a_i L11^-H, one warp per row (lane c
//      holds column c; one FP64 chain of nb steps per row);
//  (3) the trailing update a_ij -= sum_c l_ic conj(l_jc), i >= j, in CHOL_TS
//      square tiles spread over the CTAs.
// One cooperative launch runs all panels with a grid barrier after (2) and
// after (3); where the cooperative launch is refused, (1)+(2) and (3) run as
// one launch each per panel.
constexpr int CHOL_TS = 16;

__device__ void chol_factor_diag(const double2 *a, int ld, int kb, int nb, double floor_,
                                 double2 (*sD)[NBK + 1], double *s_l, double *s_il, int *s_drop) {
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
        const int r = t / nb, c = t % nb;
        sD[r][c] = c <= r ? ldcg2(a + (size_t)(kb + r) * ld + kb + c) : make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int c = 0; c < nb; ++c) {
        if (threadIdx.x == 0) {
            const double d = sD[c][c].x;
            const int dr = !(d > floor_);
            s_drop[c] = dr;
            s_l[c] = dr ? 1.0 : sqrt(d);
            s_il[c] = dr ? 1.0 : rcp_nr(s_l[c]);
            sD[c][c] = make_double2(s_l[c], 0.0);
        }
        __syncthreads();
        const int dr = s_drop[c];
        const double inv = s_il[c];
        for (int i = c + 1 + threadIdx.x; i < nb; i += blockDim.x) {
            const double2 x = sD[i][c];
            sD[i][c] = dr ? make_double2(0.0, 0.0) : make_double2(x.x * inv, x.y * inv);
        }
        __syncthreads();
        if (!dr) {
            // lower triangle of the trailing block, (i, c2) with c2 <= i, packed:
            // t -> row offset ri with ri (ri + 1) / 2 <= t
            const int m = nb - (c + 1);
            for (int t = threadIdx.x; t < m * (m + 1) / 2; t += blockDim.x) {
                int ri = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
                while (ri * (ri + 1) / 2 > t) --ri;
                while ((ri + 1) * (ri + 2) / 2 <= t) ++ri;
                const int i = c + 1 + ri, c2 = c + 1 + (t - ri * (ri + 1) / 2);
                // -= l_i conj(l_c2), as four FMAs
                const double2 p = sD[i][c], q = sD[c2][c];
                double2 x = sD[i][c2];
                x.x = fma(-p.x, q.x, fma(-p.y, q.y, x.x));
                x.y = fma(-p.y, q.x, fma(p.x, q.y, x.y));
                sD[i][c2] = x;
            }
        }
        __syncthreads();
    }
}

// The same factorisation of the diagonal block in double-float (dfloat.h), for
// pivot floors >= 1e-6 (the mixed form): the block's columns are a sequential
// chain of a square root, a reciprocal and small updates, all on the FP32 pipe
// (an FP64 square root or reciprocal is a chain of FP64 instructions of 64
// cycles each on GB300).  sD holds complex double-floats (float4, the size of a
// double2) during the factorisation and the FP64 factor at the end.
__device__ void chol_factor_diag_df(const double2 *a, int ld, int kb, int nb, double floor_,
                                    double2 (*sD)[NBK + 1], double *s_l, double *s_il, int *s_drop) {
    float4(*sF)[NBK + 1] = reinterpret_cast<float4(*)[NBK + 1]>(sD);
    __shared__ float2 s_ildf[NBK];
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
        const int r = t / nb, c = t % nb;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c <= r) {
            const double2 x = ldcg2(a + (size_t)(kb + r) * ld + kb + c);
            const dfl::df xr = dfl::from_double(x.x), xi = dfl::from_double(x.y);
            v = make_float4(xr.h, xr.l, xi.h, xi.l);
        }
        sF[r][c] = v;
    }
    __syncthreads();
    for (int c = 0; c < nb; ++c) {
        if (threadIdx.x == 0) {
            const dfl::df d{sF[c][c].x, sF[c][c].y};
            const int dr = !(dfl::to_double(d) > floor_);
            s_drop[c] = dr;
            const dfl::df l = dr ? dfl::mk(1.0f) : dfl::sqrt(d);
            const dfl::df il = dr ? dfl::mk(1.0f) : dfl::div(dfl::mk(1.0f), l);
            s_l[c] = dfl::to_double(l);
            s_il[c] = dfl::to_double(il);
            s_ildf[c] = make_float2(il.h, il.l);
            sF[c][c] = make_float4(l.h, l.l, 0.f, 0.f);
        }
        __syncthreads();
        const int dr = s_drop[c];
        const dfl::df inv{s_ildf[c].x, s_ildf[c].y};
        for (int i = c + 1 + threadIdx.x; i < nb; i += blockDim.x) {
            const float4 x = sF[i][c];
            if (dr) {
                sF[i][c] = make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                const dfl::df xr = dfl::mul(dfl::df{x.x, x.y}, inv), xi = dfl::mul(dfl::df{x.z, x.w}, inv);
                sF[i][c] = make_float4(xr.h, xr.l, xi.h, xi.l);
            }
        }
        __syncthreads();
        if (!dr) {
            const int m = nb - (c + 1);
            for (int t = threadIdx.x; t < m * (m + 1) / 2; t += blockDim.x) {
                int ri = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
                while (ri * (ri + 1) / 2 > t) --ri;
                while ((ri + 1) * (ri + 2) / 2 <= t) ++ri;
                const int i = c + 1 + ri, c2 = c + 1 + (t - ri * (ri + 1) / 2);
                // -= l_i conj(l_c2)
                const float4 p = sF[i][c], q = sF[c2][c], x = sF[i][c2];
                const dfl::df pr{p.x, p.y}, pi{p.z, p.w}, qr{q.x, q.y}, qi{q.z, q.w};
                const dfl::df re = dfl::sub(dfl::df{x.x, x.y}, dfl::add(dfl::mul(pr, qr), dfl::mul(pi, qi)));
                const dfl::df im = dfl::sub(dfl::df{x.z, x.w}, dfl::sub(dfl::mul(pi, qr), dfl::mul(pr, qi)));
                sF[i][c2] = make_float4(re.h, re.l, im.h, im.l);
            }
        }
        __syncthreads();
    }
    // to FP64 in place (each element read and written by one thread)
    for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
        const int r = t / nb, c = t % nb;
        const float4 v = sF[r][c];
        sD[r][c] = make_double2(dfl::to_double(dfl::df{v.x, v.y}), dfl::to_double(dfl::df{v.z, v.w}));
    }
    __syncthreads();
}

// Rows i >= kb+nb of the panel: l_i = a_i L11^-H by forward substitution, warp
// wid of nw takes rows kb+nb+wid, kb+nb+wid+nw, ...
__device__ void chol_panel_rows(double2 *a, int k, int ld, int kb, int nb, const double2 (*sD)[NBK + 1],
                                const double *s_il, const int *s_drop, int wid, int nw) {
    const int lane = threadIdx.x & 31;
    for (int i = kb + nb + wid; i < k; i += nw) {
        double2 *row = a + (size_t)i * ld + kb;
        double2 v = lane < nb ? ldcg2(row + lane) : make_double2(0.0, 0.0);
        for (int c = 0; c < nb; ++c) {
            double2 x = make_double2(0.0, 0.0);
            if (lane == c && !s_drop[c]) {
                const double inv = s_il[c];
                x = make_double2(v.x * inv, v.y * inv);
            }
            x.x = __shfl_sync(0xffffffffu, x.x, c);
            x.y = __shfl_sync(0xffffffffu, x.y, c);
            if (lane == c) v = x;
            else if (lane > c && lane < nb) {   // v -= x conj(l_lane,c)
                const double2 q = sD[lane][c];
                v.x = fma(-x.x, q.x, fma(-x.y, q.y, v.x));
                v.y = fma(-x.y, q.x, fma(x.x, q.y, v.y));
            }
        }
        if (lane < nb) row[lane] = v;
    }
}

// Trailing-update tile (ti, tj), ti >= tj, of the rows/columns >= kb+nb:
// a[i][j] -= sum_{c in panel} l[i][c] conj(l[j][c]) for j <= i.
__device__ void chol_update_tile(double2 *a, int k, int ld, int kb, int nb, int ti, int tj,
                                 double2 (*Li)[NBK + 1], double2 (*Lj)[NBK + 1]) {
    const int t0 = kb + nb;
    const int i0 = t0 + ti * CHOL_TS, j0 = t0 + tj * CHOL_TS;
    __syncthreads();   // the previous tile's readers of Li, Lj are done
    for (int t = threadIdx.x; t < CHOL_TS * nb; t += blockDim.x) {
        const int r = t / nb, c = t % nb;
        Li[r][c] = (i0 + r < k) ? ldcg2(a + (size_t)(i0 + r) * ld + kb + c) : make_double2(0.0, 0.0);
        Lj[r][c] = (j0 + r < k) ? ldcg2(a + (size_t)(j0 + r) * ld + kb + c) : make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < CHOL_TS * CHOL_TS; t += blockDim.x) {
        const int r = t / CHOL_TS, s = t % CHOL_TS;
        const int i = i0 + r, j = j0 + s;
        if (i >= k || j >= k || j > i) continue;
        double sx = 0.0, sy = 0.0;
        for (int c = 0; c < nb; ++c) {   // l_i conj(l_j) as four FMAs
            const double2 p = Li[r][c], q = Lj[s][c];
            sx = fma(p.x, q.x, fma(p.y, q.y, sx));
            sy = fma(p.y, q.x, fma(-p.x, q.y, sy));
        }
        double2 *x = a + (size_t)i * ld + j;
        const double2 x0 = ldcg2(x);
        *x = make_double2(x0.x - sx, x0.y - sy);
    }
}

__device__ __forceinline__ void tri_index(int t, int &ti, int &tj) {
    int r = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while (r * (r + 1) / 2 > t) --r;
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    ti = r;
    tj = t - r * (r + 1) / 2;
}

// All panels in one cooperative launch; drop flags to drop[0..k), and the
// kept-column list (keep[0..kc), keep[k] = kc) at the end.
template <bool DF>
__global__ void __launch_bounds__(256)
k_chol_coop(double2 *a, int k, int ld, const double *floorp, int *drop, int *keep, GridSync *gs, long long limit) {
    __shared__ double2 sD[NBK][NBK + 1];
    __shared__ double2 Li[CHOL_TS][NBK + 1], Lj[CHOL_TS][NBK + 1];
    __shared__ double s_l[NBK], s_il[NBK];
    __shared__ int s_drop[NBK];
    __shared__ int s_ok;
    unsigned int epoch = 0;
    const double floor_ = floorp[0];
    const int nw = (int)(gridDim.x * (blockDim.x >> 5));
    const int wid = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
    for (int kb = 0; kb < k; kb += NBK) {
        const int nb = min(NBK, k - kb);
        if (DF) chol_factor_diag_df(a, ld, kb, nb, floor_, sD, s_l, s_il, s_drop);
        else chol_factor_diag(a, ld, kb, nb, floor_, sD, s_l, s_il, s_drop);
        if (blockIdx.x == 0)
            for (int c = threadIdx.x; c < nb; c += blockDim.x) drop[kb + c] = s_drop[c];
        chol_panel_rows(a, k, ld, kb, nb, sD, s_il, s_drop, wid, nw);
        const int rest = k - kb - nb;
        if (rest > 0 && !grid_sync(gs, gridDim.x, limit, &s_ok, epoch)) return;
        // every CTA has read the diagonal block: store its factor
        if (blockIdx.x == 0) {
            for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
                const int r = t / nb, c = t % nb;
                if (c <= r) a[(size_t)(kb + r) * ld + kb + c] = sD[r][c];
            }
        }
        if (rest > 0) {
            const int nt = (rest + CHOL_TS - 1) / CHOL_TS;
            for (int t = blockIdx.x; t < nt * (nt + 1) / 2; t += gridDim.x) {
                int ti, tj;
                tri_index(t, ti, tj);
                chol_update_tile(a, k, ld, kb, nb, ti, tj, Li, Lj);
            }
            if (!grid_sync(gs, gridDim.x, limit, &s_ok, epoch)) return;
        }
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int c = 0;
        for (int i = 0; i < k; ++i)
            if (!drop[i]) keep[c++] = i;
        keep[k] = c;
    }
}

// Fallback, one panel per pair of launches: (1)+(2) with the factored block
// to diag_out (other CTAs of the launch may not have read the original yet),
// then (3) with block (0, 0) storing the factored block from diag_out.
__global__ void __launch_bounds__(256)
k_chol_panel(double2 *a, int k, int ld, int kb, int nb, const double *floorp, int *drop, double2 *diag_out) {
    __shared__ double2 sD[NBK][NBK + 1];
    __shared__ double s_l[NBK], s_il[NBK];
    __shared__ int s_drop[NBK];
    chol_factor_diag(a, ld, kb, nb, floorp[0], sD, s_l, s_il, s_drop);
    if (blockIdx.x == 0) {
        for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) diag_out[t] = sD[t / nb][t % nb];
        for (int c = threadIdx.x; c < nb; c += blockDim.x) drop[kb + c] = s_drop[c];
    }
    chol_panel_rows(a, k, ld, kb, nb, sD, s_il, s_drop,
                    (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)), (int)(gridDim.x * (blockDim.x >> 5)));
}

__global__ void __launch_bounds__(256)
k_chol_update(double2 *a, int k, int ld, int kb, int nb, const double2 *__restrict__ diag) {
    __shared__ double2 Li[CHOL_TS][NBK + 1], Lj[CHOL_TS][NBK + 1];
    if (blockIdx.x == 0 && blockIdx.y == 0) {
        for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
            const int r = t / nb, c = t % nb;
            if (c <= r) a[(size_t)(kb + r) * ld + kb + c] = diag[t];
        }
    }
    if (kb + nb >= k || blockIdx.x > blockIdx.y) return;   // uniform over the block
    chol_update_tile(a, k, ld, kb, nb, blockIdx.y, blockIdx.x, Li, Lj);
}

__global__ void k_keep_scan(const int *drop, int k, int *keep) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int c = 0;
    for (int i = 0; i < k; ++i)
        if (!drop[i]) keep[c++] = i;
    keep[k] = c;
}

// out[r][s] = in[keep[r]][keep[s]] for r, s < kc.
__global__ void k_gather_sq(const double2 *__restrict__ in, int ldi, const int *__restrict__ keep,
                            int kc, double2 *__restrict__ out, int ldo) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)kc * kc) return;
    const int r = (int)(idx / kc), s = (int)(idx % kc);
    out[(size_t)r * ldo + s] = in[(size_t)keep[r] * ldi + keep[s]];
}

// out = (in^H), kc x kc
__global__ void k_conj_transpose(const double2 *__restrict__ in, int ldi, int kc,
                                 double2 *__restrict__ out, int ldo) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)kc * kc) return;
    const int r = (int)(idx / kc), s = (int)(idx % kc);
    out[(size_t)r * ldo + s] = c_conj(in[(size_t)s * ldi + r]);
}

// out = (a + a^H) / 2, kc x kc (out may not alias a)
__global__ void k_hermitise(const double2 *__restrict__ a, int lda, int kc, double2 *__restrict__ out,
                            int ldo) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)kc * kc) return;
    const int r = (int)(idx / kc), s = (int)(idx % kc);
    const double2 x = a[(size_t)r * lda + s], y = a[(size_t)s * lda + r];
    out[(size_t)r * ldo + s] = make_double2(0.5 * (x.x + y.x), 0.5 * (x.y - y.y));
}

// ---- triangular solves with the lower factor L (kc x kc) ----------------------------
// All columns of B (kc x ncol, ld ldb) in place: BACK = false solves L X = B
// (block rows of 32 from the top), BACK = true solves L^H X = B (from the
// bottom).  Columns are independent, so there is no grid-wide step: one warp
// per column, four columns per CTA; lane r holds row r of the current block
// row.  For each block row the CTA stages the 32 x 32 tiles of L (of L^H) that
// multiply the already solved block rows in shared memory, shared by its four
// columns; the diagonal block is then solved by column-oriented substitution
// (x_c final, the rows below subtract it).
template <bool BACK>
__device__ __forceinline__ double2 trsm_tile_elem(const double2 *__restrict__ L, int ldl, int r0, int nr, int c0,
                                                  int nc, int t) {
    if (!BACK) {   // L[r0+r][c0+j], j fastest (coalesced)
        const int r = t >> 5, j = t & 31;
        return (r < nr && j < nc) ? L[(size_t)(r0 + r) * ldl + c0 + j] : make_double2(0.0, 0.0);
    }
    // (L^H)[r0+r][c0+j] = conj(L[c0+j][r0+r]), r fastest (coalesced)
    const int j = t >> 5, r = t & 31;
    return (r < nr && j < nc) ? c_conj(L[(size_t)(c0 + j) * ldl + r0 + r]) : make_double2(0.0, 0.0);
}

template <bool BACK>
__global__ void __launch_bounds__(128)
k_trsm_cols(const double2 *__restrict__ L, int ldl, int kc, double2 *b, int ldb, int ncol) {
    __shared__ double2 Ts[32][33];
    __shared__ double Linv[32];
    constexpr int PER = 32 * 32 / 128;   // tile elements staged per thread
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int col = blockIdx.x * 4 + warp;
    const bool act = col < ncol;          // uniform over the warp
    const int nblk = (kc + 31) / 32;
    const double2 zero = make_double2(0.0, 0.0);
    for (int s = 0; s < nblk; ++s) {
        const int rb = BACK ? nblk - 1 - s : s;
        const int r0 = rb * 32, nr = min(32, kc - r0);
        double2 acc = (act && lane < nr) ? b[(size_t)(r0 + lane) * ldb + col] : zero;
        const int j_lo = BACK ? rb + 1 : 0, j_hi = BACK ? nblk : rb;
        // the next tile is fetched into registers while the current one is used
        double2 pre[PER];
        if (j_lo < j_hi) {
            const int c0 = j_lo * 32, nc = min(32, kc - c0);
#pragma unroll
            for (int q = 0; q < PER; ++q) pre[q] = trsm_tile_elem<BACK>(L, ldl, r0, nr, c0, nc, threadIdx.x + q * 128);
        }
        for (int jb = j_lo; jb < j_hi; ++jb) {
            const int c0 = jb * 32, nc = min(32, kc - c0);
            __syncthreads();   // the previous tile's readers are done
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int t = threadIdx.x + q * 128;
                if (!BACK) Ts[t >> 5][t & 31] = pre[q];
                else Ts[t & 31][t >> 5] = pre[q];
            }
            __syncthreads();
            if (jb + 1 < j_hi) {
                const int c1 = c0 + 32, nc1 = min(32, kc - c1);
#pragma unroll
                for (int q = 0; q < PER; ++q)
                    pre[q] = trsm_tile_elem<BACK>(L, ldl, r0, nr, c1, nc1, threadIdx.x + q * 128);
            }
            // solved rows c0.. of this column (written by this lane earlier)
            const double2 xj = (act && lane < nc) ? b[(size_t)(c0 + lane) * ldb + col] : zero;
#pragma unroll 8
            for (int j = 0; j < 32; ++j) {
                double2 x;
                x.x = __shfl_sync(0xffffffffu, xj.x, j);
                x.y = __shfl_sync(0xffffffffu, xj.y, j);
                c_fms(acc, Ts[lane][j], x);
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
            const int r = t >> 5, j = t & 31;
            Ts[r][j] = (r < nr && j < nr) ? L[(size_t)(r0 + r) * ldl + r0 + j] : zero;
        }
        if (threadIdx.x < nr) Linv[threadIdx.x] = 1.0 / L[(size_t)(r0 + threadIdx.x) * ldl + r0 + threadIdx.x].x;
        __syncthreads();
        double2 v = acc;
        if (!BACK) {
            for (int c = 0; c < nr; ++c) {
                const double inv = Linv[c];   // real positive diagonal
                double2 x = make_double2(v.x * inv, v.y * inv);
                x.x = __shfl_sync(0xffffffffu, x.x, c);
                x.y = __shfl_sync(0xffffffffu, x.y, c);
                if (lane == c) v = x;
                else if (lane > c && lane < nr) c_fms(v, Ts[lane][c], x);
            }
        } else {   // (L^H)[r][c] = conj(L[c][r])
            for (int c = nr - 1; c >= 0; --c) {
                const double inv = Linv[c];
                double2 x = make_double2(v.x * inv, v.y * inv);
                x.x = __shfl_sync(0xffffffffu, x.x, c);
                x.y = __shfl_sync(0xffffffffu, x.y, c);
                if (lane == c) v = x;
                else if (lane < c) c_fms(v, c_conj(Ts[c][lane]), x);
            }
        }
        if (act && lane < nr) b[(size_t)(r0 + lane) * ldb + col] = v;
    }
}

static rsdft_status trsm_lower(rsdft_ctx *ctx, const double2 *L, int ldl, int kc, double2 *b,
                               int ldb, int ncol, cudaStream_t st) {
    if (kc <= 0 || ncol <= 0) return RSDFT_OK;
    k_trsm_cols<false><<<cdiv(ncol, 4), 128, 0, st>>>(L, ldl, kc, b, ldb, ncol);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "trsm_lower");
    return RSDFT_OK;
}

static rsdft_status trsm_upperH(rsdft_ctx *ctx, const double2 *L, int ldl, int kc, double2 *b,
                                int ldb, int ncol, cudaStream_t st) {
    if (kc <= 0 || ncol <= 0) return RSDFT_OK;
    k_trsm_cols<true><<<cdiv(ncol, 4), 128, 0, st>>>(L, ldl, kc, b, ldb, ncol);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "trsm_upperH");
    return RSDFT_OK;
}

// ---- Hermitian eigensolver ----------------------------------------------------------
// Householder step i (LAPACK zhetd2 convention, lower): reflector H = I - tau v v^H
// with v[0] = 1 such that H^H (alpha, x)^T = (beta, 0)^T, beta real.
__global__ void k_house_reflector(double2 *a, int k, int ld, int i, double2 *vh, int ldv,
                                  double2 *tau, double *d, double *e) {
    __shared__ double sh[33];
    const int L = k - i - 1;
    const double2 alpha = a[(size_t)(i + 1) * ld + i];
    double s = 0.0;
    for (int r = 1 + threadIdx.x; r < L; r += blockDim.x) {
        const double2 x = a[(size_t)(i + 1 + r) * ld + i];
        s += x.x * x.x + x.y * x.y;
    }
    const double xnorm2 = block_sum(s, sh);
    double2 t;
    double beta;
    double2 scal = make_double2(0.0, 0.0);
    if (xnorm2 == 0.0 && alpha.y == 0.0) {
        t = make_double2(0.0, 0.0);
        beta = alpha.x;
    } else {
        beta = -copysign(sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xnorm2), alpha.x);
        t = make_double2((beta - alpha.x) / beta, -alpha.y / beta);
        // scal = 1 / (alpha - beta)
        const double2 den = make_double2(alpha.x - beta, alpha.y);
        const double dd = den.x * den.x + den.y * den.y;
        scal = make_double2(den.x / dd, -den.y / dd);
    }
    double2 *v = vh + (size_t)i * ldv + (i + 1);
    for (int r = threadIdx.x; r < L; r += blockDim.x) {
        if (r == 0) v[0] = make_double2(1.0, 0.0);
        else v[r] = c_mul(a[(size_t)(i + 1 + r) * ld + i], scal);
    }
    if (threadIdx.x == 0) {
        tau[i] = t;
        e[i] = beta;
        d[i] = a[(size_t)i * ld + i].x;
    }
}

// w[r] = tau * sum_c A22[r][c] v[c]; one warp per row.
__global__ void k_house_matvec(const double2 *__restrict__ a, int k, int ld, int i,
                               const double2 *__restrict__ vh, int ldv, const double2 *__restrict__ tau,
                               double2 *__restrict__ w) {
    const int L = k - i - 1;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= L) return;
    const double2 *row = a + (size_t)(i + 1 + warp) * ld + (i + 1);
    const double2 *v = vh + (size_t)i * ldv + (i + 1);
    double sx = 0.0, sy = 0.0;
    for (int c = lane; c < L; c += 32) {
        const double2 p = c_mul(row[c], v[c]);
        sx += p.x;
        sy += p.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_down_sync(0xffffffffu, sx, o);
        sy += __shfl_down_sync(0xffffffffu, sy, o);
    }
    if (lane == 0) w[warp] = c_mul(tau[i], make_double2(sx, sy));
}

// alpha = -1/2 tau (w^H v); w += alpha v
__global__ void k_house_w(int k, int i, const double2 *__restrict__ vh, int ldv,
                          const double2 *__restrict__ tau, double2 *w) {
    __shared__ double sh[33];
    const int L = k - i - 1;
    const double2 *v = vh + (size_t)i * ldv + (i + 1);
    double sx = 0.0, sy = 0.0;
    for (int r = threadIdx.x; r < L; r += blockDim.x) {
        const double2 p = c_mul(c_conj(w[r]), v[r]);
        sx += p.x;
        sy += p.y;
    }
    sx = block_sum(sx, sh);
    sy = block_sum(sy, sh);
    const double2 tw = c_mul(tau[i], make_double2(sx, sy));
    const double2 alpha = make_double2(-0.5 * tw.x, -0.5 * tw.y);
    for (int r = threadIdx.x; r < L; r += blockDim.x) {
        const double2 p = c_mul(alpha, v[r]);
        w[r].x += p.x;
        w[r].y += p.y;
    }
}

// A22 -= v w^H + w v^H
__global__ void k_house_rank2(double2 *a, int k, int ld, int i, const double2 *__restrict__ vh, int ldv,
                              const double2 *__restrict__ w) {
    const int L = k - i - 1;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (c >= L || r >= L) return;
    const double2 *v = vh + (size_t)i * ldv + (i + 1);
    const double2 p = c_mulc(v[r], w[c]);
    const double2 q = c_mulc(w[r], v[c]);
    double2 &x = a[(size_t)(i + 1 + r) * ld + (i + 1 + c)];
    x.x -= p.x + q.x;
    x.y -= p.y + q.y;
}

// ---- cooperative tridiagonalisation ------------------------------------------------
// All Householder steps in one cooperative launch with ONE grid barrier per
// step.  With A^(i) the matrix after i reflectors, v_i the i-th reflector (on
// rows/columns i+1..k-1, v_i[0] = 1) and w_i = tau_i A^(i)_22 v_i known to all
// blocks after a barrier, step i is, in every block:
//   w'_i = w_i - 1/2 tau_i (w_i^H v_i) v_i                      (redundant, O(k))
//   column i+1 of A^(i+1) = column i+1 of A^(i) - v_i conj(w'_i[0]) - w'_i
//   and its diagonal      -> reflector v_{i+1}, tau_{i+1}, beta  (redundant, O(k))
// then, over rows r >= i+2 spread over all blocks (row r stays with one warp
// for the whole launch), the rank-2 update A -= v_i w'^H_i + w'_i v^H_i on
// columns >= i+2 fused with the next matvec w_{i+1} = tau_{i+1} A^(i+1) v_{i+1}
//                                                               -> grid barrier.
// w alternates between two buffers (w_{i+1} is written while slower blocks may
// still read w_i).

// Block-wide sum of one complex value.
__device__ double2 block_sum_c(double2 v, double2 *sh2) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh2[warp] = v;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        double2 s = lane < nw ? sh2[lane] : make_double2(0.0, 0.0);
        for (int o = 16; o > 0; o >>= 1) {
            s.x += __shfl_down_sync(0xffffffffu, s.x, o);
            s.y += __shfl_down_sync(0xffffffffu, s.y, o);
        }
        if (lane == 0) sh2[32] = s;
    }
    __syncthreads();
    return sh2[32];
}

// In place: x[0..L) (x[0] = alpha) -> reflector v (v[0] = 1), with tau and
// beta (LAPACK zlarfg convention: H^H x = beta e_0, H = I - tau v v^H).
// Block-wide; every thread returns the same tau and beta.
__device__ void house_inplace(double2 *x, int L, double2 &tau, double &beta, double *sh) {
    const double2 alpha = x[0];
    double s = 0.0;
    for (int r = 1 + threadIdx.x; r < L; r += blockDim.x) s += x[r].x * x[r].x + x[r].y * x[r].y;
    const double xnorm2 = block_sum(s, sh);   // its barriers also order the reads of x[0]
    // the square root and divisions once per block (FP64 division and sqrt are
    // long instruction sequences on this part), shared through sh[0..5]
    if (threadIdx.x == 0) {
        double2 t = make_double2(0.0, 0.0), scal = make_double2(0.0, 0.0);
        double b;
        if (xnorm2 == 0.0 && alpha.y == 0.0) {
            b = alpha.x;
        } else {
            b = -copysign(sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xnorm2), alpha.x);
            const double ib = rcp_nr(b);
            t = make_double2((b - alpha.x) * ib, -alpha.y * ib);
            const double2 den = make_double2(alpha.x - b, alpha.y);
            const double idd = rcp_nr(den.x * den.x + den.y * den.y);
            scal = make_double2(den.x * idd, -den.y * idd);
        }
        sh[0] = t.x;
        sh[1] = t.y;
        sh[2] = b;
        sh[3] = scal.x;
        sh[4] = scal.y;
    }
    __syncthreads();
    tau = make_double2(sh[0], sh[1]);
    beta = sh[2];
    const double2 scal = make_double2(sh[3], sh[4]);
    for (int r = threadIdx.x; r < L; r += blockDim.x) x[r] = r == 0 ? make_double2(1.0, 0.0) : c_mul(x[r], scal);
    __syncthreads();
}

// Column segments per row of the fused update + matvec of one step: enough items
// for one per SM sub-partition (4 nb) when rows are few, at least 32 columns each.
constexpr int TRI_PARTS = 4;
__device__ __forceinline__ int tri_parts(int rows, int nb) {
    const int by_warps = rows > 0 ? (4 * nb) / rows : 1;
    const int by_cols = rows / 32;
    return max(1, min(TRI_PARTS, min(by_warps, by_cols)));
}

__global__ void __launch_bounds__(256)
k_tridiag_coop(double2 *a, int k, int ld, double2 *vh, int ldv, double2 *tau, double *d, double *e,
               double2 *wbuf, GridSync *gs, long long limit) {
    __shared__ double sh[33];
    __shared__ double2 sh2[33];
    __shared__ int s_ok;
    extern __shared__ double2 s_vw[];      // v_i, w'_i, v_{i+1}: 3k entries
    double2 *sv = s_vw, *sw = s_vw + k, *sn = s_vw + 2 * k;
    const int nb = (int)gridDim.x;
    const int wib = threadIdx.x >> 5, nwb = blockDim.x >> 5, lane = threadIdx.x & 31;
    unsigned int epoch = 0;   // barriers passed so far (same in every thread)
    if (k == 1) {
        if (blockIdx.x == 0 && threadIdx.x == 0) d[0] = a[0].x;
        return;
    }
    // reflector 0 from column 0 (every block), then w_0 = tau_0 A[1:,1:] v_0
    int L = k - 1;
    for (int r = threadIdx.x; r < L; r += blockDim.x) sv[r] = ldcg2(a + (size_t)(1 + r) * ld);
    __syncthreads();
    double2 ti;
    double beta;
    house_inplace(sv, L, ti, beta, sh);
    if (blockIdx.x == 0) {
        for (int r = threadIdx.x; r < L; r += blockDim.x) vh[1 + r] = sv[r];
        if (threadIdx.x == 0) {
            tau[0] = ti;
            e[0] = beta;
            d[0] = ldcg2(a).x;
        }
    }
    for (int r = blockIdx.x + nb * wib; r < k; r += nb * nwb) {
        if (r < 1) continue;
        const double2 *row = a + (size_t)r * ld + 1;
        double sx = 0.0, sy = 0.0;
        for (int c = lane; c < L; c += 32) {
            const double2 p = c_mul(ldcg2(row + c), sv[c]);
            sx += p.x;
            sy += p.y;
        }
        for (int o = 16; o > 0; o >>= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
        }
        if (lane == 0) wbuf[r - 1] = c_mul(ti, make_double2(sx, sy));
    }
    if (!grid_sync(gs, nb, limit, &s_ok, epoch)) return;
    int pw = 1;   // parts the current w is split into (summed on reading)
    for (int i = 0; i < k - 1; ++i) {
        L = k - i - 1;
        const double2 *w = wbuf + (size_t)(i & 1) * TRI_PARTS * k;
        double2 *wn = wbuf + (size_t)((i + 1) & 1) * TRI_PARTS * k;
        // w' = w + alpha v, alpha = -1/2 tau (w^H v); the raw column i+1 is
        // fetched in the same sweep
        // (every FP64 instruction costs the same whether or not it fuses, so the
        // redundant per-block loops below are written as FMA chains)
        double2 acc = make_double2(0.0, 0.0);
        for (int r = threadIdx.x; r < L; r += blockDim.x) {
            double2 wr = ldcg2(w + r);
            for (int p = 1; p < pw; ++p) {
                const double2 q = ldcg2(w + (size_t)p * k + r);
                wr.x += q.x;
                wr.y += q.y;
            }
            const double2 vr = sv[r];
            sw[r] = wr;
            acc.x = fma(wr.x, vr.x, acc.x);        // conj(w) v
            acc.x = fma(wr.y, vr.y, acc.x);
            acc.y = fma(wr.x, vr.y, acc.y);
            acc.y = fma(-wr.y, vr.x, acc.y);
            if (r >= 1) sn[r - 1] = ldcg2(a + (size_t)(i + 1 + r) * ld + (i + 1));
        }
        acc = block_sum_c(acc, sh2);
        const double2 tw = c_mul(ti, acc);
        const double2 alpha = make_double2(-0.5 * tw.x, -0.5 * tw.y);
        for (int r = threadIdx.x; r < L; r += blockDim.x) {
            const double2 vr = sv[r];
            double2 x = sw[r];
            x.x = fma(alpha.x, vr.x, fma(-alpha.y, vr.y, x.x));
            x.y = fma(alpha.x, vr.y, fma(alpha.y, vr.x, x.y));
            sw[r] = x;
        }
        __syncthreads();
        const double dnext = ldcg2(a + (size_t)(i + 1) * ld + (i + 1)).x - 2.0 * sw[0].x;
        if (i == k - 2) {
            if (blockIdx.x == 0 && threadIdx.x == 0) d[k - 1] = dnext;
            break;
        }
        // updated column i+1 below the diagonal -> reflector i+1
        const int Ln = L - 1;
        const double2 w0 = sw[0];
        for (int q = threadIdx.x; q < Ln; q += blockDim.x) {
            // sn - v conj(w'_0) - w'
            const double2 vq = sv[q + 1], pw = sw[q + 1];
            double2 x = sn[q];
            x.x = fma(-vq.y, w0.y, fma(-vq.x, w0.x, x.x - pw.x));
            x.y = fma(vq.x, w0.y, fma(-vq.y, w0.x, x.y - pw.y));
            sn[q] = x;
        }
        __syncthreads();
        double2 tn;
        double bn;
        house_inplace(sn, Ln, tn, bn, sh);
        if (blockIdx.x == 0) {
            for (int q = threadIdx.x; q < Ln; q += blockDim.x) vh[(size_t)(i + 1) * ldv + (i + 2) + q] = sn[q];
            if (threadIdx.x == 0) {
                tau[i + 1] = tn;
                e[i + 1] = bn;
                d[i + 1] = dnext;
            }
        }
        // rows >= i+2: A -= v w'^H + w' v^H on columns >= i+2, fused with
        // w_{i+1} = tau_{i+1} A^(i+1) v_{i+1}
        // work items (row, column segment): P segments per row when there are few
        // rows, so that up to one item lands on each SM sub-partition (warps w and
        // w + 4 of a CTA share one; items fill warp slots 0-3 of every CTA first)
        const int o = i + 1;
        const int rows = k - i - 2;
        const int P = tri_parts(rows, nb);
        const int seg = ((rows + P - 1) / P + 31) & ~31;
        for (int t = blockIdx.x + nb * wib; t < rows * P; t += nb * nwb) {
            const int rr = t / P, p = t - rr * P;
            const int r = i + 2 + rr;
            const int c0 = i + 2 + p * seg, c1 = min(k, c0 + seg);
            double2 *row = a + (size_t)r * ld;
            const double2 vr = sv[r - o], wr = sw[r - o];
            double sx = 0.0, sy = 0.0;
            // x = a - v_r conj(w_c) - w_r conj(v_c) and the matvec term x s_c as 12
            // FMAs per element (an FP64 instruction costs the same whatever it fuses)
            for (int c = c0 + lane; c < c1; c += 32) {
                const double2 xv = ldcg2(row + c);
                const double2 wc = sw[c - o], vc = sv[c - o], sc = sn[c - i - 2];
                double xr = fma(-vr.x, wc.x, xv.x);
                xr = fma(-vr.y, wc.y, xr);
                xr = fma(-wr.x, vc.x, xr);
                xr = fma(-wr.y, vc.y, xr);
                double xi = fma(-vr.y, wc.x, xv.y);
                xi = fma(vr.x, wc.y, xi);
                xi = fma(-wr.y, vc.x, xi);
                xi = fma(wr.x, vc.y, xi);
                row[c] = make_double2(xr, xi);
                sx = fma(xr, sc.x, sx);
                sx = fma(-xi, sc.y, sx);
                sy = fma(xr, sc.y, sy);
                sy = fma(xi, sc.x, sy);
            }
            for (int o2 = 16; o2 > 0; o2 >>= 1) {
                sx += __shfl_xor_sync(0xffffffffu, sx, o2);
                sy += __shfl_xor_sync(0xffffffffu, sy, o2);
            }
            if (lane == 0) wn[(size_t)p * k + rr] = c_mul(tn, make_double2(sx, sy));
        }
        pw = P;
        if (!grid_sync(gs, nb, limit, &s_ok, epoch)) return;
        double2 *t = sv;
        sv = sn;
        sn = t;
        ti = tn;
    }
}

__global__ void k_house_last(const double2 *a, int k, int ld, double *d) {
    d[k - 1] = a[(size_t)(k - 1) * ld + (k - 1)].x;
}

// Sturm count: number of eigenvalues of T below x, from the characteristic
// polynomials of the leading submatrices, p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2}
// (p_{-1} = 1): q_i = p_i / p_{i-1} < 0 exactly when consecutive p change sign, so
// the count needs no division (three FP64 operations per step).  An exact p_i = 0
// stands for q_i = 0, which counts as negative (as in the ratio form with a
// -pivmin pivot): it is replaced by -p_{i-1} 2^-400.  Both p_i and p_{i-1} are
// multiplied by the same power of two whenever the larger leaves [2^-500, 2^500]
// (exact; a value that underflows keeps its sign).  Signs are read from the bits.
__device__ int sturm_count(const double *__restrict__ d, const double *__restrict__ e2, int k, double x) {
    double pm = 1.0;            // p_{i-1}
    double p = d[0] - x;        // p_0
    if (p == 0.0) p = -0x1p-400;
    int cnt = __double2hiint(p) < 0 ? 1 : 0;
    for (int i = 1; i < k; ++i) {
        double pn = fma(d[i] - x, p, -(e2[i - 1] * pm));
        const int hn = __double2hiint(pn);
        if (((hn << 1) | __double2loint(pn)) == 0) pn = -p * 0x1p-400;
        cnt += (__double2hiint(pn) ^ __double2hiint(p)) < 0 ? 1 : 0;
        const int ea = (__double2hiint(pn) >> 20) & 0x7FF, eb = (__double2hiint(p) >> 20) & 0x7FF;
        const int ex = max(ea, eb);
        if (ex > 1023 + 500 || ex < 1023 - 500) {
            const double sc = __hiloint2double((2046 - ex) << 20, 0);   // 2^(1023 - ex)
            pn *= sc;
            p *= sc;
        }
        pm = p;
        p = pn;
    }
    return cnt;
}

// scr: [0] tnorm, [1] glo, [2] ghi, [3] pivmin, then e2[k]
__device__ double block_reduce_max(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double r = lane < nw ? sh[lane] : -1e300;
        for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_down_sync(0xffffffffu, r, o));
        if (lane == 0) sh[32] = r;
    }
    __syncthreads();
    return sh[32];
}

// Gershgorin bracket, norm and e^2 of T (one CTA).
__global__ void k_tri_prep(const double *d, const double *e, int k, double *scr) {
    __shared__ double sh[33];
    double *e2 = scr + 8;
    double tn = 0.0, nlo = -1e300, hi = -1e300, emax2 = 0.0;   // nlo = -min
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const double el = i > 0 ? fabs(e[i - 1]) : 0.0;
        const double er = i < k - 1 ? fabs(e[i]) : 0.0;
        tn = fmax(tn, fabs(d[i]) + el + er);
        nlo = fmax(nlo, -(d[i] - el - er));
        hi = fmax(hi, d[i] + el + er);
        if (i < k - 1) {
            e2[i] = e[i] * e[i];
            emax2 = fmax(emax2, e2[i]);
        }
    }
    tn = block_reduce_max(tn, sh);
    nlo = block_reduce_max(nlo, sh);
    hi = block_reduce_max(hi, sh);
    emax2 = block_reduce_max(emax2, sh);
    if (threadIdx.x == 0) {
        const double pad = 2.0 * DBL_EPSILON * fmax(tn, 1e-300) + 1e-300;
        scr[0] = tn;
        scr[1] = -nlo - pad;
        scr[2] = hi + pad;
        scr[3] = DBL_MIN * fmax(1.0, emax2);
    }
}

// Multisection for the lowest nkeep eigenvalues of T, one 128-thread CTA per
// eigenvalue j (one warp per SM sub-partition, so the four Sturm chains of a
// round run side by side): each round the threads take Sturm counts at 128
// interior points of the bracket [lo, hi] and the bracket shrinks to the
// sub-interval that holds the j-th eigenvalue (counts are monotone in x, so
// the points with count > j form a suffix); a round divides the bracket by 129
// (against 33 with one warp, so about 30% fewer sequential rounds).  Stops at
// a bracket of 4 ulps of ||T||.
constexpr int BIS_T = 128;
__global__ void __launch_bounds__(BIS_T) k_bisect(const double *d, int k, int nkeep, const double *scr, double *lam) {
    const int j = blockIdx.x;
    if (j >= nkeep) return;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    __shared__ unsigned s_ball[BIS_T / 32];
    __shared__ double s_x[BIS_T];
    const double *e2 = scr + 8;
    const double step = 1.0 / (double)(BIS_T + 1);
    double lo = scr[1], hi = scr[2];
    // the bracket is final at 4 ulps of ||T|| (absolute, as in LAPACK's bisection
    // with abstol = ulp ||T||): eigenvalues near zero need no more rounds than
    // the others
    const double tol_abs = 4.0 * DBL_EPSILON * fmax(scr[0], 1e-300);
    for (int round = 0; round < 40; ++round) {
        // lo and hi are the same in every thread (taken from shared memory)
        if (hi - lo <= tol_abs) break;
        const double x = lo + (hi - lo) * ((double)(t + 1) * step);
        const int c = sturm_count(d, e2, k, x);
        const unsigned ball = __ballot_sync(0xffffffffu, c > j);
        if (lane == 0) s_ball[warp] = ball;
        s_x[t] = x;
        __syncthreads();
        int f = -1;
        for (int w = 0; w < BIS_T / 32; ++w)
            if (s_ball[w]) {
                f = w * 32 + __ffs(s_ball[w]) - 1;
                break;
            }
        if (f < 0) {
            lo = s_x[BIS_T - 1];
        } else {
            if (f > 0) lo = s_x[f - 1];
            hi = s_x[f];
        }
        __syncthreads();
    }
    if (t == 0) lam[j] = 0.5 * (lo + hi);
}

__device__ __forceinline__ double hash_uniform(unsigned long long x) {
    x += 0x9e3779b97f4a7c15ULL;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
    x ^= x >> 31;
    return ((double)(x >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;
}

// Inverse iteration for eigenvalue j: two solves of (T - lam_j I) y = x with
// partial pivoting (row interchanges), normalising after each solve; the
// start vector is a fixed pseudo-random one.  Vector j goes to zt[j][0..k).
// One warp per eigenvalue (one CTA each, so the eigenvalues spread over the
// SMs): lane 0 runs the sequential elimination and substitutions, the warp
// does the element-wise parts.  The factors live in shared memory when 6k
// doubles fit (smem != 0), else in the per-eigenvalue scratch fac[j][6][k].
__global__ void __launch_bounds__(32)
k_inverse_iter(const double *d, const double *e, int k, int nkeep, const double *lam,
               const double *scr, double *fac, double *zt, int smem) {
    extern __shared__ double s_fac[];
    const int j = blockIdx.x;
    if (j >= nkeep) return;
    const int lane = threadIdx.x;
    const double tiny = DBL_EPSILON * fmax(scr[0], 1e-300);
    double *D = smem ? s_fac : fac + (size_t)j * 6 * k;
    double *U1 = D + k, *U2 = U1 + k, *M = U2 + k, *F = M + k, *x = F + k;
    const double s = lam[j];
    for (int i = lane; i < k; i += 32) {
        D[i] = d[i] - s;
        U1[i] = i < k - 1 ? e[i] : 0.0;
        U2[i] = 0.0;
        M[i] = 0.0;
        F[i] = 0.0;
        x[i] = hash_uniform(((unsigned long long)(j + 1) << 32) + (unsigned long long)i);
    }
    __syncwarp();
    if (lane == 0) {
        for (int i = 0; i < k - 1; ++i) {
            const double sub = e[i];
            if (fabs(D[i]) >= fabs(sub)) {
                if (D[i] == 0.0) D[i] = tiny;
                M[i] = sub * rcp_nr(D[i]);
                D[i + 1] -= M[i] * U1[i];
            } else {
                // interchange rows i and i+1, then eliminate
                const double mult = D[i] / sub;
                const double dk1 = D[i + 1], uk = U1[i], uk1 = U1[i + 1];
                D[i] = sub;
                U1[i] = dk1;
                U2[i] = uk1;
                D[i + 1] = uk - mult * dk1;
                U1[i + 1] = -mult * uk1;
                M[i] = mult;
                F[i] = 1.0;
            }
        }
    }
    __syncwarp();
    // clamp tiny pivots, then keep 1/D for the substitutions
    for (int i = lane; i < k; i += 32) {
        double di = D[i];
        if (fabs(di) < tiny) di = di < 0.0 ? -tiny : tiny;
        D[i] = 1.0 / di;
    }
    __syncwarp();
    for (int it = 0; it < 2; ++it) {
        if (lane == 0) {
            for (int i = 0; i < k - 1; ++i) {
                if (F[i] != 0.0) {
                    const double t = x[i];
                    x[i] = x[i + 1];
                    x[i + 1] = t - M[i] * x[i];
                } else {
                    x[i + 1] -= M[i] * x[i];
                }
            }
            x[k - 1] *= D[k - 1];
            if (k >= 2) x[k - 2] = (x[k - 2] - U1[k - 2] * x[k - 1]) * D[k - 2];
            for (int i = k - 3; i >= 0; --i) x[i] = (x[i] - U1[i] * x[i + 1] - U2[i] * x[i + 2]) * D[i];
        }
        __syncwarp();
        double nrm = 0.0;
        for (int i = lane; i < k; i += 32) nrm += x[i] * x[i];
        for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
        nrm = 1.0 / sqrt(nrm);
        for (int i = lane; i < k; i += 32) x[i] *= nrm;
        __syncwarp();
    }
    double *out = zt + (size_t)j * k;
    for (int i = lane; i < k; i += 32) out[i] = x[i];
}

// Gram-Schmidt (two passes) of each vector against the earlier vectors of its
// eigenvalue cluster (a maximal run of consecutive eigenvalues with gaps of at
// most 1e-6 ||T||), then normalisation.  Inverse iteration leaves two vectors
// whose eigenvalues are g apart orthogonal to about eps ||T|| / g, so outside
// such clusters the loss is below 3e-10; a wider threshold (LAPACK's 1e-3 ||T||)
// merged hundreds of distinct eigenvalues of a 1440 x 1440 problem into one
// cluster, whose Gram-Schmidt on one CTA then took most of the solve.  Clusters
// are independent: CTA j handles the cluster that starts at eigenvalue j;
// singletons are left as inverse iteration normalised them.
__global__ void k_cluster_gs(int k, int nkeep, const double *lam, const double *scr, double *zt) {
    __shared__ double sh[33];
    __shared__ double dots[1024];
    const double ortol = 1e-6 * scr[0];
    const int cstart = blockIdx.x;
    if (cstart >= nkeep) return;
    if (cstart > 0 && lam[cstart] - lam[cstart - 1] <= ortol) return;   // not a cluster start
    int cend = cstart + 1;
    while (cend < nkeep && lam[cend] - lam[cend - 1] <= ortol) ++cend;
    if (cend - cstart < 2) return;
    for (int j = cstart + 1; j < cend; ++j) {
        double *x = zt + (size_t)j * k;
        for (int pass = 0; pass < 2; ++pass) {
            for (int i0 = cstart; i0 < j; i0 += 1024) {
                const int cnt = min(1024, j - i0);
                const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
                for (int q = warp; q < cnt; q += nw) {
                    const double *y = zt + (size_t)(i0 + q) * k;
                    double s = 0.0;
                    for (int r = lane; r < k; r += 32) s += y[r] * x[r];
                    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
                    if (lane == 0) dots[q] = s;
                }
                __syncthreads();
                for (int r = threadIdx.x; r < k; r += blockDim.x) {
                    double v = x[r];
                    for (int q = 0; q < cnt; ++q) v -= dots[q] * zt[(size_t)(i0 + q) * k + r];
                    x[r] = v;
                }
                __syncthreads();
            }
        }
        double s = 0.0;
        for (int r = threadIdx.x; r < k; r += blockDim.x) s += x[r] * x[r];
        s = block_sum(s, sh);
        const double inv = 1.0 / sqrt(s);
        for (int r = threadIdx.x; r < k; r += blockDim.x) x[r] *= inv;
        __syncthreads();
    }
}

// ---- back-transformation, compact WY blocks of 32 reflectors -------------------------
// Q = H(0) H(1) ... H(k-2), H(i) = I - tau_i v_i v_i^H, v_i stored in row i of
// vh from column i+1 on (v_i[i+1] = 1; columns <= i are not part of it).  A
// block of reflectors i0 .. i0+nr-1 is H(i0) ... H(i0+nr-1) = I - V T V^H with
// T upper triangular (the forward, column-wise compact WY form of Schreiber and
// Van Loan): T[j][j] = tau_j, T[0:j][j] = -tau_j T[0:j][0:j] (V[:, 0:j]^H v_j).
constexpr int WY_NB = 32;

// S[a][j] = <v_a|v_j> (a < j, rows r > i0+j) of every block into tw[blk][a][j]:
// grid (blocks, WY_G), the block's pairs spread over WY_G CTAs of 8 warps (the dot
// products are FP64 chains: a warp FP64 instruction holds its GB300 sub-partition
// for 64 cycles, so the pairs are spread over as many SMs as there are).
constexpr int WY_G = 8;
__global__ void __launch_bounds__(256)
k_wy_gram(int k, const double2 *__restrict__ vh, int ldv, double2 *__restrict__ tw) {
    const int i0 = blockIdx.x * WY_NB, nr = min(WY_NB, (k - 1) - i0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double2 *S = tw + (size_t)blockIdx.x * WY_NB * WY_NB;
    for (int p = blockIdx.y * nw + warp; p < WY_NB * WY_NB; p += nw * gridDim.y) {
        const int a = p / WY_NB, j = p % WY_NB;
        if (a >= j || j >= nr) continue;   // uniform over the warp
        const double2 *va = vh + (size_t)(i0 + a) * ldv, *vj = vh + (size_t)(i0 + j) * ldv;
        double sx = 0.0, sy = 0.0;
        for (int r = i0 + j + 1 + lane; r < k; r += 32) {   // conj(v_a) v_j
            const double2 x = va[r], y = vj[r];
            sx = fma(x.x, y.x, fma(x.y, y.y, sx));
            sy = fma(x.x, y.y, fma(-x.y, y.x, sy));
        }
        for (int o = 16; o > 0; o >>= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
        }
        if (lane == 0) S[a * WY_NB + j] = make_double2(sx, sy);
    }
}

// One CTA (one warp) per block: T column by column from the S that k_wy_gram left in
// tw, then T over it; tw[blk][32][32] row-major.
__global__ void __launch_bounds__(32)
k_wy_tfactor(int k, const double2 *__restrict__ tau, double2 *__restrict__ tw) {
    __shared__ double2 S[WY_NB][WY_NB + 1], T[WY_NB][WY_NB + 1];
    const int i0 = blockIdx.x * WY_NB, nr = min(WY_NB, (k - 1) - i0);
    const int lane = threadIdx.x;
    double2 *g = tw + (size_t)blockIdx.x * WY_NB * WY_NB;
    for (int a = 0; a < WY_NB; ++a) S[a][lane] = (a < lane && lane < nr) ? g[a * WY_NB + lane] : make_double2(0.0, 0.0);
    __syncwarp();
    for (int j = 0; j < WY_NB; ++j) {
        const double2 tj = j < nr ? tau[i0 + j] : make_double2(0.0, 0.0);
        double2 t = make_double2(0.0, 0.0);
        if (lane < j && j < nr) {
            double2 acc = make_double2(0.0, 0.0);
            for (int c = lane; c < j; ++c) c_fma(acc, T[lane][c], S[c][j]);
            t = c_mul(make_double2(-tj.x, -tj.y), acc);
        } else if (lane == j) {
            t = tj;
        }
        T[lane][j] = t;
        __syncwarp();
    }
    for (int c = 0; c < WY_NB; ++c) g[lane * WY_NB + c] = T[lane][c];
}

// z_j = Q zt_j for each wanted eigenvector j (one CTA each, the vector in shared
// memory): blocks from the last to the first, z -= V (T (V^H z)).
__global__ void __launch_bounds__(256)
k_backtransform_wy(int k, const double2 *__restrict__ vh, int ldv, const double2 *__restrict__ tw,
                   const double *__restrict__ zt, double2 *z, int ldz) {
    extern __shared__ double2 sz[];   // [k]
    __shared__ double2 y[WY_NB], u[WY_NB];
    const int j = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r = threadIdx.x; r < k; r += blockDim.x) sz[r] = make_double2(zt[(size_t)j * k + r], 0.0);
    __syncthreads();
    const int nblk = (k - 1 + WY_NB - 1) / WY_NB;
    for (int blk = nblk - 1; blk >= 0; --blk) {
        const int i0 = blk * WY_NB, nr = min(WY_NB, (k - 1) - i0);
        // y_a = <v_a|z>, rows r > i0 + a
        for (int a = warp; a < nr; a += nw) {
            const double2 *va = vh + (size_t)(i0 + a) * ldv;
            double sx = 0.0, sy = 0.0;
            for (int r = i0 + a + 1 + lane; r < k; r += 32) {
                const double2 x = va[r], q = sz[r];
                sx = fma(x.x, q.x, fma(x.y, q.y, sx));
                sy = fma(x.x, q.y, fma(-x.y, q.x, sy));
            }
            for (int o = 16; o > 0; o >>= 1) {
                sx += __shfl_xor_sync(0xffffffffu, sx, o);
                sy += __shfl_xor_sync(0xffffffffu, sy, o);
            }
            if (lane == 0) y[a] = make_double2(sx, sy);
        }
        __syncthreads();
        if (warp == 0 && lane < nr) {   // u = T y, T upper triangular
            const double2 *Tr = tw + (size_t)blk * WY_NB * WY_NB + lane * WY_NB;
            double2 acc = make_double2(0.0, 0.0);
            for (int c = lane; c < nr; ++c) c_fma(acc, Tr[c], y[c]);
            u[lane] = acc;
        }
        __syncthreads();
        // z[r] -= sum_a v_a[r] u_a over a with r > i0 + a
        for (int r = i0 + 1 + threadIdx.x; r < k; r += blockDim.x) {
            double2 acc = sz[r];
            const int amax = min(nr, r - i0);
            for (int a = 0; a < amax; ++a) c_fms(acc, vh[(size_t)(i0 + a) * ldv + r], u[a]);
            sz[r] = acc;
        }
        __syncthreads();
    }
    for (int r = threadIdx.x; r < k; r += blockDim.x) z[(size_t)r * ldz + j] = sz[r];
}

rsdft_status eigh_lowest(rsdft_ctx *ctx, double2 *a, int k, int nkeep, double *lam_dev,
                         double2 *z, int ldz, cudaStream_t st, bool df) {
    Workspace &w = ctx->ws;
    if (k <= 0 || nkeep <= 0) return RSDFT_OK;
    if (k > w.cap_k) return fail(ctx, RSDFT_E_INVALID, "subspace %d exceeds workspace %d", k, w.cap_k);
    if (k == 1) {
        // 1 x 1: eigenvalue is the real diagonal, eigenvector 1
        RS_CUDA(ctx, cudaMemcpyAsync(lam_dev, a, sizeof(double), cudaMemcpyDeviceToDevice, st));
        double2 one = make_double2(1.0, 0.0);
        RS_CUDA(ctx, cudaMemcpyAsync(z, &one, sizeof(double2), cudaMemcpyHostToDevice, st));
        return RSDFT_OK;
    }
    const int ld = k;
    bool coop_done = false;
    std::unique_lock<std::mutex> coop_lock;
    const double kd = (double)k;
    {
        ProfScope ps(ctx, RSDFT_K_TRIDIAG, 16.0 / 3.0 * kd * kd * kd, 0.0, st, 0);
        bool cluster_done = false;
        if (df) RS_TRY(tridiag_cluster(ctx, a, k, ld, w.Vh, k, w.tau, w.d, w.e, st, &cluster_done));
        // else one cooperative launch for all Householder steps (occupancy queried
        // once, thread-safe static initialisation)
        static const int occ = [] {
            int dev = 0, coop = 0, o = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
            // the opt-in shared memory size first: the occupancy query below
            // asks for more than the default 48 KB
            if (coop == 0 ||
                cudaFuncSetAttribute(k_tridiag_coop, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     3 * MAX_K_COOP * sizeof(double2)) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_tridiag_coop, 256,
                                                              3 * MAX_K_COOP * sizeof(double2)) != cudaSuccess)
                o = 0;
            cudaGetLastError();
            return o;
        }();
        // cooperative grids of different contexts (batched cells on other streams)
        // never run at the same time: the lock is held until this call's final
        // stream synchronisation
        if (cluster_done) coop_done = true;
        const bool try_coop = !cluster_done && occ > 0 && k <= MAX_K_COOP;
        if (try_coop) coop_lock = std::unique_lock<std::mutex>(coop_mutex());
        if (try_coop) {
            int nb = std::max(1, std::min(ctx->num_sms * std::min(occ, 1), cdiv((long long)k * k, 1024)));
            GridSync *gs = reinterpret_cast<GridSync *>(w.gsync);
            RS_CUDA(ctx, cudaMemsetAsync(gs, 0, sizeof(GridSync), st));
            long long limit = 4000000000LL;   // ~2 s of SM clock per barrier wait
            double2 *vh = w.Vh, *tau = w.tau, *wv = w.wv;
            double *dd = w.d, *ee = w.e;
            int kk = k, ldd = ld, ldv = k;
            void *args[] = {&a, &kk, &ldd, &vh, &ldv, &tau, &dd, &ee, &wv, &gs, &limit};
            cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_tridiag_coop, dim3(nb), dim3(256),
                                                        args, 3 * (size_t)k * sizeof(double2), st);
            if (e == cudaSuccess) {
                count_launch(ctx);
                coop_done = true;
            } else {
                cudaGetLastError();   // fall back to one launch per phase
                ++ctx->coop_fallbacks;
                ctx->coop_last_error = (int)e;
            }
        }
        for (int i = 0; i < k - 1 && !coop_done; ++i) {
            const int L = k - i - 1;
            k_house_reflector<<<1, 256, 0, st>>>(a, k, ld, i, w.Vh, k, w.tau, w.d, w.e);
            count_launch(ctx);
            k_house_matvec<<<cdiv((long long)L * 32, 256), 256, 0, st>>>(a, k, ld, i, w.Vh, k, w.tau, w.wv);
            count_launch(ctx);
            k_house_w<<<1, 256, 0, st>>>(k, i, w.Vh, k, w.tau, w.wv);
            count_launch(ctx);
            dim3 g(cdiv(L, 128), L);
            k_house_rank2<<<g, 128, 0, st>>>(a, k, ld, i, w.Vh, k, w.wv);
            count_launch(ctx);
        }
        if (!coop_done) {
            k_house_last<<<1, 1, 0, st>>>(a, k, ld, w.d);
            count_launch(ctx);
        }
        RS_LAUNCHED(ctx, "householder");
    }
    {
        ProfScope ps(ctx, RSDFT_K_TRIEIG, kd * nkeep * (3.0 * 52.0 + 20.0), 0.0, st, 0);
        k_tri_prep<<<1, 256, 0, st>>>(w.d, w.e, k, w.dscr);
        count_launch(ctx);
        // one CTA per eigenvalue: the Sturm counts and the substitutions are
        // sequential chains, so the eigenvalues spread over the SMs.  The counts in
        // double-float (df) or FP64; the inverse iteration stays FP64 either way
        // (its vectors for eigenvalues g apart are orthogonal only to ~u ||T|| / g,
        // with u the working precision)
        if (df) {
            RS_TRY(bisect_df(ctx, k, nkeep, lam_dev, st));
        } else {
            k_bisect<<<nkeep, BIS_T, 0, st>>>(w.d, k, nkeep, w.dscr, lam_dev);
            count_launch(ctx);
        }
        const size_t ii_smem = (size_t)6 * k * sizeof(double);
        static std::mutex ii_mutex;
        static size_t ii_smem_max = 0;
        bool use_smem = ii_smem <= 48 * 1024;
        if (!use_smem && ii_smem <= 200 * 1024) {
            std::lock_guard<std::mutex> g(ii_mutex);
            if (ii_smem > ii_smem_max &&
                cudaFuncSetAttribute(k_inverse_iter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ii_smem) ==
                    cudaSuccess)
                ii_smem_max = ii_smem;
            cudaGetLastError();
            use_smem = ii_smem <= ii_smem_max;
        }
        k_inverse_iter<<<nkeep, 32, use_smem ? ii_smem : 0, st>>>(w.d, w.e, k, nkeep, lam_dev, w.dscr,
                                                                   w.fac, w.zt, use_smem ? 1 : 0);
        count_launch(ctx);
        k_cluster_gs<<<nkeep, 256, 0, st>>>(k, nkeep, lam_dev, w.dscr, w.zt);
        count_launch(ctx);
    }
    {
        ProfScope ps(ctx, RSDFT_K_BACKTRANSFORM, 8.0 * kd * kd * nkeep, 0.0, st, 0);
        const size_t bt_smem = (size_t)k * sizeof(double2);
        static std::mutex bt_mutex;
        static size_t bt_smem_max = 48 * 1024;
        if (bt_smem > bt_smem_max) {
            std::lock_guard<std::mutex> g(bt_mutex);
            if (bt_smem > bt_smem_max && bt_smem <= 200 * 1024 &&
                cudaFuncSetAttribute(k_backtransform_wy, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)bt_smem) == cudaSuccess)
                bt_smem_max = bt_smem;
            cudaGetLastError();
        }
        if (bt_smem > bt_smem_max)
            return fail(ctx, RSDFT_E_INVALID, "subspace %d too large for the back-transformation", k);
        k_wy_gram<<<dim3(cdiv(k - 1, WY_NB), WY_G), 256, 0, st>>>(k, w.Vh, k, w.Tw);
        k_wy_tfactor<<<cdiv(k - 1, WY_NB), 32, 0, st>>>(k, w.tau, w.Tw);
        count_launch(ctx, 2);
        k_backtransform_wy<<<nkeep, 256, bt_smem, st>>>(k, w.Vh, k, w.Tw, w.zt, z, ldz);
        count_launch(ctx);
    }
    RS_LAUNCHED(ctx, "tridiagonal eigensolve");
    if (coop_lock.owns_lock()) {
        // a barrier wait of the cooperative kernel that gave up leaves err set
        int *slot = reinterpret_cast<int *>(w.hbuf + w.hbuf_elems - 16);
        RS_CUDA(ctx, cudaMemcpyAsync(slot, &reinterpret_cast<GridSync *>(w.gsync)->err, sizeof(int),
                                     cudaMemcpyDeviceToHost, st));
        RS_CUDA(ctx, cudaStreamSynchronize(st));
        if (*slot != 0)
            return fail(ctx, RSDFT_E_TIMEOUT, "tridiagonalisation: a grid barrier wait timed out");
    }
    return RSDFT_OK;
}

// Cholesky of w.Lm (k x k) with dropping, the floor in w.dscr[4]: one
// cooperative launch, or one pair of launches per panel where the cooperative
// launch is refused.  Leaves the drop flags in w.drop and the kept columns in
// w.keep (keep[k] = their count).  After a cooperative launch *coop is set and
// `lock` holds the process-wide cooperative-launch mutex, which the caller
// releases once the stream has synchronised.  df: the diagonal blocks are
// factored in double-float (pivot floors >= 1e-6 only).
static rsdft_status cholesky(rsdft_ctx *ctx, int k, cudaStream_t st, std::unique_lock<std::mutex> &lock,
                             bool *coop, bool df) {
    Workspace &w = ctx->ws;
    *coop = false;
    static const int occ = [] {
        int dev = 0, cp = 0, o = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&cp, cudaDevAttrCooperativeLaunch, dev);
        int o2 = 0;
        if (cp == 0 || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_chol_coop<false>, 256, 0) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, k_chol_coop<true>, 256, 0) != cudaSuccess)
            o = 0;
        o = std::min(o, o2);
        cudaGetLastError();
        return o;
    }();
    if (occ > 0) {
        lock = std::unique_lock<std::mutex>(coop_mutex());
        const int rest = k - std::min(NBK, k);
        const int nt = cdiv(rest, CHOL_TS);
        // enough CTAs for one warp per panel row and one tile per CTA, at most one per SM
        const int want = std::max(cdiv(k, 8), nt * (nt + 1) / 2);
        const int nb = std::max(1, std::min(ctx->num_sms, want));
        GridSync *gs = reinterpret_cast<GridSync *>(w.gsync);
        RS_CUDA(ctx, cudaMemsetAsync(gs, 0, sizeof(GridSync), st));
        long long limit = 4000000000LL;   // ~2 s of SM clock per barrier wait
        double2 *a = w.Lm;
        int kk = k, ld = k;
        const double *fl = w.dscr + 4;
        int *dr = w.drop, *kp = w.keep;
        void *args[] = {&a, &kk, &ld, &fl, &dr, &kp, &gs, &limit};
        const void *fn = df ? (const void *)k_chol_coop<true> : (const void *)k_chol_coop<false>;
        const cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(nb), dim3(256), args, 0, st);
        if (e == cudaSuccess) {
            count_launch(ctx);
            *coop = true;
            RS_LAUNCHED(ctx, "cholesky");
            return RSDFT_OK;
        }
        cudaGetLastError();
        ++ctx->coop_fallbacks;
        ctx->coop_last_error = (int)e;
        lock.unlock();
    }
    for (int kb = 0; kb < k; kb += NBK) {
        const int nb = std::min(NBK, k - kb);
        // w.Km is free until the compaction: scratch for the factored block
        k_chol_panel<<<std::max(1, cdiv(k - kb - nb, 8)), 256, 0, st>>>(w.Lm, k, k, kb, nb, w.dscr + 4,
                                                                         w.drop, w.Km);
        count_launch(ctx);
        const int rest = k - kb - nb;
        dim3 g(std::max(1, cdiv(rest, CHOL_TS)), std::max(1, cdiv(rest, CHOL_TS)));
        k_chol_update<<<g, 256, 0, st>>>(w.Lm, k, k, kb, nb, w.Km);
        count_launch(ctx);
    }
    k_keep_scan<<<1, 1, 0, st>>>(w.drop, k, w.keep);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "cholesky");
    return RSDFT_OK;
}

__global__ void k_place_rows(const double2 *__restrict__ cc, int kc, int ncol,
                             const int *__restrict__ keep, double2 *__restrict__ out) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)kc * ncol) return;
    const int r = (int)(idx / ncol), c = (int)(idx % ncol);
    out[(size_t)keep[r] * ncol + c] = cc[idx];
}

rsdft_status rayleigh_ritz(rsdft_ctx *ctx, const double2 *gh, const double2 *gs, int k,
                           int nkeep, double pivot_tol, double *lam_dev, double2 *c_out,
                           int *ndropped, cudaStream_t st, bool df) {
    Workspace &w = ctx->ws;
    if (k > w.cap_k) return fail(ctx, RSDFT_E_INVALID, "subspace %d exceeds workspace %d", k, w.cap_k);
    if (nkeep > k || nkeep <= 0) return fail(ctx, RSDFT_E_INVALID, "bad nkeep");
    const size_t kk = (size_t)k * k;
    const double kd = (double)k;
    ProfScope ps(ctx, RSDFT_K_DENSE, kd * kd * kd * (4.0 / 3.0 + 8.0 + 16.0 / 3.0) +
                 kd * nkeep * (12.0 * kd + 176.0), 0.0, st, 0);
    RS_CUDA(ctx, cudaMemcpyAsync(w.Lm, gs, kk * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    k_maxdiag<<<1, 256, 0, st>>>(gs, k, k, pivot_tol, w.dscr + 4);
    count_launch(ctx);
    std::unique_lock<std::mutex> coop_lock;
    bool coop = false;
    {
        ProfScope pc(ctx, RSDFT_K_CHOL, 4.0 / 3.0 * kd * kd * kd, 0.0, st, 0);
        RS_TRY(cholesky(ctx, k, st, coop_lock, &coop, df && pivot_tol >= 1e-6));
    }
    int kc = 0;
    int *slot = reinterpret_cast<int *>(w.hbuf + w.hbuf_elems - 8);   // the front of hbuf holds LOBPCG residuals
    RS_CUDA(ctx, cudaMemcpyAsync(slot, w.keep + k, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (coop)
        RS_CUDA(ctx, cudaMemcpyAsync(slot + 1, &reinterpret_cast<GridSync *>(w.gsync)->err, sizeof(int),
                                     cudaMemcpyDeviceToHost, st));
    RS_CUDA(ctx, cudaStreamSynchronize(st));
    if (coop_lock.owns_lock()) coop_lock.unlock();
    if (coop && slot[1] != 0) return fail(ctx, RSDFT_E_TIMEOUT, "cholesky: a grid barrier wait timed out");
    kc = slot[0];
    if (ndropped) *ndropped = k - kc;
    if (kc < nkeep)
        return fail(ctx, RSDFT_E_NOT_SPD, "overlap has %d independent columns, %d wanted", kc, nkeep);
    const int T = 256;
    const long long kc2 = (long long)kc * kc;
    // compact L -> Km, G_H -> Ym
    k_gather_sq<<<cdiv(kc2, T), T, 0, st>>>(w.Lm, k, w.keep, kc, w.Km, kc);
    count_launch(ctx);
    k_gather_sq<<<cdiv(kc2, T), T, 0, st>>>(gh, k, w.keep, kc, w.Ym, kc);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "compaction");
    const double kcd = (double)kc;
    // the solves in double-float where the pivot floor keeps L well conditioned
    // (L^-1 amplifies the solve's relative error by at most ~1 / sqrt(floor))
    const bool trsm_in_df = df && pivot_tol >= 1e-6;
    float4 *Ldf = reinterpret_cast<float4 *>(w.Lm);   // free after the compaction
    {
        ProfScope pt(ctx, RSDFT_K_TRSM, 8.0 * kcd * kcd * kcd, 0.0, st, 0);
        if (trsm_in_df) RS_TRY(to_df(ctx, w.Km, kc, kc, Ldf, st));
        // first TRSM: Y = L^-1 G_H
        if (trsm_in_df) RS_TRY(trsm_df(ctx, false, Ldf, kc, w.Ym, kc, kc, st));
        else RS_TRY(trsm_lower(ctx, w.Km, kc, kc, w.Ym, kc, kc, st));
        // second TRSM: K = L^-1 Y^H
        k_conj_transpose<<<cdiv(kc2, T), T, 0, st>>>(w.Ym, kc, kc, w.Vh, kc);
        count_launch(ctx);
        if (trsm_in_df) RS_TRY(trsm_df(ctx, false, Ldf, kc, w.Vh, kc, kc, st));
        else RS_TRY(trsm_lower(ctx, w.Km, kc, kc, w.Vh, kc, kc, st));
    }
    k_hermitise<<<cdiv(kc2, T), T, 0, st>>>(w.Vh, kc, kc, w.Ym, kc);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "reduction");
    // eigenpairs of K (destroys Ym; the reflectors overwrite Vh)
    RS_TRY(eigh_lowest(ctx, w.Ym, kc, nkeep, lam_dev, w.Zc, nkeep, st, df));
    // C = L^-H Z
    {
        ProfScope pt(ctx, RSDFT_K_TRSM, 4.0 * kcd * kcd * nkeep, 0.0, st, 0);
        if (trsm_in_df) RS_TRY(trsm_df(ctx, true, Ldf, kc, w.Zc, nkeep, nkeep, st));
        else RS_TRY(trsm_upperH(ctx, w.Km, kc, kc, w.Zc, nkeep, nkeep, st));
    }
    RS_CUDA(ctx, cudaMemsetAsync(c_out, 0, (size_t)k * nkeep * sizeof(double2), st));
    k_place_rows<<<cdiv((long long)kc * nkeep, T), T, 0, st>>>(w.Zc, kc, nkeep, w.keep, c_out);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "back-substitution");
    return RSDFT_OK;
}

}  // namespace rsdft

using namespace rsdft;

extern "C" {

rsdft_status rsdft_rayleigh_ritz(rsdft_ctx *ctx, const void *gh_dev, const void *gs_dev, int k,
                                 int nkeep, double pivot_tol, double *lam_host, void *c_dev,
                                 int *ndropped_host, void *stream) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (k <= 0 || nkeep <= 0 || nkeep > k || !gh_dev || !gs_dev || !lam_host || !c_dev)
        return fail(ctx, RSDFT_E_INVALID, "bad rayleigh_ritz arguments");
    RS_TRY(ensure_workspace(ctx, cdiv(k, 3)));
    cudaStream_t st = as_stream(stream);
    int nd = 0;
    RS_TRY(rayleigh_ritz(ctx, (const double2 *)gh_dev, (const double2 *)gs_dev, k, nkeep, pivot_tol,
                         ctx->ws.lam, (double2 *)c_dev, &nd, st, ctx->dense_mode == RSDFT_DENSE_DF));
    RS_CUDA(ctx, cudaMemcpyAsync(lam_host, ctx->ws.lam, nkeep * sizeof(double), cudaMemcpyDeviceToHost, st));
    RS_CUDA(ctx, cudaStreamSynchronize(st));
    if (ndropped_host) *ndropped_host = nd;
    return RSDFT_OK;
}

rsdft_status rsdft_eigh(rsdft_ctx *ctx, const void *a_dev, int k, int nkeep, double *lam_host,
                        void *z_dev, void *stream) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (k <= 0 || nkeep <= 0 || nkeep > k || !a_dev || !lam_host || !z_dev)
        return fail(ctx, RSDFT_E_INVALID, "bad eigh arguments");
    RS_TRY(ensure_workspace(ctx, cdiv(k, 3)));
    cudaStream_t st = as_stream(stream);
    RS_CUDA(ctx, cudaMemcpyAsync(ctx->ws.Ym, a_dev, (size_t)k * k * sizeof(double2),
                                 cudaMemcpyDeviceToDevice, st));
    RS_TRY(eigh_lowest(ctx, ctx->ws.Ym, k, nkeep, ctx->ws.lam, (double2 *)z_dev, nkeep, st,
                       ctx->dense_mode == RSDFT_DENSE_DF));
    RS_CUDA(ctx, cudaMemcpyAsync(lam_host, ctx->ws.lam, nkeep * sizeof(double), cudaMemcpyDeviceToHost, st));
    RS_CUDA(ctx, cudaStreamSynchronize(st));
    return RSDFT_OK;
}

rsdft_status rsdft_set_dense(rsdft_ctx *ctx, int mode) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (mode != RSDFT_DENSE_AUTO && mode != RSDFT_DENSE_FP64 && mode != RSDFT_DENSE_DF)
        return fail(ctx, RSDFT_E_INVALID, "unknown dense mode %d", mode);
    ctx->dense_mode = mode;
    return RSDFT_OK;
}

}  // extern "C"
