// Householder tridiagonalisation of a Hermitian k x k matrix (k <= 448) by one
// thread-block cluster of 16 CTAs, the matrix resident in their shared memory
// and all arithmetic in double-float (dfloat.h).
//
// The reduction is the unblocked one of the cooperative FP64 kernel in dense.cu
// (LAPACK zhetd2 order, lower form), step i = 0 .. k-2 with L = k-1-i:
//   x = A[i+1:, i] -> reflector v_i (v_i[0] = 1), tau_i, beta_i = e_i; d_i = A[i][i]
//   y = A[i+1:, i+1:] v_i,  w = tau_i y,  w' = w - 1/2 tau_i (w^H v_i) v_i
//   A[i+1:, i+1:] -= v_i w'^H + w' v_i^H.
// On GB300 that kernel is bound by the latency of its per-step FP64 chains
// (a warp FP64 instruction takes 64 cycles of its sub-partition) and by a grid
// barrier per step.  Here:
//   - the matrix lives in distributed shared memory: row r in CTA r mod 16,
//     full rows of complex double-floats (16 B), so k <= 448 fits in 227 KB;
//   - A is Hermitian, so column i below the diagonal is the conjugate of row i,
//     which one CTA (the owner of row i) holds whole: it brings row i up to date
//     and forms the reflector's scalars (norm, beta, tau, the scale of v) alone,
//     while the other CTAs apply the previous step's rank-2 update to their rows
//     (the update of step i-1 is applied lazily at step i);
//   - two cluster barriers per step: after the scalars and the updates (every
//     CTA then reads row i from the owner's shared memory and forms v_i itself),
//     and after the matrix-vector products, whose results y_r and per-warp
//     partial sums of y^H v each CTA has stored into every CTA's shared memory
//     (every CTA then forms w' redundantly from local data);
//   - the FP64 outputs are written off the owner's path: vh row i by one warp of
//     each CTA, d_i, e_i, tau_i by the next CTA;
//   - double-float keeps about 48 significant bits, so the reduction's backward
//     error is a small multiple of 2^-46 |A| instead of 2^-53 |A|.
// Outputs as the FP64 kernel: d, e (real), tau, and v_i in vh row i (columns
// i+1 .. k-1), for the compact-WY back-transformation.
#include <cooperative_groups.h>

#include <algorithm>

#include "dfloat.h"
#include "rsdft_internal.h"

namespace rsdft {

namespace cg = cooperative_groups;
using namespace dfl;

constexpr int TC_C = 16;     // CTAs in the cluster
constexpr int TC_T = 512;    // threads per CTA
constexpr int TC_W = TC_T / 32;
constexpr int TC_KMAX = 448;   // largest k whose rows fit the cluster's shared memory

__device__ __forceinline__ cdf ld4(const float4 &v) { return cdf{df{v.x, v.y}, df{v.z, v.w}}; }
__device__ __forceinline__ float4 st4(const cdf &c) { return make_float4(c.re.h, c.re.l, c.im.h, c.im.l); }

__device__ __forceinline__ void cl_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// s + sum of one product's exact pieces: the running sum keeps its hi part by
// TwoSum and collects every rounding error in lo (one renormalisation at the end)
struct Acc {
    float h, l;
};
__device__ __forceinline__ void acc_prod(Acc &s, float ah, float al, float bh, float bl) {
    const df p = two_prod(ah, bh);
    const df t = two_sum(s.h, p.h);
    s.h = t.h;
    s.l = fadd(s.l, fadd(t.l, ffma(ah, bl, ffma(al, bh, p.l))));
}
__device__ __forceinline__ void acc_df(Acc &s, df x) {
    const df t = two_sum(s.h, x.h);
    s.h = t.h;
    s.l = fadd(s.l, fadd(t.l, x.l));
}
__device__ __forceinline__ df acc_get(const Acc &s) { return fast_two_sum(s.h, s.l); }

// a - v_r conj(w_c) - w_r conj(v_c), all complex double-float
__device__ __forceinline__ cdf rank2(const cdf &a, const cdf &vr, const cdf &wr, const cdf &vc, const cdf &wc) {
    // re: a.re - (vr.re wc.re + vr.im wc.im + wr.re vc.re + wr.im vc.im)
    Acc re{a.re.h, a.re.l}, im{a.im.h, a.im.l};
    acc_prod(re, -vr.re.h, -vr.re.l, wc.re.h, wc.re.l);
    acc_prod(re, -vr.im.h, -vr.im.l, wc.im.h, wc.im.l);
    acc_prod(re, -wr.re.h, -wr.re.l, vc.re.h, vc.re.l);
    acc_prod(re, -wr.im.h, -wr.im.l, vc.im.h, vc.im.l);
    // im: a.im - (vr.im wc.re - vr.re wc.im + wr.im vc.re - wr.re vc.im)
    acc_prod(im, -vr.im.h, -vr.im.l, wc.re.h, wc.re.l);
    acc_prod(im, vr.re.h, vr.re.l, wc.im.h, wc.im.l);
    acc_prod(im, -wr.im.h, -wr.im.l, vc.re.h, vc.re.l);
    acc_prod(im, wr.re.h, wr.re.l, vc.im.h, vc.im.l);
    return cdf{acc_get(re), acc_get(im)};
}

__device__ __forceinline__ df shfl_df(df x, int o) {
    return df{__shfl_xor_sync(0xffffffffu, x.h, o), __shfl_xor_sync(0xffffffffu, x.l, o)};
}

// Block-wide sum of a complex double-float; every thread gets the result.
__device__ cdf block_sum_cdf(cdf v, float4 *scratch) {
    for (int o = 16; o > 0; o >>= 1) {
        v.re = add(v.re, shfl_df(v.re, o));
        v.im = add(v.im, shfl_df(v.im, o));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) scratch[warp] = st4(v);
    __syncthreads();
    if (warp == 0) {
        cdf s = lane < TC_W ? ld4(scratch[lane]) : cdf{df{0.f, 0.f}, df{0.f, 0.f}};
        for (int o = 16; o > 0; o >>= 1) {
            s.re = add(s.re, shfl_df(s.re, o));
            s.im = add(s.im, shfl_df(s.im, o));
        }
        if (lane == 0) scratch[TC_W] = st4(s);
    }
    __syncthreads();
    return ld4(scratch[TC_W]);
}

__global__ void __launch_bounds__(TC_T, 1)
k_tridiag_cluster(const double2 *__restrict__ a, int k, int ld, double2 *__restrict__ vh, int ldv,
                  double2 *__restrict__ tau, double *__restrict__ d, double *__restrict__ e) {
    cg::cluster_group cl = cg::this_cluster();
    const int me = (int)cl.block_rank();
    const int R = (k + TC_C - 1) / TC_C;   // row slots per CTA
    extern __shared__ float4 sm[];
    float4 *A = sm;                        // [R][k]: row me + 16 lr in slot lr
    float4 *Vb0 = A + (size_t)R * k;       // v of even steps, [k]
    float4 *Vb1 = Vb0 + k;                 // v of odd steps
    float4 *YW = Vb1 + k;                  // [k]: y of all rows (pushed by their owners), then w'
    __shared__ float4 scratch[TC_W + 1];
    __shared__ float4 bc[4];               // scalars broadcast inside the CTA
    __shared__ float4 pub[3];              // owner of the step: tau, scal, (beta, d_i)
    __shared__ float4 loc[3];              // every CTA: its copy of the owner's pub
    __shared__ float4 Sall[TC_C * TC_W];   // every warp's part of y^H v (pushed)
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const cdf zero{df{0.f, 0.f}, df{0.f, 0.f}};
    const cdf one{df{1.f, 0.f}, df{0.f, 0.f}};

    for (int idx = tid; idx < R * k; idx += TC_T) {
        const int lr = idx / k, c = idx - lr * k;
        const int r = me + TC_C * lr;
        cdf v = zero;
        if (r < k) {
            const double2 x = a[(size_t)r * ld + c];
            v = cdf{from_double(x.x), from_double(x.y)};
        }
        A[idx] = st4(v);
    }
    __syncthreads();
    cl_barrier();

    for (int i = 0; i < k - 1; ++i) {
        const int L = k - 1 - i;
        float4 *Vp = (i & 1) ? Vb0 : Vb1;   // v_{i-1}: rows/columns i .. k-1 at [c - i]
        float4 *Vc = (i & 1) ? Vb1 : Vb0;   // v_i: rows/columns i+1 .. k-1 at [c - i - 1]
        const int owner = i % TC_C;
        // first own row slot with a row > i
        const int lr_first = (i + 1 - me + TC_C - 1) / TC_C > 0 ? (i + 1 - me + TC_C - 1) / TC_C : 0;
        const int nrow = max(0, R - lr_first - ((me + TC_C * (R - 1) >= k) ? 1 : 0));
        if (me == owner) {
            // ---- phase 1: row i up to date, then its reflector
            const int li = i / TC_C;
            float4 *row = A + (size_t)li * k;
            if (i > 0) {
                const cdf vr = ld4(Vp[0]), wr = ld4(YW[0]);
                for (int c = i + tid; c < k; c += TC_T)
                    row[c] = st4(rank2(ld4(row[c]), vr, wr, ld4(Vp[c - i]), ld4(YW[c - i])));
                __syncthreads();
            }
            // x_q = conj(A[i][i+1+q]); alpha = x_0
            df nrm{0.f, 0.f};
            for (int q = 1 + tid; q < L; q += TC_T) nrm = add(nrm, cabs2(ld4(row[i + 1 + q])));
            const cdf ns = block_sum_cdf(cdf{nrm, df{0.f, 0.f}}, scratch);
            if (tid == 0) {
                const cdf x0 = cconj(ld4(row[i + 1]));
                const df xnorm2 = ns.re;
                cdf t = zero, scal = zero;
                df beta;
                // a column below 1e-18 (squares near FP32's underflow) is taken as
                // reduced already: H = I, beta = Re alpha (an absolute change below
                // 1e-18, far under the rounding of an Ha-scale matrix)
                const df nb2 = add(cabs2(x0), xnorm2);
                if ((xnorm2.h == 0.f && x0.im.h == 0.f) || !(nb2.h > 1e-36f)) {
                    beta = x0.re;
                } else {
                    // beta = -sign(Re alpha) |(alpha, x)|, tau = (beta - alpha) / beta,
                    // scal = 1 / (alpha - beta) = conj(alpha - beta) / |alpha - beta|^2
                    const df nb = sqrt(nb2);
                    beta = x0.re.h >= 0.f ? neg(nb) : nb;
                    const df rb = div(mk(1.0f), beta);
                    t = cdf{mul(sub(beta, x0.re), rb), neg(mul(x0.im, rb))};
                    const cdf den{sub(x0.re, beta), x0.im};
                    const df rd = div(mk(1.0f), cabs2(den));
                    scal = cdf{mul(den.re, rd), neg(mul(den.im, rd))};
                }
                // published for every CTA (which form v_i from row i themselves)
                const df di = ld4(row[i]).re;
                pub[0] = st4(t);
                pub[1] = st4(scal);
                pub[2] = make_float4(beta.h, beta.l, di.h, di.l);
            }
        }
        // ---- phase 2: step i-1's update of this CTA's rows > i (columns > i)
        if (i > 0 && nrow > 0) {
            const int total = nrow * L;
            const int dj = TC_T / L, dc = TC_T - dj * L;
            int j = tid / L, c = tid - j * L;
            for (int t = tid; t < total; t += TC_T) {
                const int r = me + TC_C * (lr_first + j);
                float4 *p = A + (size_t)(lr_first + j) * k + (i + 1 + c);
                *p = st4(rank2(ld4(*p), ld4(Vp[r - i]), ld4(YW[r - i]), ld4(Vp[i + 1 + c - i]),
                               ld4(YW[i + 1 + c - i])));
                j += dj;
                c += dc;
                if (c >= L) {
                    c -= L;
                    ++j;
                }
            }
        }
        cl_barrier();
        // ---- phase 3: v_i from the owner's row i and scalars, y = A v_i for own rows > i
        {
            const float4 *prow = cl.map_shared_rank(A, owner) + (size_t)(i / TC_C) * k + (i + 1);
            const float4 x = tid < L ? prow[tid] : make_float4(0.f, 0.f, 0.f, 0.f);   // L < TC_T
            if (tid < 3) loc[tid] = cl.map_shared_rank(pub, owner)[tid];
            __syncthreads();
            const cdf scal = ld4(loc[1]);
            if (tid < L) {
                const cdf vq = tid == 0 ? one : cmul(cconj(ld4(x)), scal);
                Vc[tid] = st4(vq);
                // the FP64 copy for the back-transformation: one warp's range per CTA
                if (warp == me) vh[(size_t)i * ldv + i + 1 + tid] = make_double2(to_double(vq.re), to_double(vq.im));
            }
            if (me == (owner + 1) % TC_C && tid == 0) {
                const float4 bd = loc[2], tq = loc[0];
                d[i] = to_double(df{bd.z, bd.w});
                e[i] = to_double(df{bd.x, bd.y});
                tau[i] = make_double2(to_double(df{tq.x, tq.y}), to_double(df{tq.z, tq.w}));
            }
        }
        __syncthreads();
        cdf sp = zero;   // sum over own rows of conj(y_r) v_r
        for (int j = warp; j < nrow; j += TC_W) {
            const int lr = lr_first + j;
            const int r = me + TC_C * lr;
            const float4 *row = A + (size_t)lr * k + (i + 1);
            Acc yr{0.f, 0.f}, yi{0.f, 0.f};
            for (int q = lane; q < L; q += 32) {
                const cdf x = ld4(row[q]), v = ld4(Vc[q]);
                acc_prod(yr, x.re.h, x.re.l, v.re.h, v.re.l);
                acc_prod(yr, -x.im.h, -x.im.l, v.im.h, v.im.l);
                acc_prod(yi, x.re.h, x.re.l, v.im.h, v.im.l);
                acc_prod(yi, x.im.h, x.im.l, v.re.h, v.re.l);
            }
            cdf y{acc_get(yr), acc_get(yi)};
            for (int o = 16; o > 0; o >>= 1) {
                y.re = add(y.re, shfl_df(y.re, o));
                y.im = add(y.im, shfl_df(y.im, o));
            }
            // y_r into every CTA's YW (one remote store per lane; the stores need no
            // reply, and the cluster barrier below makes them visible)
            if (lane < TC_C) cl.map_shared_rank(YW, lane)[r - i - 1] = st4(y);
            if (lane == 0) sp = cadd(sp, cmulc(y, ld4(Vc[r - i - 1])));
        }
        {   // this warp's part of y^H v into every CTA
            const float4 sp4 = st4(sp);
            const float4 b{__shfl_sync(0xffffffffu, sp4.x, 0), __shfl_sync(0xffffffffu, sp4.y, 0),
                           __shfl_sync(0xffffffffu, sp4.z, 0), __shfl_sync(0xffffffffu, sp4.w, 0)};
            if (lane < TC_C) cl.map_shared_rank(Sall, lane)[me * TC_W + warp] = b;
        }
        cl_barrier();
        // ---- phase 4: y^H v, then w' = tau y - 1/2 |tau|^2 (y^H v) v
        if (warp == 0) {
            // y^H v: the TC_C x TC_W per-warp parts, TC_C * TC_W / 32 per lane
            float4 part[TC_C * TC_W / 32];
#pragma unroll
            for (int u = 0; u < TC_C * TC_W / 32; ++u) part[u] = Sall[lane + 32 * u];
            cdf s = zero;
#pragma unroll
            for (int u = 0; u < TC_C * TC_W / 32; ++u) s = cadd(s, ld4(part[u]));
            for (int o = 16; o > 0; o >>= 1) {
                s.re = add(s.re, shfl_df(s.re, o));
                s.im = add(s.im, shfl_df(s.im, o));
            }
            if (lane == 0) {
                const cdf t = ld4(loc[0]);
                const df h = mul_f(cabs2(t), -0.5f);
                bc[3] = st4(cdf{mul(h, s.re), mul(h, s.im)});
            }
        }
        __syncthreads();
        {
            const cdf t = ld4(loc[0]), al = ld4(bc[3]);
            for (int q = tid; q < L; q += TC_T) YW[q] = st4(cadd(cmul(t, ld4(YW[q])), cmul(al, ld4(Vc[q]))));
        }
        __syncthreads();
    }
    // d[k-1]: row k-1 after the last update, v_{k-2} = (1)
    if (me == (k - 1) % TC_C && tid == 0) {
        const cdf x = ld4(A[(size_t)((k - 1) / TC_C) * k + (k - 1)]);
        const cdf w = ld4(YW[0]);
        d[k - 1] = to_double(sub(x.re, mul_f(w.re, 2.0f)));
    }
    cl_barrier();   // no CTA leaves while another may still read its shared memory
}

// Each reflector made unitary in FP64.  H = I - tau v v^H is unitary exactly when
// 2 Re(tau) = |tau|^2 |v|^2; the double-float reduction leaves that true to about
// 2^-46, and the back-transformed eigenvectors would be orthonormal only to
// ~k 2^-46.  Re(tau) is reset to the root of nu a^2 - 2 a + nu b^2 = 0 (b = Im tau,
// nu = |v|^2 summed in FP64) nearest its value: a change of ~2^-46 relative, within
// the reduction's own backward error.  One warp per reflector.
__global__ void __launch_bounds__(256)
k_unitarize(int k, const double2 *__restrict__ vh, int ldv, double2 *__restrict__ tau) {
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= k - 1) return;
    const double2 *v = vh + (size_t)i * ldv;
    double s = 0.0;
    for (int c = i + 1 + lane; c < k; c += 32) s = fma(v[c].x, v[c].x, fma(v[c].y, v[c].y, s));
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane != 0 || !(s > 0.0)) return;
    const double2 t = tau[i];
    const double disc = 1.0 - s * s * t.y * t.y;
    if (!(disc >= 0.0)) return;
    const double r = ::sqrt(disc);
    const double a_lo = s * t.y * t.y / (1.0 + r);   // (1 - r) / nu without cancellation
    const double a_hi = (1.0 + r) / s;
    tau[i].x = fabs(t.x - a_lo) <= fabs(t.x - a_hi) ? a_lo : a_hi;
}

size_t tridiag_cluster_smem(int k) {
    const size_t R = (size_t)(k + TC_C - 1) / TC_C;
    return (R * k + 3 * (size_t)k) * sizeof(float4);
}

bool tridiag_cluster_fits(int k) { return k >= 2 && k <= TC_KMAX; }

rsdft_status tridiag_cluster(rsdft_ctx *ctx, const double2 *a, int k, int ld, double2 *vh, int ldv, double2 *tau,
                             double *d, double *e, cudaStream_t st, bool *done) {
    *done = false;
    if (!tridiag_cluster_fits(k)) return RSDFT_OK;
    const size_t smem = tridiag_cluster_smem(k);
    // the attributes once per process (largest size), then a residency check
    static const bool ok = [] {
        bool good = cudaFuncSetAttribute(k_tridiag_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                        cudaSuccess &&
                    cudaFuncSetAttribute(k_tridiag_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tridiag_cluster_smem(TC_KMAX)) == cudaSuccess;
        if (good) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = TC_C;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(TC_C);
            cfg.blockDim = dim3(TC_T);
            cfg.dynamicSmemBytes = tridiag_cluster_smem(TC_KMAX);
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int ncl = 0;
            good = cudaOccupancyMaxActiveClusters(&ncl, k_tridiag_cluster, &cfg) == cudaSuccess && ncl >= 1;
        }
        cudaGetLastError();
        return good;
    }();
    if (!ok) return RSDFT_OK;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = TC_C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(TC_C);
    cfg.blockDim = dim3(TC_T);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const cudaError_t err = cudaLaunchKernelEx(&cfg, k_tridiag_cluster, a, k, ld, vh, ldv, tau, d, e);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return RSDFT_OK;   // the caller falls back to the cooperative FP64 kernel
    }
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_tridiag_cluster");
    k_unitarize<<<cdiv(k - 1, 8), 256, 0, st>>>(k, vh, ldv, tau);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_unitarize");
    *done = true;
    return RSDFT_OK;
}

}  // namespace rsdft
