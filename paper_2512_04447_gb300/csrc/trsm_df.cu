// The triangular solves of Eq. 1 in double-float (dfloat.h), for subspace solves
// whose Cholesky pivots are floored at >= 1e-6 of the largest (the mixed form's
// FP32 phase and refinement use 1e-3): the layout and order of k_trsm_cols in
// dense.cu (one warp per right-hand-side column, lane r holding row r of the
// current block row, 32 x 32 tiles of L staged in shared memory and shared by the
// CTA's four columns), with each complex multiply-add as four double-float
// products on the FP32 pipe instead of four FP64 FMAs.  A warp FP64 instruction
// occupies its GB300 sub-partition for 64 cycles, and this solve has one warp per
// column, so the FP64 kernel is bound by that issue rate.
// Accuracy: backward error ~ kc 2^-48 |L| per solve; with L_jj^2 >= 1e-6 max
// diag(G_S) the condition of L stays below ~1e3 and the solution keeps ~1e-11
// relative accuracy at worst, far below the FP32 Gram matrices' own error.
#include "dfloat.h"
#include "rsdft_internal.h"

namespace rsdft {

using namespace dfl;

namespace {

__device__ __forceinline__ cdf ld4t(const float4 &v) { return cdf{df{v.x, v.y}, df{v.z, v.w}}; }
__device__ __forceinline__ float4 st4t(const cdf &c) { return make_float4(c.re.h, c.re.l, c.im.h, c.im.l); }

struct AccT {
    float h, l;
};
__device__ __forceinline__ void acc_mad(AccT &s, float ah, float al, float bh, float bl) {
    const df p = two_prod(ah, bh);
    const df t = two_sum(s.h, p.h);
    s.h = t.h;
    s.l = fadd(s.l, fadd(t.l, ffma(ah, bl, ffma(al, bh, p.l))));
}
// v -= a x (complex)
__device__ __forceinline__ void cfms_df(AccT &vr, AccT &vi, const cdf &a, const cdf &x) {
    acc_mad(vr, -a.re.h, -a.re.l, x.re.h, x.re.l);
    acc_mad(vr, a.im.h, a.im.l, x.im.h, x.im.l);
    acc_mad(vi, -a.re.h, -a.re.l, x.im.h, x.im.l);
    acc_mad(vi, -a.im.h, -a.im.l, x.re.h, x.re.l);
}
__device__ __forceinline__ cdf acc_val(const AccT &r, const AccT &i) {
    return cdf{fast_two_sum(r.h, r.l), fast_two_sum(i.h, i.l)};
}

}  // namespace

// L (FP64, kc x kc, ld ldl) -> double-float rows (ld kc)
__global__ void k_to_df(const double2 *__restrict__ L, int ldl, int kc, float4 *__restrict__ out) {
    const long long n = (long long)kc * kc;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / kc), c = (int)(i - (long long)r * kc);
        const double2 v = L[(size_t)r * ldl + c];
        out[i] = st4t(cdf{from_double(v.x), from_double(v.y)});
    }
}

template <bool BACK>
__device__ __forceinline__ float4 tile_elem_df(const float4 *__restrict__ L, int kc, int r0, int nr, int c0, int nc,
                                               int t) {
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!BACK) {   // L[r0+r][c0+j]
        const int r = t >> 5, j = t & 31;
        return (r < nr && j < nc) ? L[(size_t)(r0 + r) * kc + c0 + j] : z;
    }
    // (L^H)[r0+r][c0+j] = conj(L[c0+j][r0+r])
    const int j = t >> 5, r = t & 31;
    if (!(r < nr && j < nc)) return z;
    const float4 v = L[(size_t)(c0 + j) * kc + r0 + r];
    return make_float4(v.x, v.y, -v.z, -v.w);
}

template <bool BACK>
__global__ void __launch_bounds__(128)
k_trsm_cols_df(const float4 *__restrict__ L, int kc, double2 *b, int ldb, int ncol) {
    __shared__ float4 Ts[32][33];
    __shared__ float4 Xs[4][32];   // per warp: the solved rows of the current tile
    __shared__ float2 Linv[32];
    constexpr int PER = 32 * 32 / 128;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int col = blockIdx.x * 4 + warp;
    const bool act = col < ncol;
    const int nblk = (kc + 31) / 32;
    const cdf zero{df{0.f, 0.f}, df{0.f, 0.f}};
    for (int s = 0; s < nblk; ++s) {
        const int rb = BACK ? nblk - 1 - s : s;
        const int r0 = rb * 32, nr = min(32, kc - r0);
        cdf a0 = zero;
        if (act && lane < nr) {
            const double2 v = b[(size_t)(r0 + lane) * ldb + col];
            a0 = cdf{from_double(v.x), from_double(v.y)};
        }
        // two accumulator pairs (even and odd j) halve the dependent TwoSum chains
        AccT ar{a0.re.h, a0.re.l}, ai{a0.im.h, a0.im.l}, br{0.f, 0.f}, bi{0.f, 0.f};
        const int j_lo = BACK ? rb + 1 : 0, j_hi = BACK ? nblk : rb;
        float4 pre[PER];
        if (j_lo < j_hi) {
            const int c0 = j_lo * 32, nc = min(32, kc - c0);
#pragma unroll
            for (int q = 0; q < PER; ++q) pre[q] = tile_elem_df<BACK>(L, kc, r0, nr, c0, nc, threadIdx.x + q * 128);
        }
        for (int jb = j_lo; jb < j_hi; ++jb) {
            const int c0 = jb * 32, nc = min(32, kc - c0);
            __syncthreads();
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
                    pre[q] = tile_elem_df<BACK>(L, kc, r0, nr, c1, nc1, threadIdx.x + q * 128);
            }
            // solved rows c0.. of this column, as double-float, through shared memory
            cdf xj = zero;
            if (act && lane < nc) {
                const double2 v = b[(size_t)(c0 + lane) * ldb + col];
                xj = cdf{from_double(v.x), from_double(v.y)};
            }
            __syncwarp();
            Xs[warp][lane] = st4t(xj);
            __syncwarp();
#pragma unroll 4
            for (int j = 0; j < 32; j += 2) {
                cfms_df(ar, ai, ld4t(Ts[lane][j]), ld4t(Xs[warp][j]));
                cfms_df(br, bi, ld4t(Ts[lane][j + 1]), ld4t(Xs[warp][j + 1]));
            }
        }
        {
            const df er = fast_two_sum(br.h, br.l), ei = fast_two_sum(bi.h, bi.l);
            const df t1 = two_sum(ar.h, er.h), t2 = two_sum(ai.h, ei.h);
            ar = AccT{t1.h, fadd(ar.l, fadd(t1.l, er.l))};
            ai = AccT{t2.h, fadd(ai.l, fadd(t2.l, ei.l))};
        }
        __syncthreads();
        for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
            const int r = t >> 5, j = t & 31;
            Ts[r][j] = (r < nr && j < nr) ? L[(size_t)(r0 + r) * kc + r0 + j] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (threadIdx.x < nr) {
            const float4 dgl = L[(size_t)(r0 + threadIdx.x) * kc + r0 + threadIdx.x];
            const df inv = div(mk(1.0f), df{dgl.x, dgl.y});   // real positive diagonal
            Linv[threadIdx.x] = make_float2(inv.h, inv.l);
        }
        __syncthreads();
        cdf v = acc_val(ar, ai);
        if (!BACK) {
            for (int c = 0; c < nr; ++c) {
                const df inv{Linv[c].x, Linv[c].y};
                const cdf xc{mul(v.re, inv), mul(v.im, inv)};
                cdf x;
                x.re.h = __shfl_sync(0xffffffffu, xc.re.h, c);
                x.re.l = __shfl_sync(0xffffffffu, xc.re.l, c);
                x.im.h = __shfl_sync(0xffffffffu, xc.im.h, c);
                x.im.l = __shfl_sync(0xffffffffu, xc.im.l, c);
                if (lane == c) {
                    v = x;
                } else if (lane > c && lane < nr) {
                    AccT r{v.re.h, v.re.l}, i{v.im.h, v.im.l};
                    cfms_df(r, i, ld4t(Ts[lane][c]), x);
                    v = acc_val(r, i);
                }
            }
        } else {   // (L^H)[r][c] = conj(L[c][r])
            for (int c = nr - 1; c >= 0; --c) {
                const df inv{Linv[c].x, Linv[c].y};
                const cdf xc{mul(v.re, inv), mul(v.im, inv)};
                cdf x;
                x.re.h = __shfl_sync(0xffffffffu, xc.re.h, c);
                x.re.l = __shfl_sync(0xffffffffu, xc.re.l, c);
                x.im.h = __shfl_sync(0xffffffffu, xc.im.h, c);
                x.im.l = __shfl_sync(0xffffffffu, xc.im.l, c);
                if (lane == c) {
                    v = x;
                } else if (lane < c) {
                    AccT r{v.re.h, v.re.l}, i{v.im.h, v.im.l};
                    cfms_df(r, i, cconj(ld4t(Ts[c][lane])), x);
                    v = acc_val(r, i);
                }
            }
        }
        if (act && lane < nr) b[(size_t)(r0 + lane) * ldb + col] = make_double2(to_double(v.re), to_double(v.im));
    }
}

rsdft_status to_df(rsdft_ctx *ctx, const double2 *L, int ldl, int kc, float4 *out, cudaStream_t st) {
    if (kc <= 0) return RSDFT_OK;
    k_to_df<<<std::min(cdiv((long long)kc * kc, 256), 2048), 256, 0, st>>>(L, ldl, kc, out);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_to_df");
    return RSDFT_OK;
}

rsdft_status trsm_df(rsdft_ctx *ctx, bool back, const float4 *L, int kc, double2 *b, int ldb, int ncol,
                     cudaStream_t st) {
    if (kc <= 0 || ncol <= 0) return RSDFT_OK;
    if (back) k_trsm_cols_df<true><<<cdiv(ncol, 4), 128, 0, st>>>(L, kc, b, ldb, ncol);
    else k_trsm_cols_df<false><<<cdiv(ncol, 4), 128, 0, st>>>(L, kc, b, ldb, ncol);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_trsm_cols_df");
    return RSDFT_OK;
}

}  // namespace rsdft
