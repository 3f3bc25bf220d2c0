// FP64-accurate Gram matrices and rotations on the FP32 pipe ("double-float"),
// for the refinement of the mixed form.  GB300 issues FP32 at 64 times its
// FP64 rate (128 against 2 lanes per clock and SM), so a product carried as a
// pair of FP32 values beats the FP64 pipe even at a dozen FP32 operations per
// real product:
//   - an FP64 value x is held as hi = fl32(x), lo = fl32(x - hi) (48 bits);
//   - a product a b = ah bh + (ah bl + al bh) (+ al bl, below 2^-48, dropped),
//     with ah bh split exactly into p + e (TwoProduct: p = fl(ah bh),
//     e = fma(ah, bh, -p)) and the cross terms in FP32;
//   - sums in (s_hi, s_lo) pairs: s_hi takes p by TwoSum (Knuth), its rounding
//     error, e and the cross terms go to s_lo;
//   - per-tile pair sums go out as FP64 (hi + lo) and split-K partials are summed
//     in FP64, as in gemm.cu.
// The relative error per product is about 2^-46, against 2^-53 in FP64: well
// below the refinement's 1e-8 floor.  All operations use the _rn intrinsics so
// that the compiler cannot fuse the error-free steps.
#include <algorithm>
#include <string>

#include "rsdft_internal.h"

namespace rsdft {

constexpr int DF_T = 64;       // output tile edge of the Gram (16 x 16 threads, 4 x 4 each)
constexpr int DF_K = 16;       // reduction chunk per shared-memory stage
constexpr int DF_THREADS = 256;

__device__ __forceinline__ const float2 *row_of_df(const RowBlocksT<float2> &rb, int i, long long n) {
    if (i < rb.cnt[0]) return rb.ptr[0] + (size_t)i * n;
    i -= rb.cnt[0];
    if (i < rb.cnt[1]) return rb.ptr[1] + (size_t)i * n;
    i -= rb.cnt[1];
    return rb.ptr[2] + (size_t)i * n;
}

__device__ __forceinline__ void df_mac(float &sh, float &sl, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    const float e = __fmaf_rn(ah, bh, -p);                       // ah bh = p + e exactly
    const float cr = __fmaf_rn(ah, bl, __fmul_rn(al, bh));       // cross terms
    const float s = __fadd_rn(sh, p);
    const float bb = __fsub_rn(s, sh);
    const float te = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));   // TwoSum error
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(te, __fadd_rn(e, cr)));
}

// hi/lo FP32 split of FP64 rows: h = fl32(x), l = fl32(x - h)
__global__ void k_split_df(const double2 *__restrict__ x, long long cnt, float2 *__restrict__ h,
                           float2 *__restrict__ l) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (long long)gridDim.x * blockDim.x) {
        const double2 v = x[i];
        const float hx = (float)v.x, hy = (float)v.y;
        h[i] = make_float2(hx, hy);
        l[i] = make_float2((float)(v.x - (double)hx), (float)(v.y - (double)hy));
    }
}

// Partial Gram tiles over one K-chunk: G[i][j] = sum_r conj(A_i(r)) B_j(r), A as
// (ah, al) rows, B as (bh, bl) rows (bl may be null: B exact in FP32).
__global__ void __launch_bounds__(DF_THREADS)
k_gram_df(const float2 *__restrict__ ah, const float2 *__restrict__ al, RowBlocksT<float2> bh,
          RowBlocksT<float2> bl, int na, int nb, long long n, int Tj, long long kchunk,
          double2 *__restrict__ part) {
    __shared__ float2 Ah[DF_K][DF_T + 1], Al[DF_K][DF_T + 1], Bh[DF_K][DF_T + 1], Bl[DF_K][DF_T + 1];
    const int ti = blockIdx.x / Tj, tj = blockIdx.x % Tj;
    const int split = blockIdx.y;
    const long long k0 = (long long)split * kchunk, k1 = min(n, k0 + kchunk);
    const int i0 = ti * DF_T, j0 = tj * DF_T;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const bool blo = bl.ptr[0] != nullptr || bl.ptr[1] != nullptr || bl.ptr[2] != nullptr;
    float rh[4][4], rl[4][4], ih[4][4], il[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) rh[a][b] = rl[a][b] = ih[a][b] = il[a][b] = 0.0f;
    for (long long kb = k0; kb < k1; kb += DF_K) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int idx = threadIdx.x + q * DF_THREADS;
            const int lrow = idx >> 4, lk = idx & 15;
            const long long kk = kb + lk;
            float2 xa = make_float2(0.f, 0.f), xal = xa, xb = xa, xbl = xa;
            if (kk < k1) {
                if (i0 + lrow < na) {
                    xa = ah[(size_t)(i0 + lrow) * n + kk];
                    xal = al[(size_t)(i0 + lrow) * n + kk];
                }
                if (j0 + lrow < nb) {
                    xb = row_of_df(bh, j0 + lrow, n)[kk];
                    if (blo) xbl = row_of_df(bl, j0 + lrow, n)[kk];
                }
            }
            Ah[lk][lrow] = xa;
            Al[lk][lrow] = xal;
            Bh[lk][lrow] = xb;
            Bl[lk][lrow] = xbl;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < DF_K; ++k) {
            float2 a[4], a2[4], b[4], b2[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = Ah[k][ty + 16 * q];
                a2[q] = Al[k][ty + 16 * q];
                b[q] = Bh[k][tx + 16 * q];
                b2[q] = Bl[k][tx + 16 * q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    // conj(a) b: re = ax bx + ay by, im = ax by - ay bx
                    df_mac(rh[p][q], rl[p][q], a[p].x, a2[p].x, b[q].x, b2[q].x);
                    df_mac(rh[p][q], rl[p][q], a[p].y, a2[p].y, b[q].y, b2[q].y);
                    df_mac(ih[p][q], il[p][q], a[p].x, a2[p].x, b[q].y, b2[q].y);
                    df_mac(ih[p][q], il[p][q], -a[p].y, -a2[p].y, b[q].x, b2[q].x);
                }
        }
        __syncthreads();
    }
    double2 *pp = part + (size_t)split * na * nb;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int i = i0 + ty + 16 * p;
        if (i >= na) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = j0 + tx + 16 * q;
            if (j < nb)
                pp[(size_t)i * nb + j] = make_double2((double)rh[p][q] + (double)rl[p][q],
                                                      (double)ih[p][q] + (double)il[p][q]);
        }
    }
}

// out[b][r] = sum_i c[i][b] Y_i(r), Y as (yh, yl) rows [k][n], c FP64 [k][ldc]
// (split to pairs on staging), out FP64; tile 64 bands x 64 points.
__global__ void __launch_bounds__(DF_THREADS)
k_rotate_df(const float2 *__restrict__ yh, const float2 *__restrict__ yl, int k, const double2 *__restrict__ c,
            int ldc, int m, long long n, double2 *__restrict__ out) {
    __shared__ float2 Ch[DF_K][DF_T + 1], Cl[DF_K][DF_T + 1], Yh[DF_K][DF_T + 1], Yl[DF_K][DF_T + 1];
    const int b0 = blockIdx.x * DF_T;
    const long long r0 = (long long)blockIdx.y * DF_T;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float xh[4][4], xl[4][4], yh_[4][4], yl_[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) xh[a][b] = xl[a][b] = yh_[a][b] = yl_[a][b] = 0.0f;
    for (int kb = 0; kb < k; kb += DF_K) {
        for (int idx = threadIdx.x; idx < DF_K * DF_T; idx += DF_THREADS) {
            const int kk = idx / DF_T, cc = idx % DF_T;
            const int i = kb + kk;
            float2 vh = make_float2(0.f, 0.f), vl = vh, wh = vh, wl = vh;
            if (i < k && r0 + cc < n) {
                vh = yh[(size_t)i * n + r0 + cc];
                vl = yl[(size_t)i * n + r0 + cc];
            }
            if (i < k && b0 + cc < m) {
                const double2 cd = c[(size_t)i * ldc + b0 + cc];
                wh = make_float2((float)cd.x, (float)cd.y);
                wl = make_float2((float)(cd.x - (double)wh.x), (float)(cd.y - (double)wh.y));
            }
            Yh[kk][cc] = vh;
            Yl[kk][cc] = vl;
            Ch[kk][cc] = wh;
            Cl[kk][cc] = wl;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < DF_K; ++kk) {
            float2 cv[4], cl[4], yv[4], yw[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                cv[q] = Ch[kk][ty + 16 * q];
                cl[q] = Cl[kk][ty + 16 * q];
                yv[q] = Yh[kk][tx + 16 * q];
                yw[q] = Yl[kk][tx + 16 * q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    // c y: re = cx yx - cy yy, im = cx yy + cy yx
                    df_mac(xh[p][q], xl[p][q], cv[p].x, cl[p].x, yv[q].x, yw[q].x);
                    df_mac(xh[p][q], xl[p][q], -cv[p].y, -cl[p].y, yv[q].y, yw[q].y);
                    df_mac(yh_[p][q], yl_[p][q], cv[p].x, cl[p].x, yv[q].y, yw[q].y);
                    df_mac(yh_[p][q], yl_[p][q], cv[p].y, cl[p].y, yv[q].x, yw[q].x);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int b = b0 + ty + 16 * p;
        if (b >= m) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const long long r = r0 + tx + 16 * q;
            if (r < n)
                out[(size_t)b * n + r] = make_double2((double)xh[p][q] + (double)xl[p][q],
                                                      (double)yh_[p][q] + (double)yl_[p][q]);
        }
    }
}

rsdft_status split_df(rsdft_ctx *ctx, const double2 *x, long long cnt, float2 *h, float2 *l, cudaStream_t st) {
    k_split_df<<<std::max(1, std::min(cdiv(cnt, 256), 8 * ctx->num_sms)), 256, 0, st>>>(x, cnt, h, l);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_split_df");
    return RSDFT_OK;
}

rsdft_status gram_df(rsdft_ctx *ctx, const float2 *ah, const float2 *al, int na, const RowBlocksT<float2> &bh,
                     const RowBlocksT<float2> &bl, double2 *g, int ldg, double scale, cudaStream_t st) {
    const int nb = bh.cnt[0] + bh.cnt[1] + bh.cnt[2];
    if (na <= 0 || nb <= 0) return RSDFT_OK;
    const long long n = ctx->n;
    const int Ti = cdiv(na, DF_T), Tj = cdiv(nb, DF_T);
    const int tiles = Ti * Tj;
    // whole waves of (one CTA per SM x 2), at least 2048 points per CTA
    const int want = std::max(1, cdiv(2LL * ctx->num_sms, tiles));
    const int nsplit = std::max(1, std::min(want, (int)std::max(1LL, n / 2048)));
    long long kchunk = (n + nsplit - 1) / nsplit;
    kchunk = (kchunk + DF_K - 1) / DF_K * DF_K;
    const int ns = (int)((n + kchunk - 1) / kchunk);
    RS_TRY(ensure_gram_partials(ctx, (size_t)ns * na * nb));
    {
        ProfScope ps(ctx, RSDFT_K_GRAM, 8.0 * (double)n * na * nb, 16.0 * (double)n * (na + nb), st);
        k_gram_df<<<dim3(tiles, ns), DF_THREADS, 0, st>>>(ah, al, bh, bl, na, nb, n, Tj, kchunk, ctx->ws.gram_part);
    }
    RS_LAUNCHED(ctx, "k_gram_df");
    return gram_reduce(ctx, ns, na, nb, false, DF_T, scale, g, ldg, st);
}

rsdft_status rotate_df(rsdft_ctx *ctx, const float2 *yh, const float2 *yl, int k, const double2 *c, int ldc, int m,
                       double2 *out, cudaStream_t st) {
    if (m <= 0 || k <= 0) return RSDFT_OK;
    const long long n = ctx->n;
    dim3 grid(cdiv(m, DF_T), cdiv(n, DF_T));
    {
        ProfScope ps(ctx, RSDFT_K_ROTATE, 8.0 * (double)n * k * m, 16.0 * (double)n * (k + m), st);
        k_rotate_df<<<grid, DF_THREADS, 0, st>>>(yh, yl, k, c, ldc, m, n, out);
    }
    RS_LAUNCHED(ctx, "k_rotate_df");
    return RSDFT_OK;
}

}  // namespace rsdft
