// GEMM-shaped kernels of the LOBPCG iteration (SCF task (2)), FP64 complex:
//   gram   : G[i][j] = scale * sum_r conj(A_i(r)) B_j(r)  (reduction length n,
//            split-K over CTAs, partial tiles reduced in a fixed order)
//   rotate : out[b][r] = base[b][r] + sign * sum_i c[i][b] Y_i(r)
// Both read the orbital blocks in their native band-major layout.
#include <algorithm>
#include <mutex>

#include <string>

#include "rsdft_internal.h"

namespace rsdft {

constexpr int GT = 64;      // output tile edge
constexpr int GKC = 16;     // reduction chunk per shared-memory stage
constexpr int GTHREADS = 256;

template <typename V>
__device__ __forceinline__ const V *row_of(const RowBlocksT<V> &rb, int i, long long n) {
    if (i < rb.cnt[0]) return rb.ptr[0] + (size_t)i * n;
    i -= rb.cnt[0];
    if (i < rb.cnt[1]) return rb.ptr[1] + (size_t)i * n;
    i -= rb.cnt[1];
    return rb.ptr[2] + (size_t)i * n;
}

// Upper-triangular tile enumeration: t -> (ti, tj), ti <= tj, row by row.
__device__ __forceinline__ void upper_tile(int t, int T, int &ti, int &tj) {
    int i = 0;
    while (t >= T - i) { t -= T - i; ++i; }
    ti = i;
    tj = i + t;
}

// Partial tiles of G over one K-chunk.  V = double2 (FP64) or float2 (the
// mixed form: FP32 products and accumulation inside the CTA); the partials are
// stored in FP64 and reduced in FP64 by k_gram_reduce.  Output tile edge 16*P
// (each of the 16 x 16 threads owns P x P entries).
template <typename V, int P>
__global__ void __launch_bounds__(GTHREADS)
k_gram_partial(RowBlocksT<V> A, RowBlocksT<V> B, int na, int nb, long long n, int hermitian, int Ti,
               int Tj, long long kchunk, double2 *__restrict__ part) {
    using T = decltype(V{}.x);
    constexpr int TE = 16 * P;
    __shared__ V As[GKC][TE + 1];
    __shared__ V Bs[GKC][TE + 1];
    int ti, tj;
    if (hermitian) upper_tile(blockIdx.x, Ti, ti, tj);
    else { ti = blockIdx.x / Tj; tj = blockIdx.x % Tj; }
    const int split = blockIdx.y;
    const long long k0 = (long long)split * kchunk;
    const long long k1 = min(n, k0 + kchunk);
    const int i0 = ti * TE, j0 = tj * TE;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T ar[P][P], ai[P][P];
#pragma unroll
    for (int a = 0; a < P; ++a)
#pragma unroll
        for (int b = 0; b < P; ++b) ar[a][b] = ai[a][b] = (T)0;
    // loader: TE rows x 16 k per stage; 16 consecutive threads read one row's chunk
    for (long long kb = k0; kb < k1; kb += GKC) {
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int idx = threadIdx.x + q * GTHREADS;
            const int lrow = idx >> 4, lk = idx & 15;
            const long long kk = kb + lk;
            V va, vb;
            va.x = va.y = vb.x = vb.y = (T)0;
            if (kk < k1) {
                if (i0 + lrow < na) va = row_of(A, i0 + lrow, n)[kk];
                if (j0 + lrow < nb) vb = row_of(B, j0 + lrow, n)[kk];
            }
            As[lk][lrow] = va;
            Bs[lk][lrow] = vb;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < GKC; ++k) {
            V a[P], b[P];
#pragma unroll
            for (int q = 0; q < P; ++q) {
                a[q] = As[k][ty + 16 * q];
                b[q] = Bs[k][tx + 16 * q];
            }
#pragma unroll
            for (int p = 0; p < P; ++p)
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    // conj(a) * b
                    ar[p][q] = fma(a[p].x, b[q].x, fma(a[p].y, b[q].y, ar[p][q]));
                    ai[p][q] = fma(a[p].x, b[q].y, fma(-a[p].y, b[q].x, ai[p][q]));
                }
        }
        __syncthreads();
    }
    double2 *pp = part + (size_t)split * na * nb;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int i = i0 + ty + 16 * p;
        if (i >= na) continue;
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int j = j0 + tx + 16 * q;
            if (j < nb) pp[(size_t)i * nb + j] = make_double2((double)ar[p][q], (double)ai[p][q]);
        }
    }
}

__global__ void k_gram_reduce(const double2 *__restrict__ part, int nsplit, int na, int nb,
                              int hermitian, int te, double scale, double2 *__restrict__ g, int ldg) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)na * nb) return;
    const int i = (int)(idx / nb), j = (int)(idx % nb);
    const size_t stride = (size_t)na * nb;
    auto sum_at = [&](int r, int c) {
        double sx = 0.0, sy = 0.0;
        for (int s = 0; s < nsplit; ++s) {
            double2 v = part[s * stride + (size_t)r * nb + c];
            sx += v.x;
            sy += v.y;
        }
        return make_double2(sx, sy);
    };
    double2 val;
    if (!hermitian) {
        val = sum_at(i, j);
    } else {
        const int ti = i / te, tj = j / te;
        if (ti < tj) val = sum_at(i, j);
        else if (ti > tj) { double2 t = sum_at(j, i); val = make_double2(t.x, -t.y); }
        else {
            double2 a = sum_at(i, j), b = sum_at(j, i);
            val = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
        }
    }
    g[(size_t)i * ldg + j] = make_double2(val.x * scale, val.y * scale);
}

static rsdft_status ensure_gram_part(rsdft_ctx *ctx, size_t elems) {
    Workspace &w = ctx->ws;
    if (elems <= w.gram_part_elems) return RSDFT_OK;
    if (w.gram_part) {
        cudaFree(w.gram_part);
        for (auto &p : ctx->owned)
            if (p == w.gram_part) p = nullptr;
    }
    w.gram_part = nullptr;
    w.gram_part_elems = 0;
    RS_TRY(dev_alloc(ctx, (void **)&w.gram_part, elems * sizeof(double2)));
    w.gram_part_elems = elems;
    return RSDFT_OK;
}

rsdft_status ensure_gram_partials(rsdft_ctx *ctx, size_t elems) { return ensure_gram_part(ctx, elems); }

rsdft_status gram_reduce(rsdft_ctx *ctx, int nsplit, int na, int nb, bool hermitian, int te, double scale,
                         double2 *g, int ldg, cudaStream_t st) {
    const long long tot = (long long)na * nb;
    k_gram_reduce<<<cdiv(tot, 256), 256, 0, st>>>(ctx->ws.gram_part, nsplit, na, nb, hermitian ? 1 : 0, te, scale,
                                                   g, ldg);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_gram_reduce");
    return RSDFT_OK;
}

// Resident CTAs of a kernel per SM (queried once per instantiation).
template <typename K> static int occupancy(K kernel, int threads) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, 0) != cudaSuccess) {
        cudaGetLastError();
        occ = 1;
    }
    return std::max(1, occ);
}

// Output tile edge 16*P with the least padding over an extent (ties: larger P).
static int pick_p(int extent_a, int extent_b) {
    int best = 4;
    long long bestpad = -1;
    for (int P = 4; P >= 2; --P) {
        const long long te = 16 * P;
        const long long pad = (long long)cdiv(extent_a, te) * te * cdiv(extent_b, te) * te;
        if (bestpad < 0 || pad < bestpad) { bestpad = pad; best = P; }
    }
    return best;
}

// Split count for `tiles` output tiles: the first count whose grid fills whole
// waves of the resident-CTA capacity to 97% (else the best seen), keeping at
// least 512 reduction points per CTA.
static int pick_splits(int tiles, long long n, int capacity) {
    int best = 1;
    double besteff = 0.0;
    for (int ns = 1; ns <= 128; ++ns) {
        if (ns > 1 && n / ns < 512) break;
        const long long ctas = (long long)tiles * ns;
        const long long waves = (ctas + capacity - 1) / capacity;
        const double eff = (double)ctas / (double)(waves * capacity);
        if (eff > besteff + 1e-9) { besteff = eff; best = ns; }
        if (eff >= 0.97) return ns;
    }
    return best;
}

template <typename V, int P>
static rsdft_status gram_launch(rsdft_ctx *ctx, const RowBlocksT<V> &A, const RowBlocksT<V> &B,
                                int na, int nb, double2 *g, int ldg, bool hermitian, double scale,
                                cudaStream_t st) {
    constexpr int TE = 16 * P;
    static int occ = occupancy(k_gram_partial<V, P>, GTHREADS);
    const int Ti = cdiv(na, TE), Tj = cdiv(nb, TE);
    const int tiles = hermitian ? Ti * (Ti + 1) / 2 : Ti * Tj;
    const long long n = ctx->n;
    int nsplit = pick_splits(tiles, n, ctx->num_sms * occ);
    long long kchunk = (n + nsplit - 1) / nsplit;
    kchunk = (kchunk + GKC - 1) / GKC * GKC;
    nsplit = (int)((n + kchunk - 1) / kchunk);
    RS_TRY(ensure_gram_part(ctx, (size_t)nsplit * na * nb));
    dim3 grid(tiles, nsplit);
    {
        const bool same = (const void *)A.ptr[0] == (const void *)B.ptr[0] &&
                          (const void *)A.ptr[1] == (const void *)B.ptr[1] &&
                          (const void *)A.ptr[2] == (const void *)B.ptr[2];
        const double entries = hermitian ? 0.5 * na * (na + 1.0) : (double)na * nb;
        ProfScope ps(ctx, RSDFT_K_GRAM, 8.0 * (double)n * entries,
                     (double)n * sizeof(V) * (same ? na : na + nb), st);
        k_gram_partial<V, P><<<grid, GTHREADS, 0, st>>>(A, B, na, nb, n, hermitian ? 1 : 0, Ti, Tj, kchunk,
                                                        ctx->ws.gram_part);
    }
    RS_LAUNCHED(ctx, "k_gram_partial");
    const long long tot = (long long)na * nb;
    k_gram_reduce<<<cdiv(tot, 256), 256, 0, st>>>(ctx->ws.gram_part, nsplit, na, nb,
                                                   hermitian ? 1 : 0, TE, scale, g, ldg);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_gram_reduce");
    return RSDFT_OK;
}

template <typename V>
rsdft_status gram_t(rsdft_ctx *ctx, const RowBlocksT<V> &A, const RowBlocksT<V> &B, double2 *g, int ldg,
                    bool hermitian, double scale, cudaStream_t st) {
    const int na = A.cnt[0] + A.cnt[1] + A.cnt[2];
    const int nb = B.cnt[0] + B.cnt[1] + B.cnt[2];
    if (na <= 0 || nb <= 0) return RSDFT_OK;
    if (hermitian && na != nb) return fail(ctx, RSDFT_E_INVALID, "hermitian gram needs na == nb");
    // tile edge 16 P, P in {2, 3, 4}: the least-padding rule, or the autotuner's pick
    auto run = [&](int c) -> rsdft_status {
        switch (c + 2) {
            case 2: return gram_launch<V, 2>(ctx, A, B, na, nb, g, ldg, hermitian, scale, st);
            case 3: return gram_launch<V, 3>(ctx, A, B, na, nb, g, ldg, hermitian, scale, st);
            default: return gram_launch<V, 4>(ctx, A, B, na, nb, g, ldg, hermitian, scale, st);
        }
    };
    // shapes in buckets of 32 (the subspace size changes as bands lock)
    const std::string key = std::string(sizeof(V) == 8 ? "gram32 " : "gram64 ") +
                            std::to_string(cdiv(na, 32)) +
                            " " + std::to_string(cdiv(nb, 32)) + (hermitian ? " h" : " g");
    int chosen = 0;
    return autotune_pick(ctx, key, 3, pick_p(na, nb) - 2, st, run, &chosen);
}

rsdft_status gram(rsdft_ctx *ctx, const RowBlocks &A, const RowBlocks &B, double2 *g, int ldg,
                  bool hermitian, double scale, cudaStream_t st) {
    return gram_t<double2>(ctx, A, B, g, ldg, hermitian, scale, st);
}
rsdft_status gram32(rsdft_ctx *ctx, const RowBlocksT<float2> &A, const RowBlocksT<float2> &B,
                    double2 *g, int ldg, bool hermitian, double scale, cudaStream_t st) {
    return gram_t<float2>(ctx, A, B, g, ldg, hermitian, scale, st);
}


// ---- rotation ----------------------------------------------------------------------
// Tile: 64 bands x 64 points.  Rows of Y are consumed block 1, block 2, then
// block 0, so that out1 (the W/P part alone) is available before the X part is
// added.
template <typename V, int PB>
__global__ void __launch_bounds__(GTHREADS)
k_rotate(RowBlocksT<V> Y, const double2 *__restrict__ c, int ldc, int m, long long n,
         const V *base, int sign, V *out0, V *out1) {
    using T = decltype(V{}.x);
    constexpr int TB = 16 * PB;   // bands per tile (the points per tile are GT = 64)
    __shared__ V Cs[GKC][TB + 1];
    __shared__ V Ys[GKC][GT + 1];
    const int b0 = blockIdx.x * TB;
    const long long r0 = (long long)blockIdx.y * GT;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T accx[PB][4], accy[PB][4];
#pragma unroll
    for (int p = 0; p < PB; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) accx[p][q] = accy[p][q] = (T)0;
#pragma unroll
    for (int oi = 0; oi < 3; ++oi) {
        // blocks in the order 1, 2, 0; crow0 = first row of the block in c
        const int cnt = oi == 0 ? Y.cnt[1] : (oi == 1 ? Y.cnt[2] : Y.cnt[0]);
        const V *yb = oi == 0 ? Y.ptr[1] : (oi == 1 ? Y.ptr[2] : Y.ptr[0]);
        const int crow0 = oi == 0 ? Y.cnt[0] : (oi == 1 ? Y.cnt[0] + Y.cnt[1] : 0);
        for (int kb = 0; kb < cnt; kb += GKC) {
            for (int idx = threadIdx.x; idx < GKC * GT; idx += GTHREADS) {
                const int kk = idx / GT, cc = idx % GT;
                const int i = kb + kk;
                V yv;
                yv.x = yv.y = (T)0;
                if (i < cnt && r0 + cc < n) yv = yb[(size_t)i * n + r0 + cc];
                Ys[kk][cc] = yv;
            }
            for (int idx = threadIdx.x; idx < GKC * TB; idx += GTHREADS) {
                const int kk = idx / TB, cc = idx % TB;
                const int i = kb + kk;
                V cv;
                cv.x = cv.y = (T)0;
                if (i < cnt && b0 + cc < m) {
                    const double2 cd = c[(size_t)(crow0 + i) * ldc + b0 + cc];
                    cv.x = (T)cd.x;
                    cv.y = (T)cd.y;
                }
                Cs[kk][cc] = cv;
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < GKC; ++k) {
                V cv[PB], yv[4];
#pragma unroll
                for (int q = 0; q < PB; ++q) cv[q] = Cs[k][ty + 16 * q];
#pragma unroll
                for (int q = 0; q < 4; ++q) yv[q] = Ys[k][tx + 16 * q];
#pragma unroll
                for (int p = 0; p < PB; ++p)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        accx[p][q] = fma(cv[p].x, yv[q].x, fma(-cv[p].y, yv[q].y, accx[p][q]));
                        accy[p][q] = fma(cv[p].x, yv[q].y, fma(cv[p].y, yv[q].x, accy[p][q]));
                    }
            }
            __syncthreads();
        }
        if (oi == 1 && out1) {
#pragma unroll
            for (int p = 0; p < PB; ++p) {
                const int b = b0 + ty + 16 * p;
                if (b >= m) continue;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const long long r = r0 + tx + 16 * q;
                    if (r < n) {
                        V o;
                        o.x = accx[p][q];
                        o.y = accy[p][q];
                        out1[(size_t)b * n + r] = o;
                    }
                }
            }
        }
    }
    const T sg = (T)sign;
#pragma unroll
    for (int p = 0; p < PB; ++p) {
        const int b = b0 + ty + 16 * p;
        if (b >= m) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const long long r = r0 + tx + 16 * q;
            if (r >= n) continue;
            T ox = sg * accx[p][q], oy = sg * accy[p][q];
            if (base) {
                const V bv = base[(size_t)b * n + r];
                ox += bv.x;
                oy += bv.y;
            }
            V o;
            o.x = ox;
            o.y = oy;
            out0[(size_t)b * n + r] = o;
        }
    }
}

template <typename V, int PB>
static rsdft_status rotate_launch(rsdft_ctx *ctx, const RowBlocksT<V> &Y, const double2 *c, int ldc,
                                  int m, const V *base, int sign, V *out0, V *out1, cudaStream_t st) {
    dim3 grid(cdiv(m, 16 * PB), cdiv(ctx->n, GT));
    const int k = Y.cnt[0] + Y.cnt[1] + Y.cnt[2];
    ProfScope ps(ctx, RSDFT_K_ROTATE, 8.0 * (double)ctx->n * k * m,
                 (double)sizeof(V) * (double)ctx->n * (k + m + (out1 ? m : 0) + (base ? m : 0)), st);
    k_rotate<V, PB><<<grid, GTHREADS, 0, st>>>(Y, c, ldc, m, ctx->n, base, sign, out0, out1);
    RS_LAUNCHED(ctx, "k_rotate");
    return RSDFT_OK;
}

// Band tile 16*PB with the least padding over m bands (ties: larger PB).
template <typename V>
rsdft_status rotate_t(rsdft_ctx *ctx, const RowBlocksT<V> &Y, const double2 *c, int ldc, int m,
                      const V *base, int sign, V *out0, V *out1, cudaStream_t st) {
    if (m <= 0) return RSDFT_OK;
    int best = 4, bestpad = 1 << 30;
    for (int pb = 4; pb >= 1; --pb) {
        const int pad = cdiv(m, 16 * pb) * 16 * pb - m;
        if (pad < bestpad) { bestpad = pad; best = pb; }
    }
    auto run = [&](int cand) -> rsdft_status {
        switch (cand + 1) {
            case 1: return rotate_launch<V, 1>(ctx, Y, c, ldc, m, base, sign, out0, out1, st);
            case 2: return rotate_launch<V, 2>(ctx, Y, c, ldc, m, base, sign, out0, out1, st);
            case 3: return rotate_launch<V, 3>(ctx, Y, c, ldc, m, base, sign, out0, out1, st);
            default: return rotate_launch<V, 4>(ctx, Y, c, ldc, m, base, sign, out0, out1, st);
        }
    };
    // an update in place (base) may not run twice: the least-padding rule only
    if (base) return run(best - 1);
    const int k = Y.cnt[0] + Y.cnt[1] + Y.cnt[2];
    const std::string key = std::string(sizeof(V) == 8 ? "rot32 " : "rot64 ") + std::to_string(cdiv(k, 32)) +
                            " " + std::to_string(cdiv(m, 32)) + (out1 ? " p" : " x");
    int chosen = 0;
    return autotune_pick(ctx, key, 4, best - 1, st, run, &chosen);
}

rsdft_status rotate(rsdft_ctx *ctx, const RowBlocks &Y, const double2 *c, int ldc, int m,
                    const double2 *base, int sign, double2 *out0, double2 *out1,
                    cudaStream_t st) {
    return rotate_t<double2>(ctx, Y, c, ldc, m, base, sign, out0, out1, st);
}
rsdft_status rotate32(rsdft_ctx *ctx, const RowBlocksT<float2> &Y, const double2 *c, int ldc, int m,
                      const float2 *base, int sign, float2 *out0, float2 *out1, cudaStream_t st) {
    return rotate_t<float2>(ctx, Y, c, ldc, m, base, sign, out0, out1, st);
}

// ---- Gram without allocation -------------------------------------------------------
// Split-K partial tiles of rsdft_gram_static live in this fixed array, which
// every GPU that loads the library holds until the process exits.
constexpr size_t STATIC_GRAM_ELEMS = (size_t)1 << 21;   // complex128 entries, 32 MiB
static __device__ __align__(256) double2 g_static_gram_part[STATIC_GRAM_ELEMS];

constexpr int STATIC_MAX_DEVICES = 64;
static std::mutex g_static_mu;
static double2 *g_static_addr[STATIC_MAX_DEVICES] = {};

// Device address of g_static_gram_part on the current device, looked up once
// per device (the host-side name is only a stand-in for it).
static rsdft_status static_gram_scratch(double2 **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, RSDFT_E_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    }
    if (dev < 0 || dev >= STATIC_MAX_DEVICES)
        return fail(nullptr, RSDFT_E_INVALID, "device %d beyond the %d supported", dev, STATIC_MAX_DEVICES);
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_gram_part);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail(nullptr, RSDFT_E_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        }
        g_static_addr[dev] = static_cast<double2 *>(p);
    }
    *out = g_static_addr[dev];
    return RSDFT_OK;
}

}  // namespace rsdft

using namespace rsdft;

extern "C" {

rsdft_status rsdft_gram_static(const void *a_dev, int na, const void *b_dev, int nb, long long n,
                               double scale, void *g_dev, void *stream) {
    if (na < 0 || nb < 0 || n <= 0)
        return fail(nullptr, RSDFT_E_INVALID, "need na >= 0, nb >= 0, n > 0");
    if (na == 0 || nb == 0) return RSDFT_OK;
    if (!a_dev || !b_dev || !g_dev) return fail(nullptr, RSDFT_E_INVALID, "null pointer argument");
    if ((size_t)na * (size_t)nb > STATIC_GRAM_ELEMS)
        return fail(nullptr, RSDFT_E_INVALID,
                    "na*nb = %lld exceeds the fixed scratch of %zu entries (rsdft_gram_static)",
                    (long long)na * nb, STATIC_GRAM_ELEMS);
    double2 *part = nullptr;
    RS_TRY(static_gram_scratch(&part));
    cudaStream_t st = as_stream(stream);
    const int Ti = cdiv(na, GT), Tj = cdiv(nb, GT);
    const int tiles = Ti * Tj;
    int nsplit = std::max(1, std::min(cdiv(1216, tiles), 16));
    while (nsplit > 1 && n / nsplit < 2048) --nsplit;
    nsplit = std::max(1, std::min<int>(nsplit, (int)(STATIC_GRAM_ELEMS / ((size_t)na * nb))));
    long long kchunk = (n + nsplit - 1) / nsplit;
    kchunk = (kchunk + GKC - 1) / GKC * GKC;
    nsplit = (int)((n + kchunk - 1) / kchunk);
    RowBlocks A{{(const double2 *)a_dev, nullptr, nullptr}, {na, 0, 0}};
    RowBlocks B{{(const double2 *)b_dev, nullptr, nullptr}, {nb, 0, 0}};
    // every partial entry the reduction reads is written by this launch first,
    // so nothing left by an earlier call is read
    k_gram_partial<double2, 4><<<dim3(tiles, nsplit), GTHREADS, 0, st>>>(A, B, na, nb, n, 0, Ti, Tj, kchunk, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(nullptr, RSDFT_E_CUDA, "k_gram_partial: %s", cudaGetErrorString(e));
    k_gram_reduce<<<cdiv((long long)na * nb, 256), 256, 0, st>>>(part, nsplit, na, nb, 0, GT, scale,
                                                                 (double2 *)g_dev, nb);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(nullptr, RSDFT_E_CUDA, "k_gram_reduce: %s", cudaGetErrorString(e));
    return RSDFT_OK;
}

rsdft_status rsdft_gram(rsdft_ctx *ctx, const void *a_dev, int na, const void *b_dev, int nb,
                        void *g_dev, void *stream) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (na < 0 || nb < 0 || ((na > 0 && nb > 0) && (!a_dev || !b_dev || !g_dev)))
        return fail(ctx, RSDFT_E_INVALID, "bad gram arguments");
    RowBlocks A{{(const double2 *)a_dev, nullptr, nullptr}, {na, 0, 0}};
    RowBlocks B{{(const double2 *)b_dev, nullptr, nullptr}, {nb, 0, 0}};
    return gram(ctx, A, B, (double2 *)g_dev, nb, false, ctx->dV, as_stream(stream));
}

rsdft_status rsdft_rotate(rsdft_ctx *ctx, const void *y_dev, int k, const void *c_dev, int m,
                          const void *base_dev, int sign, void *out_dev, void *stream) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (k < 0 || m < 0 || (m > 0 && (!out_dev || (k > 0 && (!y_dev || !c_dev)))) ||
        (sign != 1 && sign != -1))
        return fail(ctx, RSDFT_E_INVALID, "bad rotate arguments");
    RowBlocks Y{{(const double2 *)y_dev, nullptr, nullptr}, {k, 0, 0}};
    return rotate(ctx, Y, (const double2 *)c_dev, m, m, (const double2 *)base_dev, sign,
                  (double2 *)out_dev, nullptr, as_stream(stream));
}

}  // extern "C"
