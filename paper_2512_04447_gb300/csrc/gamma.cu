// The real-arithmetic Gamma-point form of the LOBPCG block iteration: the
// paper's real-symmetric case (its eigensolver benchmark, Fig. 3a beside the
// Hermitian Fig. 3b), FP64.
//
// At Gamma, with a real local potential and real Kleinman-Bylander projectors,
// H maps real grid functions to real ones, and the lowest eigenvectors can be
// taken real.  Layout: two real bands share one complex "pair row" -- band b is
// component (b & 1) (.x or .y) of row b / 2 of a [ceil(c / 2)][n] complex block;
// when a block holds an odd number c of bands, the .y half of its last row is
// padding (zero, or rounding noise after H) and takes no part in any result.
//  - H psi: H is real-linear and preserves real functions, so H (x_a + i x_b) =
//    H x_a + i H x_b; the complex H psi kernels (fft.cu) transform two real bands
//    for the price of one complex band, half the FFT work of the complex form,
//    as a real-to-complex transform would.  The projector coefficients come out
//    as pairs too (<beta|x_a>, <beta|x_b>).
//  - Gram matrices: a tile of pair rows is loaded like a complex tile and gives
//    the four real products x_a y_a, x_a y_b, x_b y_a, x_b y_b per pair of
//    elements: over m real bands, m^2 n multiply-adds, a quarter of the complex
//    form's 4 m^2 n.  The rotation alike.
//  - TPA: the factor K((|G|^2/2) / t_b) depends on the band, so the two bands of
//    a pair cannot share its transform; residuals go through the complex TPA
//    passes one band per row (imaginary part zero) and only the real part of
//    the result is kept.
//  - Eq. 1 is real symmetric here.  It runs through the Hermitian dense core
//    (dense.cu) with zero imaginary parts: its reflectors are formed by the
//    LAPACK zlarfg rule, which for a real leading entry and a real column gives
//    real tau and v, its tridiagonal eigenvectors are real, and every product
//    with a zero imaginary part is an exact zero, so the coefficients C come
//    back real and the rotations read their real parts.
#include <algorithm>
#include <cmath>
#include <string>

#include "rsdft_internal.h"

namespace rsdft {

namespace {

constexpr int GR_THREADS = 256;
constexpr int GRK = 16;      // reduction chunk (points for the Gram, input pair rows for the rotation)
constexpr int GRPTS = 64;    // points per rotation tile

__host__ __device__ __forceinline__ int pairs_of(int c) { return (c + 1) >> 1; }
__device__ __forceinline__ double comp(double2 v, int h) { return h ? v.y : v.x; }

__device__ __forceinline__ double block_sum(double v, double *sh) {
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

__device__ __forceinline__ void slice_range(long long n, int S, int s, long long &i0, long long &i1) {
    const long long c = (n + S - 1) / S;
    i0 = (long long)s * c;
    i1 = i0 + c < n ? i0 + c : n;
}

// slices per row: about 8 CTAs per SM over all rows, at least 4096 points each
int slices_for(const rsdft_ctx *ctx, int rows) {
    const int want = cdiv(8 * ctx->num_sms, std::max(rows, 1));
    const int most = (int)std::max(1LL, ctx->n / 4096);
    return std::max(1, std::min(std::min(want, most), 64));
}

dim3 row_grid(long long n, int rows) { return dim3(std::min(cdiv(n, 256), 1024), rows); }

}  // namespace

// ---- layout conversion -------------------------------------------------------------
// pair row j <- (x[2j], x[2j+1]); the .y half is 0 past the last band
__global__ void k_pack_pairs(const double *__restrict__ x, int m, long long n, double2 *__restrict__ out) {
    const int j = blockIdx.y;
    const double *a = x + (size_t)(2 * j) * n;
    const double *b = 2 * j + 1 < m ? x + (size_t)(2 * j + 1) * n : nullptr;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[(size_t)j * n + i] = make_double2(a[i], b ? b[i] : 0.0);
}

__global__ void k_unpack_pairs(const double2 *__restrict__ in, int m, long long n, double *__restrict__ x) {
    const int j = blockIdx.y;
    double *a = x + (size_t)(2 * j) * n;
    double *b = 2 * j + 1 < m ? x + (size_t)(2 * j + 1) * n : nullptr;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double2 v = in[(size_t)j * n + i];
        a[i] = v.x;
        if (b) b[i] = v.y;
    }
}

// pair row j <- (Re in[2j], Re in[2j+1]) from complex rows (one band each)
__global__ void k_real_to_pairs(const double2 *__restrict__ in, int cnt, long long n, double2 *__restrict__ w) {
    const int j = blockIdx.y;
    const double2 *a = in + (size_t)(2 * j) * n;
    const double2 *b = 2 * j + 1 < cnt ? in + (size_t)(2 * j + 1) * n : nullptr;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        w[(size_t)j * n + i] = make_double2(a[i].x, b ? b[i].x : 0.0);
}

// ---- per-band reductions -----------------------------------------------------------
// part[(j S + s) 2]     = (|r_2j|^2, |r_2j+1|^2) over slice s, r_b = hx_b - theta_b x_b
// part[(j S + s) 2 + 1] = (sum V x_2j^2, sum V x_2j+1^2)
__global__ void __launch_bounds__(GR_THREADS)
k_resid_pair_part(const double2 *__restrict__ hx, const double2 *__restrict__ x, const double *__restrict__ theta,
                  const double *__restrict__ v, int m, long long n, int S, double2 *__restrict__ part) {
    __shared__ double sh[33];
    const int s_ = blockIdx.x, j = blockIdx.y;
    long long i0, i1;
    slice_range(n, S, s_, i0, i1);
    const double ta = theta[2 * j], tb = 2 * j + 1 < m ? theta[2 * j + 1] : 0.0;
    const double2 *h = hx + (size_t)j * n, *xx = x + (size_t)j * n;
    double sa = 0.0, sb = 0.0, va = 0.0, vb = 0.0;
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const double2 a = h[i], c = xx[i];
        const double vv = v[i];
        const double ra = a.x - ta * c.x, rb = a.y - tb * c.y;
        sa = fma(ra, ra, sa);
        sb = fma(rb, rb, sb);
        va = fma(vv * c.x, c.x, va);
        vb = fma(vv * c.y, c.y, vb);
    }
    sa = block_sum(sa, sh);
    sb = block_sum(sb, sh);
    va = block_sum(va, sh);
    vb = block_sum(vb, sh);
    if (threadIdx.x == 0) {
        part[((size_t)j * S + s_) * 2] = make_double2(sa, sb);
        part[((size_t)j * S + s_) * 2 + 1] = make_double2(va, vb);
    }
}

// res[b] = ||r_b|| (dV metric), vexp[b] = <x_b|V|x_b>
__global__ void k_resid_pair_fin(const double2 *__restrict__ part, int S, int m, double dV, double *res, double *vexp) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= m) return;
    const int j = b >> 1, hf = b & 1;
    double s = 0.0, sv = 0.0;
    for (int q = 0; q < S; ++q) {
        s += comp(part[((size_t)j * S + q) * 2], hf);
        sv += comp(part[((size_t)j * S + q) * 2 + 1], hf);
    }
    res[b] = sqrt(s * dV);
    vexp[b] = sv * dV;
}

// part[j S + s] = (sum x_2j^2, sum x_2j+1^2) over slice s
__global__ void __launch_bounds__(GR_THREADS)
k_rownorm_pair_part(const double2 *__restrict__ a, long long n, int S, double2 *__restrict__ part) {
    __shared__ double sh[33];
    const int s_ = blockIdx.x, j = blockIdx.y;
    long long i0, i1;
    slice_range(n, S, s_, i0, i1);
    const double2 *r = a + (size_t)j * n;
    double sa = 0.0, sb = 0.0;
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const double2 v = r[i];
        sa = fma(v.x, v.x, sa);
        sb = fma(v.y, v.y, sb);
    }
    sa = block_sum(sa, sh);
    sb = block_sum(sb, sh);
    if (threadIdx.x == 0) part[(size_t)j * S + s_] = make_double2(sa, sb);
}

__global__ void k_rownorm_pair_fin(const double2 *__restrict__ part, int S, int cnt, double dV, double *out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= cnt) return;
    double s = 0.0;
    for (int q = 0; q < S; ++q) s += comp(part[(size_t)(b >> 1) * S + q], b & 1);
    out[b] = sqrt(s * dV);
}

// t_b = theta_b - <x_b|V|x_b> - sum_q E_q <beta_q|x_b>^2 for the active bands
// (compact index j); p holds the projections of the pair rows of X
__global__ void k_tkin_pair(const double *__restrict__ theta, const double *__restrict__ vexp,
                            const double2 *__restrict__ p, ProjTables pt, const int *__restrict__ act, int na,
                            double *tkin) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= na) return;
    const int b = act[j];
    const int np = pt.natom * pt.nproj;
    double nl = 0.0;
    for (int q = 0; q < np; ++q) {
        const double c = comp(p[(size_t)(b >> 1) * np + q], b & 1);
        nl += pt.e_kb[q] * c * c;
    }
    tkin[j] = theta[b] - vexp[b] - nl;
}

// ---- row kernels ---------------------------------------------------------------------
// complex row j <- (r_b, 0), b = act[j]: one band per row for the TPA transforms
__global__ void k_resid_rows_cplx(const double2 *__restrict__ hx, const double2 *__restrict__ x,
                                  const double *__restrict__ theta, const int *__restrict__ act, long long n,
                                  double2 *__restrict__ out) {
    const int j = blockIdx.y;
    const int b = act[j], hf = b & 1;
    const double th = theta[b];
    const double2 *h = hx + (size_t)(b >> 1) * n, *xx = x + (size_t)(b >> 1) * n;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[(size_t)j * n + i] = make_double2(comp(h[i], hf) - th * comp(xx[i], hf), 0.0);
}

// pair row j <- (r_act[2j], r_act[2j+1]) (0 past na)
__global__ void k_resid_rows_pair(const double2 *__restrict__ hx, const double2 *__restrict__ x,
                                  const double *__restrict__ theta, const int *__restrict__ act, int na,
                                  long long n, double2 *__restrict__ w) {
    const int j = blockIdx.y;
    const int ba = act[2 * j], bb = 2 * j + 1 < na ? act[2 * j + 1] : -1;
    const double ta = theta[ba], tb = bb >= 0 ? theta[bb] : 0.0;
    const double2 *ha = hx + (size_t)(ba >> 1) * n, *xa = x + (size_t)(ba >> 1) * n;
    const double2 *hb = bb >= 0 ? hx + (size_t)(bb >> 1) * n : nullptr;
    const double2 *xb = bb >= 0 ? x + (size_t)(bb >> 1) * n : nullptr;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double ra = comp(ha[i], ba & 1) - ta * comp(xa[i], ba & 1);
        const double rb = hb ? comp(hb[i], bb & 1) - tb * comp(xb[i], bb & 1) : 0.0;
        w[(size_t)j * n + i] = make_double2(ra, rb);
    }
}

// the two bands of pair row j divided by their norms (the padding half unchanged)
__global__ void k_scale_pairs(double2 *a, double2 *a2, int cnt, long long n, const double *__restrict__ nrm) {
    const int j = blockIdx.y;
    const double sa = 1.0 / nrm[2 * j];
    const double sb = 2 * j + 1 < cnt ? 1.0 / nrm[2 * j + 1] : 1.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double2 &x = a[(size_t)j * n + i];
        x.x *= sa;
        x.y *= sb;
        if (a2) {
            double2 &y = a2[(size_t)j * n + i];
            y.x *= sa;
            y.y *= sb;
        }
    }
}

// dst pair row j <- (band act[2j], band act[2j+1]) of src (0 past cnt); dst2 alike
__global__ void k_gather_pairs(const double2 *__restrict__ src, const double2 *__restrict__ src2,
                               const int *__restrict__ act, int cnt, long long n, double2 *__restrict__ dst,
                               double2 *__restrict__ dst2) {
    const int j = blockIdx.y;
    const int ba = act[2 * j], bb = 2 * j + 1 < cnt ? act[2 * j + 1] : -1;
    const size_t ra = (size_t)(ba >> 1) * n, rb = bb >= 0 ? (size_t)(bb >> 1) * n : 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        dst[(size_t)j * n + i] = make_double2(comp(src[ra + i], ba & 1), bb >= 0 ? comp(src[rb + i], bb & 1) : 0.0);
        dst2[(size_t)j * n + i] = make_double2(comp(src2[ra + i], ba & 1), bb >= 0 ? comp(src2[rb + i], bb & 1) : 0.0);
    }
}

// ---- Gram matrices on pair rows --------------------------------------------------------
__device__ __forceinline__ const double2 *pair_row(const RowBlocks &rb, int i, long long n) {
    const int p0 = pairs_of(rb.cnt[0]), p1 = pairs_of(rb.cnt[1]);
    if (i < p0) return rb.ptr[0] + (size_t)i * n;
    i -= p0;
    if (i < p1) return rb.ptr[1] + (size_t)i * n;
    i -= p1;
    return rb.ptr[2] + (size_t)i * n;
}

// position of compact real band i of blocks (c0, c1, ...) among the padded
// bands (2 per pair row)
__device__ __forceinline__ int padded_band(int c0, int c1, int i) {
    if (i < c0) return i;
    i -= c0;
    const int base = 2 * pairs_of(c0);
    if (i < c1) return base + i;
    return base + 2 * pairs_of(c1) + (i - c1);
}

__device__ __forceinline__ void upper_tile_of(int t, int T, int &ti, int &tj) {
    int i = 0;
    while (t >= T - i) { t -= T - i; ++i; }
    ti = i;
    tj = i + t;
}

// Partial sums over one reduction chunk of the padded real Gram: part[split][I][J],
// I < 2 pa, J < 2 pb.  Tile edge 16 P pair rows (32 P real bands); each of the
// 16 x 16 threads owns P x P pairs of pair rows, four real products each.
template <int P>
__global__ void __launch_bounds__(GR_THREADS)
k_gram_pair(RowBlocks A, RowBlocks B, int pa, int pb, long long n, int sym, int Ti, int Tj, long long kchunk,
            double *__restrict__ part) {
    constexpr int TE = 16 * P;
    __shared__ double2 As[GRK][TE + 1];
    __shared__ double2 Bs[GRK][TE + 1];
    int ti, tj;
    if (sym) upper_tile_of(blockIdx.x, Ti, ti, tj);
    else { ti = blockIdx.x / Tj; tj = blockIdx.x % Tj; }
    const int split = blockIdx.y;
    const long long k0 = (long long)split * kchunk;
    const long long k1 = min(n, k0 + kchunk);
    const int i0 = ti * TE, j0 = tj * TE;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[P][P][4];
#pragma unroll
    for (int a = 0; a < P; ++a)
#pragma unroll
        for (int b = 0; b < P; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.0;
    for (long long kb = k0; kb < k1; kb += GRK) {
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int idx = threadIdx.x + q * GR_THREADS;
            const int lrow = idx >> 4, lk = idx & 15;
            const long long kk = kb + lk;
            double2 va = make_double2(0.0, 0.0), vb = make_double2(0.0, 0.0);
            if (kk < k1) {
                if (i0 + lrow < pa) va = pair_row(A, i0 + lrow, n)[kk];
                if (j0 + lrow < pb) vb = pair_row(B, j0 + lrow, n)[kk];
            }
            As[lk][lrow] = va;
            Bs[lk][lrow] = vb;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < GRK; ++k) {
            double2 a[P], b[P];
#pragma unroll
            for (int q = 0; q < P; ++q) {
                a[q] = As[k][ty + 16 * q];
                b[q] = Bs[k][tx + 16 * q];
            }
#pragma unroll
            for (int p = 0; p < P; ++p)
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    acc[p][q][0] = fma(a[p].x, b[q].x, acc[p][q][0]);
                    acc[p][q][1] = fma(a[p].x, b[q].y, acc[p][q][1]);
                    acc[p][q][2] = fma(a[p].y, b[q].x, acc[p][q][2]);
                    acc[p][q][3] = fma(a[p].y, b[q].y, acc[p][q][3]);
                }
        }
        __syncthreads();
    }
    const size_t ldp = 2 * (size_t)pb;
    double *pp = part + (size_t)split * 2 * pa * ldp;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        const int i = i0 + ty + 16 * p;
        if (i >= pa) continue;
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int j = j0 + tx + 16 * q;
            if (j >= pb) continue;
            pp[(size_t)(2 * i) * ldp + 2 * j] = acc[p][q][0];
            pp[(size_t)(2 * i) * ldp + 2 * j + 1] = acc[p][q][1];
            pp[(size_t)(2 * i + 1) * ldp + 2 * j] = acc[p][q][2];
            pp[(size_t)(2 * i + 1) * ldp + 2 * j + 1] = acc[p][q][3];
        }
    }
}

// g[i][j] = (scale * sum_s part[s][I][J], 0) for compact real bands i < na,
// j < nb (I, J their padded positions).  sym: entries of tiles below the
// diagonal (pair-row tiles of edge te) are read from their mirror, diagonal
// tiles are averaged with it.
__global__ void k_gram_pair_reduce(const double *__restrict__ part, int nsplit, int pa, int pb, int a0, int a1,
                                   int b0, int b1, int na, int nb, int sym, int te, double scale,
                                   double2 *__restrict__ g, int ldg) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)na * nb) return;
    const int i = (int)(idx / nb), j = (int)(idx % nb);
    const int I = padded_band(a0, a1, i), J = padded_band(b0, b1, j);
    const size_t ldp = 2 * (size_t)pb, stride = 2 * (size_t)pa * ldp;
    auto sum_at = [&](int r, int c) {
        double s = 0.0;
        for (int q = 0; q < nsplit; ++q) s += part[q * stride + (size_t)r * ldp + c];
        return s;
    };
    double v;
    if (!sym) {
        v = sum_at(I, J);
    } else {
        const int ti = (I >> 1) / te, tj = (J >> 1) / te;
        if (ti < tj) v = sum_at(I, J);
        else if (ti > tj) v = sum_at(J, I);
        else v = 0.5 * (sum_at(I, J) + sum_at(J, I));
    }
    g[(size_t)i * ldg + j] = make_double2(v * scale, 0.0);
}

namespace {

template <typename K> int occupancy_of(K kernel) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, GR_THREADS, 0) != cudaSuccess) {
        cudaGetLastError();
        occ = 1;
    }
    return std::max(1, occ);
}

// the first split count whose grid fills whole waves to 97% (else the best
// seen), at least 512 points per CTA
int splits_for(int tiles, long long n, int capacity) {
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

template <int P>
rsdft_status gram_pair_launch(rsdft_ctx *ctx, const RowBlocks &A, const RowBlocks &B, int na, int nb, double2 *g,
                              int ldg, bool sym, double scale, cudaStream_t st) {
    constexpr int TE = 16 * P;
    static int occ = occupancy_of(k_gram_pair<P>);
    const int pa = pairs_of(A.cnt[0]) + pairs_of(A.cnt[1]) + pairs_of(A.cnt[2]);
    const int pb = pairs_of(B.cnt[0]) + pairs_of(B.cnt[1]) + pairs_of(B.cnt[2]);
    const int Ti = cdiv(pa, TE), Tj = cdiv(pb, TE);
    const int tiles = sym ? Ti * (Ti + 1) / 2 : Ti * Tj;
    const long long n = ctx->n;
    int nsplit = splits_for(tiles, n, ctx->num_sms * occ);
    long long kchunk = (n + nsplit - 1) / nsplit;
    kchunk = (kchunk + GRK - 1) / GRK * GRK;
    nsplit = (int)((n + kchunk - 1) / kchunk);
    // 4 pa pb doubles per split = 2 pa pb complex entries
    RS_TRY(ensure_gram_partials(ctx, (size_t)nsplit * 2 * pa * pb));
    double *part = reinterpret_cast<double *>(ctx->ws.gram_part);
    {
        const double entries = sym ? 0.5 * na * (na + 1.0) : (double)na * nb;
        ProfScope ps(ctx, RSDFT_K_GRAM, 2.0 * (double)n * entries,
                     (double)n * sizeof(double2) * (sym ? pa : pa + pb), st);
        k_gram_pair<P><<<dim3(tiles, nsplit), GR_THREADS, 0, st>>>(A, B, pa, pb, n, sym ? 1 : 0, Ti, Tj, kchunk,
                                                                     part);
    }
    RS_LAUNCHED(ctx, "k_gram_pair");
    const long long tot = (long long)na * nb;
    k_gram_pair_reduce<<<cdiv(tot, 256), 256, 0, st>>>(part, nsplit, pa, pb, A.cnt[0], A.cnt[1], B.cnt[0], B.cnt[1],
                                                       na, nb, sym ? 1 : 0, TE, scale, g, ldg);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_gram_pair_reduce");
    return RSDFT_OK;
}

}  // namespace

// g[i][j] = (scale <a_i|b_j>, 0) over the real bands of pair-row blocks A (na =
// sum of its counts) and B; sym: A and B have the same counts and G is
// symmetric (G_S = <Y|Y>, or G_H = <Y|HY> with H symmetric), so only tiles on
// and above the diagonal are formed.  ldg: leading dimension of g.
rsdft_status gram_pair(rsdft_ctx *ctx, const RowBlocks &A, const RowBlocks &B, double2 *g, int ldg, bool sym,
                       double scale, cudaStream_t st) {
    const int na = A.cnt[0] + A.cnt[1] + A.cnt[2];
    const int nb = B.cnt[0] + B.cnt[1] + B.cnt[2];
    if (na <= 0 || nb <= 0) return RSDFT_OK;
    if (sym && na != nb) return fail(ctx, RSDFT_E_INVALID, "symmetric gram needs na == nb");
    // Tile edge 16, 32 or 64 pair rows, the one that computes the fewest pair
    // products (padding, and for sym the full diagonal tiles); ties: the larger.
    // The kernel is bound by the FP64 pipe alone, so the smaller tiles' extra
    // shared-memory loads cost nothing.
    const int pa = pairs_of(A.cnt[0]) + pairs_of(A.cnt[1]) + pairs_of(A.cnt[2]);
    const int pb = pairs_of(B.cnt[0]) + pairs_of(B.cnt[1]) + pairs_of(B.cnt[2]);
    auto work = [&](long long te) {
        const long long ti = (pa + te - 1) / te, tj = (pb + te - 1) / te;
        return (sym ? ti * (ti + 1) / 2 : ti * tj) * te * te;
    };
    const long long w1 = work(16), w2 = work(32), w4 = work(64);
    if (w4 <= w2 && w4 <= w1) return gram_pair_launch<4>(ctx, A, B, na, nb, g, ldg, sym, scale, st);
    if (w2 <= w1) return gram_pair_launch<2>(ctx, A, B, na, nb, g, ldg, sym, scale, st);
    return gram_pair_launch<1>(ctx, A, B, na, nb, g, ldg, sym, scale, st);
}

// ---- Ritz rotation on pair rows ---------------------------------------------------------
// out0[b] = base[b] + sign sum_i Re c[i][b] y_i over the real bands y_i of the
// pair-row blocks of Y, for m output bands (pairs_of(m) pair rows; the .y half
// of the last row is base's, or 0, when m is odd).  Blocks are consumed in the
// order 1, 2, 0 so that out1 (optional) = the block 1-2 part alone.  Tile: 16 PB
// output pair rows x 64 points; thread (ty, tx) owns pair rows ty + 16 p and
// points tx + 16 q.
template <int PB>
__global__ void __launch_bounds__(GR_THREADS)
k_rotate_pair(RowBlocks Y, const double2 *__restrict__ c, int ldc, int m, long long n, const double2 *base, int sign,
              double2 *out0, double2 *out1) {
    constexpr int TB = 16 * PB;
    __shared__ double2 Ys[GRK][GRPTS + 1];
    __shared__ double2 Ca[GRK][TB + 1];   // (c[2i][2b'], c[2i][2b'+1])   input band 2i -> output pair b'
    __shared__ double2 Cb[GRK][TB + 1];   // (c[2i+1][2b'], c[2i+1][2b'+1])
    const int b0 = blockIdx.x * TB;
    const long long r0 = (long long)blockIdx.y * GRPTS;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int mp = pairs_of(m);
    double ax[PB][4], ay[PB][4];
#pragma unroll
    for (int p = 0; p < PB; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) ax[p][q] = ay[p][q] = 0.0;
#pragma unroll 1
    for (int oi = 0; oi < 3; ++oi) {
        // blocks in the order 1, 2, 0 (selects, not a run-time index into the
        // parameter arrays, which would go through local memory)
        const int cnt = oi == 0 ? Y.cnt[1] : (oi == 1 ? Y.cnt[2] : Y.cnt[0]);
        const double2 *yb = oi == 0 ? Y.ptr[1] : (oi == 1 ? Y.ptr[2] : Y.ptr[0]);
        const int crow0 = oi == 0 ? Y.cnt[0] : (oi == 1 ? Y.cnt[0] + Y.cnt[1] : 0);
        const int pc = pairs_of(cnt);
        for (int kb = 0; kb < pc; kb += GRK) {
            for (int idx = threadIdx.x; idx < GRK * GRPTS; idx += GR_THREADS) {
                const int kk = idx / GRPTS, cc = idx % GRPTS;
                const int i = kb + kk;
                double2 yv = make_double2(0.0, 0.0);
                if (i < pc && r0 + cc < n) yv = yb[(size_t)i * n + r0 + cc];
                Ys[kk][cc] = yv;
            }
            for (int idx = threadIdx.x; idx < GRK * TB; idx += GR_THREADS) {
                const int kk = idx / TB, cc = idx % TB;
                const int ra = 2 * (kb + kk), rb = ra + 1;       // input bands within the block
                const int oa = 2 * (b0 + cc), ob = oa + 1;       // output bands
                double2 va = make_double2(0.0, 0.0), vb = make_double2(0.0, 0.0);
                if (ra < cnt) {
                    const double2 *cr = c + (size_t)(crow0 + ra) * ldc;
                    if (oa < m) va.x = cr[oa].x;
                    if (ob < m) va.y = cr[ob].x;
                }
                if (rb < cnt) {
                    const double2 *cr = c + (size_t)(crow0 + rb) * ldc;
                    if (oa < m) vb.x = cr[oa].x;
                    if (ob < m) vb.y = cr[ob].x;
                }
                Ca[kk][cc] = va;
                Cb[kk][cc] = vb;
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < GRK; ++k) {
                double2 ca[PB], cb[PB], yv[4];
#pragma unroll
                for (int p = 0; p < PB; ++p) {
                    ca[p] = Ca[k][ty + 16 * p];
                    cb[p] = Cb[k][ty + 16 * p];
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) yv[q] = Ys[k][tx + 16 * q];
#pragma unroll
                for (int p = 0; p < PB; ++p)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        ax[p][q] = fma(yv[q].x, ca[p].x, fma(yv[q].y, cb[p].x, ax[p][q]));
                        ay[p][q] = fma(yv[q].x, ca[p].y, fma(yv[q].y, cb[p].y, ay[p][q]));
                    }
            }
            __syncthreads();
        }
        if (oi == 1 && out1) {
#pragma unroll
            for (int p = 0; p < PB; ++p) {
                const int bp = b0 + ty + 16 * p;
                if (bp >= mp) continue;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const long long r = r0 + tx + 16 * q;
                    if (r < n) out1[(size_t)bp * n + r] = make_double2(ax[p][q], ay[p][q]);
                }
            }
        }
    }
    const double sg = (double)sign;
#pragma unroll
    for (int p = 0; p < PB; ++p) {
        const int bp = b0 + ty + 16 * p;
        if (bp >= mp) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const long long r = r0 + tx + 16 * q;
            if (r >= n) continue;
            double ox = sg * ax[p][q], oy = sg * ay[p][q];
            if (base) {
                const double2 bv = base[(size_t)bp * n + r];
                ox += bv.x;
                oy += bv.y;
            }
            out0[(size_t)bp * n + r] = make_double2(ox, oy);
        }
    }
}

rsdft_status rotate_pair(rsdft_ctx *ctx, const RowBlocks &Y, const double2 *c, int ldc, int m, const double2 *base,
                         int sign, double2 *out0, double2 *out1, cudaStream_t st) {
    if (m <= 0) return RSDFT_OK;
    const int k = Y.cnt[0] + Y.cnt[1] + Y.cnt[2];
    const int kp = pairs_of(Y.cnt[0]) + pairs_of(Y.cnt[1]) + pairs_of(Y.cnt[2]);
    const int mp = pairs_of(m);
    ProfScope ps(ctx, RSDFT_K_ROTATE, 2.0 * (double)ctx->n * k * m,
                 (double)sizeof(double2) * (double)ctx->n * (kp + mp + (out1 ? mp : 0) + (base ? mp : 0)), st);
    // output tile of 16 or 32 pair rows, the one with less padding (ties: 32)
    if (cdiv(mp, 16) * 16 < cdiv(mp, 32) * 32)
        k_rotate_pair<1><<<dim3(cdiv(mp, 16), cdiv(ctx->n, GRPTS)), GR_THREADS, 0, st>>>(Y, c, ldc, m, ctx->n, base,
                                                                                        sign, out0, out1);
    else
        k_rotate_pair<2><<<dim3(cdiv(mp, 32), cdiv(ctx->n, GRPTS)), GR_THREADS, 0, st>>>(Y, c, ldc, m, ctx->n, base,
                                                                                        sign, out0, out1);
    RS_LAUNCHED(ctx, "k_rotate_pair");
    return RSDFT_OK;
}

// ---- per-band wrappers --------------------------------------------------------------------
static rsdft_status resid_pairs(rsdft_ctx *ctx, const double2 *hx, const double2 *x, int m, cudaStream_t st) {
    Workspace &w = ctx->ws;
    const int mp = pairs_of(m);
    const int S = slices_for(ctx, mp);
    // 2 S mp complex entries; the Gram partial buffer (free between Gram calls)
    // holds at least 32 (3 m)^2
    double2 *part = w.gram_part;
    k_resid_pair_part<<<dim3(S, mp), GR_THREADS, 0, st>>>(hx, x, w.theta, ctx->v, m, ctx->n, S, part);
    k_resid_pair_fin<<<cdiv(m, 128), 128, 0, st>>>(part, S, m, ctx->dV, w.res, w.vexp);
    count_launch(ctx, 2);
    RS_LAUNCHED(ctx, "k_resid_pair");
    return RSDFT_OK;
}

static rsdft_status norms_pairs(rsdft_ctx *ctx, const double2 *a, int cnt, double *out, cudaStream_t st) {
    if (cnt <= 0) return RSDFT_OK;
    const int mp = pairs_of(cnt);
    const int S = slices_for(ctx, mp);
    double2 *part = ctx->ws.gram_part;
    k_rownorm_pair_part<<<dim3(S, mp), GR_THREADS, 0, st>>>(a, ctx->n, S, part);
    k_rownorm_pair_fin<<<cdiv(cnt, 128), 128, 0, st>>>(part, S, cnt, ctx->dV, out);
    count_launch(ctx, 2);
    RS_LAUNCHED(ctx, "k_rownorm_pair");
    return RSDFT_OK;
}

static rsdft_status pack(rsdft_ctx *ctx, const double *x, int m, double2 *out, cudaStream_t st) {
    if (m <= 0) return RSDFT_OK;
    k_pack_pairs<<<row_grid(ctx->n, pairs_of(m)), 256, 0, st>>>(x, m, ctx->n, out);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_pack_pairs");
    return RSDFT_OK;
}

static rsdft_status unpack(rsdft_ctx *ctx, const double2 *in, int m, double *x, cudaStream_t st) {
    if (m <= 0) return RSDFT_OK;
    k_unpack_pairs<<<row_grid(ctx->n, pairs_of(m)), 256, 0, st>>>(in, m, ctx->n, x);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_unpack_pairs");
    return RSDFT_OK;
}

// ---- the iteration ------------------------------------------------------------------------
// One FP64 LOBPCG run on the pair rows in the workspace (X holds the start
// block).  The steps, stopping rule, soft locking, pivot floor and restart
// guard are those of the complex FP64 iteration (lobpcg.cu).
static rsdft_status lobpcg_pairs(rsdft_ctx *ctx, int m, const rsdft_lobpcg_opts &o, int *iters, int *dropped,
                                 bool *converged, double *hres, cudaStream_t st) {
    Workspace &w = ctx->ws;
    const long long n = ctx->n;
    const double dV = ctx->dV;
    const int nconv = (o.nconv <= 0 || o.nconv > m) ? m : o.nconv;
    const bool df = o.dense == RSDFT_DENSE_DF;
    const int mp = pairs_of(m);
    double2 *X = w.X, *HX = w.HX, *Xn = w.Xn, *HXn = w.HXn, *W = w.W, *HW = w.HW, *P = w.P, *HP = w.HP;
    double2 *Pn = w.Pn, *HPn = w.HPn, *T1 = w.T1;
    int *hact = reinterpret_cast<int *>(w.hbuf + m);
    RS_TRY(apply_h64(ctx, X, HX, mp, st));
    {
        RowBlocks Y{{X, nullptr, nullptr}, {m, 0, 0}};
        RowBlocks HY{{HX, nullptr, nullptr}, {m, 0, 0}};
        RS_TRY(gram_pair(ctx, Y, Y, w.GS, m, true, dV, st));
        RS_TRY(gram_pair(ctx, Y, HY, w.GH, m, true, dV, st));
        int nd = 0;
        RS_TRY(rayleigh_ritz(ctx, w.GH, w.GS, m, m, o.pivot_tol, w.theta, w.Cfull, &nd, st, df));
        RS_TRY(rotate_pair(ctx, Y, w.Cfull, m, m, nullptr, 1, Xn, nullptr, st));
        RS_TRY(rotate_pair(ctx, HY, w.Cfull, m, m, nullptr, 1, HXn, nullptr, st));
        std::swap(X, Xn);
        std::swap(HX, HXn);
    }
    bool haveP = false;
    int it = 0;
    double best = -1.0;
    rsdft_status result = RSDFT_OK;
    *converged = false;
    for (;;) {
        RS_TRY(resid_pairs(ctx, HX, X, m, st));
        RS_CUDA(ctx, cudaMemcpyAsync(hres, w.res, m * sizeof(double), cudaMemcpyDeviceToHost, st));
        RS_CUDA(ctx, cudaStreamSynchronize(st));
        double rmax = 0.0;
        bool bad = false;
        for (int b = 0; b < m; ++b) {
            if (!std::isfinite(hres[b])) bad = true;
            if (b < nconv) rmax = std::max(rmax, hres[b]);
        }
        if (bad) { result = fail(ctx, RSDFT_E_NUMERIC, "non-finite residual at iteration %d", it); break; }
        *converged = rmax <= o.tol;
        if (*converged || it >= o.maxit) break;
        // restart without P when, below 1e-6, the max residual rises above
        // twice its best (the complex FP64 iteration's guard)
        if (haveP && best > 0.0 && best < 1e-6 && rmax > 2.0 * best) haveP = false;
        best = best > 0.0 ? std::min(best, rmax) : rmax;
        int na = 0;
        for (int b = 0; b < m; ++b)
            if (hres[b] > o.lock_tol) hact[na++] = b;
        if (na == 0) break;
        RS_CUDA(ctx, cudaMemcpyAsync(w.act, hact, na * sizeof(int), cudaMemcpyHostToDevice, st));
        const int nap = pairs_of(na);
        // ---- W = TPA(R) (or R), as pair rows
        if (o.precond == RSDFT_PRECOND_TPA) {
            RS_TRY(project(ctx, X, w.proj, mp, st));
            k_tkin_pair<<<cdiv(na, 128), 128, 0, st>>>(w.theta, w.vexp, w.proj, ctx->pt, w.act, na, w.tkin);
            k_resid_rows_cplx<<<row_grid(n, na), 256, 0, st>>>(HX, X, w.theta, w.act, n, HW);
            count_launch(ctx, 2);
            RS_LAUNCHED(ctx, "k_tkin_pair");
            RS_TRY(fft_xy_forward(ctx, Src::Plain, HW, nullptr, nullptr, nullptr, nullptr, T1, na, st));
            RS_TRY(fft_z_mid(ctx, Mid::Tpa, T1, w.tkin, na, st));
            RS_TRY(fft_xy_inverse(ctx, T1, nullptr, nullptr, HW, nullptr, na, st));
            k_real_to_pairs<<<row_grid(n, nap), 256, 0, st>>>(HW, na, n, W);
            count_launch(ctx);
            RS_LAUNCHED(ctx, "k_real_to_pairs");
        } else {
            k_resid_rows_pair<<<row_grid(n, nap), 256, 0, st>>>(HX, X, w.theta, w.act, na, n, W);
            count_launch(ctx);
            RS_LAUNCHED(ctx, "k_resid_rows_pair");
        }
        // ---- W <- W - X <X|W>
        {
            RowBlocks YX{{X, nullptr, nullptr}, {m, 0, 0}};
            RowBlocks YW{{W, nullptr, nullptr}, {na, 0, 0}};
            RS_TRY(gram_pair(ctx, YX, YW, w.C, na, false, dV, st));
            RS_TRY(rotate_pair(ctx, YX, w.C, na, na, W, -1, W, nullptr, st));
        }
        RS_TRY(apply_h64(ctx, W, HW, nap, st));
        RS_TRY(norms_pairs(ctx, W, na, w.nrm, st));
        k_scale_pairs<<<row_grid(n, nap), 256, 0, st>>>(W, HW, na, n, w.nrm);
        count_launch(ctx);
        RS_LAUNCHED(ctx, "k_scale_pairs");
        int np_ = 0;
        if (haveP) {
            np_ = na;   // every active band keeps its P column (FP64)
            k_gather_pairs<<<row_grid(n, nap), 256, 0, st>>>(P, HP, w.act, np_, n, Pn, HPn);
            count_launch(ctx);
            RS_LAUNCHED(ctx, "k_gather_pairs");
            RS_TRY(norms_pairs(ctx, Pn, np_, w.nrm, st));
            k_scale_pairs<<<row_grid(n, nap), 256, 0, st>>>(Pn, HPn, np_, n, w.nrm);
            count_launch(ctx);
            RS_LAUNCHED(ctx, "k_scale_pairs");
        }
        const int k = m + na + np_;
        RowBlocks Y{{X, W, Pn}, {m, na, np_}};
        RowBlocks HY{{HX, HW, HPn}, {m, na, np_}};
        RS_TRY(gram_pair(ctx, Y, Y, w.GS, k, true, dV, st));
        RS_TRY(gram_pair(ctx, Y, HY, w.GH, k, true, dV, st));
        int nd = 0;
        RS_TRY(rayleigh_ritz(ctx, w.GH, w.GS, k, m, o.pivot_tol, w.lam, w.Cfull, &nd, st, df));
        *dropped += nd;
        RS_TRY(rotate_pair(ctx, Y, w.Cfull, m, m, nullptr, 1, Xn, P, st));
        RS_TRY(rotate_pair(ctx, HY, w.Cfull, m, m, nullptr, 1, HXn, HP, st));
        RS_CUDA(ctx, cudaMemcpyAsync(w.theta, w.lam, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
        std::swap(X, Xn);
        std::swap(HX, HXn);
        haveP = true;
        ++it;
    }
    *iters = it;
    // the result stays in X (the workspace pointers follow the swaps)
    w.X = X; w.Xn = Xn; w.HX = HX; w.HXn = HXn;
    return result;
}

}  // namespace rsdft

using namespace rsdft;

extern "C" {

rsdft_status rsdft_apply_h_real(rsdft_ctx *ctx, const void *x_dev, void *hx_dev, int nband, void *stream) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (nband < 0 || (nband > 0 && (!x_dev || !hx_dev))) return fail(ctx, RSDFT_E_INVALID, "bad apply_h_real arguments");
    if (nband == 0) return RSDFT_OK;
    cudaStream_t st = as_stream(stream);
    RS_TRY(ensure_workspace(ctx, pairs_of(nband)));
    Workspace &w = ctx->ws;
    RS_TRY(pack(ctx, (const double *)x_dev, nband, w.X, st));
    RS_TRY(apply_h64(ctx, w.X, w.HX, pairs_of(nband), st));
    return unpack(ctx, w.HX, nband, (double *)hx_dev, st);
}

rsdft_status rsdft_gram_real(rsdft_ctx *ctx, const void *a_dev, int na, const void *b_dev, int nb, void *g_dev,
                             void *stream) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (na < 0 || nb < 0 || ((na > 0 && nb > 0) && (!a_dev || !b_dev || !g_dev)))
        return fail(ctx, RSDFT_E_INVALID, "bad gram_real arguments");
    if (na == 0 || nb == 0) return RSDFT_OK;
    cudaStream_t st = as_stream(stream);
    // the workspace's k x k subspace matrices hold the na x nb result
    RS_TRY(ensure_workspace(ctx, std::max(cdiv(std::max(na, nb), 3), pairs_of(std::max(na, nb)))));
    Workspace &w = ctx->ws;
    const bool sym = a_dev == b_dev && na == nb;
    RS_TRY(pack(ctx, (const double *)a_dev, na, w.X, st));
    if (!sym) RS_TRY(pack(ctx, (const double *)b_dev, nb, w.W, st));
    RowBlocks A{{w.X, nullptr, nullptr}, {na, 0, 0}};
    RowBlocks B{{sym ? w.X : w.W, nullptr, nullptr}, {nb, 0, 0}};
    RS_TRY(gram_pair(ctx, A, B, w.C, nb, sym, ctx->dV, st));
    // the real parts out, as a [na][nb] real matrix
    RS_CUDA(ctx, cudaMemcpy2DAsync(g_dev, sizeof(double), w.C, sizeof(double2), sizeof(double), (size_t)na * nb,
                                   cudaMemcpyDeviceToDevice, st));
    return RSDFT_OK;
}

rsdft_status rsdft_rotate_real(rsdft_ctx *ctx, const void *y_dev, int k, const void *c_dev, int m,
                               const void *base_dev, int sign, void *out_dev, void *stream) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (k < 0 || m < 0 || (m > 0 && (!out_dev || (k > 0 && (!y_dev || !c_dev)))) || (sign != 1 && sign != -1))
        return fail(ctx, RSDFT_E_INVALID, "bad rotate_real arguments");
    if (m == 0) return RSDFT_OK;
    cudaStream_t st = as_stream(stream);
    RS_TRY(ensure_workspace(ctx, std::max(cdiv(std::max(k, m), 3), pairs_of(std::max(k, m)))));
    Workspace &w = ctx->ws;
    if (k > 0) {
        RS_TRY(pack(ctx, (const double *)y_dev, k, w.X, st));
        // c (real [k][m]) into the .x parts of a complex [k][m] matrix
        RS_CUDA(ctx, cudaMemsetAsync(w.Cfull, 0, (size_t)k * m * sizeof(double2), st));
        RS_CUDA(ctx, cudaMemcpy2DAsync(w.Cfull, sizeof(double2), c_dev, sizeof(double), sizeof(double), (size_t)k * m,
                                       cudaMemcpyDeviceToDevice, st));
    }
    if (base_dev) RS_TRY(pack(ctx, (const double *)base_dev, m, w.W, st));
    RowBlocks Y{{w.X, nullptr, nullptr}, {k, 0, 0}};
    RS_TRY(rotate_pair(ctx, Y, w.Cfull, m, m, base_dev ? w.W : nullptr, sign, w.Xn, nullptr, st));
    return unpack(ctx, w.Xn, m, (double *)out_dev, st);
}

rsdft_status rsdft_lobpcg_real(rsdft_ctx *ctx, void *x_dev, int nband, const rsdft_lobpcg_opts *opts,
                               double *eig_host, double *resnorm_host, rsdft_lobpcg_stats *stats, void *stream) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (!x_dev || nband <= 0 || 3LL * nband > ctx->n)
        return fail(ctx, RSDFT_E_INVALID, "need x and 0 < nband <= n/3");
    rsdft_lobpcg_opts o;
    rsdft_lobpcg_default_opts(&o);
    if (opts) o = *opts;
    if (o.maxit < 0 || !(o.tol >= 0.0) || !(o.pivot_tol >= 0.0) || !(o.lock_tol >= 0.0))
        return fail(ctx, RSDFT_E_INVALID, "bad LOBPCG options");
    if (o.precision != RSDFT_FP64)
        return fail(ctx, RSDFT_E_INVALID, "the real Gamma-point form runs in FP64 only");
    if (o.precond != RSDFT_PRECOND_TPA && o.precond != RSDFT_PRECOND_NONE)
        return fail(ctx, RSDFT_E_INVALID, "the real Gamma-point form takes the TPA or no preconditioner");
    if (o.dense != RSDFT_DENSE_AUTO && o.dense != RSDFT_DENSE_FP64 && o.dense != RSDFT_DENSE_DF)
        return fail(ctx, RSDFT_E_INVALID, "unknown dense mode");
    if (stats) *stats = rsdft_lobpcg_stats{};
    cudaStream_t st = as_stream(stream);
    // the orbital buffers hold nband complex rows, twice what the pair rows
    // need; the subspace buffers are sized for k <= 3 nband real columns
    RS_TRY(ensure_workspace(ctx, nband));
    Workspace &w = ctx->ws;
    const long long fallbacks0 = ctx->coop_fallbacks;
    RS_TRY(pack(ctx, (const double *)x_dev, nband, w.X, st));
    int iters = 0, dropped = 0;
    bool converged = false;
    double *hres = w.hbuf;
    const rsdft_status r = lobpcg_pairs(ctx, nband, o, &iters, &dropped, &converged, hres, st);
    if (r == RSDFT_OK) RS_TRY(unpack(ctx, w.X, nband, (double *)x_dev, st));
    if (stats) {
        stats->iterations = iters;
        stats->converged = converged ? 1 : 0;
        stats->dropped = dropped;
        stats->coop_fallbacks = (int)(ctx->coop_fallbacks - fallbacks0);
        stats->coop_last_error = stats->coop_fallbacks ? ctx->coop_last_error : 0;
    }
    if (eig_host) RS_CUDA(ctx, cudaMemcpyAsync(eig_host, w.theta, nband * sizeof(double), cudaMemcpyDeviceToHost, st));
    RS_CUDA(ctx, cudaStreamSynchronize(st));
    if (resnorm_host) memcpy(resnorm_host, hres, nband * sizeof(double));
    if (r != RSDFT_OK) return r;
    return converged || o.tol <= 0.0 ? RSDFT_OK : RSDFT_E_NOT_CONVERGED;
}

}  // extern "C"
