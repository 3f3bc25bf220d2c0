// Tensor-core Gram matrices for the mixed form (SCF task (2)): split-BF16
// products on the 5th-generation tensor cores (tcgen05, FP32 accumulation in
// TMEM), operands staged by TMA into 128-byte-swizzled shared memory.
//
// Complex to real: with each orbital row stored as interleaved reals
// (re0, im0, re1, im1, ...) of length K = 2n,
//   Re <a|b> = sum_k a[k] b[k],   Im <a|b> = sum_k a[k] brot[k],
//   brot = (im0, -re0, im1, -re1, ...).
// Each FP32 value x is split x = hi + lo, hi = bf16(x), lo = bf16(x - hi); the
// product uses hi*hi' + hi*lo' + lo*hi' (the lo*lo' term is below FP32
// rounding).  One launch forms C = A B^T for A = [rows of Y] and B = the stacked
// operand rows ([Y; Yrot] for G_S, [HY; HYrot] for G_H), split over K; the FP32
// partial tiles are reduced in FP64 and assembled into complex G.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>

#include "rsdft_internal.h"

namespace rsdft {
namespace tc {

constexpr int BM = 128;             // tile rows (A)
constexpr int BN = 128;             // tile cols (B rows)
constexpr int BK = 64;              // bf16 elements per 128-byte swizzled row
constexpr int STAGES = 3;
constexpr int TILE_BYTES = BM * BK * 2;                 // 16 KB per operand tile
constexpr int STAGE_BYTES = 4 * TILE_BYTES;             // A_hi, A_lo, B_hi, B_lo
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024; // + alignment slack
constexpr int THREADS = 128;
constexpr long long WAIT_LIMIT = 4000000000LL;          // SM cycles (~2 s) per wait

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait on an mbarrier phase; false on timeout or when *abort is set.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > WAIT_LIMIT) {
            *abort = 1;
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x,
                                            int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups of
// 1024 bytes (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(const void *p) {
    const uint64_t addr = (smem_u32(p) & 0x3FFFFu) >> 4;
    uint64_t d = addr;                      // start address  [0, 14)
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset [32, 46)
    d |= (uint64_t)1 << 46;                 // version
    d |= (uint64_t)2 << 61;                 // layout: 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: BF16 x BF16 -> FP32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4)                        // accumulator F32
           | (1u << 7)                      // A: BF16
           | (1u << 10)                     // B: BF16
           | ((uint32_t)(n >> 3) << 17)     // N / 8
           | ((uint32_t)(m >> 4) << 24);    // M / 16
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}


// Split FP32 complex rows into BF16 hi/lo rows of interleaved reals.
// rot = 1 stores (im, -re) pairs.  dst rows dst_row0 + r, leading dimension ldk
// (>= 2n, multiple of 8); the columns 2n..ldk-1 are zeroed.
__global__ void k_split_bf16(RowBlocksT<float2> src, int nrows, long long n, int ldk, int rot,
                             __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ lo,
                             int dst_row0) {
    const int r = blockIdx.y;
    if (r >= nrows) return;
    int i = r, blk = 0;
    while (blk < 2 && i >= src.cnt[blk]) { i -= src.cnt[blk]; ++blk; }
    const float2 *row = src.ptr[blk] + (size_t)i * n;
    __nv_bfloat162 *h2 = reinterpret_cast<__nv_bfloat162 *>(hi + (size_t)(dst_row0 + r) * ldk);
    __nv_bfloat162 *l2 = reinterpret_cast<__nv_bfloat162 *>(lo + (size_t)(dst_row0 + r) * ldk);
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const float2 v = row[p];
        const float x0 = rot ? v.y : v.x, x1 = rot ? -v.x : v.y;
        const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
        const __nv_bfloat16 g0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
        const __nv_bfloat16 g1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
        h2[p] = __halves2bfloat162(h0, h1);
        l2[p] = __halves2bfloat162(g0, g1);
    }
    if (blockIdx.x == 0 && threadIdx.x < ldk - 2 * n) {
        const size_t c = (size_t)(dst_row0 + r) * ldk + 2 * n + threadIdx.x;
        hi[c] = __float2bfloat16_rn(0.0f);
        lo[c] = __float2bfloat16_rn(0.0f);
    }
}

// part[split][M][N] (FP32) = the split's K range of A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T.
// Grid (N tiles, M tiles, splits), 128 threads, one 128 x 128 FP32 accumulator
// in TMEM.  Warp 0 lane 0 issues TMA, warp 1 lane 0 issues MMAs, all four
// warps read the accumulator (warp w owns TMEM lanes 32w..32w+31).
__global__ void __launch_bounds__(THREADS, 1)
k_gram_tc(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
          const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl, int M,
          int N, int kb_total, int kb_per_split, int tpb, int blk_rows, float *__restrict__ part, int *err) {
    // tpb > 0: B is a stack of N / blk_rows blocks of blk_rows rows, each Hermitian
    // against A; blockIdx.x = block * tpb + tile within the block, and tiles below
    // the diagonal (tile < tm) are skipped (the reduction mirrors them).
    int brow0, ncol0, nvalid;
    if (tpb > 0) {
        const int blk = blockIdx.x / tpb, tnb = blockIdx.x - blk * tpb;
        if (tnb < (int)blockIdx.y) return;
        brow0 = blk * blk_rows + tnb * BN;
        ncol0 = brow0;
        nvalid = blk_rows - tnb * BN;
    } else {
        brow0 = ncol0 = blockIdx.x * BN;
        nvalid = N - ncol0;
    }
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[STAGES];
    __shared__ __align__(8) uint64_t empty_bar[STAGES];
    __shared__ __align__(8) uint64_t acc_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    const int tm = blockIdx.y, split = blockIdx.z;
    const int kb0 = split * kb_per_split;
    const int nkb = max(0, min(kb_total, kb0 + kb_per_split) - kb0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&acc_bar, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&tmem_base, BN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    volatile int *abort = &s_abort;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer
        int issued = 0;
        for (int it = 0; it < nkb; ++it) {
            const int s = it % STAGES, r = it / STAGES;
            if (r > 0 && !mbar_wait(&empty_bar[s], (r - 1) & 1, abort)) break;
            unsigned char *st = smem + s * STAGE_BYTES;
            mbar_expect_tx(&full_bar[s], STAGE_BYTES);
            const int kx = (kb0 + it) * BK;
            tma_load_2d(st, &mAh, &full_bar[s], kx, tm * BM);
            tma_load_2d(st + TILE_BYTES, &mAl, &full_bar[s], kx, tm * BM);
            tma_load_2d(st + 2 * TILE_BYTES, &mBh, &full_bar[s], kx, brow0);
            tma_load_2d(st + 3 * TILE_BYTES, &mBl, &full_bar[s], kx, brow0);
            issued = it + 1;
        }
        if (*abort) {
            // let the copies still in flight land before the CTA leaves
            for (int it = max(0, issued - STAGES); it < issued; ++it) {
                const long long t0 = clock64();
                while (!mbar_try_wait(&full_bar[it % STAGES], (it / STAGES) & 1) &&
                       clock64() - t0 < WAIT_LIMIT) {
                }
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        const uint32_t idesc = idesc_bf16(BM, BN);
        for (int it = 0; it < nkb; ++it) {
            const int s = it % STAGES, r = it / STAGES;
            if (!mbar_wait(&full_bar[s], r & 1, abort)) break;
            tc_fence_after();
            unsigned char *st = smem + s * STAGE_BYTES;
            const uint64_t ah = smem_desc(st), al = smem_desc(st + TILE_BYTES);
            const uint64_t bh = smem_desc(st + 2 * TILE_BYTES), bl = smem_desc(st + 3 * TILE_BYTES);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
                const uint64_t off = (uint64_t)((kk * 32) >> 4);   // 16 bf16 = 32 bytes
                mma_bf16(tmem, ah + off, bh + off, idesc, (it | kk) != 0 ? 1u : 0u);
                mma_bf16(tmem, ah + off, bl + off, idesc, 1u);
                mma_bf16(tmem, al + off, bh + off, idesc, 1u);
            }
            mma_commit(&empty_bar[s]);
        }
        mma_commit(&acc_bar);   // arrives once every MMA issued above has completed
    }
    __syncwarp();
    // ---- epilogue: wait for the accumulator (time-bounded even after an abort,
    // since TMEM may only be released once the MMAs are done)
    bool ready = true;
    {
        const long long t0 = clock64();
        while (!mbar_try_wait(&acc_bar, 0)) {
            if (clock64() - t0 > WAIT_LIMIT) { *abort = 1; ready = false; break; }
        }
    }
    tc_fence_after();
    const bool write = ready && nkb > 0 && !*abort;
    const int row = tm * BM + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        if (write && row < M) {
            float *dst = part + ((size_t)split * M + row) * N + (size_t)ncol0 + c0;
            const int cmax = min(32, nvalid - c0);
#pragma unroll
            for (int i = 0; i < 32; ++i)
                if (i < cmax) dst[i] = v[i];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, BN);
    }
    if (threadIdx.x == 0 && *abort) atomicExch(err, 1);
}

// G_S and G_H of the LOBPCG basis from the split partials of
// C = A [Y; Yrot; HY; HYrot]^T (N = 4k, upper 128-tiles of each block computed):
// scaled by dV, FP64 sums; entries of tiles above the diagonal are taken as
// computed, below it as the conjugate of the mirrored entry, and on diagonal
// tiles the two are averaged (as the FP64 path does).
__global__ void k_gram_tc_reduce_sh(const float *__restrict__ part, int splits, int k, double scale,
                                    double2 *__restrict__ gs, double2 *__restrict__ gh, int ld) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)k * k) return;
    const int i = (int)(idx / k), j = (int)(idx % k);
    const size_t N = 4 * (size_t)k, plane = (size_t)k * N;
    auto sum4 = [&](int r, int c, double &sr, double &si, double &hr, double &hi) {
        sr = si = hr = hi = 0.0;
        for (int s = 0; s < splits; ++s) {
            const float *pr = part + s * plane + (size_t)r * N;
            sr += (double)pr[c];
            si += (double)pr[k + c];
            hr += (double)pr[2 * k + c];
            hi += (double)pr[3 * k + c];
        }
    };
    const int ti = i / BM, tj = j / BN;
    double sr, si, hr, hi;
    if (ti < tj) {
        sum4(i, j, sr, si, hr, hi);
    } else if (ti > tj) {
        sum4(j, i, sr, si, hr, hi);
        si = -si;
        hi = -hi;
    } else {
        double sr2, si2, hr2, hi2;
        sum4(i, j, sr, si, hr, hi);
        sum4(j, i, sr2, si2, hr2, hi2);
        sr = 0.5 * (sr + sr2);
        si = 0.5 * (si - si2);
        hr = 0.5 * (hr + hr2);
        hi = 0.5 * (hi - hi2);
    }
    gs[(size_t)i * ld + j] = make_double2(scale * sr, scale * si);
    gh[(size_t)i * ld + j] = make_double2(scale * hr, scale * hi);
}

// General G = A^H B from the partials of C = A [B; Brot]^T (N = 2 nb).
__global__ void k_gram_tc_reduce(const float *__restrict__ part, int splits, int na, int nb,
                                 double scale, double2 *__restrict__ g, int ld) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)na * nb) return;
    const int i = (int)(idx / nb), j = (int)(idx % nb);
    const size_t N = 2 * (size_t)nb, plane = (size_t)na * N;
    double re = 0, im = 0;
    for (int s = 0; s < splits; ++s) {
        re += (double)part[s * plane + (size_t)i * N + j];
        im += (double)part[s * plane + (size_t)i * N + nb + j];
    }
    g[(size_t)i * ld + j] = make_double2(scale * re, scale * im);
}


// ---- Ritz rotation: out[b][:] = sum_j C[j][b] Y[j][:] ------------------------------
// As a real GEMM D[p][q] = sum_j A[p][j] B[j][q] with p the interleaved real index
// of a grid point (M, 2n), j the row of Y (K) and q in [0, 2 nh) (N): the first nh
// columns of B hold Re C[j][b], the next nh Im C[j][b].  Then for the pair of rows
// (re, im) of one point, out_re = D[re][b] - D[im][nh + b] and
// out_im = D[im][b] + D[re][nh + b]; the epilogue forms them with one shuffle.
// A is Y itself, read MN-major (the grid index is contiguous, K runs over rows);
// B is the small coefficient matrix, K-major.  Per 128-row tile the [W P] rows
// are accumulated first and written as the new P, then the X rows accumulate on
// top and the sum is written as the new X (= X C_X + P).
constexpr int RBK = 64;               // K rows (of Y) per pipeline stage
constexpr int RSTAGES = 2;
constexpr int RTHREADS = 320;         // warp 0 TMA, warp 1 MMA, warps 2..9 epilogue
constexpr int REPI = 8;               // epilogue warps (two per TMEM lane quarter)
constexpr int RA_CHUNK = 64 * RBK * 2;  // one 64-column chunk of A: 8 KB
constexpr int MAX_NH = 240;

__host__ __device__ constexpr int rot_stage_bytes(int nh) { return 4 * RA_CHUNK + 4 * nh * 128; }

// Shared-memory descriptor of an MN-major operand with 128-byte swizzle: 64
// contiguous MN elements per 128-byte row, 8 K-rows per 1024-byte group; lbo =
// byte distance between 64-element MN chunks, sbo = between 8-row K groups.
__device__ __forceinline__ uint64_t smem_desc_mn(const void *p, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (smem_u32(p) & 0x3FFFFu) >> 4;
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Split C (FP64 complex, rows j0..j0+nrows of [k][ldc], m columns) into the K-major
// bf16 hi/lo operand [2 nh][kpad]: row q < nh is Re C[j0 + t][q], row nh + q is
// Im C[j0 + t][q] at column t; zero outside (t >= nrows or q >= m).
__global__ void k_rot_coef(const double2 *__restrict__ c, int ldc, int j0, int nrows, int m, int nh,
                           int kpad, __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ lo) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 2LL * nh * kpad) return;
    const int row = (int)(idx / kpad), t = (int)(idx % kpad);
    const int q = row < nh ? row : row - nh;
    float v = 0.0f;
    if (t < nrows && q < m) {
        const double2 z = c[(size_t)(j0 + t) * ldc + q];
        v = (float)(row < nh ? z.x : z.y);
    }
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[idx] = h;
    lo[idx] = __float2bfloat16_rn(v - __bfloat162float(h));
}

__global__ void __launch_bounds__(RTHREADS, 1)
k_rot_tc(const __grid_constant__ CUtensorMap mWPh, const __grid_constant__ CUtensorMap mWPl,
         const __grid_constant__ CUtensorMap mXh, const __grid_constant__ CUtensorMap mXl,
         const __grid_constant__ CUtensorMap mBWPh, const __grid_constant__ CUtensorMap mBWPl,
         const __grid_constant__ CUtensorMap mBXh, const __grid_constant__ CUtensorMap mBXl, int nh,
         int m, int kb_wp, int kb_x, long long two_n, int ntiles, float *out0,
         float *__restrict__ out1, const float *base, float sign, int *err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[RSTAGES];
    __shared__ __align__(8) uint64_t empty_bar[RSTAGES];
    __shared__ __align__(8) uint64_t accf_bar;   // accumulator ready (MMA -> epilogue)
    __shared__ __align__(8) uint64_t acce_bar;   // accumulator drained (epilogue -> MMA)
    __shared__ __align__(8) uint64_t done_bar;   // every MMA issued has completed
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int stage_bytes = rot_stage_bytes(nh);
    const int bpart = nh * 128;               // one half (re or im) of B hi or lo
    if (threadIdx.x == 0) {
        for (int s = 0; s < RSTAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&accf_bar, 1);
        mbar_init(&acce_bar, REPI);
        mbar_init(&done_bar, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(&tmem_base, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    volatile int *abort = &s_abort;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer: k-blocks of ([W P] rows, then X rows) for each tile
        int it = 0;
        bool stop = false;
        for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
            const int m0 = t * 128;
            for (int ph = 0; ph < 2 && !stop; ++ph) {
                const int nkb = ph == 0 ? kb_wp : kb_x;
                const CUtensorMap *ah = ph == 0 ? &mWPh : &mXh, *al = ph == 0 ? &mWPl : &mXl;
                const CUtensorMap *bh = ph == 0 ? &mBWPh : &mBXh, *bl = ph == 0 ? &mBWPl : &mBXl;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = it % RSTAGES, r = it / RSTAGES;
                    if (r > 0 && !mbar_wait(&empty_bar[s], (r - 1) & 1, abort)) { stop = true; break; }
                    unsigned char *st = smem + s * stage_bytes;
                    mbar_expect_tx(&full_bar[s], stage_bytes);
                    const int y = kb * RBK;
                    tma_load_2d(st, ah, &full_bar[s], m0, y);
                    tma_load_2d(st + RA_CHUNK, ah, &full_bar[s], m0 + 64, y);
                    tma_load_2d(st + 2 * RA_CHUNK, al, &full_bar[s], m0, y);
                    tma_load_2d(st + 3 * RA_CHUNK, al, &full_bar[s], m0 + 64, y);
                    unsigned char *sb = st + 4 * RA_CHUNK;
                    tma_load_2d(sb, bh, &full_bar[s], y, 0);
                    tma_load_2d(sb + bpart, bh, &full_bar[s], y, nh);
                    tma_load_2d(sb + 2 * bpart, bl, &full_bar[s], y, 0);
                    tma_load_2d(sb + 3 * bpart, bl, &full_bar[s], y, nh);
                }
            }
        }
        if (*abort) {
            // let the copies still in flight land before the CTA leaves
            for (int j = max(0, it - RSTAGES); j < it; ++j) {
                const long long t0 = clock64();
                while (!mbar_try_wait(&full_bar[j % RSTAGES], (j / RSTAGES) & 1) && clock64() - t0 < WAIT_LIMIT) {
                }
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        const uint32_t idesc = idesc_bf16(128, nh) | (1u << 15);   // A MN-major
        int it = 0, ap = 0;
        bool stop = false;
        for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
            bool fresh = true;   // the tile's first MMA overwrites the accumulator
            for (int ph = 0; ph < 2 && !stop; ++ph) {
                const int nkb = ph == 0 ? kb_wp : kb_x;
                if (nkb == 0) continue;   // no [W P] rows: X phase only
                if (ap > 0 && !mbar_wait(&acce_bar, (ap - 1) & 1, abort)) { stop = true; break; }
                tc_fence_after();
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = it % RSTAGES, r = it / RSTAGES;
                    if (!mbar_wait(&full_bar[s], r & 1, abort)) { stop = true; break; }
                    tc_fence_after();
                    unsigned char *st = smem + s * stage_bytes;
                    unsigned char *sb = st + 4 * RA_CHUNK;
#pragma unroll
                    for (int kk = 0; kk < RBK / 16; ++kk) {
                        // A: 16 K-rows = two 8-row groups of 1024 B; B: 16 bf16 = 32 B
                        const uint64_t ah = smem_desc_mn(st + kk * 2048, RA_CHUNK, 1024);
                        const uint64_t al = smem_desc_mn(st + 2 * RA_CHUNK + kk * 2048, RA_CHUNK, 1024);
#pragma unroll
                        for (int half = 0; half < 2; ++half) {
                            const uint64_t bh = smem_desc(sb + half * bpart + kk * 32);
                            const uint64_t bl = smem_desc(sb + (2 + half) * bpart + kk * 32);
                            const uint32_t d = tmem + (uint32_t)(half * nh);
                            const uint32_t acc = fresh ? 0u : 1u;
                            mma_bf16(d, ah, bh, idesc, acc);
                            mma_bf16(d, ah, bl, idesc, 1u);
                            mma_bf16(d, al, bh, idesc, 1u);
                        }
                        fresh = false;
                    }
                    mma_commit(&empty_bar[s]);
                }
                if (stop) break;
                mma_commit(&accf_bar);
                ++ap;
            }
        }
        // every MMA issued so far must finish before TMEM is released (bounded)
        mma_commit(&done_bar);
        const long long t0 = clock64();
        while (!mbar_try_wait(&done_bar, 0)) {
            if (clock64() - t0 > WAIT_LIMIT) { *abort = 1; break; }
        }
    } else if (warp >= 2) {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31; the two warps of
        // a lane quarter take alternate 32-column chunks
        const int q = warp & 3, half = (warp - 2) >> 2;
        int ap = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const long long m0 = (long long)t * 128;
            for (int ph = 0; ph < 2; ++ph) {
                if ((ph == 0 ? kb_wp : kb_x) == 0) continue;
                if (!mbar_wait(&accf_bar, ap & 1, abort)) break;
                tc_fence_after();
                float *out = ph == 0 ? out1 : out0;
                const float *bse = ph == 0 ? nullptr : base;
                const long long p = m0 + q * 32 + lane;
                for (int b0 = half * 32; b0 < m; b0 += 64) {
                    float vr[32], vi[32], bv[32];
                    tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)b0, vr);
                    tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(nh + b0), vi);
                    if (bse) {
                        // all base loads of the chunk before any store (out may alias base)
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            bv[i] = (b0 + i < m && p < two_n) ? bse[(size_t)(b0 + i) * two_n + p] : 0.0f;
                    }
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        const float pv = __shfl_xor_sync(0xffffffffu, vi[i], 1);
                        const float v = (lane & 1) ? vr[i] + pv : vr[i] - pv;
                        if (out && b0 + i < m && p < two_n) {
                            const size_t o = (size_t)(b0 + i) * two_n + p;
                            out[o] = bse ? bv[i] + sign * v : v;
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acce_bar);
                ++ap;
            }
            if (*abort) break;
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
    if (threadIdx.x == 0 && *abort) atomicExch(err, 1);
}
}  // namespace tc
}  // namespace rsdft

namespace rsdft {
namespace tc {

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static rsdft_status encoder(rsdft_ctx *ctx) {
    if (g_encode) return RSDFT_OK;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return fail(ctx, RSDFT_E_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    }
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    return RSDFT_OK;
}

// 2D BF16 operand [rows][ldk] with kvalid valid columns; box 64 x box_rows,
// 128-byte swizzle (rows beyond `rows` and columns beyond kvalid read as zero).
static rsdft_status make_map(rsdft_ctx *ctx, CUtensorMap *m, const void *base, long long kvalid,
                             int rows, long long ldk, int box_rows = BM) {
    if ((reinterpret_cast<uintptr_t>(base) & 15u) || ((ldk * 2) & 15))
        return fail(ctx, RSDFT_E_INVALID, "tensor map base or stride not 16-byte aligned");
    cuuint64_t dims[2] = {(cuuint64_t)kvalid, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ldk * 2)};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims,
                          strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ctx, RSDFT_E_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return RSDFT_OK;
}

struct Buffers {
    __nv_bfloat16 *ah, *al, *bh, *bl;
    long long ldk;
};

// Operand storage for a rows x cols problem (bytes grow on demand).
static rsdft_status buffers(rsdft_ctx *ctx, int arows, int brows, Buffers &b) {
    Workspace &w = ctx->ws;
    const long long K = 2 * ctx->n;
    b.ldk = (K + 7) / 8 * 8;
    const size_t per = (size_t)b.ldk * sizeof(__nv_bfloat16);
    const size_t need = per * 2 * ((size_t)arows + brows) + 256;
    if (need > w.tc_bytes) {
        if (w.tcbuf) {
            cudaFree(w.tcbuf);
            for (auto &p : ctx->owned)
                if (p == w.tcbuf) p = nullptr;
        }
        w.tcbuf = nullptr;
        w.tc_bytes = 0;
        RS_TRY(dev_alloc(ctx, (void **)&w.tcbuf, need));
        w.tc_bytes = need;
    }
    unsigned char *base = reinterpret_cast<unsigned char *>(w.tcbuf);
    b.ah = reinterpret_cast<__nv_bfloat16 *>(base);
    b.al = b.ah + (size_t)arows * b.ldk;
    b.bh = b.al + (size_t)arows * b.ldk;
    b.bl = b.bh + (size_t)brows * b.ldk;
    return RSDFT_OK;
}

static rsdft_status partials(rsdft_ctx *ctx, size_t elems) {
    Workspace &w = ctx->ws;
    if (elems > w.tcpart_elems) {
        if (w.tcpart) {
            cudaFree(w.tcpart);
            for (auto &p : ctx->owned)
                if (p == w.tcpart) p = nullptr;
        }
        w.tcpart = nullptr;
        w.tcpart_elems = 0;
        RS_TRY(dev_alloc(ctx, (void **)&w.tcpart, elems * sizeof(float)));
        w.tcpart_elems = elems;
    }
    if (!w.tcerr) RS_TRY(dev_alloc(ctx, (void **)&w.tcerr, 64));
    return RSDFT_OK;
}

static rsdft_status split_rows(rsdft_ctx *ctx, const RowBlocksT<float2> &src, int rot, __nv_bfloat16 *hi,
                               __nv_bfloat16 *lo, int row0, long long ldk, cudaStream_t st) {
    const int rows = src.cnt[0] + src.cnt[1] + src.cnt[2];
    if (rows <= 0) return RSDFT_OK;
    dim3 g(std::max(1, std::min(cdiv(ctx->n, 256), 64)), rows);
    k_split_bf16<<<g, 256, 0, st>>>(src, rows, ctx->n, (int)ldk, rot, hi, lo, row0);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_split_bf16");
    return RSDFT_OK;
}

// C = A B^T over K = 2n for A rows [0, M), B rows [0, N) already split; returns
// splits.  blk_rows > 0: B is N / blk_rows blocks Hermitian against A (upper
// tiles of each block only).
static rsdft_status gemm(rsdft_ctx *ctx, const Buffers &b, int M, int N, cudaStream_t st, int *splits_out,
                         int blk_rows = 0) {
    RS_TRY(encoder(ctx));
    const long long K = 2 * ctx->n;
    CUtensorMap mAh, mAl, mBh, mBl;
    RS_TRY(make_map(ctx, &mAh, b.ah, K, M, b.ldk));
    RS_TRY(make_map(ctx, &mAl, b.al, K, M, b.ldk));
    RS_TRY(make_map(ctx, &mBh, b.bh, K, N, b.ldk));
    RS_TRY(make_map(ctx, &mBl, b.bl, K, N, b.ldk));
    const int tm = cdiv(M, BM);
    const int tpb = blk_rows > 0 ? cdiv(blk_rows, BN) : 0;
    const int tn = blk_rows > 0 ? (N / blk_rows) * tpb : cdiv(N, BN);
    // tiles that do work: all, or the upper ones of each Hermitian block
    const long long active = blk_rows > 0 ? (long long)(N / blk_rows) * tpb * (tpb + 1) / 2 : (long long)tn * tm;
    const int kb_total = (int)((K + BK - 1) / BK);
    // splits: whole waves of one CTA per SM, at least 8 k-blocks per CTA
    int splits = 1;
    double best = 0.0;
    for (int s = 1; s <= 256 && s <= kb_total; ++s) {
        if (s > 1 && kb_total / s < 8) break;
        const long long ctas = active * s;
        const long long waves = (ctas + ctx->num_sms - 1) / ctx->num_sms;
        const double eff = (double)ctas / (double)(waves * ctx->num_sms);
        if (eff > best + 1e-9) { best = eff; splits = s; }
        if (eff >= 0.97 && waves >= 2) { splits = s; break; }
    }
    const int kbs = cdiv(kb_total, splits);
    splits = cdiv(kb_total, kbs);
    RS_TRY(partials(ctx, (size_t)splits * M * N));
    RS_CUDA(ctx, cudaMemsetAsync(ctx->ws.tcerr, 0, sizeof(int), st));
    static bool attr = false;
    if (!attr) {
        RS_CUDA(ctx, cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
        attr = true;
    }
    {
        const double frac = blk_rows > 0 ? (double)active / ((double)tn * tm) : 1.0;
        ProfScope ps(ctx, RSDFT_K_GRAM_TC, 3.0 * 2.0 * (double)M * N * K * frac,
                     4.0 * (double)K * (M + N), st);
        k_gram_tc<<<dim3(tn, tm, splits), THREADS, SMEM_BYTES, st>>>(mAh, mAl, mBh, mBl, M, N, kb_total,
                                                                     kbs, tpb, blk_rows, ctx->ws.tcpart,
                                                                     ctx->ws.tcerr);
    }
    RS_LAUNCHED(ctx, "k_gram_tc");
    *splits_out = splits;
    return RSDFT_OK;
}

static rsdft_status check_err(rsdft_ctx *ctx, cudaStream_t st) {
    int *slot = reinterpret_cast<int *>(ctx->ws.hbuf + ctx->ws.hbuf_elems - 24);
    RS_CUDA(ctx, cudaMemcpyAsync(slot, ctx->ws.tcerr, sizeof(int), cudaMemcpyDeviceToHost, st));
    RS_CUDA(ctx, cudaStreamSynchronize(st));
    if (*slot) return fail(ctx, RSDFT_E_TIMEOUT, "tensor-core Gram: an mbarrier wait timed out");
    return RSDFT_OK;
}

// Coefficient operands of one rotation: [W P] part and X part, hi and lo.
struct RotCoef {
    __nv_bfloat16 *wph, *wpl, *xh, *xl;
    int kpad_wp, kpad_x;
};

// One rotation out0 = base + sign (X C_X + WP C_WP), out1 = WP C_WP (when kwp > 0):
// X = kx split rows at (xh, xl), WP = kwp split rows at (wph, wpl), leading
// dimension ldk; C rows [0, kx) multiply X, rows [kx, kx + kwp) multiply WP;
// ncol output bands.
struct RotSpec {
    const __nv_bfloat16 *xh, *xl, *wph, *wpl;
    long long ldk;
    int kx, kwp;
    const double2 *c;
    int ldc, ncol;
    float2 *out0, *out1;
    const float2 *base;
    int sign;
};

static rsdft_status rot_coef(rsdft_ctx *ctx, const RotSpec &sp, int nh, RotCoef &rc, cudaStream_t st) {
    Workspace &w = ctx->ws;
    rc.kpad_wp = cdiv(sp.kwp, RBK) * RBK;
    rc.kpad_x = cdiv(sp.kx, RBK) * RBK;
    const size_t per_wp = (size_t)2 * nh * rc.kpad_wp, per_x = (size_t)2 * nh * rc.kpad_x;
    const size_t need = 2 * (per_wp + per_x) * sizeof(__nv_bfloat16) + 256;
    if (need > w.tcrot_bytes) {
        if (w.tcrot) {
            cudaFree(w.tcrot);
            for (auto &p : ctx->owned)
                if (p == w.tcrot) p = nullptr;
        }
        w.tcrot = nullptr;
        w.tcrot_bytes = 0;
        RS_TRY(dev_alloc(ctx, &w.tcrot, need));
        w.tcrot_bytes = need;
    }
    rc.wph = reinterpret_cast<__nv_bfloat16 *>(w.tcrot);
    rc.wpl = rc.wph + per_wp;
    rc.xh = rc.wpl + per_wp;
    rc.xl = rc.xh + per_x;
    if (per_wp > 0) {
        k_rot_coef<<<cdiv((long long)per_wp, 256), 256, 0, st>>>(sp.c, sp.ldc, sp.kx, sp.kwp, sp.ncol, nh,
                                                                  rc.kpad_wp, rc.wph, rc.wpl);
        count_launch(ctx);
    }
    k_rot_coef<<<cdiv((long long)per_x, 256), 256, 0, st>>>(sp.c, sp.ldc, 0, sp.kx, sp.ncol, nh, rc.kpad_x,
                                                             rc.xh, rc.xl);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_rot_coef");
    return RSDFT_OK;
}

static rsdft_status rotate_launch(rsdft_ctx *ctx, const RotSpec &sp, cudaStream_t st) {
    RS_TRY(encoder(ctx));
    const int nh = cdiv(sp.ncol, 16) * 16;
    RotCoef rc;
    RS_TRY(rot_coef(ctx, sp, nh, rc, st));
    const long long two_n = 2 * ctx->n;
    CUtensorMap mWPh, mWPl, mXh, mXl, mBWPh, mBWPl, mBXh, mBXl;
    RS_TRY(make_map(ctx, &mXh, sp.xh, two_n, sp.kx, sp.ldk, RBK));
    RS_TRY(make_map(ctx, &mXl, sp.xl, two_n, sp.kx, sp.ldk, RBK));
    RS_TRY(make_map(ctx, &mBXh, rc.xh, rc.kpad_x, 2 * nh, rc.kpad_x, nh));
    RS_TRY(make_map(ctx, &mBXl, rc.xl, rc.kpad_x, 2 * nh, rc.kpad_x, nh));
    if (sp.kwp > 0) {
        RS_TRY(make_map(ctx, &mWPh, sp.wph, two_n, sp.kwp, sp.ldk, RBK));
        RS_TRY(make_map(ctx, &mWPl, sp.wpl, two_n, sp.kwp, sp.ldk, RBK));
        RS_TRY(make_map(ctx, &mBWPh, rc.wph, rc.kpad_wp, 2 * nh, rc.kpad_wp, nh));
        RS_TRY(make_map(ctx, &mBWPl, rc.wpl, rc.kpad_wp, 2 * nh, rc.kpad_wp, nh));
    } else {
        mWPh = mXh;   // never read: the [W P] phase has no k-blocks
        mWPl = mXl;
        mBWPh = mBXh;
        mBWPl = mBXl;
    }
    RS_TRY(partials(ctx, 0));
    RS_CUDA(ctx, cudaMemsetAsync(ctx->ws.tcerr, 0, sizeof(int), st));
    const int smem = RSTAGES * rot_stage_bytes(nh) + 1024;
    static int attr = 0;
    if (attr < smem) {
        RS_CUDA(ctx, cudaFuncSetAttribute(k_rot_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        attr = smem;
    }
    const int ntiles = (int)((two_n + 127) / 128);
    const int grid = std::min(ntiles, ctx->num_sms);
    const int k = sp.kx + sp.kwp;
    {
        ProfScope ps(ctx, RSDFT_K_ROTATE_TC, 3.0 * 2.0 * (double)two_n * (2.0 * sp.ncol) * k,
                     2.0 * 2.0 * (double)k * two_n +
                         4.0 * (double)sp.ncol * two_n * ((sp.out1 ? 2.0 : 1.0) + (sp.base ? 1.0 : 0.0)),
                     st);
        k_rot_tc<<<grid, RTHREADS, smem, st>>>(mWPh, mWPl, mXh, mXl, mBWPh, mBWPl, mBXh, mBXl, nh, sp.ncol,
                                                rc.kpad_wp / RBK, rc.kpad_x / RBK, two_n, ntiles,
                                                reinterpret_cast<float *>(sp.out0),
                                                reinterpret_cast<float *>(sp.out1),
                                                reinterpret_cast<const float *>(sp.base), (float)sp.sign,
                                                ctx->ws.tcerr);
    }
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_rot_tc");
    return check_err(ctx, st);
}

// Ritz rotation of split rows row0 .. row0 + k of b (X = the first m rows).
static rsdft_status rotate_rows(rsdft_ctx *ctx, const Buffers &b, int row0, int k, const double2 *c, int ldc,
                                int m, float2 *out0, float2 *out1, cudaStream_t st) {
    RotSpec sp;
    sp.xh = b.bh + (size_t)row0 * b.ldk;
    sp.xl = b.bl + (size_t)row0 * b.ldk;
    sp.wph = b.bh + (size_t)(row0 + m) * b.ldk;
    sp.wpl = b.bl + (size_t)(row0 + m) * b.ldk;
    sp.ldk = b.ldk;
    sp.kx = m;
    sp.kwp = k - m;
    sp.c = c;
    sp.ldc = ldc;
    sp.ncol = m;
    sp.out0 = out0;
    sp.out1 = out1;
    sp.base = nullptr;
    sp.sign = 1;
    return rotate_launch(ctx, sp, st);
}

}  // namespace tc

// G_S = <Y|Y>, G_H = <Y|HY> (Hermitised, scaled by dV) for FP32 blocks on the
// tensor cores: one GEMM of A = Y against B = [Y; Yrot; HY; HYrot] (A is read
// from the first k rows of B).  The split rows stay in the workspace for the
// Ritz rotation (rotate_tc_split).
rsdft_status gram_tc_sh(rsdft_ctx *ctx, const RowBlocksT<float2> &Y, const RowBlocksT<float2> &HY,
                        double2 *gs, double2 *gh, int ld, cudaStream_t st) {
    const int k = Y.cnt[0] + Y.cnt[1] + Y.cnt[2];
    if (k <= 0) return RSDFT_OK;
    tc::Buffers b;
    RS_TRY(tc::buffers(ctx, 0, 4 * k, b));
    b.ah = b.bh;   // A = the first k rows of B
    b.al = b.bl;
    RS_TRY(tc::split_rows(ctx, Y, 0, b.bh, b.bl, 0, b.ldk, st));
    RS_TRY(tc::split_rows(ctx, Y, 1, b.bh, b.bl, k, b.ldk, st));
    RS_TRY(tc::split_rows(ctx, HY, 0, b.bh, b.bl, 2 * k, b.ldk, st));
    RS_TRY(tc::split_rows(ctx, HY, 1, b.bh, b.bl, 3 * k, b.ldk, st));
    int splits = 0;
    RS_TRY(tc::gemm(ctx, b, k, 4 * k, st, &splits, k));
    tc::k_gram_tc_reduce_sh<<<cdiv((long long)k * k, 256), 256, 0, st>>>(ctx->ws.tcpart, splits, k, ctx->dV,
                                                                          gs, gh, ld);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_gram_tc_reduce_sh");
    return tc::check_err(ctx, st);
}

// General G = <A|B> (na x nb) for FP32 blocks on the tensor cores.
rsdft_status gram_tc(rsdft_ctx *ctx, const RowBlocksT<float2> &A, const RowBlocksT<float2> &B,
                     double2 *g, int ld, cudaStream_t st) {
    const int na = A.cnt[0] + A.cnt[1] + A.cnt[2], nb = B.cnt[0] + B.cnt[1] + B.cnt[2];
    if (na <= 0 || nb <= 0) return RSDFT_OK;
    tc::Buffers b;
    RS_TRY(tc::buffers(ctx, na, 2 * nb, b));
    RS_TRY(tc::split_rows(ctx, A, 0, b.ah, b.al, 0, b.ldk, st));
    RS_TRY(tc::split_rows(ctx, B, 0, b.bh, b.bl, 0, b.ldk, st));
    RS_TRY(tc::split_rows(ctx, B, 1, b.bh, b.bl, nb, b.ldk, st));
    int splits = 0;
    RS_TRY(tc::gemm(ctx, b, na, 2 * nb, st, &splits));
    tc::k_gram_tc_reduce<<<cdiv((long long)na * nb, 256), 256, 0, st>>>(ctx->ws.tcpart, splits, na, nb,
                                                                        ctx->dV, g, ld);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_gram_tc_reduce");
    return tc::check_err(ctx, st);
}

// W <- W - X C (C = <X|W>, m x na, ld na) on the tensor cores, from the X split
// rows that the preceding gram_tc(X, W) left in the A region of the workspace.
rsdft_status rotate_tc_ortho(rsdft_ctx *ctx, int m, int na, const double2 *c, float2 *w, cudaStream_t st) {
    if (m < 1 || na < 1 || cdiv(na, 16) * 16 > tc::MAX_NH)
        return fail(ctx, RSDFT_E_INVALID, "tensor-core orthogonalisation: m %d, na %d", m, na);
    tc::Buffers b;
    RS_TRY(tc::buffers(ctx, m, 2 * na, b));   // the layout gram_tc(X, W) wrote
    tc::RotSpec sp;
    sp.xh = b.ah;
    sp.xl = b.al;
    sp.wph = sp.wpl = nullptr;
    sp.ldk = b.ldk;
    sp.kx = m;
    sp.kwp = 0;
    sp.c = c;
    sp.ldc = na;
    sp.ncol = na;
    sp.out0 = w;
    sp.out1 = nullptr;
    sp.base = w;
    sp.sign = -1;
    return tc::rotate_launch(ctx, sp, st);
}

bool rotate_tc_fits(int k, int m) { return m >= 1 && k > m && cdiv(m, 16) * 16 <= tc::MAX_NH; }

rsdft_status rotate_tc_split(rsdft_ctx *ctx, int which, int k, const double2 *c, int ldc, int m,
                             float2 *out0, float2 *out1, cudaStream_t st) {
    // k == m (X only, no new P) is allowed when out1 is NULL
    const bool ok = rotate_tc_fits(k, m) || (k == m && !out1 && m >= 1 && cdiv(m, 16) * 16 <= tc::MAX_NH);
    if (!ok) return fail(ctx, RSDFT_E_INVALID, "tensor-core rotation: k %d, m %d", k, m);
    tc::Buffers b;
    RS_TRY(tc::buffers(ctx, 0, 4 * k, b));   // the layout gram_tc_sh wrote
    return tc::rotate_rows(ctx, b, which == 0 ? 0 : 2 * k, k, c, ldc, m, out0, out1, st);
}

rsdft_status rotate_tc(rsdft_ctx *ctx, const float2 *y, int k, const double2 *c, int ldc, int m,
                       float2 *out0, float2 *out1, cudaStream_t st) {
    if (!rotate_tc_fits(k, m)) return fail(ctx, RSDFT_E_INVALID, "tensor-core rotation: k %d, m %d", k, m);
    tc::Buffers b;
    RS_TRY(tc::buffers(ctx, 0, k, b));
    RowBlocksT<float2> Y{{y, nullptr, nullptr}, {k, 0, 0}};
    RS_TRY(tc::split_rows(ctx, Y, 0, b.bh, b.bl, 0, b.ldk, st));
    return tc::rotate_rows(ctx, b, 0, k, c, ldc, m, out0, out1, st);
}

}  // namespace rsdft

using namespace rsdft;

extern "C" rsdft_status rsdft_gram_bf16x3(rsdft_ctx *ctx, const void *a_dev, int na, const void *b_dev,
                                          int nb, void *g_dev, void *stream) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (na < 0 || nb < 0 || ((na > 0 && nb > 0) && (!a_dev || !b_dev || !g_dev)))
        return fail(ctx, RSDFT_E_INVALID, "bad gram arguments");
    RS_TRY(ensure_workspace(ctx, 1));
    RowBlocksT<float2> A{{(const float2 *)a_dev, nullptr, nullptr}, {na, 0, 0}};
    RowBlocksT<float2> B{{(const float2 *)b_dev, nullptr, nullptr}, {nb, 0, 0}};
    return gram_tc(ctx, A, B, (double2 *)g_dev, nb, as_stream(stream));
}

extern "C" rsdft_status rsdft_rotate_bf16x3(rsdft_ctx *ctx, const void *y_dev, int k, const void *c_dev, int m,
                                            void *out0_dev, void *out1_dev, void *stream) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (!y_dev || !c_dev || !out0_dev || !out1_dev) return fail(ctx, RSDFT_E_INVALID, "NULL pointer");
    if (!rotate_tc_fits(k, m)) return fail(ctx, RSDFT_E_INVALID, "rotation shape k %d, m %d unsupported", k, m);
    RS_TRY(ensure_workspace(ctx, 1));
    return rotate_tc(ctx, (const float2 *)y_dev, k, (const double2 *)c_dev, m, m, (float2 *)out0_dev,
                     (float2 *)out1_dev, as_stream(stream));
}
