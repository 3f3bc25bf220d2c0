// Tensor-core Gram matrices and Ritz rotations for the mixed form (SCF task
// (2)): split-BF16 products on the 5th-generation tensor cores (tcgen05, FP32
// accumulation in TMEM), operands staged by TMA into swizzled shared memory.
//
// Each FP32 value x is split x = hi + lo, hi = bf16(x), lo = bf16(x - hi), and a
// product uses hi*hi' + hi*lo' + lo*hi' (the lo*lo' term is below FP32
// rounding).  The split rows are planar: row j holds [Re y_j | Im y_j] (each
// plane padded to a multiple of 64 points), hi and lo in separate arrays.  A
// complex product is then four real products of planes, and the one with a
// minus sign uses the MMA's negate-A bit:
//   Gram      Re G = A_re B_re^T + A_im B_im^T,  Im G = A_re B_im^T - A_im B_re^T
//   rotation  Re out = Y_re^T C_r - Y_im^T C_i,  Im out = Y_re^T C_i + Y_im^T C_r
// with two TMEM accumulators (real and imaginary part) per tile.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "rsdft_internal.h"

namespace rsdft {
namespace tc {

constexpr int BM = 128;              // Gram tile rows (A rows)
constexpr int BN = 128;              // Gram tile cols (B rows)
constexpr int GK = 32;               // points per Gram stage: 64-byte rows, 64-byte swizzle
constexpr int GSTAGES = 3;
constexpr int GTILE = BM * GK * 2;   // 8 KB per operand tile
constexpr int GSTAGE_BYTES = 8 * GTILE;                  // A re/im hi/lo, B re/im hi/lo
constexpr int GSMEM = GSTAGES * GSTAGE_BYTES + 1024;     // + alignment slack
constexpr int GTHREADS = 192;        // warp 0: TMA, warp 1: MMA, warps 2-5: accumulator drain
constexpr int PROMOTE_KB = 32;       // k-blocks per tensor-core accumulation chunk
constexpr int PLANE_ALIGN = 64;      // plane length granularity (points)
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

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x,
                                            int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand with 64-byte swizzle:
// rows of 32 bf16 (64 bytes), 8-row groups of 512 bytes (stride byte offset),
// descriptor version 1, layout type 4 (64-byte swizzle).
__device__ __forceinline__ uint64_t smem_desc_k64(const void *p) {
    uint64_t d = (smem_u32(p) & 0x3FFFFu) >> 4;  // start address  [0, 14)
    d |= (uint64_t)1 << 16;                      // leading byte offset (unused for this layout)
    d |= (uint64_t)(512 >> 4) << 32;             // stride byte offset [32, 46)
    d |= (uint64_t)1 << 46;                      // version
    d |= (uint64_t)4 << 61;                      // layout: 64-byte swizzle
    return d;
}

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

// Instruction descriptor of kind::f16: BF16 x BF16 -> FP32, both K-major
// (bit 13 negates A, bit 15 makes A MN-major).
constexpr uint32_t IDESC_NEG_A = 1u << 13;
constexpr uint32_t IDESC_A_MN = 1u << 15;
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

// Store 32 consecutive FP32 columns of this thread's TMEM lane (waits for completion).
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float *v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
        "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
        "r"(__float_as_uint(v[15])), "r"(__float_as_uint(v[16])), "r"(__float_as_uint(v[17])),
        "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])), "r"(__float_as_uint(v[20])),
        "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])), "r"(__float_as_uint(v[23])),
        "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])), "r"(__float_as_uint(v[26])),
        "r"(__float_as_uint(v[27])), "r"(__float_as_uint(v[28])), "r"(__float_as_uint(v[29])),
        "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31]))
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Split FP32 complex rows into planar BF16 hi/lo rows [Re | Im], each plane ldh
// points long (ldh a multiple of 64, points n..ldh-1 zero).  Destination rows
// dst_row0 + r, row length 2 ldh.  Two points per thread (bf16x2 stores).
__global__ void k_split_planar(RowBlocksT<float2> src, int nrows, long long n, int ldh,
                               __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ lo, int dst_row0) {
    const int r = blockIdx.y;
    if (r >= nrows) return;
    int i = r, blk = 0;
    while (blk < 2 && i >= src.cnt[blk]) { i -= src.cnt[blk]; ++blk; }
    const float2 *row = src.ptr[blk] + (size_t)i * n;
    const size_t base = (size_t)(dst_row0 + r) * 2 * ldh;
    __nv_bfloat162 *hre = reinterpret_cast<__nv_bfloat162 *>(hi + base);
    __nv_bfloat162 *him = reinterpret_cast<__nv_bfloat162 *>(hi + base + ldh);
    __nv_bfloat162 *lre = reinterpret_cast<__nv_bfloat162 *>(lo + base);
    __nv_bfloat162 *lim = reinterpret_cast<__nv_bfloat162 *>(lo + base + ldh);
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < ldh / 2;
         q += (long long)gridDim.x * blockDim.x) {
        const long long p = 2 * q;
        const float2 v0 = p < n ? row[p] : make_float2(0.0f, 0.0f);
        const float2 v1 = p + 1 < n ? row[p + 1] : make_float2(0.0f, 0.0f);
        const __nv_bfloat16 h0 = __float2bfloat16_rn(v0.x), h1 = __float2bfloat16_rn(v1.x);
        const __nv_bfloat16 g0 = __float2bfloat16_rn(v0.y), g1 = __float2bfloat16_rn(v1.y);
        hre[q] = __halves2bfloat162(h0, h1);
        him[q] = __halves2bfloat162(g0, g1);
        lre[q] = __halves2bfloat162(__float2bfloat16_rn(v0.x - __bfloat162float(h0)),
                                    __float2bfloat16_rn(v1.x - __bfloat162float(h1)));
        lim[q] = __halves2bfloat162(__float2bfloat16_rn(v0.y - __bfloat162float(g0)),
                                    __float2bfloat16_rn(v1.y - __bfloat162float(g1)));
    }
}

// part[split][M][N] (complex, FP32) = the split's point range of conj(A) B^T from
// planar split rows.  Grid (N tiles, M tiles, splits), 192 threads: warp 0 lane 0
// issues TMA, warp 1 lane 0 issues MMAs, warps 2-5 drain the accumulator (warp w
// owns TMEM lanes 32 (w mod 4) ..).  The MMAs accumulate at most PROMOTE_KB
// k-blocks in TMEM (columns 0..255: real part 0..127, imaginary part 128..255);
// the drain warps then add that chunk to a running sum kept in TMEM columns
// 256..511 with round-to-nearest FP32 adds, and the MMAs of the next chunk start
// afresh.  The tensor cores' FP32 accumulation loses a little on every step, so
// an error proportional to the chain length would otherwise grow with the
// k-blocks per split.  tpb > 0: B is a stack of blocks of blk_rows rows, each
// Hermitian against A; blockIdx.x = block * tpb + tile in the block, and tiles
// below the diagonal are skipped.
__global__ void __launch_bounds__(GTHREADS, 1)
k_gram_pl(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
          const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl, int M, int N,
          int ldh, int kb_total, int kb_per_split, int tpb, int blk_rows, float2 *__restrict__ part,
          int *err) {
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
    __shared__ __align__(8) uint64_t full_bar[GSTAGES];
    __shared__ __align__(8) uint64_t empty_bar[GSTAGES];
    __shared__ __align__(8) uint64_t acc_full;
    __shared__ __align__(8) uint64_t acc_empty;
    __shared__ __align__(8) uint64_t acc_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    const int tm = blockIdx.y, split = blockIdx.z;
    const int kb0 = split * kb_per_split;
    const int nkb = max(0, min(kb_total, kb0 + kb_per_split) - kb0);
    const int nch = (nkb + PROMOTE_KB - 1) / PROMOTE_KB;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < GSTAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&acc_full, 1);
        mbar_init(&acc_empty, 4);   // one arrive per drain warp
        mbar_init(&acc_bar, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(&tmem_base, 4 * BN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    volatile int *abort = &s_abort;

    if (warp == 0 && lane == 0) {
        // ---- TMA producer: per stage the re and im planes of A and B, hi and lo
        int issued = 0;
        for (int it = 0; it < nkb; ++it) {
            const int s = it % GSTAGES, r = it / GSTAGES;
            if (r > 0 && !mbar_wait(&empty_bar[s], (r - 1) & 1, abort)) break;
            unsigned char *st = smem + s * GSTAGE_BYTES;
            mbar_expect_tx(&full_bar[s], GSTAGE_BYTES);
            const int xr = (kb0 + it) * GK, xi = ldh + xr;
            tma_load_2d(st + 0 * GTILE, &mAh, &full_bar[s], xr, tm * BM);
            tma_load_2d(st + 1 * GTILE, &mAl, &full_bar[s], xr, tm * BM);
            tma_load_2d(st + 2 * GTILE, &mAh, &full_bar[s], xi, tm * BM);
            tma_load_2d(st + 3 * GTILE, &mAl, &full_bar[s], xi, tm * BM);
            tma_load_2d(st + 4 * GTILE, &mBh, &full_bar[s], xr, brow0);
            tma_load_2d(st + 5 * GTILE, &mBl, &full_bar[s], xr, brow0);
            tma_load_2d(st + 6 * GTILE, &mBh, &full_bar[s], xi, brow0);
            tma_load_2d(st + 7 * GTILE, &mBl, &full_bar[s], xi, brow0);
            issued = it + 1;
        }
        if (*abort) {
            // let the copies still in flight land before the CTA leaves
            for (int it = max(0, issued - GSTAGES); it < issued; ++it) {
                const long long t0 = clock64();
                while (!mbar_try_wait(&full_bar[it % GSTAGES], (it / GSTAGES) & 1) &&
                       clock64() - t0 < WAIT_LIMIT) {
                }
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer: chunk c starts once chunk c - 1 has been drained
        const uint32_t idesc = idesc_bf16(BM, BN), idesc_neg = idesc | IDESC_NEG_A;
        const uint32_t d_re = tmem, d_im = tmem + BN;
        bool stop = false;
        for (int c = 0; c < nch && !stop; ++c) {
            if (c > 0 && !mbar_wait(&acc_empty, (c - 1) & 1, abort)) break;
            tc_fence_after();
            const int it0 = c * PROMOTE_KB, it1 = min(nkb, it0 + PROMOTE_KB);
            for (int it = it0; it < it1; ++it) {
                const int s = it % GSTAGES, r = it / GSTAGES;
                if (!mbar_wait(&full_bar[s], r & 1, abort)) {
                    stop = true;
                    break;
                }
                tc_fence_after();
                unsigned char *st = smem + s * GSTAGE_BYTES;
#pragma unroll
                for (int kk = 0; kk < GK / 16; ++kk) {
                    const int off = kk * 32;   // 16 bf16 = 32 bytes along the 64-byte row
                    const uint64_t arh = smem_desc_k64(st + 0 * GTILE + off), arl = smem_desc_k64(st + 1 * GTILE + off);
                    const uint64_t aih = smem_desc_k64(st + 2 * GTILE + off), ail = smem_desc_k64(st + 3 * GTILE + off);
                    const uint64_t brh = smem_desc_k64(st + 4 * GTILE + off), brl = smem_desc_k64(st + 5 * GTILE + off);
                    const uint64_t bih = smem_desc_k64(st + 6 * GTILE + off), bil = smem_desc_k64(st + 7 * GTILE + off);
                    const uint32_t acc = (it != it0 || kk != 0) ? 1u : 0u;
                    // Re += A_re B_re + A_im B_im
                    mma_bf16(d_re, arh, brh, idesc, acc);
                    mma_bf16(d_re, arh, brl, idesc, 1u);
                    mma_bf16(d_re, arl, brh, idesc, 1u);
                    mma_bf16(d_re, aih, bih, idesc, 1u);
                    mma_bf16(d_re, aih, bil, idesc, 1u);
                    mma_bf16(d_re, ail, bih, idesc, 1u);
                    // Im += A_re B_im - A_im B_re
                    mma_bf16(d_im, arh, bih, idesc, acc);
                    mma_bf16(d_im, arh, bil, idesc, 1u);
                    mma_bf16(d_im, arl, bih, idesc, 1u);
                    mma_bf16(d_im, aih, brh, idesc_neg, 1u);
                    mma_bf16(d_im, aih, brl, idesc_neg, 1u);
                    mma_bf16(d_im, ail, brh, idesc_neg, 1u);
                }
                mma_commit(&empty_bar[s]);
            }
            if (!stop) mma_commit(&acc_full);   // arrives when the chunk's MMAs are done
        }
        mma_commit(&acc_bar);   // arrives once every MMA issued above has completed
    } else if (warp >= 2) {
        // ---- drain: running sum (TMEM columns 256..511) += chunk; the last chunk
        // goes with the sum to this split's partial
        const int q = warp & 3;   // TMEM lane quarter
        const int row = tm * BM + q * 32 + lane;
        float2 *dst_row = part + ((size_t)split * M + row) * N + (size_t)ncol0;
        const uint32_t lanes = (uint32_t)(q * 32) << 16;
        const uint32_t acc = tmem + lanes, sum = tmem + lanes + (uint32_t)(2 * BN);
        for (int c = 0; c < nch; ++c) {
            // warp-uniform bounded wait (the TMEM loads below are warp-collective)
            bool ok = true;
            const long long t0 = clock64();
            while (true) {
                const bool done = mbar_try_wait(&acc_full, c & 1);
                if (__all_sync(0xffffffffu, done)) break;
                if (__any_sync(0xffffffffu, *abort || clock64() - t0 > WAIT_LIMIT)) {
                    ok = false;
                    break;
                }
            }
            if (!ok) {
                *abort = 1;
                break;
            }
            tc_fence_after();
            const bool last = c == nch - 1;
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 32) {
                float vr[32], vi[32];
                tmem_ld32(acc + (uint32_t)c0, vr);
                tmem_ld32(acc + (uint32_t)(BN + c0), vi);
                if (c > 0) {
                    float sr[32], si[32];
                    tmem_ld32(sum + (uint32_t)c0, sr);
                    tmem_ld32(sum + (uint32_t)(BN + c0), si);
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        vr[i] += sr[i];
                        vi[i] += si[i];
                    }
                }
                if (!last) {
                    tmem_st32(sum + (uint32_t)c0, vr);
                    tmem_st32(sum + (uint32_t)(BN + c0), vi);
                } else if (row < M && !*abort) {
                    float2 *dst = dst_row + c0;
                    const int cmax = min(32, nvalid - c0);
#pragma unroll
                    for (int i = 0; i < 32; ++i)
                        if (i < cmax) dst[i] = make_float2(vr[i], vi[i]);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty);
        }
    }
    __syncwarp();
    // TMEM is released only once every MMA issued has completed (time-bounded)
    if (warp == 0) {
        const long long t0 = clock64();
        while (!mbar_try_wait(&acc_bar, 0)) {
            if (clock64() - t0 > WAIT_LIMIT) {
                *abort = 1;
                break;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 4 * BN);
    }
    if (threadIdx.x == 0 && *abort) atomicExch(err, 1);
}

// G_S and G_H of the LOBPCG basis from the split partials of conj(Y) [Y; HY]^T
// (N = 2k, upper 128-tiles of each block computed): scaled by dV, FP64 sums;
// entries of tiles above the diagonal are taken as computed, below it as the
// conjugate of the mirrored entry, and on diagonal tiles the two are averaged
// (as the FP64 path does).
__global__ void k_gram_pl_reduce_sh(const float2 *__restrict__ part, int splits, int k, double scale,
                                    double2 *__restrict__ gs, double2 *__restrict__ gh, int ld) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)k * k) return;
    const int i = (int)(idx / k), j = (int)(idx % k);
    const size_t N = 2 * (size_t)k, plane = (size_t)k * N;
    auto sum2 = [&](int r, int c, double2 &s, double2 &h) {
        s = h = make_double2(0.0, 0.0);
        for (int q = 0; q < splits; ++q) {
            const float2 *pr = part + q * plane + (size_t)r * N;
            s.x += (double)pr[c].x;
            s.y += (double)pr[c].y;
            h.x += (double)pr[k + c].x;
            h.y += (double)pr[k + c].y;
        }
    };
    const int ti = i / BM, tj = j / BN;
    double2 s, h;
    if (ti < tj) {
        sum2(i, j, s, h);
    } else if (ti > tj) {
        sum2(j, i, s, h);
        s.y = -s.y;
        h.y = -h.y;
    } else {
        double2 s2, h2;
        sum2(i, j, s, h);
        sum2(j, i, s2, h2);
        s = make_double2(0.5 * (s.x + s2.x), 0.5 * (s.y - s2.y));
        h = make_double2(0.5 * (h.x + h2.x), 0.5 * (h.y - h2.y));
    }
    gs[(size_t)i * ld + j] = make_double2(scale * s.x, scale * s.y);
    gh[(size_t)i * ld + j] = make_double2(scale * h.x, scale * h.y);
}

// General G = conj(A) B^T (na x nb) from the split partials.
__global__ void k_gram_pl_reduce(const float2 *__restrict__ part, int splits, int na, int nb, double scale,
                                 double2 *__restrict__ g, int ld) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)na * nb) return;
    const int i = (int)(idx / nb), j = (int)(idx % nb);
    const size_t plane = (size_t)na * nb;
    double re = 0.0, im = 0.0;
    for (int q = 0; q < splits; ++q) {
        const float2 v = part[q * plane + (size_t)i * nb + j];
        re += (double)v.x;
        im += (double)v.y;
    }
    g[(size_t)i * ld + j] = make_double2(scale * re, scale * im);
}

// ---- Ritz rotation: out[b][:] = sum_j C[j][b] Y[j][:] ------------------------------
// As real GEMMs with M = grid points (128 per tile), N = bands (nh, a multiple of
// 16) and K = rows of Y: A = the planar split rows read MN-major by TMA (128-byte
// swizzle, 64 points per row), B = the coefficient planes C_r, C_i (K-major,
// 64-byte swizzle, 32 rows per stage).  Per 128-point tile the [W P] rows are
// accumulated first and written as the new P, then the X rows accumulate on top
// and the sum is written as the new X (= X C_X + P).
constexpr int RK = 32;                  // Y rows per pipeline stage
constexpr int RMAX_STAGES = 4;
constexpr int RTHREADS = 320;           // warp 0 TMA, warp 1 MMA, warps 2..9 epilogue
constexpr int REPI = 8;                 // epilogue warps (two per TMEM lane quarter)
constexpr int RA_CHUNK = 64 * RK * 2;   // 64 points x 32 rows of bf16: 4 KB
constexpr int MAX_NH = 240;

__host__ __device__ constexpr int rot_stage_bytes(int nh) { return 8 * RA_CHUNK + 4 * nh * 64; }
__host__ __device__ constexpr int rot_stages(int nh) {
    return (227 * 1024 - 1024) / rot_stage_bytes(nh) < RMAX_STAGES ? (227 * 1024 - 1024) / rot_stage_bytes(nh)
                                                                     : RMAX_STAGES;
}

// Split C (FP64 complex, rows j0..j0+nrows of [k][ldc], m columns) into the
// K-major bf16 hi/lo operand [2 nh][kpad]: row q < nh is Re C[j0 + t][q], row
// nh + q is Im C[j0 + t][q] at column t; zero outside (t >= nrows or q >= m).
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
k_rot_pl(const __grid_constant__ CUtensorMap mWPh, const __grid_constant__ CUtensorMap mWPl,
         const __grid_constant__ CUtensorMap mXh, const __grid_constant__ CUtensorMap mXl,
         const __grid_constant__ CUtensorMap mBWPh, const __grid_constant__ CUtensorMap mBWPl,
         const __grid_constant__ CUtensorMap mBXh, const __grid_constant__ CUtensorMap mBXl, int nh, int m,
         int kb_wp, int kb_x, int ldh, long long n, int ntiles, int stages, float2 *out0,
         float2 *__restrict__ out1, const float2 *base, float sign, int *err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[RMAX_STAGES];
    __shared__ __align__(8) uint64_t empty_bar[RMAX_STAGES];
    __shared__ __align__(8) uint64_t accf_bar;   // accumulators ready (MMA -> epilogue)
    __shared__ __align__(8) uint64_t acce_bar;   // accumulators drained (epilogue -> MMA)
    __shared__ __align__(8) uint64_t done_bar;   // every MMA issued has completed
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int stage_bytes = rot_stage_bytes(nh);
    const int bpart = nh * 64;                // one coefficient plane (re or im), hi or lo
    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
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
            const int p0 = t * 128;
            for (int ph = 0; ph < 2 && !stop; ++ph) {
                const int nkb = ph == 0 ? kb_wp : kb_x;
                const CUtensorMap *ah = ph == 0 ? &mWPh : &mXh, *al = ph == 0 ? &mWPl : &mXl;
                const CUtensorMap *bh = ph == 0 ? &mBWPh : &mBXh, *bl = ph == 0 ? &mBWPl : &mBXl;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = it % stages, r = it / stages;
                    if (r > 0 && !mbar_wait(&empty_bar[s], (r - 1) & 1, abort)) { stop = true; break; }
                    unsigned char *st = smem + s * stage_bytes;
                    mbar_expect_tx(&full_bar[s], stage_bytes);
                    const int y = kb * RK;
                    // A: re hi (2 chunks), re lo, im hi, im lo
                    tma_load_2d(st + 0 * RA_CHUNK, ah, &full_bar[s], p0, y);
                    tma_load_2d(st + 1 * RA_CHUNK, ah, &full_bar[s], p0 + 64, y);
                    tma_load_2d(st + 2 * RA_CHUNK, al, &full_bar[s], p0, y);
                    tma_load_2d(st + 3 * RA_CHUNK, al, &full_bar[s], p0 + 64, y);
                    tma_load_2d(st + 4 * RA_CHUNK, ah, &full_bar[s], ldh + p0, y);
                    tma_load_2d(st + 5 * RA_CHUNK, ah, &full_bar[s], ldh + p0 + 64, y);
                    tma_load_2d(st + 6 * RA_CHUNK, al, &full_bar[s], ldh + p0, y);
                    tma_load_2d(st + 7 * RA_CHUNK, al, &full_bar[s], ldh + p0 + 64, y);
                    // B: C_r hi, C_i hi, C_r lo, C_i lo
                    unsigned char *sb = st + 8 * RA_CHUNK;
                    tma_load_2d(sb, bh, &full_bar[s], y, 0);
                    tma_load_2d(sb + bpart, bh, &full_bar[s], y, nh);
                    tma_load_2d(sb + 2 * bpart, bl, &full_bar[s], y, 0);
                    tma_load_2d(sb + 3 * bpart, bl, &full_bar[s], y, nh);
                }
            }
        }
        if (*abort) {
            // let the copies still in flight land before the CTA leaves
            for (int j = max(0, it - stages); j < it; ++j) {
                const long long t0 = clock64();
                while (!mbar_try_wait(&full_bar[j % stages], (j / stages) & 1) && clock64() - t0 < WAIT_LIMIT) {
                }
            }
        }
    } else if (warp == 1 && lane == 0) {
        // ---- MMA issuer
        const uint32_t idesc = idesc_bf16(128, nh) | IDESC_A_MN, idesc_neg = idesc | IDESC_NEG_A;
        const uint32_t d_re = tmem, d_im = tmem + (uint32_t)nh;
        int it = 0, ap = 0;
        bool stop = false;
        for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
            bool fresh = true;   // the tile's first MMAs overwrite the accumulators
            for (int ph = 0; ph < 2 && !stop; ++ph) {
                const int nkb = ph == 0 ? kb_wp : kb_x;
                if (nkb == 0) continue;   // no [W P] rows: X phase only
                if (ap > 0 && !mbar_wait(&acce_bar, (ap - 1) & 1, abort)) { stop = true; break; }
                tc_fence_after();
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = it % stages, r = it / stages;
                    if (!mbar_wait(&full_bar[s], r & 1, abort)) { stop = true; break; }
                    tc_fence_after();
                    unsigned char *st = smem + s * stage_bytes;
                    unsigned char *sb = st + 8 * RA_CHUNK;
#pragma unroll
                    for (int kk = 0; kk < RK / 16; ++kk) {
                        // A: 16 rows = two 8-row groups of 1024 B; B: 16 bf16 = 32 B
                        const uint64_t arh = smem_desc_mn(st + 0 * RA_CHUNK + kk * 2048, RA_CHUNK, 1024);
                        const uint64_t arl = smem_desc_mn(st + 2 * RA_CHUNK + kk * 2048, RA_CHUNK, 1024);
                        const uint64_t aih = smem_desc_mn(st + 4 * RA_CHUNK + kk * 2048, RA_CHUNK, 1024);
                        const uint64_t ail = smem_desc_mn(st + 6 * RA_CHUNK + kk * 2048, RA_CHUNK, 1024);
                        const uint64_t crh = smem_desc_k64(sb + kk * 32), cih = smem_desc_k64(sb + bpart + kk * 32);
                        const uint64_t crl = smem_desc_k64(sb + 2 * bpart + kk * 32);
                        const uint64_t cil = smem_desc_k64(sb + 3 * bpart + kk * 32);
                        const uint32_t acc = fresh ? 0u : 1u;
                        // Re += Y_re C_r - Y_im C_i
                        mma_bf16(d_re, arh, crh, idesc, acc);
                        mma_bf16(d_re, arh, crl, idesc, 1u);
                        mma_bf16(d_re, arl, crh, idesc, 1u);
                        mma_bf16(d_re, aih, cih, idesc_neg, 1u);
                        mma_bf16(d_re, aih, cil, idesc_neg, 1u);
                        mma_bf16(d_re, ail, cih, idesc_neg, 1u);
                        // Im += Y_re C_i + Y_im C_r
                        mma_bf16(d_im, arh, cih, idesc, acc);
                        mma_bf16(d_im, arh, cil, idesc, 1u);
                        mma_bf16(d_im, arl, cih, idesc, 1u);
                        mma_bf16(d_im, aih, crh, idesc, 1u);
                        mma_bf16(d_im, aih, crl, idesc, 1u);
                        mma_bf16(d_im, ail, crh, idesc, 1u);
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
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (the tile's
        // points); the two warps of a lane quarter take alternate 32-band chunks
        const int q = warp & 3, half = (warp - 2) >> 2;
        int ap = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const long long p = (long long)t * 128 + q * 32 + lane;
            for (int ph = 0; ph < 2; ++ph) {
                if ((ph == 0 ? kb_wp : kb_x) == 0) continue;
                if (!mbar_wait(&accf_bar, ap & 1, abort)) break;
                tc_fence_after();
                float2 *out = ph == 0 ? out1 : out0;
                const float2 *bse = ph == 0 ? nullptr : base;
                for (int b0 = half * 32; b0 < m; b0 += 64) {
                    float vr[32], vi[32];
                    float2 bv[32];
                    tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)b0, vr);
                    tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(nh + b0), vi);
                    if (bse) {
                        // all base loads of the chunk before any store (out may alias base)
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            bv[i] = (b0 + i < m && p < n) ? bse[(size_t)(b0 + i) * n + p] : make_float2(0.0f, 0.0f);
                    }
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        if (out && b0 + i < m && p < n) {
                            const size_t o = (size_t)(b0 + i) * n + p;
                            out[o] = bse ? make_float2(bv[i].x + sign * vr[i], bv[i].y + sign * vi[i])
                                         : make_float2(vr[i], vi[i]);
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
    static std::mutex mu;
    std::lock_guard<std::mutex> g(mu);
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

// 2D BF16 operand [rows][ld] with xvalid valid columns, box box_x x box_y (box_x
// bf16 = the swizzle span); rows beyond `rows` and columns beyond xvalid read
// as zero.
static rsdft_status make_map(rsdft_ctx *ctx, CUtensorMap *m, const void *base, long long xvalid, int rows,
                             long long ld, int box_x, int box_y, CUtensorMapSwizzle swz) {
    if ((reinterpret_cast<uintptr_t>(base) & 15u) || ((ld * 2) & 15))
        return fail(ctx, RSDFT_E_INVALID, "tensor map base or stride not 16-byte aligned");
    cuuint64_t dims[2] = {(cuuint64_t)xvalid, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    cuuint32_t box[2] = {(cuuint32_t)box_x, (cuuint32_t)box_y};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ctx, RSDFT_E_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return RSDFT_OK;
}

// Planar split rows: row r of a region holds [Re | Im], ldh points each
// (ldh = n rounded up to 64), hi and lo in separate arrays of the workspace.
struct Buffers {
    __nv_bfloat16 *ah, *al, *bh, *bl;
    int ldh;          // points per plane
    long long ld;     // bf16 per row (2 ldh)
};

static rsdft_status buffers(rsdft_ctx *ctx, int arows, int brows, Buffers &b) {
    Workspace &w = ctx->ws;
    b.ldh = (int)((ctx->n + PLANE_ALIGN - 1) / PLANE_ALIGN * PLANE_ALIGN);
    b.ld = 2LL * b.ldh;
    const size_t per = (size_t)b.ld * sizeof(__nv_bfloat16);
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
    b.al = b.ah + (size_t)arows * b.ld;
    b.bh = b.al + (size_t)arows * b.ld;
    b.bl = b.bh + (size_t)brows * b.ld;
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
        RS_TRY(dev_alloc(ctx, (void **)&w.tcpart, elems * sizeof(float2)));
        w.tcpart_elems = elems;
    }
    if (!w.tcerr) RS_TRY(dev_alloc(ctx, (void **)&w.tcerr, 64));
    return RSDFT_OK;
}

static rsdft_status split_rows(rsdft_ctx *ctx, const RowBlocksT<float2> &src, __nv_bfloat16 *hi,
                               __nv_bfloat16 *lo, int row0, int ldh, cudaStream_t st) {
    const int rows = src.cnt[0] + src.cnt[1] + src.cnt[2];
    if (rows <= 0) return RSDFT_OK;
    dim3 g(std::max(1, std::min(cdiv(ldh / 2, 256), 64)), rows);
    k_split_planar<<<g, 256, 0, st>>>(src, rows, ctx->n, ldh, hi, lo, row0);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_split_planar");
    return RSDFT_OK;
}

// conj(A) B^T over the points for A rows [0, M), B rows [0, N) already split;
// returns splits.  blk_rows > 0: B is N / blk_rows blocks Hermitian against A
// (upper tiles of each block only).
static rsdft_status gemm(rsdft_ctx *ctx, const Buffers &b, int M, int N, cudaStream_t st, int *splits_out,
                         int blk_rows = 0, int scale_splits = 0) {
    RS_TRY(encoder(ctx));
    CUtensorMap mAh, mAl, mBh, mBl;
    RS_TRY(make_map(ctx, &mAh, b.ah, b.ld, M, b.ld, GK, BM, CU_TENSOR_MAP_SWIZZLE_64B));
    RS_TRY(make_map(ctx, &mAl, b.al, b.ld, M, b.ld, GK, BM, CU_TENSOR_MAP_SWIZZLE_64B));
    RS_TRY(make_map(ctx, &mBh, b.bh, b.ld, N, b.ld, GK, BN, CU_TENSOR_MAP_SWIZZLE_64B));
    RS_TRY(make_map(ctx, &mBl, b.bl, b.ld, N, b.ld, GK, BN, CU_TENSOR_MAP_SWIZZLE_64B));
    const int tm = cdiv(M, BM);
    const int tpb = blk_rows > 0 ? cdiv(blk_rows, BN) : 0;
    const int tn = blk_rows > 0 ? (N / blk_rows) * tpb : cdiv(N, BN);
    // tiles that do work: all, or the upper ones of each Hermitian block
    const long long active = blk_rows > 0 ? (long long)(N / blk_rows) * tpb * (tpb + 1) / 2 : (long long)tn * tm;
    const int kb_total = b.ldh / GK;   // whole plane; the padding is zero
    // splits: whole waves of one CTA per SM, at least 16 k-blocks per CTA
    int splits = 1;
    double best = 0.0;
    for (int s = 1; s <= 256 && s <= kb_total; ++s) {
        if (s > 1 && kb_total / s < 16) break;
        const long long ctas = active * s;
        const long long waves = (ctas + ctx->num_sms - 1) / ctx->num_sms;
        const double eff = (double)ctas / (double)(waves * ctx->num_sms);
        if (eff > best + 1e-9) { best = eff; splits = s; }
        if (eff >= 0.97 && waves >= 2) { splits = s; break; }
    }
    // autotuner candidates: the wave rule's count (0), half of it (1), twice it (2)
    if (scale_splits == 1) splits = std::max(1, splits / 2);
    if (scale_splits == 2) splits = std::min(std::max(1, kb_total / 4), 2 * splits);
    const int kbs = cdiv(kb_total, splits);
    splits = cdiv(kb_total, kbs);
    RS_TRY(partials(ctx, (size_t)splits * M * N));
    RS_CUDA(ctx, cudaMemsetAsync(ctx->ws.tcerr, 0, sizeof(int), st));
    static const cudaError_t attr = cudaFuncSetAttribute(k_gram_pl, cudaFuncAttributeMaxDynamicSharedMemorySize, GSMEM);
    RS_CUDA(ctx, attr);
    {
        const double frac = blk_rows > 0 ? (double)active / ((double)tn * tm) : 1.0;
        const double K = 2.0 * (double)ctx->n;   // real products per complex entry pair
        ProfScope ps(ctx, RSDFT_K_GRAM_TC, 3.0 * 2.0 * 2.0 * (double)M * N * K * frac,
                     2.0 * 2.0 * K * (double)(M + N), st);
        k_gram_pl<<<dim3(tn, tm, splits), GTHREADS, GSMEM, st>>>(mAh, mAl, mBh, mBl, M, N, b.ldh, kb_total, kbs,
                                                                   tpb, blk_rows, ctx->ws.tcpart, ctx->ws.tcerr);
    }
    RS_LAUNCHED(ctx, "k_gram_pl");
    *splits_out = splits;
    return RSDFT_OK;
}

static rsdft_status check_err(rsdft_ctx *ctx, cudaStream_t st) {
    int *slot = reinterpret_cast<int *>(ctx->ws.hbuf + ctx->ws.hbuf_elems - 24);
    RS_CUDA(ctx, cudaMemcpyAsync(slot, ctx->ws.tcerr, sizeof(int), cudaMemcpyDeviceToHost, st));
    RS_CUDA(ctx, cudaStreamSynchronize(st));
    if (*slot) return fail(ctx, RSDFT_E_TIMEOUT, "tensor-core GEMM: an mbarrier wait timed out");
    return RSDFT_OK;
}

// Coefficient operands of one rotation: [W P] part and X part, hi and lo.
struct RotCoef {
    __nv_bfloat16 *wph, *wpl, *xh, *xl;
    int kpad_wp, kpad_x;
};

// One rotation out0 = base + sign (X C_X + WP C_WP), out1 = WP C_WP (when kwp > 0):
// X = kx split rows at (xh, xl), WP = kwp split rows at (wph, wpl); C rows
// [0, kx) multiply X, rows [kx, kx + kwp) multiply WP; ncol output bands.
struct RotSpec {
    const __nv_bfloat16 *xh, *xl, *wph, *wpl;
    int ldh;
    long long ld;
    int kx, kwp;
    const double2 *c;
    int ldc, ncol;
    float2 *out0, *out1;
    const float2 *base;
    int sign;
};

static rsdft_status rot_coef(rsdft_ctx *ctx, const RotSpec &sp, int nh, RotCoef &rc, cudaStream_t st) {
    Workspace &w = ctx->ws;
    rc.kpad_wp = cdiv(sp.kwp, RK) * RK;
    rc.kpad_x = cdiv(sp.kx, RK) * RK;
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
    const long long n = ctx->n;
    CUtensorMap mWPh, mWPl, mXh, mXl, mBWPh, mBWPl, mBXh, mBXl;
    const CUtensorMapSwizzle S128 = CU_TENSOR_MAP_SWIZZLE_128B, S64 = CU_TENSOR_MAP_SWIZZLE_64B;
    RS_TRY(make_map(ctx, &mXh, sp.xh, sp.ld, sp.kx, sp.ld, 64, RK, S128));
    RS_TRY(make_map(ctx, &mXl, sp.xl, sp.ld, sp.kx, sp.ld, 64, RK, S128));
    RS_TRY(make_map(ctx, &mBXh, rc.xh, rc.kpad_x, 2 * nh, rc.kpad_x, RK, nh, S64));
    RS_TRY(make_map(ctx, &mBXl, rc.xl, rc.kpad_x, 2 * nh, rc.kpad_x, RK, nh, S64));
    if (sp.kwp > 0) {
        RS_TRY(make_map(ctx, &mWPh, sp.wph, sp.ld, sp.kwp, sp.ld, 64, RK, S128));
        RS_TRY(make_map(ctx, &mWPl, sp.wpl, sp.ld, sp.kwp, sp.ld, 64, RK, S128));
        RS_TRY(make_map(ctx, &mBWPh, rc.wph, rc.kpad_wp, 2 * nh, rc.kpad_wp, RK, nh, S64));
        RS_TRY(make_map(ctx, &mBWPl, rc.wpl, rc.kpad_wp, 2 * nh, rc.kpad_wp, RK, nh, S64));
    } else {
        mWPh = mXh;   // never read: the [W P] phase has no k-blocks
        mWPl = mXl;
        mBWPh = mBXh;
        mBWPl = mBXl;
    }
    RS_TRY(partials(ctx, 0));
    RS_CUDA(ctx, cudaMemsetAsync(ctx->ws.tcerr, 0, sizeof(int), st));
    const int stages = rot_stages(nh);
    const int smem = stages * rot_stage_bytes(nh) + 1024;
    {
        static std::mutex mu;
        static int attr = 0;
        std::lock_guard<std::mutex> g(mu);
        if (attr < smem) {
            RS_CUDA(ctx, cudaFuncSetAttribute(k_rot_pl, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            attr = smem;
        }
    }
    const int ntiles = (int)((n + 127) / 128);
    const int grid = std::min(ntiles, ctx->num_sms);
    const int k = sp.kx + sp.kwp;
    {
        ProfScope ps(ctx, RSDFT_K_ROTATE_TC, 3.0 * 8.0 * (double)n * sp.ncol * k,
                     2.0 * 2.0 * 2.0 * (double)k * n +
                         8.0 * (double)sp.ncol * n * ((sp.out1 ? 2.0 : 1.0) + (sp.base ? 1.0 : 0.0)),
                     st);
        k_rot_pl<<<grid, RTHREADS, smem, st>>>(mWPh, mWPl, mXh, mXl, mBWPh, mBWPl, mBXh, mBXl, nh, sp.ncol,
                                                rc.kpad_wp / RK, rc.kpad_x / RK, sp.ldh, n, ntiles, stages,
                                                sp.out0, sp.out1, sp.base, (float)sp.sign, ctx->ws.tcerr);
    }
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_rot_pl");
    return check_err(ctx, st);
}

// More output bands than one TMEM accumulator pair holds (MAX_NH): the bands go
// in chunks of at most MAX_NH (multiples of 16, balanced), one launch each;
// every chunk reads all the split rows of Y again.
static rsdft_status rotate_chunked(rsdft_ctx *ctx, const RotSpec &sp, cudaStream_t st) {
    if (sp.ncol <= MAX_NH) return rotate_launch(ctx, sp, st);
    const int nchunk = cdiv(sp.ncol, MAX_NH);
    const int mc = cdiv(cdiv(sp.ncol, nchunk), 16) * 16;
    const long long n = ctx->n;
    for (int b0 = 0; b0 < sp.ncol; b0 += mc) {
        RotSpec c = sp;
        c.c = sp.c + b0;
        c.ncol = std::min(mc, sp.ncol - b0);
        c.out0 = sp.out0 ? sp.out0 + (size_t)b0 * n : nullptr;
        c.out1 = sp.out1 ? sp.out1 + (size_t)b0 * n : nullptr;
        c.base = sp.base ? sp.base + (size_t)b0 * n : nullptr;
        RS_TRY(rotate_launch(ctx, c, st));
    }
    return RSDFT_OK;
}

// Ritz rotation of split rows row0 .. row0 + k of b's B region (X = the first m rows).
static rsdft_status rotate_rows(rsdft_ctx *ctx, const Buffers &b, int row0, int k, const double2 *c, int ldc,
                                int m, float2 *out0, float2 *out1, cudaStream_t st) {
    RotSpec sp;
    sp.xh = b.bh + (size_t)row0 * b.ld;
    sp.xl = b.bl + (size_t)row0 * b.ld;
    sp.wph = b.bh + (size_t)(row0 + m) * b.ld;
    sp.wpl = b.bl + (size_t)(row0 + m) * b.ld;
    sp.ldh = b.ldh;
    sp.ld = b.ld;
    sp.kx = m;
    sp.kwp = k - m;
    sp.c = c;
    sp.ldc = ldc;
    sp.ncol = m;
    sp.out0 = out0;
    sp.out1 = out1;
    sp.base = nullptr;
    sp.sign = 1;
    return rotate_chunked(ctx, sp, st);
}

}  // namespace tc

// G_S = <Y|Y>, G_H = <Y|HY> (Hermitised, scaled by dV) for FP32 blocks on the
// tensor cores: one GEMM of A = Y against B = [Y; HY] (A is read from the first
// k rows of B).  The split rows stay in the workspace for the Ritz rotation
// (rotate_tc_split).
rsdft_status gram_tc_sh(rsdft_ctx *ctx, const RowBlocksT<float2> &Y, const RowBlocksT<float2> &HY,
                        double2 *gs, double2 *gh, int ld, cudaStream_t st) {
    const int k = Y.cnt[0] + Y.cnt[1] + Y.cnt[2];
    if (k <= 0) return RSDFT_OK;
    tc::Buffers b;
    RS_TRY(tc::buffers(ctx, 0, 2 * k, b));
    b.ah = b.bh;   // A = the first k rows of B
    b.al = b.bl;
    RS_TRY(tc::split_rows(ctx, Y, b.bh, b.bl, 0, b.ldh, st));
    RS_TRY(tc::split_rows(ctx, HY, b.bh, b.bl, k, b.ldh, st));
    auto run = [&](int cand) -> rsdft_status {
        int splits = 0;
        RS_TRY(tc::gemm(ctx, b, k, 2 * k, st, &splits, k, cand));
        tc::k_gram_pl_reduce_sh<<<cdiv((long long)k * k, 256), 256, 0, st>>>(ctx->ws.tcpart, splits, k, ctx->dV,
                                                                              gs, gh, ld);
        count_launch(ctx);
        RS_LAUNCHED(ctx, "k_gram_pl_reduce_sh");
        return RSDFT_OK;
    };
    int chosen = 0;
    RS_TRY(autotune_pick(ctx, "gramtc " + std::to_string(cdiv(k, 32)), 3, 0, st, run, &chosen));
    return tc::check_err(ctx, st);
}

// General G = <A|B> (na x nb) for FP32 blocks on the tensor cores.
rsdft_status gram_tc(rsdft_ctx *ctx, const RowBlocksT<float2> &A, const RowBlocksT<float2> &B,
                     double2 *g, int ld, cudaStream_t st) {
    const int na = A.cnt[0] + A.cnt[1] + A.cnt[2], nb = B.cnt[0] + B.cnt[1] + B.cnt[2];
    if (na <= 0 || nb <= 0) return RSDFT_OK;
    tc::Buffers b;
    RS_TRY(tc::buffers(ctx, na, nb, b));
    RS_TRY(tc::split_rows(ctx, A, b.ah, b.al, 0, b.ldh, st));
    RS_TRY(tc::split_rows(ctx, B, b.bh, b.bl, 0, b.ldh, st));
    int splits = 0;
    RS_TRY(tc::gemm(ctx, b, na, nb, st, &splits));
    tc::k_gram_pl_reduce<<<cdiv((long long)na * nb, 256), 256, 0, st>>>(ctx->ws.tcpart, splits, na, nb, ctx->dV,
                                                                        g, ld);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_gram_pl_reduce");
    return tc::check_err(ctx, st);
}

// W <- W - X C (C = <X|W>, m x na, ld na) on the tensor cores, from the X split
// rows that the preceding gram_tc(X, W) left in the A region of the workspace.
rsdft_status rotate_tc_ortho(rsdft_ctx *ctx, int m, int na, const double2 *c, float2 *w, cudaStream_t st) {
    if (m < 1 || na < 1)
        return fail(ctx, RSDFT_E_INVALID, "tensor-core orthogonalisation: m %d, na %d", m, na);
    tc::Buffers b;
    RS_TRY(tc::buffers(ctx, m, na, b));   // the layout gram_tc(X, W) wrote
    tc::RotSpec sp;
    sp.xh = b.ah;
    sp.xl = b.al;
    sp.wph = sp.wpl = nullptr;
    sp.ldh = b.ldh;
    sp.ld = b.ld;
    sp.kx = m;
    sp.kwp = 0;
    sp.c = c;
    sp.ldc = na;
    sp.ncol = na;
    sp.out0 = w;
    sp.out1 = nullptr;
    sp.base = w;
    sp.sign = -1;
    return tc::rotate_chunked(ctx, sp, st);
}

bool rotate_tc_fits(int k, int m) { return m >= 1 && k > m; }

rsdft_status rotate_tc_split(rsdft_ctx *ctx, int which, int k, const double2 *c, int ldc, int m,
                             float2 *out0, float2 *out1, cudaStream_t st) {
    // k == m (X only, no new P) is allowed when out1 is NULL
    const bool ok = rotate_tc_fits(k, m) || (k == m && !out1 && m >= 1);
    if (!ok) return fail(ctx, RSDFT_E_INVALID, "tensor-core rotation: k %d, m %d", k, m);
    tc::Buffers b;
    RS_TRY(tc::buffers(ctx, 0, 2 * k, b));   // the layout gram_tc_sh wrote: [Y; HY]
    return tc::rotate_rows(ctx, b, which == 0 ? 0 : k, k, c, ldc, m, out0, out1, st);
}

rsdft_status rotate_tc(rsdft_ctx *ctx, const float2 *y, int k, const double2 *c, int ldc, int m,
                       float2 *out0, float2 *out1, cudaStream_t st) {
    if (!rotate_tc_fits(k, m)) return fail(ctx, RSDFT_E_INVALID, "tensor-core rotation: k %d, m %d", k, m);
    tc::Buffers b;
    RS_TRY(tc::buffers(ctx, 0, k, b));
    RowBlocksT<float2> Y{{y, nullptr, nullptr}, {k, 0, 0}};
    RS_TRY(tc::split_rows(ctx, Y, b.bh, b.bl, 0, b.ldh, st));
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

extern "C" rsdft_status rsdft_gram_sh_bf16x3(rsdft_ctx *ctx, const void *y_dev, const void *hy_dev, int k,
                                             void *gs_dev, void *gh_dev, void *stream) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (k < 0 || (k > 0 && (!y_dev || !hy_dev || !gs_dev || !gh_dev)))
        return fail(ctx, RSDFT_E_INVALID, "bad gram arguments");
    RS_TRY(ensure_workspace(ctx, 1));
    RowBlocksT<float2> Y{{(const float2 *)y_dev, nullptr, nullptr}, {k, 0, 0}};
    RowBlocksT<float2> HY{{(const float2 *)hy_dev, nullptr, nullptr}, {k, 0, 0}};
    return gram_tc_sh(ctx, Y, HY, (double2 *)gs_dev, (double2 *)gh_dev, k, as_stream(stream));
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
