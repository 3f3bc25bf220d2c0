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
          int N, int kb_total, int kb_per_split, float *__restrict__ part, int *err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[STAGES];
    __shared__ __align__(8) uint64_t empty_bar[STAGES];
    __shared__ __align__(8) uint64_t acc_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    const int tn = blockIdx.x, tm = blockIdx.y, split = blockIdx.z;
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
            tma_load_2d(st + 2 * TILE_BYTES, &mBh, &full_bar[s], kx, tn * BN);
            tma_load_2d(st + 3 * TILE_BYTES, &mBl, &full_bar[s], kx, tn * BN);
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
            float *dst = part + ((size_t)split * M + row) * N + (size_t)tn * BN + c0;
            const int cmax = min(32, N - (tn * BN + c0));
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
// C = A [Y; Yrot; HY; HYrot]^T (N = 4k): Hermitised, scaled by dV, FP64 sums.
__global__ void k_gram_tc_reduce_sh(const float *__restrict__ part, int splits, int k, double scale,
                                    double2 *__restrict__ gs, double2 *__restrict__ gh, int ld) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)k * k) return;
    const int i = (int)(idx / k), j = (int)(idx % k);
    const size_t N = 4 * (size_t)k, plane = (size_t)k * N;
    double sr = 0, si = 0, hr = 0, hi = 0;
    for (int s = 0; s < splits; ++s) {
        const float *pi = part + s * plane + (size_t)i * N, *pj = part + s * plane + (size_t)j * N;
        sr += (double)pi[j] + (double)pj[i];
        si += (double)pi[k + j] - (double)pj[k + i];
        hr += (double)pi[2 * k + j] + (double)pj[2 * k + i];
        hi += (double)pi[3 * k + j] - (double)pj[3 * k + i];
    }
    const double h = 0.5 * scale;
    gs[(size_t)i * ld + j] = make_double2(h * sr, h * si);
    gh[(size_t)i * ld + j] = make_double2(h * hr, h * hi);
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

// 2D BF16 operand [rows][ldk] with kvalid valid columns; box 64 x 128, 128-byte swizzle.
static rsdft_status make_map(rsdft_ctx *ctx, CUtensorMap *m, const void *base, long long kvalid,
                             int rows, long long ldk) {
    if ((reinterpret_cast<uintptr_t>(base) & 15u) || ((ldk * 2) & 15))
        return fail(ctx, RSDFT_E_INVALID, "tensor map base or stride not 16-byte aligned");
    cuuint64_t dims[2] = {(cuuint64_t)kvalid, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ldk * 2)};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)BM};
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

// C = A B^T over K = 2n for A rows [0, M), B rows [0, N) already split; returns splits.
static rsdft_status gemm(rsdft_ctx *ctx, const Buffers &b, int M, int N, cudaStream_t st, int *splits_out) {
    RS_TRY(encoder(ctx));
    const long long K = 2 * ctx->n;
    CUtensorMap mAh, mAl, mBh, mBl;
    RS_TRY(make_map(ctx, &mAh, b.ah, K, M, b.ldk));
    RS_TRY(make_map(ctx, &mAl, b.al, K, M, b.ldk));
    RS_TRY(make_map(ctx, &mBh, b.bh, K, N, b.ldk));
    RS_TRY(make_map(ctx, &mBl, b.bl, K, N, b.ldk));
    const int tn = cdiv(N, BN), tm = cdiv(M, BM);
    const int kb_total = (int)((K + BK - 1) / BK);
    // splits: whole waves of one CTA per SM, at least 8 k-blocks per CTA
    int splits = 1;
    double best = 0.0;
    for (int s = 1; s <= 256 && s <= kb_total; ++s) {
        if (s > 1 && kb_total / s < 8) break;
        const long long ctas = (long long)tn * tm * s;
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
        ProfScope ps(ctx, RSDFT_K_GRAM_TC, 3.0 * 2.0 * (double)M * N * K,
                     4.0 * (double)K * (M + N), st);
        k_gram_tc<<<dim3(tn, tm, splits), THREADS, SMEM_BYTES, st>>>(mAh, mAl, mBh, mBl, M, N, kb_total,
                                                                     kbs, ctx->ws.tcpart, ctx->ws.tcerr);
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

}  // namespace tc

// G_S = <Y|Y>, G_H = <Y|HY> (Hermitised, scaled by dV) for FP32 blocks on the
// tensor cores: one GEMM of A = Y against B = [Y; Yrot; HY; HYrot].
rsdft_status gram_tc_sh(rsdft_ctx *ctx, const RowBlocksT<float2> &Y, const RowBlocksT<float2> &HY,
                        double2 *gs, double2 *gh, int ld, cudaStream_t st) {
    const int k = Y.cnt[0] + Y.cnt[1] + Y.cnt[2];
    if (k <= 0) return RSDFT_OK;
    tc::Buffers b;
    RS_TRY(tc::buffers(ctx, k, 4 * k, b));
    RS_TRY(tc::split_rows(ctx, Y, 0, b.ah, b.al, 0, b.ldk, st));
    RS_TRY(tc::split_rows(ctx, Y, 0, b.bh, b.bl, 0, b.ldk, st));
    RS_TRY(tc::split_rows(ctx, Y, 1, b.bh, b.bl, k, b.ldk, st));
    RS_TRY(tc::split_rows(ctx, HY, 0, b.bh, b.bl, 2 * k, b.ldk, st));
    RS_TRY(tc::split_rows(ctx, HY, 1, b.bh, b.bl, 3 * k, b.ldk, st));
    int splits = 0;
    RS_TRY(tc::gemm(ctx, b, k, 4 * k, st, &splits));
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
