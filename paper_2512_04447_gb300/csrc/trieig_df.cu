// The lowest eigenvalues of the real symmetric tridiagonal T (diagonal d,
// off-diagonal e) by the multisection of dense.cu with its Sturm counts in
// double-float (dfloat.h).  On GB300 a warp FP64 instruction occupies its
// sub-partition for 64 cycles whether one lane or 32 are active, so the FP64
// kernel is bound by the FP64 issue of its sequential count chains; a
// double-float step costs a few dozen FP32 instructions of one cycle each.
//   - Sturm count: the product form p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2}
//     (p_{-1} = 1); the count is the number of sign changes.  An exact p_i = 0
//     counts as negative (replaced by -p_{i-1} 2^-50); p_i and p_{i-1} are scaled
//     by one power of two when the larger leaves [2^-60, 2^60] (FP32 range).
//   - The bracket stops at 2^-44 ||T|| (the counts are exact for a T perturbed by a
//     few units of 2^-48 relative), against 4 eps ||T|| in FP64.
// The eigenvectors stay with the FP64 inverse iteration: its vectors for
// eigenvalues g apart are orthogonal to ~u ||T|| / g, u the working precision, and
// 2^-46 instead of 2^-53 left them 1e-10 from orthogonal on a test spectrum.
#include "dfloat.h"
#include "rsdft_internal.h"
#include "sturm_df.h"

namespace rsdft {

using namespace dfl;

// df tables after the FP64 ones in scr: d at scr + 8 + k, e^2 at scr + 8 + 2k (one
// float2 per double slot)
__device__ __forceinline__ float2 *df_d(double *scr, int k) { return reinterpret_cast<float2 *>(scr + 8 + k); }
__device__ __forceinline__ float2 *df_e2(double *scr, int k) { return reinterpret_cast<float2 *>(scr + 8 + 2 * k); }

__global__ void k_tri_prep_df(const double *__restrict__ d, const double *__restrict__ e, int k, double *scr) {
    float2 *dt = df_d(scr, k), *et = df_e2(scr, k);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
        const df di = from_double(d[i]);
        dt[i] = make_float2(di.h, di.l);
        if (i < k - 1) {
            const df e2 = sqr(from_double(e[i]));
            et[i] = make_float2(e2.h, e2.l);
        }
    }
}

// One CTA of BISD_T threads per eigenvalue j: each round the threads take Sturm
// counts at BISD_T interior points of [lo, hi] and keep the sub-interval holding
// the j-th eigenvalue (counts > j form a suffix of the points).
constexpr int BISD_T = 256;
__global__ void __launch_bounds__(BISD_T)
k_bisect_df(int k, int nkeep, double *scr, double *__restrict__ lam) {
    const int j = blockIdx.x;
    if (j >= nkeep) return;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    __shared__ unsigned s_ball[BISD_T / 32];
    __shared__ double s_x[BISD_T];
    const float2 *dt = df_d(scr, k), *et = df_e2(scr, k);
    const double step = 1.0 / (double)(BISD_T + 1);
    double lo = scr[1], hi = scr[2];
    const double tol_abs = 0x1p-44 * fmax(scr[0], 1e-300);
    for (int round = 0; round < 40; ++round) {
        if (hi - lo <= tol_abs) break;
        const double x = lo + (hi - lo) * ((double)(t + 1) * step);
        const int c = sturm_count_df(dt, et, k, from_double(x));
        const unsigned ball = __ballot_sync(0xffffffffu, c > j);
        if (lane == 0) s_ball[warp] = ball;
        s_x[t] = x;
        __syncthreads();
        int f = -1;
        for (int w = 0; w < BISD_T / 32; ++w)
            if (s_ball[w]) {
                f = w * 32 + __ffs(s_ball[w]) - 1;
                break;
            }
        if (f < 0) {
            lo = s_x[BISD_T - 1];
        } else {
            if (f > 0) lo = s_x[f - 1];
            hi = s_x[f];
        }
        __syncthreads();
    }
    if (t == 0) lam[j] = 0.5 * (lo + hi);
}

rsdft_status bisect_df(rsdft_ctx *ctx, int k, int nkeep, double *lam_dev, cudaStream_t st) {
    Workspace &w = ctx->ws;
    k_tri_prep_df<<<cdiv(k, 256), 256, 0, st>>>(w.d, w.e, k, w.dscr);
    k_bisect_df<<<nkeep, BISD_T, 0, st>>>(k, nkeep, w.dscr, lam_dev);
    count_launch(ctx, 2);
    RS_LAUNCHED(ctx, "k_bisect_df");
    return RSDFT_OK;
}

}  // namespace rsdft
