// Real-time propagation of the orbitals (RS-TDDFT, the application the paper's
// real-space code is built for): psi <- exp(-i H dt) psi by the truncated Taylor
// series of the exponential, term by term on the FFT H psi of fft.cu:
//   T_0 = psi,  T_j = (-i dt / j) H T_{j-1},  psi_new = sum_{j <= order} T_j.
// Each term is one batched H psi over all bands and one fused pass that scales
// H T_{j-1} into T_j and adds it to psi.  FP64; V is held fixed over the call.
#include <algorithm>
#include <cmath>

#include "rsdft_internal.h"

namespace rsdft {

// t = c h with c = -i a (a real), psi += t, t kept for the next term
__global__ void k_taylor_term(double2 *__restrict__ t, const double2 *__restrict__ h, double2 *__restrict__ psi,
                              long long cnt, double a) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (long long)gridDim.x * blockDim.x) {
        const double2 hv = h[i];
        const double2 tv = make_double2(a * hv.y, -a * hv.x);   // -i a (x + i y) = a y - i a x
        t[i] = tv;
        double2 p = psi[i];
        p.x += tv.x;
        p.y += tv.y;
        psi[i] = p;
    }
}

}  // namespace rsdft

using namespace rsdft;

extern "C" rsdft_status rsdft_propagate(rsdft_ctx *ctx, void *psi_dev, int nband, double dt, int nsteps, int order,
                                        void *stream) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (!psi_dev || nband <= 0 || nsteps < 0 || order < 1 || order > 16 || !std::isfinite(dt))
        return fail(ctx, RSDFT_E_INVALID, "bad propagation arguments");
    RS_TRY(ensure_workspace(ctx, nband));
    cudaStream_t st = as_stream(stream);
    double2 *psi = static_cast<double2 *>(psi_dev);
    double2 *t = ctx->ws.W, *ht = ctx->ws.HW;
    const long long cnt = (long long)nband * ctx->n;
    const int grid = std::max(1, std::min(cdiv(cnt, 256), 8 * ctx->num_sms));
    for (int s = 0; s < nsteps; ++s) {
        RS_CUDA(ctx, cudaMemcpyAsync(t, psi, (size_t)cnt * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        for (int j = 1; j <= order; ++j) {
            RS_TRY(apply_h64(ctx, t, ht, nband, st));
            k_taylor_term<<<grid, 256, 0, st>>>(t, ht, psi, cnt, dt / j);
            count_launch(ctx);
            RS_LAUNCHED(ctx, "k_taylor_term");
        }
    }
    return RSDFT_OK;
}
