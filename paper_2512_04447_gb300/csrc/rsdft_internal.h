// Internal declarations of the rsdft CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cstdio>
#include <cstring>
#include <string>
#include <functional>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/rsdft.h"

namespace rsdft {

constexpr int MAX_N = 128;          // largest grid dimension
constexpr int MAX_STAGES = 8;       // FFT stages per axis

// One axis of the 3D FFT: N = prod radix[s]; stage s works on blocks of
// length len[s] with sub-stride sub[s] = len[s] / radix[s].  Forward stages run
// in order (decimation in frequency, natural order in, digit-reversed out),
// inverse stages in reverse order (decimation in time, digit-reversed in,
// natural out), so a forward-scale-inverse round trip needs no reordering.
struct AxisPlan {
    int N;
    int nstage;
    int radix[MAX_STAGES];
    int len[MAX_STAGES];
    int sub[MAX_STAGES];
    // multiply-high divisors: x / d == __umulhi(x, mag) for x < 2^16 (mag = 0 for d = 1)
    unsigned nmag;                  // d = N
    unsigned submag[MAX_STAGES];    // d = sub[s]
    unsigned bfmag[MAX_STAGES];     // d = N / radix[s]
};

struct Fft3Plan {
    AxisPlan ax[3];          // x, y, z
    const double2 *tw64[3];  // [N] exp(-2 pi i k / N), device
    const float2 *tw32[3];
    const double *g2pos[3];  // G_a^2 at each digit-reversed position, device
    const float *g2pos32[3];
    const double *gpos[3];   // G_a at each digit-reversed position (0 on the
                             // Nyquist plane of an even axis), device
};

// Device views handed to kernels (T = double for the FP64 form, float for the
// FP32 data path of the mixed form; the index arrays are shared).
template <typename T> struct ProjT {
    int natom, nproj;
    const int *a_start;      // [natom+1] atom-major entry ranges
    const int *a_idx;        // [nent] grid index
    const T *a_beta;         // [nent][4] beta values (unused slots 0)
    const int *c_rowptr;     // [n+1] point-major CSR
    const int *c_atom;       // [nent]
    const T *c_beta;         // [nent][4]
    const T *e_kb;           // [natom*nproj]
};
using ProjTables = ProjT<double>;

struct Workspace {
    int cap_band = 0;        // bands the buffers are sized for
    // orbital-sized buffers, each cap_band * n complex128
    double2 *X = nullptr, *HX = nullptr, *W = nullptr, *HW = nullptr, *P = nullptr,
            *HP = nullptr, *T1 = nullptr, *Xn = nullptr, *HXn = nullptr, *Pn = nullptr,
            *HPn = nullptr;
    float2 *Xs = nullptr;    // FP32 orbital block of the mixed form [cap_band][n]
    // projector coefficients [cap_band][natom*nproj]
    double2 *proj = nullptr;
    // subspace: k = 3 * cap_band
    int cap_k = 0;
    double2 *GS = nullptr, *GH = nullptr, *C = nullptr, *Cfull = nullptr;
    double2 *gram_part = nullptr;  size_t gram_part_elems = 0;
    // dense core scratch
    double2 *Lm = nullptr, *Km = nullptr, *Ym = nullptr, *Vh = nullptr, *Zc = nullptr;
    double2 *tau = nullptr, *wv = nullptr;
    double2 *Tw = nullptr;   // compact-WY T factors of the reflector blocks [k/32][32][32]
    double *d = nullptr, *e = nullptr, *lam = nullptr, *zt = nullptr, *dscr = nullptr;
    double *fac = nullptr;   // inverse-iteration factors and vector [k][6][k] (shared-memory overflow)
    int *drop = nullptr, *keep = nullptr, *ikeep = nullptr;
    unsigned int *gsync = nullptr;  // grid-barrier state of the cooperative kernels
    // tensor-core Gram: BF16 hi/lo operands, FP32 split partials, error flag
    void *tcbuf = nullptr;  size_t tc_bytes = 0;
    float2 *tcpart = nullptr;  size_t tcpart_elems = 0;   // tensor-core split-K partials (complex)
    int *tcerr = nullptr;
    void *tcrot = nullptr;  size_t tcrot_bytes = 0;   // split rotation coefficients
    // per-band vectors [cap_band]
    double *theta = nullptr, *res = nullptr, *vexp = nullptr, *tkin = nullptr, *nrm = nullptr;
    int *act = nullptr;      // [active bands (m) | P columns kept (m)]
    double *hbuf = nullptr;  // pinned host scratch
    size_t hbuf_elems = 0;
};

struct ScfWork {
    int ready = 0;
    int nband = 0;
    int step = 0;
    double *rho_in = nullptr, *rho_out = nullptr, *vh = nullptr, *eps = nullptr, *vxc = nullptr;
    double *veff = nullptr;
    double *hist_rho = nullptr, *hist_f = nullptr;   // [depth+1][n]
    int hist_count = 0, hist_cap = 0;
    double *f = nullptr, *eig = nullptr;             // [nband]
    double *red = nullptr;                           // reduction scratch
    double2 *cbuf = nullptr;                         // [n] complex scratch (FFT)
    double *gga = nullptr;                           // [4][n] PBE: grad rho, then the flux terms
};

// Learned preconditioner: weights, Adam state and scratch (precond_nn.cu).
struct NnState {
    int ready = 0;                   // weights set
    float *w = nullptr, *wt = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;   // [RSDFT_NN_WEIGHTS] each
    float *vhat = nullptr;           // [n] standardised potential
    double *dred = nullptr;          // reduction scratch
    float *act = nullptr;  size_t act_cap = 0;     // inference activations
    float *part = nullptr; size_t part_cap = 0;    // weight-gradient partials
    float *bs = nullptr;   size_t bs_cap = 0;      // band scales
    float *tr = nullptr;   size_t tr_cap = 0;      // training activations and gradients
};

struct Profiler {
    bool on = false;
    struct Rec { cudaEvent_t a, b; int id; double flops, bytes; };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    double ms[RSDFT_K_COUNT] = {}, flops[RSDFT_K_COUNT] = {}, bytes[RSDFT_K_COUNT] = {};
    long long count[RSDFT_K_COUNT] = {};
};

}  // namespace rsdft

struct rsdft_ctx {
    int N[3];
    double L[3];
    long long n;
    double dV;
    int num_sms = 1;                 // SMs of the device the context was made on
    rsdft::Fft3Plan fft;
    std::vector<void *> owned;       // device allocations freed at destroy
    double *vloc = nullptr;          // [n] the V_loc given at create
    double *v = nullptr;             // [n] potential used by H
    float *v32 = nullptr;            // [n] FP32 copy of v for the mixed form
    rsdft::ProjTables pt{};
    rsdft::ProjT<float> pt32{};
    long long nent = 0;
    rsdft::Workspace ws;
    rsdft::ScfWork scf;
    rsdft::Profiler prof;
    rsdft::NnState nn;
    long long launches = 0;          // every kernel launched on this context
    long long coop_fallbacks = 0;    // tridiagonalisations that could not launch cooperatively
    int coop_last_error = 0;         // cudaError_t of the last such launch
    int dense_mode = 0;              // rsdft_eigh / rsdft_rayleigh_ritz: RSDFT_DENSE_*
    bool autotune = false;           // time the tile candidates on the first call of a shape
    std::map<std::string, int> tuned;   // shape key -> chosen candidate
    std::string err;
};

namespace rsdft {

// ---- error helpers --------------------------------------------------------
rsdft_status fail(rsdft_ctx *ctx, rsdft_status st, const char *fmt, ...);
rsdft_status cuda_check(rsdft_ctx *ctx, cudaError_t e, const char *what);
#define RS_CUDA(ctx, call)                                                     \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) return ::rsdft::cuda_check((ctx), e_, #call);   \
    } while (0)
#define RS_LAUNCHED(ctx, what)                                                 \
    do {                                                                       \
        cudaError_t e_ = cudaGetLastError();                                   \
        if (e_ != cudaSuccess) return ::rsdft::cuda_check((ctx), e_, what);    \
    } while (0)
#define RS_TRY(expr)                                                           \
    do {                                                                       \
        rsdft_status s_ = (expr);                                              \
        if (s_ != RSDFT_OK) return s_;                                         \
    } while (0)

rsdft_status dev_alloc(rsdft_ctx *ctx, void **p, size_t bytes);

// Brackets the launches of one hot kernel with CUDA events when profiling is
// on; always counts the launches.
struct ProfScope {
    rsdft_ctx *ctx;
    cudaStream_t st;
    int id;
    double flops, bytes;
    cudaEvent_t a = nullptr;
    ProfScope(rsdft_ctx *c, int kid, double fl, double by, cudaStream_t s, int nlaunch = 1);
    ~ProfScope();
};
inline void count_launch(rsdft_ctx *ctx, int n = 1) { ctx->launches += n; }
rsdft_status ensure_workspace(rsdft_ctx *ctx, int nband);
inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }
inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// ---- FFT / H psi (fft.cu) ---------------------------------------------------
enum class Mid { Kinetic, Tpa, Hartree, Scale, GradX, GradY, GradZ };
enum class Src { Plain, Residual, RealField };
// Forward xy-plane pass: src -> dst ([nb][n] complex).  Src::Residual reads
// hx[act[b]] - theta[act[b]] x[act[b]]; Src::RealField reads a real [n] field
// (nb must be 1).
rsdft_status fft_xy_forward(rsdft_ctx *ctx, Src kind, const double2 *src, const double2 *src2,
                            const double *theta, const int *act, const double *rsrc,
                            double2 *dst, int nb, cudaStream_t st);
// z pass: forward z FFT, multiply by the Mid factor, inverse z FFT (in place).
rsdft_status fft_z_mid(rsdft_ctx *ctx, Mid mid, double2 *buf, const double *tkin, int nb,
                       cudaStream_t st);
// Inverse xy pass.  When psi != nullptr: out = T psi + V psi + NL(p) (H psi);
// else out = buf transformed (plain).  When rout != nullptr (nb == 1) the real
// part is written to rout instead.
rsdft_status fft_xy_inverse(rsdft_ctx *ctx, const double2 *buf, const double2 *psi,
                            const double2 *p, double2 *out, double *rout, int nb,
                            cudaStream_t st);
rsdft_status project(rsdft_ctx *ctx, const double2 *psi, double2 *p, int nb, cudaStream_t st);
rsdft_status apply_h64(rsdft_ctx *ctx, const double2 *psi, double2 *hpsi, int nb,
                       cudaStream_t st);
// FP32 data path of the mixed form
rsdft_status fft_xy_forward32(rsdft_ctx *ctx, Src kind, const float2 *src, const float2 *src2,
                              const double *theta, const int *act, float2 *dst, int nb,
                              cudaStream_t st);
rsdft_status fft_z_mid32(rsdft_ctx *ctx, Mid mid, float2 *buf, const double *tkin, int nb,
                         cudaStream_t st);
rsdft_status fft_xy_inverse32(rsdft_ctx *ctx, const float2 *buf, const float2 *psi,
                              const float2 *p, float2 *out, int nb, cudaStream_t st);
rsdft_status project32(rsdft_ctx *ctx, const float2 *psi, float2 *p, int nb, cudaStream_t st);
rsdft_status apply_h32(rsdft_ctx *ctx, const float2 *psi, float2 *hpsi, int nb, cudaStream_t st);
rsdft_status refresh_v32(rsdft_ctx *ctx, cudaStream_t st);

// ---- GEMM-shaped kernels (gemm.cu) -------------------------------------------
template <typename V> struct RowBlocksT {
    const V *ptr[3];
    int cnt[3];
};
using RowBlocks = RowBlocksT<double2>;
// g[i][j] = scale * sum_r conj(A_i) B_j over rows of A (na) and B (nb).
// hermitian: A and B index the same basis; only tiles with ti <= tj are formed
// and g is completed as a Hermitian matrix.  ldg = leading dimension of g.
rsdft_status gram(rsdft_ctx *ctx, const RowBlocks &A, const RowBlocks &B, double2 *g, int ldg,
                  bool hermitian, double scale, cudaStream_t st);
// out1 (optional) = sum over blocks 1..2 of c rows; out0 = out1 + block-0 part
// (+ sign * ... and base handling as in rsdft_rotate).  c is [k][ldc].
rsdft_status rotate(rsdft_ctx *ctx, const RowBlocks &Y, const double2 *c, int ldc, int m,
                    const double2 *base, int sign, double2 *out0, double2 *out1,
                    cudaStream_t st);
// FP32 operands (mixed form): products and CTA-level sums in FP32, Gram
// partials reduced in FP64; rotation coefficients rounded to FP32.
rsdft_status gram32(rsdft_ctx *ctx, const RowBlocksT<float2> &A, const RowBlocksT<float2> &B,
                    double2 *g, int ldg, bool hermitian, double scale, cudaStream_t st);
// Split-K partial buffer of the Gram kernels (grown when needed) and its FP64
// reduction into g (hermitian: tiles of edge te below the diagonal mirrored).
rsdft_status ensure_gram_partials(rsdft_ctx *ctx, size_t elems);
rsdft_status gram_reduce(rsdft_ctx *ctx, int nsplit, int na, int nb, bool hermitian, int te, double scale,
                         double2 *g, int ldg, cudaStream_t st);
// FP64-accurate products on the FP32 pipe (gemm_df.cu): FP64 rows held as
// FP32 hi/lo pairs (split_df), error-free products, TwoSum accumulation.
rsdft_status split_df(rsdft_ctx *ctx, const double2 *x, long long cnt, float2 *h, float2 *l, cudaStream_t st);
// g[i][j] = scale * sum_r conj(A_i) B_j, A = (ah, al) [na][n], B = (bh, bl) row
// blocks (bl all null: B exact in FP32).
rsdft_status gram_df(rsdft_ctx *ctx, const float2 *ah, const float2 *al, int na, const RowBlocksT<float2> &bh,
                     const RowBlocksT<float2> &bl, double2 *g, int ldg, double scale, cudaStream_t st);
// out[b] = sum_{i < k} c[i][b] Y_i, Y = (yh, yl) [k][n], c [k][ldc] FP64, out [m][n] FP64.
rsdft_status rotate_df(rsdft_ctx *ctx, const float2 *yh, const float2 *yl, int k, const double2 *c, int ldc, int m,
                       double2 *out, cudaStream_t st);
rsdft_status rotate32(rsdft_ctx *ctx, const RowBlocksT<float2> &Y, const double2 *c, int ldc, int m,
                      const float2 *base, int sign, float2 *out0, float2 *out1, cudaStream_t st);
// Tensor-core (split-BF16, tcgen05) Grams of FP32 blocks (gram_tc.cu).
rsdft_status gram_tc_sh(rsdft_ctx *ctx, const RowBlocksT<float2> &Y, const RowBlocksT<float2> &HY,
                        double2 *gs, double2 *gh, int ld, cudaStream_t st);
rsdft_status gram_tc(rsdft_ctx *ctx, const RowBlocksT<float2> &A, const RowBlocksT<float2> &B,
                     double2 *g, int ld, cudaStream_t st);
// Ritz rotation on the tensor cores from the split-BF16 rows that the last
// gram_tc_sh left in the workspace (which = 0: Y, which = 1: HY):
// out0 = Y C (all k rows), out1 = Y[m:k] C[m:k] (the new P).  rotate_tc_fits
// says whether the shape is supported (k > m >= 1; more than 240 bands go in
// groups of at most 240).
bool rotate_tc_fits(int k, int m);
rsdft_status rotate_tc_split(rsdft_ctx *ctx, int which, int k, const double2 *c, int ldc, int m,
                             float2 *out0, float2 *out1, cudaStream_t st);
// W <- W - X C (C = <X|W>, m x na) from the X split rows that the preceding
// gram_tc(X, W) left in the workspace.
rsdft_status rotate_tc_ortho(rsdft_ctx *ctx, int m, int na, const double2 *c, float2 *w, cudaStream_t st);
// Same for an arbitrary FP32 block y [k][n] (splits it first).
rsdft_status rotate_tc(rsdft_ctx *ctx, const float2 *y, int k, const double2 *c, int ldc, int m,
                       float2 *out0, float2 *out1, cudaStream_t st);

// ---- autotuner (context.cu) --------------------------------------------------
// With ctx->autotune set, the first call of a shape runs each candidate once
// untimed and twice timed with CUDA events on the stream, and remembers the one
// with the fastest timed run under `key` (later calls reuse it; without
// autotune the closed-form choice is used).  run(i) launches candidate i; the
// winner is run last so that its result is the one left in the outputs.  Only
// for calls whose outputs do not alias inputs.
rsdft_status autotune_pick(rsdft_ctx *ctx, const std::string &key, int ncand, int fallback, cudaStream_t st,
                           const std::function<rsdft_status(int)> &run, int *chosen);

// ---- dense core (dense.cu) ----------------------------------------------------
// Held from a cooperative launch until the stream that launched it has
// synchronised: cooperative grids of different contexts never overlap.
std::mutex &coop_mutex();
// df: the double-float cluster tridiagonalisation where it fits (tridiag_cl.cu)
rsdft_status rayleigh_ritz(rsdft_ctx *ctx, const double2 *gh, const double2 *gs, int k,
                           int nkeep, double pivot_tol, double *lam_dev, double2 *c_out,
                           int *ndropped, cudaStream_t st, bool df = false);
rsdft_status eigh_lowest(rsdft_ctx *ctx, double2 *a, int k, int nkeep, double *lam_dev,
                         double2 *z, int ldz, cudaStream_t st, bool df = false);
// Householder tridiagonalisation of the Hermitian a (k x k, ld) in double-float
// on one 16-CTA cluster; *done = false (and nothing launched) where k does not
// fit in the cluster's shared memory or the cluster launch is refused.
bool tridiag_cluster_fits(int k);
// Lowest nkeep eigenvalues (lam_dev) of the tridiagonal ws.d, ws.e by
// multisection on double-float Sturm counts; ws.dscr must hold k_tri_prep's norm
// and bracket (trieig_df.cu).
rsdft_status bisect_df(rsdft_ctx *ctx, int k, int nkeep, double *lam_dev, cudaStream_t st);
// L (kc x kc, FP64) to double-float rows, and the column-parallel triangular
// solves L X = B (back = false) or L^H X = B (back = true) on them (trsm_df.cu)
rsdft_status to_df(rsdft_ctx *ctx, const double2 *L, int ldl, int kc, float4 *out, cudaStream_t st);
rsdft_status trsm_df(rsdft_ctx *ctx, bool back, const float4 *L, int kc, double2 *b, int ldb, int ncol,
                     cudaStream_t st);
rsdft_status tridiag_cluster(rsdft_ctx *ctx, const double2 *a, int k, int ld, double2 *vh, int ldv, double2 *tau,
                             double *d, double *e, cudaStream_t st, bool *done);

// ---- small vector kernels (lobpcg.cu / scf.cu) ----------------------------------
rsdft_status colnorms(rsdft_ctx *ctx, const double2 *a, int nb, double *out, cudaStream_t st);

// W[b] += s_b NN(R_b / s_b) (the learned preconditioner's correction) for the
// nb compact rows of R; requires weights (RSDFT_E_INVALID otherwise).
template <typename V>
rsdft_status learned_correction(rsdft_ctx *ctx, const V *R, int nb, V *W, cudaStream_t st);

}  // namespace rsdft
