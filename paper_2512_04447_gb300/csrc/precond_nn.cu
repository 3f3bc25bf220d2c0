// Learned preconditioner: TPA plus a small periodic 3D convolutional network
// on the LOBPCG residuals (residual form), its training kernels, and the
// projected-correction targets it is trained on.
//
// Network (the paper gives none; the readings are fixed here and in the
// header): per real plane u of a normalised residual r_b / s_b (Re and Im are
// separate samples: at the Gamma point H is real, so (H - e)^-1 maps them
// independently), input channels (u, u * vhat) with vhat the standardised
// potential, four 3x3x3 periodic convolutions without biases, channels
// 2 -> 8 -> 8 -> 8 -> 1, tanh between them.  w_b = TPA(r_b) + s_b NN(r_b / s_b).
// Weights: layer after layer, each [27][cin][cout] float32, tap = (dz + 1) 9 +
// (dy + 1) 3 + (dx + 1), out[co](p) = sum_ci sum_d w[tap(d)][ci][co] in[ci](p + d).
//
// Kernels.  One CTA computes a 16 x 8 x 4 (x, y, z) output tile of one sample:
// the (18 x 10 x 6) x cin halo tile and the layer's weights go to shared
// memory, thread (x, y) keeps its z column of 4 points x cout accumulators and
// reuses each loaded column of 6 inputs for the three z offsets.  Activations
// are channel planes [sample][c][n] in HBM (coalesced along x).  The backward
// pass uses the same kernel with the flipped, transposed weights (the adjoint
// of a periodic correlation) and a weight-gradient kernel that reduces
// per-CTA partials deterministically.
#include "rsdft_internal.h"

#include <cmath>
#include <vector>

namespace rsdft {
namespace nn {

constexpr int C = RSDFT_NN_HIDDEN;
constexpr int TX = 16, TY = 8, TZ = 4;
constexpr int HXW = TX + 2, HYW = TY + 2, HZW = TZ + 2;
constexpr int HALO = HXW * HYW * HZW;        // 1080 points
constexpr int TILE = TX * TY * TZ;           // 512 points
constexpr int NT = TX * TY;                  // 128 threads
constexpr int OFF1 = 27 * 2 * C, OFF2 = OFF1 + 27 * C * C, OFF3 = OFF2 + 27 * C * C;
constexpr int WCOUNT = OFF3 + 27 * C;
static_assert(WCOUNT == RSDFT_NN_WEIGHTS, "weight count");
constexpr float ADAM_B1 = 0.9f, ADAM_B2 = 0.999f, ADAM_EPS = 1e-8f;

struct Geo {
    int Nx, Ny, Nz;
    int tx, ty, tz;    // tiles per axis
    long long n;
};

static Geo geo_of(const rsdft_ctx *ctx) {
    Geo g;
    g.Nx = ctx->N[0];
    g.Ny = ctx->N[1];
    g.Nz = ctx->N[2];
    g.tx = cdiv(g.Nx, TX);
    g.ty = cdiv(g.Ny, TY);
    g.tz = cdiv(g.Nz, TZ);
    g.n = ctx->n;
    return g;
}

__device__ __forceinline__ void tile_origin(const Geo &g, int &x0, int &y0, int &z0) {
    const int t = blockIdx.x;
    const int tx = t % g.tx, r = t / g.tx;
    x0 = tx * TX;
    y0 = (r % g.ty) * TY;
    z0 = (r / g.ty) * TZ;
}

// a mod N in [0, N) (tiles may overhang grids smaller than a tile)
__device__ __forceinline__ int wrap(int a, int N) {
    const int r = a % N;
    return r < 0 ? r + N : r;
}

// ---- sources of a layer's input channels -------------------------------------
// Layer-1 features from float planes u[idx[s]] (training samples).
struct SrcPlane {
    const float *u;
    const int *idx;      // sample map (nullptr: identity)
    const float *vhat;
    long long n;
    __device__ __forceinline__ void fetch(int s, long long i, float (&v)[2]) const {
        const int q = idx ? idx[s] : s;
        const float a = u[(size_t)q * n + i];
        v[0] = a;
        v[1] = a * vhat[i];
    }
};

// Layer-1 features from a complex residual block: sample g0 + s is the real
// (g < nb) or imaginary (g >= nb) plane of band g mod nb, scaled by 1 / s_b.
template <typename V> struct SrcResid {
    const V *r;
    const float *inv_s;
    const float *vhat;
    int nb, g0;
    long long n;
    __device__ __forceinline__ void fetch(int s, long long i, float (&v)[2]) const {
        const int g = g0 + s;
        const int im = g >= nb, b = g - im * nb;
        const V z = r[(size_t)b * n + i];
        const float a = (float)(im ? z.y : z.x) * inv_s[b];
        v[0] = a;
        v[1] = a * vhat[i];
    }
};

// Channel planes act[s][CIN][n].
template <int CIN> struct SrcAct {
    const float *a;
    long long n;
    __device__ __forceinline__ void fetch(int s, long long i, float (&v)[CIN]) const {
#pragma unroll
        for (int c = 0; c < CIN; ++c) v[c] = a[((size_t)s * CIN + c) * n + i];
    }
};

// ---- epilogues --------------------------------------------------------------
// out[s][co][i] = tanh(acc)
struct EpiTanh {
    float *out;
    long long n;
    template <int COUT> __device__ __forceinline__ float3 put(int s, long long i, const float (&a)[COUT]) const {
#pragma unroll
        for (int c = 0; c < COUT; ++c) out[((size_t)s * COUT + c) * n + i] = tanhf(a[c]);
        return make_float3(0.0f, 0.0f, 0.0f);
    }
    __device__ __forceinline__ void finish(float3) const {}
};

// out[s][co][i] = acc * (1 - act[s][co][i]^2): the adjoint through tanh
struct EpiDtanh {
    float *out;
    const float *act;
    long long n;
    template <int COUT> __device__ __forceinline__ float3 put(int s, long long i, const float (&a)[COUT]) const {
#pragma unroll
        for (int c = 0; c < COUT; ++c) {
            const size_t o = ((size_t)s * COUT + c) * n + i;
            const float t = act[o];
            out[o] = a[c] * (1.0f - t * t);
        }
        return make_float3(0.0f, 0.0f, 0.0f);
    }
    __device__ __forceinline__ void finish(float3) const {}
};

// Training output: p = b + o (into pout) and the per-CTA partials of the loss
// sums <p, y>, <p, p>, <y, y> of the CTA's sample.
struct EpiLoss {
    const float *b, *y;
    const int *idx;
    float *pout;
    double *part;        // [gridDim.y * gridDim.x][3]
    long long n;
    template <int COUT> __device__ __forceinline__ float3 put(int s, long long i, const float (&a)[COUT]) const {
        const int q = idx ? idx[s] : s;
        const float p = b[(size_t)q * n + i] + a[0], yy = y[(size_t)q * n + i];
        pout[(size_t)s * n + i] = p;
        return make_float3(p * yy, p * p, yy * yy);
    }
    __device__ void finish(float3 acc) const;
};

// Inference output: w[b].(x or y) += s_b o for sample g0 + s.
template <typename V> struct EpiAdd {
    V *w;
    const float *sc;
    int nb, g0;
    long long n;
    template <int COUT> __device__ __forceinline__ float3 put(int s, long long i, const float (&a)[COUT]) const {
        const int g = g0 + s;
        const int im = g >= nb, b = g - im * nb;
        V &z = w[(size_t)b * n + i];
        using T = decltype(V{}.x);
        if (im) z.y += (T)(sc[b] * a[0]);
        else z.x += (T)(sc[b] * a[0]);
        return make_float3(0.0f, 0.0f, 0.0f);
    }
    __device__ __forceinline__ void finish(float3) const {}
};

__device__ double block_sum_d(double v) {
    __shared__ double sh[NT / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NT / 32; ++w) t += sh[w];
    return t;
}

__device__ void EpiLoss::finish(float3 acc) const {
    const size_t o = 3 * ((size_t)blockIdx.y * gridDim.x + blockIdx.x);
    double t = block_sum_d((double)acc.x);
    if (threadIdx.x == 0) part[o] = t;
    __syncthreads();
    t = block_sum_d((double)acc.y);
    if (threadIdx.x == 0) part[o + 1] = t;
    __syncthreads();
    t = block_sum_d((double)acc.z);
    if (threadIdx.x == 0) part[o + 2] = t;
}

// ---- the convolution ----------------------------------------------------------
// Loads the halo tile of sample blockIdx.y (channel planes s_in[ci][HALO]).
template <int CIN, class Src>
__device__ __forceinline__ void load_halo(const Src &src, const Geo &g, int x0, int y0, int z0, float *s_in) {
    const int s = blockIdx.y;
    for (int hp = threadIdx.x; hp < HALO; hp += NT) {
        const int hx = hp % HXW, r = hp / HXW;
        const int hy = r % HYW, hz = r / HYW;
        const int x = wrap(x0 + hx - 1, g.Nx), y = wrap(y0 + hy - 1, g.Ny), z = wrap(z0 + hz - 1, g.Nz);
        const long long i = ((long long)z * g.Ny + y) * g.Nx + x;
        float v[CIN];
        src.fetch(s, i, v);
#pragma unroll
        for (int c = 0; c < CIN; ++c) s_in[c * HALO + hp] = v[c];
    }
}

// out = epi(conv(src, w)); grid (tiles, samples), NT threads.
template <int CIN, int COUT, class Src, class Epi>
__global__ void __launch_bounds__(NT) k_conv(Src src, const float *__restrict__ w, Epi epi, Geo g) {
    extern __shared__ float sm[];
    float *s_w = sm;                        // [27][CIN][COUT]
    float *s_in = sm + 27 * CIN * COUT;     // [CIN][HALO]
    int x0, y0, z0;
    tile_origin(g, x0, y0, z0);
    for (int q = threadIdx.x; q < 27 * CIN * COUT; q += NT) s_w[q] = w[q];
    load_halo<CIN>(src, g, x0, y0, z0, s_in);
    __syncthreads();
    const int x = threadIdx.x % TX, y = threadIdx.x / TX;
    float acc[TZ][COUT];
#pragma unroll
    for (int z = 0; z < TZ; ++z)
#pragma unroll
        for (int c = 0; c < COUT; ++c) acc[z][c] = 0.0f;
#pragma unroll 1
    for (int dy = 0; dy < 3; ++dy) {
#pragma unroll 1
        for (int dx = 0; dx < 3; ++dx) {
            const int col0 = (y + dy) * HXW + (x + dx);
#pragma unroll 2
            for (int ci = 0; ci < CIN; ++ci) {
                float col[TZ + 2];
#pragma unroll
                for (int q = 0; q < TZ + 2; ++q) col[q] = s_in[ci * HALO + q * (HYW * HXW) + col0];
#pragma unroll
                for (int dz = 0; dz < 3; ++dz) {
                    const float *wp = s_w + ((dz * 9 + dy * 3 + dx) * CIN + ci) * COUT;
                    float wv[COUT];
#pragma unroll
                    for (int c = 0; c < COUT; ++c) wv[c] = wp[c];
#pragma unroll
                    for (int z = 0; z < TZ; ++z)
#pragma unroll
                        for (int c = 0; c < COUT; ++c) acc[z][c] = fmaf(col[z + dz], wv[c], acc[z][c]);
                }
            }
        }
    }
    const int gx = x0 + x, gy = y0 + y;
    float3 lsum = make_float3(0.0f, 0.0f, 0.0f);
#pragma unroll
    for (int z = 0; z < TZ; ++z) {
        const int gz = z0 + z;
        if (gx < g.Nx && gy < g.Ny && gz < g.Nz) {
            const float3 t = epi.template put<COUT>(blockIdx.y, ((long long)gz * g.Ny + gy) * g.Nx + gx, acc[z]);
            lsum.x += t.x;
            lsum.y += t.y;
            lsum.z += t.z;
        }
    }
    epi.finish(lsum);
}

// Per-CTA partials of dw[tap][ci][co] = sum_p in[ci](p + d) gout[co](p) over the
// CTA's tile (points outside the grid carry gout = 0).
template <int CIN, int COUT, class Src>
__global__ void __launch_bounds__(NT) k_wgrad(Src src, const float *__restrict__ gout, Geo g,
                                              float *__restrict__ part) {
    extern __shared__ float sm[];
    float *s_in = sm;                  // [CIN][HALO]
    float *s_g = sm + CIN * HALO;      // [TILE][COUT]
    int x0, y0, z0;
    tile_origin(g, x0, y0, z0);
    load_halo<CIN>(src, g, x0, y0, z0, s_in);
    const int s = blockIdx.y;
    for (int q = threadIdx.x; q < TILE; q += NT) {
        const int x = q % TX, r = q / TX;
        const int y = r % TY, z = r / TY;
        const int gx = x0 + x, gy = y0 + y, gz = z0 + z;
        const bool in = gx < g.Nx && gy < g.Ny && gz < g.Nz;
        const long long i = ((long long)gz * g.Ny + gy) * g.Nx + gx;
#pragma unroll
        for (int c = 0; c < COUT; ++c) s_g[q * COUT + c] = in ? gout[((size_t)s * COUT + c) * g.n + i] : 0.0f;
    }
    __syncthreads();
    float *dst = part + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * (27 * CIN * COUT);
    for (int item = threadIdx.x; item < 27 * CIN; item += NT) {
        const int tap = item / CIN, ci = item - tap * CIN;
        const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
        float acc[COUT];
#pragma unroll
        for (int c = 0; c < COUT; ++c) acc[c] = 0.0f;
        const float *base = s_in + ci * HALO;
#pragma unroll 1
        for (int z = 0; z < TZ; ++z)
#pragma unroll 1
            for (int y = 0; y < TY; ++y) {
                const float *row = base + ((z + dz) * HYW + (y + dy)) * HXW + dx;
                const float *grow = s_g + ((z * TY + y) * TX) * COUT;
#pragma unroll 4
                for (int x = 0; x < TX; ++x) {
                    const float a = row[x];
#pragma unroll
                    for (int c = 0; c < COUT; ++c) acc[c] = fmaf(a, grow[x * COUT + c], acc[c]);
                }
            }
#pragma unroll
        for (int c = 0; c < COUT; ++c) dst[item * COUT + c] = acc[c];
    }
}

// out[j] = sum over partials (FP64), j < cnt
__global__ void k_sum_parts(const float *__restrict__ part, int nparts, int cnt, float *__restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cnt) return;
    double s = 0.0;
    for (int q = 0; q < nparts; ++q) s += (double)part[(size_t)q * cnt + j];
    out[j] = (float)s;
}

// Per sample s (block s): al = <p, y>, be = <p, p>, ga = <y, y> from the tile
// partials (fixed order), its loss 1 - al^2 / (be ga) into ls[s] and the
// gradient coefficients of dL/dp = cy y + cp p (with the 1 / S of the batch mean).
__global__ void k_cos_coef(const double *__restrict__ part, int tiles, int S, float *coef, double *ls) {
    const int s = blockIdx.x;
    double a = 0.0, b = 0.0, c = 0.0;
    for (int t = threadIdx.x; t < tiles; t += blockDim.x) {
        const double *q = part + 3 * ((size_t)s * tiles + t);
        a += q[0];
        b += q[1];
        c += q[2];
    }
    a = block_sum_d(a);
    __syncthreads();
    b = block_sum_d(b);
    __syncthreads();
    c = block_sum_d(c);
    if (threadIdx.x == 0) {
        const double bc = fmax(b, 1e-300) * fmax(c, 1e-300);
        ls[s] = 1.0 - a * a / bc;
        coef[2 * s] = (float)(-2.0 * a / bc / S);
        coef[2 * s + 1] = (float)(2.0 * a * a / (fmax(b, 1e-300) * bc) / S);
    }
}

// loss = mean over the batch of the per-sample losses
__global__ void k_loss_mean(const double *__restrict__ ls, int S, float *loss) {
    if (threadIdx.x != 0) return;
    double t = 0.0;
    for (int s = 0; s < S; ++s) t += ls[s];
    *loss = (float)(t / S);
}

// g = cy y + cp p per sample, in place over p
__global__ void k_cos_grad(float *pg, const float *__restrict__ y, const int *idx, const float *__restrict__ coef,
                           long long n) {
    const int s = blockIdx.y;
    const int q = idx ? idx[s] : s;
    const float cy = coef[2 * s], cp = coef[2 * s + 1];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const size_t o = (size_t)s * n + i;
        pg[o] = cy * y[(size_t)q * n + i] + cp * pg[o];
    }
}

// wt[26 - tap][co][ci] = w[tap][ci][co]: the weights of the adjoint convolution
__global__ void k_flip(const float *__restrict__ w, int cin, int cout, float *__restrict__ wt) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= 27 * cin * cout) return;
    const int co = q % cout, r = q / cout;
    const int ci = r % cin, tap = r / cin;
    wt[((26 - tap) * cout + co) * cin + ci] = w[q];
}

// Adam (Kingma and Ba 2015, Algorithm 1); lr_t = lr / (1 - b1^t), vc = 1 / (1 - b2^t).
__global__ void k_adam(float *w, const float *__restrict__ g, float *m, float *v, int cnt, float lr_t, float vc) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cnt) return;
    const float gj = g[j];
    const float mj = ADAM_B1 * m[j] + (1.0f - ADAM_B1) * gj;
    const float vj = ADAM_B2 * v[j] + (1.0f - ADAM_B2) * gj * gj;
    m[j] = mj;
    v[j] = vj;
    w[j] -= lr_t * mj / (sqrtf(vj * vc) + ADAM_EPS);
}

// ---- potential standardisation and band scales ------------------------------------
__global__ void k_sum_part(const double *__restrict__ v, long long n, const double *mean, double *part) {
    double s = 0.0;
    const double mu = mean ? *mean : 0.0;
    for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT) {
        const double d = v[i] - mu;
        s += mean ? d * d : v[i];
    }
    s = block_sum_d(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_sum_fin(const double *__restrict__ part, int np, long long n, double *out, int take_sqrt) {
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int q = 0; q < np; ++q) s += part[q];
    s /= (double)n;
    *out = take_sqrt ? sqrt(s) : s;
}

__global__ void k_vhat(const double *__restrict__ v, long long n, const double *mean, const double *sd,
                       float *vhat) {
    const double mu = *mean, s = *sd;
    const double inv = 1.0 / (s > 1e-12 ? s : 1.0);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        vhat[i] = (float)((v[i] - mu) * inv);
}

// part[b][q] = sum over slice q of |r_b|^2
template <typename V>
__global__ void k_band_sumsq(const V *__restrict__ r, long long n, int S, double *part) {
    const int q = blockIdx.x, b = blockIdx.y;
    const long long c = (n + S - 1) / S, i0 = (long long)q * c, i1 = i0 + c < n ? i0 + c : n;
    double s = 0.0;
    for (long long i = i0 + threadIdx.x; i < i1; i += NT) {
        const V z = r[(size_t)b * n + i];
        s += (double)z.x * z.x + (double)z.y * z.y;
    }
    s = block_sum_d(s);
    if (threadIdx.x == 0) part[(size_t)b * S + q] = s;
}

// s_b = sqrt(sum |r_b|^2 / n); inv_s = 1 / s_b (0 where s_b = 0)
__global__ void k_band_scale(const double *__restrict__ part, int S, int nb, long long n, float *sc, float *inv) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    double s = 0.0;
    for (int q = 0; q < S; ++q) s += part[(size_t)b * S + q];
    const double r = sqrt(s / (double)n);
    sc[b] = (float)r;
    inv[b] = r > 0.0 ? (float)(1.0 / r) : 0.0f;
}

// ---- state ---------------------------------------------------------------------
static rsdft_status ensure(rsdft_ctx *ctx, float **p, size_t *cap, size_t elems) {
    if (*cap >= elems && *p) return RSDFT_OK;
    if (*p) {
        cudaFree(*p);
        for (auto &q : ctx->owned)
            if (q == *p) q = nullptr;
        *p = nullptr;
        *cap = 0;
    }
    void *v = nullptr;
    RS_TRY(dev_alloc(ctx, &v, elems * sizeof(float)));
    *p = static_cast<float *>(v);
    *cap = elems;
    return RSDFT_OK;
}

static rsdft_status ensure_weights(rsdft_ctx *ctx) {
    NnState &s = ctx->nn;
    if (s.w) return RSDFT_OK;
    void *v = nullptr;
    // weights, flipped weights, gradient, two Adam moments
    RS_TRY(dev_alloc(ctx, &v, 5 * (size_t)WCOUNT * sizeof(float)));
    s.w = static_cast<float *>(v);
    s.wt = s.w + WCOUNT;
    s.g = s.wt + WCOUNT;
    s.m = s.g + WCOUNT;
    s.v = s.m + WCOUNT;
    // vhat, then the reduction scratch at an even float offset (8-byte aligned for any n)
    const size_t off = ((size_t)ctx->n + 65) & ~(size_t)1;
    RS_TRY(dev_alloc(ctx, &v, off * sizeof(float) + 1024 * sizeof(double)));
    s.vhat = static_cast<float *>(v);
    s.dred = reinterpret_cast<double *>(s.vhat + off);
    return RSDFT_OK;
}

// vhat = (V - mean V) / std V of the context's current potential
static rsdft_status make_vhat(rsdft_ctx *ctx, cudaStream_t st) {
    NnState &s = ctx->nn;
    const int np = std::max(1, std::min(cdiv(ctx->n, NT * 8), 512));
    double *part = s.dred, *mean = s.dred + 512, *sd = s.dred + 513;
    k_sum_part<<<np, NT, 0, st>>>(ctx->v, ctx->n, nullptr, part);
    k_sum_fin<<<1, 32, 0, st>>>(part, np, ctx->n, mean, 0);
    k_sum_part<<<np, NT, 0, st>>>(ctx->v, ctx->n, mean, part);
    k_sum_fin<<<1, 32, 0, st>>>(part, np, ctx->n, sd, 1);
    k_vhat<<<std::max(1, std::min(cdiv(ctx->n, 256), 1024)), 256, 0, st>>>(ctx->v, ctx->n, mean, sd, s.vhat);
    count_launch(ctx, 5);
    RS_LAUNCHED(ctx, "k_vhat");
    return RSDFT_OK;
}

static rsdft_status flip_all(rsdft_ctx *ctx, cudaStream_t st) {
    NnState &s = ctx->nn;
    const int cin[4] = {2, C, C, C}, cout[4] = {C, C, C, 1}, off[4] = {0, OFF1, OFF2, OFF3};
    for (int l = 1; l < 4; ++l) {   // the first layer's adjoint is never needed
        const int cnt = 27 * cin[l] * cout[l];
        k_flip<<<cdiv(cnt, 256), 256, 0, st>>>(s.w + off[l], cin[l], cout[l], s.wt + off[l]);
    }
    count_launch(ctx, 3);
    RS_LAUNCHED(ctx, "k_flip");
    return RSDFT_OK;
}

template <int CIN, int COUT, class Src, class Epi>
static rsdft_status conv(rsdft_ctx *ctx, const Src &src, const float *w, const Epi &epi, int S, cudaStream_t st) {
    const Geo g = geo_of(ctx);
    const size_t smem = (27 * CIN * COUT + CIN * HALO) * sizeof(float);
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_conv<CIN, COUT, Src, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    RS_CUDA(ctx, attr);
    k_conv<CIN, COUT, Src, Epi><<<dim3(g.tx * g.ty * g.tz, S), NT, smem, st>>>(src, w, epi, g);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_conv");
    return RSDFT_OK;
}

template <int CIN, int COUT, class Src>
static rsdft_status wgrad(rsdft_ctx *ctx, const Src &src, const float *gout, int S, float *dw, cudaStream_t st) {
    NnState &s = ctx->nn;
    const Geo g = geo_of(ctx);
    const int tiles = g.tx * g.ty * g.tz, cnt = 27 * CIN * COUT;
    RS_TRY(ensure(ctx, &s.part, &s.part_cap, (size_t)tiles * S * cnt));
    const size_t smem = (CIN * HALO + TILE * COUT) * sizeof(float);
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_wgrad<CIN, COUT, Src>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    RS_CUDA(ctx, attr);
    k_wgrad<CIN, COUT, Src><<<dim3(tiles, S), NT, smem, st>>>(src, gout, g, s.part);
    k_sum_parts<<<cdiv(cnt, 128), 128, 0, st>>>(s.part, tiles * S, cnt, dw);
    count_launch(ctx, 2);
    RS_LAUNCHED(ctx, "k_wgrad");
    return RSDFT_OK;
}

}  // namespace nn

// W[b] += s_b NN(R_b / s_b) for the nb rows of R (compact); V = double2 or float2.
template <typename V>
rsdft_status learned_correction(rsdft_ctx *ctx, const V *R, int nb, V *W, cudaStream_t st) {
    using namespace nn;
    NnState &s = ctx->nn;
    if (!s.ready) return fail(ctx, RSDFT_E_INVALID, "learned preconditioner: no weights set");
    if (nb <= 0) return RSDFT_OK;
    RS_TRY(make_vhat(ctx, st));
    // per-band scales
    const int S = std::max(1, std::min(64, cdiv(ctx->n, 8192)));
    RS_TRY(ensure(ctx, &s.bs, &s.bs_cap, (size_t)2 * nb + (size_t)nb * S * 2));
    float *sc = s.bs, *inv = s.bs + nb;
    double *part = reinterpret_cast<double *>(s.bs + 2 * nb);   // 8-byte aligned: 2 nb floats
    k_band_sumsq<V><<<dim3(S, nb), NT, 0, st>>>(R, ctx->n, S, part);
    k_band_scale<<<cdiv(nb, 128), 128, 0, st>>>(part, S, nb, ctx->n, sc, inv);
    count_launch(ctx, 2);
    // samples in chunks whose two activation buffers stay near 64 MB (L2-resident)
    const int total = 2 * nb;
    const size_t per = (size_t)C * ctx->n;
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>(total, (size_t)(8u << 20) / per));
    RS_TRY(ensure(ctx, &s.act, &s.act_cap, 2 * per * chunk));
    float *A = s.act, *B = s.act + per * chunk;
    for (int g0 = 0; g0 < total; g0 += chunk) {
        const int cs = std::min(chunk, total - g0);
        SrcResid<V> src{R, inv, s.vhat, nb, g0, ctx->n};
        RS_TRY((conv<2, C>(ctx, src, s.w, EpiTanh{A, ctx->n}, cs, st)));
        RS_TRY((conv<C, C>(ctx, SrcAct<C>{A, ctx->n}, s.w + OFF1, EpiTanh{B, ctx->n}, cs, st)));
        RS_TRY((conv<C, C>(ctx, SrcAct<C>{B, ctx->n}, s.w + OFF2, EpiTanh{A, ctx->n}, cs, st)));
        RS_TRY((conv<C, 1>(ctx, SrcAct<C>{A, ctx->n}, s.w + OFF3, EpiAdd<V>{W, sc, nb, g0, ctx->n}, cs, st)));
    }
    return RSDFT_OK;
}
template rsdft_status learned_correction<double2>(rsdft_ctx *, const double2 *, int, double2 *, cudaStream_t);
template rsdft_status learned_correction<float2>(rsdft_ctx *, const float2 *, int, float2 *, cudaStream_t);

}  // namespace rsdft

namespace rsdft {
namespace nn {

// Scratch of one training batch: activations, gradients, loss partials.
struct Batch {
    float *a1, *a2, *a3, *ga, *gb, *gout, *loss, *coef;
    double *lossp, *ls;
};

static rsdft_status batch_buffers(rsdft_ctx *ctx, int batch, int nloss, Batch &bb) {
    NnState &s = ctx->nn;
    const long long n = ctx->n;
    const Geo g = geo_of(ctx);
    const int tiles = g.tx * g.ty * g.tz;
    const size_t per = (size_t)C * n * batch;
    // a1 a2 a3 ga gb [batch][C][n], gout [batch][n], losses, gradient coefficients
    // [batch][2], then (doubles) loss partials [batch][tiles][3] and sample losses
    const size_t lp_off = (5 * per + (size_t)batch * n + (size_t)nloss + 2 * (size_t)batch + 1) & ~(size_t)1;
    RS_TRY(ensure(ctx, &s.tr, &s.tr_cap, lp_off + 2 * (3 * (size_t)tiles * batch + batch) + 8));
    bb.a1 = s.tr;
    bb.a2 = bb.a1 + per;
    bb.a3 = bb.a2 + per;
    bb.ga = bb.a3 + per;
    bb.gb = bb.ga + per;
    bb.gout = bb.gb + per;
    bb.loss = bb.gout + (size_t)batch * n;
    bb.coef = bb.loss + nloss;
    bb.lossp = reinterpret_cast<double *>(s.tr + lp_off);
    bb.ls = bb.lossp + 3 * (size_t)tiles * batch;
    return RSDFT_OK;
}

// Loss of one batch (samples idx[0..batch), or 0..batch when idx is null) into
// *loss_dev and its gradient in the weights into s.g (the flipped weights s.wt
// must be current).
static rsdft_status forward_backward(rsdft_ctx *ctx, const float *u, const float *b, const float *y, const int *idx,
                                     int batch, const Batch &bb, float *loss_dev, cudaStream_t st) {
    NnState &s = ctx->nn;
    const long long n = ctx->n;
    const Geo g = geo_of(ctx);
    const int tiles = g.tx * g.ty * g.tz;
    const SrcPlane p{u, idx, s.vhat, n};
    RS_TRY((conv<2, C>(ctx, p, s.w, EpiTanh{bb.a1, n}, batch, st)));
    RS_TRY((conv<C, C>(ctx, SrcAct<C>{bb.a1, n}, s.w + OFF1, EpiTanh{bb.a2, n}, batch, st)));
    RS_TRY((conv<C, C>(ctx, SrcAct<C>{bb.a2, n}, s.w + OFF2, EpiTanh{bb.a3, n}, batch, st)));
    RS_TRY((conv<C, 1>(ctx, SrcAct<C>{bb.a3, n}, s.w + OFF3, EpiLoss{b, y, idx, bb.gout, bb.lossp, n}, batch, st)));
    // loss 1 - cos^2(p, y) per sample, its mean, and dL/dp in place of p
    k_cos_coef<<<batch, NT, 0, st>>>(bb.lossp, tiles, batch, bb.coef, bb.ls);
    k_loss_mean<<<1, 32, 0, st>>>(bb.ls, batch, loss_dev);
    k_cos_grad<<<dim3(std::max(1, std::min(cdiv(n, 256), 256)), batch), 256, 0, st>>>(bb.gout, y, idx, bb.coef, n);
    count_launch(ctx, 3);
    RS_LAUNCHED(ctx, "k_cos");
    // reverse mode, last layer first
    RS_TRY((wgrad<C, 1>(ctx, SrcAct<C>{bb.a3, n}, bb.gout, batch, s.g + OFF3, st)));
    RS_TRY((conv<1, C>(ctx, SrcAct<1>{bb.gout, n}, s.wt + OFF3, EpiDtanh{bb.ga, bb.a3, n}, batch, st)));
    RS_TRY((wgrad<C, C>(ctx, SrcAct<C>{bb.a2, n}, bb.ga, batch, s.g + OFF2, st)));
    RS_TRY((conv<C, C>(ctx, SrcAct<C>{bb.ga, n}, s.wt + OFF2, EpiDtanh{bb.gb, bb.a2, n}, batch, st)));
    RS_TRY((wgrad<C, C>(ctx, SrcAct<C>{bb.a1, n}, bb.gb, batch, s.g + OFF1, st)));
    RS_TRY((conv<C, C>(ctx, SrcAct<C>{bb.gb, n}, s.wt + OFF1, EpiDtanh{bb.ga, bb.a1, n}, batch, st)));
    return wgrad<2, C>(ctx, p, bb.ga, batch, s.g, st);
}

// Loss and gradient over all S samples as one batch.
static rsdft_status loss_grad(rsdft_ctx *ctx, const float *u, const float *b, const float *y, int S, float *loss_host,
                              float *grad_host, cudaStream_t st) {
    NnState &s = ctx->nn;
    Batch bb;
    RS_TRY(batch_buffers(ctx, S, 1, bb));
    RS_TRY(make_vhat(ctx, st));
    RS_TRY(flip_all(ctx, st));
    RS_TRY(forward_backward(ctx, u, b, y, nullptr, S, bb, bb.loss, st));
    if (loss_host) RS_CUDA(ctx, cudaMemcpyAsync(loss_host, bb.loss, sizeof(float), cudaMemcpyDeviceToHost, st));
    if (grad_host) RS_CUDA(ctx, cudaMemcpyAsync(grad_host, s.g, WCOUNT * sizeof(float), cudaMemcpyDeviceToHost, st));
    RS_CUDA(ctx, cudaStreamSynchronize(st));
    return RSDFT_OK;
}

// Adam on cyclic mini-batches of the samples (u, b, y: [S][n] float planes);
// the loss of each step's batch (before its update) goes to loss_host[steps].
static rsdft_status train(rsdft_ctx *ctx, const float *u, const float *b, const float *y, long long S, int steps,
                          int batch, float lr, float *loss_host, cudaStream_t st) {
    NnState &s = ctx->nn;
    Batch bb;
    RS_TRY(batch_buffers(ctx, batch, steps, bb));
    // cyclic batch order: batch k holds samples (k batch + j) mod S
    std::vector<int> idx((size_t)steps * batch);
    for (long long k = 0; k < steps; ++k)
        for (int j = 0; j < batch; ++j) idx[(size_t)k * batch + j] = (int)((k * batch + j) % S);
    int *idx_dev = nullptr;
    RS_CUDA(ctx, cudaMallocAsync(reinterpret_cast<void **>(&idx_dev), idx.size() * sizeof(int), st));
    RS_CUDA(ctx, cudaMemcpyAsync(idx_dev, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    RS_TRY(make_vhat(ctx, st));
    RS_CUDA(ctx, cudaMemsetAsync(s.m, 0, 2 * (size_t)WCOUNT * sizeof(float), st));
    RS_TRY(flip_all(ctx, st));
    float *loss_dev = bb.loss;
    rsdft_status rc = RSDFT_OK;
    for (int k = 0; k < steps && rc == RSDFT_OK; ++k) {
        const int *ik = idx_dev + (size_t)k * batch;
        auto step = [&]() -> rsdft_status {
            RS_TRY(forward_backward(ctx, u, b, y, ik, batch, bb, loss_dev + k, st));
            const double t = (double)(k + 1);
            const float lr_t = (float)(lr / (1.0 - std::pow((double)ADAM_B1, t)));
            const float vc = (float)(1.0 / (1.0 - std::pow((double)ADAM_B2, t)));
            k_adam<<<cdiv(WCOUNT, 256), 256, 0, st>>>(s.w, s.g, s.m, s.v, WCOUNT, lr_t, vc);
            count_launch(ctx);
            RS_LAUNCHED(ctx, "k_adam");
            return flip_all(ctx, st);
        };
        rc = step();
    }
    if (rc == RSDFT_OK && loss_host) {
        const cudaError_t e = cudaMemcpyAsync(loss_host, loss_dev, (size_t)steps * sizeof(float),
                                              cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = cuda_check(ctx, e, "loss copy");
    }
    cudaFreeAsync(idx_dev, st);
    const cudaError_t e = cudaStreamSynchronize(st);
    if (rc == RSDFT_OK && e != cudaSuccess) rc = cuda_check(ctx, e, "train sync");
    return rc;
}

// ---- projected correction targets (batched MINRES, Paige and Saunders 1975) ----
constexpr int BT = 256;

__device__ double2 block_sum_c(double2 v) {
    __shared__ double2 sh[BT / 32];
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double2 t = make_double2(0.0, 0.0);
    if (threadIdx.x == 0)
        for (int w = 0; w < BT / 32; ++w) {
            t.x += sh[w].x;
            t.y += sh[w].y;
        }
    return t;
}

// part[b][q] = sum over slice q of conj(a_b) c_b (times wt when given)
__global__ void k_bdot_part(const double2 *__restrict__ a, const double2 *__restrict__ c,
                            const double *__restrict__ wt, long long n, int S, double2 *part) {
    const int q = blockIdx.x, b = blockIdx.y;
    const long long len = (n + S - 1) / S, i0 = (long long)q * len, i1 = i0 + len < n ? i0 + len : n;
    double2 s = make_double2(0.0, 0.0);
    for (long long i = i0 + threadIdx.x; i < i1; i += BT) {
        const double2 x = a[(size_t)b * n + i], z = c[(size_t)b * n + i];
        const double w = wt ? wt[i] : 1.0;
        s.x += w * (x.x * z.x + x.y * z.y);
        s.y += w * (x.x * z.y - x.y * z.x);
    }
    s = block_sum_c(s);
    if (threadIdx.x == 0) part[(size_t)b * S + q] = s;
}

__global__ void k_bdot_fin(const double2 *__restrict__ part, int S, int nb, double scale, double2 *out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    double2 s = make_double2(0.0, 0.0);
    for (int q = 0; q < S; ++q) {
        s.x += part[(size_t)b * S + q].x;
        s.y += part[(size_t)b * S + q].y;
    }
    out[b] = make_double2(scale * s.x, scale * s.y);
}

struct MrState {
    double *beta, *cp, *sp, *cpp, *spp, *phi, *beta1;
    double *inv_gamma, *delta, *eps, *tau, *inv_bnext;
    int *done, *upd, *iters;
};

// z_b = hq_b - e_b q_b (in place in hq)
__global__ void k_mr_shift(double2 *hq, const double2 *__restrict__ q, const double *__restrict__ e, long long n,
                           const int *done) {
    const int b = blockIdx.y;
    if (done && done[b]) return;
    const double eb = e[b];
    for (long long i = (long long)blockIdx.x * BT + threadIdx.x; i < n; i += (long long)gridDim.x * BT) {
        const size_t o = (size_t)b * n + i;
        const double2 h = hq[o], v = q[o];
        hq[o] = make_double2(h.x - eb * v.x, h.y - eb * v.y);
    }
}

// p_b -= alpha_b v_b + beta_b v_prev_b, alpha_b = Re <v_b|p_b>
__global__ void k_mr_lanczos(double2 *p, const double2 *__restrict__ v, const double2 *__restrict__ vp,
                             const double2 *__restrict__ dvp, MrState ms, long long n) {
    const int b = blockIdx.y;
    if (ms.done[b]) return;
    const double al = dvp[b].x, be = ms.beta[b];
    for (long long i = (long long)blockIdx.x * BT + threadIdx.x; i < n; i += (long long)gridDim.x * BT) {
        const size_t o = (size_t)b * n + i;
        const double2 a = p[o], x = v[o], y = vp[o];
        p[o] = make_double2(a.x - al * x.x - be * y.x, a.y - al * x.y - be * y.y);
    }
}

// The MINRES scalars of one iteration per band: the new tridiagonal column
// (beta_k, alpha_k, beta_k+1) through the two previous Givens rotations, the
// new rotation, and the coefficients of the direction and solution updates.
__global__ void k_mr_scalars(MrState ms, const double2 *__restrict__ dvp, const double2 *__restrict__ dpp, int nb,
                             double rtol) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    ms.upd[b] = 0;
    if (ms.done[b]) return;
    const double alpha = dvp[b].x, bnext = sqrt(fmax(dpp[b].x, 0.0)), beta = ms.beta[b];
    const double eps = ms.spp[b] * beta, dbar = ms.cpp[b] * beta;
    const double delta = ms.cp[b] * dbar + ms.sp[b] * alpha;
    const double gbar = -ms.sp[b] * dbar + ms.cp[b] * alpha;
    const double gamma = hypot(gbar, bnext);
    if (gamma == 0.0) {
        ms.done[b] = 1;
        return;
    }
    const double c = gbar / gamma, s = bnext / gamma;
    const double phi = ms.phi[b];
    ms.inv_gamma[b] = 1.0 / gamma;
    ms.delta[b] = delta;
    ms.eps[b] = eps;
    ms.tau[b] = c * phi;
    ms.inv_bnext[b] = bnext > 0.0 ? 1.0 / bnext : 0.0;
    ms.phi[b] = -s * phi;
    ms.cpp[b] = ms.cp[b];
    ms.spp[b] = ms.sp[b];
    ms.cp[b] = c;
    ms.sp[b] = s;
    ms.beta[b] = bnext;
    ms.upd[b] = 1;
    ms.iters[b] += 1;
    if (fabs(s * phi) <= rtol * ms.beta1[b] || bnext == 0.0) ms.done[b] = 1;
}

// d_new = (v - delta d_prev - eps d_pp) / gamma (into d_pp's buffer), t += tau d_new,
// v_new = p / beta_k+1 (into v_prev's buffer)
__global__ void k_mr_update(double2 *dpp, const double2 *__restrict__ v, const double2 *__restrict__ dp, double2 *t,
                            const double2 *__restrict__ p, double2 *vnew, MrState ms, long long n) {
    const int b = blockIdx.y;
    if (!ms.upd[b]) return;
    const double ig = ms.inv_gamma[b], de = ms.delta[b], ep = ms.eps[b], ta = ms.tau[b], ib = ms.inv_bnext[b];
    for (long long i = (long long)blockIdx.x * BT + threadIdx.x; i < n; i += (long long)gridDim.x * BT) {
        const size_t o = (size_t)b * n + i;
        const double2 vv = v[o], d1 = dp[o], d2 = dpp[o], pp = p[o];
        const double2 d = make_double2((vv.x - de * d1.x - ep * d2.x) * ig, (vv.y - de * d1.y - ep * d2.y) * ig);
        dpp[o] = d;
        const double2 tt = t[o];
        t[o] = make_double2(tt.x + ta * d.x, tt.y + ta * d.y);
        vnew[o] = make_double2(pp.x * ib, pp.y * ib);
    }
}

// MINRES start: beta1 = ||rhs||, v = rhs / beta1, state reset
__global__ void k_mr_init(MrState ms, const double2 *__restrict__ dbb, int nb) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const double b1 = sqrt(fmax(dbb[b].x, 0.0));
    ms.beta1[b] = b1;
    ms.phi[b] = b1;
    ms.beta[b] = 0.0;
    ms.cp[b] = ms.cpp[b] = 1.0;
    ms.sp[b] = ms.spp[b] = 0.0;
    ms.done[b] = b1 == 0.0;
    ms.upd[b] = 0;
    ms.iters[b] = 0;
    ms.inv_bnext[b] = b1 > 0.0 ? 1.0 / b1 : 0.0;
}

__global__ void k_mr_scale(double2 *v, const double2 *__restrict__ rhs, MrState ms, long long n) {
    const int b = blockIdx.y;
    const double s = ms.inv_bnext[b];
    for (long long i = (long long)blockIdx.x * BT + threadIdx.x; i < n; i += (long long)gridDim.x * BT) {
        const size_t o = (size_t)b * n + i;
        v[o] = make_double2(rhs[o].x * s, rhs[o].y * s);
    }
}

// r_b = hx_b - e_b x_b with e_b = Re <x_b|hx_b> dV; t_b = e_b - <x_b|V|x_b> - sum E |p|^2
__global__ void k_samples_setup(const double2 *__restrict__ exh, const double2 *__restrict__ evx,
                                const double2 *__restrict__ p, ProjTables pt, int nb, double *e, double *tkin) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int np = pt.natom * pt.nproj;
    double nl = 0.0;
    for (int q = 0; q < np; ++q) {
        const double2 c = p[(size_t)b * np + q];
        nl += pt.e_kb[q] * (c.x * c.x + c.y * c.y);
    }
    e[b] = exh[b].x;
    tkin[b] = exh[b].x - evx[b].x - nl;
}

// u = [Re r / s; Im r / s], bp = base / s, yp = c t / s as float planes, with
// c = sign(Re<t|base>) ||base|| / ||t|| (t rescaled to the TPA norm, pointing along it)
__global__ void k_planes(const double2 *__restrict__ r, const double2 *__restrict__ base, const double2 *__restrict__ t,
                         const double2 *__restrict__ dtb, const double2 *__restrict__ dtt, const double2 *__restrict__ drr,
                         const double2 *__restrict__ dbb, int nb, long long n, float *u, float *bp, float *yp) {
    const int b = blockIdx.y;
    const double s = sqrt(drr[b].x / (double)n);
    const double inv = s > 0.0 ? 1.0 / s : 1.0;
    const double c = dtt[b].x > 0.0 ? (dtb[b].x < 0.0 ? -1.0 : 1.0) * sqrt(dbb[b].x / dtt[b].x) : 0.0;
    for (long long i = (long long)blockIdx.x * BT + threadIdx.x; i < n; i += (long long)gridDim.x * BT) {
        const size_t o = (size_t)b * n + i, o2 = (size_t)(b + nb) * n + i;
        const double2 rr = r[o], bb = base[o], tt = t[o];
        u[o] = (float)(rr.x * inv);
        u[o2] = (float)(rr.y * inv);
        bp[o] = (float)(bb.x * inv);
        bp[o2] = (float)(bb.y * inv);
        yp[o] = (float)(c * tt.x * inv);
        yp[o2] = (float)(c * tt.y * inv);
    }
}

static rsdft_status bdot(rsdft_ctx *ctx, const double2 *a, const double2 *c, const double *wt, int nb, double scale,
                         double2 *part, int S, double2 *out, cudaStream_t st) {
    k_bdot_part<<<dim3(S, nb), BT, 0, st>>>(a, c, wt, ctx->n, S, part);
    k_bdot_fin<<<cdiv(nb, 128), 128, 0, st>>>(part, S, nb, scale, out);
    count_launch(ctx, 2);
    RS_LAUNCHED(ctx, "k_bdot");
    return RSDFT_OK;
}

// out = Q in with Q = I - X X^H (all nb bands of the block; dV metric): a Gram
// against X and a rotation.  out may alias in.
static rsdft_status block_project(rsdft_ctx *ctx, const double2 *X, int nb, const double2 *in, double2 *out,
                                  cudaStream_t st) {
    RowBlocks YX{{X, nullptr, nullptr}, {nb, 0, 0}};
    RowBlocks YI{{in, nullptr, nullptr}, {nb, 0, 0}};
    RS_TRY(gram(ctx, YX, YI, ctx->ws.C, nb, false, ctx->dV, st));
    return rotate(ctx, YX, ctx->ws.C, nb, nb, in, -1, out, nullptr, st);
}

static rsdft_status samples(rsdft_ctx *ctx, const double2 *X, int nb, double rtol, int maxit, float *U, float *B,
                            float *Y, int *iters_host, cudaStream_t st) {
    const long long n = ctx->n;
    const size_t blk = (size_t)nb * n;
    RS_TRY(ensure_workspace(ctx, nb));
    // R, base, V, VP, D1, D2, T, Q, HQ, P
    double2 *buf = nullptr;
    RS_CUDA(ctx, cudaMallocAsync(reinterpret_cast<void **>(&buf), 10 * blk * sizeof(double2), st));
    const int S = std::max(1, std::min(64, cdiv(n, 8192)));
    const int nsc = 16;   // per-band scalar arrays
    double *sc = nullptr;
    RS_CUDA(ctx, cudaMallocAsync(reinterpret_cast<void **>(&sc), ((size_t)nsc * nb + 2 * (size_t)nb * S * 2 + 16 * (size_t)nb) * sizeof(double), st));
    double2 *R = buf, *Bs = R + blk, *V = Bs + blk, *VP = V + blk, *D1 = VP + blk, *D2 = D1 + blk, *T = D2 + blk,
            *Q = T + blk, *HQ = Q + blk, *P = HQ + blk;
    MrState ms;
    double *q = sc;
    ms.beta = q; q += nb; ms.cp = q; q += nb; ms.sp = q; q += nb; ms.cpp = q; q += nb; ms.spp = q; q += nb;
    ms.phi = q; q += nb; ms.beta1 = q; q += nb; ms.inv_gamma = q; q += nb; ms.delta = q; q += nb;
    ms.eps = q; q += nb; ms.tau = q; q += nb; ms.inv_bnext = q; q += nb;
    double *e = q; q += nb;
    double *tkin = q; q += nb;
    int *iq = reinterpret_cast<int *>(q);
    ms.done = iq; ms.upd = iq + nb; ms.iters = iq + 2 * nb;
    q += 2 * nb;   // room for three int arrays
    double2 *part = reinterpret_cast<double2 *>(q);
    double2 *d1 = part + (size_t)nb * S, *d2 = d1 + nb, *d3 = d2 + nb, *d4 = d3 + nb, *d5 = d4 + nb;
    const dim3 rg(std::max(1, std::min(cdiv(n, BT * 4), 256)), nb);
    const double dV = ctx->dV;
    rsdft_status rc = [&]() -> rsdft_status {
        // residuals, kinetic energies, TPA base
        RS_TRY(apply_h64(ctx, X, HQ, nb, st));
        RS_TRY(bdot(ctx, X, HQ, nullptr, nb, dV, part, S, d1, st));        // e_b
        RS_TRY(bdot(ctx, X, X, ctx->v, nb, dV, part, S, d2, st));          // <x|V|x>
        RS_TRY(project(ctx, X, ctx->ws.proj, nb, st));
        k_samples_setup<<<cdiv(nb, 128), 128, 0, st>>>(d1, d2, ctx->ws.proj, ctx->pt, nb, e, tkin);
        RS_CUDA(ctx, cudaMemcpyAsync(R, HQ, blk * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        k_mr_shift<<<rg, BT, 0, st>>>(R, X, e, n, nullptr);
        count_launch(ctx, 2);
        RS_LAUNCHED(ctx, "k_samples_setup");
        RS_TRY(fft_xy_forward(ctx, Src::Plain, R, nullptr, nullptr, nullptr, nullptr, ctx->ws.T1, nb, st));
        RS_TRY(fft_z_mid(ctx, Mid::Tpa, ctx->ws.T1, tkin, nb, st));
        RS_TRY(fft_xy_inverse(ctx, ctx->ws.T1, nullptr, nullptr, Bs, nullptr, nb, st));
        // MINRES on A t' = Q r (into VP as scratch), Q = I - X X^H off the whole
        // block; the target is t = -t'
        RS_TRY(block_project(ctx, X, nb, R, VP, st));
        RS_TRY(bdot(ctx, VP, VP, nullptr, nb, 1.0, part, S, d2, st));
        k_mr_init<<<cdiv(nb, 128), 128, 0, st>>>(ms, d2, nb);
        k_mr_scale<<<rg, BT, 0, st>>>(V, VP, ms, n);   // v = rhs / beta1
        count_launch(ctx, 3);
        RS_CUDA(ctx, cudaMemsetAsync(VP, 0, blk * sizeof(double2), st));
        RS_CUDA(ctx, cudaMemsetAsync(D1, 0, blk * sizeof(double2), st));
        RS_CUDA(ctx, cudaMemsetAsync(D2, 0, blk * sizeof(double2), st));
        RS_CUDA(ctx, cudaMemsetAsync(T, 0, blk * sizeof(double2), st));
        std::vector<int> hdone(nb);
        for (int it = 0; it < maxit; ++it) {
            // p = Q (H - e) Q v (converged bands are computed too; the MINRES
            // kernels below leave their state untouched)
            RS_TRY(block_project(ctx, X, nb, V, Q, st));
            RS_TRY(apply_h64(ctx, Q, HQ, nb, st));
            k_mr_shift<<<rg, BT, 0, st>>>(HQ, Q, e, n, ms.done);
            count_launch(ctx);
            RS_TRY(block_project(ctx, X, nb, HQ, P, st));
            // Lanczos step and its scalars
            RS_TRY(bdot(ctx, V, P, nullptr, nb, 1.0, part, S, d3, st));
            k_mr_lanczos<<<rg, BT, 0, st>>>(P, V, VP, d3, ms, n);
            count_launch(ctx);
            RS_TRY(bdot(ctx, P, P, nullptr, nb, 1.0, part, S, d4, st));
            k_mr_scalars<<<cdiv(nb, 128), 128, 0, st>>>(ms, d3, d4, nb, rtol);
            k_mr_update<<<rg, BT, 0, st>>>(D2, V, D1, T, P, VP, ms, n);
            count_launch(ctx, 2);
            RS_LAUNCHED(ctx, "k_mr");
            std::swap(D1, D2);   // d_prev <- d_new, d_pp <- old d_prev
            std::swap(V, VP);    // v <- v_new, v_prev <- old v
            if ((it & 7) == 7 || it == maxit - 1) {
                RS_CUDA(ctx, cudaMemcpyAsync(hdone.data(), ms.done, nb * sizeof(int), cudaMemcpyDeviceToHost, st));
                RS_CUDA(ctx, cudaStreamSynchronize(st));
                bool all = true;
                for (int bb = 0; bb < nb; ++bb) all = all && hdone[bb];
                if (all) break;
            }
        }
        // t' <- Q t'.  With t = -t' the target sign(Re<t|base>) t equals
        // sign(Re<t'|base>) t', so the planes come from t' directly.
        RS_TRY(block_project(ctx, X, nb, T, Q, st));
        RS_TRY(bdot(ctx, Q, Bs, nullptr, nb, 1.0, part, S, d2, st));
        RS_TRY(bdot(ctx, Q, Q, nullptr, nb, 1.0, part, S, d3, st));
        RS_TRY(bdot(ctx, Bs, Bs, nullptr, nb, 1.0, part, S, d4, st));
        RS_TRY(bdot(ctx, R, R, nullptr, nb, 1.0, part, S, d5, st));
        k_planes<<<rg, BT, 0, st>>>(R, Bs, Q, d2, d3, d5, d4, nb, n, U, B, Y);
        count_launch(ctx);
        RS_LAUNCHED(ctx, "k_planes");
        if (iters_host)
            RS_CUDA(ctx, cudaMemcpyAsync(iters_host, ms.iters, nb * sizeof(int), cudaMemcpyDeviceToHost, st));
        RS_CUDA(ctx, cudaStreamSynchronize(st));
        return RSDFT_OK;
    }();
    cudaFreeAsync(sc, st);
    cudaFreeAsync(buf, st);
    cudaStreamSynchronize(st);
    return rc;
}

}  // namespace nn
}  // namespace rsdft

using namespace rsdft;

extern "C" {

rsdft_status rsdft_set_precond_weights(rsdft_ctx *ctx, const float *w_host, long long count) {
    if (!ctx || !w_host) return fail(ctx, RSDFT_E_INVALID, "ctx and weights are required");
    if (count != RSDFT_NN_WEIGHTS) return fail(ctx, RSDFT_E_INVALID, "weight count %lld, expected %d", count,
                                                RSDFT_NN_WEIGHTS);
    for (long long i = 0; i < count; ++i)
        if (!std::isfinite(w_host[i])) return fail(ctx, RSDFT_E_INVALID, "non-finite weight %lld", i);
    RS_TRY(nn::ensure_weights(ctx));
    RS_CUDA(ctx, cudaMemcpy(ctx->nn.w, w_host, count * sizeof(float), cudaMemcpyHostToDevice));
    ctx->nn.ready = 1;
    return RSDFT_OK;
}

rsdft_status rsdft_get_precond_weights(rsdft_ctx *ctx, float *w_host, long long count) {
    if (!ctx || !w_host) return fail(ctx, RSDFT_E_INVALID, "ctx and weights are required");
    if (count != RSDFT_NN_WEIGHTS) return fail(ctx, RSDFT_E_INVALID, "weight count %lld, expected %d", count,
                                                RSDFT_NN_WEIGHTS);
    if (!ctx->nn.ready) return fail(ctx, RSDFT_E_INVALID, "no weights set");
    RS_CUDA(ctx, cudaMemcpy(w_host, ctx->nn.w, count * sizeof(float), cudaMemcpyDeviceToHost));
    return RSDFT_OK;
}

rsdft_status rsdft_precond_learned(rsdft_ctx *ctx, const void *r_dev, const void *base_dev, void *w_dev, int nband,
                                   void *stream) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (nband < 0 || (nband > 0 && (!r_dev || !base_dev || !w_dev))) return fail(ctx, RSDFT_E_INVALID, "bad arguments");
    if (nband == 0) return RSDFT_OK;
    cudaStream_t st = as_stream(stream);
    if (w_dev != base_dev)
        RS_CUDA(ctx, cudaMemcpyAsync(w_dev, base_dev, (size_t)nband * ctx->n * sizeof(double2),
                                     cudaMemcpyDeviceToDevice, st));
    return learned_correction<double2>(ctx, static_cast<const double2 *>(r_dev), nband,
                                       static_cast<double2 *>(w_dev), st);
}

rsdft_status rsdft_precond_samples(rsdft_ctx *ctx, const void *x_dev, int nband, double rtol, int maxit,
                                   float *u_dev, float *b_dev, float *y_dev, int *iters_host, void *stream) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (nband <= 0 || !x_dev || !u_dev || !b_dev || !y_dev || maxit < 1 || !(rtol >= 0.0))
        return fail(ctx, RSDFT_E_INVALID, "bad arguments");
    return nn::samples(ctx, static_cast<const double2 *>(x_dev), nband, rtol, maxit, u_dev, b_dev, y_dev, iters_host,
                       as_stream(stream));
}

rsdft_status rsdft_precond_loss_grad(rsdft_ctx *ctx, const float *u_dev, const float *b_dev, const float *y_dev,
                                     int nsample, float *loss_host, float *grad_host, void *stream) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (!u_dev || !b_dev || !y_dev || nsample < 1 || nsample > 65535) return fail(ctx, RSDFT_E_INVALID, "bad arguments");
    if (!ctx->nn.ready) return fail(ctx, RSDFT_E_INVALID, "set weights first");
    return nn::loss_grad(ctx, u_dev, b_dev, y_dev, nsample, loss_host, grad_host, as_stream(stream));
}

rsdft_status rsdft_precond_train(rsdft_ctx *ctx, const float *u_dev, const float *b_dev, const float *y_dev,
                                 long long nsample, int steps, int batch, float lr, float *loss_host, void *stream) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (!u_dev || !b_dev || !y_dev || nsample < 1 || steps < 1 || batch < 1 || batch > 65535 || !(lr > 0.0f))
        return fail(ctx, RSDFT_E_INVALID, "bad arguments");
    if (!ctx->nn.ready) return fail(ctx, RSDFT_E_INVALID, "set initial weights first");
    return nn::train(ctx, u_dev, b_dev, y_dev, nsample, steps, batch, lr, loss_host, as_stream(stream));
}

}  // extern "C"
