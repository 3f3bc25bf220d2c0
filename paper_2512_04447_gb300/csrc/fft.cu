// Batched 3D FFT kernels and H psi (SCF tasks (1) and (4)).
//
// Layout: orbital block [band][z][y][x] complex, x fastest.  A 3D transform is
// three shared-memory passes over HBM:
//   xy-forward  (one CTA per (band, z) plane: x lines then y lines, DIF)
//   z-mid       (one CTA per (band, y) slab: z DIF, multiply by a function of
//                |G|^2 at the digit-reversed position, z DIT)
//   xy-inverse  (one CTA per (band, z) plane: y and x DIT, then the epilogue:
//                + V psi and the point-major projector scatter for H psi)
// Forward stages leave the spectrum in mixed-radix digit-reversed order and
// the inverse stages take it back to natural order, so the per-G factor is
// applied through position-indexed |G|^2 tables and no permutation pass exists.
#include <cmath>

#include "rsdft_internal.h"

namespace rsdft {

// ---- complex helpers (double2 / float2) ---------------------------------------
template <typename V> struct Sc;
template <> struct Sc<double2> { using T = double; };
template <> struct Sc<float2> { using T = float; };

template <typename V> __device__ __forceinline__ V mk(typename Sc<V>::T x, typename Sc<V>::T y) {
    V r; r.x = x; r.y = y; return r;
}
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return mk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return mk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
    return mk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename V> __device__ __forceinline__ V cmulconj(V a, V b) {  // a * conj(b)
    return mk<V>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename V> __device__ __forceinline__ V cscale(V a, typename Sc<V>::T s) { return mk<V>(a.x * s, a.y * s); }
// multiply by -i (forward sign) or +i (inverse sign)
template <typename V, bool INV> __device__ __forceinline__ V rot(V a) {
    return INV ? mk<V>(-a.y, a.x) : mk<V>(a.y, -a.x);
}

// ---- small DFTs: y_p = sum_q x_q exp(-+2 pi i p q / R) ----------------------
// Constants are cos/sin of 2 pi k / R written out to 30 digits.
#define RS_SQRT3_2 0.866025403784438646763723170753
#define RS_SQRT1_2 0.707106781186547524400844362105
#define RS_C1_5 0.309016994374947424102293417183
#define RS_C2_5 (-0.809016994374947424102293417183)
#define RS_S1_5 0.951056516295153572116439333379
#define RS_S2_5 0.587785252292473129168705954639

template <typename V, bool INV> __device__ __forceinline__ void dft2(V *v) {
    V a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}
template <typename V, bool INV> __device__ __forceinline__ void dft3(V *v) {
    using T = typename Sc<V>::T;
    V t1 = cadd(v[1], v[2]);
    V t2 = csub(v[0], cscale(t1, (T)0.5));
    V t3 = cscale(csub(v[1], v[2]), (T)RS_SQRT3_2);
    v[0] = cadd(v[0], t1);
    V r = rot<V, INV>(t3);  // -i t3 (forward)
    v[1] = cadd(t2, r);
    v[2] = csub(t2, r);
}
template <typename V, bool INV> __device__ __forceinline__ void dft4(V *v) {
    V a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
    V a2 = cadd(v[1], v[3]), a3 = rot<V, INV>(csub(v[1], v[3]));
    v[0] = cadd(a0, a2);
    v[2] = csub(a0, a2);
    v[1] = cadd(a1, a3);
    v[3] = csub(a1, a3);
}
template <typename V, bool INV> __device__ __forceinline__ void dft5(V *v) {
    using T = typename Sc<V>::T;
    V a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
    V a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
    V x0 = v[0];
    v[0] = cadd(x0, cadd(a1, a2));
    V r1 = cadd(x0, cadd(cscale(a1, (T)RS_C1_5), cscale(a2, (T)RS_C2_5)));
    V i1 = rot<V, INV>(cadd(cscale(b1, (T)RS_S1_5), cscale(b2, (T)RS_S2_5)));
    V r2 = cadd(x0, cadd(cscale(a1, (T)RS_C2_5), cscale(a2, (T)RS_C1_5)));
    V i2 = rot<V, INV>(csub(cscale(b1, (T)RS_S2_5), cscale(b2, (T)RS_S1_5)));
    v[1] = cadd(r1, i1);
    v[4] = csub(r1, i1);
    v[2] = cadd(r2, i2);
    v[3] = csub(r2, i2);
}
template <typename V, bool INV> __device__ __forceinline__ void dft8(V *v) {
    using T = typename Sc<V>::T;
    V e[4] = {v[0], v[2], v[4], v[6]};
    V o[4] = {v[1], v[3], v[5], v[7]};
    dft4<V, INV>(e);
    dft4<V, INV>(o);
    // o_p *= w8^p, w8 = exp(-+ i pi / 4)
    const T h = (T)RS_SQRT1_2;
    V o1 = o[1], o3 = o[3];
    // (1 -+ i) h * o1
    o[1] = cscale(cadd(o1, rot<V, INV>(o1)), h);
    o[2] = rot<V, INV>(o[2]);
    // (-1 -+ i) h * o3
    o[3] = cscale(csub(rot<V, INV>(o3), o3), h);
    for (int p = 0; p < 4; ++p) {
        v[p] = cadd(e[p], o[p]);
        v[p + 4] = csub(e[p], o[p]);
    }
}

template <typename V, int R, bool INV> __device__ __forceinline__ void dftR(V *v) {
    if constexpr (R == 2) dft2<V, INV>(v);
    else if constexpr (R == 3) dft3<V, INV>(v);
    else if constexpr (R == 4) dft4<V, INV>(v);
    else if constexpr (R == 5) dft5<V, INV>(v);
    else dft8<V, INV>(v);
}

template <typename V> __device__ __forceinline__ V ldtw(const V *tw, int k) { return __ldg(tw + k); }

// One radix-R butterfly of a stage, in place in shared memory.
template <typename V, int R, bool INV>
__device__ __forceinline__ void bfly(V *s, int base, int step, int j, int twstep, const V *tw) {
    V v[R];
    if (!INV) {
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = s[base + q * step];
        dftR<V, R, false>(v);
#pragma unroll
        for (int p = 1; p < R; ++p) v[p] = cmul(v[p], ldtw(tw, j * p * twstep));
    } else {
#pragma unroll
        for (int p = 0; p < R; ++p) v[p] = s[base + p * step];
#pragma unroll
        for (int p = 1; p < R; ++p) v[p] = cmulconj(v[p], ldtw(tw, j * p * twstep));
        dftR<V, R, true>(v);
    }
#pragma unroll
    for (int q = 0; q < R; ++q) s[base + q * step] = v[q];
}

// All stages of nlines 1D transforms of length ax.N in shared memory.
// Element e of line l sits at s[l * lstride + e * es].  lines_fast selects the
// thread mapping: consecutive threads take consecutive lines (use when es > 1
// and lstride == 1), else consecutive butterflies of one line.
template <typename V, bool INV>
__device__ void fft_lines(V *s, const AxisPlan &ax, const V *tw, int nlines, int lstride, int es,
                          bool lines_fast) {
    const int N = ax.N;
    for (int t = 0; t < ax.nstage; ++t) {
        const int st = INV ? ax.nstage - 1 - t : t;
        const int r = ax.radix[st], len = ax.len[st], sub = ax.sub[st];
        const int nbf = N / r;
        const int total = nbf * nlines;
        const int twstep = N / len;
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            int line, bf;
            if (lines_fast) { line = idx % nlines; bf = idx / nlines; }
            else { bf = idx % nbf; line = idx / nbf; }
            const int b = bf / sub, j = bf - b * sub;
            const int base = line * lstride + (b * len + j) * es;
            const int step = sub * es;
            switch (r) {
                case 2: bfly<V, 2, INV>(s, base, step, j, twstep, tw); break;
                case 3: bfly<V, 3, INV>(s, base, step, j, twstep, tw); break;
                case 4: bfly<V, 4, INV>(s, base, step, j, twstep, tw); break;
                case 5: bfly<V, 5, INV>(s, base, step, j, twstep, tw); break;
                default: bfly<V, 8, INV>(s, base, step, j, twstep, tw); break;
            }
        }
        __syncthreads();
    }
}

constexpr int FFT_THREADS = 512;

// ---- xy forward pass ------------------------------------------------------------
template <Src SRC>
__global__ void __launch_bounds__(FFT_THREADS)
k_xy_forward(Fft3Plan plan, const double2 *__restrict__ src, const double2 *__restrict__ src2,
             const double *__restrict__ theta, const int *__restrict__ act,
             const double *__restrict__ rsrc, double2 *__restrict__ dst) {
    extern __shared__ double2 s_plane[];
    const int Nx = plan.ax[0].N, Ny = plan.ax[1].N, Nz = plan.ax[2].N;
    const int z = blockIdx.x, band = blockIdx.y;
    const size_t n = (size_t)Nx * Ny * Nz;
    const size_t plane = (size_t)Nx * Ny;
    const size_t off = (size_t)z * plane;
    if (SRC == Src::Plain) {
        const double2 *in = src + band * n + off;
        for (int i = threadIdx.x; i < (int)plane; i += blockDim.x) s_plane[i] = in[i];
    } else if (SRC == Src::Residual) {
        const int b = act[band];
        const double th = theta[b];
        const double2 *hx = src + b * n + off;
        const double2 *x = src2 + b * n + off;
        for (int i = threadIdx.x; i < (int)plane; i += blockDim.x) {
            double2 h = hx[i], v = x[i];
            s_plane[i] = make_double2(h.x - th * v.x, h.y - th * v.y);
        }
    } else {
        const double *in = rsrc + off;
        for (int i = threadIdx.x; i < (int)plane; i += blockDim.x) s_plane[i] = make_double2(in[i], 0.0);
    }
    __syncthreads();
    fft_lines<double2, false>(s_plane, plan.ax[0], plan.tw64[0], Ny, Nx, 1, false);
    fft_lines<double2, false>(s_plane, plan.ax[1], plan.tw64[1], Nx, 1, Nx, true);
    double2 *out = dst + band * n + off;
    for (int i = threadIdx.x; i < (int)plane; i += blockDim.x) out[i] = s_plane[i];
}

// ---- z pass with the per-G factor ------------------------------------------------
__device__ __forceinline__ double tpa_k(double x) {
    double num = 27.0 + x * (18.0 + x * (12.0 + 8.0 * x));
    return num / (num + 16.0 * x * x * x * x);
}

template <Mid MID>
__global__ void __launch_bounds__(FFT_THREADS)
k_z_mid(Fft3Plan plan, double2 *__restrict__ buf, const double *__restrict__ tkin) {
    extern __shared__ double2 s_slab[];
    const int Nx = plan.ax[0].N, Ny = plan.ax[1].N, Nz = plan.ax[2].N;
    const int y = blockIdx.x, band = blockIdx.y;
    const size_t n = (size_t)Nx * Ny * Nz;
    const size_t zstride = (size_t)Nx * Ny;
    double2 *base = buf + band * n + (size_t)y * Nx;
    const int tot = Nx * Nz;
    for (int i = threadIdx.x; i < tot; i += blockDim.x) {
        int z = i / Nx, x = i - z * Nx;
        s_slab[i] = base[z * zstride + x];
    }
    __syncthreads();
    fft_lines<double2, false>(s_slab, plan.ax[2], plan.tw64[2], Nx, 1, Nx, true);
    const double inv_n = 1.0 / (double)n;
    const double gy2 = plan.g2pos[1][y];
    double tb = 1.0;
    if (MID == Mid::Tpa) {
        tb = tkin[band];
        if (!(tb >= 1e-12)) tb = 1.0;
    }
    for (int i = threadIdx.x; i < tot; i += blockDim.x) {
        int z = i / Nx, x = i - z * Nx;
        double g2 = plan.g2pos[0][x] + gy2 + plan.g2pos[2][z];
        double f;
        if (MID == Mid::Kinetic) f = 0.5 * g2 * inv_n;
        else if (MID == Mid::Tpa) f = tpa_k(0.5 * g2 / tb) * inv_n;
        else if (MID == Mid::Hartree) f = g2 > 0.0 ? 4.0 * M_PI / g2 * inv_n : 0.0;
        else f = inv_n;
        s_slab[i] = make_double2(s_slab[i].x * f, s_slab[i].y * f);
    }
    __syncthreads();
    fft_lines<double2, true>(s_slab, plan.ax[2], plan.tw64[2], Nx, 1, Nx, true);
    for (int i = threadIdx.x; i < tot; i += blockDim.x) {
        int z = i / Nx, x = i - z * Nx;
        base[z * zstride + x] = s_slab[i];
    }
}

// ---- xy inverse pass + epilogue ------------------------------------------------------
enum class Epi { Plain, Hpsi, Real };

template <Epi EPI>
__global__ void __launch_bounds__(FFT_THREADS)
k_xy_inverse(Fft3Plan plan, const double2 *__restrict__ buf, const double2 *__restrict__ psi,
             const double *__restrict__ v, ProjTables pt, const double2 *__restrict__ p,
             double2 *__restrict__ out, double *__restrict__ rout) {
    extern __shared__ double2 s_plane[];
    const int Nx = plan.ax[0].N, Ny = plan.ax[1].N, Nz = plan.ax[2].N;
    const int z = blockIdx.x, band = blockIdx.y;
    const size_t n = (size_t)Nx * Ny * Nz;
    const size_t plane = (size_t)Nx * Ny;
    const size_t off = (size_t)z * plane;
    const double2 *in = buf + band * n + off;
    for (int i = threadIdx.x; i < (int)plane; i += blockDim.x) s_plane[i] = in[i];
    __syncthreads();
    fft_lines<double2, true>(s_plane, plan.ax[1], plan.tw64[1], Nx, 1, Nx, true);
    fft_lines<double2, true>(s_plane, plan.ax[0], plan.tw64[0], Ny, Nx, 1, false);
    if (EPI == Epi::Plain) {
        double2 *o = out + band * n + off;
        for (int i = threadIdx.x; i < (int)plane; i += blockDim.x) o[i] = s_plane[i];
    } else if (EPI == Epi::Real) {
        double *o = rout + off;
        for (int i = threadIdx.x; i < (int)plane; i += blockDim.x) o[i] = s_plane[i].x;
    } else {
        const double2 *ps = psi + band * n + off;
        const double *vv = v + off;
        const int np = pt.natom * pt.nproj;
        const double2 *pb = p + (size_t)band * np;
        double2 *o = out + band * n + off;
        for (int i = threadIdx.x; i < (int)plane; i += blockDim.x) {
            double2 t = s_plane[i];
            double2 y = ps[i];
            double vi = vv[i];
            double ax = t.x + vi * y.x, ay = t.y + vi * y.y;
            const int g = (int)off + i;
            const int e0 = pt.c_rowptr[g], e1 = pt.c_rowptr[g + 1];
            for (int e = e0; e < e1; ++e) {
                const int a = pt.c_atom[e];
                const double *bt = pt.c_beta + 4 * (size_t)e;
                for (int j = 0; j < pt.nproj; ++j) {
                    const int aj = a * pt.nproj + j;
                    const double c = bt[j] * pt.e_kb[aj];
                    const double2 q = pb[aj];
                    ax += c * q.x;
                    ay += c * q.y;
                }
            }
            o[i] = make_double2(ax, ay);
        }
    }
}

// ---- projection <beta|psi> (atom-major gather) ------------------------------------------
constexpr int PROJ_THREADS = 256;
constexpr int PROJ_BANDS = 4;

__global__ void __launch_bounds__(PROJ_THREADS)
k_project(ProjTables pt, const double2 *__restrict__ psi, double2 *__restrict__ p, int nb,
          long long n, double dV) {
    const int a = blockIdx.x;
    const int b0 = blockIdx.y * PROJ_BANDS;
    const int e0 = pt.a_start[a], e1 = pt.a_start[a + 1];
    double acc[PROJ_BANDS][4][2];
#pragma unroll
    for (int bb = 0; bb < PROJ_BANDS; ++bb)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[bb][j][0] = acc[bb][j][1] = 0.0;
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int g = pt.a_idx[e];
        const double *bt = pt.a_beta + 4 * (size_t)e;
        const double be[4] = {bt[0], bt[1], bt[2], bt[3]};
#pragma unroll
        for (int bb = 0; bb < PROJ_BANDS; ++bb) {
            const int band = b0 + bb;
            if (band >= nb) break;
            const double2 v = psi[(size_t)band * n + g];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                acc[bb][j][0] += be[j] * v.x;
                acc[bb][j][1] += be[j] * v.y;
            }
        }
    }
    // block reduction, fixed order
    __shared__ double red[PROJ_THREADS / 32][PROJ_BANDS * 8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int bb = 0; bb < PROJ_BANDS; ++bb)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                double s = acc[bb][j][c];
                for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
                if (lane == 0) red[warp][(bb * 4 + j) * 2 + c] = s;
            }
    __syncthreads();
    if (threadIdx.x < PROJ_BANDS * 8) {
        double s = 0.0;
        for (int w = 0; w < PROJ_THREADS / 32; ++w) s += red[w][threadIdx.x];
        const int bb = threadIdx.x / 8, j = (threadIdx.x / 2) % 4, c = threadIdx.x % 2;
        const int band = b0 + bb;
        if (band < nb && j < pt.nproj) {
            double *dst = reinterpret_cast<double *>(p + (size_t)band * pt.natom * pt.nproj +
                                                     a * pt.nproj + j);
            dst[c] = s * dV;
        }
    }
}

// ---- launchers -------------------------------------------------------------------------
static size_t plane_bytes(const rsdft_ctx *ctx) { return (size_t)ctx->N[0] * ctx->N[1] * sizeof(double2); }
static size_t slab_bytes(const rsdft_ctx *ctx) { return (size_t)ctx->N[0] * ctx->N[2] * sizeof(double2); }

template <typename K> static rsdft_status set_smem(rsdft_ctx *ctx, K kernel, size_t bytes) {
    if (bytes > 48 * 1024)
        RS_CUDA(ctx, cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return RSDFT_OK;
}

rsdft_status fft_xy_forward(rsdft_ctx *ctx, Src kind, const double2 *src, const double2 *src2,
                            const double *theta, const int *act, const double *rsrc,
                            double2 *dst, int nb, cudaStream_t st) {
    if (nb <= 0) return RSDFT_OK;
    const size_t sm = plane_bytes(ctx);
    dim3 grid(ctx->N[2], nb);
    const double nxy = (double)ctx->N[0] * ctx->N[1];
    const double bpp = kind == Src::Plain ? 32.0 : (kind == Src::Residual ? 48.0 : 24.0);
    ProfScope ps(ctx, RSDFT_K_FFT_XY_FWD, 5.0 * nxy * std::log2(nxy) * ctx->N[2] * nb,
                 bpp * (double)ctx->n * nb, st);
    switch (kind) {
        case Src::Plain:
            RS_TRY(set_smem(ctx, k_xy_forward<Src::Plain>, sm));
            k_xy_forward<Src::Plain><<<grid, FFT_THREADS, sm, st>>>(ctx->fft, src, src2, theta, act, rsrc, dst);
            break;
        case Src::Residual:
            RS_TRY(set_smem(ctx, k_xy_forward<Src::Residual>, sm));
            k_xy_forward<Src::Residual><<<grid, FFT_THREADS, sm, st>>>(ctx->fft, src, src2, theta, act, rsrc, dst);
            break;
        case Src::RealField:
            RS_TRY(set_smem(ctx, k_xy_forward<Src::RealField>, sm));
            k_xy_forward<Src::RealField><<<grid, FFT_THREADS, sm, st>>>(ctx->fft, src, src2, theta, act, rsrc, dst);
            break;
    }
    RS_LAUNCHED(ctx, "k_xy_forward");
    return RSDFT_OK;
}

rsdft_status fft_z_mid(rsdft_ctx *ctx, Mid mid, double2 *buf, const double *tkin, int nb,
                       cudaStream_t st) {
    if (nb <= 0) return RSDFT_OK;
    const size_t sm = slab_bytes(ctx);
    dim3 grid(ctx->N[1], nb);
    ProfScope ps(ctx, RSDFT_K_FFT_Z, 10.0 * (double)ctx->n * std::log2((double)ctx->N[2]) * nb,
                 32.0 * (double)ctx->n * nb, st);
    switch (mid) {
        case Mid::Kinetic:
            RS_TRY(set_smem(ctx, k_z_mid<Mid::Kinetic>, sm));
            k_z_mid<Mid::Kinetic><<<grid, FFT_THREADS, sm, st>>>(ctx->fft, buf, tkin);
            break;
        case Mid::Tpa:
            RS_TRY(set_smem(ctx, k_z_mid<Mid::Tpa>, sm));
            k_z_mid<Mid::Tpa><<<grid, FFT_THREADS, sm, st>>>(ctx->fft, buf, tkin);
            break;
        case Mid::Hartree:
            RS_TRY(set_smem(ctx, k_z_mid<Mid::Hartree>, sm));
            k_z_mid<Mid::Hartree><<<grid, FFT_THREADS, sm, st>>>(ctx->fft, buf, tkin);
            break;
        case Mid::Scale:
            RS_TRY(set_smem(ctx, k_z_mid<Mid::Scale>, sm));
            k_z_mid<Mid::Scale><<<grid, FFT_THREADS, sm, st>>>(ctx->fft, buf, tkin);
            break;
    }
    RS_LAUNCHED(ctx, "k_z_mid");
    return RSDFT_OK;
}

rsdft_status fft_xy_inverse(rsdft_ctx *ctx, const double2 *buf, const double2 *psi,
                            const double2 *p, double2 *out, double *rout, int nb,
                            cudaStream_t st) {
    if (nb <= 0) return RSDFT_OK;
    const size_t sm = plane_bytes(ctx);
    dim3 grid(ctx->N[2], nb);
    const double nxy = (double)ctx->N[0] * ctx->N[1];
    const double bpp = rout ? 24.0 : (psi ? 48.0 : 32.0);
    ProfScope ps(ctx, RSDFT_K_FFT_XY_INV, 5.0 * nxy * std::log2(nxy) * ctx->N[2] * nb,
                 bpp * (double)ctx->n * nb + (psi ? 8.0 * (double)ctx->n : 0.0), st);
    if (rout) {
        RS_TRY(set_smem(ctx, k_xy_inverse<Epi::Real>, sm));
        k_xy_inverse<Epi::Real><<<grid, FFT_THREADS, sm, st>>>(ctx->fft, buf, psi, ctx->v, ctx->pt, p, out, rout);
    } else if (psi) {
        RS_TRY(set_smem(ctx, k_xy_inverse<Epi::Hpsi>, sm));
        k_xy_inverse<Epi::Hpsi><<<grid, FFT_THREADS, sm, st>>>(ctx->fft, buf, psi, ctx->v, ctx->pt, p, out, rout);
    } else {
        RS_TRY(set_smem(ctx, k_xy_inverse<Epi::Plain>, sm));
        k_xy_inverse<Epi::Plain><<<grid, FFT_THREADS, sm, st>>>(ctx->fft, buf, psi, ctx->v, ctx->pt, p, out, rout);
    }
    RS_LAUNCHED(ctx, "k_xy_inverse");
    return RSDFT_OK;
}

rsdft_status project(rsdft_ctx *ctx, const double2 *psi, double2 *p, int nb, cudaStream_t st) {
    if (nb <= 0 || ctx->pt.natom == 0) return RSDFT_OK;
    dim3 grid(ctx->pt.natom, cdiv(nb, PROJ_BANDS));
    const double ne = (double)ctx->nent;
    ProfScope ps(ctx, RSDFT_K_PROJECT, 4.0 * ctx->pt.nproj * ne * nb, 16.0 * ne * nb + 36.0 * ne, st);
    k_project<<<grid, PROJ_THREADS, 0, st>>>(ctx->pt, psi, p, nb, ctx->n, ctx->dV);
    RS_LAUNCHED(ctx, "k_project");
    return RSDFT_OK;
}

rsdft_status apply_h64(rsdft_ctx *ctx, const double2 *psi, double2 *hpsi, int nb, cudaStream_t st) {
    if (nb <= 0) return RSDFT_OK;
    RS_TRY(ensure_workspace(ctx, nb));
    RS_TRY(project(ctx, psi, ctx->ws.proj, nb, st));
    RS_TRY(fft_xy_forward(ctx, Src::Plain, psi, nullptr, nullptr, nullptr, nullptr, ctx->ws.T1, nb, st));
    RS_TRY(fft_z_mid(ctx, Mid::Kinetic, ctx->ws.T1, nullptr, nb, st));
    RS_TRY(fft_xy_inverse(ctx, ctx->ws.T1, psi, ctx->ws.proj, hpsi, nullptr, nb, st));
    return RSDFT_OK;
}

}  // namespace rsdft

using namespace rsdft;

extern "C" {

rsdft_status rsdft_apply_h(rsdft_ctx *ctx, const void *psi_dev, void *hpsi_dev, int nband,
                           rsdft_precision prec, void *stream) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (nband < 0 || (nband > 0 && (!psi_dev || !hpsi_dev)))
        return fail(ctx, RSDFT_E_INVALID, "bad psi/hpsi/nband");
    if (psi_dev == hpsi_dev && nband > 0) return fail(ctx, RSDFT_E_INVALID, "psi and hpsi must not overlap");
    if (prec != RSDFT_FP64) return fail(ctx, RSDFT_E_INVALID, "only RSDFT_FP64 is available");
    return apply_h64(ctx, (const double2 *)psi_dev, (double2 *)hpsi_dev, nband, as_stream(stream));
}

rsdft_status rsdft_project(rsdft_ctx *ctx, const void *psi_dev, void *p_dev, int nband, void *stream) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (nband < 0 || (nband > 0 && (!psi_dev || !p_dev))) return fail(ctx, RSDFT_E_INVALID, "bad arguments");
    return project(ctx, (const double2 *)psi_dev, (double2 *)p_dev, nband, as_stream(stream));
}

rsdft_status rsdft_precondition_tpa(rsdft_ctx *ctx, const void *r_dev, void *w_dev,
                                    const double *tkin_dev, int nband, void *stream) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (nband < 0 || (nband > 0 && (!r_dev || !w_dev || !tkin_dev)))
        return fail(ctx, RSDFT_E_INVALID, "bad arguments");
    if (nband == 0) return RSDFT_OK;
    cudaStream_t st = as_stream(stream);
    RS_TRY(ensure_workspace(ctx, nband));
    RS_TRY(fft_xy_forward(ctx, Src::Plain, (const double2 *)r_dev, nullptr, nullptr, nullptr, nullptr,
                          ctx->ws.T1, nband, st));
    RS_TRY(fft_z_mid(ctx, Mid::Tpa, ctx->ws.T1, tkin_dev, nband, st));
    RS_TRY(fft_xy_inverse(ctx, ctx->ws.T1, nullptr, nullptr, (double2 *)w_dev, nullptr, nband, st));
    return RSDFT_OK;
}

}  // extern "C"
