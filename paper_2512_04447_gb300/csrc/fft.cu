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
#include <algorithm>
#include <cmath>

#include <mutex>
#include <vector>

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
// x / d for x < 2^16 from the multiply-high divisor of d (mag = 0 means d = 1).
__device__ __forceinline__ int qdiv(int x, unsigned mag) { return mag ? (int)__umulhi((unsigned)x, mag) : x; }

// xy planes live in shared memory with an odd row stride RS = Nx | 1 (complex
// values): the lines of both transform directions are then read by consecutive
// threads without bank conflicts (successive rows start two banks apart).
__device__ __forceinline__ int plane_rs(int Nx) { return Nx | 1; }
// shared-memory index of plane element i = y Nx + x
__device__ __forceinline__ int pidx(int i, int Nx, int RS, unsigned nxmag) { return i + qdiv(i, nxmag) * (RS - Nx); }

// nlmag: multiply-high divisor of nlines.  Quotients and remainders of the
// index decomposition use it instead of integer division (total < 2^16).
template <typename V, bool INV>
__device__ void fft_lines(V *s, const AxisPlan &ax, const V *tw, int nlines, unsigned nlmag, int lstride,
                          int es, bool lines_fast) {
    const int N = ax.N;
    for (int t = 0; t < ax.nstage; ++t) {
        const int st = INV ? ax.nstage - 1 - t : t;
        const int r = ax.radix[st], len = ax.len[st], sub = ax.sub[st];
        const unsigned smag = ax.submag[st], bmag = ax.bfmag[st];
        const int nbf = N / r;
        const int total = nbf * nlines;
        const int twstep = N / len;
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            int line, bf;
            if (lines_fast) { bf = qdiv(idx, nlmag); line = idx - bf * nlines; }
            else { line = qdiv(idx, bmag); bf = idx - line * nbf; }
            const int b = qdiv(bf, smag), j = bf - b * sub;
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

// Tables of one precision: twiddles exp(-2 pi i k/N) and G_a^2 at each
// digit-reversed position.
template <typename V> struct FftTabs {
    AxisPlan ax[3];
    const V *tw[3];
    const typename Sc<V>::T *g2[3];
    const double *g1[3];   // G_a (first derivatives; FP64 real fields only)
    double inv_n;   // 1 / (Nx Ny Nz), formed on the host
};

static FftTabs<double2> tabs_of(const rsdft_ctx *ctx, double2 *) {
    FftTabs<double2> t;
    for (int a = 0; a < 3; ++a) {
        t.ax[a] = ctx->fft.ax[a];
        t.tw[a] = ctx->fft.tw64[a];
        t.g2[a] = ctx->fft.g2pos[a];
        t.g1[a] = ctx->fft.gpos[a];
    }
    t.inv_n = 1.0 / (double)ctx->n;
    return t;
}
static FftTabs<float2> tabs_of(const rsdft_ctx *ctx, float2 *) {
    FftTabs<float2> t;
    for (int a = 0; a < 3; ++a) {
        t.ax[a] = ctx->fft.ax[a];
        t.tw[a] = ctx->fft.tw32[a];
        t.g2[a] = ctx->fft.g2pos32[a];
        t.g1[a] = ctx->fft.gpos[a];
    }
    t.inv_n = 1.0 / (double)ctx->n;
    return t;
}
static const ProjT<double> &proj_of(const rsdft_ctx *ctx, double2 *) { return ctx->pt; }
static const ProjT<float> &proj_of(const rsdft_ctx *ctx, float2 *) { return ctx->pt32; }
static const double *v_of(const rsdft_ctx *ctx, double2 *) { return ctx->v; }
static const float *v_of(const rsdft_ctx *ctx, float2 *) { return ctx->v32; }

// Global -> shared copy of a plane or slab with several loads in flight per thread:
// each batch issues its loads (src(i)) before any of its stores (dst(i, v)); the
// plain loop would leave one load per thread in flight, and the passes stalled on
// load latency well below the HBM rate.
template <typename V, typename SrcF, typename DstF>
__device__ __forceinline__ void stage_in(int tot, SrcF src, DstF dst) {
    constexpr int U = sizeof(V) == 8 ? 8 : 2;
    for (int i0 = threadIdx.x; i0 < tot; i0 += U * blockDim.x) {
        V r[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < tot) r[u] = src(i);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < tot) dst(i, r[u]);
        }
    }
}

// ---- xy forward pass ------------------------------------------------------------
template <typename V, Src SRC>
__global__ void __launch_bounds__(FFT_THREADS, sizeof(V) == 8 ? 3 : 1)
k_xy_forward(FftTabs<V> tb, const V *__restrict__ src, const V *__restrict__ src2,
             const double *__restrict__ theta, const int *__restrict__ act,
             const double *__restrict__ rsrc, V *__restrict__ dst) {
    using T = typename Sc<V>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *s_plane = reinterpret_cast<V *>(smem_raw);
    const int Nx = tb.ax[0].N, Ny = tb.ax[1].N, Nz = tb.ax[2].N;
    const int z = blockIdx.x, band = blockIdx.y;
    const size_t n = (size_t)Nx * Ny * Nz;
    const size_t plane = (size_t)Nx * Ny;
    const size_t off = (size_t)z * plane;
    const int RS = plane_rs(Nx);
    const unsigned nxm = tb.ax[0].nmag;
    auto put = [&](int i, V v) { s_plane[pidx(i, Nx, RS, nxm)] = v; };
    if (SRC == Src::Plain) {
        const V *in = src + band * n + off;
        stage_in<V>((int)plane, [&](int i) { return in[i]; }, put);
    } else if (SRC == Src::Residual) {
        const int b = act[band];
        const T th = (T)theta[b];
        const V *hx = src + b * n + off;
        const V *x = src2 + b * n + off;
        stage_in<V>((int)plane, [&](int i) {
            const V h = hx[i], v = x[i];
            return mk<V>(h.x - th * v.x, h.y - th * v.y);
        }, put);
    } else {
        const double *in = rsrc + off;
        stage_in<V>((int)plane, [&](int i) { return mk<V>((T)in[i], (T)0); }, put);
    }
    __syncthreads();
    fft_lines<V, false>(s_plane, tb.ax[0], tb.tw[0], Ny, tb.ax[1].nmag, RS, 1, true);
    fft_lines<V, false>(s_plane, tb.ax[1], tb.tw[1], Nx, tb.ax[0].nmag, 1, RS, true);
    V *out = dst + band * n + off;
    for (int i = threadIdx.x; i < (int)plane; i += blockDim.x) out[i] = s_plane[pidx(i, Nx, RS, nxm)];
}

// ---- z pass with the per-G factor ------------------------------------------------
template <typename T> __device__ __forceinline__ T tpa_k(T x) {
    T num = (T)27 + x * ((T)18 + x * ((T)12 + (T)8 * x));
    return num / (num + (T)16 * x * x * x * x);
}

template <typename V, Mid MID>
__global__ void __launch_bounds__(FFT_THREADS, sizeof(V) == 8 ? 3 : 1)
k_z_mid(FftTabs<V> tb, V *__restrict__ buf, const double *__restrict__ tkin) {
    using T = typename Sc<V>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *s_slab = reinterpret_cast<V *>(smem_raw);
    const int Nx = tb.ax[0].N, Ny = tb.ax[1].N, Nz = tb.ax[2].N;
    const int y = blockIdx.x, band = blockIdx.y;
    const size_t n = (size_t)Nx * Ny * Nz;
    const size_t zstride = (size_t)Nx * Ny;
    V *base = buf + band * n + (size_t)y * Nx;
    const int tot = Nx * Nz;
    stage_in<V>(tot, [&](int i) {
        const int z = qdiv(i, tb.ax[0].nmag), x = i - z * Nx;
        return base[z * zstride + x];
    }, [&](int i, V v) { s_slab[i] = v; });
    __syncthreads();
    fft_lines<V, false>(s_slab, tb.ax[2], tb.tw[2], Nx, tb.ax[0].nmag, 1, Nx, true);
    const T inv_n = (T)tb.inv_n;
    const T gy2 = tb.g2[1][y];
    T tk = (T)1;
    if (MID == Mid::Tpa) {
        double t = tkin[band];
        if (!(t >= 1e-12)) t = 1.0;
        tk = (T)t;
    }
    if constexpr (MID == Mid::GradX || MID == Mid::GradY || MID == Mid::GradZ) {
        // i G_a / n: (re, im) -> (-f im, f re)
        for (int i = threadIdx.x; i < tot; i += blockDim.x) {
            const int z = qdiv(i, tb.ax[0].nmag), x = i - z * Nx;
            const T ga = (T)(MID == Mid::GradX ? tb.g1[0][x] : (MID == Mid::GradY ? tb.g1[1][y] : tb.g1[2][z]));
            const T f = ga * inv_n;
            s_slab[i] = mk<V>(-f * s_slab[i].y, f * s_slab[i].x);
        }
        __syncthreads();
        fft_lines<V, true>(s_slab, tb.ax[2], tb.tw[2], Nx, tb.ax[0].nmag, 1, Nx, true);
        for (int i = threadIdx.x; i < tot; i += blockDim.x) {
            const int z = qdiv(i, tb.ax[0].nmag), x = i - z * Nx;
            base[z * zstride + x] = s_slab[i];
        }
    } else {
        for (int i = threadIdx.x; i < tot; i += blockDim.x) {
            const int z = qdiv(i, tb.ax[0].nmag), x = i - z * Nx;
            T g2 = tb.g2[0][x] + gy2 + tb.g2[2][z];
            T f;
            if (MID == Mid::Kinetic) f = (T)0.5 * g2 * inv_n;
            else if (MID == Mid::Tpa) f = tpa_k<T>((T)0.5 * g2 / tk) * inv_n;
            else if (MID == Mid::Hartree) f = g2 > (T)0 ? (T)(4.0 * M_PI) / g2 * inv_n : (T)0;
            else f = inv_n;
            s_slab[i] = mk<V>(s_slab[i].x * f, s_slab[i].y * f);
        }
        __syncthreads();
        fft_lines<V, true>(s_slab, tb.ax[2], tb.tw[2], Nx, tb.ax[0].nmag, 1, Nx, true);
        for (int i = threadIdx.x; i < tot; i += blockDim.x) {
            const int z = qdiv(i, tb.ax[0].nmag), x = i - z * Nx;
            base[z * zstride + x] = s_slab[i];
        }
    }
}

// The four beta values of one projector-table entry (16- or 32-byte aligned: the
// tables are [nent][4]) in one 16-byte load (FP32) or two (FP64), instead of four
// scalar loads that each cost the L1 a wavefront per thread.
__device__ __forceinline__ void beta4(const float *bt, float b[4]) {
    const float4 q = *reinterpret_cast<const float4 *>(bt);
    b[0] = q.x;
    b[1] = q.y;
    b[2] = q.z;
    b[3] = q.w;
}
__device__ __forceinline__ void beta4(const double *bt, double b[4]) {
    const double2 q0 = reinterpret_cast<const double2 *>(bt)[0], q1 = reinterpret_cast<const double2 *>(bt)[1];
    b[0] = q0.x;
    b[1] = q0.y;
    b[2] = q1.x;
    b[3] = q1.y;
}

// ---- xy inverse pass + epilogue ------------------------------------------------------
enum class Epi { Plain, Hpsi, Real };

template <typename V, Epi EPI>
__global__ void __launch_bounds__(FFT_THREADS, sizeof(V) == 8 ? 3 : 1)
k_xy_inverse(FftTabs<V> tb, const V *__restrict__ buf, const V *__restrict__ psi,
             const typename Sc<V>::T *__restrict__ v, ProjT<typename Sc<V>::T> pt,
             const V *__restrict__ p, V *__restrict__ out, double *__restrict__ rout, int stage_pe) {
    using T = typename Sc<V>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *s_plane = reinterpret_cast<V *>(smem_raw);
    const int Nx = tb.ax[0].N, Ny = tb.ax[1].N, Nz = tb.ax[2].N;
    const int z = blockIdx.x, band = blockIdx.y;
    const size_t n = (size_t)Nx * Ny * Nz;
    const size_t plane = (size_t)Nx * Ny;
    const size_t off = (size_t)z * plane;
    const V *in = buf + band * n + off;
    const int RS = plane_rs(Nx);
    const unsigned nxm = tb.ax[0].nmag;
    stage_in<V>((int)plane, [&](int i) { return in[i]; }, [&](int i, V v) { s_plane[pidx(i, Nx, RS, nxm)] = v; });
    __syncthreads();
    fft_lines<V, true>(s_plane, tb.ax[1], tb.tw[1], Nx, tb.ax[0].nmag, 1, RS, true);
    fft_lines<V, true>(s_plane, tb.ax[0], tb.tw[0], Ny, tb.ax[1].nmag, RS, 1, true);
    if (EPI == Epi::Plain) {
        V *o = out + band * n + off;
        for (int i = threadIdx.x; i < (int)plane; i += blockDim.x) o[i] = s_plane[pidx(i, Nx, RS, nxm)];
    } else if (EPI == Epi::Real) {
        double *o = rout + off;
        for (int i = threadIdx.x; i < (int)plane; i += blockDim.x) o[i] = (double)s_plane[pidx(i, Nx, RS, nxm)].x;
    } else {
        const V *ps = psi + band * n + off;
        const T *vv = v + off;
        const int np = pt.natom * pt.nproj;
        const V *pb = p + (size_t)band * np;
        // E_aj <beta_aj|psi> of this band, staged once per CTA after the plane
        // (when it fits; else read from global memory)
        V *s_pe = s_plane + (size_t)Ny * RS;
        if (stage_pe) {
            for (int q = threadIdx.x; q < np; q += blockDim.x) {
                const V c = pb[q];
                const T e = pt.e_kb[q];
                s_pe[q] = mk<V>(e * c.x, e * c.y);
            }
            __syncthreads();
        }
        V *o = out + band * n + off;
        for (int i = threadIdx.x; i < (int)plane; i += blockDim.x) {
            V t = s_plane[pidx(i, Nx, RS, nxm)];
            V y = ps[i];
            T vi = vv[i];
            T ax = t.x + vi * y.x, ay = t.y + vi * y.y;
            const int g = (int)off + i;
            const int e0 = pt.c_rowptr[g], e1 = pt.c_rowptr[g + 1];
            for (int e = e0; e < e1; ++e) {
                const int a0 = pt.c_atom[e] * pt.nproj;
                T bt[4];
                beta4(pt.c_beta + 4 * (size_t)e, bt);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (j >= pt.nproj) break;
                    V q;
                    if (stage_pe) {
                        q = s_pe[a0 + j];
                    } else {
                        const V c = pb[a0 + j];
                        const T ek = pt.e_kb[a0 + j];
                        q = mk<V>(ek * c.x, ek * c.y);
                    }
                    const T c = bt[j];
                    ax += c * q.x;
                    ay += c * q.y;
                }
            }
            o[i] = mk<V>(ax, ay);
        }
    }
}

// ---- projection <beta|psi> (atom-major gather) ------------------------------------------
constexpr int PROJ_THREADS = 256;
constexpr int PROJ_BANDS = 4;

template <typename V>
__global__ void __launch_bounds__(PROJ_THREADS)
k_project(ProjT<typename Sc<V>::T> pt, const V *__restrict__ psi, V *__restrict__ p, int nb,
          long long n, double dV) {
    using T = typename Sc<V>::T;
    const int a = blockIdx.x;
    const int b0 = blockIdx.y * PROJ_BANDS;
    const int e0 = pt.a_start[a], e1 = pt.a_start[a + 1];
    T acc[PROJ_BANDS][4][2];
#pragma unroll
    for (int bb = 0; bb < PROJ_BANDS; ++bb)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[bb][j][0] = acc[bb][j][1] = (T)0;
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int g = pt.a_idx[e];
        T be[4];
        beta4(pt.a_beta + 4 * (size_t)e, be);
#pragma unroll
        for (int bb = 0; bb < PROJ_BANDS; ++bb) {
            const int band = b0 + bb;
            if (band >= nb) break;
            const V v = psi[(size_t)band * n + g];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                acc[bb][j][0] += be[j] * v.x;
                acc[bb][j][1] += be[j] * v.y;
            }
        }
    }
    // block reduction, fixed order
    __shared__ T red[PROJ_THREADS / 32][PROJ_BANDS * 8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int bb = 0; bb < PROJ_BANDS; ++bb)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                T s = acc[bb][j][c];
                for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
                if (lane == 0) red[warp][(bb * 4 + j) * 2 + c] = s;
            }
    __syncthreads();
    if (threadIdx.x < PROJ_BANDS * 8) {
        T s = (T)0;
        for (int w = 0; w < PROJ_THREADS / 32; ++w) s += red[w][threadIdx.x];
        const int bb = threadIdx.x / 8, j = (threadIdx.x / 2) % 4, c = threadIdx.x % 2;
        const int band = b0 + bb;
        if (band < nb && j < pt.nproj) {
            T *dst = reinterpret_cast<T *>(p + (size_t)band * pt.natom * pt.nproj + a * pt.nproj + j);
            dst[c] = s * (T)dV;
        }
    }
}

__global__ void k_to_float(const double *__restrict__ in, long long n, float *__restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

// ---- launchers -------------------------------------------------------------------------
template <typename V> static size_t plane_bytes(const rsdft_ctx *ctx) {
    return (size_t)(ctx->N[0] | 1) * ctx->N[1] * sizeof(V);   // odd row stride
}
template <typename V> static size_t slab_bytes(const rsdft_ctx *ctx) {
    return (size_t)ctx->N[0] * ctx->N[2] * sizeof(V);
}

constexpr size_t MAX_DYN_SMEM = 227 * 1024;   // largest dynamic shared memory of one CTA

// The attribute is per function and process-wide, so it is raised once to the
// largest size (occupancy follows each launch's own dynamic size); lowering it
// per launch would race with launches of other contexts on other threads.
template <typename K> static rsdft_status set_smem(rsdft_ctx *ctx, K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return RSDFT_OK;
    if (bytes > MAX_DYN_SMEM) return fail(ctx, RSDFT_E_INVALID, "plane needs %zu B of shared memory", bytes);
    static std::mutex mu;
    static std::vector<const void *> done;
    std::lock_guard<std::mutex> g(mu);
    const void *key = reinterpret_cast<const void *>(kernel);
    if (std::find(done.begin(), done.end(), key) == done.end()) {
        RS_CUDA(ctx, cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MAX_DYN_SMEM));
        done.push_back(key);
    }
    return RSDFT_OK;
}

template <typename V>
rsdft_status fft_xy_forward_t(rsdft_ctx *ctx, Src kind, const V *src, const V *src2,
                              const double *theta, const int *act, const double *rsrc, V *dst,
                              int nb, cudaStream_t st) {
    if (nb <= 0) return RSDFT_OK;
    const size_t sm = plane_bytes<V>(ctx);
    dim3 grid(ctx->N[2], nb);
    const double nxy = (double)ctx->N[0] * ctx->N[1];
    const double e = (double)sizeof(V);
    const double bpp = kind == Src::Plain ? 2 * e : (kind == Src::Residual ? 3 * e : 8.0 + e);
    ProfScope ps(ctx, RSDFT_K_FFT_XY_FWD, 5.0 * nxy * std::log2(nxy) * ctx->N[2] * nb,
                 bpp * (double)ctx->n * nb, st);
    const FftTabs<V> tb = tabs_of(ctx, (V *)nullptr);
    switch (kind) {
        case Src::Plain:
            RS_TRY(set_smem(ctx, k_xy_forward<V, Src::Plain>, sm));
            k_xy_forward<V, Src::Plain><<<grid, FFT_THREADS, sm, st>>>(tb, src, src2, theta, act, rsrc, dst);
            break;
        case Src::Residual:
            RS_TRY(set_smem(ctx, k_xy_forward<V, Src::Residual>, sm));
            k_xy_forward<V, Src::Residual><<<grid, FFT_THREADS, sm, st>>>(tb, src, src2, theta, act, rsrc, dst);
            break;
        case Src::RealField:
            RS_TRY(set_smem(ctx, k_xy_forward<V, Src::RealField>, sm));
            k_xy_forward<V, Src::RealField><<<grid, FFT_THREADS, sm, st>>>(tb, src, src2, theta, act, rsrc, dst);
            break;
    }
    RS_LAUNCHED(ctx, "k_xy_forward");
    return RSDFT_OK;
}

template <typename V>
rsdft_status fft_z_mid_t(rsdft_ctx *ctx, Mid mid, V *buf, const double *tkin, int nb,
                         cudaStream_t st) {
    if (nb <= 0) return RSDFT_OK;
    const size_t sm = slab_bytes<V>(ctx);
    dim3 grid(ctx->N[1], nb);
    ProfScope ps(ctx, RSDFT_K_FFT_Z, 10.0 * (double)ctx->n * std::log2((double)ctx->N[2]) * nb,
                 2.0 * sizeof(V) * (double)ctx->n * nb, st);
    const FftTabs<V> tb = tabs_of(ctx, (V *)nullptr);
    switch (mid) {
        case Mid::Kinetic:
            RS_TRY(set_smem(ctx, k_z_mid<V, Mid::Kinetic>, sm));
            k_z_mid<V, Mid::Kinetic><<<grid, FFT_THREADS, sm, st>>>(tb, buf, tkin);
            break;
        case Mid::Tpa:
            RS_TRY(set_smem(ctx, k_z_mid<V, Mid::Tpa>, sm));
            k_z_mid<V, Mid::Tpa><<<grid, FFT_THREADS, sm, st>>>(tb, buf, tkin);
            break;
        case Mid::Hartree:
            RS_TRY(set_smem(ctx, k_z_mid<V, Mid::Hartree>, sm));
            k_z_mid<V, Mid::Hartree><<<grid, FFT_THREADS, sm, st>>>(tb, buf, tkin);
            break;
        case Mid::Scale:
            RS_TRY(set_smem(ctx, k_z_mid<V, Mid::Scale>, sm));
            k_z_mid<V, Mid::Scale><<<grid, FFT_THREADS, sm, st>>>(tb, buf, tkin);
            break;
        case Mid::GradX:
            RS_TRY(set_smem(ctx, k_z_mid<V, Mid::GradX>, sm));
            k_z_mid<V, Mid::GradX><<<grid, FFT_THREADS, sm, st>>>(tb, buf, tkin);
            break;
        case Mid::GradY:
            RS_TRY(set_smem(ctx, k_z_mid<V, Mid::GradY>, sm));
            k_z_mid<V, Mid::GradY><<<grid, FFT_THREADS, sm, st>>>(tb, buf, tkin);
            break;
        case Mid::GradZ:
            RS_TRY(set_smem(ctx, k_z_mid<V, Mid::GradZ>, sm));
            k_z_mid<V, Mid::GradZ><<<grid, FFT_THREADS, sm, st>>>(tb, buf, tkin);
            break;
    }
    RS_LAUNCHED(ctx, "k_z_mid");
    return RSDFT_OK;
}

template <typename V>
rsdft_status fft_xy_inverse_t(rsdft_ctx *ctx, const V *buf, const V *psi, const V *p, V *out,
                              double *rout, int nb, cudaStream_t st) {
    if (nb <= 0) return RSDFT_OK;
    const size_t sm = plane_bytes<V>(ctx);
    dim3 grid(ctx->N[2], nb);
    const double nxy = (double)ctx->N[0] * ctx->N[1];
    const double e = (double)sizeof(V);
    const double bpp = rout ? e + 8.0 : (psi ? 3 * e : 2 * e);
    ProfScope ps(ctx, RSDFT_K_FFT_XY_INV, 5.0 * nxy * std::log2(nxy) * ctx->N[2] * nb,
                 bpp * (double)ctx->n * nb + (psi ? 0.5 * e * (double)ctx->n : 0.0), st);
    const FftTabs<V> tb = tabs_of(ctx, (V *)nullptr);
    const auto &pt = proj_of(ctx, (V *)nullptr);
    const auto *v = v_of(ctx, (V *)nullptr);
    if (rout) {
        RS_TRY(set_smem(ctx, k_xy_inverse<V, Epi::Real>, sm));
        k_xy_inverse<V, Epi::Real><<<grid, FFT_THREADS, sm, st>>>(tb, buf, psi, v, pt, p, out, rout, 0);
    } else if (psi) {
        // the plane plus, when it fits, the band's E_aj <beta_aj|psi> after it
        const size_t smh = sm + (size_t)pt.natom * pt.nproj * sizeof(V);
        const int stage = smh <= MAX_DYN_SMEM ? 1 : 0;
        const size_t smu = stage ? smh : sm;
        RS_TRY(set_smem(ctx, k_xy_inverse<V, Epi::Hpsi>, smu));
        k_xy_inverse<V, Epi::Hpsi><<<grid, FFT_THREADS, smu, st>>>(tb, buf, psi, v, pt, p, out, rout, stage);
    } else {
        RS_TRY(set_smem(ctx, k_xy_inverse<V, Epi::Plain>, sm));
        k_xy_inverse<V, Epi::Plain><<<grid, FFT_THREADS, sm, st>>>(tb, buf, psi, v, pt, p, out, rout, 0);
    }
    RS_LAUNCHED(ctx, "k_xy_inverse");
    return RSDFT_OK;
}

template <typename V>
rsdft_status project_t(rsdft_ctx *ctx, const V *psi, V *p, int nb, cudaStream_t st) {
    if (nb <= 0 || ctx->pt.natom == 0) return RSDFT_OK;
    dim3 grid(ctx->pt.natom, cdiv(nb, PROJ_BANDS));
    const double ne = (double)ctx->nent;
    const double e = (double)sizeof(V);
    ProfScope ps(ctx, RSDFT_K_PROJECT, 4.0 * ctx->pt.nproj * ne * nb, e * ne * nb + (4 + 2 * e) * ne, st);
    k_project<V><<<grid, PROJ_THREADS, 0, st>>>(proj_of(ctx, (V *)nullptr), psi, p, nb, ctx->n, ctx->dV);
    RS_LAUNCHED(ctx, "k_project");
    return RSDFT_OK;
}

rsdft_status fft_xy_forward(rsdft_ctx *ctx, Src kind, const double2 *src, const double2 *src2,
                            const double *theta, const int *act, const double *rsrc,
                            double2 *dst, int nb, cudaStream_t st) {
    return fft_xy_forward_t<double2>(ctx, kind, src, src2, theta, act, rsrc, dst, nb, st);
}
rsdft_status fft_xy_forward32(rsdft_ctx *ctx, Src kind, const float2 *src, const float2 *src2,
                              const double *theta, const int *act, float2 *dst, int nb,
                              cudaStream_t st) {
    return fft_xy_forward_t<float2>(ctx, kind, src, src2, theta, act, nullptr, dst, nb, st);
}
rsdft_status fft_z_mid(rsdft_ctx *ctx, Mid mid, double2 *buf, const double *tkin, int nb,
                       cudaStream_t st) {
    return fft_z_mid_t<double2>(ctx, mid, buf, tkin, nb, st);
}
rsdft_status fft_z_mid32(rsdft_ctx *ctx, Mid mid, float2 *buf, const double *tkin, int nb,
                         cudaStream_t st) {
    return fft_z_mid_t<float2>(ctx, mid, buf, tkin, nb, st);
}
rsdft_status fft_xy_inverse(rsdft_ctx *ctx, const double2 *buf, const double2 *psi,
                            const double2 *p, double2 *out, double *rout, int nb,
                            cudaStream_t st) {
    return fft_xy_inverse_t<double2>(ctx, buf, psi, p, out, rout, nb, st);
}
rsdft_status fft_xy_inverse32(rsdft_ctx *ctx, const float2 *buf, const float2 *psi,
                              const float2 *p, float2 *out, int nb, cudaStream_t st) {
    return fft_xy_inverse_t<float2>(ctx, buf, psi, p, out, nullptr, nb, st);
}
rsdft_status project(rsdft_ctx *ctx, const double2 *psi, double2 *p, int nb, cudaStream_t st) {
    return project_t<double2>(ctx, psi, p, nb, st);
}
rsdft_status project32(rsdft_ctx *ctx, const float2 *psi, float2 *p, int nb, cudaStream_t st) {
    return project_t<float2>(ctx, psi, p, nb, st);
}

rsdft_status refresh_v32(rsdft_ctx *ctx, cudaStream_t st) {
    k_to_float<<<std::max(1, std::min(cdiv(ctx->n, 256), 608)), 256, 0, st>>>(ctx->v, ctx->n, ctx->v32);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_to_float");
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

// FP32 H psi; the FP32 copy of V must be current (refresh_v32).
rsdft_status apply_h32(rsdft_ctx *ctx, const float2 *psi, float2 *hpsi, int nb, cudaStream_t st) {
    if (nb <= 0) return RSDFT_OK;
    RS_TRY(ensure_workspace(ctx, nb));
    float2 *proj = reinterpret_cast<float2 *>(ctx->ws.proj);
    float2 *t1 = reinterpret_cast<float2 *>(ctx->ws.T1);
    RS_TRY(project32(ctx, psi, proj, nb, st));
    RS_TRY(fft_xy_forward32(ctx, Src::Plain, psi, nullptr, nullptr, nullptr, t1, nb, st));
    RS_TRY(fft_z_mid32(ctx, Mid::Kinetic, t1, nullptr, nb, st));
    RS_TRY(fft_xy_inverse32(ctx, t1, psi, proj, hpsi, nb, st));
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
    if (prec == RSDFT_MIXED) {
        RS_TRY(refresh_v32(ctx, as_stream(stream)));
        return apply_h32(ctx, (const float2 *)psi_dev, (float2 *)hpsi_dev, nband, as_stream(stream));
    }
    if (prec != RSDFT_FP64) return fail(ctx, RSDFT_E_INVALID, "unknown precision");
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
