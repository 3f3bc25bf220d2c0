// SCF step around LOBPCG (the density and potential updates that the paper
// counts as "Others" in Fig. 1): density, FFT Hartree, LDA (Slater exchange +
// Perdew-Zunger 1981 correlation) or GGA-PBE, occupations (aufbau / Fermi-Dirac with mu
// by bisection), energies, Anderson mixing.  All FP64, all on the device;
// reductions are two-stage with a fixed order.
#include <cmath>
#include <algorithm>

#include "rsdft_internal.h"

namespace rsdft {

rsdft_status lobpcg_run(rsdft_ctx *ctx, double2 *x, int m, const rsdft_lobpcg_opts &o,
                        double *eig_host, double *res_host, rsdft_lobpcg_stats *stats,
                        cudaStream_t st);

constexpr double PZ_GAMMA = -0.1423, PZ_B1 = 1.0529, PZ_B2 = 0.3334;
constexpr double PZ_A = 0.0311, PZ_B = -0.048, PZ_C = 0.0020, PZ_D = -0.0116;
constexpr double RHO_MIN = 1e-12;
constexpr double ANDERSON_REG = 1e-10;
constexpr int RED_BLOCKS = 304;    // 2 x 152 SMs
constexpr int RED_THREADS = 256;
// layout of ScfWork::red (doubles)
constexpr int RED_PART = 0;                          // [56][RED_BLOCKS] partial sums
constexpr int RED_ANDERSON = 56 * RED_BLOCKS;        // [56] Anderson A and b
constexpr int RED_GAMMA = RED_ANDERSON + 64;         // [8] gamma, fallback flag
constexpr int RED_ENERGY = RED_GAMMA + 16;           // [8] energy sums
constexpr int RED_OCC = RED_ENERGY + 16;             // [2] mu, entropy
constexpr int RED_TOTAL = RED_OCC + 16;

__global__ void k_density(const double2 *__restrict__ x, const double *__restrict__ f, int nb,
                          long long n, double *__restrict__ rho) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) {
            const double2 v = x[(size_t)b * n + i];
            s += f[b] * (v.x * v.x + v.y * v.y);
        }
        rho[i] = s;
    }
}

// rho = sum_b f_b x_b^2 over real orbitals [nb][n] (the real Gamma-point form)
__global__ void k_density_real(const double *__restrict__ x, const double *__restrict__ f, int nb, long long n,
                               double *__restrict__ rho) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) {
            const double v = x[(size_t)b * n + i];
            s += f[b] * v * v;
        }
        rho[i] = s;
    }
}

__device__ __forceinline__ void lda_point(double rho, double &eps, double &v) {
    if (!(rho >= RHO_MIN)) { eps = 0.0; v = 0.0; return; }
    const double cx = -0.75 * cbrt(3.0 / M_PI);
    const double ex = cx * cbrt(rho);
    const double vx = (4.0 / 3.0) * ex;
    const double rs = cbrt(3.0 / (4.0 * M_PI * rho));
    double ec, vc;
    if (rs >= 1.0) {
        const double s = sqrt(rs);
        const double den = 1.0 + PZ_B1 * s + PZ_B2 * rs;
        ec = PZ_GAMMA / den;
        vc = ec * (1.0 + 7.0 / 6.0 * PZ_B1 * s + 4.0 / 3.0 * PZ_B2 * rs) / den;
    } else {
        const double ln = log(rs);
        ec = PZ_A * ln + PZ_B + PZ_C * rs * ln + PZ_D * rs;
        vc = PZ_A * ln + (PZ_B - PZ_A / 3.0) + 2.0 / 3.0 * PZ_C * rs * ln + (2.0 * PZ_D - PZ_C) / 3.0 * rs;
    }
    eps = ex + ec;
    v = vx + vc;
}

__global__ void k_lda(const double *__restrict__ rho, long long n, double *eps, double *vxc) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double e, v;
        lda_point(rho[i], e, v);
        eps[i] = e;
        vxc[i] = v;
    }
}

// ---- GGA: PBE (Perdew, Burke, Ernzerhof 1996; PW92 correlation of the uniform gas)
// e(rho, sigma) = rho (eps_x + eps_c), sigma = |grad rho|^2, spin-unpolarised:
//   eps_x = -(3/(4 pi)) k_F F_x(s), k_F = (3 pi^2 rho)^(1/3), s^2 = sigma/(4 k_F^2 rho^2),
//   F_x = 1 + kappa - kappa/(1 + mu s^2/kappa);
//   eps_c = eps_c^PW92(r_s) + H, t^2 = sigma/(4 k_s^2 rho^2), k_s^2 = 4 k_F/pi,
//   H = gamma ln(1 + (beta/gamma) t^2 (1 + A t^2)/(1 + A t^2 + A^2 t^4)),
//   A = (beta/gamma)/(exp(-eps_c^PW92/gamma) - 1).
// de/drho and de/dsigma by forward-mode differentiation: every quantity carries
// its two partial derivatives (Dual2), with the exact rules of each operation.
constexpr double PBE_KAPPA = 0.804, PBE_BETA = 0.06672455060314922;
constexpr double PW92_A0 = 0.031091, PW92_A1 = 0.21370;
constexpr double PW92_B1 = 7.5957, PW92_B2 = 3.5876, PW92_B3 = 1.6382, PW92_B4 = 0.49294;

struct Dual2 { double v, r, s; };   // value, d/drho, d/dsigma
__device__ __forceinline__ Dual2 dconst(double c) { return Dual2{c, 0.0, 0.0}; }
__device__ __forceinline__ Dual2 operator+(Dual2 a, Dual2 b) { return Dual2{a.v + b.v, a.r + b.r, a.s + b.s}; }
__device__ __forceinline__ Dual2 operator-(Dual2 a, Dual2 b) { return Dual2{a.v - b.v, a.r - b.r, a.s - b.s}; }
__device__ __forceinline__ Dual2 operator*(Dual2 a, Dual2 b) {
    return Dual2{a.v * b.v, a.r * b.v + a.v * b.r, a.s * b.v + a.v * b.s};
}
__device__ __forceinline__ Dual2 operator*(double c, Dual2 a) { return Dual2{c * a.v, c * a.r, c * a.s}; }
__device__ __forceinline__ Dual2 operator+(double c, Dual2 a) { return Dual2{c + a.v, a.r, a.s}; }
__device__ __forceinline__ Dual2 operator/(Dual2 a, Dual2 b) {
    const double q = a.v / b.v;
    return Dual2{q, (a.r - q * b.r) / b.v, (a.s - q * b.s) / b.v};
}
__device__ __forceinline__ Dual2 dlog(Dual2 a) { return Dual2{log(a.v), a.r / a.v, a.s / a.v}; }
__device__ __forceinline__ Dual2 dexp(Dual2 a) {
    const double e = exp(a.v);
    return Dual2{e, e * a.r, e * a.s};
}
__device__ __forceinline__ Dual2 dsqrt(Dual2 a) {
    const double q = sqrt(a.v);
    return Dual2{q, 0.5 * a.r / q, 0.5 * a.s / q};
}
__device__ __forceinline__ Dual2 dcbrt(Dual2 a) {
    const double c = cbrt(a.v);
    const double f = c / (3.0 * a.v);
    return Dual2{c, f * a.r, f * a.s};
}

__device__ Dual2 pbe_e(Dual2 rho, Dual2 sigma) {
    const double gamma = (1.0 - M_LN2) / (M_PI * M_PI);
    const double mu = PBE_BETA * M_PI * M_PI / 3.0;
    const Dual2 kf = dcbrt((3.0 * M_PI * M_PI) * rho);
    const Dual2 ex_unif = (-0.75 / M_PI) * kf;
    const Dual2 rho2 = rho * rho;
    const Dual2 s2 = sigma / (4.0 * (kf * kf * rho2));
    const Dual2 fx = dconst(1.0 + PBE_KAPPA) - PBE_KAPPA * (dconst(1.0) / (1.0 + (mu / PBE_KAPPA) * s2));
    const Dual2 rs = dcbrt(dconst(3.0 / (4.0 * M_PI)) / rho);
    const Dual2 srs = dsqrt(rs);
    const Dual2 den = (2.0 * PW92_A0) * (PW92_B1 * srs + PW92_B2 * rs + PW92_B3 * (rs * srs) + PW92_B4 * (rs * rs));
    const Dual2 ec = (-2.0 * PW92_A0) * ((1.0 + PW92_A1 * rs) * dlog(1.0 + dconst(1.0) / den));
    const Dual2 t2 = sigma / ((16.0 / M_PI) * (kf * rho2));
    const Dual2 A = dconst(PBE_BETA / gamma) / (dexp((-1.0 / gamma) * ec) - dconst(1.0));
    const Dual2 at2 = A * t2;
    const Dual2 H = gamma * dlog(1.0 + (PBE_BETA / gamma) * ((t2 * (1.0 + at2)) / (1.0 + at2 + at2 * at2)));
    return rho * (ex_unif * fx + ec + H);
}

// Per point: eps = e/rho, vloc = de/drho, and the flux h_a = 2 de/dsigma d_a rho
// in place of the gradient (zero where rho < 1e-12).
__global__ void k_pbe(const double *__restrict__ rho, double *__restrict__ g0, double *__restrict__ g1,
                      double *__restrict__ g2, long long n, double *__restrict__ eps, double *__restrict__ vloc) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double r = rho[i];
        if (!(r >= RHO_MIN)) {
            eps[i] = 0.0;
            vloc[i] = 0.0;
            g0[i] = g1[i] = g2[i] = 0.0;
            continue;
        }
        const double a = g0[i], b = g1[i], c = g2[i];
        const double sg = a * a + b * b + c * c;
        const Dual2 e = pbe_e(Dual2{r, 1.0, 0.0}, Dual2{sg, 0.0, 1.0});
        eps[i] = e.v / r;
        vloc[i] = e.r;
        const double f = 2.0 * e.s;
        g0[i] = f * a;
        g1[i] = f * b;
        g2[i] = f * c;
    }
}

__global__ void k_sub_acc(double *v, const double *__restrict__ d, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        v[i] -= d[i];
}

__global__ void k_add3(const double *a, const double *b, const double *c, long long n, double *out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = a[i] + b[i] + c[i];
}

// Occupations: one block; eig ascending.  out: [0] mu, [1] entropy.
__global__ void k_occupations(const double *__restrict__ eig, int m, double ne, double kT,
                              double *f, double *out) {
    __shared__ double sh[33];
    __shared__ double s_mu;
    if (kT <= 0.0) {
        const int full = (int)floor(ne / 2.0);
        const double rest = ne - 2.0 * full;
        for (int b = threadIdx.x; b < m; b += blockDim.x)
            f[b] = b < full ? 2.0 : (b == full && rest > 0.0 ? rest : 0.0);
        if (threadIdx.x == 0) {
            out[0] = eig[min(full, m - 1)];
            out[1] = 0.0;
        }
        return;
    }
    double lo = eig[0] - 50.0 * kT - 1.0, hi = eig[m - 1] + 50.0 * kT + 1.0;
    for (int it = 0; it < 200; ++it) {
        const double mu = 0.5 * (lo + hi);
        double s = 0.0;
        for (int b = threadIdx.x; b < m; b += blockDim.x) s += 2.0 / (1.0 + exp((eig[b] - mu) / kT));
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
            sh[32] = t;
        }
        __syncthreads();
        if (sh[32] > ne) hi = mu;
        else lo = mu;
    }
    if (threadIdx.x == 0) s_mu = 0.5 * (lo + hi);
    __syncthreads();
    const double mu = s_mu;
    double s = 0.0;
    for (int b = threadIdx.x; b < m; b += blockDim.x) {
        const double ft = 1.0 / (1.0 + exp((eig[b] - mu) / kT));
        f[b] = 2.0 * ft;
        double t = 0.0;
        if (ft > 0.0) t += ft * log(ft);
        if (ft < 1.0) t += (1.0 - ft) * log1p(-ft);
        s += t;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        out[0] = mu;
        out[1] = -2.0 * t;
    }
}

// Per-block partial sums of several point-wise products; then k_red_final.
// q = 0: vh*rho_in, 1: eps*rho_in, 2: vxc*rho_in, 3: (rho_out - rho_in)^2, 4: rho_out
__global__ void __launch_bounds__(RED_THREADS)
k_energy_partials(const double *__restrict__ rin, const double *__restrict__ rout,
                  const double *__restrict__ vh, const double *__restrict__ eps,
                  const double *__restrict__ vxc, long long n, double *part) {
    __shared__ double sh[5][RED_THREADS / 32];
    double acc[5] = {0, 0, 0, 0, 0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double r = rin[i], o = rout[i];
        acc[0] += vh[i] * r;
        acc[1] += eps[i] * r;
        acc[2] += vxc[i] * r;
        acc[3] += (o - r) * (o - r);
        acc[4] += o;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = 0; q < 5; ++q) {
        double s = acc[q];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) sh[q][warp] = s;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double s = 0.0;
        for (int w = 0; w < RED_THREADS / 32; ++w) s += sh[threadIdx.x][w];
        part[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
    }
}

__global__ void k_red_final(const double *part, int nblocks, int nq, double scale, double *out) {
    const int q = threadIdx.x;
    if (q >= nq) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[(size_t)q * nblocks + b];
    out[q] = s * scale;
}

// Anderson: with the history F_0..F_k (ring slots given by idx[0..k]), form
// A_ij = <dF_i|dF_j>, b_i = <dF_i|F_k>, dF_j = F_{j+1} - F_j, per block.
struct Hist {
    const double *f[8];
    const double *r[8];
};

__global__ void __launch_bounds__(RED_THREADS)
k_anderson_partials(Hist h, int k, long long n, double *part) {
    // k <= 7 differences -> k*k + k <= 56 sums
    __shared__ double sh[RED_THREADS / 32];
    const int nq = k * k + k;
    for (int q = 0; q < nq; ++q) {
        double s = 0.0;
        const int i = q < k * k ? q / k : q - k * k;
        const int j = q < k * k ? q % k : -1;
        for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
             p += (long long)gridDim.x * blockDim.x) {
            const double di = h.f[i + 1][p] - h.f[i][p];
            const double other = j >= 0 ? h.f[j + 1][p] - h.f[j][p] : h.f[k][p];
            s += di * other;
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < RED_THREADS / 32; ++w) t += sh[w];
            part[(size_t)q * gridDim.x + blockIdx.x] = t;
        }
    }
}

// Solve (A + reg max(diag A) I) gamma = b by Gaussian elimination with partial
// pivoting (k <= 7), sums[0..k*k) = A, sums[k*k..) = b.  gamma -> out[0..k);
// out[7] = 1 if the linear-mixing fallback applies (max diag A not > 0).
__global__ void k_anderson_solve(const double *sums, int k, double *out) {
    if (threadIdx.x != 0) return;
    double A[7][8];
    double scale = 0.0;
    for (int i = 0; i < k; ++i) scale = fmax(scale, sums[i * k + i]);
    if (!(scale > 0.0)) {
        for (int i = 0; i < 8; ++i) out[i] = 0.0;
        out[7] = 1.0;
        return;
    }
    for (int i = 0; i < k; ++i) {
        for (int j = 0; j < k; ++j) A[i][j] = sums[i * k + j] + (i == j ? ANDERSON_REG * scale : 0.0);
        A[i][k] = sums[k * k + i];
    }
    for (int c = 0; c < k; ++c) {
        int p = c;
        for (int r = c + 1; r < k; ++r)
            if (fabs(A[r][c]) > fabs(A[p][c])) p = r;
        if (p != c)
            for (int j = 0; j <= k; ++j) { double t = A[c][j]; A[c][j] = A[p][j]; A[p][j] = t; }
        for (int r = c + 1; r < k; ++r) {
            const double f = A[r][c] / A[c][c];
            for (int j = c; j <= k; ++j) A[r][j] -= f * A[c][j];
        }
    }
    double g[7];
    for (int i = k - 1; i >= 0; --i) {
        double s = A[i][k];
        for (int j = i + 1; j < k; ++j) s -= A[i][j] * g[j];
        g[i] = s / A[i][i];
    }
    for (int i = 0; i < 8; ++i) out[i] = 0.0;
    for (int i = 0; i < k; ++i) out[i] = g[i];
}

// rho_in <- (rho_k - sum g_j dR_j) + beta (F_k - sum g_j dF_j)
__global__ void k_anderson_update(Hist h, int k, const double *__restrict__ gam, double beta,
                                  long long n, double *rho_new) {
    const bool linear = k == 0 || gam[7] != 0.0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        double rb = h.r[k][p], fb = h.f[k][p];
        if (!linear)
            for (int j = 0; j < k; ++j) {
                rb -= gam[j] * (h.r[j + 1][p] - h.r[j][p]);
                fb -= gam[j] * (h.f[j + 1][p] - h.f[j][p]);
            }
        rho_new[p] = rb + beta * fb;
    }
}

__global__ void k_sub(const double *a, const double *b, long long n, double *out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = a[i] - b[i];
}

__global__ void k_fill(double *a, long long n, double v) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        a[i] = v;
}

__global__ void k_eband(const double *f, const double *eig, int m, double *out) {
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int b = 0; b < m; ++b) s += f[b] * eig[b];
    out[0] = s;
}

static int grid_for(long long n) { return std::max(1, std::min(cdiv(n, 256), 4 * 152)); }

rsdft_status density(rsdft_ctx *ctx, const double2 *x, const double *f, int nb, double *rho,
                     cudaStream_t st) {
    k_density<<<grid_for(ctx->n), 256, 0, st>>>(x, f, nb, ctx->n, rho);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_density");
    return RSDFT_OK;
}

static rsdft_status ensure_scf(rsdft_ctx *ctx, int nband, int depth) {
    ScfWork &s = ctx->scf;
    const size_t n = (size_t)ctx->n;
    if (!s.rho_in) {
        for (double **b : {&s.rho_in, &s.rho_out, &s.vh, &s.eps, &s.vxc, &s.veff})
            RS_TRY(dev_alloc(ctx, (void **)b, n * sizeof(double)));
        RS_TRY(dev_alloc(ctx, (void **)&s.cbuf, n * sizeof(double2)));
        RS_TRY(dev_alloc(ctx, (void **)&s.red, (size_t)RED_TOTAL * sizeof(double)));
    }
    if (depth + 1 > s.hist_cap) {
        RS_TRY(dev_alloc(ctx, (void **)&s.hist_rho, (size_t)(depth + 1) * n * sizeof(double)));
        RS_TRY(dev_alloc(ctx, (void **)&s.hist_f, (size_t)(depth + 1) * n * sizeof(double)));
        s.hist_cap = depth + 1;
    }
    if (nband > s.nband) {
        RS_TRY(dev_alloc(ctx, (void **)&s.f, nband * sizeof(double)));
        RS_TRY(dev_alloc(ctx, (void **)&s.eig, nband * sizeof(double)));
        s.nband = nband;
    }
    return RSDFT_OK;
}

rsdft_status hartree(rsdft_ctx *ctx, const double *rho, double *vh, cudaStream_t st) {
    RS_TRY(ensure_scf(ctx, 1, 0));
    RS_TRY(fft_xy_forward(ctx, Src::RealField, nullptr, nullptr, nullptr, nullptr, rho, ctx->scf.cbuf, 1, st));
    RS_TRY(fft_z_mid(ctx, Mid::Hartree, ctx->scf.cbuf, nullptr, 1, st));
    RS_TRY(fft_xy_inverse(ctx, ctx->scf.cbuf, nullptr, nullptr, nullptr, vh, 1, st));
    return RSDFT_OK;
}

// d_a f of a real field by FFT (i G_a; the Nyquist plane of an even axis is 0)
static rsdft_status real_derivative(rsdft_ctx *ctx, const double *f, int axis, double *out, cudaStream_t st) {
    const Mid mid = axis == 0 ? Mid::GradX : (axis == 1 ? Mid::GradY : Mid::GradZ);
    RS_TRY(fft_xy_forward(ctx, Src::RealField, nullptr, nullptr, nullptr, nullptr, f, ctx->scf.cbuf, 1, st));
    RS_TRY(fft_z_mid(ctx, mid, ctx->scf.cbuf, nullptr, 1, st));
    RS_TRY(fft_xy_inverse(ctx, ctx->scf.cbuf, nullptr, nullptr, nullptr, out, 1, st));
    return RSDFT_OK;
}

// PBE: eps_xc and v_xc = de/drho - sum_a d_a (2 de/dsigma d_a rho)
rsdft_status pbe(rsdft_ctx *ctx, const double *rho, double *eps, double *vxc, cudaStream_t st) {
    RS_TRY(ensure_scf(ctx, 1, 0));
    ScfWork &s = ctx->scf;
    const long long n = ctx->n;
    if (!s.gga) RS_TRY(dev_alloc(ctx, (void **)&s.gga, 4 * (size_t)n * sizeof(double)));
    double *g[3] = {s.gga, s.gga + n, s.gga + 2 * n};
    double *d = s.gga + 3 * n;
    for (int a = 0; a < 3; ++a) RS_TRY(real_derivative(ctx, rho, a, g[a], st));
    k_pbe<<<grid_for(n), 256, 0, st>>>(rho, g[0], g[1], g[2], n, eps, vxc);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_pbe");
    for (int a = 0; a < 3; ++a) {
        RS_TRY(real_derivative(ctx, g[a], a, d, st));
        k_sub_acc<<<grid_for(n), 256, 0, st>>>(vxc, d, n);
        count_launch(ctx);
        RS_LAUNCHED(ctx, "k_sub_acc");
    }
    return RSDFT_OK;
}

rsdft_status lda(rsdft_ctx *ctx, const double *rho, double *eps, double *vxc, cudaStream_t st) {
    k_lda<<<grid_for(ctx->n), 256, 0, st>>>(rho, ctx->n, eps, vxc);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_lda");
    return RSDFT_OK;
}

}  // namespace rsdft

using namespace rsdft;

extern "C" {

void rsdft_scf_default_opts(rsdft_scf_opts *o) {
    if (!o) return;
    o->n_electrons = 0.0;
    o->kT = 0.0;
    o->beta = 0.3;
    o->depth = 4;
    o->k_lobpcg = 3;
    o->first_maxit = 200;
    o->tol = 1e-6;
    o->precond = RSDFT_PRECOND_TPA;
    o->precision = RSDFT_FP64;
    o->tensor_cores = 0;
    o->later_tol = 0.0;
    o->xc = RSDFT_XC_LDA;
}

static rsdft_status check_scf_opts(rsdft_ctx *ctx, const rsdft_scf_opts *o, int nband) {
    if (!o || !(o->n_electrons > 0.0) || o->n_electrons > 2.0 * nband || !(o->kT >= 0.0) ||
        o->depth < 0 || o->depth > 7 || o->k_lobpcg < 0 || o->first_maxit < 0 || !(o->tol >= 0.0) ||
        !(o->later_tol >= 0.0) || (o->xc != RSDFT_XC_LDA && o->xc != RSDFT_XC_PBE) ||
        (o->precision != RSDFT_FP64 && o->precision != RSDFT_MIXED))
        return fail(ctx, RSDFT_E_INVALID, "bad SCF options");
    return RSDFT_OK;
}

rsdft_status rsdft_scf_init(rsdft_ctx *ctx, int nband, const rsdft_scf_opts *opts, void *stream) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (nband <= 0) return fail(ctx, RSDFT_E_INVALID, "nband must be positive");
    RS_TRY(check_scf_opts(ctx, opts, nband));
    RS_TRY(ensure_scf(ctx, nband, opts->depth));
    ScfWork &s = ctx->scf;
    const double vol = ctx->L[0] * ctx->L[1] * ctx->L[2];
    k_fill<<<grid_for(ctx->n), 256, 0, as_stream(stream)>>>(s.rho_in, ctx->n, opts->n_electrons / vol);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_fill");
    s.step = 0;
    s.hist_count = 0;
    s.ready = 1;
    return RSDFT_OK;
}

const double *rsdft_scf_density(const rsdft_ctx *ctx) {
    return (ctx && ctx->scf.ready) ? ctx->scf.rho_in : nullptr;
}

// One SCF step on complex orbitals (real = false) or on the real orbitals of the
// Gamma-point form (real = true: float64 [nband][n], FP64 only).
static rsdft_status scf_step_impl(rsdft_ctx *ctx, void *x_dev, int nband, const rsdft_scf_opts *opts,
                                  rsdft_scf_out *out, double *eig_host, double *occ_host, void *stream, bool real) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (!x_dev || nband <= 0 || 3LL * nband > ctx->n) return fail(ctx, RSDFT_E_INVALID, "bad x/nband");
    RS_TRY(check_scf_opts(ctx, opts, nband));
    if (real && opts->precision != RSDFT_FP64)
        return fail(ctx, RSDFT_E_INVALID, "the real Gamma-point SCF step runs in FP64 only");
    ScfWork &s = ctx->scf;
    if (!s.ready) return fail(ctx, RSDFT_E_INVALID, "call rsdft_scf_init first");
    if (opts->depth + 1 > s.hist_cap || nband > s.nband)
        return fail(ctx, RSDFT_E_INVALID, "options changed since rsdft_scf_init");
    cudaStream_t st = as_stream(stream);
    const long long n = ctx->n;
    const double dV = ctx->dV;
    // 1. effective potential from rho_in
    RS_TRY(hartree(ctx, s.rho_in, s.vh, st));
    if (opts->xc == RSDFT_XC_PBE) RS_TRY(pbe(ctx, s.rho_in, s.eps, s.vxc, st));
    else RS_TRY(lda(ctx, s.rho_in, s.eps, s.vxc, st));
    k_add3<<<grid_for(n), 256, 0, st>>>(ctx->vloc, s.vh, s.vxc, n, s.veff);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_add3");
    RS_CUDA(ctx, cudaMemcpyAsync(ctx->v, s.veff, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    // 2. LOBPCG
    rsdft_lobpcg_opts lo;
    rsdft_lobpcg_default_opts(&lo);
    lo.precond = opts->precond;
    lo.nconv = opts->kT > 0.0 ? nband : (int)std::min<double>(nband, std::ceil(opts->n_electrons / 2.0));
    lo.precision = opts->precision;
    lo.tensor_cores = opts->tensor_cores;
    if (s.step == 0) { lo.maxit = opts->first_maxit; lo.tol = opts->tol; }
    else if (opts->later_tol > 0.0) { lo.maxit = opts->first_maxit; lo.tol = opts->later_tol; }
    else { lo.maxit = opts->k_lobpcg; lo.tol = 0.0; lo.switch_tol = 0.0; }
    rsdft_lobpcg_stats ls{};
    rsdft_status lst = real ? rsdft_lobpcg_real(ctx, x_dev, nband, &lo, nullptr, nullptr, &ls, stream)
                            : lobpcg_run(ctx, (double2 *)x_dev, nband, lo, nullptr, nullptr, &ls, st);
    if (lst != RSDFT_OK && lst != RSDFT_E_NOT_CONVERGED) return lst;
    double *eig = ctx->ws.theta;
    // 3. occupations
    k_occupations<<<1, 512, 0, st>>>(eig, nband, opts->n_electrons, opts->kT, s.f, s.red + RED_OCC);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_occupations");
    // 4. rho_out
    if (real) {
        k_density_real<<<grid_for(n), 256, 0, st>>>((const double *)x_dev, s.f, nband, n, s.rho_out);
        count_launch(ctx);
        RS_LAUNCHED(ctx, "k_density_real");
    } else {
        RS_TRY(density(ctx, (const double2 *)x_dev, s.f, nband, s.rho_out, st));
    }
    // 5. energies
    double *part = s.red + RED_PART;
    double *sums = s.red + RED_ENERGY;
    k_energy_partials<<<RED_BLOCKS, RED_THREADS, 0, st>>>(s.rho_in, s.rho_out, s.vh, s.eps, s.vxc, n, part);
    count_launch(ctx);
    k_red_final<<<1, 32, 0, st>>>(part, RED_BLOCKS, 5, dV, sums);
    count_launch(ctx);
    k_eband<<<1, 32, 0, st>>>(s.f, eig, nband, sums + 5);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "energies");
    // 6. Anderson mixing: push (rho_in, F) into the ring
    const int cap = opts->depth + 1;
    const int slot = s.hist_count % cap;
    double *hr = s.hist_rho + (size_t)slot * n, *hf = s.hist_f + (size_t)slot * n;
    RS_CUDA(ctx, cudaMemcpyAsync(hr, s.rho_in, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    k_sub<<<grid_for(n), 256, 0, st>>>(s.rho_out, s.rho_in, n, hf);
    count_launch(ctx);
    s.hist_count++;
    const int have = std::min(s.hist_count, cap);
    const int k = opts->depth == 0 ? 0 : have - 1;
    Hist h{};
    for (int j = 0; j <= k; ++j) {
        const int sl = (s.hist_count - 1 - k + j) % cap;
        h.r[j] = s.hist_rho + (size_t)sl * n;
        h.f[j] = s.hist_f + (size_t)sl * n;
    }
    double *gam = s.red + RED_GAMMA;
    if (k > 0) {
        k_anderson_partials<<<RED_BLOCKS, RED_THREADS, 0, st>>>(h, k, n, part);
        count_launch(ctx);
        k_red_final<<<1, 64, 0, st>>>(part, RED_BLOCKS, k * k + k, dV, s.red + RED_ANDERSON);
        count_launch(ctx);
        k_anderson_solve<<<1, 32, 0, st>>>(s.red + RED_ANDERSON, k, gam);
        count_launch(ctx);
    }
    k_anderson_update<<<grid_for(n), 256, 0, st>>>(h, k, gam, opts->beta, n, s.rho_in);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "anderson");
    // outputs
    double hsum[8], occ2[2];
    RS_CUDA(ctx, cudaMemcpyAsync(hsum, sums, 6 * sizeof(double), cudaMemcpyDeviceToHost, st));
    RS_CUDA(ctx, cudaMemcpyAsync(occ2, s.red + RED_OCC, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (eig_host) RS_CUDA(ctx, cudaMemcpyAsync(eig_host, eig, nband * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (occ_host) RS_CUDA(ctx, cudaMemcpyAsync(occ_host, s.f, nband * sizeof(double), cudaMemcpyDeviceToHost, st));
    RS_CUDA(ctx, cudaStreamSynchronize(st));
    const double e_h = 0.5 * hsum[0], e_xc = hsum[1], e_vxc = hsum[2];
    const double drho = std::sqrt(hsum[3]);
    const double e_band = hsum[5];
    if (out) {
        out->e_band = e_band;
        out->e_h = e_h;
        out->e_xc = e_xc;
        out->e_vxc = e_vxc;
        out->e_tot = e_band - e_h - e_vxc + e_xc;
        out->mu = occ2[0];
        out->entropy = occ2[1];
        out->free_energy = out->e_tot - opts->kT * occ2[1];
        out->drho = drho;
        out->lobpcg_iterations = ls.iterations;
        out->lobpcg_iterations_mixed = ls.iterations_mixed;
        out->step = s.step;
    }
    s.step++;
    if (!std::isfinite(e_band) || !std::isfinite(drho))
        return fail(ctx, RSDFT_E_NUMERIC, "non-finite SCF energy or density change");
    return RSDFT_OK;
}

rsdft_status rsdft_scf_step(rsdft_ctx *ctx, void *x_dev, int nband, const rsdft_scf_opts *opts,
                            rsdft_scf_out *out, double *eig_host, double *occ_host, void *stream) {
    return scf_step_impl(ctx, x_dev, nband, opts, out, eig_host, occ_host, stream, false);
}

rsdft_status rsdft_scf_step_real(rsdft_ctx *ctx, void *x_dev, int nband, const rsdft_scf_opts *opts,
                                 rsdft_scf_out *out, double *eig_host, double *occ_host, void *stream) {
    return scf_step_impl(ctx, x_dev, nband, opts, out, eig_host, occ_host, stream, true);
}

rsdft_status rsdft_density(rsdft_ctx *ctx, const void *x_dev, const double *f_dev, int nband,
                           double *rho_dev, void *stream) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (nband < 0 || !rho_dev || (nband > 0 && (!x_dev || !f_dev)))
        return fail(ctx, RSDFT_E_INVALID, "bad density arguments");
    return density(ctx, (const double2 *)x_dev, f_dev, nband, rho_dev, as_stream(stream));
}

rsdft_status rsdft_hartree(rsdft_ctx *ctx, const double *rho_dev, double *vh_dev, void *stream) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (!rho_dev || !vh_dev) return fail(ctx, RSDFT_E_INVALID, "bad hartree arguments");
    return hartree(ctx, rho_dev, vh_dev, as_stream(stream));
}

rsdft_status rsdft_lda(rsdft_ctx *ctx, const double *rho_dev, double *eps_dev, double *vxc_dev,
                       void *stream) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (!rho_dev || !eps_dev || !vxc_dev) return fail(ctx, RSDFT_E_INVALID, "bad lda arguments");
    return lda(ctx, rho_dev, eps_dev, vxc_dev, as_stream(stream));
}

rsdft_status rsdft_xc_pbe(rsdft_ctx *ctx, const double *rho_dev, double *eps_dev, double *vxc_dev, void *stream) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (!rho_dev || !eps_dev || !vxc_dev) return fail(ctx, RSDFT_E_INVALID, "bad pbe arguments");
    return pbe(ctx, rho_dev, eps_dev, vxc_dev, as_stream(stream));
}

rsdft_status rsdft_occupations(rsdft_ctx *ctx, const double *eig_dev, int nband, double n_electrons,
                               double kT, double *f_dev, double *mu_host, double *entropy_host,
                               void *stream) {
    if (!ctx) return fail(nullptr, RSDFT_E_INVALID, "ctx is NULL");
    if (nband <= 0 || !eig_dev || !f_dev || !(n_electrons >= 0.0) || n_electrons > 2.0 * nband ||
        !(kT >= 0.0))
        return fail(ctx, RSDFT_E_INVALID, "bad occupation arguments");
    RS_TRY(ensure_scf(ctx, nband, 0));
    cudaStream_t st = as_stream(stream);
    double *o = ctx->scf.red + RED_OCC;
    k_occupations<<<1, 512, 0, st>>>(eig_dev, nband, n_electrons, kT, f_dev, o);
    count_launch(ctx);
    RS_LAUNCHED(ctx, "k_occupations");
    double h[2];
    RS_CUDA(ctx, cudaMemcpyAsync(h, o, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    RS_CUDA(ctx, cudaStreamSynchronize(st));
    if (mu_host) *mu_host = h[0];
    if (entropy_host) *entropy_host = h[1];
    return RSDFT_OK;
}

}  // extern "C"
