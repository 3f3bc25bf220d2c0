/*
 * rsdft.h -- C ABI of the GB300-native real-space Kohn-Sham LOBPCG path.
 *
 * The method is the SCF iteration of Ito's QUMASUN paper (arXiv 2512.04447):
 * per iteration, (1) the FFT Laplacian on all orbitals at once, (2) GEMMs that
 * form the subspace matrices H and S in LOBPCG, (3) the generalised Hermitian
 * eigenproblem reduced by a Cholesky factorisation and two triangular solves
 * (Eq. 1), and (4) the Kleinman-Bylander nonlocal operator, plus the density
 * and potential updates ("Others", Fig. 1).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Cell: orthorhombic, edges (Lx, Ly, Lz) bohr.  Grid (Nx, Ny, Nz), each
 *    N 5-smooth (2^a 3^b 5^c) with 2 <= N <= 128 (RSDFT_E_GRID_NOT_5SMOOTH
 *    otherwise).  Point r = (ix Lx/Nx, iy Ly/Ny, iz Lz/Nz); linear index
 *    i = (iz*Ny + iy)*Nx + ix (x fastest); n = Nx*Ny*Nz; dV = Lx*Ly*Lz/n.
 *  - Orbital blocks: [nband][n] complex128 (interleaved re, im), band-major.
 *    Inner product <a|b> = sum_r conj(a(r)) b(r) dV; orbitals are
 *    normalised in that metric.
 *  - Kinetic operator: T psi = IFFT(|G|^2/2 FFT(psi)), G = 2 pi k / L with k
 *    in FFT order (0..N/2-1, -N/2..-1).
 *  - Nonlocal operator: sum_{a,j} |beta_aj> E_aj <beta_aj|psi>, with
 *    projectors s, p_x, p_y, p_z = (1, d_x/rc, d_y/rc, d_z/rc) exp(-|d|^2/(2 rc^2)),
 *    d the minimal-image displacement from atom a, truncated to |d| < rcut and
 *    normalised on the grid (sum beta^2 dV = 1).
 *  - Pointers named *_dev are device memory owned by the caller; *_host are
 *    host memory owned by the caller.  Nothing is retained after a call
 *    returns except by rsdft_create (which copies its inputs).
 *  - Every call returns an rsdft_status.  No call aborts or throws.  On
 *    failure rsdft_last_error(ctx) describes it; caller-owned outputs are left
 *    in their last valid state.  A context is used by one host thread at a
 *    time; work is issued on the CUDA stream passed in (NULL = legacy stream),
 *    and calls that return host values synchronise that stream first.
 */
#ifndef RSDFT_H
#define RSDFT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rsdft_ctx rsdft_ctx;

typedef enum {
    RSDFT_OK = 0,
    RSDFT_E_INVALID = 1,           /* bad argument (null, size, range)            */
    RSDFT_E_GRID_NOT_5SMOOTH = 2,  /* a grid dimension is not 2^a 3^b 5^c <= 128  */
    RSDFT_E_OOM = 3,               /* device allocation failed                    */
    RSDFT_E_CUDA = 4,              /* a CUDA runtime call or launch failed        */
    RSDFT_E_NOT_SPD = 5,           /* overlap matrix has fewer independent columns
                                      than wanted eigenpairs                       */
    RSDFT_E_NUMERIC = 6,           /* NaN/Inf met in residuals or energies        */
    RSDFT_E_TIMEOUT = 7,           /* reserved: a bounded device wait gave up     */
    RSDFT_E_NOT_CONVERGED = 8      /* informational: outputs valid, tol not met   */
} rsdft_status;

typedef enum { RSDFT_FP64 = 0, RSDFT_MIXED = 1 } rsdft_precision;
/* RSDFT_PRECOND_LEARNED: TPA plus the learned network correction (weights set
 * with rsdft_set_precond_weights; RSDFT_E_INVALID without them). */
typedef enum { RSDFT_PRECOND_NONE = 0, RSDFT_PRECOND_TPA = 1, RSDFT_PRECOND_LEARNED = 2 } rsdft_precond;

/* Lattice vectors as rows, bohr.  Only diagonal (orthorhombic) cells are
 * accepted; off-diagonal entries must be 0 (RSDFT_E_INVALID otherwise). */
typedef struct { double a[3][3]; } rsdft_cell;

/* Grid points along x, y, z. */
typedef struct { int n[3]; } rsdft_grid;

/* Gaussian KB projectors (the synthetic pseudo-atoms of the workloads). */
typedef struct {
    int natom;             /* >= 0                                               */
    const double *pos;     /* [natom][3] bohr, host                              */
    int nproj;             /* 1 (s) or 4 (s, p_x, p_y, p_z)                      */
    double rc;             /* Gaussian radius, bohr, > 0                         */
    double rcut;           /* truncation radius, 0 < rcut < min(L)/2             */
    const double *e_kb;    /* [natom][nproj] KB energies, Ha, host               */
} rsdft_projectors;

/* ---------------------------------------------------------------------------
 * Context: grid, FFT tables, local potential, projector tables, device arena.
 * Follows the paper's statement of the problem (H = T + V + V_NL on a
 * real-space grid).  v_loc_host: [n] local potential, Ha, copied.  proj may be
 * NULL (no nonlocal term).  On success *out owns all device memory it uses;
 * release it with rsdft_destroy.
 */
rsdft_status rsdft_create(const rsdft_cell *cell, const rsdft_grid *grid,
                          const double *v_loc_host, const rsdft_projectors *proj,
                          rsdft_ctx **out);
void rsdft_destroy(rsdft_ctx *ctx);

/* Text of the last error on ctx (or, when ctx is NULL, of the last failed
 * rsdft_create or context-free call on this thread).  Valid until the next
 * call on the same ctx. */
const char *rsdft_last_error(const rsdft_ctx *ctx);

/* Input builder for the synthetic workloads: V(r) = sum_a -Z exp(-|d_a|^2 /
 * (2 sigma^2)), minimal-image d_a.  Host only; out_host is [n] doubles. */
rsdft_status rsdft_gaussian_vloc(const rsdft_cell *cell, const rsdft_grid *grid, int natom,
                                 const double *pos_host, double Z, double sigma,
                                 double *out_host);

/* Replace the local potential V(r) used by H (e.g. V_loc + V_H + V_xc).
 * v: [n] doubles, on the device when on_device != 0, else on the host. */
rsdft_status rsdft_set_potential(rsdft_ctx *ctx, const double *v, int on_device, void *stream);

/* Number of projector table entries (points inside all spheres, summed over
 * atoms), for sizing and roofline accounting. */
long long rsdft_projector_entries(const rsdft_ctx *ctx);

/* ---------------------------------------------------------------------------
 * H psi for a block of orbitals (SCF tasks (1) and (4)): batched 3D FFT
 * kinetic term with the local-potential product and the projector scatter
 * fused into the last pass.  psi_dev, hpsi_dev: [nband][n] complex128
 * (RSDFT_FP64) or complex64 (RSDFT_MIXED); must not overlap.  nband >= 0.
 */
rsdft_status rsdft_apply_h(rsdft_ctx *ctx, const void *psi_dev, void *hpsi_dev, int nband,
                           rsdft_precision prec, void *stream);

/* Projector coefficients p[b][a*nproj + j] = <beta_aj|psi_b> (complex128).
 * psi_dev: [nband][n] complex128; p_dev: [nband][natom*nproj] complex128. */
rsdft_status rsdft_project(rsdft_ctx *ctx, const void *psi_dev, void *p_dev, int nband,
                           void *stream);

/* Teter-Payne-Allan preconditioner: w_b = IFFT(K(|G|^2/2 / t_b) FFT(r_b)),
 * K(x) = (27+18x+12x^2+8x^3)/(27+18x+12x^2+8x^3+16x^4); t_b < 1e-12 is
 * replaced by 1.  r_dev, w_dev: [nband][n] complex128 (may alias);
 * tkin_dev: [nband] doubles. */
rsdft_status rsdft_precondition_tpa(rsdft_ctx *ctx, const void *r_dev, void *w_dev,
                                    const double *tkin_dev, int nband, void *stream);

/* ---------------------------------------------------------------------------
 * Subspace building blocks of the LOBPCG iteration (SCF tasks (2)-(3)).
 *
 * Gram matrix G[i][j] = <a_i|b_j> = dV sum_r conj(a_i(r)) b_j(r).
 * a_dev: [na][n], b_dev: [nb][n], g_dev: [na][nb] row-major, complex128.
 */
rsdft_status rsdft_gram(rsdft_ctx *ctx, const void *a_dev, int na, const void *b_dev, int nb,
                        void *g_dev, void *stream);

/* Gram matrix without any device allocation, for callers that cannot call
 * cudaMalloc: for example a time-stepping driver (RS-TDDFT, Ehrenfest MD)
 * that reserves all device memory before its loop and must not allocate or
 * free inside it, because each allocation synchronises the device and
 * fragments its fixed pool.  The paper has no counterpart; it is an extra
 * entry point of this library.  Needs no context.
 *   g[i][j] = scale * sum_{r<n} conj(a_i(r)) b_j(r); a_dev: [na][n],
 *   b_dev: [nb][n], g_dev: [na][nb] row-major, complex128, caller-owned
 *   device memory.
 * The split-K partial sums go to one fixed device array of 2^21 complex128
 * entries (32 MiB) inside the library, held by every GPU that loads it until
 * the process exits; na * nb above 2^21 is rejected with RSDFT_E_INVALID.
 * The first call on a device looks up that array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  All calls share the array: calls that overlap on the GPU (other
 * streams, other host threads on the same device) race and give wrong results.
 * No earlier contents are read (every entry used is written first).  Errors:
 * rsdft_last_error(NULL). */
rsdft_status rsdft_gram_static(const void *a_dev, int na, const void *b_dev, int nb, long long n,
                               double scale, void *g_dev, void *stream);

/* Gram matrix of complex64 blocks on the tensor cores (the mixed form):
 * G[i][j] = dV sum_r conj(a_i(r)) b_j(r) with each FP32 value split into
 * bf16 hi + lo and the products hi*hi + hi*lo + lo*hi accumulated in FP32 on
 * tcgen05 (TMEM), FP32 partials over K blocks summed in FP64 (SCF task (2),
 * mixed precision).  a_dev: [na][n], b_dev: [nb][n] complex64; g_dev: [na][nb]
 * complex128.  Relative error about 1e-5 of max |G|. */
rsdft_status rsdft_gram_bf16x3(rsdft_ctx *ctx, const void *a_dev, int na, const void *b_dev, int nb,
                               void *g_dev, void *stream);

/* The Hermitian pair of the LOBPCG Rayleigh-Ritz step on the tensor cores:
 * G_S = dV Y^H Y and G_H = dV Y^H (HY) as one split-BF16 GEMM of Y against
 * [Y; HY], computing only the tiles that hold entries on or above the
 * diagonal; entries below it are the conjugates of their mirrors (exactly
 * Hermitian).  y_dev, hy_dev: [k][n] complex64; gs_dev, gh_dev: [k][k]
 * complex128, row-major. */
rsdft_status rsdft_gram_sh_bf16x3(rsdft_ctx *ctx, const void *y_dev, const void *hy_dev, int k, void *gs_dev,
                                  void *gh_dev, void *stream);

/* Ritz rotation of a complex64 block on the tensor cores (the mixed form's
 * rotation, SCF task (2)): with Y = y_dev [k][n] complex64 and C = c_dev [k][m]
 * complex128 row-major (rows 0..m-1 multiply the X part, m..k-1 the [W P] part),
 *   out1[b] = sum_{i >= m} C[i][b] Y[i]        (the new P)
 *   out0[b] = sum_{i <  m} C[i][b] Y[i] + out1[b]   (the new X)
 * as real GEMMs over the interleaved grid index with Y and C split into bf16
 * hi + lo and the products hi*hi + hi*lo + lo*hi accumulated in FP32 in TMEM.
 * out0_dev, out1_dev: [m][n] complex64, caller-owned, must not alias y_dev.
 * Shape limits: m >= 1 and k > m, else RSDFT_E_INVALID (more than 240 bands
 * are rotated in balanced groups of at most 240, one launch each).  Relative
 * error about 1e-5 of the largest |C[i][b] Y[i](r)| term. */
rsdft_status rsdft_rotate_bf16x3(rsdft_ctx *ctx, const void *y_dev, int k, const void *c_dev, int m,
                                 void *out0_dev, void *out1_dev, void *stream);

/* Rotation out[b] = sum_i c[i][b] y[i] (+ base[b] when base_dev != NULL;
 * base may alias out).  y_dev: [k][n]; c_dev: [k][m] row-major;
 * out_dev, base_dev: [m][n]; complex128.  sign = +1 adds, -1 subtracts the sum. */
rsdft_status rsdft_rotate(rsdft_ctx *ctx, const void *y_dev, int k, const void *c_dev, int m,
                          const void *base_dev, int sign, void *out_dev, void *stream);

/* Rayleigh-Ritz of Eq. 1 on a k x k Hermitian pair (row-major complex128 on
 * the device; inputs are not modified): G_S = L L^H (columns whose pivot
 * falls to pivot_tol * max diag are dropped), K = L^-1 G_H L^-H by two
 * triangular solves, K Z = Z Lambda for the lowest nkeep, C = L^-H Z.
 * lam_host: [nkeep] ascending; c_dev: [k][nkeep] (zero rows for dropped
 * columns); *ndropped_host: columns dropped.  RSDFT_E_NOT_SPD if fewer than
 * nkeep columns are independent. */
rsdft_status rsdft_rayleigh_ritz(rsdft_ctx *ctx, const void *gh_dev, const void *gs_dev, int k,
                                 int nkeep, double pivot_tol, double *lam_host, void *c_dev,
                                 int *ndropped_host, void *stream);

/* Subspace Hermitian eigensolve alone: the lowest nkeep eigenpairs of a k x k
 * Hermitian matrix (row-major complex128, device, not modified).
 * lam_host: [nkeep]; z_dev: [k][nkeep] orthonormal columns. */
rsdft_status rsdft_eigh(rsdft_ctx *ctx, const void *a_dev, int k, int nkeep, double *lam_host,
                        void *z_dev, void *stream);

/* Arithmetic of the subspace solve inside rsdft_eigh and rsdft_rayleigh_ritz
 * for this context: RSDFT_DENSE_FP64 (default; AUTO means the same here) or
 * RSDFT_DENSE_DF (as rsdft_lobpcg_opts.dense, the pivot_tol argument deciding
 * the Cholesky and the triangular solves).
 * RSDFT_E_INVALID for another value. */
rsdft_status rsdft_set_dense(rsdft_ctx *ctx, int mode);

/* ---------------------------------------------------------------------------
 * LOBPCG for the lowest nband eigenpairs of H (the paper's eigensolver,
 * Knyazev's block method with the Rayleigh-Ritz of Eq. 1).  RSDFT_FP64 keeps
 * everything in FP64.  RSDFT_MIXED runs H psi, the FFTs, the Gram and rotation
 * GEMMs on FP32 orbitals (FP32 products, FP64 sums across GEMM blocks) while the
 * residual norms, Cholesky, triangular solves and eigensolve stay FP64, and
 * finishes with FP64 iterations to tol.
 * x_dev: in/out [nband][n] complex128 (initial guess in, Ritz vectors out,
 * orthonormal).  eig_host, resnorm_host: [nband].
 */
typedef struct {
    int maxit;             /* iterations cap (>= 0)                                */
    double tol;            /* stop when max residual over the first nconv <= tol   */
    int nconv;             /* bands checked for tol; <= 0 means nband              */
    int precond;           /* rsdft_precond                                        */
    int precision;         /* rsdft_precision                                      */
    double lock_tol;       /* soft-lock bands with residual <= lock_tol (1e-10)    */
    double pivot_tol;      /* relative Cholesky pivot floor for G_S (1e-8; the FP32
                              data path of RSDFT_MIXED uses at least 1e-3 and soft-
                              locks bands at residual <= 1e-6)                    */
    double switch_tol;     /* RSDFT_MIXED: FP32 data path until the max residual
                              is <= max(tol, switch_tol) (3e-5) or stagnates (3
                              iterations gaining < 10%), then FP64 to tol; 0 runs
                              FP32 iterations to maxit                            */
    int tensor_cores;      /* RSDFT_MIXED: 0 runs the FP32 phase's Gram matrices
                              and Ritz rotations on FP32 CUDA cores; 1 forms the
                              Gram matrices with split-BF16 tcgen05 GEMMs; 2 does
                              the Ritz rotations that way too (default 0)         */
    int learned_iters;     /* RSDFT_PRECOND_LEARNED: add the network correction in
                              the first learned_iters iterations only, TPA alone
                              after them; 0 = in every iteration (default 0)      */
    int refine;            /* RSDFT_MIXED, iterations after the FP32 phase:
                              RSDFT_REFINE_FP32_CORRECTIONS (default) keeps X and
                              HX in FP64 (residuals, residual norms, T_b, the X-X
                              blocks of G_S and G_H, the X part of the rotation)
                              and forms W = TPA(R), H W, P, H P and the Gram blocks
                              that involve them on the FP32 path (recomputing H P
                              each iteration) down to a residual of 1e-7 (30
                              iterations at most); FP64 iterations finish tighter
                              tolerances, and take over
                              when it stalls (three iterations each gaining less
                              than 10%, or a residual ten times its best);
                              RSDFT_REFINE_FP64 runs them all in FP64.  Both stop
                              on the FP64 residual norms.                         */
    int dense;             /* arithmetic of the subspace solve's sequential parts:
                              RSDFT_DENSE_AUTO (default) = double-float in
                              RSDFT_MIXED, FP64 in RSDFT_FP64; RSDFT_DENSE_FP64;
                              RSDFT_DENSE_DF = double-float (FP32 pairs, ~2^-46
                              relative per operation) for the Householder
                              tridiagonalisation (one 16-CTA thread-block
                              cluster with the matrix in its shared memory, for
                              subspaces up to 448; FP64 above), the Sturm
                              bisection and inverse iteration, and, where the
                              Cholesky pivot floor is >= 1e-6 (the FP32 phase and
                              the refinement), the Cholesky's diagonal blocks
                              and the three triangular solves.  Results are
                              returned in FP64 in every case.                     */
} rsdft_lobpcg_opts;

enum { RSDFT_REFINE_FP64 = 0, RSDFT_REFINE_FP32_CORRECTIONS = 1 };
enum { RSDFT_DENSE_AUTO = 0, RSDFT_DENSE_FP64 = 1, RSDFT_DENSE_DF = 2 };

typedef struct {
    int iterations;        /* full iterations done (both phases)                   */
    int iterations_mixed;  /* of which in the FP32 data path (RSDFT_MIXED)         */
    int converged;         /* 1 if the tolerance test passed                       */
    int dropped;           /* basis columns dropped by the Cholesky, summed        */
    int coop_fallbacks;    /* subspace tridiagonalisations that ran as one launch
                              per Householder step because the cooperative launch
                              was refused (same result up to rounding)           */
    int coop_last_error;   /* cudaError_t of the last refused cooperative launch   */
    double ms_hpsi, ms_precond, ms_gram, ms_dense, ms_rotate, ms_other;
} rsdft_lobpcg_stats;

void rsdft_lobpcg_default_opts(rsdft_lobpcg_opts *opts);

rsdft_status rsdft_lobpcg(rsdft_ctx *ctx, void *x_dev, int nband, const rsdft_lobpcg_opts *opts,
                          double *eig_host, double *resnorm_host, rsdft_lobpcg_stats *stats,
                          void *stream);

/* Batched LOBPCG (the batched form of the solve: many independent cells of
 * uneven grid and band counts on one GPU).  ncell cells, each with its own
 * context ctxs[c] and orbital block x_dev[c] ([nband[c]][n_c] complex128,
 * device, in/out), solved with options opts[c] (one entry per cell, e.g. a
 * different nconv per cell; NULL = defaults for all).  Up to max_concurrent cells
 * (<= 0: min(ncell, 8)) are in flight at a time, each on its own stream driven
 * by its own host thread, so that one cell's latency-bound subspace eigensolve
 * overlaps the FFT and GEMM work of the others; the cooperative
 * tridiagonalisations of different cells never run at the same time.  The call
 * first waits for all work already issued on the device (the cells' streams do
 * not order against the caller's streams) and returns after every cell's work
 * has completed.  Per cell
 * the results equal those of rsdft_lobpcg with the same options (same kernels,
 * same launch shapes).  eig_host[c], res_host[c]: [nband[c]] host outputs (the
 * arrays may be NULL); stats: ncell entries or NULL.  Returns the first failing
 * cell's status and its index in *failed_cell (-1 when all succeed; may be
 * NULL); the other cells still complete.  Contexts must not be shared between
 * cells or used by other threads during the call. */
rsdft_status rsdft_lobpcg_batched(rsdft_ctx *const *ctxs, int ncell, void *const *x_dev, const int *nband,
                                  const rsdft_lobpcg_opts *opts /* [ncell] */, double *const *eig_host,
                                  double *const *res_host, rsdft_lobpcg_stats *stats, int max_concurrent,
                                  int *failed_cell);

/* ---------------------------------------------------------------------------
 * Real Gamma-point form (the paper's real-symmetric case: its eigensolver
 * benchmark for real-symmetric matrices, Fig. 3a, beside the Hermitian Fig. 3b).
 * At Gamma, with the context's real V_loc and real projectors, H is real
 * symmetric and the orbitals are real.  Orbital blocks here are float64
 * [nband][n] real arrays on the device (x fastest, as the complex blocks).
 * Internally two real bands share one complex row, so each complex H psi
 * transform carries two bands, and the Gram and rotation kernels form real
 * products only (a quarter of the complex form's arithmetic).  The subspace
 * problem of Eq. 1 is real symmetric; it runs through the Hermitian dense core
 * with zero imaginary parts, which stay exactly zero.  Same ownership, stream
 * and error rules as the complex calls; the workspace of the context is reused
 * (these calls and the complex ones may alternate on one context).
 * ------------------------------------------------------------------------- */

/* hx = H x for nband real orbitals (x, hx: float64 [nband][n], device; they
 * must not overlap).  nband == 0 is a no-op. */
rsdft_status rsdft_apply_h_real(rsdft_ctx *ctx, const void *x_dev, void *hx_dev, int nband, void *stream);

/* g[i][j] = sum_r a_i(r) b_j(r) dV (float64 [na][nb], device) over real rows
 * a [na][n] and b [nb][n].  When a_dev == b_dev and na == nb, G is formed as a
 * symmetric matrix (tiles on and above the diagonal, the rest mirrored). */
rsdft_status rsdft_gram_real(rsdft_ctx *ctx, const void *a_dev, int na, const void *b_dev, int nb, void *g_dev,
                             void *stream);

/* out[b] = base[b] + sign * sum_{i<k} c[i][b] y_i for b < m: y float64 [k][n],
 * c float64 [k][m], base float64 [m][n] or NULL (then 0), sign +-1, out float64
 * [m][n] (may equal base).  All device. */
rsdft_status rsdft_rotate_real(rsdft_ctx *ctx, const void *y_dev, int k, const void *c_dev, int m,
                               const void *base_dev, int sign, void *out_dev, void *stream);

/* LOBPCG of the real form: x_dev float64 [nband][n] (device, in/out: start
 * block in, Ritz vectors out, <x_i|x_j> = delta_ij).  Options as rsdft_lobpcg
 * with precision RSDFT_FP64 only and precond RSDFT_PRECOND_TPA or
 * RSDFT_PRECOND_NONE (RSDFT_E_INVALID otherwise); nconv, tol, maxit,
 * lock_tol, pivot_tol and dense keep their meaning.  The stats' per-phase
 * times are not filled.  Returns RSDFT_E_NOT_CONVERGED when tol > 0 was not
 * met within maxit (the block is still written back). */
rsdft_status rsdft_lobpcg_real(rsdft_ctx *ctx, void *x_dev, int nband, const rsdft_lobpcg_opts *opts,
                               double *eig_host, double *resnorm_host, rsdft_lobpcg_stats *stats, void *stream);

/* ---------------------------------------------------------------------------
 * SCF step: V_eff = V_loc + V_H[rho_in] + v_xc[rho_in] (FFT Hartree, LDA
 * Slater + Perdew-Zunger 1981), LOBPCG (converged on the first step, k_lobpcg
 * iterations afterwards), occupations (aufbau, or Fermi-Dirac at kT > 0),
 * rho_out = sum f |psi|^2, energies, Anderson mixing of rho_in.  The density
 * and the mixing history live in the context (rsdft_scf_init resets them to
 * the uniform density N_e / volume).
 */
typedef struct {
    double n_electrons;    /* spin-degenerate electron count (> 0)                 */
    double kT;             /* Ha; 0 = aufbau                                       */
    double beta;           /* Anderson weight (0.3)                                */
    int depth;             /* Anderson history depth (4)                           */
    int k_lobpcg;          /* LOBPCG iterations per step after the first (3)       */
    int first_maxit;       /* iteration cap of the first, converged, solve (200)   */
    double tol;            /* residual tolerance of the first solve (1e-6)         */
    int precond;           /* rsdft_precond                                        */
    int precision;         /* rsdft_precision of the LOBPCG: RSDFT_MIXED runs the
                              first solve in the mixed form (FP32 data path to the
                              default switch_tol, then the default refinement to
                              tol) and the later steps' k_lobpcg iterations on the
                              FP32 data path                                      */
    int tensor_cores;      /* as rsdft_lobpcg_opts.tensor_cores                    */
    double later_tol;      /* 0 (default): the steps after the first run k_lobpcg
                              LOBPCG iterations; > 0: they also converge to
                              later_tol (at most first_maxit iterations; the mixed
                              form as in the first solve), so that each step is a
                              function of rho_in alone                            */
    int xc;                /* RSDFT_XC_LDA (default) or RSDFT_XC_PBE               */
} rsdft_scf_opts;

enum { RSDFT_XC_LDA = 0, RSDFT_XC_PBE = 1 };

typedef struct {
    double e_tot;          /* sum f eps - E_H - int v_xc rho + E_xc (at rho_in)    */
    double free_energy;    /* e_tot - kT S                                         */
    double e_band, e_h, e_xc, e_vxc, mu, entropy;
    double drho;           /* ||rho_out - rho_in|| sqrt(dV)                        */
    int lobpcg_iterations;
    int lobpcg_iterations_mixed;  /* of which on the FP32 data path (RSDFT_MIXED)  */
    int step;              /* index of the step just done (0-based)                */
} rsdft_scf_out;

void rsdft_scf_default_opts(rsdft_scf_opts *opts);
rsdft_status rsdft_scf_init(rsdft_ctx *ctx, int nband, const rsdft_scf_opts *opts, void *stream);
/* eig_host, occ_host: [nband] outputs (may be NULL). */
rsdft_status rsdft_scf_step(rsdft_ctx *ctx, void *x_dev, int nband, const rsdft_scf_opts *opts,
                            rsdft_scf_out *out, double *eig_host, double *occ_host, void *stream);

/* The same SCF step on the real orbitals of the Gamma-point form (x_dev: float64
 * [nband][n], device, in/out): LOBPCG by rsdft_lobpcg_real, rho = sum_b f_b x_b^2.
 * opts->precision must be RSDFT_FP64 (RSDFT_E_INVALID otherwise); tensor_cores
 * is ignored; precond RSDFT_PRECOND_TPA or RSDFT_PRECOND_NONE.  Shares the SCF
 * state of rsdft_scf_init with the complex step (one kind of step per run). */
rsdft_status rsdft_scf_step_real(rsdft_ctx *ctx, void *x_dev, int nband, const rsdft_scf_opts *opts,
                                 rsdft_scf_out *out, double *eig_host, double *occ_host, void *stream);

/* SCF field pieces, each on [n] doubles on the device:
 * rho = sum_b f_b |x_b|^2 (x_dev [nband][n] complex128, f_dev [nband]);
 * V_H by FFT Poisson (G = 0 term removed);
 * LDA eps_xc and v_xc (rho < 1e-12 gives 0). */
rsdft_status rsdft_density(rsdft_ctx *ctx, const void *x_dev, const double *f_dev, int nband,
                           double *rho_dev, void *stream);
rsdft_status rsdft_hartree(rsdft_ctx *ctx, const double *rho_dev, double *vh_dev, void *stream);
rsdft_status rsdft_lda(rsdft_ctx *ctx, const double *rho_dev, double *eps_dev, double *vxc_dev,
                       void *stream);
/* GGA exchange-correlation of Perdew, Burke and Ernzerhof (PBE, the paper's
 * functional), spin-unpolarised, with PW92 correlation of the uniform gas:
 * eps_dev = e / rho and vxc_dev = de/drho - div(2 de/dsigma grad rho) for
 * e(rho, sigma = |grad rho|^2); gradients and the divergence by FFT (i G_a,
 * the Nyquist plane of an even axis set to zero); points with rho < 1e-12
 * contribute nothing.  [n] doubles on the device. */
rsdft_status rsdft_xc_pbe(rsdft_ctx *ctx, const double *rho_dev, double *eps_dev, double *vxc_dev, void *stream);
/* Occupations on the device: eig_dev [nband] ascending -> f_dev [nband];
 * mu_host, entropy_host may be NULL. */
rsdft_status rsdft_occupations(rsdft_ctx *ctx, const double *eig_dev, int nband,
                               double n_electrons, double kT, double *f_dev, double *mu_host,
                               double *entropy_host, void *stream);
/* Density rho_in as held by the SCF state (device, [n]); NULL before init. */
const double *rsdft_scf_density(const rsdft_ctx *ctx);

/* ---------------------------------------------------------------------------
 * Real-time propagation (RS-TDDFT: i d psi/dt = H psi, the application the
 * paper's real-space code serves, in its introduction), V held fixed:
 * nsteps steps of psi <- sum_{j=0}^{order} (-i dt H)^j / j! psi, the truncated
 * Taylor series of exp(-i H dt), each term one batched H psi (FP64).
 * psi_dev: [nband][n] complex128, device, in/out.  1 <= order <= 16,
 * nsteps >= 0, dt finite (Ha^-1 time units), else RSDFT_E_INVALID.  Uses the
 * context's workspace (no allocation after the first call for nband bands).
 * Asynchronous on the stream.
 */
rsdft_status rsdft_propagate(rsdft_ctx *ctx, void *psi_dev, int nband, double dt, int nsteps, int order,
                             void *stream);

/* ---------------------------------------------------------------------------
 * Per-kernel timing (the per-component breakdown of Fig. 1, finer grained).
 * When enabled, each launch of the hot kernels below is bracketed by CUDA
 * events on its stream and its algorithmic work is recorded: flops counted
 * from the operation's definition (complex MAC = 8, FFT = 5 N log2 N per
 * transform) and bytes = the minimum HBM traffic of the operation (each
 * operand read once, each result written once).  Reading synchronises the
 * events.  Enabling resets the counters.
 */
typedef enum {
    RSDFT_K_GRAM = 0,        /* Gram partial tiles (split-K)                    */
    RSDFT_K_ROTATE = 1,      /* Ritz rotation / block update                    */
    RSDFT_K_FFT_XY_FWD = 2,  /* xy-plane forward FFT pass                       */
    RSDFT_K_FFT_Z = 3,       /* z pass: forward, per-G factor, inverse          */
    RSDFT_K_FFT_XY_INV = 4,  /* xy-plane inverse pass (+ V psi + projectors)    */
    RSDFT_K_PROJECT = 5,     /* projector gather <beta|psi>                     */
    RSDFT_K_DENSE = 6,       /* the whole Rayleigh-Ritz solve of Eq. 1 (a group:
                                the ids below time its parts)                   */
    RSDFT_K_GRAM_TC = 7,     /* tensor-core split-BF16 Gram (tcgen05)           */
    RSDFT_K_ROTATE_TC = 8,   /* tensor-core split-BF16 Ritz rotation (tcgen05)  */
    RSDFT_K_CHOL = 9,        /* Cholesky of G_S with dropping: (4/3) k^3 flop   */
    RSDFT_K_TRSM = 10,       /* the triangular solves of Eq. 1 and C = L^-H Z:
                                4 k^2 per right-hand side                       */
    RSDFT_K_TRIDIAG = 11,    /* Householder tridiagonalisation: (16/3) k^3      */
    RSDFT_K_TRIEIG = 12,     /* bisection + inverse iteration on the tridiagonal
                                matrix: k (3 x 52 + 20) per wanted eigenpair    */
    RSDFT_K_BACKTRANSFORM = 13, /* Q Z in compact WY blocks: 8 k^2 per vector   */
    RSDFT_K_COUNT = 14
} rsdft_kernel_id;

rsdft_status rsdft_profile_enable(rsdft_ctx *ctx, int on);
/* Totals since enabling for one kernel id: summed event time (ms), launches,
 * algorithmic flops and bytes.  Any pointer may be NULL. */
rsdft_status rsdft_profile_read(rsdft_ctx *ctx, int kernel_id, double *ms, long long *launches,
                                double *flops, double *bytes);
/* Kernels launched on ctx since creation (every kernel, profiled or not). */
long long rsdft_launch_count(const rsdft_ctx *ctx);

/* Autotuner (off by default).  When on, the first call of each shape of the
 * Gram GEMMs (tile edge 16 P, P = 2, 3, 4), the Ritz rotations (band tile
 * 16 PB, PB = 1..4; not the in-place W update) and the tensor-core Gram (split
 * count: the wave rule's, half, double) runs every candidate once, timed with
 * CUDA events on the call's stream (the call synchronises), and later calls of
 * that shape on this context use the fastest.  Candidates differ only in the
 * summation order, so results agree to rounding.  on = 0 switches it off and
 * forgets the choices. */
rsdft_status rsdft_set_autotune(rsdft_ctx *ctx, int on);

/* ---------------------------------------------------------------------------
 * Learned preconditioner (the learned form of the LOBPCG preconditioner; the
 * paper's LOBPCG uses a kinetic-energy preconditioner, here Teter-Payne-Allan).
 *
 * w_b = TPA(r_b) + s_b (NN(Re r_b / s_b) + i NN(Im r_b / s_b)),
 * s_b = sqrt(sum_p |r_b(p)|^2 / n) (no correction where s_b = 0).
 * NN maps a real plane u to a real plane: input channels (u, u vhat) with
 * vhat = (V - mean V) / std V of the context's current potential, then four
 * periodic 3x3x3 convolutions without biases, channels
 * 2 -> RSDFT_NN_HIDDEN -> RSDFT_NN_HIDDEN -> RSDFT_NN_HIDDEN -> 1, tanh after
 * the first three.  A convolution is out[co](p) = sum_ci sum_d
 * w[tap(d)][ci][co] in[ci](p + d) over d in {-1,0,1}^3 with periodic wrap,
 * tap(d) = (dz+1)*9 + (dy+1)*3 + (dx+1).  Weights: float32, the four layers one
 * after the other, each [27][cin][cout]; RSDFT_NN_WEIGHTS in all.  The network
 * computes in FP32.
 */
#define RSDFT_NN_HIDDEN 8
#define RSDFT_NN_WEIGHTS (27 * (2 * RSDFT_NN_HIDDEN + 2 * RSDFT_NN_HIDDEN * RSDFT_NN_HIDDEN + RSDFT_NN_HIDDEN))

/* Copy the network weights in (w_host: count = RSDFT_NN_WEIGHTS finite floats,
 * else RSDFT_E_INVALID) or out (RSDFT_E_INVALID before any were set).
 * Synchronous. */
rsdft_status rsdft_set_precond_weights(rsdft_ctx *ctx, const float *w_host, long long count);
rsdft_status rsdft_get_precond_weights(rsdft_ctx *ctx, float *w_host, long long count);

/* w = base + the network correction of r (formula above), per band.
 * r_dev, base_dev, w_dev: [nband][n] complex128; w may alias base, not r. */
rsdft_status rsdft_precond_learned(rsdft_ctx *ctx, const void *r_dev, const void *base_dev, void *w_dev,
                                   int nband, void *stream);

/* Training samples from a block of normalised approximate orbitals x_dev
 * ([nband][n] complex128, e.g. LOBPCG iterates): per band e = <x|H|x>,
 * r = H x - e x, s = sqrt(sum |r|^2 / n), base = TPA(r) (T_b = <x|T|x>), and
 * t perpendicular to the whole block solving Q (H - e) Q t = -Q r, Q = I - X X^H
 * with X all nband orbitals (orthonormal), by MINRES (Paige-Saunders) to
 * relative residual rtol or maxit iterations (FP64);
 * c = sign(Re<t|base>) ||base|| / ||t|| (t rescaled to the TPA norm, pointing
 * along it: LOBPCG uses only the direction).  Writes float planes
 * [2 nband][n] (real parts of every band, then imaginary parts): u = r / s,
 * b = base / s, y = c t / s.
 * iters_host (optional, [nband]): MINRES iterations per band.  Allocates and
 * frees its own scratch (about 10 nband n complex128); synchronises. */
rsdft_status rsdft_precond_samples(rsdft_ctx *ctx, const void *x_dev, int nband, double rtol, int maxit,
                                   float *u_dev, float *b_dev, float *y_dev, int *iters_host, void *stream);

/* Loss over all nsample planes (u, b, y: [nsample][n] float, device), the mean
 * over planes of 1 - cos^2(p, y) = 1 - <p, y>^2 / (<p, p> <y, y>) with
 * p = b + NN(u) (scale- and sign-free: LOBPCG uses only the span of a
 * preconditioned residual), and its gradient in the weights (grad_host:
 * RSDFT_NN_WEIGHTS floats), with the context's current weights and potential.
 * Synchronises. */
rsdft_status rsdft_precond_loss_grad(rsdft_ctx *ctx, const float *u_dev, const float *b_dev, const float *y_dev,
                                     int nsample, float *loss_host, float *grad_host, void *stream);

/* Train the context's weights (set initial ones first) on nsample float planes
 * u, b, y ([nsample][n], device) from rsdft_precond_samples of this context's
 * potential: Adam (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr, fresh
 * moments each call) for `steps` steps on mini-batches of `batch` samples taken
 * cyclically (batch k = samples (k batch + j) mod nsample), minimising the
 * loss of rsdft_precond_loss_grad.  loss_host (optional, [steps]): each
 * step's batch loss before its update.  Synchronises. */
rsdft_status rsdft_precond_train(rsdft_ctx *ctx, const float *u_dev, const float *b_dev, const float *y_dev,
                                 long long nsample, int steps, int batch, float lr, float *loss_host,
                                 void *stream);

#ifdef __cplusplus
}
#endif

#endif /* RSDFT_H */
