"""The mixed form (FP32 orbitals for H psi, FFTs, Gram and rotation GEMMs; FP64
residual norms, Cholesky, triangular solves, eigensolve; FP64 refinement at
the end) against the FP64 oracle.  Intermediate FP32 results carry stated
tolerances derived from FP32 rounding; after the FP64 refinement the results
must meet the FP64 bars (1e-9 Ha per eigenvalue, 1e-7 subspace distance)."""
import numpy as np
import pytest

from oracle.lobpcg import lobpcg as oracle_lobpcg
from oracle.scf import scf_init, scf_step
from tests.gpu_common import PREFIX8, R, dev, host, need_gpu, pair, rel_err, subspace_distance, torch
from workloads import diamond8_24, draw_x0, small_cell

pytestmark = pytest.mark.gpu

# FP32 H psi: each of the ~log2(n) butterfly stages and the V/projector terms
# round at 2^-24 relative to the largest entries; 2e-6 of max|H psi| bounds it.
FP32_HPSI_TOL = 2e-6


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("case", [0, 1, 2])
def test_apply_h_fp32_matches_oracle(case):
    wl = [lambda: small_cell(N=(12, 10, 8), L=(6.0, 5.5, 5.0), natom=2, rcut=2.2),
          lambda: small_cell(N=(45, 45, 45), L=(9.0, 9.0, 9.0), natom=4, rcut=3.0),
          diamond8_24][case]()
    ctx, ham, _ = pair(wl)
    psi = draw_x0(case + 50, 5, ham.grid.n).astype(np.complex64)
    out = torch.empty((5, ham.grid.n), dtype=torch.complex64, device="cuda")
    ctx.apply_h(dev(psi), out, precision=R.MIXED)
    ref = ham.apply(psi.astype(np.complex128))
    assert rel_err(host(out).astype(np.complex128), ref) < FP32_HPSI_TOL


def test_mixed_lobpcg_meets_fp64_bars_after_refinement():
    wl = diamond8_24()
    ctx, ham, _ = pair(wl)
    x0 = wl.x0(24)
    x = dev(x0)
    eig, res, stats, st = ctx.lobpcg(x, ctx.lobpcg_opts(maxit=200, tol=1e-9, precision=R.MIXED))
    o = oracle_lobpcg(ham, x0, maxit=200, tol=1e-9)
    assert stats.converged and stats.iterations_mixed > 0
    assert stats.iterations > stats.iterations_mixed
    assert np.max(res) <= 1e-9
    assert np.max(np.abs(eig - o.eig)) < 1e-9
    assert subspace_distance(host(x)[:PREFIX8], o.X[:PREFIX8], ham.dV) < 1e-7


def test_mixed_iterations_alone_reach_fp32_level():
    """FP32 data path only (switch_tol = 0, no refinement): the error of the
    eigenvalues against the converged FP64 oracle is stated, not pinned to
    the FP64 bar; it must be at the FP32 level (below 1e-4 Ha)."""
    wl = diamond8_24()
    ctx, ham, _ = pair(wl)
    x0 = wl.x0(24)
    x = dev(x0)
    eig, res, stats, st = ctx.lobpcg(x, ctx.lobpcg_opts(maxit=60, tol=0.0, precision=R.MIXED,
                                                        switch_tol=0.0))
    o = oracle_lobpcg(ham, x0, maxit=200, tol=1e-9)
    assert stats.iterations_mixed == stats.iterations
    err = np.max(np.abs(eig[:16] - o.eig[:16]))
    print(f"FP32-path eigenvalue error after 60 iterations: {err:.2e} Ha")
    assert err < 1e-4


def test_mixed_scf_steps_track_fp64_oracle():
    """SCF with the mixed form: the first step refines to tol in FP64, later
    steps run their 3 LOBPCG iterations on the FP32 data path.  Energies stay
    within a stated 1e-5 Ha/atom of the FP64 oracle's SCF."""
    wl = small_cell(N=(12, 12, 12), L=(6.0, 6.0, 6.0), natom=2, nband=6)
    ctx, ham, v_loc = pair(wl)
    n_el = 8.0
    x0 = wl.x0()
    opts = ctx.scf_opts(n_electrons=n_el, k_lobpcg=3, first_maxit=200, tol=1e-8,
                        precision=R.MIXED)
    ctx.scf_init(6, opts)
    st = scf_init(ham.grid, n_el, x0)
    x = dev(x0)
    for step in range(6):
        out, eig, occ = ctx.scf_step(x, opts)
        o = scf_step(ham, v_loc, st, n_el, 0.0, k_lobpcg=3, first_maxit=200, tol=1e-8)
        assert abs(out.e_tot - o.e_tot) / wl.natom < 1e-5, step
        assert np.max(np.abs(eig - o.eig)) < 1e-4, step
