"""GPU parity of the whole LOBPCG iteration and of the SCF step against the
FP64 oracle; full-size invariants in the launch configuration the bench uses."""
import numpy as np
import pytest

from oracle.grid import Grid
from oracle.hamiltonian import inner
from oracle.lobpcg import lobpcg as oracle_lobpcg
from oracle.scf import scf_init, scf_step
from tests.gpu_common import R, dev, host, need_gpu, pair, subspace_distance, torch
from tests.oracle_refs import hamiltonian_dense
from workloads import diamond8_24, diamond64_64, small_cell

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _gap_prefix(eig_all, m, gap=1e-4):
    """Largest prefix length <= m (< len(eig_all)) ending at a gap >= gap."""
    for p in range(min(m, len(eig_all) - 1), 0, -1):
        if eig_all[p] - eig_all[p - 1] >= gap:
            return p
    return 0


def test_lobpcg_converged_matches_brute_force_12cubed():
    wl = small_cell(N=(12, 12, 12), L=(6.0, 6.0, 6.0), natom=2, nband=8)
    ctx, ham, v = pair(wl)
    x = dev(wl.x0())
    eig, res, stats, st = ctx.lobpcg(x, ctx.lobpcg_opts(maxit=300, tol=1e-8))
    assert st == R.OK and stats.converged
    Hd = hamiltonian_dense(wl.N, wl.L, v, ham.proj.B.toarray(), ham.proj.E)
    ref = np.linalg.eigvalsh(Hd)
    assert np.max(np.abs(eig - ref[:8])) < 1e-9
    X = host(x)
    assert np.allclose(inner(X, X, ham.dV), np.eye(8), atol=1e-12)
    r = ham.apply(X) - eig[:, None] * X
    assert np.allclose(np.sqrt(np.sum(np.abs(r) ** 2, 1) * ham.dV), res, atol=1e-11)
    assert np.max(res) <= 1e-8


def test_lobpcg_diamond8_24_forty_iterations_matches_oracle():
    """The fixed-potential workload as specified: 16 bands, 40 iterations.  The
    16th band is not converged after 40 iterations (its gap to the 17th is
    9e-4 Ha), so this compares trajectories: eigenvalues to the 1e-9 Ha bar,
    residual norms, and the spanned subspace to 1e-6."""
    wl = diamond8_24()
    ctx, ham, _ = pair(wl)
    x0 = wl.x0()
    x = dev(x0)
    eig, res, stats, st = ctx.lobpcg(x, ctx.lobpcg_opts(maxit=40, tol=0.0))
    o = oracle_lobpcg(ham, x0, maxit=40, tol=0.0)
    assert stats.iterations == o.iterations
    assert np.max(np.abs(eig - o.eig)) < 1e-9
    assert np.max(np.abs(res - o.resnorm)) < 1e-7
    X = host(x)
    assert subspace_distance(X, o.X, ham.dV) < 1e-6
    assert np.allclose(inner(X, X, ham.dV), np.eye(16), atol=1e-12)


def test_lobpcg_diamond8_24_converged_occupied_subspace():
    """Converged run with 24 bands: the 16 occupied bands' eigenvalues within
    1e-9 Ha and their subspace within a projector distance of 1e-7."""
    wl = diamond8_24()
    ctx, ham, _ = pair(wl)
    x0 = wl.x0(24)
    x = dev(x0)
    eig, res, stats, st = ctx.lobpcg(x, ctx.lobpcg_opts(maxit=200, tol=1e-9))
    o = oracle_lobpcg(ham, x0, maxit=200, tol=1e-9)
    assert stats.converged and o.converged
    assert np.max(np.abs(eig - o.eig)) < 1e-9
    p = _gap_prefix(o.eig, 16)
    assert p == 16
    X = host(x)
    assert subspace_distance(X[:p], o.X[:p], ham.dV) < 1e-7


def test_lobpcg_without_preconditioner_and_with_locking():
    wl = small_cell(N=(10, 12, 8), L=(5.0, 6.0, 4.5), natom=2, nband=5, rcut=2.0)
    ctx, ham, _ = pair(wl)
    x0 = wl.x0()
    x = dev(x0)
    eig, res, stats, st = ctx.lobpcg(x, ctx.lobpcg_opts(maxit=400, tol=1e-9, precond=R.PRECOND_NONE))
    o = oracle_lobpcg(ham, x0, maxit=400, tol=1e-9, precond="none")
    assert stats.converged and o.converged
    assert np.max(np.abs(eig - o.eig)) < 1e-9


def test_lobpcg_rejects_nan_input():
    wl = small_cell(N=(12, 12, 12), L=(6.0, 6.0, 6.0), natom=2, nband=4)
    ctx, ham, _ = pair(wl)
    x0 = wl.x0()
    x0[1, 17] = np.nan
    with pytest.raises(R.RsdftError) as e:
        ctx.lobpcg(dev(x0), ctx.lobpcg_opts(maxit=5, tol=0.0))
    assert e.value.status in (R.E_NUMERIC, R.E_NOT_SPD)


def test_scf_steps_match_oracle_small_cell():
    wl = small_cell(N=(12, 12, 12), L=(6.0, 6.0, 6.0), natom=2, nband=6)
    ctx, ham, v_loc = pair(wl)
    n_el = 8.0
    x0 = wl.x0()
    opts = ctx.scf_opts(n_electrons=n_el, kT=0.0, beta=0.3, depth=4, k_lobpcg=3, first_maxit=200,
                        tol=1e-8)
    ctx.scf_init(6, opts)
    st = scf_init(ham.grid, n_el, x0, beta=0.3, depth=4)
    x = dev(x0)
    for step in range(8):
        out, eig, occ = ctx.scf_step(x, opts)
        o = scf_step(ham, v_loc, st, n_el, 0.0, k_lobpcg=3, first_maxit=200, tol=1e-8)
        assert abs(out.e_tot - o.e_tot) / wl.natom < 1e-8, step
        assert np.max(np.abs(eig - o.eig)) < 1e-9, step
        assert abs(out.drho - o.drho) < 1e-8, step
        assert np.array_equal(occ, o.f)
    rho = torch.empty(ham.grid.n, dtype=torch.float64, device="cuda")
    ctx.density(x, dev(occ), rho)
    assert abs(host(rho).sum() * ham.dV - n_el) < 1e-10


def test_scf_fermi_dirac_matches_oracle():
    wl = small_cell(N=(12, 12, 12), L=(6.0, 6.0, 6.0), natom=2, nband=8)
    ctx, ham, v_loc = pair(wl)
    n_el, kT = 9.0, 0.01
    x0 = wl.x0()
    opts = ctx.scf_opts(n_electrons=n_el, kT=kT, k_lobpcg=3, first_maxit=200, tol=1e-8)
    ctx.scf_init(8, opts)
    st = scf_init(ham.grid, n_el, x0)
    x = dev(x0)
    for step in range(4):
        out, eig, occ = ctx.scf_step(x, opts)
        o = scf_step(ham, v_loc, st, n_el, kT, k_lobpcg=3, first_maxit=200, tol=1e-8)
        assert abs(out.free_energy - o.free_energy) / wl.natom < 1e-8, step
        assert abs(out.mu - o.mu) < 1e-9 and np.allclose(occ, o.f, atol=1e-8)


def test_full_size_apply_h_sampled_against_oracle():
    """64^3, 144 bands (the SCF bench workload) in the bench's launch
    configuration; eight sampled bands checked against the oracle."""
    wl = diamond64_64()
    ctx, ham, _ = pair(wl)
    x0 = wl.x0()
    x = dev(x0)
    hx = torch.empty_like(x)
    ctx.apply_h(x, hx)
    idx = [0, 1, 37, 63, 64, 100, 142, 143]
    ref = ham.apply(x0[idx])
    got = host(hx)[idx]
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 1e-12


def test_full_size_scf_step_invariants():
    """One SCF step of the bench workload: orthonormal orbitals, electron count,
    residuals consistent with the returned pairs (checked on sampled bands)."""
    wl = diamond64_64()
    ctx, ham, _ = pair(wl)
    opts = ctx.scf_opts(n_electrons=wl.n_electrons, first_maxit=3, tol=0.0)
    ctx.scf_init(wl.nband, opts)
    x = dev(wl.x0())
    out, eig, occ = ctx.scf_step(x, opts)
    X = host(x)
    idx = [0, 5, 70, 127, 143]
    G = inner(X[idx], X[idx], ham.dV)
    assert np.allclose(G, np.eye(len(idx)), atol=1e-11)
    assert abs(occ.sum() - wl.n_electrons) < 1e-12
    assert np.all(np.diff(eig) >= -1e-12)
    assert np.isfinite(out.e_tot)
