"""GPU parity of the real Gamma-point form (through the C ABI) against
oracle.gamma: H x on real blocks (two bands per complex transform, odd counts
included), the real Gram and rotation kernels, the reading that the Hermitian
dense core returns real coefficients for a real symmetric problem, and the real
LOBPCG (trajectory and converged) against the oracle and the complex form."""
import numpy as np
import pytest

from oracle.gamma import apply_h_real, gram_real, lobpcg_gamma
from oracle.linalg import rayleigh_ritz as oracle_rr
from tests.gpu_common import PREFIX8, R, dev, host, need_gpu, pair, rel_err, subspace_distance, torch
from workloads import diamond8_24, diamond64_64, draw_x0_real, small_cell

pytestmark = pytest.mark.gpu

CASES = [
    lambda: small_cell(N=(12, 10, 8), L=(6.0, 5.5, 5.0), natom=2, rcut=2.2),
    lambda: small_cell(N=(27, 25, 32), L=(6.0, 6.0, 7.0), natom=2, rcut=2.5),
    lambda: small_cell(N=(45, 45, 45), L=(9.0, 9.0, 9.0), natom=4, rcut=3.0),
    diamond8_24,
]


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _real(shape):
    return torch.empty(shape, dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("nb", [1, 5, 6])
def test_apply_h_real_matches_oracle(case, nb):
    wl = CASES[case]()
    ctx, ham, _ = pair(wl)
    x = draw_x0_real(case + 20, nb, ham.grid.n)
    out = _real((nb, ham.grid.n))
    ctx.apply_h_real(dev(x), out)
    assert rel_err(host(out), apply_h_real(ham, x)) < 1e-12


def _ctx(N=(20, 18, 15), L=(5.0, 5.0, 5.0)):
    return R.Context(L, N, np.zeros(N[0] * N[1] * N[2]))


# tiles of 16 pair rows for most shapes; 32 for (64, 64) and 64 for (256, 256),
# where the computed work ties
@pytest.mark.parametrize("na,nb", [(1, 1), (7, 5), (64, 64), (67, 130), (129, 3), (256, 256)])
def test_gram_real_matches_oracle(na, nb):
    ctx = _ctx()
    a, b = draw_x0_real(1, na, ctx.n), draw_x0_real(2, nb, ctx.n)
    g = _real((na, nb))
    ctx.gram_real(dev(a), dev(b), g)
    assert rel_err(host(g), gram_real(a, b, ctx.dV)) < 1e-13


@pytest.mark.parametrize("na", [1, 2, 33, 64, 65, 131, 260])
def test_gram_real_symmetric_tiles(na):
    """Same buffer on both sides: only tiles on and above the diagonal are formed."""
    ctx = _ctx()
    a = draw_x0_real(3, na, ctx.n)
    ad = dev(a)
    g = _real((na, na))
    ctx.gram_real(ad, ad, g)
    G = host(g)
    assert rel_err(G, gram_real(a, a, ctx.dV)) < 1e-13
    assert np.array_equal(G, G.T)


# output tiles of 16 pair rows (m = 1, 3, 19, 67) and of 32 (m = 60, 128)
@pytest.mark.parametrize("k,m,with_base", [(1, 1, False), (5, 3, True), (45, 19, True), (130, 67, False),
                                           (70, 60, True), (200, 128, False)])
def test_rotate_real_matches_oracle(k, m, with_base):
    ctx = _ctx()
    y = draw_x0_real(4, k, ctx.n)
    c = np.random.default_rng(5).standard_normal((k, m))
    base = draw_x0_real(6, m, ctx.n) if with_base else None
    out = _real((m, ctx.n))
    sign = -1 if with_base else 1
    ctx.rotate_real(dev(y), dev(c), out, base=dev(base) if with_base else None, sign=sign)
    ref = sign * (c.T @ y) + (base if with_base else 0.0)
    assert rel_err(host(out), ref) < 1e-13


@pytest.mark.parametrize("dense", [R.DENSE_FP64, R.DENSE_DF])
@pytest.mark.parametrize("k", [7, 60, 300])
def test_dense_core_keeps_real_symmetric_problems_real(dense, k):
    """The real form reads the real parts of C from the Hermitian dense core;
    for a real symmetric G_H, G_S its imaginary parts are exactly zero, and
    the pairs match the oracle's real Rayleigh-Ritz."""
    ctx = _ctx()
    ctx.set_dense(dense)
    rng = np.random.default_rng(k)
    a = rng.standard_normal((k, k))
    gh = a + a.T
    q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    gs = (q * rng.uniform(0.5, 2.0, k)) @ q.T
    gs = 0.5 * (gs + gs.T)
    nkeep = max(1, k // 3)
    c = torch.empty((k, nkeep), dtype=torch.complex128, device="cuda")
    lam, nd = ctx.rayleigh_ritz(dev(gh.astype(np.complex128)), dev(gs.astype(np.complex128)), nkeep, c,
                                pivot_tol=1e-8)
    C = host(c)
    assert np.all(C.imag == 0.0)
    lam_o, _, nd_o = oracle_rr(gh, gs, nkeep, pivot_tol=1e-8)
    scale = max(1.0, np.max(np.abs(lam_o)))
    assert nd == nd_o == 0
    assert np.max(np.abs(lam - lam_o)) < (2e-11 if dense == R.DENSE_DF else 1e-11) * scale
    Cr = C.real
    assert np.allclose(Cr.T @ gs @ Cr, np.eye(nkeep), atol=1e-10)


@pytest.mark.parametrize("m", [16, 9])
def test_lobpcg_real_forty_iterations_matches_oracle(m):
    """diamond8_24 from a real start, 40 iterations: eigenvalues to the 1e-9 Ha
    bar, residual norms, the spanned subspace and orthonormality (9 bands: an
    odd count, so every block has a padded half row)."""
    wl = diamond8_24()
    ctx, ham, _ = pair(wl)
    x0 = wl.x0_real(m)
    x = dev(x0)
    eig, res, stats, st = ctx.lobpcg_real(x, ctx.lobpcg_opts(maxit=40, tol=0.0))
    o = lobpcg_gamma(ham, x0, maxit=40, tol=0.0)
    assert stats.iterations == o.iterations
    assert np.max(np.abs(eig - o.eig)) < 1e-9
    assert np.max(np.abs(res - o.resnorm)) < 1e-7
    X = host(x)
    assert subspace_distance(X, o.X, ham.dV) < 1e-6
    assert np.allclose(gram_real(X, X, ham.dV), np.eye(m), atol=1e-12)


def test_lobpcg_real_converged_equals_complex_form():
    """24 bands to a 1e-9 Ha residual: the real form's eigenvalues equal the
    complex form's from the same (real) start, and so do the first 8 bands'
    span (gap 0.256 Ha to the 9th)."""
    wl = diamond8_24()
    ctx, ham, _ = pair(wl)
    x0 = wl.x0_real(24)
    xr = dev(x0)
    xc = dev(x0.astype(np.complex128))
    opts = ctx.lobpcg_opts(maxit=200, tol=1e-9)
    eig_r, _, st_r, _ = ctx.lobpcg_real(xr, opts)
    eig_c, _, st_c, _ = ctx.lobpcg(xc, opts)
    assert st_r.converged and st_c.converged
    assert np.max(np.abs(eig_r - eig_c)) < 1e-9
    Xr, Xc = host(xr), host(xc)
    assert subspace_distance(Xr[:PREFIX8].astype(np.complex128), Xc[:PREFIX8], ham.dV) < 1e-7


def test_lobpcg_real_without_preconditioner_odd_bands():
    wl = small_cell(N=(10, 12, 8), L=(5.0, 6.0, 4.5), natom=2, nband=5, rcut=2.0)
    ctx, ham, _ = pair(wl)
    x0 = wl.x0_real()
    x = dev(x0)
    eig, res, stats, st = ctx.lobpcg_real(x, ctx.lobpcg_opts(maxit=600, tol=1e-8, precond=R.PRECOND_NONE))
    o = lobpcg_gamma(ham, x0, maxit=600, tol=1e-8, precond="none")
    assert stats.converged and o.converged
    assert np.max(np.abs(eig - o.eig)) < 1e-9
    assert np.max(res) <= 1e-8


def test_full_size_real_form_tracks_complex_form():
    """diamond64_64 (64^3, 144 bands), three iterations from one real start:
    the real and complex forms run the same algorithm on the same data, so
    their Ritz values agree to rounding; H x at this size against the oracle on
    a few bands."""
    wl = diamond64_64()
    ctx, ham, _ = pair(wl)
    x0 = wl.x0_real(wl.nband)
    xr = dev(x0)
    xc = dev(x0.astype(np.complex128))
    opts = ctx.lobpcg_opts(maxit=3, tol=0.0)
    eig_r, res_r, st_r, _ = ctx.lobpcg_real(xr, opts)
    eig_c, res_c, st_c, _ = ctx.lobpcg(xc, opts)
    assert st_r.iterations == st_c.iterations == 3
    assert np.max(np.abs(eig_r - eig_c)) < 1e-9
    assert np.max(np.abs(res_r - res_c)) < 1e-7
    xs = x0[[0, 77, 143]]
    out = _real(xs.shape)
    ctx.apply_h_real(dev(xs), out)
    assert rel_err(host(out), apply_h_real(ham, xs)) < 1e-12


@pytest.mark.parametrize("kw", [dict(precision=R.MIXED), dict(precond=R.PRECOND_LEARNED), dict(tol=-1.0)])
def test_lobpcg_real_rejects_unsupported_options(kw):
    ctx = _ctx()
    x = dev(draw_x0_real(7, 4, ctx.n))
    with pytest.raises(R.RsdftError) as e:
        ctx.lobpcg_real(x, ctx.lobpcg_opts(**kw))
    assert e.value.status == R.E_INVALID


def test_scf_steps_real_match_oracle_small_cell():
    """Eight SCF steps of the real form against the oracle's SCF steps from the
    same real start (the oracle's complex LOBPCG keeps a real start real, and its
    first-step eigenpairs equal the Gamma-point oracle's, test_oracle_gamma)."""
    from oracle.scf import scf_init, scf_step
    wl = small_cell(N=(12, 12, 12), L=(6.0, 6.0, 6.0), natom=2, nband=6)
    ctx, ham, v_loc = pair(wl)
    n_el = 8.0
    x0 = wl.x0_real()
    opts = ctx.scf_opts(n_electrons=n_el, kT=0.0, beta=0.3, depth=4, k_lobpcg=3, first_maxit=200, tol=1e-8)
    ctx.scf_init(6, opts)
    st = scf_init(ham.grid, n_el, x0.astype(np.complex128), beta=0.3, depth=4)
    x = dev(x0)
    for step in range(8):
        out, eig, occ = ctx.scf_step_real(x, opts)
        o = scf_step(ham, v_loc, st, n_el, 0.0, k_lobpcg=3, first_maxit=200, tol=1e-8)
        assert abs(out.e_tot - o.e_tot) / wl.natom < 1e-8, step
        assert np.max(np.abs(eig - o.eig)) < 1e-9, step
        assert abs(out.drho - o.drho) < 1e-8, step
        assert np.array_equal(occ, o.f)
    X = host(x)
    assert np.allclose(gram_real(X, X, ham.dV), np.eye(6), atol=1e-12)


def test_scf_step_real_rejects_mixed_precision():
    wl = small_cell(N=(12, 12, 12), L=(6.0, 6.0, 6.0), natom=2, nband=6)
    ctx, ham, _ = pair(wl)
    opts = ctx.scf_opts(n_electrons=8.0, kT=0.0, precision=R.MIXED)
    ctx.scf_init(6, opts)
    with pytest.raises(R.RsdftError) as e:
        ctx.scf_step_real(dev(wl.x0_real()), opts)
    assert e.value.status == R.E_INVALID


def test_real_form_empty_and_degenerate_blocks():
    """Empty blocks are no-ops; a rotation with no input rows leaves base (or
    zeros); one band runs the iteration on a single padded pair row."""
    ctx = _ctx()
    n = ctx.n
    empty = _real((0, n))
    ctx.apply_h_real(empty, _real((0, n)))
    ctx.gram_real(empty, dev(draw_x0_real(8, 3, n)), _real((0, 3)))
    base = draw_x0_real(9, 5, n)
    out = _real((5, n))
    ctx.rotate_real(empty, _real((0, 5)), out, base=dev(base), sign=-1)
    assert np.array_equal(host(out), base)
    out.fill_(1.0)
    ctx.rotate_real(empty, _real((0, 5)), out)
    assert np.all(host(out) == 0.0)


def test_lobpcg_real_one_band_matches_oracle():
    wl = diamond8_24()
    ctx, ham, _ = pair(wl)
    x0 = wl.x0_real(1)
    x = dev(x0)
    eig, res, stats, st = ctx.lobpcg_real(x, ctx.lobpcg_opts(maxit=10, tol=0.0))
    o = lobpcg_gamma(ham, x0, maxit=10, tol=0.0)
    assert stats.iterations == o.iterations == 10
    assert abs(eig[0] - o.eig[0]) < 1e-9
    assert abs(res[0] - o.resnorm[0]) < 1e-7
