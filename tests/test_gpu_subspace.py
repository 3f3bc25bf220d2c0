"""GPU parity of the subspace pieces of the LOBPCG iteration: Gram matrices,
rotation, and the Rayleigh-Ritz of Eq. 1 (Cholesky with dropping, two TRSMs,
eigensolve, back-substitution), against the oracle and library routines."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.hamiltonian import inner
from oracle.linalg import rayleigh_ritz as oracle_rr
from tests.gpu_common import R, dev, host, need_gpu, rel_err, torch
from workloads import draw_x0

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _ctx(N=(20, 18, 15), L=(5.0, 5.0, 5.0)):
    return R.Context(L, N, np.zeros(N[0] * N[1] * N[2]))


@pytest.mark.parametrize("na,nb", [(1, 1), (7, 5), (64, 64), (67, 130)])
def test_gram_matches_oracle(na, nb):
    ctx = _ctx()
    a, b = draw_x0(1, na, ctx.n), draw_x0(2, nb, ctx.n)
    g = torch.empty((na, nb), dtype=torch.complex128, device="cuda")
    ctx.gram(dev(a), dev(b), g)
    assert rel_err(host(g), inner(a, b, ctx.dV)) < 1e-13


@pytest.mark.parametrize("k,m", [(3, 2), (9, 4), (70, 65), (130, 64)])
def test_rotate_matches_numpy(k, m):
    ctx = _ctx()
    y = draw_x0(3, k, ctx.n)
    c = draw_x0(4, k, m)
    base = draw_x0(5, m, ctx.n)
    out = torch.empty((m, ctx.n), dtype=torch.complex128, device="cuda")
    ctx.rotate(dev(y), dev(c), out)
    assert rel_err(host(out), c.T @ y) < 1e-13
    bt = dev(base)
    ctx.rotate(dev(y), dev(c), bt, base=bt, sign=-1)     # in place on the base
    assert rel_err(host(bt), base - c.T @ y) < 1e-13


def _pair(k, seed, cond=None):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k))
    gh = a + a.conj().T
    q, _ = np.linalg.qr(rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k)))
    s = rng.uniform(0.5, 2.0, k) if cond is None else np.logspace(0, -np.log10(cond), k)
    gs = (q * s) @ q.conj().T
    return gh, 0.5 * (gs + gs.conj().T)


@pytest.mark.parametrize("k", [1, 2, 6, 33, 48, 100, 432])
def test_rayleigh_ritz_matches_oracle(k):
    ctx = _ctx()
    nkeep = max(1, k // 3)
    gh, gs = _pair(k, k)
    c = torch.empty((k, nkeep), dtype=torch.complex128, device="cuda")
    lam, nd = ctx.rayleigh_ritz(dev(gh), dev(gs), nkeep, c, pivot_tol=1e-8)
    lam_o, c_o, nd_o = oracle_rr(gh, gs, nkeep, pivot_tol=1e-8)
    scale = max(1.0, np.max(np.abs(lam_o)))
    assert nd == nd_o == 0
    assert np.max(np.abs(lam - lam_o)) < 1e-11 * scale
    C = host(c)
    assert np.allclose(C.conj().T @ gs @ C, np.eye(nkeep), atol=1e-11)
    assert np.allclose(C.conj().T @ gh @ C, np.diag(lam), atol=1e-10 * scale)


def test_rayleigh_ritz_ill_conditioned():
    ctx = _ctx()
    gh, gs = _pair(96, 7, cond=1e7)
    c = torch.empty((96, 20), dtype=torch.complex128, device="cuda")
    lam, nd = ctx.rayleigh_ritz(dev(gh), dev(gs), 20, c, pivot_tol=1e-8)
    ref = sla.eigh(gh, gs, eigvals_only=True)[:20]
    assert nd == 0 and np.allclose(lam, ref, rtol=1e-6, atol=0)


def test_rayleigh_ritz_drops_dependent_columns_like_oracle():
    ctx = _ctx()
    rng = np.random.default_rng(9)
    B = rng.standard_normal((40, 40)) + 1j * rng.standard_normal((40, 40))
    B[:, 17] = 0.5 * B[:, 2] - 1j * B[:, 4]
    B[:, 33] = B[:, 17] + 2.0 * B[:, 21]
    gs = B.conj().T @ B
    gh, _ = _pair(40, 3)
    c = torch.empty((40, 10), dtype=torch.complex128, device="cuda")
    lam, nd = ctx.rayleigh_ritz(dev(gh), dev(gs), 10, c, pivot_tol=1e-10)
    lam_o, c_o, nd_o = oracle_rr(gh, gs, 10, pivot_tol=1e-10)
    assert nd == nd_o == 2
    assert np.max(np.abs(lam - lam_o)) < 1e-8 * np.max(np.abs(lam_o))
    C = host(c)
    assert np.all(C[[17, 33]] == 0)


def test_rayleigh_ritz_not_spd_is_reported():
    ctx = _ctx()
    gh, gs = _pair(12, 4)
    gs[:, 5:] = 0.0
    gs[5:, :] = 0.0
    c = torch.empty((12, 8), dtype=torch.complex128, device="cuda")
    with pytest.raises(R.RsdftError) as e:
        ctx.rayleigh_ritz(dev(gh), dev(gs), 8, c)
    assert e.value.status == R.E_NOT_SPD


@pytest.mark.parametrize("k,nkeep", [(50, 50), (200, 70), (432, 144)])
def test_eigh_with_degenerate_clusters(k, nkeep):
    ctx = _ctx()
    rng = np.random.default_rng(k)
    w = np.sort(rng.uniform(-3, 5, k))
    # exact multiplets (2, 3, 6-fold) and a near-degenerate pair at the cut
    w[10:12] = w[10]
    w[20:23] = w[20]
    w[30:36] = w[30]
    w = np.sort(w)
    q, _ = np.linalg.qr(rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k)))
    a = (q * w) @ q.conj().T
    a = 0.5 * (a + a.conj().T)
    z = torch.empty((k, nkeep), dtype=torch.complex128, device="cuda")
    lam = ctx.eigh(dev(a), nkeep, z)
    Z = host(z)
    ref = np.linalg.eigvalsh(a)[:nkeep]
    nrm = np.max(np.abs(w))
    assert np.max(np.abs(lam - ref)) < 1e-12 * nrm
    assert np.allclose(Z.conj().T @ Z, np.eye(nkeep), atol=1e-12)
    assert np.max(np.abs(a @ Z - Z * lam)) < 1e-11 * nrm


def _hermitian_with_multiplets(k, seed):
    """Hermitian k x k with exact 2-, 3- and 6-fold eigenvalues where they fit."""
    rng = np.random.default_rng(seed)
    w = np.sort(rng.uniform(-3, 5, k))
    for lo, hi in ((10, 12), (20, 23), (30, 36)):
        if hi <= k:
            w[lo:hi] = w[lo]
    w = np.sort(w)
    q, _ = np.linalg.qr(rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k)))
    a = (q * w) @ q.conj().T
    return 0.5 * (a + a.conj().T), float(np.max(np.abs(w)))


# Double-float keeps ~48 bits (unit 2^-48 = 3.6e-15); the Householder reduction's
# backward error is a few units per step over k <= 448 steps, ~1e-11 |A| at worst.
# Orthonormality is the inverse iteration's (FP64 in both forms): vectors whose
# eigenvalues are g apart come out orthogonal to ~eps ||T|| / g, and eigenvalues
# more than 1e-6 ||T|| apart are not re-orthogonalised, hence 3e-10.
DF_BAR = 2e-11
ORTH_BAR = 3e-10


@pytest.mark.parametrize("k,nkeep", [(2, 1), (17, 5), (50, 50), (200, 70), (432, 144), (448, 150), (600, 200)])
def test_eigh_double_float_cluster(k, nkeep):
    """RSDFT_DENSE_DF: the tridiagonalisation on one 16-CTA cluster in double-float
    (k <= 448; k = 600 takes the FP64 kernel) against LAPACK's eigenvalues."""
    ctx = _ctx()
    ctx.set_dense(R.DENSE_DF)
    a, nrm = _hermitian_with_multiplets(k, 1000 + k)
    z = torch.empty((k, nkeep), dtype=torch.complex128, device="cuda")
    lam = ctx.eigh(dev(a), nkeep, z)
    Z = host(z)
    ref = np.linalg.eigvalsh(a)[:nkeep]
    e_lam = np.max(np.abs(lam - ref)) / nrm
    e_orth = np.max(np.abs(Z.conj().T @ Z - np.eye(nkeep)))
    e_res = np.max(np.abs(a @ Z - Z * lam)) / nrm
    print(f"k {k}: eigenvalues {e_lam:.1e}, orthonormality {e_orth:.1e}, residual {e_res:.1e} (of |A|)")
    assert e_lam < DF_BAR and e_orth < ORTH_BAR and e_res < DF_BAR


@pytest.mark.parametrize("k,pivot_tol", [(432, 1e-8), (432, 1e-3), (300, 1e-3), (37, 1e-3)])
def test_rayleigh_ritz_double_float_matches_oracle(k, pivot_tol):
    """RSDFT_DENSE_DF: double-float tridiagonalisation and tridiagonal eigensolve;
    with a pivot floor >= 1e-6 the triangular solves run in double-float too."""
    ctx = _ctx()
    ctx.set_dense(R.DENSE_DF)
    nkeep = max(1, k // 3)
    gh, gs = _pair(k, k)
    c = torch.empty((k, nkeep), dtype=torch.complex128, device="cuda")
    lam, nd = ctx.rayleigh_ritz(dev(gh), dev(gs), nkeep, c, pivot_tol=pivot_tol)
    lam_o, _, nd_o = oracle_rr(gh, gs, nkeep, pivot_tol=pivot_tol)
    scale = max(1.0, np.max(np.abs(lam_o)))
    assert nd == nd_o == 0
    assert np.max(np.abs(lam - lam_o)) < DF_BAR * scale
    C = host(c)
    assert np.allclose(C.conj().T @ gs @ C, np.eye(nkeep), atol=ORTH_BAR)
    assert np.allclose(C.conj().T @ gh @ C, np.diag(lam), atol=DF_BAR * scale)


def test_set_dense_rejects_unknown_mode():
    ctx = _ctx()
    with pytest.raises(R.RsdftError) as e:
        ctx.set_dense(7)
    assert e.value.status == R.E_INVALID
