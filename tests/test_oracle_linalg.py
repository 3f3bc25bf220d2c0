"""Pins for oracle.linalg (Eq. 1): the Cholesky + two-TRSM route agrees with
the generalised library solver scipy.linalg.eigh(G_H, G_S)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.linalg import NotPositiveDefinite, cholesky_dropping, cholesky_lower, rayleigh_ritz


def _pair(k, seed, cond=None):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k))
    gh = a + a.conj().T
    q, _ = np.linalg.qr(rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k)))
    if cond is None:
        s = rng.uniform(0.5, 2.0, k)
    else:
        s = np.logspace(0, -np.log10(cond), k)
    gs = (q * s) @ q.conj().T
    return gh, 0.5 * (gs + gs.conj().T)


@pytest.mark.parametrize("k,nkeep", [(48, 16), (96, 32), (144, 48)])
def test_matches_generalised_eigh(k, nkeep):
    gh, gs = _pair(k, k)
    lam, C, _ = rayleigh_ritz(gh, gs, nkeep)
    ref = sla.eigh(gh, gs, eigvals_only=True)[:nkeep]
    assert np.allclose(lam, ref, rtol=0, atol=1e-11 * np.max(np.abs(ref)))
    assert np.allclose(C.conj().T @ gs @ C, np.eye(nkeep), atol=1e-12)
    assert np.allclose(C.conj().T @ gh @ C, np.diag(lam), atol=1e-11)


def test_ill_conditioned_overlap():
    gh, gs = _pair(64, 1, cond=1e8)
    lam, C, _ = rayleigh_ritz(gh, gs, 8)
    ref = sla.eigh(gh, gs, eigvals_only=True)[:8]
    assert np.allclose(lam, ref, rtol=1e-6)
    assert np.allclose(C.conj().T @ gs @ C, np.eye(8), atol=1e-7)


def test_not_positive_definite_raises():
    gh, gs = _pair(16, 2)
    gs[3, 3] = -1.0
    with pytest.raises(NotPositiveDefinite):
        cholesky_lower(gs)


def test_dropping_equals_cholesky_of_kept_submatrix():
    rng = np.random.default_rng(9)
    gh, gs = _pair(20, 3)
    # make columns 7 and 15 exact combinations of earlier ones
    B = rng.standard_normal((20, 20)) + 1j * rng.standard_normal((20, 20))
    B[:, 7] = 0.5 * B[:, 2] - 1j * B[:, 4]
    B[:, 15] = B[:, 7] + 2.0 * B[:, 11]
    gs = B.conj().T @ B
    L, dropped = cholesky_dropping(gs, 1e-10)
    assert dropped.tolist() == [i in (7, 15) for i in range(20)]
    keep = ~dropped
    ref = cholesky_lower(gs[np.ix_(keep, keep)])
    assert np.allclose(L[np.ix_(keep, keep)], ref, atol=1e-12)
    lam, C, nd = rayleigh_ritz(gh, gs, 6, pivot_tol=1e-10)
    assert nd == 2 and np.all(C[~keep] == 0)
    ref_lam = sla.eigh(gh[np.ix_(keep, keep)], gs[np.ix_(keep, keep)], eigvals_only=True)[:6]
    assert np.allclose(lam, ref_lam, atol=1e-8 * np.max(np.abs(ref_lam)))
