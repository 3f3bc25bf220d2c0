"""Oracle: the generalised Hermitian subspace problem of LOBPCG (Eq. 1).

Test infrastructure only (see ``oracle/__init__``).

The Rayleigh-Ritz step solves G_H C = G_S C Lambda.  Following Eq. 1, the
overlap is factorised G_S = L L^H (Cholesky), the problem is reduced to the
standard one K Z = Z Lambda with K = L^-1 G_H L^-H by two triangular solves
(the TRSM route the paper proposes in place of xHEGST), K is diagonalised, and
the coefficients come back through a third triangular solve C = L^-H Z.

The paper does not say what happens when G_S is numerically singular (LOBPCG
bases lose rank near convergence).  Reading used here and in the CUDA path:
the Cholesky drops a column whose pivot falls to a relative floor, which
removes that basis vector from the Rayleigh-Ritz problem (the reduction and
the eigensolve run on the kept columns).

Pins (tests/test_oracle_linalg.py): eigenvalues equal scipy.linalg.eigh(G_H,
G_S) (the HEGST-style library path the paper compares against); C^H G_S C = I;
C^H G_H C = diag(Lambda); ill-conditioned G_S (cond 1e8); a non-positive G_S
raises NotPositiveDefinite; column dropping equals the Cholesky of the kept
submatrix and returns zero coefficients on dropped columns.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


class NotPositiveDefinite(np.linalg.LinAlgError):
    pass



def hermitise(a: np.ndarray) -> np.ndarray:
    return 0.5 * (a + a.conj().T)


def cholesky_lower(gs: np.ndarray, pivot_tol: float = 0.0) -> np.ndarray:
    """G_S = L L^H, L lower triangular (Eq. 1), via the library routine.

    Raises NotPositiveDefinite when the factorisation breaks down or when a
    pivot L_kk^2 is at most pivot_tol * max_i G_S[i, i].
    """
    try:
        L = sla.cholesky(gs, lower=True)
    except np.linalg.LinAlgError as exc:
        raise NotPositiveDefinite(str(exc)) from exc
    piv = np.real(np.diag(L)) ** 2
    floor = pivot_tol * np.max(np.real(np.diag(gs)))
    if np.any(piv <= floor):
        raise NotPositiveDefinite(f"pivot {int(np.argmin(piv))} below {floor:g}")
    return L


def cholesky_dropping(gs: np.ndarray, pivot_tol: float):
    """Right-looking Cholesky G_S = L L^H that drops dependent columns.

    Column k is factorised against the columns kept before it.  When its
    pivot (the Schur complement G_S[k,k] - sum_j |L[k,j]|^2) is at most
    pivot_tol * max_i G_S[i,i], the column is dropped: L[:, k] = e_k and it
    takes no part in the trailing update.  The kept rows and columns of L are
    then exactly the Cholesky factor of G_S restricted to the kept columns.
    Returns (L, dropped_mask).
    """
    a = np.array(gs, dtype=np.complex128 if np.iscomplexobj(gs) else np.float64)
    k_tot = a.shape[0]
    floor = pivot_tol * np.max(np.real(np.diag(a)))
    L = np.zeros_like(a)
    dropped = np.zeros(k_tot, dtype=bool)
    for k in range(k_tot):
        d = np.real(a[k, k])
        if not d > floor:
            dropped[k] = True
            L[k, k] = 1.0
            continue
        lkk = np.sqrt(d)
        L[k, k] = lkk
        col = a[k + 1:, k] / lkk
        L[k + 1:, k] = col
        a[k + 1:, k + 1:] -= np.outer(col, col.conj())
    return L, dropped


def reduce_to_standard(gh: np.ndarray, L: np.ndarray) -> np.ndarray:
    """K = L^-1 G_H L^-H by two triangular solves (Eq. 1, the TRSM route).

    First TRSM: Y = L^-1 G_H.  Second TRSM: K = L^-1 Y^H, which equals
    L^-1 G_H L^-H because G_H is Hermitian.  K is then Hermitised.
    """
    y = sla.solve_triangular(L, gh, lower=True)
    k = sla.solve_triangular(L, y.conj().T, lower=True)
    return hermitise(k)


def rayleigh_ritz(gh: np.ndarray, gs: np.ndarray, nkeep: int, pivot_tol: float = 0.0):
    """Lowest nkeep eigenpairs of G_H c = lambda G_S c via Eq. 1.

    G_S is factorised by ``cholesky_dropping``; the reduction, the
    eigensolve and the back-substitution then run on the kept rows and
    columns only, and dropped basis vectors get zero coefficients.  Raises
    NotPositiveDefinite if fewer than nkeep columns survive.

    Returns (lam[nkeep] ascending, C[k, nkeep] with C = L^-H Z on the kept
    rows and 0 elsewhere, number of dropped columns).
    """
    L, dropped = cholesky_dropping(gs, pivot_tol)
    keep = ~dropped
    if np.count_nonzero(keep) < nkeep:
        raise NotPositiveDefinite("fewer independent columns than wanted pairs")
    Lk = L[np.ix_(keep, keep)]
    k = reduce_to_standard(gh[np.ix_(keep, keep)], Lk)
    lam, z = np.linalg.eigh(k)
    c = np.zeros((gs.shape[0], nkeep), dtype=Lk.dtype)
    c[keep] = sla.solve_triangular(Lk.conj().T, z[:, :nkeep], lower=False)
    return lam[:nkeep], c, int(np.count_nonzero(dropped))
