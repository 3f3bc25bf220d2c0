"""Oracle: Knyazev's LOBPCG for the lowest m Kohn-Sham orbitals.

Test infrastructure only (see ``oracle/__init__``).

The paper forms H and S on the LOBPCG subspace by GEMM (SCF task (2)) and
solves the generalised problem through Eq. 1 (task (3)); it cites Knyazev for
the method and gives no further detail, so the variant here is the plain
block form (the readings are listed in the design notes):

1.  X <- X0; HX <- H X; Rayleigh-Ritz on span(X) (Eq. 1) -> X, HX, Theta.
2.  Repeat:
    a. R = HX - X Theta; res_b = ||r_b|| (dV metric).  Stop when
       max_b res_b <= tol over the first ``nconv`` bands, or after maxit.
    b. Active set A = {b : res_b > lock_tol} (soft locking: a band whose
       residual is at round-off level keeps its place in X but contributes
       no W or P column, since its preconditioned residual is noise).
    c. W = T_prec(R_A) (Teter-Payne-Allan, TPA plus the learned network
       correction of ``oracle.precond``, or identity), then W <- W - X <X|W>
       (Hetmaniuk-Lehoucq orthogonalisation against X); HW = H W.
    d. Normalise the columns of W and P_A, scaling HW and HP_A alike.
    e. Y = [X W P_A] (first iteration [X W]), HY = [HX HW HP_A];
       G_S = <Y|Y>, G_H = <Y|HY> in full, Hermitised.
    f. Rayleigh-Ritz via Eq. 1 -> lowest m (Lambda, C).  The Cholesky of G_S
       drops every column whose pivot falls to pivot_tol * max_i G_S[i,i] or
       below (a numerically dependent W or P direction); dropped columns get
       zero coefficients (``linalg.rayleigh_ritz``).
    g. P <- [W P_A] C[m:], HP <- [HW HP_A] C[m:];
       X <- X C[:m] + P, HX <- HX C[:m] + HP; Theta <- Lambda.

Teter-Payne-Allan (PRB 40, 12255 (1989)): W_b = IFFT(K(x_G) FFT(R_b)) with
x_G = (|G|^2/2) / T_b, T_b = <x_b|T|x_b> (1 if below 1e-12) and
K(x) = (27 + 18x + 12x^2 + 8x^3) / (27 + 18x + 12x^2 + 8x^3 + 16x^4).

Pins (tests/test_oracle_lobpcg.py): free-electron spectrum (2pi/L)^2 |k|^2 / 2
with closed shells; separable potential = sums of three 1D dense spectra on a
non-cubic grid; constant-potential shift; 12^3 brute-force dense
diagonalisation; X^H X dV = I; Ritz values non-increasing (Courant-Fischer);
rank-1 secular equation of a lone s projector.  TPA itself
(tests/test_oracle_pins_closed_form.py): a plane wave maps to K(x_G) times
itself, with t_b chosen so that K takes the exact rational values 40/41,
65/81 and 175/431, per G in a sum of plane waves, and t_b < 1e-12 read as 1.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np
import scipy.fft as sfft

from .hamiltonian import Hamiltonian, inner
from .linalg import hermitise, rayleigh_ritz
from .precond import learned_apply, standardise


LOCK_TOL = 1e-10     # residual (Ha) at or below which a band is soft-locked
PIVOT_TOL = 1e-8     # relative Cholesky pivot floor for G_S


@dataclasses.dataclass
class LobpcgResult:
    eig: np.ndarray            # Theta [m]
    X: np.ndarray              # [m][n], <x_i|x_j> = delta_ij
    HX: np.ndarray
    resnorm: np.ndarray        # [m] final residual norms
    iterations: int            # full iterations done
    converged: bool
    ritz_history: List[np.ndarray]
    res_history: List[np.ndarray]
    p_dropped: int             # basis columns dropped by the Cholesky, summed
    P: Optional[np.ndarray] = None
    HP: Optional[np.ndarray] = None


def tpa_factor(x: np.ndarray) -> np.ndarray:
    """Teter-Payne-Allan K(x)."""
    num = 27.0 + x * (18.0 + x * (12.0 + 8.0 * x))
    return num / (num + 16.0 * x ** 4)


def tpa_precondition(ham: Hamiltonian, R: np.ndarray, X: np.ndarray) -> np.ndarray:
    """W_b = IFFT(K((|G|^2/2)/T_b) FFT(R_b)), T_b = <x_b|T|x_b>."""
    return tpa_apply(ham, R, ham.kinetic_energy(X))


def tpa_apply(ham: Hamiltonian, R: np.ndarray, tb: np.ndarray) -> np.ndarray:
    """W_b = IFFT(K((|G|^2/2)/t_b) FFT(R_b)) for given t_b (< 1e-12 -> 1)."""
    tb = np.where(tb < 1e-12, 1.0, tb)
    m = R.shape[0]
    shape = ham.grid.shape
    f = sfft.fftn(R.reshape((m,) + shape), axes=(1, 2, 3), workers=ham.workers)
    f *= tpa_factor(ham.t_g[None] / tb[:, None, None, None])
    return sfft.ifftn(f, axes=(1, 2, 3), workers=ham.workers).reshape(m, -1)


def _colnorms(a: np.ndarray, dV: float) -> np.ndarray:
    return np.sqrt(np.sum(np.abs(a) ** 2, axis=1) * dV)


def _rotate(C: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """out[b] = sum_i C[i, b] Y[i]."""
    return C.T @ Y


def rayleigh_ritz_block(ham: Hamiltonian, X: np.ndarray, HX: np.ndarray):
    """Initial Rayleigh-Ritz on span(X)."""
    dV = ham.dV
    gs = hermitise(inner(X, X, dV))
    gh = hermitise(inner(X, HX, dV))
    lam, C, _ = rayleigh_ritz(gh, gs, X.shape[0], pivot_tol=PIVOT_TOL)
    return lam, _rotate(C, X), _rotate(C, HX)


def lobpcg(ham: Hamiltonian, X0: np.ndarray, maxit: int, tol: float = 0.0,
           nconv: Optional[int] = None, precond: str = "tpa",
           P0: Optional[np.ndarray] = None, HP0: Optional[np.ndarray] = None,
           initial_rr: bool = True, lock_tol: float = LOCK_TOL,
           pivot_tol: float = PIVOT_TOL, nn_weights: Optional[np.ndarray] = None,
           nn_hidden: int = 8) -> LobpcgResult:
    dV = ham.dV
    m = X0.shape[0]
    nconv = m if nconv is None else nconv
    X = np.array(X0, dtype=np.complex128)
    HX = ham.apply(X)
    if initial_rr:
        theta, X, HX = rayleigh_ritz_block(ham, X, HX)
    else:
        theta = np.real(np.sum(X.conj() * HX, axis=1)) * dV
    P, HP = P0, HP0
    ritz_hist, res_hist = [theta.copy()], []
    dropped = 0
    it = 0
    while True:
        R = HX - theta[:, None] * X
        res = _colnorms(R, dV)
        res_hist.append(res)
        converged = bool(np.max(res[:nconv]) <= tol) if nconv > 0 else True
        if converged or it >= maxit:
            break
        act = np.nonzero(res > lock_tol)[0]
        if act.size == 0:
            break
        if precond == "tpa":
            W = tpa_precondition(ham, R[act], X[act])
        elif precond == "learned":
            # TPA plus the network correction (oracle.precond, residual form)
            W = learned_apply(R[act], tpa_precondition(ham, R[act], X[act]), standardise(ham.v),
                              nn_weights, ham.grid.shape, nn_hidden)
        elif precond == "none":
            W = R[act].copy()
        else:
            raise ValueError(precond)
        W = W - _rotate(inner(X, W, dV), X)
        HW = ham.apply(W)
        nw = _colnorms(W, dV)
        W /= nw[:, None]
        HW /= nw[:, None]
        blocks = [X, W]
        hblocks = [HX, HW]
        if P is not None:
            Pa, HPa = P[act], HP[act]
            npn = _colnorms(Pa, dV)
            blocks.append(Pa / npn[:, None])
            hblocks.append(HPa / npn[:, None])
        Y = np.concatenate(blocks)
        HY = np.concatenate(hblocks)
        gs = hermitise(inner(Y, Y, dV))
        gh = hermitise(inner(Y, HY, dV))
        lam, C, ndrop = rayleigh_ritz(gh, gs, m, pivot_tol=pivot_tol)
        dropped += ndrop
        P = _rotate(C[m:], Y[m:])
        HP = _rotate(C[m:], HY[m:])
        X = _rotate(C[:m], X) + P
        HX = _rotate(C[:m], HX) + HP
        theta = lam
        ritz_hist.append(theta.copy())
        it += 1
    return LobpcgResult(eig=theta, X=X, HX=HX, resnorm=res, iterations=it,
                        converged=converged, ritz_history=ritz_hist, res_history=res_hist,
                        p_dropped=dropped, P=P, HP=HP)
