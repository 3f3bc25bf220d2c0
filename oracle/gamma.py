"""Oracle: the real-arithmetic Gamma-point form of the LOBPCG block iteration.

Test infrastructure only (see ``oracle/__init__``).

At the Gamma point with a real local potential and real Kleinman-Bylander
projectors (the truncated Gaussian s, p_x, p_y, p_z of ``grid.kb_projectors``),
H is a real symmetric operator on real grid functions and its eigenvectors can
be taken real.  The paper benchmarks the real-symmetric eigensolver of this
case beside the Hermitian one (Fig. 3a against Fig. 3b).  The iteration here is
``oracle.lobpcg``'s (its steps a-g, the same soft locking, pivot floor and
Hetmaniuk-Lehoucq orthogonalisation) with every block real:

* H x for real x: T x by a real-to-complex transform (``scipy.fft.rfftn``) --
  the multiplier |G|^2/2 is real and even in G, so T maps real functions to
  real functions and the half spectrum determines the result; V x pointwise;
  sum_aj beta_aj E_aj <beta_aj|x> with real beta;
* TPA: K((|G|^2/2) / t_b) is real and even in G, applied through the same
  real transform, so W is real;
* Gram matrices G = Y Z^T dV, real symmetric;
* Rayleigh-Ritz: Eq. 1 in real arithmetic (``linalg.rayleigh_ritz`` keeps a
  real input real: real Cholesky with the dropping rule, two real triangular
  solves, a real symmetric eigensolve).

Pins (tests/test_oracle_gamma.py): cos(G.r) and sin(G.r) are eigenfunctions of
the real kinetic operator with eigenvalue |G|^2/2, and TPA maps them to
K(x_G) times themselves (closed forms); the real H applied to real blocks
equals the complex oracle's H on the same blocks with an imaginary part at
rounding level (fftn against rfftn); H(x_a + i x_b) = H x_a + i H x_b, the
identity that lets two real bands share one complex transform; the real
Rayleigh-Ritz matches scipy.linalg.eigh(G_H, G_S) and gives C^T G_S C = I; on
a 12^3 cell with projectors the converged eigenvalues equal the lowest of the
dense real symmetric H built independently (Kronecker sum of explicit 1D
kinetic matrices, diagonal V, projector outer products); on the 24^3 diamond
cell they equal the complex oracle's LOBPCG eigenvalues.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np
import scipy.fft as sfft

from .hamiltonian import Hamiltonian
from .linalg import hermitise, rayleigh_ritz
from .lobpcg import LOCK_TOL, PIVOT_TOL, tpa_factor


def _half_t(ham: Hamiltonian) -> np.ndarray:
    """|G|^2/2 on the half spectrum of a real transform over (z, y, x): x
    frequencies 0 .. Nx/2, the layout of ``rfftn`` along its last axis."""
    nx = ham.grid.shape[2]
    return ham.t_g[:, :, : nx // 2 + 1]


def kinetic_real(ham: Hamiltonian, X: np.ndarray) -> np.ndarray:
    """T x_b = IRFFT(|G|^2/2 RFFT(x_b)) for real rows x_b."""
    X = np.asarray(X, dtype=np.float64)
    m = X.shape[0]
    shape = ham.grid.shape
    f = sfft.rfftn(X.reshape((m,) + shape), axes=(1, 2, 3), workers=ham.workers)
    f *= _half_t(ham)
    return sfft.irfftn(f, s=shape, axes=(1, 2, 3), workers=ham.workers).reshape(m, -1)


def apply_h_real(ham: Hamiltonian, X: np.ndarray) -> np.ndarray:
    """H x_b = T x_b + V x_b + sum_aj beta_aj E_aj <beta_aj|x_b>, real rows."""
    X = np.asarray(X, dtype=np.float64)
    out = kinetic_real(ham, X) + ham.v[None, :] * X
    if ham.proj is not None:
        p = (ham.proj.B @ X.T) * ham.dV
        out += (ham.proj.B.T @ (ham.proj.E[:, None] * p)).T
    return out


def kinetic_energy_real(ham: Hamiltonian, X: np.ndarray) -> np.ndarray:
    """t_b = <x_b|T|x_b> per real band."""
    return np.sum(X * kinetic_real(ham, X), axis=1) * ham.dV


def tpa_apply_real(ham: Hamiltonian, R: np.ndarray, tb: np.ndarray) -> np.ndarray:
    """W_b = IRFFT(K((|G|^2/2)/t_b) RFFT(R_b)) for real rows (t_b < 1e-12 -> 1)."""
    tb = np.where(tb < 1e-12, 1.0, tb)
    m = R.shape[0]
    shape = ham.grid.shape
    f = sfft.rfftn(np.asarray(R, dtype=np.float64).reshape((m,) + shape), axes=(1, 2, 3),
                   workers=ham.workers)
    f *= tpa_factor(_half_t(ham)[None] / tb[:, None, None, None])
    return sfft.irfftn(f, s=shape, axes=(1, 2, 3), workers=ham.workers).reshape(m, -1)


def gram_real(A: np.ndarray, B: np.ndarray, dV: float) -> np.ndarray:
    """G[i, j] = <a_i|b_j> = sum_r a_i(r) b_j(r) dV for real rows."""
    return (A @ B.T) * dV


def _colnorms(a: np.ndarray, dV: float) -> np.ndarray:
    return np.sqrt(np.sum(a * a, axis=1) * dV)


def _rotate(C: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """out[b] = sum_i C[i, b] Y[i]."""
    return C.T @ Y


@dataclasses.dataclass
class GammaResult:
    eig: np.ndarray            # Theta [m]
    X: np.ndarray              # real [m][n], <x_i|x_j> = delta_ij
    HX: np.ndarray
    resnorm: np.ndarray
    iterations: int
    converged: bool
    ritz_history: List[np.ndarray]
    res_history: List[np.ndarray]
    p_dropped: int


def lobpcg_gamma(ham: Hamiltonian, X0: np.ndarray, maxit: int, tol: float = 0.0,
                 nconv: Optional[int] = None, precond: str = "tpa",
                 lock_tol: float = LOCK_TOL, pivot_tol: float = PIVOT_TOL) -> GammaResult:
    """LOBPCG for the lowest m eigenpairs of the real symmetric H (real X0)."""
    dV = ham.dV
    X = np.array(X0, dtype=np.float64)
    if X.ndim != 2:
        raise ValueError("X0 must be [m][n]")
    m = X.shape[0]
    nconv = m if nconv is None else nconv
    HX = apply_h_real(ham, X)
    gs = hermitise(gram_real(X, X, dV))
    gh = hermitise(gram_real(X, HX, dV))
    theta, C, _ = rayleigh_ritz(gh, gs, m, pivot_tol=PIVOT_TOL)
    X, HX = _rotate(C, X), _rotate(C, HX)
    P = HP = None
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
            W = tpa_apply_real(ham, R[act], kinetic_energy_real(ham, X[act]))
        elif precond == "none":
            W = R[act].copy()
        else:
            raise ValueError(precond)
        W = W - _rotate(gram_real(X, W, dV), X)
        HW = apply_h_real(ham, W)
        nw = _colnorms(W, dV)
        W /= nw[:, None]
        HW /= nw[:, None]
        blocks, hblocks = [X, W], [HX, HW]
        if P is not None:
            Pa, HPa = P[act], HP[act]
            npn = _colnorms(Pa, dV)
            blocks.append(Pa / npn[:, None])
            hblocks.append(HPa / npn[:, None])
        Y = np.concatenate(blocks)
        HY = np.concatenate(hblocks)
        gs = hermitise(gram_real(Y, Y, dV))
        gh = hermitise(gram_real(Y, HY, dV))
        lam, C, ndrop = rayleigh_ritz(gh, gs, m, pivot_tol=pivot_tol)
        dropped += ndrop
        P = _rotate(C[m:], Y[m:])
        HP = _rotate(C[m:], HY[m:])
        X = _rotate(C[:m], X) + P
        HX = _rotate(C[:m], HX) + HP
        theta = lam
        ritz_hist.append(theta.copy())
        it += 1
    return GammaResult(eig=theta, X=X, HX=HX, resnorm=res, iterations=it, converged=converged,
                       ritz_history=ritz_hist, res_history=res_hist, p_dropped=dropped)
