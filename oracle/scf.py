"""Oracle: the self-consistent-field step around LOBPCG.

Test infrastructure only (see ``oracle/__init__``).

The paper's SCF iteration is its four tasks plus "Others" (density and
potential updates, Fig. 1).  The potential pieces used here are the ones the
synthetic workloads specify: FFT Hartree, LDA exchange-correlation (Slater
exchange + Perdew-Zunger 1981 correlation, spin-unpolarised), Anderson
density mixing, aufbau or Fermi-Dirac occupations.

Definitions (orbitals normalised with <psi|psi> = sum |psi|^2 dV = 1):

* rho(r) = sum_b f_b |psi_b(r)|^2, f_b in [0, 2]; sum rho dV = sum f = N_e.
* V_H(G) = 4 pi rho(G) / |G|^2, V_H(G = 0) = 0;  E_H = 1/2 sum V_H rho dV.
* Slater: eps_x = -(3/4)(3/pi)^(1/3) rho^(1/3), v_x = (4/3) eps_x.
* PZ81 (unpolarised), r_s = (3 / (4 pi rho))^(1/3):
    r_s >= 1: eps_c = g / (1 + b1 sqrt(r_s) + b2 r_s),
              v_c = eps_c (1 + 7/6 b1 sqrt(r_s) + 4/3 b2 r_s) / (1 + b1 sqrt(r_s) + b2 r_s)
    r_s <  1: eps_c = A ln r_s + B + C r_s ln r_s + D r_s,
              v_c = A ln r_s + (B - A/3) + 2/3 C r_s ln r_s + (2D - C)/3 r_s
    g = -0.1423, b1 = 1.0529, b2 = 0.3334, A = 0.0311, B = -0.048,
    C = 0.0020, D = -0.0116.  rho < 1e-12 gives eps = v = 0.
* Occupations: aufbau (kT = 0) or f = 2 / (1 + exp((eps - mu)/kT)) with mu
  from bisection on sum f = N_e; entropy S = -2 sum [f~ ln f~ + (1-f~) ln(1-f~)],
  f~ = f/2.
* Anderson mixing (depth M, weight beta): F = rho_out - rho_in; with the last
  min(k, M) differences dR_j = rho_in^{j+1} - rho_in^j, dF_j = F^{j+1} - F^j,
  gamma solves (dF^T dF + 1e-10 max(diag) I) gamma = dF^T F (dV inner
  products, LU solve; the small Tikhonov term keeps the system solvable as the
  differences vanish near convergence);
  rho_in <- (rho_in - dR gamma) + beta (F - dF gamma).  M = 0 is linear mixing.
* Energy (Harris-Foulkes / double-counting form, evaluated at rho_in):
  E = sum f eps - E_H[rho_in] - int v_xc[rho_in] rho_in + E_xc[rho_in];
  free energy E - kT S.  The ion-ion term is constant and omitted.

Pins (tests/test_oracle_scf.py): sum rho dV = N_e; Hartree of cos(G.r) is
(4 pi / |G|^2) cos(G.r); eps_x = -0.458165 / r_s; v_xc equals a central finite
difference of d(rho eps_xc)/d rho; the PZ81 branches meet at r_s = 1 to 4e-5;
sum f = N_e; kT -> 0 gives aufbau; the entropy equals -dOmega/dT at fixed mu
(central difference of the fermion grand potential) and is 2 ln 2 for one
half-filled level (tests/test_oracle_pins_closed_form.py); Anderson depth 0 is linear mixing and keeps
a fixed point; at self-consistency the double-counting energy equals the direct
functional T_s + int V_loc rho + E_NL + E_H + E_xc.
The absolute SCF energies of the synthetic pseudo-atoms have no external value
and are parity-unpinned (oracle vs CUDA only).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np
import scipy.fft as sfft
from scipy.special import expit

from .gga import pbe_xc
from .grid import Grid
from .hamiltonian import Hamiltonian
from .lobpcg import LobpcgResult, lobpcg

PZ_GAMMA, PZ_B1, PZ_B2 = -0.1423, 1.0529, 0.3334
PZ_A, PZ_B, PZ_C, PZ_D = 0.0311, -0.048, 0.0020, -0.0116
RHO_MIN = 1e-12
ANDERSON_REG = 1e-10   # Tikhonov term, relative to max diag of dF^T dF


def density(X: np.ndarray, f: np.ndarray) -> np.ndarray:
    return np.einsum("b,bi->i", f, np.abs(X) ** 2)


def hartree(grid: Grid, rho: np.ndarray) -> np.ndarray:
    g2 = grid.g2()
    rg = sfft.fftn(rho.reshape(grid.shape))
    with np.errstate(divide="ignore", invalid="ignore"):
        vg = np.where(g2 > 0.0, 4.0 * np.pi * rg / np.where(g2 > 0.0, g2, 1.0), 0.0)
    return np.real(sfft.ifftn(vg)).reshape(-1)


def slater_exchange(rho: np.ndarray):
    """(eps_x, v_x) per point for rho >= RHO_MIN (no clamping here)."""
    cx = -0.75 * (3.0 / np.pi) ** (1.0 / 3.0)
    ex = cx * np.cbrt(rho)
    return ex, (4.0 / 3.0) * ex


def pz81_correlation(rho: np.ndarray):
    """(eps_c, v_c) per point, Perdew-Zunger 1981 unpolarised, rho >= RHO_MIN."""
    rs = np.cbrt(3.0 / (4.0 * np.pi * rho))
    ec = np.empty_like(rs)
    vc = np.empty_like(rs)
    hi = rs >= 1.0
    s = np.sqrt(rs[hi])
    den = 1.0 + PZ_B1 * s + PZ_B2 * rs[hi]
    ec[hi] = PZ_GAMMA / den
    vc[hi] = ec[hi] * (1.0 + 7.0 / 6.0 * PZ_B1 * s + 4.0 / 3.0 * PZ_B2 * rs[hi]) / den
    lo = ~hi
    rl = rs[lo]
    ln = np.log(rl)
    ec[lo] = PZ_A * ln + PZ_B + PZ_C * rl * ln + PZ_D * rl
    vc[lo] = PZ_A * ln + (PZ_B - PZ_A / 3.0) + 2.0 / 3.0 * PZ_C * rl * ln + (2.0 * PZ_D - PZ_C) / 3.0 * rl
    return ec, vc


def lda_xc(rho: np.ndarray):
    """(eps_xc, v_xc) per point, Slater exchange + PZ81 correlation;
    points with rho < 1e-12 get eps = v = 0."""
    rho = np.asarray(rho, dtype=np.float64)
    eps = np.zeros_like(rho)
    v = np.zeros_like(rho)
    ok = rho >= RHO_MIN
    ex, vx = slater_exchange(rho[ok])
    ec, vc = pz81_correlation(rho[ok])
    eps[ok] = ex + ec
    v[ok] = vx + vc
    return eps, v


def occupations(eig: np.ndarray, n_electrons: float, kT: float):
    """(f, mu, S).  kT = 0: aufbau (f = 2 on the lowest N_e/2 bands)."""
    eig = np.asarray(eig, dtype=np.float64)
    m = eig.size
    if n_electrons > 2.0 * m:
        raise ValueError("more electrons than band slots")
    if kT <= 0.0:
        f = np.zeros(m)
        full = int(np.floor(n_electrons / 2.0))
        f[:full] = 2.0
        rest = n_electrons - 2.0 * full
        if rest > 0:
            f[full] = rest
        mu = eig[min(full, m - 1)]
        return f, float(mu), 0.0
    lo = eig.min() - 50.0 * kT - 1.0
    hi = eig.max() + 50.0 * kT + 1.0
    for _ in range(200):
        mu = 0.5 * (lo + hi)
        if np.sum(2.0 * expit(-(eig - mu) / kT)) > n_electrons:
            hi = mu
        else:
            lo = mu
    mu = 0.5 * (lo + hi)
    ft = expit(-(eig - mu) / kT)
    f = 2.0 * ft
    with np.errstate(divide="ignore", invalid="ignore"):
        s_terms = np.where(ft > 0, ft * np.log(ft), 0.0) + np.where(ft < 1, (1 - ft) * np.log1p(-ft), 0.0)
    return f, float(mu), float(-2.0 * np.sum(s_terms))


@dataclasses.dataclass
class AndersonMixer:
    beta: float = 0.3
    depth: int = 4
    rho_hist: List[np.ndarray] = dataclasses.field(default_factory=list)
    f_hist: List[np.ndarray] = dataclasses.field(default_factory=list)

    def mix(self, rho_in: np.ndarray, rho_out: np.ndarray, dV: float) -> np.ndarray:
        F = rho_out - rho_in
        self.rho_hist.append(rho_in.copy())
        self.f_hist.append(F.copy())
        keep = self.depth + 1
        self.rho_hist = self.rho_hist[-keep:]
        self.f_hist = self.f_hist[-keep:]
        k = len(self.f_hist) - 1
        if self.depth == 0 or k == 0:
            return rho_in + self.beta * F
        dR = np.stack([self.rho_hist[j + 1] - self.rho_hist[j] for j in range(k)])
        dF = np.stack([self.f_hist[j + 1] - self.f_hist[j] for j in range(k)])
        A = (dF @ dF.T) * dV
        b = (dF @ F) * dV
        scale = float(np.max(np.diag(A)))
        if not scale > 0.0:
            return rho_in + self.beta * F
        gamma = np.linalg.solve(A + ANDERSON_REG * scale * np.eye(k), b)
        rho_bar = rho_in - gamma @ dR
        f_bar = F - gamma @ dF
        return rho_bar + self.beta * f_bar


@dataclasses.dataclass
class ScfState:
    rho_in: np.ndarray
    X: np.ndarray
    mixer: AndersonMixer
    step: int = 0
    eig: Optional[np.ndarray] = None


@dataclasses.dataclass
class ScfOut:
    e_tot: float
    free_energy: float
    e_band: float
    e_h: float
    e_xc: float
    e_vxc: float
    mu: float
    entropy: float
    drho: float
    eig: np.ndarray
    f: np.ndarray
    rho_out: np.ndarray
    lobpcg: LobpcgResult


def effective_potential(grid: Grid, v_loc: np.ndarray, rho: np.ndarray, xc: str = "lda"):
    vh = hartree(grid, rho)
    if xc == "pbe":
        eps, vxc = pbe_xc(grid, rho)
    elif xc == "lda":
        eps, vxc = lda_xc(rho)
    else:
        raise ValueError(xc)
    return v_loc + vh + vxc, vh, eps, vxc


def scf_init(grid: Grid, n_electrons: float, X0: np.ndarray, beta=0.3, depth=4) -> ScfState:
    """Start from the uniform density N_e / volume."""
    rho = np.full(grid.n, n_electrons / (grid.n * grid.dV))
    return ScfState(rho_in=rho, X=np.array(X0, dtype=np.complex128),
                    mixer=AndersonMixer(beta=beta, depth=depth))


def scf_step(ham: Hamiltonian, v_loc: np.ndarray, state: ScfState, n_electrons: float,
             kT: float, k_lobpcg: int = 3, first_maxit: int = 200, tol: float = 1e-6,
             precond: str = "tpa", later_tol: float = 0.0, xc: str = "lda") -> ScfOut:
    """One SCF step.  The first step converges LOBPCG to ``tol``; later steps
    run ``k_lobpcg`` iterations, or, with ``later_tol > 0``, also converge to
    ``later_tol`` (at most ``first_maxit`` iterations), which makes each step a
    function of rho_in alone (the eigenpairs no longer depend on the iteration
    path)."""
    grid = ham.grid
    dV = grid.dV
    v_eff, vh, eps_xc, vxc = effective_potential(grid, v_loc, state.rho_in, xc)
    ham.set_potential(v_eff)
    m = state.X.shape[0]
    nocc = int(min(m, np.ceil(n_electrons / 2.0))) if kT <= 0 else m
    if state.step == 0:
        res = lobpcg(ham, state.X, maxit=first_maxit, tol=tol, nconv=nocc, precond=precond)
    elif later_tol > 0.0:
        res = lobpcg(ham, state.X, maxit=first_maxit, tol=later_tol, nconv=nocc, precond=precond)
    else:
        res = lobpcg(ham, state.X, maxit=k_lobpcg, tol=0.0, nconv=nocc, precond=precond)
    f, mu, S = occupations(res.eig, n_electrons, kT)
    rho_out = density(res.X, f)
    e_band = float(np.sum(f * res.eig))
    e_h = 0.5 * float(np.sum(vh * state.rho_in)) * dV
    e_xc = float(np.sum(eps_xc * state.rho_in)) * dV
    e_vxc = float(np.sum(vxc * state.rho_in)) * dV
    e_tot = e_band - e_h - e_vxc + e_xc
    drho = float(np.sqrt(np.sum((rho_out - state.rho_in) ** 2) * dV))
    state.rho_in = state.mixer.mix(state.rho_in, rho_out, dV)
    state.X = res.X
    state.eig = res.eig
    state.step += 1
    return ScfOut(e_tot=e_tot, free_energy=e_tot - kT * S, e_band=e_band, e_h=e_h, e_xc=e_xc,
                  e_vxc=e_vxc, mu=mu, entropy=S, drho=drho, eig=res.eig, f=f, rho_out=rho_out,
                  lobpcg=res)


def direct_energy(ham: Hamiltonian, v_loc: np.ndarray, X: np.ndarray, f: np.ndarray):
    """E_KS[rho] = T_s + int V_loc rho + E_NL + E_H[rho] + E_xc[rho], rho from X, f."""
    grid = ham.grid
    dV = grid.dV
    rho = density(X, f)
    ts = float(np.sum(f * ham.kinetic_energy(X)))
    e_loc = float(np.sum(v_loc * rho)) * dV
    e_nl = float(np.sum(f * np.real(np.sum(X.conj() * ham.nonlocal_(X), axis=1)))) * dV
    vh = hartree(grid, rho)
    eps, _ = lda_xc(rho)
    return ts + e_loc + e_nl + 0.5 * float(np.sum(vh * rho)) * dV + float(np.sum(eps * rho)) * dV
