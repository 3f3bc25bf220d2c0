"""Oracle: the GGA exchange-correlation of Perdew, Burke and Ernzerhof (PBE).

Test infrastructure only (see ``oracle/__init__``).

The paper's benchmarks use GGA-PBE (its benchmark-target paragraph); the
synthetic workloads default to LDA, and this module is the PBE alternative of
the SCF step, spin-unpolarised:

* Energy density e(rho, sigma) = rho (eps_x + eps_c), sigma = |grad rho|^2:
  - exchange (PBE 1996): eps_x = -(3/(4 pi)) k_F F_x(s), k_F = (3 pi^2 rho)^(1/3),
    s^2 = sigma / (4 k_F^2 rho^2), F_x = 1 + kappa - kappa / (1 + mu s^2 / kappa),
    kappa = 0.804, mu = beta pi^2 / 3;
  - correlation: eps_c = eps_c^PW92(r_s) + H, r_s = (3 / (4 pi rho))^(1/3),
    t^2 = sigma / (4 k_s^2 rho^2), k_s^2 = 4 k_F / pi,
    H = gamma ln(1 + (beta/gamma) t^2 (1 + A t^2) / (1 + A t^2 + A^2 t^4)),
    A = (beta/gamma) / (exp(-eps_c^PW92 / gamma) - 1), beta = 0.06672455060314922,
    gamma = (1 - ln 2) / pi^2;
  - eps_c^PW92 (Perdew and Wang 1992, unpolarised):
    -2 A0 (1 + a1 r_s) ln(1 + 1 / (2 A0 (b1 r_s^1/2 + b2 r_s + b3 r_s^3/2 + b4 r_s^2))),
    A0 = 0.031091, a1 = 0.21370, b1 = 7.5957, b2 = 3.5876, b3 = 1.6382, b4 = 0.49294.
  Points with rho < 1e-12 contribute nothing (as the LDA's clamp).
* de/drho and de/dsigma by complex-step differentiation (Squire and Trapp 1998):
  f'(x) = Im f(x + i h) / h, exact to rounding for the analytic e (written in
  sigma, not |grad rho|, so sigma = 0 is regular).
* Gradients by FFT, d_a f = IFFT(i G_a FFT(f)), real part, with the Nyquist
  plane of an even axis set to zero (for a real field its derivative is purely
  imaginary, so this equals taking the real part).
* v_xc = de/drho - sum_a d_a (2 de/dsigma d_a rho); E_xc = sum e dV.

Pins (tests/test_oracle_gga.py): the FFT gradient of cos(G.r + phi) is
-G sin(G.r + phi) and of a Nyquist plane is 0; at sigma = 0 exchange is
Slater's; PW92 agrees with the pinned PZ81 within 6e-4 Ha for r_s in
[0.1, 20]; the design limits F_x -> 1 + kappa (s -> inf), F_x = 1 + mu s^2 +
O(s^4), H = beta t^2 + O(t^4), eps_c^PW92 + H -> 0 (t -> inf); de/dsigma = 0
at sigma = 0 (mu = beta pi^2 / 3 cancels the second-order terms of exchange and
correlation, which fixes the scalings of s and t); v_xc equals the directional
derivative of E_xc by central differences; the complex-step derivatives match
central differences pointwise.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

from .grid import Grid

PBE_KAPPA = 0.804
PBE_BETA = 0.06672455060314922
PBE_MU = PBE_BETA * np.pi ** 2 / 3.0
PBE_GAMMA = (1.0 - np.log(2.0)) / np.pi ** 2
PW92_A0, PW92_A1 = 0.031091, 0.21370
PW92_B = (7.5957, 3.5876, 1.6382, 0.49294)
RHO_MIN = 1e-12
CSTEP = 1e-20


def pw92_correlation(rs):
    """eps_c of the uniform gas (PW92, unpolarised); rs may be complex."""
    srs = np.sqrt(rs)
    den = 2.0 * PW92_A0 * (PW92_B[0] * srs + PW92_B[1] * rs + PW92_B[2] * rs * srs + PW92_B[3] * rs * rs)
    return -2.0 * PW92_A0 * (1.0 + PW92_A1 * rs) * np.log(1.0 + 1.0 / den)


def exchange_enhancement(s2):
    return 1.0 + PBE_KAPPA - PBE_KAPPA / (1.0 + PBE_MU * s2 / PBE_KAPPA)


def correlation_gradient_term(ec_unif, t2):
    """H(eps_c^unif, t^2)."""
    A = (PBE_BETA / PBE_GAMMA) / (np.exp(-ec_unif / PBE_GAMMA) - 1.0)
    at2 = A * t2
    return PBE_GAMMA * np.log(1.0 + (PBE_BETA / PBE_GAMMA) * t2 * (1.0 + at2) / (1.0 + at2 + at2 * at2))


def energy_density(rho, sigma):
    """e = rho (eps_x + eps_c) for rho > 0 (rho, sigma may be complex)."""
    kf = np.exp(np.log(3.0 * np.pi ** 2 * rho) / 3.0)
    ex_unif = -0.75 / np.pi * kf
    s2 = sigma / (4.0 * kf * kf * rho * rho)
    rs = np.exp(np.log(3.0 / (4.0 * np.pi * rho)) / 3.0)
    ec = pw92_correlation(rs)
    t2 = sigma / (4.0 * (4.0 * kf / np.pi) * rho * rho)
    return rho * (ex_unif * exchange_enhancement(s2) + ec + correlation_gradient_term(ec, t2))


def energy_density_and_derivatives(rho, sigma):
    """(e, de/drho, de/dsigma) per point; zero where rho < 1e-12."""
    rho = np.asarray(rho, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    e = np.zeros_like(rho)
    dr = np.zeros_like(rho)
    ds = np.zeros_like(rho)
    ok = rho >= RHO_MIN
    r, s = rho[ok], sigma[ok]
    e[ok] = np.real(energy_density(r + 0j, s + 0j))
    hr = CSTEP * r
    dr[ok] = np.imag(energy_density(r + 1j * hr, s + 0j)) / hr
    hs = CSTEP * np.maximum(s, 1e-30)
    ds[ok] = np.imag(energy_density(r + 0j, s + 1j * hs)) / hs
    return e, dr, ds


def gradient(grid: Grid, f: np.ndarray):
    """[3][n] spectral derivatives of a real field (Nyquist planes zeroed)."""
    fg = sfft.fftn(f.reshape(grid.shape))
    out = []
    gx, gy, gz = grid.g_axes()
    for a, (g, N) in enumerate(zip((gx, gy, gz), grid.N)):
        g = np.array(g, dtype=np.float64)
        if N % 2 == 0:
            g[N // 2] = 0.0
        shape = [1, 1, 1]
        shape[2 - a] = N          # grid.shape is (Nz, Ny, Nx)
        out.append(np.real(sfft.ifftn(1j * g.reshape(shape) * fg)).reshape(-1))
    return np.stack(out)


def divergence(grid: Grid, h: np.ndarray) -> np.ndarray:
    """sum_a d_a h_a of a real vector field [3][n]."""
    return sum(gradient(grid, h[a])[a] for a in range(3))


def pbe_xc(grid: Grid, rho: np.ndarray):
    """(eps_xc, v_xc) per point, eps_xc = e / rho (0 where rho < 1e-12)."""
    rho = np.asarray(rho, dtype=np.float64)
    g = gradient(grid, rho)
    sigma = np.sum(g * g, axis=0)
    e, dr, ds = energy_density_and_derivatives(rho, sigma)
    v = dr - divergence(grid, 2.0 * ds[None, :] * g)
    eps = np.where(rho >= RHO_MIN, e / np.where(rho >= RHO_MIN, rho, 1.0), 0.0)
    return eps, v


def pbe_energy(grid: Grid, rho: np.ndarray) -> float:
    g = gradient(grid, rho)
    e, _, _ = energy_density_and_derivatives(rho, np.sum(g * g, axis=0))
    return float(np.sum(e)) * grid.dV
