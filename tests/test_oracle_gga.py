"""Pins for oracle.gga (PBE): spectral gradient closed forms, the uniform-gas
limit, PW92 against the pinned PZ81, the functional's design limits, and
v_xc as the functional derivative of E_xc."""
import numpy as np
import pytest

from oracle import gga
from oracle.grid import Grid
from oracle.scf import pz81_correlation, slater_exchange


def test_gradient_of_cosines_and_nyquist():
    g = Grid(L=(7.0, 6.0, 5.0), N=(10, 12, 9))
    x, y, z = (c.reshape(-1) for c in g.coords())
    G = (2 * np.pi / 7.0 * 2, 2 * np.pi / 6.0 * -1, 2 * np.pi / 5.0 * 3)
    ph = 0.37
    f = np.cos(G[0] * x + G[1] * y + G[2] * z + ph)
    d = gga.gradient(g, f)
    s = np.sin(G[0] * x + G[1] * y + G[2] * z + ph)
    for a in range(3):
        assert np.allclose(d[a], -G[a] * s, atol=1e-12, rtol=0)
    nyq = np.cos(np.pi * 10 / 7.0 * x)          # the Nyquist plane of Nx = 10
    assert np.allclose(gga.gradient(g, nyq), 0.0, atol=1e-12)


def test_uniform_gas_exchange_is_slater_and_pw92_tracks_pz81():
    rho = np.array([1e-3, 1e-2, 0.1, 1.0])
    e, dr, ds = gga.energy_density_and_derivatives(rho, np.zeros_like(rho))
    ex, vx = slater_exchange(rho)
    rs = np.cbrt(3.0 / (4.0 * np.pi * rho))
    ec = gga.pw92_correlation(rs)
    assert np.allclose(e, rho * (ex + ec), rtol=1e-14, atol=0)
    rsg = np.array([0.1, 0.3, 0.5, 1.0, 2.0, 5.0, 10.0, 20.0])
    pz, _ = pz81_correlation(3.0 / (4.0 * np.pi * rsg ** 3))
    assert np.max(np.abs(gga.pw92_correlation(rsg) - pz)) < 6e-4


def test_design_limits():
    # exchange: F_x -> 1 + kappa (Lieb-Oxford), F_x = 1 + mu s^2 + O(s^4)
    assert abs(gga.exchange_enhancement(1e12) - (1.0 + gga.PBE_KAPPA)) < 1e-9
    s2 = 1e-6
    assert abs((gga.exchange_enhancement(s2) - 1.0) / s2 - gga.PBE_MU) < 1e-6
    assert abs(gga.PBE_MU - 0.2195149727645171) < 1e-15
    # correlation: H = beta t^2 + O(t^4); eps_c + H -> 0 as t -> inf
    for rs in (0.5, 2.0, 8.0):
        ec = gga.pw92_correlation(rs)
        t2 = 1e-7
        assert abs(gga.correlation_gradient_term(ec, t2) / t2 - gga.PBE_BETA) < 1e-5
        assert abs(ec + gga.correlation_gradient_term(ec, 1e14)) < 1e-9


def _smooth_density(g, amp=0.4):
    x, y, z = (c.reshape(-1) for c in g.coords())
    L = g.L
    return 0.05 * (1.0 + amp * np.cos(2 * np.pi * x / L[0]) * np.cos(2 * np.pi * y / L[1])
                   + 0.3 * np.sin(4 * np.pi * z / L[2] + 0.2))


@pytest.mark.parametrize("N", [(12, 10, 8), (9, 12, 10)])
def test_vxc_is_the_functional_derivative(N):
    g = Grid(L=(6.0, 5.0, 4.5), N=N)
    rho = _smooth_density(g)
    x, y, z = (c.reshape(-1) for c in g.coords())
    # a perturbation with structure (so the gradient terms count) and a projection
    # on v_xc of the size of E_xc (so the difference is far above rounding)
    eta = rho * (1.0 + 0.5 * np.cos(2 * np.pi * (x / g.L[0] + 2 * z / g.L[2]))
                 + 0.3 * np.sin(2 * np.pi * y / g.L[1]))
    _, v = gga.pbe_xc(g, rho)
    h = 1e-4
    fd = (gga.pbe_energy(g, rho + h * eta) - gga.pbe_energy(g, rho - h * eta)) / (2 * h)
    an = float(np.sum(v * eta)) * g.dV
    assert abs(fd - an) <= 1e-8 * abs(an)


def test_complex_step_matches_finite_differences_pointwise():
    rho = np.array([3e-3, 0.02, 0.4])
    sigma = np.array([1e-5, 2e-3, 0.3])
    _, dr, ds = gga.energy_density_and_derivatives(rho, sigma)
    for i in range(3):
        h = 1e-6 * rho[i]
        fr = (gga.energy_density(rho[i] + h, sigma[i]) - gga.energy_density(rho[i] - h, sigma[i])) / (2 * h)
        hs = 1e-6 * sigma[i]
        fs = (gga.energy_density(rho[i], sigma[i] + hs) - gga.energy_density(rho[i], sigma[i] - hs)) / (2 * hs)
        assert abs(fr - dr[i]) < 1e-7 * abs(dr[i]) and abs(fs - ds[i]) < 1e-6 * abs(ds[i])


def test_second_order_gradient_terms_cancel():
    """PBE takes mu = beta pi^2 / 3 so that the s^2 term of exchange,
    -3 mu / (16 pi k_F rho) per unit sigma, cancels the t^2 term of correlation,
    beta pi / (16 k_F rho) (t^2 = sigma / (4 k_s^2 rho^2), k_s^2 = 4 k_F / pi):
    de/dsigma vanishes at sigma = 0, which fixes the scalings of s and t."""
    rho = np.array([1e-3, 0.02, 0.3, 2.0])
    _, _, ds = gga.energy_density_and_derivatives(rho, np.zeros_like(rho))
    kf = np.cbrt(3.0 * np.pi ** 2 * rho)
    term = 3.0 * gga.PBE_MU / (16.0 * np.pi * kf * rho)
    assert np.all(np.abs(ds) < 1e-10 * term)
