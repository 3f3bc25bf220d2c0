"""Closed-form pins for oracle functions that the LOBPCG/SCF pins do not fix.

* ``tpa_apply``: a plane wave e^{iG.r} is mapped to K(x_G) e^{iG.r} with
  x_G = (|G|^2/2) / t_b.  The t_b values are chosen so that x_G is 1/2, 1 or 2,
  where the Teter-Payne-Allan factor K(x) = (27+18x+12x^2+8x^3) /
  (27+18x+12x^2+8x^3+16x^4) is the exact rational 40/41, 65/81 or 175/431: an
  inverted ratio t_b / (|G|^2/2) swaps the first and the last, |G|^2 in place
  of |G|^2/2 moves every x.
* ``Hamiltonian.kinetic_energy``: a normalised plane wave has <T> = |G|^2/2; an
  equal mix of two orthogonal plane waves has the mean of the two.
* ``occupations`` entropy: S = -(dOmega/dT) at fixed mu, with the grand potential
  Omega = -2 T sum_b ln(1 + exp(-(e_b - mu)/T)) of spin-degenerate fermions,
  by a central finite difference; one level at mu (f = 1) gives S = 2 ln 2.
* ``learned_apply``: a network whose only nonzero weights are centre taps on
  channel 0 is the pointwise map u -> tanh(tanh(tanh(a u + c u vhat))); the
  complex result is base + s (NN(Re r / s) + i NN(Im r / s)), s the rms of r.
"""
import numpy as np
import pytest

from oracle import precond as P
from oracle.grid import Grid
from oracle.hamiltonian import Hamiltonian
from oracle.lobpcg import tpa_apply
from oracle.scf import occupations


def _plane_wave(g, k):
    x, y, z = g.coords()
    G = [2.0 * np.pi / g.L[a] * k[a] for a in range(3)]
    return np.exp(1j * (G[0] * x + G[1] * y + G[2] * z)).reshape(-1), 0.5 * sum(c * c for c in G)


@pytest.mark.parametrize("k", [(1, 0, 0), (2, -1, 3), (0, 0, -4)])
def test_tpa_apply_plane_wave_rational_factors(k):
    g = Grid(L=(7.0, 6.0, 5.0), N=(10, 12, 8))   # k_z = -4 is the Nyquist plane of N_z = 8
    ham = Hamiltonian(g, np.zeros(g.n))
    pw, half_g2 = _plane_wave(g, k)
    # x = half_g2 / t_b = 1/2, 1, 2  ->  K = 40/41, 65/81, 175/431
    tb = np.array([2.0 * half_g2, half_g2, 0.5 * half_g2])
    R = np.stack([pw, pw, pw])
    W = tpa_apply(ham, R, tb)
    for b, kx in enumerate((40.0 / 41.0, 65.0 / 81.0, 175.0 / 431.0)):
        assert np.allclose(W[b], kx * pw, atol=1e-13, rtol=0)


def test_tpa_apply_acts_per_g_and_replaces_tiny_tb():
    g = Grid(L=(7.0, 6.0, 5.0), N=(10, 12, 8))
    ham = Hamiltonian(g, np.zeros(g.n))
    p1, h1 = _plane_wave(g, (1, 0, 0))
    p2, h2 = _plane_wave(g, (0, 2, 1))
    tb = h1 / 2.0                        # x_1 = 2, x_2 = 2 h2 / h1
    W = tpa_apply(ham, (p1 + p2)[None], np.array([tb]))
    x2 = h2 / tb
    k2 = (27 + 18 * x2 + 12 * x2 ** 2 + 8 * x2 ** 3) / (27 + 18 * x2 + 12 * x2 ** 2 + 8 * x2 ** 3 + 16 * x2 ** 4)
    assert np.allclose(W[0], 175.0 / 431.0 * p1 + k2 * p2, atol=1e-13, rtol=0)
    # t_b below 1e-12 is read as 1: with |G|^2/2 = 1 (scaled cell) x = 1 -> 65/81
    L = 2.0 * np.pi / np.sqrt(2.0)       # |G|^2 / 2 = 1 for k = (1, 0, 0)
    g1 = Grid(L=(L, L, L), N=(6, 6, 6))
    ham1 = Hamiltonian(g1, np.zeros(g1.n))
    q, hq = _plane_wave(g1, (1, 0, 0))
    assert abs(hq - 1.0) < 1e-14
    W1 = tpa_apply(ham1, q[None], np.array([1e-13]))
    assert np.allclose(W1[0], 65.0 / 81.0 * q, atol=1e-13, rtol=0)


def test_kinetic_energy_of_plane_waves():
    g = Grid(L=(7.0, 6.0, 5.0), N=(10, 12, 8))
    ham = Hamiltonian(g, np.zeros(g.n))
    omega = 7.0 * 6.0 * 5.0
    p1, h1 = _plane_wave(g, (2, -1, 3))
    p2, h2 = _plane_wave(g, (-5, 0, -4))   # Nyquist on x and z
    X = np.stack([p1, p2, (p1 + p2) / np.sqrt(2.0)]) / np.sqrt(omega)
    t = ham.kinetic_energy(X)
    assert np.allclose(t, [h1, h2, 0.5 * (h1 + h2)], atol=1e-12, rtol=0)
    # the same numbers written out from the lattice: (2 pi / L)^2 k^2 / 2 per axis
    ref1 = 0.5 * ((2 * np.pi * 2 / 7.0) ** 2 + (2 * np.pi / 6.0) ** 2 + (2 * np.pi * 3 / 5.0) ** 2)
    assert abs(t[0] - ref1) < 1e-12


@pytest.mark.parametrize("kT", [0.01, 0.1])
def test_fermi_dirac_entropy_is_minus_dOmega_dT(kT):
    eig = np.sort(np.random.default_rng(7).uniform(-1.0, 1.0, 30))
    f, mu, S = occupations(eig, 23.0, kT)

    def omega(T):
        return -2.0 * T * np.sum(np.logaddexp(0.0, -(eig - mu) / T))

    h = 1e-4 * kT
    s_fd = -(omega(kT + h) - omega(kT - h)) / (2.0 * h)
    assert S > 0.1
    assert abs(S - s_fd) <= 1e-7 * S


def test_fermi_dirac_entropy_of_a_half_filled_level():
    f, mu, S = occupations(np.array([0.0]), 1.0, 0.05)
    assert abs(f[0] - 1.0) < 1e-12
    assert abs(S - 2.0 * np.log(2.0)) < 1e-12


def _centre_tap_weights(a, c, hidden=P.HIDDEN):
    w = np.zeros(P.weight_count(hidden))
    layers = P.unpack(w, hidden)      # views into w
    centre = 13                        # d = (0, 0, 0)
    layers[0][centre, 0, 0] = a        # u channel -> hidden 0
    layers[0][centre, 1, 0] = c        # u * vhat channel -> hidden 0
    layers[1][centre, 0, 0] = 1.0
    layers[2][centre, 0, 0] = 1.0
    layers[3][centre, 0, 0] = 1.0
    return w


def test_learned_apply_pointwise_closed_form():
    g = Grid(L=(5.0, 4.0, 4.5), N=(6, 5, 4))
    rng = np.random.default_rng(11)
    r = rng.standard_normal((3, g.n)) + 1j * rng.standard_normal((3, g.n))
    r[1] *= 1e-3                       # the correction scales with the band's residual
    r[2] = 0.0                         # no residual: base unchanged
    base = rng.standard_normal((3, g.n)) + 1j * rng.standard_normal((3, g.n))
    vhat = P.standardise(rng.uniform(-2.0, 1.0, g.n))
    a, c = 0.7, -0.4
    w = _centre_tap_weights(a, c)
    out = P.learned_apply(r, base, vhat, w, g.shape)
    for b in range(3):
        s = np.sqrt(np.sum(np.abs(r[b]) ** 2) / g.n)
        if s == 0.0:
            assert np.array_equal(out[b], base[b])
            continue

        def nn(u):
            return np.tanh(np.tanh(np.tanh(a * u + c * u * vhat)))

        ref = base[b] + s * (nn(r[b].real / s) + 1j * nn(r[b].imag / s))
        assert np.allclose(out[b], ref, atol=1e-14 * max(1.0, s), rtol=0)


def test_learned_apply_commutes_with_positive_and_imaginary_scalings():
    g = Grid(L=(5.0, 4.0, 4.5), N=(6, 5, 4))
    rng = np.random.default_rng(12)
    r = rng.standard_normal((2, g.n)) + 1j * rng.standard_normal((2, g.n))
    base = rng.standard_normal((2, g.n)) + 1j * rng.standard_normal((2, g.n))
    vhat = P.standardise(rng.uniform(-2.0, 1.0, g.n))
    w = rng.standard_normal(P.weight_count()) * 0.3
    ref = P.learned_apply(r, base, vhat, w, g.shape)
    for c in (3.7, 1e-4):
        assert np.allclose(P.learned_apply(c * r, c * base, vhat, w, g.shape), c * ref,
                           atol=1e-12 * c, rtol=0)
    # Re/Im planes through one odd real network: multiplying by i commutes
    assert np.allclose(P.learned_apply(1j * r, 1j * base, vhat, w, g.shape), 1j * ref, atol=1e-12, rtol=0)
