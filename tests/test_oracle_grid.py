"""Pins for oracle.grid: reciprocal vectors, local potential, KB projectors.

The references here are independent restatements evaluated point by point in
pure Python on tiny grids (brute force), plus plane-wave identities.
"""
import math

import numpy as np
import pytest

from oracle.grid import Grid, kb_projectors, local_potential
from oracle.hamiltonian import Hamiltonian


def _mi(d, L):
    # nearest periodic image, written without numpy
    return d - L * math.floor(d / L + 0.5)


def test_fft_order_even_and_odd():
    g = Grid(L=(6.0, 5.0, 3.0), N=(6, 5, 4))
    gx, gy, gz = g.g_axes()
    assert np.allclose(gx, 2 * np.pi / 6.0 * np.array([0, 1, 2, -3, -2, -1]))
    assert np.allclose(gy, 2 * np.pi / 5.0 * np.array([0, 1, 2, -2, -1]))
    assert np.allclose(gz, 2 * np.pi / 3.0 * np.array([0, 1, -2, -1]))


@pytest.mark.parametrize("k", [(0, 0, 0), (1, 0, 0), (0, -2, 1), (3, 2, -1), (-4, 0, 3)])
def test_plane_wave_is_kinetic_eigenvector(k):
    g = Grid(L=(7.0, 6.0, 5.0), N=(8, 10, 9))
    x, y, z = g.coords()
    G = [2 * np.pi / g.L[a] * k[a] for a in range(3)]
    pw = np.exp(1j * (G[0] * x + G[1] * y + G[2] * z)).reshape(1, -1)
    ham = Hamiltonian(g, np.zeros(g.n))
    t = ham.kinetic(pw)
    # Nyquist (k_x = -4 on Nx = 8) carries |G|^2 of -N/2, identical to +N/2
    assert np.allclose(t, 0.5 * sum(gg * gg for gg in G) * pw, atol=1e-12)


def test_local_potential_matches_pointwise_loop():
    g = Grid(L=(4.0, 5.0, 6.0), N=(4, 5, 6))
    pos = np.array([[0.3, 4.6, 0.2], [2.1, 1.0, 5.7]])
    Z, sigma = 3.0, 0.7
    v = local_potential(g, pos, Z, sigma).reshape(g.shape)
    for iz in range(6):
        for iy in range(5):
            for ix in range(4):
                r = (ix * 1.0, iy * 1.0, iz * 1.0)
                ref = 0.0
                for R in pos:
                    d2 = sum(_mi(r[a] - R[a], g.L[a]) ** 2 for a in range(3))
                    ref += -Z * math.exp(-d2 / (2 * sigma * sigma))
                assert abs(v[iz, iy, ix] - ref) < 1e-14


def test_projectors_match_pointwise_loop_and_wrap_boundary():
    g = Grid(L=(6.0, 7.0, 8.0), N=(12, 14, 16))
    # the first atom sits next to the origin corner: its sphere wraps all faces
    pos = np.array([[0.1, 6.9, 0.2], [3.0, 3.5, 4.0]])
    rc, rcut = 0.8, 2.2
    ekb = np.array([[0.7, 1.1, 1.3, 1.9], [0.6, 0.8, 1.0, 1.2]])
    P = kb_projectors(g, pos, rc, rcut, ekb)
    B = P.B.toarray()
    dV = g.dV
    hx, hy, hz = g.h
    for a, R in enumerate(pos):
        raw = np.zeros((4, g.n))
        for iz in range(16):
            for iy in range(14):
                for ix in range(12):
                    d = (_mi(ix * hx - R[0], 6.0), _mi(iy * hy - R[1], 7.0), _mi(iz * hz - R[2], 8.0))
                    d2 = d[0] ** 2 + d[1] ** 2 + d[2] ** 2
                    if d2 < rcut * rcut:
                        e = math.exp(-d2 / (2 * rc * rc))
                        i = (iz * 14 + iy) * 12 + ix
                        raw[:, i] = [e, d[0] / rc * e, d[1] / rc * e, d[2] / rc * e]
        for j in range(4):
            ref = raw[j] / math.sqrt(float(np.sum(raw[j] ** 2)) * dV)
            assert np.allclose(B[4 * a + j], ref, atol=1e-15, rtol=0)
            assert abs(np.sum(B[4 * a + j] ** 2) * dV - 1.0) < 1e-13
    # wrapping: atom 0 reaches points on the far side of every face
    idx = np.nonzero(B[0])[0]
    iz, iy, ix = np.unravel_index(idx, g.shape)
    assert ix.max() == 11 and iy.min() == 0 and iz.max() == 15
    assert np.allclose(P.E, ekb.reshape(-1))


def test_rcut_beyond_half_cell_rejected():
    g = Grid(L=(4.0, 4.0, 4.0), N=(8, 8, 8))
    with pytest.raises(ValueError):
        kb_projectors(g, np.zeros((1, 3)), 1.0, 2.0, np.ones((1, 4)))
