"""Pins for oracle.gamma: the real-arithmetic Gamma-point LOBPCG.

Closed forms (cos/sin eigenfunctions of T, TPA on them), the complex oracle's
H as an independent route (fftn against rfftn), the two-bands-per-transform
identity, the real Rayleigh-Ritz against scipy's generalised eigensolver, and
converged eigenvalues against a dense real symmetric H and the complex LOBPCG.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.gamma import (apply_h_real, gram_real, kinetic_energy_real, kinetic_real,
                          lobpcg_gamma, tpa_apply_real)
from oracle.grid import Grid, kb_projectors, local_potential
from oracle.hamiltonian import Hamiltonian
from oracle.linalg import rayleigh_ritz
from oracle.lobpcg import lobpcg, tpa_factor
from tests.oracle_refs import hamiltonian_dense
from workloads import diamond8_24, draw_x0_real, small_cell


def _cell_ham(wl):
    g = Grid(L=wl.L, N=wl.N)
    v = local_potential(g, wl.positions, wl.Z, wl.sigma)
    P = kb_projectors(g, wl.positions, wl.rc, wl.rcut, wl.e_kb())
    return Hamiltonian(g, v, P)


def _plane_cos_sin(g, k):
    """cos(G.r), sin(G.r) on the grid for G = 2 pi k / L, and |G|^2/2."""
    x, y, z = g.coords()
    G = [2 * np.pi * k[a] / g.L[a] for a in range(3)]
    ph = (G[0] * x + G[1] * y + G[2] * z).reshape(-1)
    return np.cos(ph), np.sin(ph), 0.5 * sum(c * c for c in G)


@pytest.mark.parametrize("N,L", [((12, 12, 12), (10.0, 10.0, 10.0)), ((10, 12, 9), (5.0, 6.0, 4.5))])
def test_cos_sin_are_kinetic_eigenfunctions(N, L):
    g = Grid(L=L, N=N)
    ham = Hamiltonian(g, np.zeros(g.n))
    for k in [(1, 0, 0), (0, 2, 1), (1, -1, 2), (2, 3, -1)]:
        c, s, t = _plane_cos_sin(g, k)
        out = kinetic_real(ham, np.stack([c, s]))
        assert np.allclose(out[0], t * c, atol=1e-12 * max(t, 1.0))
        assert np.allclose(out[1], t * s, atol=1e-12 * max(t, 1.0))
        # <x|T|x> of a normalised cosine is |G|^2/2
        cn = c / np.sqrt(np.sum(c * c) * g.dV)
        assert abs(kinetic_energy_real(ham, cn[None])[0] - t) < 1e-12 * max(t, 1.0)


def test_tpa_real_on_cosines_is_the_factor():
    g = Grid(L=(10.0, 10.0, 10.0), N=(12, 12, 12))
    ham = Hamiltonian(g, np.zeros(g.n))
    c1, _, t1 = _plane_cos_sin(g, (1, 0, 0))
    _, s2, t2 = _plane_cos_sin(g, (1, 2, 0))
    tb = np.array([t1, 0.5 * t2])   # x = 1 and x = 2: K = 65/81 and 175/431... per G
    out = tpa_apply_real(ham, np.stack([c1, s2]), tb)
    assert np.allclose(out[0], tpa_factor(np.array(1.0)) * c1, atol=1e-13)
    assert np.allclose(out[1], tpa_factor(np.array(2.0)) * s2, atol=1e-13)
    assert abs(tpa_factor(np.array(1.0)) - 65.0 / 81.0) < 1e-15
    # t_b below 1e-12 is read as 1
    out0 = tpa_apply_real(ham, c1[None], np.array([0.0]))
    assert np.allclose(out0[0], tpa_factor(np.array(t1)) * c1, atol=1e-13)


def test_real_h_equals_complex_h_on_real_blocks():
    wl = small_cell(N=(12, 14, 10), L=(6.5, 7.0, 6.2), natom=2, nband=5)
    ham = _cell_ham(wl)
    X = draw_x0_real(5, 5, ham.grid.n)
    hr = apply_h_real(ham, X)
    hc = ham.apply(X.astype(np.complex128))
    scale = np.max(np.abs(hc))
    assert np.max(np.abs(hc.imag)) < 1e-13 * scale
    assert np.max(np.abs(hr - hc.real)) < 1e-13 * scale


def test_two_real_bands_share_one_complex_transform():
    wl = small_cell(N=(12, 12, 12), L=(6.0, 6.0, 6.0), natom=2, nband=4)
    ham = _cell_ham(wl)
    X = draw_x0_real(6, 4, ham.grid.n)
    packed = X[0::2] + 1j * X[1::2]
    hp = ham.apply(packed)
    hr = apply_h_real(ham, X)
    scale = np.max(np.abs(hr))
    assert np.max(np.abs(hp.real - hr[0::2])) < 1e-13 * scale
    assert np.max(np.abs(hp.imag - hr[1::2])) < 1e-13 * scale


def test_real_rayleigh_ritz_against_generalised_eigensolver():
    rng = np.random.default_rng(11)
    k, m = 30, 9
    a = rng.standard_normal((k, k))
    gs = a @ a.T + 0.5 * np.eye(k)
    b = rng.standard_normal((k, k))
    gh = 0.5 * (b + b.T)
    lam, C, nd = rayleigh_ritz(gh, gs, m, pivot_tol=1e-12)
    assert nd == 0 and C.dtype == np.float64
    ref = sla.eigh(gh, gs, eigvals_only=True)[:m]
    assert np.allclose(lam, ref, atol=1e-11 * np.max(np.abs(ref)))
    assert np.allclose(C.T @ gs @ C, np.eye(m), atol=1e-10)
    assert np.allclose(C.T @ gh @ C, np.diag(lam), atol=1e-10 * np.max(np.abs(lam)))


def test_gram_real_brute_force():
    rng = np.random.default_rng(12)
    A, B = rng.standard_normal((3, 7)), rng.standard_normal((2, 7))
    g = gram_real(A, B, 0.25)
    for i in range(3):
        for j in range(2):
            assert abs(g[i, j] - 0.25 * sum(A[i, r] * B[j, r] for r in range(7))) < 1e-14


def test_gamma_lobpcg_brute_force_12cubed():
    wl = small_cell(N=(12, 12, 12), L=(6.0, 6.0, 6.0), natom=2, nband=8)
    ham = _cell_ham(wl)
    g = ham.grid
    P = ham.proj
    Hd = hamiltonian_dense(g.N, g.L, ham.v, P.B.toarray(), P.E)
    assert np.max(np.abs(Hd.imag)) == 0.0
    ref = np.linalg.eigvalsh(Hd.real)
    assert ref[8] - ref[7] > 1e-4
    res = lobpcg_gamma(ham, draw_x0_real(wl.seed, 8, g.n), maxit=300, tol=1e-8)
    assert res.converged and res.X.dtype == np.float64
    assert np.allclose(res.eig, ref[:8], atol=1e-10, rtol=0)
    assert np.allclose(gram_real(res.X, res.X, g.dV), np.eye(8), atol=1e-12)
    hist = np.array(res.ritz_history)
    assert np.all(np.diff(hist, axis=0) <= 1e-12 * np.max(np.abs(hist)))
    r = apply_h_real(ham, res.X) - res.eig[:, None] * res.X
    assert np.allclose(np.sqrt(np.sum(r * r, 1) * g.dV), res.resnorm, atol=1e-12)


@pytest.mark.parametrize("m", [16, 9])
def test_gamma_lobpcg_matches_complex_lobpcg_diamond8_24(m):
    # 16 bands (the cell's own count) and an odd count that ends at a gap of
    # 1.5e-2 Ha (band 9 at 0.590 Ha, band 10 at 0.605 Ha)
    wl = diamond8_24()
    ham = _cell_ham(wl)
    X0 = wl.x0_real(m)
    rr = lobpcg_gamma(ham, X0, maxit=200, tol=1e-8)
    rc = lobpcg(ham, X0.astype(np.complex128), maxit=200, tol=1e-8)
    assert rr.converged and rc.converged
    # residual 1e-8 bounds each eigenvalue error by ~res^2 / gap
    assert np.allclose(rr.eig, rc.eig, atol=1e-10, rtol=0)


def test_gamma_lobpcg_without_preconditioner_brute_force_12cubed():
    wl = small_cell(N=(12, 12, 12), L=(6.0, 6.0, 6.0), natom=2, nband=5)
    ham = _cell_ham(wl)
    g, P = ham.grid, ham.proj
    ref = np.linalg.eigvalsh(hamiltonian_dense(g.N, g.L, ham.v, P.B.toarray(), P.E).real)
    assert ref[5] - ref[4] > 1e-4
    res = lobpcg_gamma(ham, draw_x0_real(wl.seed, 5, g.n), maxit=1000, tol=1e-8, precond="none")
    assert res.converged
    assert np.allclose(res.eig, ref[:5], atol=1e-10, rtol=0)
