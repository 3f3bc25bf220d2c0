"""Pins for oracle.lobpcg: closed-form spectra, brute force, invariants."""
import numpy as np
import pytest
import scipy.fft as sfft
from scipy.optimize import brentq

from oracle.grid import Grid, kb_projectors, local_potential
from oracle.hamiltonian import Hamiltonian, inner
from oracle.lobpcg import lobpcg, tpa_factor
from tests.oracle_refs import hamiltonian_dense, kinetic_1d
from workloads import draw_x0, small_cell


def _free_electron_levels(L, kmax=3):
    ks = np.arange(-kmax, kmax + 1)
    kx, ky, kz = np.meshgrid(ks, ks, ks, indexing="ij")
    return np.sort(0.5 * (2 * np.pi / L) ** 2 * (kx ** 2 + ky ** 2 + kz ** 2).ravel())


@pytest.mark.parametrize("m", [7, 19])
def test_free_electron_closed_shells(m):
    g = Grid(L=(10.0, 10.0, 10.0), N=(12, 12, 12))
    ham = Hamiltonian(g, np.zeros(g.n))
    res = lobpcg(ham, draw_x0(1, m, g.n), maxit=200, tol=1e-8)
    assert res.converged
    ref = _free_electron_levels(10.0)[:m]
    assert abs(ref[1] - 0.19739208802178717) < 1e-15
    assert np.allclose(res.eig, ref, atol=1e-10, rtol=0)


def test_constant_potential_shifts_spectrum():
    g = Grid(L=(10.0, 10.0, 10.0), N=(12, 12, 12))
    ham = Hamiltonian(g, np.full(g.n, 0.7))
    res = lobpcg(ham, draw_x0(2, 7, g.n), maxit=200, tol=1e-8)
    assert np.allclose(res.eig, _free_electron_levels(10.0)[:7] + 0.7, atol=1e-10, rtol=0)


def test_separable_potential_non_cubic():
    N, L = (10, 12, 8), (5.0, 6.0, 4.5)
    g = Grid(L=L, N=N)
    x, y, z = (np.arange(N[a]) * L[a] / N[a] for a in range(3))
    vx = -1.2 * np.cos(2 * np.pi * x / L[0]) + 0.3 * np.sin(4 * np.pi * x / L[0])
    vy = -0.8 * np.cos(2 * np.pi * y / L[1]) + 0.2 * np.cos(6 * np.pi * y / L[1])
    vz = -0.5 * np.cos(2 * np.pi * z / L[2]) - 0.1 * np.sin(2 * np.pi * z / L[2])
    v = (vz[:, None, None] + vy[None, :, None] + vx[None, None, :]).reshape(-1)
    e1 = [np.linalg.eigvalsh(kinetic_1d(N[a], L[a]) + np.diag(va))
          for a, va in enumerate((vx, vy, vz))]
    sums = np.sort((e1[2][:, None, None] + e1[1][None, :, None] + e1[0][None, None, :]).ravel())
    m = 10
    assert sums[m] - sums[m - 1] > 1e-3
    ham = Hamiltonian(g, v)
    res = lobpcg(ham, draw_x0(3, m, g.n), maxit=300, tol=1e-8)
    assert res.converged
    assert np.allclose(res.eig, sums[:m], atol=1e-10, rtol=0)


def test_brute_force_12cubed_with_projectors_and_invariants():
    wl = small_cell(N=(12, 12, 12), L=(6.0, 6.0, 6.0), natom=2, nband=8)
    g = Grid(L=wl.L, N=wl.N)
    v = local_potential(g, wl.positions, wl.Z, wl.sigma)
    P = kb_projectors(g, wl.positions, wl.rc, wl.rcut, wl.e_kb())
    ham = Hamiltonian(g, v, P)
    Hd = hamiltonian_dense(g.N, g.L, v, P.B.toarray(), P.E)
    ref = np.linalg.eigvalsh(Hd)
    assert ref[8] - ref[7] > 1e-4
    res = lobpcg(ham, draw_x0(wl.seed, 8, g.n), maxit=300, tol=1e-8)
    assert res.converged
    assert np.allclose(res.eig, ref[:8], atol=1e-10, rtol=0)
    # X^H X dV = I
    assert np.allclose(inner(res.X, res.X, g.dV), np.eye(8), atol=1e-12)
    # Ritz values never increase (Courant-Fischer on nested subspaces)
    hist = np.array(res.ritz_history)
    assert np.all(np.diff(hist, axis=0) <= 1e-12 * np.max(np.abs(hist)))
    # residuals reported are those of the returned pairs
    r = ham.apply(res.X) - res.eig[:, None] * res.X
    assert np.allclose(np.sqrt(np.sum(np.abs(r) ** 2, 1) * g.dV), res.resnorm, atol=1e-12)


def test_lone_s_projector_secular_equation():
    L, N, E = 8.0, 16, 1.5
    g = Grid(L=(L, L, L), N=(N, N, N))
    P = kb_projectors(g, np.array([[1.3, 2.9, 4.1]]), 1.0, 3.0, np.array([[E]]), nproj=1)
    ham = Hamiltonian(g, np.zeros(g.n), P)
    beta = P.B.toarray()[0].reshape(g.shape)
    omega = L ** 3
    b = sfft.fftn(beta) * g.dV / np.sqrt(omega)     # <phi_G|beta>, phi_G = e^{iGr}/sqrt(omega)
    t = 0.5 * g.g2()
    w = np.abs(b.ravel()) ** 2
    tv = t.ravel()

    def secular(eps):
        return 1.0 - E * np.sum(w / (eps - tv))

    t1 = 0.5 * (2 * np.pi / L) ** 2
    root = brentq(secular, 1e-12, t1 - 1e-12, xtol=1e-15)
    res = lobpcg(ham, draw_x0(4, 6, g.n), maxit=300, tol=1e-8)
    assert res.converged
    assert abs(res.eig[0] - root) < 1e-10
    # five of the six |k| = 1 plane-wave combinations do not couple
    assert np.allclose(res.eig[1:6], t1, atol=1e-10)


def test_tpa_factor_limits():
    x = np.array([0.0, 1e-8, 1.0, 1e4])
    k = tpa_factor(x)
    assert k[0] == 1.0 and abs(k[1] - 1.0) < 1e-7
    assert abs(k[2] - 65.0 / 81.0) < 1e-15
    assert abs(k[3] - 1.0 / (2.0 * 1e4)) < 1e-7     # K ~ 8x^3 / 16x^4 = 1/(2x)
