"""Pins for oracle.tddft: plane-wave closed forms, the dense matrix exponential."""
import math

import numpy as np
import scipy.linalg as sla

from oracle.grid import Grid, kb_projectors, local_potential
from oracle.hamiltonian import Hamiltonian
from oracle.tddft import propagate
from tests.oracle_refs import hamiltonian_dense
from workloads import draw_x0, small_cell


def _pw(g, k):
    x, y, z = g.coords()
    G = [2.0 * np.pi / g.L[a] * k[a] for a in range(3)]
    return np.exp(1j * (G[0] * x + G[1] * y + G[2] * z)).reshape(-1), 0.5 * sum(c * c for c in G)


def test_plane_waves_get_their_scalar_series():
    g = Grid(L=(7.0, 6.0, 5.0), N=(10, 12, 8))
    ham = Hamiltonian(g, np.zeros(g.n))
    p1, e1 = _pw(g, (1, 0, 0))
    p2, e2 = _pw(g, (2, -1, 3))
    dt, nsteps, order = 0.05, 7, 4

    def series(e):
        return sum((-1j * e * dt) ** j / math.factorial(j) for j in range(order + 1)) ** nsteps

    psi = propagate(ham, np.stack([p1, p1 + p2]), dt, nsteps, order)
    assert np.allclose(psi[0], series(e1) * p1, atol=1e-13, rtol=0)
    assert np.allclose(psi[1], series(e1) * p1 + series(e2) * p2, atol=1e-13, rtol=0)
    # a constant potential V0 multiplies by the series of e + V0
    ham_v = Hamiltonian(g, np.full(g.n, 0.3))
    psi_v = propagate(ham_v, p2[None], dt, nsteps, order)
    assert np.allclose(psi_v[0], series(e2 + 0.3) * p2, atol=1e-13, rtol=0)


def test_matches_dense_matrix_exponential_with_projectors():
    wl = small_cell(N=(12, 12, 12), L=(6.0, 6.0, 6.0), natom=2, nband=3)
    g = Grid(L=wl.L, N=wl.N)
    v = local_potential(g, wl.positions, wl.Z, wl.sigma)
    P = kb_projectors(g, wl.positions, wl.rc, wl.rcut, wl.e_kb())
    ham = Hamiltonian(g, v, P)
    Hd = hamiltonian_dense(g.N, g.L, v, P.B.toarray(), P.E)
    x0 = draw_x0(3, 3, g.n)
    dt, nsteps = 0.002, 5
    ref = (sla.expm(-1j * dt * nsteps * Hd) @ x0.T).T
    out = propagate(ham, x0, dt, nsteps, 12)
    assert np.max(np.abs(out - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_norm_drift_is_the_taylor_remainder():
    wl = small_cell(N=(10, 10, 10), L=(5.0, 5.0, 5.0), natom=1, nband=2, rcut=2.0)
    g = Grid(L=wl.L, N=wl.N)
    ham = Hamiltonian(g, local_potential(g, wl.positions, wl.Z, wl.sigma),
                      kb_projectors(g, wl.positions, wl.rc, wl.rcut, wl.e_kb()))
    x0 = draw_x0(4, 2, g.n)
    x0 /= np.sqrt(np.sum(np.abs(x0) ** 2, axis=1) * g.dV)[:, None]
    for order, bound in ((4, 1e-3), (8, 1e-9)):
        out = propagate(ham, x0, 0.001, 20, order)
        nrm = np.sum(np.abs(out) ** 2, axis=1) * g.dV
        assert np.max(np.abs(nrm - 1.0)) < bound
