"""Pins for oracle.hamiltonian: Hermiticity, projector identity, dense brute force."""
import numpy as np

from oracle.grid import Grid, kb_projectors, local_potential
from oracle.hamiltonian import Hamiltonian, inner
from tests.oracle_refs import hamiltonian_dense
from workloads import small_cell


def _ham(wl):
    g = Grid(L=wl.L, N=wl.N)
    v = local_potential(g, wl.positions, wl.Z, wl.sigma)
    P = kb_projectors(g, wl.positions, wl.rc, wl.rcut, wl.e_kb())
    return g, Hamiltonian(g, v, P)


def test_hermitian():
    wl = small_cell(N=(10, 12, 8), L=(5.5, 6.0, 5.0), natom=3, rcut=2.2)
    g, ham = _ham(wl)
    rng = np.random.default_rng(5)
    a = rng.standard_normal((3, g.n)) + 1j * rng.standard_normal((3, g.n))
    b = rng.standard_normal((3, g.n)) + 1j * rng.standard_normal((3, g.n))
    lhs = inner(a, ham.apply(b), g.dV)
    rhs = inner(ham.apply(a), b, g.dV)
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * np.max(np.abs(lhs))


def test_lone_projector_is_eigenvector_of_vnl():
    g = Grid(L=(8.0, 8.0, 8.0), N=(16, 16, 16))
    P = kb_projectors(g, np.array([[2.0, 3.0, 4.5]]), 1.0, 3.0, np.array([[1.7]]), nproj=1)
    ham = Hamiltonian(g, np.zeros(g.n), P)
    beta = P.B.toarray().astype(np.complex128)
    assert np.allclose(ham.nonlocal_(beta), 1.7 * beta, atol=1e-13)


def test_matches_independent_dense_matrix():
    wl = small_cell(N=(6, 8, 10), L=(4.5, 5.0, 5.5), natom=2, rcut=2.0)
    g, ham = _ham(wl)
    Hd = hamiltonian_dense(g.N, g.L, ham.v, ham.proj.B.toarray(), ham.proj.E)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((4, g.n)) + 1j * rng.standard_normal((4, g.n))
    assert np.allclose(ham.apply(x), (Hd @ x.T).T, atol=1e-11)
