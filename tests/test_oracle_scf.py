"""Pins for oracle.scf: density, Hartree, LDA, occupations, mixing, energies."""
import numpy as np
import pytest

from oracle.grid import Grid, kb_projectors, local_potential
from oracle.hamiltonian import Hamiltonian, inner
from oracle.scf import (AndersonMixer, density, direct_energy, hartree, lda_xc, occupations,
                        pz81_correlation, scf_init, scf_step, slater_exchange)
from workloads import draw_x0, small_cell


def test_density_integrates_to_occupation_sum():
    g = Grid(L=(5.0, 6.0, 7.0), N=(10, 12, 14))
    X = draw_x0(0, 5, g.n)
    q, _ = np.linalg.qr(X.T)
    X = q.T / np.sqrt(g.dV)
    assert np.allclose(inner(X, X, g.dV), np.eye(5), atol=1e-13)
    f = np.array([2.0, 2.0, 1.5, 0.3, 0.0])
    rho = density(X, f)
    assert abs(np.sum(rho) * g.dV - f.sum()) < 1e-12


@pytest.mark.parametrize("k", [(1, 0, 0), (1, 2, -1), (0, -3, 2)])
def test_hartree_of_cosine(k):
    g = Grid(L=(5.0, 6.0, 7.0), N=(10, 12, 14))
    x, y, z = g.coords()
    G = [2 * np.pi / g.L[a] * k[a] for a in range(3)]
    phase = G[0] * x + G[1] * y + G[2] * z
    vh = hartree(g, np.cos(phase).reshape(-1))
    g2 = sum(gg * gg for gg in G)
    assert np.allclose(vh, (4 * np.pi / g2 * np.cos(phase)).reshape(-1), atol=1e-12)


def test_hartree_energy_nonnegative_and_constant_removed():
    g = Grid(L=(5.0, 5.0, 5.0), N=(10, 10, 10))
    rho = np.random.default_rng(1).uniform(0, 1, g.n)
    vh = hartree(g, rho)
    assert 0.5 * np.sum(vh * rho) * g.dV >= 0.0
    assert abs(np.sum(hartree(g, np.full(g.n, 3.0)))) < 1e-12


def test_slater_exchange_textbook_value():
    # eps_x = -(3/4)(9/(4 pi^2))^(1/3) / r_s = -0.458165... / r_s
    for rs in (0.5, 1.0, 2.0, 6.0):
        rho = 3.0 / (4.0 * np.pi * rs ** 3)
        ex, vx = slater_exchange(np.array([rho]))
        assert abs(ex[0] + 0.4581652932831429 / rs) < 1e-14
        assert abs(vx[0] - 4.0 / 3.0 * ex[0]) < 1e-15


def test_pz81_branches_meet_at_rs_one():
    rho1 = 3.0 / (4.0 * np.pi)
    lo = pz81_correlation(np.array([rho1 * (1 + 1e-12)]))     # r_s just below 1
    hi = pz81_correlation(np.array([rho1 * (1 - 1e-12)]))     # r_s just above 1
    assert abs(lo[0][0] - hi[0][0]) < 4e-5
    assert abs(lo[1][0] - hi[1][0]) < 1e-3
    # high-density branch at r_s = 1: B + D exactly; low-density: gamma/(1+b1+b2)
    assert abs(lo[0][0] - (-0.048 - 0.0116)) < 1e-12
    assert abs(hi[0][0] - (-0.1423 / (1 + 1.0529 + 0.3334))) < 1e-12


@pytest.mark.parametrize("rho", [1e-4, 3e-3, 0.05, 0.2, 0.9, 5.0])
def test_vxc_is_derivative_of_energy_density(rho):
    h = rho * 1e-5
    e = lambda r: (r * lda_xc(np.array([r]))[0])[0]
    fd = (e(rho + h) - e(rho - h)) / (2 * h)
    v = lda_xc(np.array([rho]))[1][0]
    assert abs(fd - v) < 1e-7 * max(1.0, abs(v))


def test_xc_clamps_tiny_and_negative_density():
    eps, v = lda_xc(np.array([-1e-3, 0.0, 5e-13]))
    assert np.all(eps == 0) and np.all(v == 0)


def test_fermi_dirac_counts_and_low_temperature_limit():
    eig = np.sort(np.random.default_rng(2).uniform(-1, 1, 40))
    for kT in (0.01, 0.1):
        f, mu, S = occupations(eig, 37.0, kT)
        assert abs(f.sum() - 37.0) < 1e-12
        assert np.all((f >= 0) & (f <= 2)) and S >= 0
    gapped = np.concatenate([np.linspace(-1, -0.5, 10), np.linspace(0.5, 1, 10)])
    f0, _, _ = occupations(gapped, 20.0, 0.0)
    f1, mu1, S1 = occupations(gapped, 20.0, 1e-4)
    assert np.allclose(f0, f1, atol=1e-12) and -0.5 < mu1 < 0.5 and S1 < 1e-12
    fa, _, _ = occupations(gapped, 7.0, 0.0)
    assert fa.tolist()[:4] == [2, 2, 2, 1] and fa[4:].sum() == 0


def test_anderson_depth0_is_linear_and_fixed_point_kept():
    rng = np.random.default_rng(3)
    a, b = rng.uniform(0, 1, 50), rng.uniform(0, 1, 50)
    mix0 = AndersonMixer(beta=0.3, depth=0)
    assert np.allclose(mix0.mix(a, b, 0.1), a + 0.3 * (b - a))
    # starting at a fixed point (F = 0 every step) the mixer never moves;
    # the history of F differences is then zero, so the first step's linear
    # update is taken and later steps see a singular system avoided by F = 0
    fixed = rng.uniform(0, 1, 50)
    mix = AndersonMixer(beta=0.3, depth=4)
    x = mix.mix(fixed, fixed, 0.1)
    assert np.array_equal(x, fixed)


def test_linear_response_exactness_of_anderson():
    # for a linear map rho_out = A rho_in + c, Anderson with enough history
    # reaches the fixed point (it is a Krylov method on the residual)
    rng = np.random.default_rng(4)
    n = 6
    A = 0.5 * np.diag(rng.uniform(-1, 1, n))
    c = rng.uniform(0, 1, n)
    fixed = np.linalg.solve(np.eye(n) - A, c)
    mix = AndersonMixer(beta=0.3, depth=n + 2)
    lin = AndersonMixer(beta=0.3, depth=0)
    x = np.zeros(n)
    y = np.zeros(n)
    for _ in range(2 * n):
        x = mix.mix(x, A @ x + c, 1.0)
        y = lin.mix(y, A @ y + c, 1.0)
    assert np.allclose(x, fixed, atol=1e-10)
    assert np.max(np.abs(y - fixed)) > 1e-3      # plain linear mixing is far slower


def test_scf_double_counting_equals_direct_functional():
    wl = small_cell(N=(12, 12, 12), L=(6.0, 6.0, 6.0), natom=2, nband=6)
    g = Grid(L=wl.L, N=wl.N)
    v_loc = local_potential(g, wl.positions, wl.Z, wl.sigma)
    P = kb_projectors(g, wl.positions, wl.rc, wl.rcut, wl.e_kb())
    ham = Hamiltonian(g, v_loc, P)
    n_el = 8.0
    st = scf_init(g, n_el, draw_x0(0, 6, g.n), beta=0.3, depth=4)
    out = None
    for _ in range(60):
        out = scf_step(ham, v_loc, st, n_el, 0.0, k_lobpcg=30, tol=1e-9)
        if out.drho < 1e-11:
            break
    assert out.drho < 1e-9
    assert abs(np.sum(out.rho_out) * g.dV - n_el) < 1e-11
    e_direct = direct_energy(ham, v_loc, out.lobpcg.X, out.f)
    assert abs(out.e_tot - e_direct) / wl.natom < 1e-8
