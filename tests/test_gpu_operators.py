"""GPU parity of H psi, the projector gather, the TPA preconditioner and the
SCF field kernels against the FP64 oracle (through the C ABI)."""
import numpy as np
import pytest

from tests.gpu_common import R, dev, host, need_gpu, pair, rel_err, torch
from workloads import diamond8_24, draw_x0, small_cell

pytestmark = pytest.mark.gpu

# grids spanning every radix (2, 3, 4, 5, 8), odd sizes, non-cubic shapes and
# projector spheres that wrap the periodic boundary
CASES = [
    lambda: small_cell(N=(12, 10, 8), L=(6.0, 5.5, 5.0), natom=2, rcut=2.2),
    lambda: small_cell(N=(16, 18, 20), L=(6.5, 7.0, 7.5), natom=3, rcut=2.5),
    lambda: small_cell(N=(30, 30, 30), L=(7.0, 7.0, 7.0), natom=3, rcut=3.0),
    lambda: small_cell(N=(45, 45, 45), L=(9.0, 9.0, 9.0), natom=4, rcut=3.0),
    lambda: small_cell(N=(27, 25, 32), L=(6.0, 6.0, 7.0), natom=2, rcut=2.5),
    diamond8_24,
]


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("nb", [1, 5])
def test_apply_h_matches_oracle(case, nb):
    wl = CASES[case]()
    ctx, ham, _ = pair(wl)
    psi = draw_x0(case + 10, nb, ham.grid.n)
    out = torch.empty((nb, ham.grid.n), dtype=torch.complex128, device="cuda")
    ctx.apply_h(dev(psi), out)
    assert rel_err(host(out), ham.apply(psi)) < 1e-12


@pytest.mark.parametrize("case", range(len(CASES)))
def test_project_matches_oracle(case):
    wl = CASES[case]()
    ctx, ham, _ = pair(wl)
    nb = 7
    psi = draw_x0(case + 20, nb, ham.grid.n)
    p = torch.empty((nb, wl.natom * wl.nproj), dtype=torch.complex128, device="cuda")
    ctx.project(dev(psi), p)
    assert rel_err(host(p), ham.project(psi).T) < 1e-13


def test_projector_table_size():
    wl = diamond8_24()
    ctx, ham, _ = pair(wl)
    assert ctx.projector_entries() == ham.proj.B.nnz // wl.nproj


@pytest.mark.parametrize("case", [0, 3, 5])
def test_tpa_matches_oracle(case):
    from oracle.lobpcg import tpa_apply
    wl = CASES[case]()
    ctx, ham, _ = pair(wl)
    nb = 5
    r = draw_x0(case + 30, nb, ham.grid.n)
    tb = np.array([0.5, 1.7, 3.0, 0.0, 1e-13])   # the last two take the t < 1e-12 rule
    w = torch.empty_like(dev(r))
    ctx.precondition_tpa(dev(r), w, dev(tb))
    assert rel_err(host(w), tpa_apply(ham, r, tb)) < 1e-12


def test_empty_band_block_is_a_no_op():
    wl = CASES[0]()
    ctx, ham, _ = pair(wl)
    psi = torch.empty((0, ham.grid.n), dtype=torch.complex128, device="cuda")
    ctx.apply_h(psi, torch.empty_like(psi))


def test_density_hartree_lda_occupations():
    from oracle import scf as S
    wl = CASES[2]()
    ctx, ham, _ = pair(wl)
    g = ham.grid
    nb = 6
    X = draw_x0(40, nb, g.n) * 0.05
    f = np.array([2.0, 2.0, 1.7, 0.6, 0.01, 0.0])
    rho = torch.empty(g.n, dtype=torch.float64, device="cuda")
    ctx.density(dev(X), dev(f), rho)
    rho_o = S.density(X, f)
    assert rel_err(host(rho), rho_o) < 1e-14
    vh = torch.empty_like(rho)
    ctx.hartree(dev(rho_o), vh)
    assert rel_err(host(vh), S.hartree(g, rho_o)) < 1e-12
    # LDA over both PZ81 branches, the clamp and negative densities
    eps = torch.empty(g.n, dtype=torch.float64, device="cuda")
    vxc = torch.empty_like(eps)
    ctx.lda(dev(rho_o), eps, vxc)
    e_o, v_o = S.lda_xc(rho_o)
    assert rel_err(host(eps), e_o) < 1e-13 and rel_err(host(vxc), v_o) < 1e-13
    field = rho_o.copy()
    field[:5] = [0.0, -1e-3, 5e-13, 3.0 / (4 * np.pi), 10.0]
    ctx.lda(dev(field), eps, vxc)
    e_o, v_o = S.lda_xc(field)
    assert rel_err(host(eps), e_o) < 1e-13 and rel_err(host(vxc), v_o) < 1e-13
    eig = np.sort(np.random.default_rng(2).uniform(-1, 1, 37))
    for ne, kT in ((30.0, 0.0), (29.0, 0.0), (30.0, 0.01), (51.3, 0.1)):
        fo, muo, So = S.occupations(eig, ne, kT)
        fd = torch.empty(37, dtype=torch.float64, device="cuda")
        mu, Sg = ctx.occupations(dev(eig), ne, kT, fd)
        assert np.allclose(host(fd), fo, atol=1e-12, rtol=0)
        assert abs(mu - muo) < 1e-12 and abs(Sg - So) < 1e-11
