"""GPU parity of GGA-PBE (rsdft_xc_pbe, the SCF step with xc = PBE) against the
oracle's PBE (oracle/gga.py: complex-step derivatives, FFT gradients)."""
import numpy as np
import pytest

from oracle import gga
from oracle.grid import Grid
from oracle.scf import scf_init, scf_step
from tests.gpu_common import R, dev, host, need_gpu, pair, torch
from workloads import small_cell

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("N", [(12, 10, 8), (15, 12, 9), (24, 24, 24)])
def test_pbe_fields_match_oracle(N):
    L = (6.0, 5.0, 4.5)
    g = Grid(L=L, N=N)
    x, y, z = (c.reshape(-1) for c in g.coords())
    rho = 0.05 * (1.0 + 0.6 * np.cos(2 * np.pi * x / L[0]) * np.cos(2 * np.pi * y / L[1])
                  + 0.3 * np.sin(4 * np.pi * z / L[2] + 0.2))
    rho[::97] = 1e-13                                 # a few points below the clamp
    ctx = R.Context(L, N, np.zeros(g.n))
    eps = torch.empty(g.n, dtype=torch.float64, device="cuda")
    vxc = torch.empty_like(eps)
    ctx.xc_pbe(dev(rho), eps, vxc)
    e_ref, v_ref = gga.pbe_xc(g, rho)
    assert np.max(np.abs(host(eps) - e_ref)) <= 1e-12 * np.max(np.abs(e_ref))
    assert np.max(np.abs(host(vxc) - v_ref)) <= 1e-11 * np.max(np.abs(v_ref))


def test_scf_steps_with_pbe_match_oracle_small_cell():
    wl = small_cell(N=(12, 12, 12), L=(6.0, 6.0, 6.0), natom=2, nband=6)
    ctx, ham, v_loc = pair(wl)
    n_el = 8.0
    x0 = wl.x0()
    opts = ctx.scf_opts(n_electrons=n_el, kT=0.0, beta=0.3, depth=4, k_lobpcg=3, first_maxit=200,
                        tol=1e-8, xc=R.XC_PBE)
    ctx.scf_init(6, opts)
    st = scf_init(ham.grid, n_el, x0, beta=0.3, depth=4)
    x = dev(x0)
    for step in range(6):
        out, eig, occ = ctx.scf_step(x, opts)
        o = scf_step(ham, v_loc, st, n_el, 0.0, k_lobpcg=3, first_maxit=200, tol=1e-8, xc="pbe")
        assert abs(out.e_tot - o.e_tot) / wl.natom < 1e-8, step
        assert np.max(np.abs(eig - o.eig)) < 1e-9, step
        assert abs(out.drho - o.drho) < 1e-8, step
