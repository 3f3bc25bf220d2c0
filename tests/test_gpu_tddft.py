"""GPU parity of the real-time propagation (rsdft_propagate) with the oracle's
Taylor propagator, on a small cell with projectors and on the 64^3 bench cell
(a few bands, one step), and its norm drift on the full 144-band block."""
import numpy as np
import pytest

import workloads
from oracle.tddft import propagate
from tests.gpu_common import dev, host, need_gpu, pair

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("order,nsteps,dt", [(4, 10, 0.01), (1, 3, 0.002), (8, 4, 0.02)])
def test_propagate_matches_oracle_small_cell(order, nsteps, dt):
    wl = workloads.small_cell(N=(12, 10, 8), L=(6.0, 5.5, 5.0), natom=2, nband=5, rcut=2.2)
    ctx, ham, _ = pair(wl)
    x0 = wl.x0()
    x = dev(x0)
    ctx.propagate(x, dt, nsteps, order)
    ref = propagate(ham, x0, dt, nsteps, order)
    err = np.max(np.abs(host(x) - ref)) / np.max(np.abs(ref))
    assert err < 1e-12, err


def test_propagate_bench_cell_few_bands_and_norm_of_full_block():
    wl = workloads.diamond64_64()
    ctx, ham, _ = pair(wl)
    x0 = wl.x0(6)
    x = dev(x0)
    ctx.propagate(x, 0.01, 1, 4)
    ref = propagate(ham, x0, 0.01, 1, 4)
    assert np.max(np.abs(host(x) - ref)) / np.max(np.abs(ref)) < 1e-12
    # the full block: orthonormalise, propagate, the norms drift by the remainder only
    import torch
    xf = torch.from_numpy(wl.x0()).cuda()
    q, _ = torch.linalg.qr(xf.T)
    xf = (q.T / np.sqrt(ham.dV)).contiguous()
    ctx.propagate(xf, 0.001, 4, 8)   # dt |H| ~ 0.34: the order-8 remainder is ~2e-10 a step
    nrm = (torch.sum(torch.abs(xf) ** 2, dim=1) * ham.dV).cpu().numpy()
    assert np.max(np.abs(nrm - 1.0)) < 1e-8
