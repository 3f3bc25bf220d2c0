"""Batched form: independent cells of uneven grid, band and atom counts solved
concurrently (rsdft_lobpcg_batched, one stream and host thread per cell in
flight).  Each cell runs the same kernels with the same launch shapes as when
it is solved alone, so the results are bit-identical to the one-cell calls;
one cell is also checked against the FP64 oracle."""
import numpy as np
import pytest

from oracle.lobpcg import lobpcg as oracle_lobpcg
from tests.gpu_common import R, dev, host, need_gpu, pair, torch
from workloads import small_cell

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _cells():
    return [small_cell(N=(12, 12, 12), L=(6.0, 6.0, 6.0), natom=2, nband=6, seed=1),
            small_cell(N=(16, 15, 12), L=(7.0, 6.5, 6.2), natom=3, nband=9, seed=2, rcut=2.4),
            small_cell(N=(20, 20, 20), L=(8.0, 8.0, 8.0), natom=4, nband=12, seed=3, rcut=2.8),
            small_cell(N=(18, 24, 20), L=(7.5, 9.0, 8.0), natom=5, nband=16, seed=4, rcut=2.8)]


@pytest.mark.parametrize("form", ["fp64", "mixed_tc"])
def test_batched_equals_one_cell_calls(form):
    cells = _cells()
    ctxs = [pair(wl)[0] for wl in cells]
    kw = dict(maxit=120, tol=1e-8)
    if form == "mixed_tc":
        kw.update(precision=R.MIXED, tensor_cores=2)
    opts = ctxs[0].lobpcg_opts(**kw)
    solo_eig, solo_x = [], []
    for ctx, wl in zip(ctxs, cells):
        x = dev(wl.x0())
        eig, res, stats, st = ctx.lobpcg(x, opts)
        torch.cuda.synchronize()
        solo_eig.append(eig)
        solo_x.append(host(x))
    xs = [dev(wl.x0()) for wl in cells]
    eigs, ress, stats, st, failed = R.lobpcg_batched(ctxs, xs, opts, max_concurrent=4)
    assert failed == -1
    for c in range(len(cells)):
        assert np.array_equal(eigs[c], solo_eig[c]), c
        assert np.array_equal(host(xs[c]), solo_x[c]), c
        assert stats[c].converged == 1


def test_batched_large_subspaces_equal_one_cell_calls():
    """Subspace 432 on small grids: the multi-CTA dense kernels (Cholesky panels,
    cooperative tridiagonalisation) of four cells run while other cells occupy
    SMs; the results must still equal the one-cell calls bit for bit."""
    cells = [small_cell(N=(32, 32, 32), L=(12.0, 12.0, 12.0), natom=8, nband=144, seed=10 + c, rcut=3.0)
             for c in range(4)]
    ctxs = [pair(wl)[0] for wl in cells]
    opts = ctxs[0].lobpcg_opts(maxit=8, tol=0.0)
    solo = []
    for ctx, wl in zip(ctxs, cells):
        x = dev(wl.x0())
        eig, res, stats, st = ctx.lobpcg(x, opts)
        solo.append(eig)
    for rep in range(2):
        xs = [dev(wl.x0()) for wl in cells]
        eigs, ress, stats, st, failed = R.lobpcg_batched(ctxs, xs, opts, max_concurrent=4)
        for c in range(4):
            assert np.array_equal(eigs[c], solo[c]), (rep, c)


def test_batched_cell_matches_oracle():
    wl = _cells()[1]
    ctx, ham, _ = pair(wl)
    x0 = wl.x0()
    xs = [dev(x0)]
    eigs, ress, stats, st, failed = R.lobpcg_batched([ctx], xs, ctx.lobpcg_opts(maxit=200, tol=1e-9))
    o = oracle_lobpcg(ham, x0, maxit=200, tol=1e-9)
    assert np.max(np.abs(eigs[0] - o.eig)) < 1e-9


def test_batched_rejects_bad_arguments():
    wl = _cells()[0]
    ctx = pair(wl)[0]
    with pytest.raises(R.RsdftError):
        R.lobpcg_batched([ctx], [torch.zeros((1000, ctx.n), dtype=torch.complex128, device="cuda")],
                         ctx.lobpcg_opts())
