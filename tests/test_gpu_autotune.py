"""The autotuner (rsdft_set_autotune): the first call of each shape times the
tile candidates and keeps the fastest.  Candidates differ only in summation
order, so a tuned solve still meets the FP64 bars against the oracle, and a
second solve on the same context (choices reused) gives the same result as the
first, bit for bit."""
import numpy as np
import pytest

from oracle.lobpcg import lobpcg as oracle_lobpcg
from tests.gpu_common import PREFIX8, R, dev, host, need_gpu, pair, subspace_distance
from workloads import diamond8_24

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("form", ["fp64", "mixed_tc"])
def test_autotuned_lobpcg_meets_fp64_bars_and_repeats(form):
    wl = diamond8_24()
    ctx, ham, _ = pair(wl)
    ctx.set_autotune(True)
    kw = dict(maxit=200, tol=1e-9)
    if form == "mixed_tc":
        kw.update(precision=R.MIXED, tensor_cores=2)
    x0 = wl.x0(24)
    x1 = dev(x0)
    eig1, res1, st1, _ = ctx.lobpcg(x1, ctx.lobpcg_opts(**kw))      # tunes
    x2 = dev(x0)
    eig2, res2, st2, _ = ctx.lobpcg(x2, ctx.lobpcg_opts(**kw))      # reuses the choices
    o = oracle_lobpcg(ham, x0, maxit=200, tol=1e-9)
    assert st1.converged and st2.converged
    assert np.max(np.abs(eig2 - o.eig)) < 1e-9
    assert subspace_distance(host(x2)[:PREFIX8], o.X[:PREFIX8], ham.dV) < 1e-7
    assert np.array_equal(eig1, eig2) or np.max(np.abs(eig1 - eig2)) < 1e-12
