"""rsdft_gram_static: the Gram matrix for callers that cannot allocate device
memory (a driver that reserves all of it before its loop and must not call
cudaMalloc inside, since each allocation synchronises the device and breaks
its fixed pool).  The entry point keeps its split-K partial sums in a fixed
device array of the library instead of allocating.  Here it is called through
the C ABI twice in a row, with different inputs, and each result is checked
against the allocating entry point rsdft_gram."""
import numpy as np
import pytest

from tests.gpu_common import R, dev, host, need_gpu, rel_err, torch
from workloads import draw_x0

pytestmark = pytest.mark.gpu


def test_gram_static_matches_gram_on_two_calls_in_a_row():
    need_gpu()
    N = (20, 18, 15)
    ctx = R.Context((5.0, 5.0, 5.0), N, np.zeros(N[0] * N[1] * N[2]))
    n = ctx.n
    # two consecutive calls, the second with other shapes and inputs, so that
    # contents left in the shared array by the first call cannot pass for results
    for call, (na, nb, seed) in enumerate([(67, 130, 1), (33, 20, 7)]):
        a = dev(draw_x0(seed, na, n))
        b = dev(draw_x0(seed + 1, nb, n))
        g_ref = torch.empty((na, nb), dtype=torch.complex128, device="cuda")
        ctx.gram(a, b, g_ref)
        g = torch.full((na, nb), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
        R.gram_static(a, b, g, ctx.dV)
        assert rel_err(host(g), host(g_ref)) < 1e-13, call
    ctx.close()


def test_gram_static_rejects_sizes_beyond_its_scratch():
    need_gpu()
    a = torch.zeros((1, 8), dtype=torch.complex128, device="cuda")
    g = torch.zeros((1, 1), dtype=torch.complex128, device="cuda")
    # 2049 * 1024 > 2^21 entries: rejected before anything is launched
    st = R.lib().rsdft_gram_static(R._ptr(a), 2049, R._ptr(a), 1024, 8, 1.0, R._ptr(g), R._stream())
    assert st == R.E_INVALID
    assert "fixed scratch" in R.lib().rsdft_last_error(None).decode()
