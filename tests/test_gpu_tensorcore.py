"""Tensor-core Gram matrix of the mixed form (split-BF16 x3 on tcgen05, FP32
accumulation in TMEM, FP64 sums of the K-split partials) against the FP64
inner products of the same FP32 inputs.

Error model: x = hi + lo with hi = bf16(x), lo = bf16(x - hi); lo keeps 8 of
the 16 bits left after hi, so each product carries a relative error of about
2^-16 = 1.5e-5 and the dropped lo*lo' term is ~2^-32.  For the random blocks
here the entry errors stay below 5e-5 of max |G|."""
import numpy as np
import pytest

from oracle.hamiltonian import inner
from tests.gpu_common import R, dev, host, need_gpu, rel_err, torch
from workloads import draw_x0

pytestmark = pytest.mark.gpu

BF16X3_TOL = 5e-5


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


@pytest.mark.parametrize("N,na,nb", [((20, 18, 15), 1, 1), ((20, 18, 15), 67, 130),
                                     ((24, 24, 24), 144, 48), ((16, 16, 16), 200, 200)])
def test_gram_bf16x3_matches_fp64(N, na, nb):
    ctx = R.Context((5.0, 5.0, 5.0), N, np.zeros(N[0] * N[1] * N[2]))
    a = draw_x0(1, na, ctx.n).astype(np.complex64)
    b = draw_x0(2, nb, ctx.n).astype(np.complex64)
    g = torch.full((na, nb), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
    ctx.gram_bf16x3(dev(a), dev(b), g)
    ref = inner(a.astype(np.complex128), b.astype(np.complex128), ctx.dV)
    err = rel_err(host(g), ref)
    print(f"split-BF16 Gram {na}x{nb} on {ctx.n} points: max error / max |G| = {err:.2e}")
    assert err < BF16X3_TOL


@pytest.mark.parametrize("N,k", [((24, 24, 24), 16), ((24, 24, 24), 144), ((20, 18, 15), 200),
                                 ((24, 24, 24), 288), ((24, 24, 24), 432), ((64, 64, 64), 144)])
def test_gram_sh_bf16x3_hermitian_pair(N, k):
    """G_S = <Y|Y> and G_H = <Y|HY> from one GEMM against [Y; HY] (the
    Rayleigh-Ritz pair; several row tiles, many K splits on the 64^3 grid)."""
    ctx = R.Context((5.0, 5.0, 5.0), N, np.zeros(N[0] * N[1] * N[2]))
    y = draw_x0(5, k, ctx.n).astype(np.complex64)
    # a Hermitian operator on the grid (a real potential), so that <Y|HY> is Hermitian
    vr = np.random.default_rng(6).uniform(-2.0, 1.0, ctx.n)
    hy = (vr[None, :] * y.astype(np.complex128)).astype(np.complex64)
    gs = torch.full((k, k), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
    gh = torch.full((k, k), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
    ctx.gram_sh_bf16x3(dev(y), dev(hy), gs, gh)
    Y64, HY64 = y.astype(np.complex128), hy.astype(np.complex128)
    rs, rh = inner(Y64, Y64, ctx.dV), inner(Y64, HY64, ctx.dV)
    rh = 0.5 * (rh + rh.conj().T)
    GS, GH = host(gs), host(gh)
    es, eh = rel_err(GS, rs), rel_err(GH, rh)
    print(f"split-BF16 Hermitian pair k={k} on {ctx.n} points: {es:.2e} (S), {eh:.2e} (H)")
    assert es < BF16X3_TOL and eh < BF16X3_TOL
    assert np.array_equal(GS, GS.conj().T) and np.array_equal(GH, GH.conj().T)


def test_gram_bf16x3_two_calls_in_a_row_and_hermitian_block():
    N = (24, 24, 24)
    ctx = R.Context((5.0, 5.0, 5.0), N, np.zeros(N[0] * N[1] * N[2]))
    y = draw_x0(3, 96, ctx.n).astype(np.complex64)
    ref = inner(y.astype(np.complex128), y.astype(np.complex128), ctx.dV)
    for _ in range(2):
        g = torch.empty((96, 96), dtype=torch.complex128, device="cuda")
        ctx.gram_bf16x3(dev(y), dev(y), g)
        G = host(g)
        assert rel_err(G, ref) < BF16X3_TOL
        assert np.max(np.abs(G - G.conj().T)) < BF16X3_TOL * np.max(np.abs(ref))


def test_mixed_lobpcg_with_tensor_core_grams_meets_fp64_bars():
    """Mixed form with the Gram matrices on the tensor cores: after the FP64
    refinement the eigenvalues meet the FP64 bar against the oracle."""
    from oracle.lobpcg import lobpcg as oracle_lobpcg
    from tests.gpu_common import PREFIX8, pair, subspace_distance
    from workloads import diamond8_24
    wl = diamond8_24()
    ctx, ham, _ = pair(wl)
    x0 = wl.x0(24)
    x = dev(x0)
    eig, res, stats, st = ctx.lobpcg(x, ctx.lobpcg_opts(maxit=200, tol=1e-9, precision=R.MIXED,
                                                        tensor_cores=1))
    o = oracle_lobpcg(ham, x0, maxit=200, tol=1e-9)
    print(f"tensor-core mixed LOBPCG: {stats.iterations_mixed} FP32 + "
          f"{stats.iterations - stats.iterations_mixed} FP64 iterations")
    assert stats.converged and stats.iterations_mixed > 0
    assert np.max(np.abs(eig - o.eig)) < 1e-9
    assert subspace_distance(host(x)[:PREFIX8], o.X[:PREFIX8], ham.dV) < 1e-7


def _rot_ref(y, c, m):
    """FP64 reference of the split rotation on the same complex64 inputs."""
    Y = y.astype(np.complex128)
    out1 = c[m:].T @ Y[m:]
    out0 = c[:m].T @ Y[:m] + out1
    scale = np.abs(c).T @ np.abs(Y)          # sum_j |C_jb| |Y_j(r)| per output entry
    return out0, out1, scale


# Split-BF16 x3 error model for one output entry: each factor keeps ~2^-18 of
# relative error after the hi/lo split, the dropped lo*lo' term is ~2^-18, and
# the FP32 accumulation over k <= 432 terms adds at most ~k 2^-24; 5e-5 of
# sum_j |C_jb||Y_j(r)| bounds the sum.
ROT_TOL = 5e-5


@pytest.mark.parametrize("N,k,m", [((24, 24, 24), 48, 16), ((20, 18, 15), 11, 5),
                                   ((24, 24, 24), 432, 144), ((16, 16, 16), 300, 144),
                                   ((20, 18, 15), 100, 33),
                                   # more bands than one accumulator pair: band groups
                                   ((16, 16, 16), 900, 480), ((20, 18, 15), 500, 250)])
def test_rotate_bf16x3_matches_fp64(N, k, m):
    ctx = R.Context((5.0, 5.0, 5.0), N, np.zeros(N[0] * N[1] * N[2]))
    y = draw_x0(11, k, ctx.n).astype(np.complex64)
    rng = np.random.default_rng(12)
    c = (rng.standard_normal((k, m)) + 1j * rng.standard_normal((k, m))) / np.sqrt(k)
    out0 = torch.full((m, ctx.n), complex(np.nan, np.nan), dtype=torch.complex64, device="cuda")
    out1 = torch.full_like(out0, complex(np.nan, np.nan))
    ctx.rotate_bf16x3(dev(y), dev(c), out0, out1)
    r0, r1, scale = _rot_ref(y, c, m)
    e0 = np.max(np.abs(host(out0) - r0) / scale)
    e1 = np.max(np.abs(host(out1) - r1) / np.maximum(np.abs(c[m:]).T @ np.abs(y[m:]), 1e-30))
    print(f"split-BF16 rotation k={k} m={m} n={ctx.n}: rel errors {e0:.2e} (X), {e1:.2e} (P)")
    assert np.isfinite(host(out0)).all() and np.isfinite(host(out1)).all()
    assert e0 < ROT_TOL and e1 < ROT_TOL


def test_rotate_bf16x3_rejects_unsupported_shapes():
    N = (12, 12, 12)
    ctx = R.Context((5.0, 5.0, 5.0), N, np.zeros(N[0] * N[1] * N[2]))
    y = torch.zeros((300, ctx.n), dtype=torch.complex64, device="cuda")
    for k, m in [(256, 256), (250, 300)]:   # k must exceed m (out1 is the new P)
        c = torch.zeros((k, m), dtype=torch.complex128, device="cuda")
        o = torch.zeros((m, ctx.n), dtype=torch.complex64, device="cuda")
        with pytest.raises(R.RsdftError):
            ctx.rotate_bf16x3(y[:k], c, o, o.clone())


def test_mixed_lobpcg_with_tensor_core_rotations_meets_fp64_bars():
    """tensor_cores = 2: Grams and Ritz rotations of the FP32 phase on tcgen05;
    after the FP64 refinement the FP64 bars hold."""
    from oracle.lobpcg import lobpcg as oracle_lobpcg
    from tests.gpu_common import PREFIX8, pair, subspace_distance
    from workloads import diamond8_24
    wl = diamond8_24()
    ctx, ham, _ = pair(wl)
    x0 = wl.x0(24)
    x = dev(x0)
    eig, res, stats, st = ctx.lobpcg(x, ctx.lobpcg_opts(maxit=200, tol=1e-9, precision=R.MIXED,
                                                        tensor_cores=2))
    o = oracle_lobpcg(ham, x0, maxit=200, tol=1e-9)
    print(f"tensor-core (Gram + rotation) mixed LOBPCG: {stats.iterations_mixed} FP32 + "
          f"{stats.iterations - stats.iterations_mixed} FP64 iterations")
    assert stats.converged and stats.iterations_mixed > 0
    assert np.max(np.abs(eig - o.eig)) < 1e-9
    assert subspace_distance(host(x)[:PREFIX8], o.X[:PREFIX8], ham.dV) < 1e-7
