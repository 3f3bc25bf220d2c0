"""GPU parity of the learned preconditioner against the FP64 oracle: the
network's forward pass, the loss gradient of the training kernels, Adam
training, the MINRES correction targets, and LOBPCG with the learned form."""
import numpy as np
import pytest

from oracle import precond as OP
from oracle.lobpcg import lobpcg as oracle_lobpcg, tpa_precondition
from tests.gpu_common import R, dev, host, need_gpu, pair, torch
from workloads import bcc_sites, draw_nn_weights, draw_x0, small_cell, Workload

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    need_gpu()


def _weights(seed, scale=0.3):
    """Random weights of every layer (the last one non-zero, so that every layer's gradient is non-zero)."""
    rng = np.random.default_rng(seed)
    w = np.empty(R.NN_WEIGHTS)
    off = 0
    for ci, co in OP.layer_channels():
        k = 27 * ci * co
        w[off:off + k] = rng.standard_normal(k) * scale / np.sqrt(27 * ci) * 3.0
        off += k
    return w.astype(np.float32).astype(np.float64)   # exactly representable in FP32


def _ragged_cell():
    # tiles are 16 x 8 x 4 points: 20 x 12 x 10 leaves a ragged tile on every axis
    return small_cell(N=(20, 12, 10), L=(7.0, 5.0, 4.6), natom=2, nband=3, rcut=2.2)


def test_weight_count():
    assert R.NN_WEIGHTS == OP.weight_count() == 4104


def test_learned_apply_matches_oracle_ragged_tiles():
    wl = _ragged_cell()
    ctx, ham, v = pair(wl)
    rng = np.random.default_rng(1)
    n, nb = ham.grid.n, 3
    r = rng.standard_normal((nb, n)) + 1j * rng.standard_normal((nb, n))
    r[1] *= 1e-3                       # a small residual: the network sees r / s
    base = rng.standard_normal((nb, n)) + 1j * rng.standard_normal((nb, n))
    w = _weights(2)
    ctx.set_precond_weights(w)
    assert np.array_equal(ctx.get_precond_weights(), w.astype(np.float32))
    out = dev(np.zeros((nb, n), dtype=np.complex128))
    ctx.precond_learned(dev(r), dev(base), out)
    got = host(out)
    ref = OP.learned_apply(r, base, OP.standardise(v), w, ham.grid.shape)
    corr = ref - base
    for b in range(nb):
        err = np.max(np.abs(got[b] - ref[b])) / np.max(np.abs(corr[b]))
        assert err < 2e-5, (b, err)
    # in place (w aliases base) gives the same
    wb = dev(base)
    ctx.precond_learned(dev(r), wb, wb)
    assert np.max(np.abs(host(wb) - got)) <= 1e-12 * np.max(np.abs(got))


def test_zero_residual_band_gets_no_correction():
    wl = small_cell(N=(8, 8, 8), L=(5.0, 5.0, 5.0), natom=1, nband=2, rcut=2.0)
    ctx, ham, v = pair(wl)
    n = ham.grid.n
    rng = np.random.default_rng(3)
    r = np.zeros((2, n), dtype=np.complex128)
    r[1] = rng.standard_normal(n)
    base = rng.standard_normal((2, n)) + 0j
    ctx.set_precond_weights(_weights(4))
    out = dev(np.zeros((2, n), dtype=np.complex128))
    ctx.precond_learned(dev(r), dev(base), out)
    got = host(out)
    assert np.array_equal(got[0], base[0])
    assert not np.allclose(got[1], base[1])


def _planes(shape, S, seed):
    rng = np.random.default_rng(seed)
    n = int(np.prod(shape))
    u = rng.standard_normal((S, n))
    b = 0.3 * rng.standard_normal((S, n))
    y = rng.standard_normal((S, n))
    return [a.astype(np.float32) for a in (u, b, y)]


def test_loss_gradient_matches_oracle():
    wl = _ragged_cell()
    ctx, ham, v = pair(wl)
    u, b, y = _planes(ham.grid.shape, 5, 5)
    w = _weights(6)
    ctx.set_precond_weights(w)
    loss, grad = ctx.precond_loss_grad(dev(u), dev(b), dev(y))
    L_ref, g_ref = OP.loss_and_grad(u.astype(np.float64), b.astype(np.float64), y.astype(np.float64),
                                    OP.standardise(v), w, ham.grid.shape)
    assert abs(loss - L_ref) <= 1e-5 * L_ref
    # per layer: the gradient entries against that layer's largest
    off = 0
    for ci, co in OP.layer_channels():
        k = 27 * ci * co
        gl, rl = grad[off:off + k], g_ref[off:off + k]
        assert np.max(np.abs(gl - rl)) <= 2e-4 * np.max(np.abs(rl)), (ci, co)
        off += k


def test_training_matches_oracle_then_reduces_loss():
    wl = small_cell(N=(16, 8, 12), L=(6.0, 4.0, 5.0), natom=2, nband=2, rcut=1.9)
    ctx, ham, v = pair(wl)
    u, b, y = _planes(ham.grid.shape, 6, 7)
    # targets a network of the same shape can reach
    w_true = _weights(8, scale=0.2)
    y = (b.astype(np.float64) + OP.forward(u.astype(np.float64), OP.standardise(v), w_true,
                                           ham.grid.shape)).astype(np.float32)
    w0 = _weights(9, scale=0.1)
    ctx.set_precond_weights(w0)
    steps, batch, lr = 4, 4, 1e-3
    loss = ctx.precond_train(dev(u), dev(b), dev(y), steps, batch, lr)
    w_ref, loss_ref = OP.train(u.astype(np.float64), b.astype(np.float64), y.astype(np.float64),
                               OP.standardise(v), w0, ham.grid.shape, steps, batch, lr)
    assert np.allclose(loss, loss_ref, rtol=1e-4, atol=0)
    dw = ctx.get_precond_weights().astype(np.float64) - w_ref
    # each Adam step moves a weight by at most about lr; FP32 rounding may
    # only perturb that move slightly
    assert np.max(np.abs(dw)) < 0.05 * lr * steps
    ctx.set_precond_weights(w0)
    loss = ctx.precond_train(dev(u), dev(b), dev(y), 60, 3, 1e-2)
    assert loss[-1] < 0.5 * loss[0]


def test_correction_samples_match_oracle():
    wl = small_cell(N=(12, 12, 12), L=(6.0, 6.0, 6.0), natom=2, nband=4, rcut=2.5)
    ctx, ham, v = pair(wl)
    X = oracle_lobpcg(ham, draw_x0(3, 4, ham.grid.n), maxit=3).X
    U, B, Y = OP.training_planes(ham, X, lambda Rr: tpa_precondition(ham, Rr, X), rtol=1e-10, maxit=600)
    n = ham.grid.n
    u, b, y = (dev(np.zeros((8, n), dtype=np.float32)) for _ in range(3))
    it = ctx.precond_samples(dev(X), u, b, y, rtol=1e-10, maxit=600)
    assert np.all(it > 3) and np.all(it < 600)
    for got, ref, name in ((host(u), U, "u"), (host(b), B, "b"), (host(y), Y, "y")):
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert err < 3e-6, (name, err)


def test_lobpcg_with_learned_preconditioner_matches_oracle():
    wl = small_cell(N=(12, 12, 12), L=(6.0, 6.0, 6.0), natom=2, nband=6, rcut=2.5)
    ctx, ham, v = pair(wl)
    w = _weights(11, scale=0.05)
    ctx.set_precond_weights(w)
    x0 = draw_x0(12, 6, ham.grid.n)
    x = dev(x0)
    eig, res, stats, st = ctx.lobpcg(x, ctx.lobpcg_opts(maxit=200, tol=1e-8, precond=R.PRECOND_LEARNED))
    assert st == R.OK and stats.converged
    ref = oracle_lobpcg(ham, x0, maxit=200, tol=1e-8, precond="learned", nn_weights=w)
    assert ref.converged
    assert np.max(np.abs(eig - ref.eig)) < 1e-9
    assert abs(stats.iterations - ref.iterations) <= 2
    # the mixed form with the learned preconditioner converges to the same values
    x = dev(x0)
    eig2, res2, stats2, st2 = ctx.lobpcg(x, ctx.lobpcg_opts(maxit=200, tol=1e-8, precond=R.PRECOND_LEARNED,
                                                            precision=R.MIXED))
    assert st2 == R.OK and stats2.converged
    assert np.max(np.abs(eig2 - ref.eig)) < 1e-9


def test_learned_preconditioner_needs_weights():
    wl = small_cell(N=(8, 8, 8), L=(5.0, 5.0, 5.0), natom=1, nband=2, rcut=2.0)
    ctx, ham, v = pair(wl)
    x = dev(draw_x0(1, 2, ham.grid.n))
    with pytest.raises(R.RsdftError):
        ctx.lobpcg(x, ctx.lobpcg_opts(maxit=3, precond=R.PRECOND_LEARNED))
    with pytest.raises(R.RsdftError):
        ctx.set_precond_weights(np.zeros(10, dtype=np.float32))
    bad = np.zeros(R.NN_WEIGHTS, dtype=np.float32)
    bad[5] = np.nan
    with pytest.raises(R.RsdftError):
        ctx.set_precond_weights(bad)
