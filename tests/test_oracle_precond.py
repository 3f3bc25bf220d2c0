"""Pins for oracle.precond: the learned preconditioner's network, training and targets."""
import numpy as np
import pytest

from oracle import precond as P
from oracle.grid import Grid, kb_projectors, local_potential
from oracle.hamiltonian import Hamiltonian
from oracle.lobpcg import lobpcg, tpa_precondition
from tests.oracle_refs import hamiltonian_dense
from workloads import draw_nn_weights, draw_x0, small_cell

SHAPE = (5, 4, 6)          # (Nz, Ny, Nx): unequal axes catch transposed indices
N = int(np.prod(SHAPE))


def _rng(seed):
    return np.random.default_rng(seed)


@pytest.mark.parametrize("d", [(1, 0, 0), (0, -1, 0), (0, 0, 1), (-1, 1, -1)])
def test_one_hot_kernel_is_a_periodic_shift(d):
    a = _rng(1).standard_normal((2, 1, N))
    w = np.zeros((27, 1, 1))
    w[P.TAPS.index(d), 0, 0] = 1.0
    out = P.conv(a, w, SHAPE)
    g = a.reshape(2, 1, *SHAPE)
    # out(p) = a(p + d): element (z, y, x) comes from (z + dz, y + dy, x + dx) mod N
    z, y, x = np.meshgrid(*(np.arange(s) for s in SHAPE), indexing="ij")
    ref = g[:, :, (z + d[0]) % SHAPE[0], (y + d[1]) % SHAPE[1], (x + d[2]) % SHAPE[2]]
    assert np.array_equal(out, ref.reshape(2, 1, N))


def test_tap_order():
    assert P.TAPS[0] == (-1, -1, -1) and P.TAPS[13] == (0, 0, 0) and P.TAPS[26] == (1, 1, 1)
    assert P.TAPS[1] == (-1, -1, 0) and P.TAPS[3] == (-1, 0, -1) and P.TAPS[9] == (0, -1, -1)


def test_single_channel_conv_is_circular_convolution_by_fft():
    r = _rng(2)
    a = r.standard_normal(N)
    w = r.standard_normal((27, 1, 1))
    # correlation with w_d = circular convolution with k, k(-d) = w_d
    k = np.zeros(SHAPE)
    for tap, (dz, dy, dx) in enumerate(P.TAPS):
        k[(-dz) % SHAPE[0], (-dy) % SHAPE[1], (-dx) % SHAPE[2]] += w[tap, 0, 0]
    ref = np.real(np.fft.ifftn(np.fft.fftn(a.reshape(SHAPE)) * np.fft.fftn(k))).reshape(-1)
    out = P.conv(a[None, None, :], w, SHAPE)[0, 0]
    assert np.allclose(out, ref, atol=1e-12, rtol=0)


def test_conv_adjoint_dot_product():
    r = _rng(3)
    a = r.standard_normal((3, 4, N))
    g = r.standard_normal((3, 5, N))
    w = r.standard_normal((27, 4, 5))
    lhs = np.sum(P.conv(a, w, SHAPE) * g)
    rhs = np.sum(a * P.conv_adjoint(g, w, SHAPE))
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_weight_grad_is_linear_functional_derivative():
    r = _rng(4)
    a = r.standard_normal((2, 3, N))
    g = r.standard_normal((2, 2, N))
    dw = P.conv_weight_grad(a, g, SHAPE)
    # sum(g * conv(a, w)) is linear in w: its value at a one-hot w is the gradient entry
    for tap, ci, co in [(0, 0, 0), (13, 2, 1), (26, 1, 0), (7, 0, 1)]:
        w = np.zeros((27, 3, 2))
        w[tap, ci, co] = 1.0
        assert abs(np.sum(g * P.conv(a, w, SHAPE)) - dw[tap, ci, co]) < 1e-11


def test_network_is_odd_and_starts_at_zero():
    r = _rng(5)
    hidden = 4
    w = r.standard_normal(P.weight_count(hidden)) * 0.3
    u = r.standard_normal((2, N))
    vhat = P.standardise(r.standard_normal(N))
    assert np.allclose(P.forward(-u, vhat, w, SHAPE, hidden), -P.forward(u, vhat, w, SHAPE, hidden),
                       atol=1e-14, rtol=0)
    w0 = draw_nn_weights(0, hidden)
    assert np.all(P.forward(u, vhat, w0, SHAPE, hidden) == 0.0)
    assert w0.size == P.weight_count(hidden) == 27 * (2 * 4 + 16 + 16 + 4)


def test_standardise():
    v = _rng(6).uniform(-3, 1, N)
    vh = P.standardise(v)
    assert abs(np.mean(vh)) < 1e-14 and abs(np.std(vh) - 1.0) < 1e-13
    assert np.all(P.standardise(np.full(N, 2.5)) == 0.0)


def test_backward_matches_finite_differences():
    r = _rng(7)
    hidden = 3
    w = r.standard_normal(P.weight_count(hidden)) * 0.4
    u = r.standard_normal((2, N))
    b = r.standard_normal((2, N))
    y = r.standard_normal((2, N))
    vhat = P.standardise(r.standard_normal(N))
    L0, g = P.loss_and_grad(u, b, y, vhat, w, SHAPE, hidden)
    h = 1e-6
    for idx in r.choice(w.size, 24, replace=False):
        wp, wm = w.copy(), w.copy()
        wp[idx] += h
        wm[idx] -= h
        fd = (P.loss_and_grad(u, b, y, vhat, wp, SHAPE, hidden)[0]
              - P.loss_and_grad(u, b, y, vhat, wm, SHAPE, hidden)[0]) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-7 * max(1.0, abs(g[idx])), (idx, fd, g[idx])


def test_first_adam_step_is_lr_sign_g():
    g = np.array([3.0, -0.5, 1e-3, -7.0])
    w = np.array([1.0, 2.0, 3.0, 4.0])
    st = P.AdamState(np.zeros(4), np.zeros(4))
    w1 = P.adam_step(w, g, st, lr=0.01)
    # m_hat = g and v_hat = g^2 after one step: the move is lr g / (|g| + eps)
    assert np.allclose(w1, w - 0.01 * g / (np.abs(g) + P.ADAM_EPS), atol=0, rtol=1e-15)
    assert np.allclose(w1 - w, -0.01 * np.sign(g), atol=1e-7, rtol=0)


def test_loss_is_one_minus_cos_squared_and_scale_free():
    r = _rng(11)
    hidden = 3
    w = r.standard_normal(P.weight_count(hidden)) * 0.3
    vhat = P.standardise(r.standard_normal(N))
    u = r.standard_normal((3, N))
    b = r.standard_normal((3, N))
    y = r.standard_normal((3, N))
    L, _ = P.loss_and_grad(u, b, y, vhat, w, SHAPE, hidden)
    pv = b + P.forward(u, vhat, w, SHAPE, hidden)
    cos = [np.dot(pv[i], y[i]) / (np.linalg.norm(pv[i]) * np.linalg.norm(y[i])) for i in range(3)]
    assert abs(L - np.mean([1.0 - c * c for c in cos])) < 1e-14
    # the target's scale and sign do not matter
    L2, _ = P.loss_and_grad(u, b, -3.0 * y, vhat, w, SHAPE, hidden)
    assert abs(L - L2) < 1e-14
    # a prediction along the target has zero loss
    w0 = draw_nn_weights(0, hidden)
    L0, g0 = P.loss_and_grad(u, b, 2.5 * b, vhat, w0, SHAPE, hidden)
    assert abs(L0) < 1e-14


def test_training_reduces_the_loss_on_a_learnable_map():
    # targets made by a fixed network: a network of the same shape can fit them
    r = _rng(8)
    hidden = 3
    w_true = r.standard_normal(P.weight_count(hidden)) * 0.3
    vhat = P.standardise(r.standard_normal(N))
    u = r.standard_normal((8, N))
    b = 0.1 * r.standard_normal((8, N))
    y = b + P.forward(u, vhat, w_true, SHAPE, hidden)
    w0 = draw_nn_weights(3, hidden)
    w, losses = P.train(u, b, y, vhat, w0, SHAPE, steps=60, batch=4, lr=0.02, hidden=hidden)
    assert losses[-1] < 0.3 * losses[0]


def test_minres_dense_indefinite_system():
    r = _rng(9)
    n = 40
    q, _ = np.linalg.qr(r.standard_normal((n, n)) + 1j * r.standard_normal((n, n)))
    lam = np.linspace(-2.0, 3.0, n) + 0.05          # indefinite, no zero eigenvalue
    A = (q * lam) @ q.conj().T
    bvec = r.standard_normal(n) + 1j * r.standard_normal(n)
    x, hist = P.minres(lambda v: A @ v, bvec, rtol=1e-12, maxit=400)
    assert np.allclose(x, np.linalg.solve(A, bvec), atol=1e-9, rtol=0)
    assert all(hist[i + 1] <= hist[i] * (1 + 1e-12) for i in range(len(hist) - 1))
    # MINRES minimises the residual over the Krylov space: after k steps no
    # worse than the Krylov least-squares solution computed densely
    k = 6
    x6, _ = P.minres(lambda v: A @ v, bvec, rtol=0.0, maxit=k)
    K = np.stack([np.linalg.matrix_power(A, j) @ bvec for j in range(k)], axis=1)
    c, *_ = np.linalg.lstsq(A @ K, bvec, rcond=None)
    assert abs(np.linalg.norm(A @ x6 - bvec) - np.linalg.norm(A @ K @ c - bvec)) < 1e-9


def test_correction_target_on_a_dense_6cubed_hamiltonian():
    w = small_cell(N=(6, 6, 6), L=(4.5, 4.5, 4.5), natom=1, nband=4, rcut=2.0)
    g = Grid(L=w.L, N=w.N)
    proj = kb_projectors(g, w.positions, w.rc, w.rcut, w.e_kb())
    ham = Hamiltonian(g, local_potential(g, w.positions, w.Z, w.sigma), proj)
    H = hamiltonian_dense(g.N, g.L, ham.v, proj.B.toarray(), proj.E)
    dV = g.dV
    res = lobpcg(ham, draw_x0(4, 4, g.n), maxit=2)
    X = res.X
    x = X[2]
    e = float(np.real(np.vdot(x, ham.apply(x[None])[0])) * dV)
    r = ham.apply(x[None])[0] - e * x
    # dense: solve the projected system in the orthogonal complement of the block
    Xn = X * np.sqrt(dV)                       # orthonormal rows in the plain metric
    for block in (X, x):                        # the whole block, and x alone
        Bn = np.atleast_2d(block) * np.sqrt(dV)
        t, hist = P.correction_target(ham, block, e, r, rtol=1e-12, maxit=2000)
        Pm = np.eye(g.n) - Bn.T @ Bn.conj()
        A = Pm @ (H - e * np.eye(g.n)) @ Pm
        ref, *_ = np.linalg.lstsq(A, -(Pm @ r), rcond=None)
        ref = Pm @ ref
        assert np.max(np.abs(np.atleast_2d(block).conj() @ t * dV)) < 1e-10 * np.linalg.norm(t)
        assert np.linalg.norm(t - ref) <= 1e-8 * np.linalg.norm(ref)
    assert np.allclose(Xn.conj() @ Xn.T, np.eye(4), atol=1e-12)


def test_training_planes_and_learned_apply():
    w = small_cell(N=(8, 8, 8), L=(5.0, 5.0, 5.0), natom=2, nband=4, rcut=2.0)
    g = Grid(L=w.L, N=w.N)
    proj = kb_projectors(g, w.positions, w.rc, w.rcut, w.e_kb())
    ham = Hamiltonian(g, local_potential(g, w.positions, w.Z, w.sigma), proj)
    res = lobpcg(ham, draw_x0(5, 4, g.n), maxit=3)
    X = res.X
    U, B, Y = P.training_planes(ham, X, lambda R: tpa_precondition(ham, R, X), maxit=300)
    assert U.shape == B.shape == Y.shape == (8, g.n)
    # u has unit complex rms per band: Re and Im planes together
    assert np.allclose(np.sum(U[:4] ** 2 + U[4:] ** 2, axis=1) / g.n, 1.0, atol=1e-12)
    # the target is t rescaled to the TPA norm, pointing along TPA, and a multiple of t
    Bc, Yc = B[:4] + 1j * B[4:], Y[:4] + 1j * Y[4:]
    HXa = ham.apply(X)
    ea = np.real(np.sum(X.conj() * HXa, axis=1)) * g.dV
    Ra = HXa - ea[:, None] * X
    for i in range(4):
        assert abs(np.linalg.norm(Yc[i]) - np.linalg.norm(Bc[i])) <= 1e-12 * np.linalg.norm(Bc[i])
        assert np.real(np.vdot(Yc[i], Bc[i])) >= 0.0
        t, _ = P.correction_target(ham, X, ea[i], Ra[i], maxit=300)
        cosang = abs(np.vdot(t, Yc[i])) / (np.linalg.norm(t) * np.linalg.norm(Yc[i]))
        assert abs(cosang - 1.0) < 1e-12
    # learned_apply with zero weights is the TPA base itself
    HX = ham.apply(X)
    e = np.real(np.sum(X.conj() * HX, axis=1)) * g.dV
    R = HX - e[:, None] * X
    base = tpa_precondition(ham, R, X)
    w0 = draw_nn_weights(1)
    vhat = P.standardise(ham.v)
    assert np.array_equal(P.learned_apply(R, base, vhat, w0, g.shape), base)
    # scale equivariance: r -> 2 r doubles the correction (the network sees r / s)
    wr = _rng(10).standard_normal(P.weight_count()) * 0.2
    a1 = P.learned_apply(R, base, vhat, wr, g.shape) - base
    a2 = P.learned_apply(2 * R, 2 * base, vhat, wr, g.shape) - 2 * base
    assert np.allclose(a2, 2 * a1, atol=1e-12, rtol=0)
