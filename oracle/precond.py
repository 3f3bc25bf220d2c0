"""Oracle: the learned preconditioner (a residual-form 3D convolutional network).

Test infrastructure only (see ``oracle/__init__``).

The learned form replaces the Teter-Payne-Allan preconditioner of the LOBPCG
residuals by TPA plus a small periodic 3D convolutional network trained on
pairs of a residual and the correction that solves the projected Newton
(Jacobi-Davidson) equation, computed by MINRES on smaller cells.  The paper
gives no network; the readings used here and in the CUDA path are:

* Real planes.  At the Gamma point H is real (real V, real projectors), so
  (H - e)^-1 maps the real and imaginary parts of a residual independently.
  The network is a real map applied to Re r and Im r as two samples, and the
  complex preconditioned residual is NN(Re r) + i NN(Im r).
* Scale.  s_b = sqrt(sum_p |r_b(p)|^2 / n); the network sees r_b / s_b and its
  output is multiplied back by s_b (s_b = 0 gives no correction).
* Inputs (2 channels): u and u * vhat, where u is the real plane and
  vhat = (V - mean V) / std V is the standardised effective potential.  Both
  channels are odd in u.
* Layers: four 3x3x3 periodic convolutions without biases, channels
  2 -> C -> C -> C -> 1 (C = 8 by default), tanh between them and none after
  the last.  With odd inputs, no biases and an odd activation the network is
  odd in u, as the exact correction is linear in r.
* Residual form: w_b = TPA(r_b) + s_b NN(r_b / s_b).
* Convolution: out[co](p) = sum_ci sum_d w[tap(d)][ci][co] in[ci](p + d) over
  the 27 offsets d in {-1, 0, 1}^3 with periodic wrap; tap(d) = (dz + 1) 9 +
  (dy + 1) 3 + (dx + 1); grid index (iz Ny + iy) Nx + ix.  Weights are stored
  layer after layer, each as [27][cin][cout] (float32 on the device).
* Training: per sample (a normalised residual plane u, its TPA plane b and the
  target plane y) the loss is 1 - cos^2(b + NN(u), y) = 1 - <w, y>^2 / (<w, w>
  <y, y>) with w = b + NN(u): LOBPCG uses only the span of a preconditioned
  residual, so the loss ignores its scale and sign (a squared-error loss lets the
  network lower it by shrinking w towards zero where y is hard to predict, which
  cancels TPA and stalls LOBPCG); the batch loss is the mean over samples; Adam
  (Kingma and Ba 2015, Algorithm 1: beta1 0.9, beta2 0.999, eps 1e-8) on
  mini-batches taken in cyclic order (batch k = samples k B .. k B + B - 1
  modulo the sample count).
* Target: t_b solves Q (H - e_b) Q t = -Q r_b with Q = I - X X^H the projector
  off the whole block X (t perpendicular to every x_c), by MINRES (Paige and
  Saunders 1975) to a relative residual of 1e-3.  Projecting off x_b alone left
  (H - e_b)^-1 to amplify the components along the other bands of the block
  whose eigenvalues lie near e_b: those dominate the single-band target, the
  network learned them, and LOBPCG, which removes span(X) from W, was left with
  the small rest (a stall at the initial residual level on both judged cells);
  LOBPCG uses only the direction of a preconditioned residual, so the target
  plane is t_b rescaled to the norm of TPA(r_b), with the sign that makes it
  point along TPA(r_b): y = c_b t_b / s_b, c_b = sign(Re<t_b|TPA(r_b)>)
  ||TPA(r_b)|| / ||t_b|| (a target that can shrink, like the least-squares
  multiple of t_b, lets the network learn to cancel TPA where t_b is nearly
  orthogonal to it).
* Acceptance: the learned form is used only where it reaches the LOBPCG
  tolerance in fewer iterations than TPA from the same start; otherwise TPA.

Pins (tests/test_oracle_precond.py): a one-hot kernel is a periodic shift
(np.roll); a single-channel convolution equals the circular convolution
theorem through numpy's FFT; the adjoint satisfies <conv a, g> = <a, conv^T g>;
the network is odd in u; the backward pass matches central finite differences;
the first Adam step moves every weight by lr sign(g); MINRES equals a dense
solve on a small indefinite Hermitian system and on the projected system of a
6^3 Hamiltonian built densely, with monotone residuals.  learned_apply
(tests/test_oracle_pins_closed_form.py): with centre-tap weights the network
is the pointwise map tanh(tanh(tanh(a u + c u vhat))), checked per band with
its rms scale and Re/Im planes; it commutes with positive and imaginary
scalings of (r, base).
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence, Tuple

import numpy as np

HIDDEN = 8
ADAM_BETA1 = 0.9
ADAM_BETA2 = 0.999
ADAM_EPS = 1e-8
MINRES_RTOL = 1e-3

# the 27 offsets d = (dz, dy, dx), tap = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)
TAPS: Tuple[Tuple[int, int, int], ...] = tuple(
    (dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1))


def layer_channels(hidden: int = HIDDEN) -> List[Tuple[int, int]]:
    """(cin, cout) of the four convolutions."""
    return [(2, hidden), (hidden, hidden), (hidden, hidden), (hidden, 1)]


def weight_count(hidden: int = HIDDEN) -> int:
    return sum(27 * ci * co for ci, co in layer_channels(hidden))


def unpack(w: np.ndarray, hidden: int = HIDDEN) -> List[np.ndarray]:
    """Flat weights -> per layer [27][cin][cout] arrays (views)."""
    w = np.asarray(w, dtype=np.float64).reshape(-1)
    if w.size != weight_count(hidden):
        raise ValueError("weight count %d, expected %d" % (w.size, weight_count(hidden)))
    out, off = [], 0
    for ci, co in layer_channels(hidden):
        k = 27 * ci * co
        out.append(w[off:off + k].reshape(27, ci, co))
        off += k
    return out


def _shift(a: np.ndarray, shape: Sequence[int], d: Tuple[int, int, int]) -> np.ndarray:
    """b[..., p] = a[..., p + d] with periodic wrap; a is [..., n], shape (Nz, Ny, Nx)."""
    lead = a.shape[:-1]
    g = a.reshape(lead + tuple(shape))
    nd = len(lead)
    g = np.roll(g, shift=(-d[0], -d[1], -d[2]), axis=(nd, nd + 1, nd + 2))
    return g.reshape(a.shape)


def conv(a: np.ndarray, w: np.ndarray, shape: Sequence[int]) -> np.ndarray:
    """out[s, co, p] = sum_ci sum_d w[tap(d), ci, co] a[s, ci, p + d] (periodic)."""
    S, cin, n = a.shape
    out = np.zeros((S, w.shape[2], n))
    for tap, d in enumerate(TAPS):
        out += np.einsum("scp,co->sop", _shift(a, shape, d), w[tap])
    return out


def conv_adjoint(g: np.ndarray, w: np.ndarray, shape: Sequence[int]) -> np.ndarray:
    """The adjoint of ``conv`` in its input: out[s, ci, p] = sum_co sum_d w[tap(d), ci, co] g[s, co, p - d]."""
    S, cout, n = g.shape
    out = np.zeros((S, w.shape[1], n))
    for tap, d in enumerate(TAPS):
        out += np.einsum("sop,co->scp", _shift(g, shape, (-d[0], -d[1], -d[2])), w[tap])
    return out


def conv_weight_grad(a: np.ndarray, g: np.ndarray, shape: Sequence[int]) -> np.ndarray:
    """d/dw of sum(g * conv(a, w)): dw[tap(d), ci, co] = sum_s sum_p a[s, ci, p + d] g[s, co, p]."""
    dw = np.zeros((27, a.shape[1], g.shape[1]))
    for tap, d in enumerate(TAPS):
        dw[tap] = np.einsum("scp,sop->co", _shift(a, shape, d), g)
    return dw


def standardise(v: np.ndarray) -> np.ndarray:
    """vhat = (V - mean V) / std V (std below 1e-12 -> 1)."""
    v = np.asarray(v, dtype=np.float64).reshape(-1)
    sd = float(np.std(v))
    return (v - np.mean(v)) / (sd if sd > 1e-12 else 1.0)


def forward(u: np.ndarray, vhat: np.ndarray, w: np.ndarray, shape: Sequence[int],
            hidden: int = HIDDEN, cache: bool = False):
    """NN(u) for real planes u [S][n]; returns [S][n] (and the activations)."""
    ws = unpack(w, hidden)
    u = np.atleast_2d(np.asarray(u, dtype=np.float64))
    acts = [np.stack([u, u * vhat[None, :]], axis=1)]
    for l, wl in enumerate(ws):
        z = conv(acts[-1], wl, shape)
        acts.append(np.tanh(z) if l < len(ws) - 1 else z)
    out = acts[-1][:, 0, :]
    return (out, acts) if cache else out


def backward(acts: List[np.ndarray], g_out: np.ndarray, w: np.ndarray, shape: Sequence[int],
             hidden: int = HIDDEN) -> np.ndarray:
    """Gradient of sum(g_out * NN(u)) in the flat weights (reverse mode, layer by layer)."""
    ws = unpack(w, hidden)
    grads = [None] * len(ws)
    g = g_out[:, None, :]
    for l in range(len(ws) - 1, -1, -1):
        grads[l] = conv_weight_grad(acts[l], g, shape)
        if l > 0:
            g = conv_adjoint(g, ws[l], shape) * (1.0 - acts[l] ** 2)   # tanh' = 1 - tanh^2
    return np.concatenate([gl.reshape(-1) for gl in grads])


def loss_and_grad(u, b, y, vhat, w, shape, hidden: int = HIDDEN):
    """loss = mean_s (1 - <p_s, y_s>^2 / (<p_s, p_s> <y_s, y_s>)), p = b + NN(u),
    and its gradient in the weights."""
    out, acts = forward(u, vhat, w, shape, hidden, cache=True)
    p = b + out
    S = p.shape[0]
    al = np.sum(p * y, axis=1)
    be = np.sum(p * p, axis=1)
    ga = np.sum(y * y, axis=1)
    loss = float(np.mean(1.0 - al * al / (be * ga)))
    # d/dp of 1 - al^2 / (be ga): -2 al / (be ga) y + 2 al^2 / (be^2 ga) p
    g = (-2.0 * al / (be * ga))[:, None] * y + (2.0 * al * al / (be * be * ga))[:, None] * p
    return loss, backward(acts, g / S, w, shape, hidden)


@dataclasses.dataclass
class AdamState:
    m: np.ndarray
    v: np.ndarray
    t: int = 0


def adam_step(w: np.ndarray, g: np.ndarray, st: AdamState, lr: float) -> np.ndarray:
    """One Adam update (Kingma and Ba 2015, Algorithm 1)."""
    st.t += 1
    st.m = ADAM_BETA1 * st.m + (1.0 - ADAM_BETA1) * g
    st.v = ADAM_BETA2 * st.v + (1.0 - ADAM_BETA2) * g * g
    mhat = st.m / (1.0 - ADAM_BETA1 ** st.t)
    vhat = st.v / (1.0 - ADAM_BETA2 ** st.t)
    return w - lr * mhat / (np.sqrt(vhat) + ADAM_EPS)


def train(u, b, y, vhat, w0, shape, steps: int, batch: int, lr: float, hidden: int = HIDDEN):
    """Adam on cyclic mini-batches; returns the weights and each step's batch loss."""
    w = np.array(w0, dtype=np.float64)
    st = AdamState(np.zeros_like(w), np.zeros_like(w))
    S = u.shape[0]
    losses = []
    for k in range(steps):
        idx = [(k * batch + j) % S for j in range(batch)]
        L, g = loss_and_grad(u[idx], b[idx], y[idx], vhat, w, shape, hidden)
        losses.append(L)
        w = adam_step(w, g, st, lr)
    return w, np.array(losses)


def rms(r: np.ndarray) -> np.ndarray:
    """s_b = sqrt(sum_p |r_b(p)|^2 / n)."""
    return np.sqrt(np.sum(np.abs(r) ** 2, axis=1) / r.shape[1])


def learned_apply(r: np.ndarray, base: np.ndarray, vhat: np.ndarray, w: np.ndarray,
                  shape: Sequence[int], hidden: int = HIDDEN) -> np.ndarray:
    """w_b = base_b + s_b (NN(Re r_b / s_b) + i NN(Im r_b / s_b))."""
    s = rms(r)
    safe = np.where(s > 0.0, s, 1.0)
    rh = r / safe[:, None]
    o_re = forward(rh.real, vhat, w, shape, hidden)
    o_im = forward(rh.imag, vhat, w, shape, hidden)
    return base + np.where(s > 0.0, s, 0.0)[:, None] * (o_re + 1j * o_im)


def minres(apply_a, b: np.ndarray, rtol: float = MINRES_RTOL, maxit: int = 500):
    """MINRES for a Hermitian (possibly indefinite) operator: x with A x ~ b.

    Paige and Saunders (1975): Lanczos on K(A, b) with the tridiagonal factored
    by Givens rotations; the residual norm |phi| is non-increasing.  Inner
    products are plain sums (the metric's dV cancels).  Returns x and the
    residual-norm history (relative to ||b||).
    """
    b = np.asarray(b, dtype=np.complex128)
    beta1 = float(np.sqrt(np.real(np.vdot(b, b))))
    x = np.zeros_like(b)
    if beta1 == 0.0:
        return x, [0.0]
    v_prev = np.zeros_like(b)
    v = b / beta1
    beta = 0.0              # beta_k (couples v_{k-1} and v_k)
    c_prev, s_prev = 1.0, 0.0   # rotation k-1
    c_pp, s_pp = 1.0, 0.0       # rotation k-2
    d_prev = np.zeros_like(b)   # search directions d_{k-1}, d_{k-2}
    d_pp = np.zeros_like(b)
    phi = beta1
    hist = [1.0]
    for _ in range(maxit):
        p = apply_a(v)
        alpha = float(np.real(np.vdot(v, p)))
        p = p - alpha * v - beta * v_prev
        beta_next = float(np.sqrt(np.real(np.vdot(p, p))))
        # the new column of the tridiagonal: (beta, alpha, beta_next) in rows k-1, k, k+1
        eps_k = s_pp * beta                    # row k-2 after the rotations
        delta_bar = c_pp * beta
        delta_k = c_prev * delta_bar + s_prev * alpha     # row k-1
        gamma_bar = -s_prev * delta_bar + c_prev * alpha  # row k (before its own rotation)
        gamma = float(np.hypot(gamma_bar, beta_next))
        if gamma == 0.0:
            break
        c, s = gamma_bar / gamma, beta_next / gamma
        d = (v - delta_k * d_prev - eps_k * d_pp) / gamma
        tau = c * phi
        phi = -s * phi
        x = x + tau * d
        hist.append(abs(phi) / beta1)
        d_pp, d_prev = d_prev, d
        c_pp, s_pp, c_prev, s_prev = c_prev, s_prev, c, s
        if abs(phi) <= rtol * beta1 or beta_next == 0.0:
            break
        v_prev, v = v, p / beta_next
        beta = beta_next
    return x, hist


def correction_target(ham, X: np.ndarray, eps: float, r: np.ndarray, rtol: float = MINRES_RTOL,
                      maxit: int = 500):
    """t perpendicular to the block X with Q (H - eps) Q t = -Q r, Q = I - X X^H
    (X [m][n] orthonormal in the dV metric; a single band is a block of one)."""
    dV = ham.dV
    X = np.atleast_2d(X)

    def proj(z):
        return z - (X.conj() @ z * dV) @ X

    def op(z):
        pz = proj(z)
        return proj(ham.apply(pz[None, :])[0] - eps * pz)

    t, hist = minres(op, -proj(r), rtol=rtol, maxit=maxit)
    return proj(t), hist


def training_planes(ham, X: np.ndarray, tpa_apply, rtol: float = MINRES_RTOL, maxit: int = 500):
    """Training samples from a block X of approximate orbitals.

    For each band: e = <x|H|x>, r = H x - e x, s = rms(r), t = the projected
    correction, base = TPA(r) (``tpa_apply(R) -> W``),
    c = sign(Re<t|base>) ||base|| / ||t|| (0 where t = 0);
    returns real planes u = r / s, b = base / s, y = c t / s, stacked as
    [Re of every band; Im of every band], each [2 m][n].
    """
    dV = ham.dV
    HX = ham.apply(X)
    e = np.real(np.sum(X.conj() * HX, axis=1)) * dV
    R = HX - e[:, None] * X
    s = rms(R)
    base = tpa_apply(R)
    T = np.zeros_like(R)
    for i in range(X.shape[0]):
        T[i], _ = correction_target(ham, X, e[i], R[i], rtol, maxit)
    tt = np.real(np.sum(T.conj() * T, axis=1))
    bb = np.real(np.sum(base.conj() * base, axis=1))
    tb = np.real(np.sum(T.conj() * base, axis=1))
    sgn = np.where(tb < 0.0, -1.0, 1.0)
    c = np.where(tt > 0.0, sgn * np.sqrt(bb / np.where(tt > 0.0, tt, 1.0)), 0.0)
    safe = np.where(s > 0.0, s, 1.0)[:, None]
    U, B, Y = R / safe, base / safe, c[:, None] * T / safe
    return (np.concatenate([U.real, U.imag]), np.concatenate([B.real, B.imag]),
            np.concatenate([Y.real, Y.imag]))
