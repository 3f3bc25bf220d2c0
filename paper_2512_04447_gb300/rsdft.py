"""Python binding of the rsdft C ABI (include/rsdft.h): argument marshalling only.

Every computation runs in the CUDA library ``librsdft.so`` built in-tree by
``paper_2512_04447_gb300.build``.  Device arrays are torch CUDA tensors (their
data pointers are passed through); host arrays are numpy arrays.  The work is
issued on torch's current CUDA stream.  If the library is missing this module
raises; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librsdft.so")
HEADER = os.path.join(HERE, "..", "include", "rsdft.h")

OK, E_INVALID, E_GRID_NOT_5SMOOTH, E_OOM, E_CUDA, E_NOT_SPD, E_NUMERIC, E_TIMEOUT, \
    E_NOT_CONVERGED = range(9)
FP64, MIXED = 0, 1
PRECOND_NONE, PRECOND_TPA, PRECOND_LEARNED = 0, 1, 2
REFINE_FP64, REFINE_FP32_CORRECTIONS = 0, 1
DENSE_AUTO, DENSE_FP64, DENSE_DF = 0, 1, 2
XC_LDA, XC_PBE = 0, 1
NN_HIDDEN = 8
NN_WEIGHTS = 27 * (2 * NN_HIDDEN + 2 * NN_HIDDEN * NN_HIDDEN + NN_HIDDEN)
STATUS_NAMES = ["OK", "E_INVALID", "E_GRID_NOT_5SMOOTH", "E_OOM", "E_CUDA", "E_NOT_SPD",
                "E_NUMERIC", "E_TIMEOUT", "E_NOT_CONVERGED"]


class RsdftError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 9 else status}: {message}")
        self.status = status


class Cell(C.Structure):
    _fields_ = [("a", (C.c_double * 3) * 3)]


class Grid(C.Structure):
    _fields_ = [("n", C.c_int * 3)]


class Projectors(C.Structure):
    _fields_ = [("natom", C.c_int), ("pos", C.c_void_p), ("nproj", C.c_int), ("rc", C.c_double),
                ("rcut", C.c_double), ("e_kb", C.c_void_p)]


class LobpcgOpts(C.Structure):
    _fields_ = [("maxit", C.c_int), ("tol", C.c_double), ("nconv", C.c_int), ("precond", C.c_int),
                ("precision", C.c_int), ("lock_tol", C.c_double), ("pivot_tol", C.c_double),
                ("switch_tol", C.c_double), ("tensor_cores", C.c_int), ("learned_iters", C.c_int),
                ("refine", C.c_int), ("dense", C.c_int)]


class LobpcgStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("iterations_mixed", C.c_int), ("converged", C.c_int),
                ("dropped", C.c_int), ("coop_fallbacks", C.c_int), ("coop_last_error", C.c_int),
                ("ms_hpsi", C.c_double), ("ms_precond", C.c_double), ("ms_gram", C.c_double),
                ("ms_dense", C.c_double), ("ms_rotate", C.c_double), ("ms_other", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ScfOpts(C.Structure):
    _fields_ = [("n_electrons", C.c_double), ("kT", C.c_double), ("beta", C.c_double),
                ("depth", C.c_int), ("k_lobpcg", C.c_int), ("first_maxit", C.c_int),
                ("tol", C.c_double), ("precond", C.c_int), ("precision", C.c_int),
                ("tensor_cores", C.c_int), ("later_tol", C.c_double), ("xc", C.c_int)]


class ScfOut(C.Structure):
    _fields_ = [("e_tot", C.c_double), ("free_energy", C.c_double), ("e_band", C.c_double),
                ("e_h", C.c_double), ("e_xc", C.c_double), ("e_vxc", C.c_double),
                ("mu", C.c_double), ("entropy", C.c_double), ("drho", C.c_double),
                ("lobpcg_iterations", C.c_int), ("lobpcg_iterations_mixed", C.c_int),
                ("step", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib: Optional[C.CDLL] = None
vp, ip, dp = C.c_void_p, C.c_int, C.c_double

_PROTOS = {
    "rsdft_create": (ip, [C.POINTER(Cell), C.POINTER(Grid), vp, C.POINTER(Projectors), C.POINTER(vp)]),
    "rsdft_destroy": (None, [vp]),
    "rsdft_last_error": (C.c_char_p, [vp]),
    "rsdft_gaussian_vloc": (ip, [C.POINTER(Cell), C.POINTER(Grid), ip, vp, dp, dp, vp]),
    "rsdft_set_potential": (ip, [vp, vp, ip, vp]),
    "rsdft_projector_entries": (C.c_longlong, [vp]),
    "rsdft_apply_h": (ip, [vp, vp, vp, ip, ip, vp]),
    "rsdft_project": (ip, [vp, vp, vp, ip, vp]),
    "rsdft_precondition_tpa": (ip, [vp, vp, vp, vp, ip, vp]),
    "rsdft_gram": (ip, [vp, vp, ip, vp, ip, vp, vp]),
    "rsdft_gram_static": (ip, [vp, ip, vp, ip, C.c_longlong, dp, vp, vp]),
    "rsdft_gram_bf16x3": (ip, [vp, vp, ip, vp, ip, vp, vp]),
    "rsdft_gram_sh_bf16x3": (ip, [vp, vp, vp, ip, vp, vp, vp]),
    "rsdft_rotate_bf16x3": (ip, [vp, vp, ip, vp, ip, vp, vp, vp]),
    "rsdft_rotate": (ip, [vp, vp, ip, vp, ip, vp, ip, vp, vp]),
    "rsdft_rayleigh_ritz": (ip, [vp, vp, vp, ip, ip, dp, vp, vp, vp, vp]),
    "rsdft_eigh": (ip, [vp, vp, ip, ip, vp, vp, vp]),
    "rsdft_set_dense": (ip, [vp, ip]),
    "rsdft_lobpcg_default_opts": (None, [C.POINTER(LobpcgOpts)]),
    "rsdft_lobpcg": (ip, [vp, vp, ip, C.POINTER(LobpcgOpts), vp, vp, C.POINTER(LobpcgStats), vp]),
    "rsdft_set_autotune": (ip, [vp, ip]),
    "rsdft_lobpcg_batched": (ip, [vp, ip, vp, vp, C.POINTER(LobpcgOpts), vp, vp, C.POINTER(LobpcgStats), ip,
                                  C.POINTER(C.c_int)]),
    "rsdft_scf_default_opts": (None, [C.POINTER(ScfOpts)]),
    "rsdft_scf_init": (ip, [vp, ip, C.POINTER(ScfOpts), vp]),
    "rsdft_scf_step": (ip, [vp, vp, ip, C.POINTER(ScfOpts), C.POINTER(ScfOut), vp, vp, vp]),
    "rsdft_density": (ip, [vp, vp, vp, ip, vp, vp]),
    "rsdft_hartree": (ip, [vp, vp, vp, vp]),
    "rsdft_lda": (ip, [vp, vp, vp, vp, vp]),
    "rsdft_xc_pbe": (ip, [vp, vp, vp, vp, vp]),
    "rsdft_occupations": (ip, [vp, vp, ip, dp, dp, vp, vp, vp, vp]),
    "rsdft_scf_density": (vp, [vp]),
    "rsdft_propagate": (ip, [vp, vp, ip, dp, ip, ip, vp]),
    "rsdft_apply_h_real": (ip, [vp, vp, vp, ip, vp]),
    "rsdft_gram_real": (ip, [vp, vp, ip, vp, ip, vp, vp]),
    "rsdft_rotate_real": (ip, [vp, vp, ip, vp, ip, vp, ip, vp, vp]),
    "rsdft_lobpcg_real": (ip, [vp, vp, ip, C.POINTER(LobpcgOpts), vp, vp, C.POINTER(LobpcgStats), vp]),
    "rsdft_scf_step_real": (ip, [vp, vp, ip, C.POINTER(ScfOpts), C.POINTER(ScfOut), vp, vp, vp]),
    "rsdft_profile_enable": (ip, [vp, ip]),
    "rsdft_profile_read": (ip, [vp, ip, vp, vp, vp, vp]),
    "rsdft_launch_count": (C.c_longlong, [vp]),
    "rsdft_set_precond_weights": (ip, [vp, vp, C.c_longlong]),
    "rsdft_get_precond_weights": (ip, [vp, vp, C.c_longlong]),
    "rsdft_precond_learned": (ip, [vp, vp, vp, vp, ip, vp]),
    "rsdft_precond_samples": (ip, [vp, vp, ip, dp, ip, vp, vp, vp, vp, vp]),
    "rsdft_precond_loss_grad": (ip, [vp, vp, vp, vp, ip, vp, vp, vp]),
    "rsdft_precond_train": (ip, [vp, vp, vp, vp, C.c_longlong, ip, ip, C.c_float, vp, vp]),
}

K_GRAM, K_ROTATE, K_FFT_XY_FWD, K_FFT_Z, K_FFT_XY_INV, K_PROJECT, K_DENSE, K_GRAM_TC = range(8)
KERNEL_NAMES = ["gram", "rotate", "fft_xy_fwd", "fft_z", "fft_xy_inv", "project", "dense", "gram_tc",
                "rotate_tc", "chol", "trsm", "tridiag", "trieig", "backtransform"]


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2512_04447_gb300.build")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _PROTOS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def header_symbols():
    """Names of the functions declared in include/rsdft.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rsdft_\w+)\s*\(", text)))


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t) -> C.c_void_p:
    if t is None:
        return C.c_void_p(0)
    if isinstance(t, np.ndarray):
        return C.c_void_p(t.ctypes.data)
    return C.c_void_p(t.data_ptr())


def _cell(L) -> Cell:
    c = Cell()
    for a in range(3):
        for b in range(3):
            c.a[a][b] = float(L[a]) if a == b else 0.0
    return c


def _grid(N) -> Grid:
    g = Grid()
    for a in range(3):
        g.n[a] = int(N[a])
    return g


def gaussian_vloc(L, N, positions, Z: float, sigma: float) -> np.ndarray:
    """rsdft_gaussian_vloc: host-only input builder."""
    pos = np.ascontiguousarray(positions, dtype=np.float64)
    out = np.zeros(int(N[0]) * int(N[1]) * int(N[2]))
    st = lib().rsdft_gaussian_vloc(C.byref(_cell(L)), C.byref(_grid(N)), pos.shape[0], _ptr(pos),
                                   float(Z), float(sigma), _ptr(out))
    if st != OK:
        raise RsdftError(st, lib().rsdft_last_error(None).decode())
    return out


def gram_static(a, b, g, scale: float) -> None:
    """rsdft_gram_static: g = scale * conj(a) @ b.T with no device allocation
    (the library's fixed scratch array holds the partial sums)."""
    st = lib().rsdft_gram_static(_ptr(a), a.shape[0], _ptr(b), b.shape[0], a.shape[1], float(scale),
                                 _ptr(g), _stream())
    if st != OK:
        raise RsdftError(st, lib().rsdft_last_error(None).decode())


def lobpcg_batched(ctxs, xs, opts, max_concurrent: int = 0):
    """rsdft_lobpcg_batched: LOBPCG on independent cells concurrently (one stream
    and host thread per cell in flight).  ctxs: Context per cell; xs: device
    [nband][n] complex128 blocks (in/out); opts: one LobpcgOpts for all cells or
    a list with one per cell.  Returns (eigs, resnorms, stats, status,
    failed_cell); RSDFT_E_NOT_CONVERGED from a cell is returned, not raised."""
    n = len(ctxs)
    assert len(xs) == n
    per = list(opts) if isinstance(opts, (list, tuple)) else [opts] * n
    assert len(per) == n
    oarr = (LobpcgOpts * n)(*per)
    h = (C.c_void_p * n)(*[c._h for c in ctxs])
    xp = (C.c_void_p * n)(*[_ptr(x) for x in xs])
    nb = (C.c_int * n)(*[int(x.shape[0]) for x in xs])
    eigs = [np.zeros(int(x.shape[0])) for x in xs]
    ress = [np.zeros(int(x.shape[0])) for x in xs]
    ep = (C.c_void_p * n)(*[_ptr(e) for e in eigs])
    rp = (C.c_void_p * n)(*[_ptr(r) for r in ress])
    stats = (LobpcgStats * n)()
    failed = C.c_int(-1)
    st = lib().rsdft_lobpcg_batched(h, n, xp, nb, oarr, ep, rp, stats, int(max_concurrent), C.byref(failed))
    if st not in (OK, E_NOT_CONVERGED):
        ctx = ctxs[failed.value] if 0 <= failed.value < n else None
        msg = lib().rsdft_last_error(ctx._h if ctx else None).decode()
        raise RsdftError(st, f"cell {failed.value}: {msg}")
    return eigs, ress, list(stats), st, failed.value


class Context:
    """rsdft_create / rsdft_destroy and the calls bound to a context."""

    def __init__(self, L, N, v_loc: np.ndarray, positions=None, rc=1.0, rcut=3.0, e_kb=None,
                 nproj=4):
        self._h = C.c_void_p(0)
        self.N = tuple(int(x) for x in N)
        self.L = tuple(float(x) for x in L)
        self.n = self.N[0] * self.N[1] * self.N[2]
        self.dV = self.L[0] * self.L[1] * self.L[2] / self.n
        v = np.ascontiguousarray(v_loc, dtype=np.float64)
        pj = None
        self._keep = [v]
        if positions is not None:
            pos = np.ascontiguousarray(positions, dtype=np.float64)
            ekb = np.ascontiguousarray(e_kb, dtype=np.float64)
            self._keep += [pos, ekb]
            pj = Projectors(pos.shape[0], _ptr(pos), nproj, rc, rcut, _ptr(ekb))
            self.natom, self.nproj = pos.shape[0], nproj
        else:
            self.natom, self.nproj = 0, nproj
        st = lib().rsdft_create(C.byref(_cell(L)), C.byref(_grid(N)), _ptr(v),
                                C.byref(pj) if pj is not None else None, C.byref(self._h))
        if st != OK:
            raise RsdftError(st, lib().rsdft_last_error(None).decode())

    def close(self):
        if self._h:
            lib().rsdft_destroy(self._h)
            self._h = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, allow=()):
        if st != OK and st not in allow:
            raise RsdftError(st, lib().rsdft_last_error(self._h).decode())
        return st

    # ---- profiling
    def profile_enable(self, on=True):
        self._check(lib().rsdft_profile_enable(self._h, 1 if on else 0))

    def profile_read(self, kid):
        ms, fl, by = C.c_double(0), C.c_double(0), C.c_double(0)
        cnt = C.c_longlong(0)
        self._check(lib().rsdft_profile_read(self._h, kid, C.byref(ms), C.byref(cnt), C.byref(fl),
                                             C.byref(by)))
        return {"ms": ms.value, "launches": cnt.value, "flops": fl.value, "bytes": by.value}

    def launch_count(self) -> int:
        return int(lib().rsdft_launch_count(self._h))

    # ---- operators
    def set_potential(self, v):
        on_dev = not isinstance(v, np.ndarray)
        if not on_dev:
            v = np.ascontiguousarray(v, dtype=np.float64)
        self._check(lib().rsdft_set_potential(self._h, _ptr(v), 1 if on_dev else 0, _stream()))

    def projector_entries(self) -> int:
        return int(lib().rsdft_projector_entries(self._h))

    def apply_h(self, psi, hpsi, precision=FP64):
        self._check(lib().rsdft_apply_h(self._h, _ptr(psi), _ptr(hpsi), psi.shape[0], precision,
                                        _stream()))

    def project(self, psi, p):
        self._check(lib().rsdft_project(self._h, _ptr(psi), _ptr(p), psi.shape[0], _stream()))

    def precondition_tpa(self, r, w, tkin):
        self._check(lib().rsdft_precondition_tpa(self._h, _ptr(r), _ptr(w), _ptr(tkin), r.shape[0],
                                                 _stream()))

    # ---- learned preconditioner
    def set_precond_weights(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        self._check(lib().rsdft_set_precond_weights(self._h, _ptr(w), w.size))

    def get_precond_weights(self) -> np.ndarray:
        w = np.zeros(NN_WEIGHTS, dtype=np.float32)
        self._check(lib().rsdft_get_precond_weights(self._h, _ptr(w), w.size))
        return w

    def precond_learned(self, r, base, w):
        self._check(lib().rsdft_precond_learned(self._h, _ptr(r), _ptr(base), _ptr(w), r.shape[0], _stream()))

    def precond_samples(self, x, u, b, y, rtol=1e-3, maxit=500) -> np.ndarray:
        """Training planes u, b, y ([2 nband][n] float32 device tensors); returns MINRES iterations."""
        it = np.zeros(x.shape[0], dtype=np.int32)
        self._check(lib().rsdft_precond_samples(self._h, _ptr(x), x.shape[0], rtol, maxit, _ptr(u), _ptr(b),
                                                _ptr(y), _ptr(it), _stream()))
        return it

    def precond_loss_grad(self, u, b, y):
        loss = np.zeros(1, dtype=np.float32)
        grad = np.zeros(NN_WEIGHTS, dtype=np.float32)
        self._check(lib().rsdft_precond_loss_grad(self._h, _ptr(u), _ptr(b), _ptr(y), u.shape[0], _ptr(loss),
                                                  _ptr(grad), _stream()))
        return float(loss[0]), grad

    def precond_train(self, u, b, y, steps, batch, lr) -> np.ndarray:
        loss = np.zeros(steps, dtype=np.float32)
        self._check(lib().rsdft_precond_train(self._h, _ptr(u), _ptr(b), _ptr(y), u.shape[0], steps, batch,
                                              lr, _ptr(loss), _stream()))
        return loss

    # ---- subspace pieces
    def gram(self, a, b, g):
        self._check(lib().rsdft_gram(self._h, _ptr(a), a.shape[0], _ptr(b), b.shape[0], _ptr(g),
                                     _stream()))

    def set_autotune(self, on: bool = True):
        self._check(lib().rsdft_set_autotune(self._h, 1 if on else 0))

    def set_dense(self, mode: int):
        self._check(lib().rsdft_set_dense(self._h, int(mode)))

    def gram_bf16x3(self, a, b, g):
        self._check(lib().rsdft_gram_bf16x3(self._h, _ptr(a), a.shape[0], _ptr(b), b.shape[0],
                                            _ptr(g), _stream()))

    def gram_sh_bf16x3(self, y, hy, gs, gh):
        self._check(lib().rsdft_gram_sh_bf16x3(self._h, _ptr(y), _ptr(hy), y.shape[0], _ptr(gs), _ptr(gh),
                                               _stream()))

    def rotate_bf16x3(self, y, c, out0, out1):
        """rsdft_rotate_bf16x3: out1 = C[m:]^T Y[m:], out0 = C[:m]^T Y[:m] + out1."""
        self._check(lib().rsdft_rotate_bf16x3(self._h, _ptr(y), y.shape[0], _ptr(c), c.shape[1],
                                              _ptr(out0), _ptr(out1), _stream()))

    def rotate(self, y, c, out, base=None, sign=1):
        self._check(lib().rsdft_rotate(self._h, _ptr(y), y.shape[0], _ptr(c), c.shape[1], _ptr(base),
                                       sign, _ptr(out), _stream()))

    def rayleigh_ritz(self, gh, gs, nkeep, c_out, pivot_tol=1e-8):
        lam = np.zeros(nkeep)
        nd = C.c_int(0)
        self._check(lib().rsdft_rayleigh_ritz(self._h, _ptr(gh), _ptr(gs), gh.shape[0], nkeep,
                                              pivot_tol, _ptr(lam), _ptr(c_out), C.byref(nd),
                                              _stream()))
        return lam, nd.value

    def eigh(self, a, nkeep, z_out):
        lam = np.zeros(nkeep)
        self._check(lib().rsdft_eigh(self._h, _ptr(a), a.shape[0], nkeep, _ptr(lam), _ptr(z_out),
                                     _stream()))
        return lam

    def propagate(self, psi, dt, nsteps, order=4):
        """rsdft_propagate: psi <- (sum_j (-i dt H)^j / j!)^nsteps psi, in place."""
        self._check(lib().rsdft_propagate(self._h, _ptr(psi), psi.shape[0], float(dt), int(nsteps), int(order),
                                          _stream()))

    # ---- LOBPCG
    @staticmethod
    def lobpcg_opts(**kw) -> LobpcgOpts:
        o = LobpcgOpts()
        lib().rsdft_lobpcg_default_opts(C.byref(o))
        for k, v in kw.items():
            setattr(o, k, v)
        return o

    def lobpcg(self, x, opts: LobpcgOpts):
        m = x.shape[0]
        eig, res = np.zeros(m), np.zeros(m)
        stats = LobpcgStats()
        st = self._check(lib().rsdft_lobpcg(self._h, _ptr(x), m, C.byref(opts), _ptr(eig), _ptr(res),
                                            C.byref(stats), _stream()), allow=(E_NOT_CONVERGED,))
        return eig, res, stats, st

    # ---- real Gamma-point form (float64 [nband][n] real blocks)
    def apply_h_real(self, x, hx):
        self._check(lib().rsdft_apply_h_real(self._h, _ptr(x), _ptr(hx), x.shape[0], _stream()))

    def gram_real(self, a, b, g):
        self._check(lib().rsdft_gram_real(self._h, _ptr(a), a.shape[0], _ptr(b), b.shape[0], _ptr(g),
                                          _stream()))

    def rotate_real(self, y, c, out, base=None, sign=1):
        self._check(lib().rsdft_rotate_real(self._h, _ptr(y), y.shape[0], _ptr(c), c.shape[1], _ptr(base),
                                            sign, _ptr(out), _stream()))

    def lobpcg_real(self, x, opts: LobpcgOpts):
        m = x.shape[0]
        eig, res = np.zeros(m), np.zeros(m)
        stats = LobpcgStats()
        st = self._check(lib().rsdft_lobpcg_real(self._h, _ptr(x), m, C.byref(opts), _ptr(eig), _ptr(res),
                                                 C.byref(stats), _stream()), allow=(E_NOT_CONVERGED,))
        return eig, res, stats, st

    # ---- SCF
    @staticmethod
    def scf_opts(**kw) -> ScfOpts:
        o = ScfOpts()
        lib().rsdft_scf_default_opts(C.byref(o))
        for k, v in kw.items():
            setattr(o, k, v)
        return o

    def scf_init(self, nband, opts: ScfOpts):
        self._check(lib().rsdft_scf_init(self._h, nband, C.byref(opts), _stream()))

    def scf_step(self, x, opts: ScfOpts):
        m = x.shape[0]
        out = ScfOut()
        eig, occ = np.zeros(m), np.zeros(m)
        self._check(lib().rsdft_scf_step(self._h, _ptr(x), m, C.byref(opts), C.byref(out), _ptr(eig),
                                         _ptr(occ), _stream()))
        return out, eig, occ

    def scf_step_real(self, x, opts: ScfOpts):
        """rsdft_scf_step_real: the SCF step on real Gamma-point orbitals (float64 [m][n])."""
        m = x.shape[0]
        out = ScfOut()
        eig, occ = np.zeros(m), np.zeros(m)
        self._check(lib().rsdft_scf_step_real(self._h, _ptr(x), m, C.byref(opts), C.byref(out), _ptr(eig),
                                              _ptr(occ), _stream()))
        return out, eig, occ

    def scf_density_ptr(self) -> int:
        return int(lib().rsdft_scf_density(self._h) or 0)

    def density(self, x, f, rho):
        self._check(lib().rsdft_density(self._h, _ptr(x), _ptr(f), x.shape[0], _ptr(rho), _stream()))

    def hartree(self, rho, vh):
        self._check(lib().rsdft_hartree(self._h, _ptr(rho), _ptr(vh), _stream()))

    def lda(self, rho, eps, vxc):
        self._check(lib().rsdft_lda(self._h, _ptr(rho), _ptr(eps), _ptr(vxc), _stream()))

    def xc_pbe(self, rho, eps, vxc):
        self._check(lib().rsdft_xc_pbe(self._h, _ptr(rho), _ptr(eps), _ptr(vxc), _stream()))

    def occupations(self, eig, n_electrons, kT, f):
        mu, S = C.c_double(0), C.c_double(0)
        self._check(lib().rsdft_occupations(self._h, _ptr(eig), eig.shape[0], float(n_electrons),
                                            float(kT), _ptr(f), C.byref(mu), C.byref(S), _stream()))
        return mu.value, S.value


def context_for(wl, v_loc: Optional[np.ndarray] = None) -> Context:
    """Context for a workloads.Workload: V_loc built by rsdft_gaussian_vloc."""
    if v_loc is None:
        v_loc = gaussian_vloc(wl.L, wl.N, wl.positions, wl.Z, wl.sigma)
    return Context(wl.L, wl.N, v_loc, wl.positions, wl.rc, wl.rcut, wl.e_kb(), wl.nproj)
