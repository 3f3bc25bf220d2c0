"""C ABI checks that need no GPU: the CUDA library builds and loads, exports
every function declared in include/rsdft.h, its host-side input builder agrees
with the oracle, and argument validation returns status codes."""
import ctypes as C

import numpy as np
import pytest

from oracle.grid import Grid, local_potential
from paper_2512_04447_gb300 import build
from paper_2512_04447_gb300 import rsdft as R
from workloads import diamond8_24, small_cell


@pytest.fixture(scope="module")
def lib():
    build.build()
    return R.lib()


def test_exports_every_declared_symbol(lib):
    syms = R.header_symbols()
    assert len(syms) >= 25
    assert [s for s in syms if not hasattr(lib, s)] == []


@pytest.mark.parametrize("wl", [diamond8_24(), small_cell(N=(12, 10, 8), L=(6.0, 5.5, 5.0), natom=3)])
def test_gaussian_vloc_matches_oracle(lib, wl):
    v = R.gaussian_vloc(wl.L, wl.N, wl.positions, wl.Z, wl.sigma)
    vo = local_potential(Grid(L=wl.L, N=wl.N), wl.positions, wl.Z, wl.sigma)
    assert np.max(np.abs(v - vo)) < 1e-14 * np.max(np.abs(vo))


def _create(L, N, v=None, pos=None, rc=1.0, rcut=3.0, ekb=None, nproj=4, cell=None):
    n = N[0] * N[1] * N[2]
    v = np.zeros(n) if v is None else v
    c = cell if cell is not None else R._cell(L)
    pj = None
    if pos is not None:
        pj = R.Projectors(len(pos), R._ptr(pos), nproj, rc, rcut, R._ptr(ekb))
    h = C.c_void_p(0)
    st = R.lib().rsdft_create(C.byref(c), C.byref(R._grid(N)), R._ptr(v),
                              C.byref(pj) if pj is not None else None, C.byref(h))
    if st == R.OK:
        R.lib().rsdft_destroy(h)
    return st, R.lib().rsdft_last_error(None).decode()


@pytest.mark.parametrize("N", [(7, 8, 8), (8, 14, 8), (8, 8, 256), (1, 8, 8), (8, 8, 0)])
def test_grid_must_be_5_smooth(lib, N):
    st, msg = _create((5.0, 5.0, 5.0), N)
    assert st == R.E_GRID_NOT_5SMOOTH, msg


def test_non_orthorhombic_cell_rejected(lib):
    c = R._cell((5.0, 5.0, 5.0))
    c.a[0][1] = 0.5
    st, msg = _create((5.0, 5.0, 5.0), (8, 8, 8), cell=c)
    assert st == R.E_INVALID and "orthorhombic" in msg


def test_projector_arguments_validated(lib):
    pos = np.zeros((1, 3))
    ekb = np.ones((1, 4))
    assert _create((5.0, 5.0, 5.0), (8, 8, 8), pos=pos, ekb=ekb, rcut=2.5)[0] == R.E_INVALID
    assert _create((5.0, 5.0, 5.0), (8, 8, 8), pos=pos, ekb=ekb, rc=0.0, rcut=2.0)[0] == R.E_INVALID
    assert _create((5.0, 5.0, 5.0), (8, 8, 8), pos=pos, ekb=ekb, nproj=3, rcut=2.0)[0] == R.E_INVALID


def test_null_arguments_rejected(lib):
    assert lib.rsdft_create(None, None, None, None, None) == R.E_INVALID
    assert lib.rsdft_apply_h(None, None, None, 1, 0, None) == R.E_INVALID
    assert lib.rsdft_lobpcg(None, None, 4, None, None, None, None, None) == R.E_INVALID
    assert lib.rsdft_launch_count(None) == 0
    # the real Gamma-point form's entry points
    assert lib.rsdft_apply_h_real(None, None, None, 1, None) == R.E_INVALID
    assert lib.rsdft_gram_real(None, None, 1, None, 1, None, None) == R.E_INVALID
    assert lib.rsdft_rotate_real(None, None, 1, None, 1, None, 1, None, None) == R.E_INVALID
    assert lib.rsdft_lobpcg_real(None, None, 4, None, None, None, None, None) == R.E_INVALID
    assert lib.rsdft_scf_step_real(None, None, 4, None, None, None, None, None) == R.E_INVALID


def test_create_without_gpu_reports_cuda_error(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    st, msg = _create((5.0, 5.0, 5.0), (8, 8, 8))
    assert st == R.E_CUDA
