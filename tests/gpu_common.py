"""Shared helpers of the GPU parity tests: build the CUDA context and the
oracle Hamiltonian for the same workload, move arrays between host and device."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.grid import Grid, kb_projectors, local_potential  # noqa: E402
from oracle.hamiltonian import Hamiltonian  # noqa: E402

from paper_2512_04447_gb300 import rsdft as R  # noqa: E402


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t) -> np.ndarray:
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def pair(wl):
    """(CUDA context, oracle Hamiltonian, oracle V_loc) for a workload; each
    side builds V_loc and the projectors with its own code."""
    g = Grid(L=wl.L, N=wl.N)
    v = local_potential(g, wl.positions, wl.Z, wl.sigma)
    P = kb_projectors(g, wl.positions, wl.rc, wl.rcut, wl.e_kb(), wl.nproj)
    ham = Hamiltonian(g, v, P)
    ctx = R.context_for(wl)
    return ctx, ham, v


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# Bands of diamond8_24 whose span the subspace checks compare: the first 8 end at a
# gap of 0.256 Ha to the 9th, while the occupied 16 end at 9.3e-4 Ha.  By the
# Davis-Kahan sin-theta bound, sin(theta) <= ||R||_2 / gap <= sqrt(p) r_max / gap,
# a residual tolerance of 1e-9 pins the 8-band span to 1.1e-8 per side, but the
# 16-band span only to 4e-6.
PREFIX8 = 8


def subspace_distance(Xa, Xb, dV):
    """sin of the largest principal angle between span(Xa) and span(Xb) (rows):
    ||(I - Qb Qb^H) Qa||_2 with both bases orthonormalised in the dV metric.  From
    sqrt(1 - s_min^2) of the raw overlap instead, a departure of d from
    orthonormality reads as an angle of sqrt(2 d) (4e-14 looks like 3e-7) and the
    result has a floor of ~2e-8."""
    qa = np.linalg.qr(Xa.T * np.sqrt(dV))[0]
    qb = np.linalg.qr(Xb.T * np.sqrt(dV))[0]
    return float(np.linalg.norm(qa - qb @ (qb.conj().T @ qa), 2))
