"""Oracle: the Kohn-Sham Hamiltonian on the periodic real-space grid.

Test infrastructure only (see ``oracle/__init__``).

H psi = T psi + V psi + sum_{a,j} |beta_aj> E_aj <beta_aj|psi>

* T psi = IFFT(|G|^2/2 * FFT(psi)): the FFT Laplacian of SCF task (1); all
  orbitals go through one batched transform, as the paper does.
* V psi: the local (effective) potential, a pointwise product.
* The Kleinman-Bylander nonlocal operator of SCF task (4), with
  <beta|psi> = sum_r beta(r) psi(r) dV.

Orbital blocks are complex128 arrays [m][n] (band-major, x fastest).

Pins (tests/test_oracle_hamiltonian.py): plane waves are eigenvectors of T with
eigenvalue |G|^2/2; Hermiticity; V_NL beta = E beta for a lone normalised
projector; on a 12^3 grid H equals a dense matrix built independently
(Kronecker sum of explicit cosine-series 1D kinetic matrices + diagonal V +
brute-force projector outer products); kinetic_energy of a normalised plane
wave is |G|^2/2 and of an equal mix of two is their mean
(tests/test_oracle_pins_closed_form.py).
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

from .grid import Grid, Projectors


class Hamiltonian:
    def __init__(self, grid: Grid, v: np.ndarray, proj: Projectors | None = None,
                 workers: int = -1):
        self.grid = grid
        self.v = np.asarray(v, dtype=np.float64).reshape(-1)
        self.proj = proj
        self.t_g = 0.5 * grid.g2()
        self.workers = workers

    @property
    def dV(self) -> float:
        return self.grid.dV

    def set_potential(self, v: np.ndarray) -> None:
        self.v = np.asarray(v, dtype=np.float64).reshape(-1)

    def kinetic(self, psi: np.ndarray) -> np.ndarray:
        """T psi = IFFT(|G|^2/2 FFT(psi)), batched over bands."""
        m = psi.shape[0]
        f = sfft.fftn(psi.reshape((m,) + self.grid.shape), axes=(1, 2, 3), workers=self.workers)
        f *= self.t_g
        return sfft.ifftn(f, axes=(1, 2, 3), workers=self.workers).reshape(m, -1)

    def project(self, psi: np.ndarray) -> np.ndarray:
        """p[aj, b] = <beta_aj|psi_b> = sum_r beta_aj(r) psi_b(r) dV."""
        return (self.proj.B @ psi.T) * self.dV

    def nonlocal_(self, psi: np.ndarray) -> np.ndarray:
        """sum_aj |beta_aj> E_aj <beta_aj|psi>."""
        if self.proj is None:
            return np.zeros_like(psi)
        p = self.project(psi)
        return (self.proj.B.T @ (self.proj.E[:, None] * p)).T

    def apply(self, psi: np.ndarray) -> np.ndarray:
        psi = np.asarray(psi, dtype=np.complex128)
        return self.kinetic(psi) + self.v[None, :] * psi + self.nonlocal_(psi)

    def kinetic_energy(self, psi: np.ndarray) -> np.ndarray:
        """<psi_b|T|psi_b> per band (real)."""
        return np.real(np.sum(psi.conj() * self.kinetic(psi), axis=1)) * self.dV


def inner(a: np.ndarray, b: np.ndarray, dV: float) -> np.ndarray:
    """Gram matrix G[i, j] = <a_i|b_j> = sum_r conj(a_i) b_j dV."""
    return (a.conj() @ b.T) * dV
