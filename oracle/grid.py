"""Oracle: real-space grid, reciprocal vectors, local potential, KB projectors.

Test infrastructure only (see ``oracle/__init__``).

Conventions (the paper gives none; these are the readings the CUDA path
follows too):

* Orthorhombic cell with edges (Lx, Ly, Lz); grid (Nx, Ny, Nz); spacing
  h_a = L_a / N_a; point r = (ix hx, iy hy, iz hz); linear index
  i = (iz Ny + iy) Nx + ix (x fastest).  Arrays shaped (Nz, Ny, Nx).
* Inner product <a|b> = sum_r conj(a) b dV, dV = Lx Ly Lz / n.
* Reciprocal vectors G_a = (2 pi / L_a) k, k in numpy.fft.fftfreq order
  (0..N/2-1, -N/2..-1 for even N).  The kinetic operator of SCF task (1) is
  T psi = IFFT(|G|^2/2 FFT(psi)) on the periodic grid.
* Minimal-image displacement d = r - R - L floor((r - R)/L + 1/2).
* Local potential V_loc(r) = sum_a -Z exp(-|d_a|^2 / (2 sigma^2)).
* Projectors (four per atom, s, p_x, p_y, p_z), truncated to |d| < rcut:
  s: exp(-|d|^2/(2 rc^2)),  p_alpha: (d_alpha / rc) exp(-|d|^2/(2 rc^2)),
  each then normalised on the grid so that sum beta^2 dV = 1.  The truncated,
  grid-normalised table is the definition of the projector.

Pins (tests/test_oracle_grid.py): fftfreq order and |G|^2 of explicit plane
waves; V_loc and projectors against pure-Python per-point loops on a tiny grid;
projector normalisation; a projector sphere that wraps the periodic boundary.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp


@dataclasses.dataclass
class Grid:
    L: tuple          # (Lx, Ly, Lz)
    N: tuple          # (Nx, Ny, Nz)

    @property
    def n(self) -> int:
        return int(self.N[0] * self.N[1] * self.N[2])

    @property
    def shape(self):
        """Array shape (Nz, Ny, Nx)."""
        return (self.N[2], self.N[1], self.N[0])

    @property
    def h(self):
        return tuple(self.L[a] / self.N[a] for a in range(3))

    @property
    def dV(self) -> float:
        return float(self.L[0] * self.L[1] * self.L[2] / self.n)

    def coords(self):
        """Point coordinates x, y, z as arrays of shape (Nz, Ny, Nx)."""
        hx, hy, hz = self.h
        iz, iy, ix = np.meshgrid(np.arange(self.N[2]), np.arange(self.N[1]),
                                 np.arange(self.N[0]), indexing="ij")
        return ix * hx, iy * hy, iz * hz

    def g_axes(self):
        """G components per axis in FFT order: (gx[Nx], gy[Ny], gz[Nz])."""
        return tuple(2.0 * np.pi / self.L[a] * np.fft.fftfreq(self.N[a], d=1.0 / self.N[a])
                     for a in range(3))

    def g2(self) -> np.ndarray:
        """|G|^2 on the (Nz, Ny, Nx) reciprocal grid."""
        gx, gy, gz = self.g_axes()
        return gz[:, None, None] ** 2 + gy[None, :, None] ** 2 + gx[None, None, :] ** 2


def minimal_image(d: np.ndarray, L: float) -> np.ndarray:
    return d - L * np.floor(d / L + 0.5)


def displacements(grid: Grid, R):
    """Minimal-image displacement components (dx, dy, dz) from atom R to every
    grid point, each shaped (Nz, Ny, Nx)."""
    x, y, z = grid.coords()
    return (minimal_image(x - R[0], grid.L[0]),
            minimal_image(y - R[1], grid.L[1]),
            minimal_image(z - R[2], grid.L[2]))


def local_potential(grid: Grid, positions: np.ndarray, Z: float, sigma: float) -> np.ndarray:
    """V_loc(r) = sum_a -Z exp(-|d_a(r)|^2 / (2 sigma^2)); returns flat [n]."""
    v = np.zeros(grid.shape)
    for R in positions:
        dx, dy, dz = displacements(grid, R)
        v -= Z * np.exp(-(dx * dx + dy * dy + dz * dz) / (2.0 * sigma * sigma))
    return v.reshape(-1)


@dataclasses.dataclass
class Projectors:
    """KB projectors as a sparse matrix B [natom*nproj, n] (row a*nproj + j),
    plus energies E [natom*nproj]."""
    B: sp.csr_matrix
    E: np.ndarray
    nproj: int

    @property
    def natom(self) -> int:
        return self.B.shape[0] // self.nproj


def kb_projectors(grid: Grid, positions: np.ndarray, rc: float, rcut: float,
                  e_kb: np.ndarray, nproj: int = 4) -> Projectors:
    """Truncated Gaussian s, p_x, p_y, p_z projectors, grid-normalised."""
    if nproj not in (1, 4):
        raise ValueError("nproj must be 1 (s) or 4 (s, px, py, pz)")
    if rcut >= 0.5 * min(grid.L):
        raise ValueError("rcut must be below half the shortest cell edge")
    rows, cols, vals = [], [], []
    dV = grid.dV
    for a, R in enumerate(positions):
        dx, dy, dz = (c.reshape(-1) for c in displacements(grid, R))
        d2 = dx * dx + dy * dy + dz * dz
        idx = np.nonzero(d2 < rcut * rcut)[0]
        g = np.exp(-d2[idx] / (2.0 * rc * rc))
        funcs = [g]
        if nproj == 4:
            funcs += [dx[idx] / rc * g, dy[idx] / rc * g, dz[idx] / rc * g]
        for j, b in enumerate(funcs):
            norm = np.sqrt(np.sum(b * b) * dV)
            rows.append(np.full(idx.size, a * nproj + j))
            cols.append(idx)
            vals.append(b / norm)
    natom = len(positions)
    B = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(natom * nproj, grid.n))
    E = np.asarray(e_kb, dtype=np.float64).reshape(natom, -1)[:, :nproj].reshape(-1)
    return Projectors(B=B, E=E, nproj=nproj)
