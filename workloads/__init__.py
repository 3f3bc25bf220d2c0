"""Seeded synthetic workloads for the real-space Kohn-Sham LOBPCG path.

This module is shared by the CUDA path, the FP64 oracle, the tests and the
bench.  It holds only input *recipes*: lattice sites, seeded random draws
(Kleinman-Bylander energies, the initial orbital block) and the sizes of the
workloads.  It holds none of the method's arithmetic: the local potential,
the projector tables, the Hamiltonian and everything downstream are built
independently by each side from these raw inputs.

The paper benchmarks 216-atom diamond and 128-atom bcc tungsten with ONCV
pseudopotentials (the benchmark-target paragraph beside Fig. 1).  Those files
are not available, so the pseudo-atoms here are synthetic: a Gaussian local
potential -Z exp(-r^2 / (2 sigma^2)) and four Gaussian KB projectors
(s, p_x, p_y, p_z) per atom with KB energies drawn from U[0.5, 2] Ha.
"""
from __future__ import annotations

import dataclasses
from typing import List, Tuple

import numpy as np

# Random streams: one numpy Generator per (seed, stream id), so that each
# draw is independent of the order in which the others are made.
_STREAM_EKB = 0
_STREAM_X0 = 1
_STREAM_NN = 2
_STREAM_PROBE = 3
_STREAM_X0_REAL = 4


def diamond_sites(a: float, reps: int) -> np.ndarray:
    """Diamond-cubic sites (fcc + fcc shifted by a/4 (1,1,1)), reps^3 cells."""
    fcc = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
    basis = np.concatenate([fcc, fcc + 0.25])
    return _replicate(basis, a, reps)


def bcc_sites(a: float, reps: int) -> np.ndarray:
    """Body-centred cubic sites, reps^3 conventional cells."""
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]])
    return _replicate(basis, a, reps)


def _replicate(basis: np.ndarray, a: float, reps: int) -> np.ndarray:
    out = []
    for i in range(reps):
        for j in range(reps):
            for k in range(reps):
                out.append((basis + np.array([i, j, k], dtype=np.float64)) * a)
    return np.ascontiguousarray(np.concatenate(out), dtype=np.float64)


def draw_e_kb(seed: int, natom: int, nproj: int = 4) -> np.ndarray:
    """KB energies E_{a,j} ~ U[0.5, 2] Ha, shape [natom][nproj], atom-major."""
    rng = np.random.default_rng([seed, _STREAM_EKB])
    return rng.uniform(0.5, 2.0, (natom, nproj))


def draw_x0(seed: int, nband: int, npts: int) -> np.ndarray:
    """Initial orbital block: complex standard normal, shape [nband][npts]."""
    rng = np.random.default_rng([seed, _STREAM_X0])
    re_im = rng.standard_normal((nband, npts, 2))
    return re_im.view(np.complex128)[..., 0]


def draw_x0_real(seed: int, nband: int, npts: int) -> np.ndarray:
    """Initial real orbital block (Gamma-point real form): standard normal,
    shape [nband][npts]."""
    rng = np.random.default_rng([seed, _STREAM_X0_REAL])
    return rng.standard_normal((nband, npts))


def draw_probes(seed: int, nprobe: int, npts: int) -> np.ndarray:
    """Probe block for subspace sketches: complex standard normal,
    shape [nprobe][npts] (test infrastructure; not an input of the method)."""
    rng = np.random.default_rng([seed, _STREAM_PROBE])
    re_im = rng.standard_normal((nprobe, npts, 2))
    return re_im.view(np.complex128)[..., 0]


def draw_nn_weights(seed: int, hidden: int = 8) -> np.ndarray:
    """Initial weights of the preconditioner network (four 3x3x3 convolutions,
    channels 2 -> hidden -> hidden -> hidden -> 1, each layer [27][cin][cout]),
    flat float64: normal with standard deviation 1/sqrt(27 cin) for the first
    three layers and zero for the last (the network starts as no correction)."""
    rng = np.random.default_rng([seed, _STREAM_NN])
    chans = [(2, hidden), (hidden, hidden), (hidden, hidden), (hidden, 1)]
    out = []
    for l, (ci, co) in enumerate(chans):
        if l == len(chans) - 1:
            out.append(np.zeros(27 * ci * co))
        else:
            out.append(rng.standard_normal(27 * ci * co) / np.sqrt(27.0 * ci))
    return np.concatenate(out)


@dataclasses.dataclass
class Workload:
    """One synthetic cell.  Lengths in bohr, energies in Hartree."""
    name: str
    L: Tuple[float, float, float]          # orthorhombic cell edges
    N: Tuple[int, int, int]                # grid points per axis (x, y, z)
    positions: np.ndarray                  # [natom][3] bohr
    Z: float = 4.0                         # Gaussian local-potential charge
    sigma: float = 0.6                     # Gaussian local-potential width
    rc: float = 1.0                        # projector Gaussian radius
    rcut: float = 3.0                      # projector truncation radius
    nproj: int = 4                         # s, p_x, p_y, p_z
    nband: int = 16
    n_electrons: float = 0.0               # spin-degenerate electron count
    kT: float = 0.0                        # Fermi-Dirac temperature (0: aufbau)
    seed: int = 0
    maxit: int = 40                        # LOBPCG iterations (fixed-count runs)
    tol: float = 1e-6                      # max residual norm, Ha

    @property
    def natom(self) -> int:
        return int(self.positions.shape[0])

    @property
    def npts(self) -> int:
        return int(self.N[0] * self.N[1] * self.N[2])

    def e_kb(self) -> np.ndarray:
        return draw_e_kb(self.seed, self.natom, self.nproj)

    def x0(self, nband: int | None = None) -> np.ndarray:
        return draw_x0(self.seed, self.nband if nband is None else nband, self.npts)

    def x0_real(self, nband: int | None = None) -> np.ndarray:
        return draw_x0_real(self.seed, self.nband if nband is None else nband, self.npts)


def _cubic(L: float) -> Tuple[float, float, float]:
    return (L, L, L)


def diamond8_24(seed: int = 0) -> Workload:
    """Fixed-potential LOBPCG: 8 C at diamond-cubic sites (a = L = 10 bohr),
    24^3 grid, 16 bands, Gamma point, 40 iterations."""
    return Workload("diamond8_24", _cubic(10.0), (24, 24, 24), diamond_sites(10.0, 1),
                    Z=4.0, nband=16, n_electrons=32.0, seed=seed, maxit=40)


def diamond64_64(seed: int = 0) -> Workload:
    """Full SCF: 64 C (2x2x2 diamond, a = 6.74, L = 13.48), 64^3, 144 bands
    (128 occupied), LDA, FFT Hartree, Anderson mixing beta = 0.3."""
    return Workload("diamond64_64", _cubic(13.48), (64, 64, 64), diamond_sites(6.74, 2),
                    Z=4.0, nband=144, n_electrons=256.0, seed=seed, maxit=200)


def diamond216_96(seed: int = 0) -> Workload:
    """216 C (3x3x3 diamond, L = 20.22), 96^3, 480 bands (432 occupied)."""
    return Workload("diamond216_96", _cubic(20.22), (96, 96, 96), diamond_sites(6.74, 3),
                    Z=4.0, nband=480, n_electrons=864.0, seed=seed, maxit=200)


def bcc128_120(seed: int = 0) -> Workload:
    """128-atom bcc metal (4x4x4, a = 5.98, L = 23.92), 120^3, Z = 6,
    460 bands, Fermi-Dirac kT = 0.01 Ha, 768 electrons."""
    return Workload("bcc128_120", _cubic(23.92), (120, 120, 120), bcc_sites(5.98, 4),
                    Z=6.0, nband=460, n_electrons=768.0, kT=0.01, seed=seed, maxit=200)


def diamond8_32(seed: int = 0) -> Workload:
    """8 C in one diamond-cubic cell (a = L = 6.74 bohr) on a 32^3 grid: the
    spacing (0.2106 bohr) and chemistry of the 64-atom 64^3 cell; 20 bands (16
    occupied).  A training cell of the learned preconditioner."""
    return Workload("diamond8_32", _cubic(6.74), (32, 32, 32), diamond_sites(6.74, 1),
                    Z=4.0, nband=20, n_electrons=32.0, seed=seed, maxit=200)


def bcc2_30(seed: int = 0) -> Workload:
    """2 atoms in one bcc cell (a = L = 5.98 bohr, Z = 6) on a 30^3 grid: the
    spacing (0.1993 bohr) and chemistry of the 128-atom 120^3 metal; 8 bands
    (6 occupied), Fermi-Dirac kT = 0.01.  The projectors are cut at 2.9 bohr,
    just below half the cell edge.  A training cell of the learned
    preconditioner."""
    return Workload("bcc2_30", _cubic(5.98), (30, 30, 30), bcc_sites(5.98, 1), Z=6.0,
                    rcut=2.9, nband=8, n_electrons=12.0, kT=0.01, seed=seed, maxit=200)


def bcc16_60(seed: int = 0) -> Workload:
    """16 atoms (2x2x2 bcc, a = 5.98, L = 11.96, Z = 6) on a 60^3 grid (the
    128-atom metal's spacing), 56 bands (48 occupied), kT = 0.01: the reduced
    metal cell on which the learned preconditioner is judged against TPA."""
    return Workload("bcc16_60", _cubic(11.96), (60, 60, 60), bcc_sites(5.98, 2), Z=6.0,
                    nband=56, n_electrons=96.0, kT=0.01, seed=seed, maxit=200)


FIVE_SMOOTH_BATCH_GRIDS = (32, 36, 40, 45, 48, 50, 54, 60, 64)


def batched_cells(ncell: int = 32) -> List[Workload]:
    """Uneven independent cells: cell c uses seed c; diamond (even c) or bcc
    (odd c); grid from the 5-smooth set 32..64; 32-160 bands; 8-64 atoms; the
    cell edge is chosen so that the spacing h lies in 0.2-0.25 bohr."""
    cells = []
    for c in range(ncell):
        rng = np.random.default_rng([c, 7])
        N = int(rng.choice(FIVE_SMOOTH_BATCH_GRIDS))
        h = float(rng.uniform(0.2, 0.25))
        L = N * h
        if c % 2 == 0:
            # diamond supercell count from the diamond lattice constant (6.74 bohr)
            reps = max(1, int(round(L / 6.74)))
            pos = diamond_sites(L / reps, reps)
            Z, ne_per_atom = 4.0, 4.0
        else:
            # a 2x2x2 bcc supercell (16 atoms): 48 occupied bands, so the band
            # count keeps its buffer above the occupied ones
            reps = 2
            pos = bcc_sites(L / reps, reps)
            Z, ne_per_atom = 6.0, 6.0
        natom = pos.shape[0]
        n_el = ne_per_atom * natom
        nband = int(min(160, max(32, int(np.ceil(n_el / 2 * 1.15)))))
        cells.append(Workload(f"cell{c:02d}_{N}", _cubic(L), (N, N, N), pos, Z=Z,
                              nband=nband, n_electrons=n_el, kT=0.01 if c % 2 else 0.0,
                              seed=c))
    return cells


def small_cell(N=(12, 12, 12), L=(6.0, 6.0, 6.0), natom: int = 2, nband: int = 8,
               Z: float = 4.0, seed: int = 0, rcut: float = 2.5) -> Workload:
    """A tiny cell for brute-force checks: natom atoms on a seeded random
    placement (not a lattice), so that no symmetry hides an index error."""
    rng = np.random.default_rng([seed, 11])
    pos = rng.uniform(0.0, 1.0, (natom, 3)) * np.asarray(L)
    return Workload(f"small{N[0]}x{N[1]}x{N[2]}", tuple(L), tuple(N), pos, Z=Z,
                    rcut=rcut, nband=nband, n_electrons=float(2 * min(nband, natom * 2)),
                    seed=seed)


REGISTRY = {
    "diamond8_24": diamond8_24,
    "diamond64_64": diamond64_64,
    "diamond216_96": diamond216_96,
    "bcc128_120": bcc128_120,
    "diamond8_32": diamond8_32,
    "bcc2_30": bcc2_30,
    "bcc16_60": bcc16_60,
}
