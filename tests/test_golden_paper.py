"""The synthetic workloads' lattice constants against the paper's printed
benchmark grids (tests/golden/paper_benchmark_grids.txt): a grid of spacing h
resolves plane waves up to |G| = pi/h, i.e. a cutoff of (pi/h)^2 Ry, so the
printed (grid, cutoff) pairs fix the cell edge L = N h and with the supercell
size the cubic lattice constant."""
import math
import pathlib

import workloads

GOLDEN = pathlib.Path(__file__).parent / "golden" / "paper_benchmark_grids.txt"


def _rows():
    out = {}
    for line in GOLDEN.read_text().splitlines():
        if line.startswith("#") or not line.strip():
            continue
        name, sc, atoms, grid, ecut = line.split()
        out[name] = (int(sc), int(atoms), int(grid), float(ecut))
    return out


def test_diamond_lattice_constant_matches_paper_cutoff():
    sc, atoms, grid, ecut = _rows()["diamond"]
    wl = workloads.diamond216_96()
    assert len(wl.positions) == atoms == 8 * sc ** 3
    h = wl.L[0] / grid                       # the paper's grid on our cell
    assert abs((math.pi / h) ** 2 - ecut) / ecut < 5e-3


def test_bcc_lattice_constant_matches_paper_cutoff():
    sc, atoms, grid, ecut = _rows()["bcc_W"]
    wl = workloads.bcc128_120()
    assert len(wl.positions) == atoms == 2 * sc ** 3
    h = wl.L[0] / grid
    assert abs((math.pi / h) ** 2 - ecut) / ecut < 5e-3
