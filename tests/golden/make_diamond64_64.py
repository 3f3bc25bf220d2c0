#!/usr/bin/env python
"""Write the oracle's SCF values of the 64-atom diamond cell (64^3 grid, 144 bands,
128 occupied; the bench configuration) to diamond64_64_scf.npz.

Calls only ``oracle/`` (and the seeded inputs of ``workloads``).  Every step's
LOBPCG is converged to 1e-10 Ha over the occupied bands, so each step is a
function of its input density alone and the CUDA path, started from the same
seeded block, must reproduce it (eigenvalues to 1e-9 Ha, energies to 1e-8 Ha per
atom, occupied subspace to a projector distance of 1e-7).

Stored per step s (0-based), step 0 from the uniform density:
  eig_s [144]      Ritz values (the first 128 converged, the rest a buffer)
  energy_s [6]     e_tot, e_band, e_h, e_xc, e_vxc, drho
  res_s [144]      final residual norms
  iters_s          LOBPCG iterations
  prefix_s         bands in the occupied prefix that ends at a gap >= 1e-4 Ha
  sketch_s [q][q]  M = C^H C, C[b][j] = <x_b|z_j> over the prefix bands, with
                   probes z_j = workloads.draw_probes(PROBE_SEED, q, n): a
                   rotation-invariant sketch of the occupied projector
                   (M = dV Z^H P Z with P the projector in the grid basis).

Run (about half an hour on 8 cores):  python tests/golden/make_diamond64_64.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402
from oracle.grid import Grid, kb_projectors, local_potential  # noqa: E402
from oracle.hamiltonian import Hamiltonian  # noqa: E402
from oracle.scf import scf_init, scf_step  # noqa: E402

STEPS = 4
TOL = 1e-10
PROBE_SEED = 100
NPROBE = 32
GAP_MIN = 1e-4


def occupied_prefix(eig, nocc):
    """Largest p <= nocc with eig[p] - eig[p-1] >= GAP_MIN (eig[nocc] the first buffer band)."""
    for p in range(nocc, 0, -1):
        if eig[p] - eig[p - 1] >= GAP_MIN:
            return p
    return 0


def main(out_path):
    wl = workloads.diamond64_64()
    g = Grid(L=wl.L, N=wl.N)
    v_loc = local_potential(g, wl.positions, wl.Z, wl.sigma)
    P = kb_projectors(g, wl.positions, wl.rc, wl.rcut, wl.e_kb())
    ham = Hamiltonian(g, v_loc, P)
    nocc = int(np.ceil(wl.n_electrons / 2))
    st = scf_init(g, wl.n_electrons, wl.x0(), beta=0.3, depth=4)
    Z = workloads.draw_probes(PROBE_SEED, NPROBE, g.n)
    rec = {"tol": TOL, "probe_seed": PROBE_SEED, "nprobe": NPROBE, "nocc": nocc, "steps": STEPS,
           "dV": g.dV}
    for s in range(STEPS):
        t0 = time.perf_counter()
        out = scf_step(ham, v_loc, st, wl.n_electrons, wl.kT, first_maxit=300, tol=TOL, later_tol=TOL)
        res = out.lobpcg
        assert res.converged, f"step {s}: not converged"
        p = occupied_prefix(out.eig, nocc)
        C = (res.X[:p].conj() @ Z.T) * g.dV
        rec[f"eig_{s}"] = out.eig
        rec[f"energy_{s}"] = np.array([out.e_tot, out.e_band, out.e_h, out.e_xc, out.e_vxc, out.drho])
        rec[f"res_{s}"] = res.resnorm
        rec[f"iters_{s}"] = res.iterations
        rec[f"prefix_{s}"] = p
        rec[f"sketch_{s}"] = C.conj().T @ C
        print(f"step {s}: {res.iterations} iterations, {time.perf_counter() - t0:.0f} s, "
              f"e_tot {out.e_tot:.12f}, drho {out.drho:.3e}, prefix {p}, "
              f"gap {out.eig[nocc] - out.eig[nocc - 1]:.3e}", flush=True)
    np.savez(out_path, **rec)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else
         os.path.join(os.path.dirname(os.path.abspath(__file__)), "diamond64_64_scf.npz"))
