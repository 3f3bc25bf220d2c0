"""Oracle: real-time propagation of Kohn-Sham orbitals by H psi (RS-TDDFT).

Test infrastructure only (see ``oracle/__init__``).

The paper motivates its real-space code by real-time TDDFT, where the orbitals
evolve under i d psi / dt = H psi and every time step is a few applications of
H to all orbitals at once (its introduction).  With a fixed H over a step of
length dt the exact step is psi <- exp(-i H dt) psi; the propagator here is the
truncated Taylor series of that exponential, the usual real-space choice:

    psi(t + dt) = sum_{j=0}^{p} (-i dt H)^j / j! psi(t)

evaluated term by term, T_0 = psi, T_j = (-i dt / j) H T_{j-1}, psi_new =
sum_j T_j, for nsteps steps (the potential is held fixed; a self-consistent
propagation would refresh V between steps).

Pins (tests/test_oracle_tddft.py): a plane wave of a free-electron cell, an
eigenvector of H with eigenvalue |G|^2/2, is multiplied per step by the scalar
series sum_j (-i e dt)^j / j!, each plane wave of a sum by its own factor;
against scipy.linalg.expm of the brute-force dense H of a 12^3 cell with
projectors (order 12, small dt) to 1e-11; the norm drifts by the Taylor
remainder only.
"""
from __future__ import annotations

import numpy as np

from .hamiltonian import Hamiltonian


def propagate(ham: Hamiltonian, psi: np.ndarray, dt: float, nsteps: int, order: int) -> np.ndarray:
    """psi [m][n] after nsteps steps of the order-p Taylor propagator."""
    psi = np.array(psi, dtype=np.complex128)
    for _ in range(nsteps):
        term = psi.copy()
        out = psi.copy()
        for j in range(1, order + 1):
            term = (-1j * dt / j) * ham.apply(term)
            out += term
        psi = out
    return psi
