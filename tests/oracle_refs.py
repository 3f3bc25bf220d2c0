"""Independent dense references used to pin the oracle (not the oracle itself).

The kinetic matrix here is built from its Fourier-series definition evaluated
term by term with cosines (no FFT), as a Kronecker sum of 1D matrices:
T1[j, l] = (1/N) sum_k (G_k^2 / 2) cos(2 pi k (j - l) / N).
"""
import numpy as np


def kinetic_1d(N: int, L: float) -> np.ndarray:
    ks = [k if k < (N + 1) // 2 else k - N for k in range(N)]
    T = np.zeros((N, N))
    for j in range(N):
        for l in range(N):
            s = 0.0
            for k in ks:
                G = 2.0 * np.pi / L * k
                s += 0.5 * G * G * np.cos(2.0 * np.pi * k * (j - l) / N)
            T[j, l] = s / N
    return T


def kinetic_dense(N, L) -> np.ndarray:
    """T on the (z, y, x)-ordered grid, x fastest."""
    Tx, Ty, Tz = (kinetic_1d(N[a], L[a]) for a in range(3))
    Ix, Iy, Iz = np.eye(N[0]), np.eye(N[1]), np.eye(N[2])
    return (np.kron(Tz, np.kron(Iy, Ix)) + np.kron(Iz, np.kron(Ty, Ix))
            + np.kron(Iz, np.kron(Iy, Tx)))


def hamiltonian_dense(N, L, v, B=None, E=None) -> np.ndarray:
    """T + diag(v) + sum_aj beta_aj E_aj beta_aj^T dV (B dense [nproj_tot][n])."""
    H = kinetic_dense(N, L).astype(np.complex128)
    H += np.diag(v)
    if B is not None:
        dV = L[0] * L[1] * L[2] / (N[0] * N[1] * N[2])
        H += (B.T * E[None, :]) @ B * dV
    return H
