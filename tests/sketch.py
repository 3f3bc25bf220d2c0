"""Rotation-invariant sketch of an occupied subspace, for comparing a subspace
with one stored as a few kilobytes (test infrastructure).

For orbitals x_b (orthonormal in the dV metric) and probes z_j whose points are
independent complex normals of variance sigma2, C[b][j] = <x_b|z_j> and
M = C^H C = dV Z^H P Z, with P the projector onto span(x) in the orthonormal
grid basis.  For two subspaces of the same dimension, D = P_a - P_b has zero
trace, so every entry of M_a - M_b has second moment (sigma2 dV)^2 ||D||_F^2;
the largest principal-angle sine is at most ||D||_F / sqrt(2) (the nonzero
singular values of D come in pairs +-sin(theta_i))."""
import numpy as np


def sketch_matrix(X, Z, dV):
    C = (X.conj() @ Z.T) * dV
    return C.conj().T @ C


def distance_from_sketches(M, M_ref, dV, sigma2=2.0):
    fro = np.sqrt(np.mean(np.abs(np.asarray(M) - np.asarray(M_ref)) ** 2)) / (sigma2 * dV)
    return float(fro / np.sqrt(2.0))
