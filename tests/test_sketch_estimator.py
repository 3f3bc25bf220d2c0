"""The subspace sketch used by the bench-configuration parity test estimates
the projector distance sin(theta_max): checked against the exact value from an
SVD on random subspaces rotated by known angles."""
import numpy as np
import pytest

import workloads
from tests.sketch import distance_from_sketches, sketch_matrix


@pytest.mark.parametrize("theta", [1e-3, 1e-6, 1e-8])
def test_sketch_distance_matches_svd(theta):
    n, p, dV = 3000, 12, 0.37
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.standard_normal((n, p + 1)) + 1j * rng.standard_normal((n, p + 1)))
    Xa = Q[:, :p].T / np.sqrt(dV)
    Xb = Xa.copy()
    # rotate one direction by theta towards the complement
    Xb[3] = (np.cos(theta) * Q[:, 3] + np.sin(theta) * Q[:, p]) / np.sqrt(dV)
    s = np.linalg.svd((Xa.conj() @ Xb.T) * dV, compute_uv=False)
    exact = np.sqrt(max(0.0, 1.0 - np.min(s) ** 2)) if theta > 1e-7 else theta
    Z = workloads.draw_probes(1, 32, n)
    est = distance_from_sketches(sketch_matrix(Xb, Z, dV), sketch_matrix(Xa, Z, dV), dV)
    assert 0.8 * exact <= est <= 1.25 * exact


def test_sketch_is_rotation_invariant():
    n, p, dV = 2000, 6, 1.3
    rng = np.random.default_rng(6)
    Q, _ = np.linalg.qr(rng.standard_normal((n, p)) + 1j * rng.standard_normal((n, p)))
    X = Q.T / np.sqrt(dV)
    U, _ = np.linalg.qr(rng.standard_normal((p, p)) + 1j * rng.standard_normal((p, p)))
    Z = workloads.draw_probes(2, 16, n)
    assert distance_from_sketches(sketch_matrix(U @ X, Z, dV), sketch_matrix(X, Z, dV), dV) < 1e-13
