"""The double-float Sturm count of the GPU bisection (csrc/sturm_df.h), compiled
for the host and checked against LAPACK's eigenvalues: at random points and at
points 1e-9 (relative to ||T||) on either side of every seventh eigenvalue, for
matrices scaled by 1e-8 to 1e6, with zero and tiny off-diagonal entries
(decoupled blocks) and a long matrix whose minors leave the FP32 range (the
power-of-two rescaling), the count equals the number of eigenvalues below x."""
import pathlib
import shutil
import subprocess

import numpy as np
import pytest
import scipy.linalg as sla

ROOT = pathlib.Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("needs g++")
    out = tmp_path_factory.mktemp("sturm") / "sturm_check"
    subprocess.run(["g++", "-O2", "-ffp-contract=off", "-std=c++17",
                    "-I", str(ROOT / "paper_2512_04447_gb300" / "csrc"),
                    str(ROOT / "tests" / "native" / "sturm_check.cpp"), "-o", str(out)], check=True)
    return out


def _counts(exe, d, e, xs):
    f = lambda a: " ".join(repr(float(v)) for v in a)
    inp = f"{len(d)}\n{f(d)}\n{f(e)}\n{len(xs)}\n{f(xs)}\n"
    out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout
    return np.array([int(v) for v in out.split()])


@pytest.mark.parametrize("k,scale,seed", [(432, 1.0, 1), (300, 1e6, 2), (200, 1e-8, 3), (48, 1.0, 4),
                                          (2000, 30.0, 5)])
def test_double_float_sturm_count_matches_eigenvalues(exe, k, scale, seed):
    rng = np.random.default_rng(seed)
    d = rng.uniform(-3, 5, k) * scale
    e = rng.standard_normal(k - 1) * scale
    e[k // 7] = 0.0
    e[k // 5] = 1e-30 * scale
    w = sla.eigh_tridiagonal(d, e, eigvals_only=True)
    tn = np.max(np.abs(d) + np.r_[0, np.abs(e)] + np.r_[np.abs(e), 0])
    xs = np.concatenate([rng.uniform(w[0] - scale, w[-1] + scale, 200),
                         w[::7] + 1e-9 * tn, w[::7] - 1e-9 * tn])
    assert np.array_equal(_counts(exe, d, e, xs), np.searchsorted(w, xs))
