"""The double-float building blocks of the CUDA library (csrc/dfloat.h), compiled
for the host without floating-point contraction and checked against long double
over random operands, cancellation included.  Bounds in units of 2^-48 (the
precision of a hi + lo pair of FP32 values): the sum relative to |x| + |y|,
products, quotients and roots relative to the exact result."""
import pathlib
import shutil
import subprocess

import pytest

ROOT = pathlib.Path(__file__).resolve().parent.parent
BOUNDS = {"add": 3.0, "norm": 1.0, "mul": 5.0, "div": 10.0, "sqrt": 5.0, "sqr": 5.0, "cmul": 6.0}


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_double_float_error_bounds(tmp_path):
    exe = tmp_path / "dfloat_check"
    subprocess.run(["g++", "-O2", "-ffp-contract=off", "-std=c++17",
                    "-I", str(ROOT / "paper_2512_04447_gb300" / "csrc"),
                    str(ROOT / "tests" / "native" / "dfloat_check.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    worst = {k: float(v) for k, v in (line.split() for line in out.strip().splitlines())}
    assert set(worst) == set(BOUNDS)
    for k, b in BOUNDS.items():
        assert worst[k] <= b, (k, worst[k])
