"""The fixed-point Matérn arithmetic of the generation kernel
(paper_2406_02701_gb300/csrc/mp_fixed.cuh), compiled for the host and
checked against long double (tests/fixed_point_check.cpp).  The bounds are
the ones the kernel's accuracy rests on: sqrt within a few units of 2^-63,
e^{-x} within 2^-58 for x <= 100 and 2^-55 up to x = 700, and the whole
entry sigma^2 P(x) e^{-x} within 0.55 + x/128 ulp of its exact value at the
same float64 squared distance (one final rounding, a few units of 2^-63 from
the products, and x's own error of at most 8 units of 2^-63 carried x-fold);
and the refinement's fixed-point copy of Sigma holds round-half-even of
v 2^(62 - E) bit for bit.
"""
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_fixed_point_entry_accuracy(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    if np.finfo(np.longdouble).nmant < 63:
        pytest.skip("long double narrower than 64 bits")
    exe = str(tmp_path / "fixed_point_check")
    r = subprocess.run([cxx, "-O2", "-std=c++17", os.path.join(HERE, "fixed_point_check.cpp"), "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = json.loads(subprocess.run([exe, "2000000"], capture_output=True, text=True, check=True).stdout)
    assert out["sqrt_units"] <= 8, out
    assert out["exp_units"] <= 32, out
    assert out["exp700_units"] <= 256, out
    assert out["entry_ulp"] <= 0.55, out
    assert out["sigma_fix_bad"] == 0, out
