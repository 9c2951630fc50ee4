"""The double-float arithmetic of the mixed-precision path's double sweeps
(csrc/lqcd_df.cuh), compiled for the host and checked against long-double
arithmetic: the integer split of a double is exact to 2^-46, sums and
products of two df numbers, a complex three-term row product (the link
multiplication) and a 48-term unnormalised chain (one output component
of a hopping sweep) keep about 44-46 bits, the way back to double is exact, and
zeros, infinities, NaN and tiny values split as documented.  These bounds
make the double sweeps' results agree with FP64 to ~1e-14 relative, far
below the 1e-10 residual the solves are run to."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_0710_0066_gb300", "csrc")


def test_df_arithmetic(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "df_check")
    subprocess.check_call([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-D__host__=", "-D__device__=",
                           "-D__forceinline__=inline", "-I", CSRC, os.path.join(HERE, "df_check", "df_check.cpp"),
                           "-o", exe, "-lm"])
    out = subprocess.check_output([exe], text=True)
    r = {k: float(v) for k, v in (line.split() for line in out.strip().splitlines())}
    assert r["split"] <= 2.0 ** -46
    assert r["add"] <= 2.0 ** -45
    assert r["mul"] <= 2.0 ** -44
    assert r["dot"] <= 2.0 ** -44
    assert r["chain"] <= 2.0 ** -43
    assert r["back"] == 0.0
    assert r["lo_ulp"] <= 1.0
    assert r["special"] == 0
