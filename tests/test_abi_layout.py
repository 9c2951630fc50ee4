"""The ctypes structures of the binding against the C header: a small C
program compiled with the host compiler prints sizeof and offsetof of
every field of lqcd_hmc_params, lqcd_hmc_result and lqcd_pf_fields, and
the binding's layout must match it field by field (a field added to one
side only would otherwise shift every later member silently)."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_0710_0066_gb300 import lqcd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = {"lqcd_hmc_params": lqcd.HmcParams, "lqcd_hmc_result": lqcd.HmcResult, "lqcd_pf_fields": lqcd.PfFields}
C_NAME = {"lam": "lambda"}  # Python keyword


def test_struct_layouts_match_the_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lqcd.h"', "int main(void) {"]
    for cname, py in STRUCTS.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, C_NAME.get(f, f)))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = str(tmp_path / "layout")
    subprocess.check_call([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", exe])
    got = dict(line.split() for line in subprocess.check_output([exe], text=True).strip().splitlines())
    for cname, py in STRUCTS.items():
        assert int(got[cname]) == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got["%s.%s" % (cname, f)]) == getattr(py, f).offset, (cname, f)


def test_solver_traffic_is_keyed_to_the_captured_sources(monkeypatch):
    """bench.py reports the ncu DRAM traffic of k_solve only while the
    sources the kernel is built from are the ones that were captured"""
    import hashlib
    import sys

    sys.path.insert(0, ROOT)
    import bench

    h = hashlib.sha256()
    for name in bench.SOLVER_SOURCES:
        with open(os.path.join(ROOT, "paper_0710_0066_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    t, d = bench.solver_traffic()
    if h.hexdigest() == bench.SOLVER_TRAFFIC["src_sha256"]:
        assert t == bench.SOLVER_TRAFFIC["block_series"] and d["global_solve_bicgstab"] == bench.SOLVER_TRAFFIC["glob"]
    else:
        assert t is None and d is None
    monkeypatch.setitem(bench.SOLVER_TRAFFIC, "src_sha256", "0" * 64)
    assert bench.solver_traffic() == (None, None)
