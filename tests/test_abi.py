"""Host-side checks of the C-ABI library (no GPU needed): it loads and
exports every entry point that include/lqcd.h declares, and the binding
covers the same names."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "lqcd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lqcd_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_0710_0066_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path_calls():
    names = declared()
    for n in ["lqcd_dslash_eo", "lqcd_block_dslash", "lqcd_block_solve_batched",
              "lqcd_schur_apply", "lqcd_pf_force", "lqcd_hmc_trajectory"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_0710_0066_gb300 import lqcd

    assert sorted(lqcd.EXPORTS) == declared()
    for n in declared():
        assert callable(getattr(lqcd, n))


def test_create_rejects_bad_geometry_without_gpu(lib):
    # geometry is validated on the host before any CUDA call
    h = ctypes.c_void_p()
    bad = [((4, 4, 4, 4), 3), ((6, 4, 4, 4), 2), ((4, 3, 4, 4), 1), ((4, 4, 4, 4), 0)]
    for L, l0 in bad:
        st = lib.lqcd_create(ctypes.byref(h), (ctypes.c_int * 4)(*L), l0, -1, None)
        assert st == -2, (L, l0, st)
    st = lib.lqcd_create(ctypes.byref(h), (ctypes.c_int * 4)(4, 4, 4, 4), 1, 3, None)
    assert st == -1


def test_create_rejects_oversized_lattice_without_gpu(lib):
    # 128 x 128^2 x 64 sites exceed the 32-bit index range of the internal
    # fields: rejected on the host
    h = ctypes.c_void_p()
    st = lib.lqcd_create(ctypes.byref(h), (ctypes.c_int * 4)(128, 128, 128, 64), 8, -1, None)
    assert st == -2


def test_static_gauge_action_validates_on_the_host(lib):
    f = lib.lqcd_gauge_action_static
    f.argtypes = [ctypes.POINTER(ctypes.c_int * 4), ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                  ctypes.c_void_p]
    dummy = ctypes.c_void_p(16)  # never dereferenced: every case fails before any device access
    ok_L = (ctypes.c_int * 4)(4, 4, 4, 4)
    assert f(ctypes.byref(ok_L), None, 5.6, dummy, None) == -1
    assert f(ctypes.byref(ok_L), dummy, 5.6, None, None) == -1
    assert f(ctypes.byref((ctypes.c_int * 4)(4, 3, 4, 4)), dummy, 5.6, dummy, None) == -2
    # more than 2,097,152 sites: beyond the fixed partial-sum array
    assert f(ctypes.byref((ctypes.c_int * 4)(128, 32, 32, 32)), dummy, 5.6, dummy, None) == -2
    # extents whose 64-bit product would overflow (2^30 each: 2^120 sites)
    # or wrap to a small value are rejected before any multiplication
    big = 1 << 30
    assert f(ctypes.byref((ctypes.c_int * 4)(big, big, big, big)), dummy, 5.6, dummy, None) == -2
    assert f(ctypes.byref((ctypes.c_int * 4)(2, 2, 2, 2147483646)), dummy, 5.6, dummy, None) == -2
    assert f(ctypes.byref((ctypes.c_int * 4)(4194304, 2, 2, 2)), dummy, 5.6, dummy, None) == -2


def test_null_handle_is_an_argument_error(lib):
    for name, args in [("lqcd_set_gauge", [None, None]), ("lqcd_launch_count", [None, None]),
                       ("lqcd_set_subslabs", [None, 0]), ("lqcd_set_global_solver", [None, 3, 4]),
                       ("lqcd_set_solver_schedule", [None, 0]), ("lqcd_set_cluster_series", [None, 1]),
                       ("lqcd_set_wait_limit", [None, ctypes.c_int64(0)])]:
        assert getattr(lib, name)(*args) == -1, name
