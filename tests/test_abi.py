"""The C-ABI library builds for sm_103a, loads, and exports every entry point ``include/vofp.h`` declares.

No compute call is made here (no GPU on the build machine)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names.update(re.findall(r"\b(vofp_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1907_00890_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_library_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert "vofp_plan_create" in names and "vofp_project" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol(lib):
    from paper_1907_00890_gb300 import vofp
    for n in declared_symbols():
        assert n in vofp.EXPORTED or n.startswith("vofp_batch") or n.startswith("vofp_server") or \
            n.startswith("vofp_tune") or n.startswith("vofp_") and hasattr(vofp, n), n


def test_error_strings_and_default_opts(lib):
    from paper_1907_00890_gb300 import vofp
    assert vofp.vofp_error_string(0) == "ok"
    assert "invalid" in vofp.vofp_error_string(-1)
    o = vofp.vofp_opts_default()
    assert o.prec == 0 and o.tol == 1e-10 and o.max_refine == 3


def test_sm103a_only_build_flags():
    from paper_1907_00890_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_entry_points_refuse_a_null_plan_on_the_host(lib):
    """Argument checks run on the host before any CUDA call: a NULL plan is INVALID_ARG (-1) everywhere."""
    P, D = ctypes.c_void_p, ctypes.c_double
    lib.vofp_project_vd.argtypes = [P] * 8 + [D] * 4 + [P] * 3
    lib.vofp_project_vd.restype = ctypes.c_int
    assert lib.vofp_project_vd(None, None, None, None, None, None, None, None, 1e-3, 1e-3, 1.0, 1.0, None, None,
                               None) == -1
    for name in ("vofp_extend_liquid_velocity", "vofp_extend_vapour_velocity"):
        f = getattr(lib, name)
        f.argtypes = [P] * 6 + [D] * 2 + [P] * 9
        f.restype = ctypes.c_int
        assert f(None, None, None, None, None, None, 100.0, 1.0, None, None, None, None, None, None, None, None,
                 None) == -1
    lib.vofp_project.argtypes = [P] * 5 + [D] + [P] * 3
    lib.vofp_project.restype = ctypes.c_int
    assert lib.vofp_project(None, None, None, None, None, 1.0, None, None, None) == -1
    lib.vofp_vof_update.argtypes = [P] * 5 + [D] + [P] * 3
    lib.vofp_vof_update.restype = ctypes.c_int
    assert lib.vofp_vof_update(None, None, None, None, None, 0.01, None, None, None) == -1


def test_bounds_checked_library_builds_and_exports_the_same_symbols():
    """The -DVOFP_CHECKED variant compiles for sm_103a and exports every declared entry point as well."""
    from paper_1907_00890_gb300 import build
    lib_c = ctypes.CDLL(build.build(checked=True))
    missing = [n for n in declared_symbols() if not hasattr(lib_c, n)]
    assert not missing, missing


def test_plain_library_check_word_is_zero_without_a_device_call(lib):
    """The plain library has no check words: status 0, zeros, and no CUDA call (this machine has no GPU)."""
    lib.vofp_debug_check_word.argtypes = [ctypes.POINTER(ctypes.c_longlong), ctypes.c_int]
    lib.vofp_debug_check_word.restype = ctypes.c_int
    w = (ctypes.c_longlong * 4)(7, 7, 7, 7)
    assert lib.vofp_debug_check_word(w, 1) == 0
    assert list(w) == [0, 0, 0, 0]
    assert lib.vofp_debug_check_word(None, 0) == -1
