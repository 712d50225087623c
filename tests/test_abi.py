"""C ABI checks that need no GPU: the library builds and loads, exports every entry point that
include/wos.h declares, the binding declares exactly those, and argument validation in host
code rejects bad calls before any CUDA work."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wos.h")


def declared_entry_points():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:wos_status|const\s+char\s*\*)\s*(wos_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2406_01713_gb300 import _lib, build

    build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for core in ["wos_domain_create", "wos_domain_destroy", "wos_solve", "wos_grad", "wos_plan_step",
                 "wos_plan_path", "wos_solve_batch", "wos_backward", "wos_status_string"]:
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_entry_points():
        assert hasattr(lib, name), name


def test_binding_declares_exactly_the_header(lib):
    from paper_2406_01713_gb300 import _lib

    assert sorted(_lib.SIGNATURES) == declared_entry_points()


def test_status_strings(lib):
    assert lib.wos_status_string(0) == b"ok"
    assert lib.wos_status_string(1) == b"invalid argument"
    assert lib.wos_status_string(99) == b"unknown status"


def test_domain_create_rejects_bad_descriptions(lib):
    from paper_2406_01713_gb300 import _lib

    h = ctypes.c_void_p()
    assert lib.wos_domain_create(None, ctypes.byref(h)) == 1
    s = _lib.DomainDesc()
    s.d = 13
    assert lib.wos_domain_create(ctypes.byref(s), ctypes.byref(h)) == 2  # unsupported d
    assert b"d = 13" in lib.wos_last_error()
    s.d = 3
    assert lib.wos_domain_create(ctypes.byref(s), ctypes.byref(h)) == 1  # no box, no outer ball
    lo = np.zeros(3)
    hi = np.ones(3)
    P = ctypes.POINTER(ctypes.c_double)
    s.box_lo = lo.ctypes.data_as(P)
    s.box_hi = hi.ctypes.data_as(P)
    c = np.zeros(3)
    r = np.array([-1.0])
    s.n_balls = 1
    s.ball_c = c.ctypes.data_as(P)
    s.ball_r = r.ctypes.data_as(P)
    assert lib.wos_domain_create(ctypes.byref(s), ctypes.byref(h)) == 1  # radius <= 0
    assert h.value is None
    s.n_balls = 0
    s.n_exp = 9
    assert lib.wos_domain_create(ctypes.byref(s), ctypes.byref(h)) == 2  # too many exp terms
    s.n_exp = 0
    s.proj_dims = 4
    assert lib.wos_domain_create(ctypes.byref(s), ctypes.byref(h)) == 1  # proj_dims > d
    assert b"proj_dims" in lib.wos_last_error()
    s.proj_dims = 2
    pts = np.zeros((4, 3))
    s.n_points = 4
    s.points = pts.ctypes.data_as(P)
    assert lib.wos_domain_create(ctypes.byref(s), ctypes.byref(h)) == 2  # extruded point set
    assert h.value is None


def test_calls_reject_null_handles(lib):
    assert lib.wos_solve(None, None, None, 1, 10, 1e-3, 1.0, None, None, None, None) == 1
    assert lib.wos_batch_run(None, None, None) == 1
    assert lib.wos_domain_destroy(None) == 0
    assert lib.wos_batch_destroy(None) == 0
    assert lib.wos_backward(None, None, None, None, -1, 2, 0, None, None, None, None) == 1
    assert lib.wos_debug_philox(0, 0, -1, 0, 0, None, None) == 1


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2406_01713_gb300 import _lib

    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.load()
