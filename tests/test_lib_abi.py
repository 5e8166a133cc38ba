"""The C-ABI library builds, loads and exports every entry point that
include/wrc.h declares; host-side argument checks need no GPU."""

import ctypes
import os
import re

import pytest

from paper_1604_08159_gb300 import binding as B
from paper_1604_08159_gb300 import build as BLD

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(wrc_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    BLD.build()
    return B.load()


def test_library_exports_every_declared_symbol(lib):
    names = declared_entry_points()
    assert "wrc_create" in names and "wrc_step" in names
    for n in names:
        assert hasattr(lib, n), n
    # and the binding wraps exactly those names
    assert set(B.SIGNATURES) == set(names)


@pytest.mark.parametrize("field,value,msg", [
    ("n0", 6, "power of two"),
    ("J", 0, "J must"),
    ("krylov_m", 40, "krylov_m"),
    ("eps", -1.0, "out of range"),
    ("dt", 0.0, "out of range"),
])
def test_create_rejects_invalid_config_without_gpu(lib, field, value, msg):
    cfg = B.WrcConfig(16, 3, 20, 0, 0, 0, 1e-3, 5000.0, 0.0, 0.0, 0.0, 1e-2)
    setattr(cfg, field, value)
    h = ctypes.c_void_p()
    st = lib.wrc_create(ctypes.byref(cfg), None, ctypes.byref(h))
    assert st == -1 and h.value is None
    assert msg in lib.wrc_last_error(None).decode()


def test_create_rejects_oversized_lattice(lib):
    cfg = B.WrcConfig(32, 8, 20, 0, 0, 0, 1e-3, 5000.0, 0.0, 0.0, 0.0, 1e-2)
    h = ctypes.c_void_p()
    assert lib.wrc_create(ctypes.byref(cfg), None, ctypes.byref(h)) == -1


def test_null_run_handles(lib):
    assert lib.wrc_step(None, 1) == -1
    assert lib.wrc_sync(None) == -1
    lib.wrc_destroy(None)


def test_ensemble_create_rejects_bad_arguments_without_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.wrc_ensemble_create(0, None, None, ctypes.byref(h)) == -1
    a = B.WrcConfig(16, 3, 20, 0, 0, 0, 1e-3, 5000.0, 0.0, 0.0, 0.0, 1e-2)
    b = B.WrcConfig(16, 3, 20, 0, 1, 0, 1e-3, 5000.0, 0.0, 0.0, 0.0, 1e-2)
    arr = (B.WrcConfig * 2)(a, b)
    assert lib.wrc_ensemble_create(2, arr, None, ctypes.byref(h)) == -1
    assert b"precision" in lib.wrc_ensemble_last_error(None)
    assert lib.wrc_ensemble_step(None, 1) == -1
    lib.wrc_ensemble_destroy(None)
