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


@pytest.mark.parametrize("order", [1, 5, -1])
def test_create_rejects_unsupported_dd_order(lib, order):
    cfg = B.WrcConfig(16, 3, 20, 0, 0, order, 1e-3, 5000.0, 0.0, 0.0, 0.0, 1e-2)
    h = ctypes.c_void_p()
    assert lib.wrc_create(ctypes.byref(cfg), None, ctypes.byref(h)) == -1
    assert b"DD order" in lib.wrc_last_error(None)


def test_create_rejects_oversized_lattice(lib):
    cfg = B.WrcConfig(32, 8, 20, 0, 0, 0, 1e-3, 5000.0, 0.0, 0.0, 0.0, 1e-2)
    h = ctypes.c_void_p()
    assert lib.wrc_create(ctypes.byref(cfg), None, ctypes.byref(h)) == -1


def test_null_run_handles(lib):
    assert lib.wrc_step(None, 1) == -1
    assert lib.wrc_sync(None, -1) == -1
    assert lib.wrc_set_wait_limit(None, 1.0) == -1
    assert lib.wrc_query_krylov_form(None, None) == -1
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


def _cfg(n0=32, J=2, prec=0, m=30):
    return B.WrcConfig(n0, J, m, 2, prec, 0, 1e-4, 5000.0, 0.17, 0.0, 0.0, 1e-2)


def test_server_estimate_is_host_arithmetic_and_ordered(lib):
    est = {}
    for J in range(2, 8):
        for prec in (0, 1):
            est[J, prec] = B.wrc_server_estimate(_cfg(J=J, prec=prec))
    for J in range(2, 8):
        # FP32 bulk arrays halve most of the footprint
        assert est[J, 1] < est[J, 0]
        if J > 2:
            assert est[J, 0] > est[J - 1, 0]
    # large lattices: the lattice arrays dominate, so doubling NJ takes ~4x
    assert 3.5 < est[7, 0] / est[6, 0] < 4.5
    # a run holds at least its seven bulk lattice arrays and five byte masks
    N = 4096 ** 2
    assert est[7, 0] > (7 * 8 + 5) * N and est[7, 1] > (7 * 4 + 5) * N
    # and 150 GB admits dozens of the largest runs, not thousands
    assert 20 < 150e9 / est[7, 1] < 200
    with pytest.raises(B.WrcError):
        B.wrc_server_estimate(_cfg(n0=6))


@pytest.mark.parametrize("field,value,msg", [
    ("policy", 5, "policy"),
    ("max_slots", 0, "max_slots"),
    ("max_slots", 5000, "max_slots"),
    ("threads_per_block", 96, "threads_per_block"),
    ("points_per_thread", 3, "threads_per_block"),   # shape given by half
    ("hbm_budget_bytes", 0.0, "budget"),
])
def test_server_create_rejects_bad_config_without_gpu(lib, field, value, msg):
    cfg = B.WrcServerConfig(0, 16, 0, 0, 150e9)
    setattr(cfg, field, value)
    h = ctypes.c_void_p()
    assert lib.wrc_server_create(ctypes.byref(cfg), ctypes.byref(h)) == -1
    assert h.value is None
    assert msg in lib.wrc_server_last_error(None).decode()


def test_server_null_handles(lib):
    rid = ctypes.c_int64()
    assert lib.wrc_server_submit(None, None, 1, None, None, None, None, 1, 0.0, ctypes.byref(rid)) == -1
    assert lib.wrc_server_wait(None, -1, 1.0) == -1
    assert lib.wrc_server_query(None, 0, None) == -1
    assert lib.wrc_server_stats(None, None) == -1
    lib.wrc_server_destroy(None)


@pytest.mark.parametrize("changes,msg", [
    (dict(model=2), "unknown model"),
    (dict(model=1, prec=1), "FP64 only"),
    (dict(model=1, sgs=2), "a-priori"),
    (dict(model=1, cpt=-1.0), "cpt"),
    (dict(model=1, coriolis=float("nan")), "cpt"),
])
def test_create_rejects_invalid_exner_config_without_gpu(lib, changes, msg):
    cfg = B.WrcConfig(16, 3, 20, 0, 0, 0, 1e-3, 5000.0, 0.0, 0.0, 0.0, 1e-2)
    for k, v in changes.items():
        setattr(cfg, k, v)
    h = ctypes.c_void_p()
    st = lib.wrc_create(ctypes.byref(cfg), None, ctypes.byref(h))
    assert st == -1 and h.value is None
    assert msg in lib.wrc_last_error(None).decode()


def test_config_struct_layout_matches_the_header():
    # six int32, six doubles, two int32, four doubles: 112 bytes, doubles 8-aligned
    assert ctypes.sizeof(B.WrcConfig) == 112
    assert B.WrcConfig.model.offset == 76 and B.WrcConfig.cpt.offset == 80
