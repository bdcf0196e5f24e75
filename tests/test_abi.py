"""C ABI checks that need no GPU: the library builds, loads, exports every
symbol include/pfb.h declares, and rejects invalid arguments before touching
the device."""

import ctypes
import os
import re

import pytest

import paper_2408_16551_gb300 as pkg
from paper_2408_16551_gb300 import build as pbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    pbuild.build()
    return pkg.lib()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"PFB_API\s+[\w\s\*]*?\b(pfb_\w+)\s*\(", src))
    return names


def test_header_declares_entry_points():
    names = _declared()
    for must in ("pfb_plan_create", "pfb_execute", "pfb_submit", "pfb_poll", "pfb_execute_batch"):
        assert must in names


def test_every_declared_symbol_is_exported(L):
    missing = [n for n in sorted(_declared()) if not hasattr(L, n)]
    assert not missing, missing
    assert set(pkg.EXPORTED) == _declared()


def test_status_strings(L):
    assert L.pfb_status_string(0) == b"PFB_OK"
    assert L.pfb_status_string(-1) == b"PFB_ERR_INVALID"
    assert L.pfb_status_string(-7) == b"PFB_ERR_UNSUPPORTED"


def _desc(**kw):
    d = pkg.pfb_plan_desc()
    d.P, d.T, d.in_dtype, d.in_scale, d.window, d.path, d.device, d.reserved = 64, 4, 1, 1.0, 0, 0, -1, 0
    for k, v in kw.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("bad", [dict(P=0), dict(P=48), dict(P=8192), dict(T=0), dict(T=65), dict(in_dtype=3),
                                 dict(window=4), dict(window=3), dict(path=3), dict(reserved=1),
                                 dict(in_dtype=2, in_scale=float("inf")), dict(hop=3), dict(hop=-2), dict(hop=65),
                                 dict(hop=1), dict(in_dtype=2, hop=4), dict(P=4096, hop=64), dict(tap_order=2),
                                 dict(tap_order=-1)])
def test_plan_create_rejects_invalid_descriptors(L, bad):
    h = ctypes.c_void_p()
    st = L.pfb_plan_create(ctypes.byref(_desc(**bad)), ctypes.byref(h))
    assert st == pkg.PFB_ERR_INVALID
    assert not h.value
    assert L.pfb_last_error()


def test_null_arguments(L):
    assert L.pfb_plan_create(None, None) == pkg.PFB_ERR_INVALID
    assert L.pfb_execute(None, None, 0, None, 0, None) == pkg.PFB_ERR_INVALID
    assert L.pfb_out_spectra(None, 10) == -1
    assert L.pfb_plan_destroy(None) == pkg.PFB_OK
    assert L.pfb_batch_destroy(None) == pkg.PFB_OK
    assert L.pfb_server_destroy(None) == pkg.PFB_OK
    assert L.pfb_poll(None, 1) == pkg.PFB_ERR_INVALID
    assert L.pfb_execute_batch(None, -1, None) == pkg.PFB_ERR_INVALID
    assert L.pfb_plan_kernel_name(None) == b""


@pytest.mark.parametrize("bad", [dict(hbm_budget_bytes=0), dict(max_slots=0), dict(max_slots=65),
                                 dict(timeout_ms=0), dict(queue_when_busy=2)])
def test_server_create_rejects_invalid(L, bad):
    d = pkg.pfb_server_desc(1 << 30, 4, 1000, 1, -1)
    for k, v in bad.items():
        setattr(d, k, v)
    h = ctypes.c_void_p()
    assert L.pfb_server_create(ctypes.byref(d), ctypes.byref(h)) == pkg.PFB_ERR_INVALID
    assert not h.value


def test_struct_layouts():
    assert ctypes.sizeof(pkg.pfb_plan_desc) == 48
    assert ctypes.sizeof(pkg.pfb_batch_item) == 40
    assert ctypes.sizeof(pkg.pfb_server_desc) == 24
    assert ctypes.sizeof(pkg.pfb_server_stats) == 11 * 8 + 3 * 8
