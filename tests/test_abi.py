"""The C-ABI library builds, loads without a GPU, and exports every entry point
that include/tbr.h declares; host-side argument checks fail without touching
the device."""
import ctypes
import os
import re

import pytest

from paper_2609_08722_b300 import tbr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tbr.h")


def declared_symbols():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"TBR_API\s+[\w\s\*]+?\b(tbr_\w+)\s*\(", src)))


def test_header_declares_the_entry_points():
    names = declared_symbols()
    assert "tbr_render_hard" in names and "tbr_render_backward" in names
    assert sorted(tbr.EXPORTED) == names


def test_library_exports_every_declared_symbol():
    lib = tbr.lib()
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_version_string():
    assert "sm_103a" in tbr.version()


def test_invalid_arguments_fail_on_the_host():
    lib = tbr.lib()
    s = tbr.TbrProgram()
    s.n, s.k = 3, 0            # k < 1
    s.color_temp = 1.0
    rc = lib.tbr_render_hard(ctypes.byref(s), 8, 8, -1, 0, None, None, None, None)
    assert rc == tbr.TBR_ERR_INVALID_ARG
    assert b"palette size" in lib.tbr_last_error()
    s.k = 2
    rc = lib.tbr_render_hard(ctypes.byref(s), 0, 8, -1, 0, ctypes.c_void_p(16), None, None, None)
    assert rc == tbr.TBR_ERR_INVALID_ARG
    opts = tbr.TbrSoftOpts(0.1, 0.0, 0, 0, 0)   # tau_min must be > 0
    s.cx = s.cy = s.theta = s.length = s.half_width = s.logits = s.palette = ctypes.c_void_p(256)
    rc = lib.tbr_render_soft(ctypes.byref(s), 8, 8, ctypes.byref(opts), ctypes.c_void_p(256), None, None)
    assert rc == tbr.TBR_ERR_INVALID_ARG
    assert lib.tbr_render_backward(None, None, None, None, None, None, None, None, None, None) == \
        tbr.TBR_ERR_INVALID_ARG
    assert lib.tbr_loss_mse(None, None, 4, None, None, None) == tbr.TBR_ERR_INVALID_ARG
    rate, ms = ctypes.c_double(), ctypes.c_double()
    tbr._fit_lib()
    assert lib.tbr_measure_peak(7, 10, ctypes.byref(rate), ctypes.byref(ms), None) == tbr.TBR_ERR_INVALID_ARG
    assert lib.tbr_measure_peak(0, 0, ctypes.byref(rate), None, None) == tbr.TBR_ERR_INVALID_ARG
