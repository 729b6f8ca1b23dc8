"""Host-side checks of the C-ABI library: it builds for sm_103a, loads, and
exports every entry point include/qpinv.h declares.  No GPU compute here."""
import ctypes
import os
import re

import pytest

from paper_2605_01464_gb300 import build as libbuild
from paper_2605_01464_gb300 import qpinv

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "qpinv.h")


def declared_symbols():
    text = open(HEADER).read()
    return set(re.findall(r"^\s*(?:int|void|const char\*)\s+(qpinv_\w+)\s*\(", text, re.M))


def test_library_builds_and_loads():
    path = libbuild.build()
    assert os.path.exists(path)
    assert qpinv.lib() is not None


def test_every_declared_symbol_is_exported():
    decl = declared_symbols()
    assert {"qpinv_init", "qpinv_solve", "qpinv_solve_batched", "qpinv_free"} <= decl
    L = qpinv.lib()
    for name in decl:
        assert hasattr(L, name), name
    assert decl == set(qpinv.EXPORTS)


def test_default_options():
    o = qpinv.qpinv_default_options()
    assert o.precision == 1 and o.polish_iters == 2 and o.qrapid_N == 5 and o.penrose == 1
    assert o.alpha_mode == 0 and o.side == 0 and o.stop_rule == 1
    # the trailing fields pin the ctypes mirror of the struct layout
    assert o.batched_tile == -1 and o.hyper_order == 19


def test_null_context_is_rejected_without_cuda():
    res = qpinv.qpinv_result()
    p = qpinv.PTR4(1, 2, 3, 4)
    rc = qpinv.qpinv_solve(None, None, 4, 4, p, 4, 3, 1e-10, 10, p, 4, res)
    assert rc == -1
    assert qpinv.lib().qpinv_last_error(None) == b"null context"


def test_init_reports_missing_device_or_succeeds():
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    h = ctypes.c_void_p()
    rc = qpinv.lib().qpinv_init(ctypes.byref(h), 0, None)
    if has_gpu:
        assert rc == 0
        qpinv.lib().qpinv_free(h)
    else:
        assert rc == -2 and not h.value


def test_invalid_options_rejected():
    o = qpinv.qpinv_default_options()
    o.alpha_mode = 3
    o.alpha_user = -1.0
    h = ctypes.c_void_p()
    rc = qpinv.lib().qpinv_init(ctypes.byref(h), 0, ctypes.byref(o))
    assert rc in (-1, -2)  # invalid (or no device, checked first)
