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


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors in the binding have the size and field offsets of
    the structs include/qpinv.h declares, as a C compiler lays them out."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = [qpinv.qpinv_options, qpinv.qpinv_result, qpinv.qpinv_stats, qpinv.qpinv_cur_result,
               qpinv.qpinv_krylov_result]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "qpinv.h"', "int main(void) {"]
    for S in mirrors:
        name = S.__name__
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for field, _ in S._fields_:
            lines.append(f'  printf("{name}.{field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = dict(line.rsplit(" ", 1) for line in out.strip().splitlines())
    for S in mirrors:
        name = S.__name__
        assert int(got[name]) == ctypes.sizeof(S), name
        for field, _ in S._fields_:
            assert int(got[f"{name}.{field}"]) == getattr(S, field).offset, (name, field)
