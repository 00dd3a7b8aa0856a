"""Host-side checks of the C-ABI library that need no GPU: it builds, loads,
and exports every function include/bchar.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bchar.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bchar_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("bchar_create_mesh", "bchar_set_velocity", "bchar_step", "bchar_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1908_05834_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_marshals_options_and_status_strings():
    from paper_1908_05834_gb300 import build
    build.build()
    from paper_1908_05834_gb300 import bchar
    o = bchar.default_options()
    assert (o.balls_per_axis, o.n_scale, o.precision) == (2, 10, bchar.FP64)
    assert o.penalty == pytest.approx(1e-7) and o.qp_tol == pytest.approx(1e-14)
    assert bchar.bchar_status_string(0) == b"ok"
    assert b"boundary" in bchar.bchar_status_string(4)
