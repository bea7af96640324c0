"""The C-ABI library loads and exports every entry point that include/ba.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ba.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ba_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ("ba_create", "ba_destroy", "ba_add_cameras", "ba_add_features", "ba_add_groups",
              "ba_add_observations", "ba_lm_step", "ba_solve"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2609_04026_b300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_default_options():
    import paper_2609_04026_b300 as B
    o = B.ba_default_options()
    assert (o.w_point, o.w_line, o.w_group, o.w_wire, o.w_vp) == (1.0, 1.0, 0.5, 0.1, 5e3)
    assert (o.cauchy_px, o.cauchy_vp) == (1.0, 0.2)
    assert o.pcg_rel_tol == 1e-6 and o.pcg_max_iters == 1000 and o.lambda0 == 1e-4
    assert ctypes.sizeof(B.ba_options) > 0
