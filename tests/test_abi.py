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


def test_raw_pointer_calls_check_their_tensors():
    """The calls that take raw device pointers (no lengths cross the ABI) refuse tensors of the wrong dtype,
    size, layout or device with BA_ERR_ARG in the binding, before anything reaches the library."""
    import numpy as np
    import torch
    import paper_2609_04026_b300 as B
    n, nnz = 3, 5
    rp = np.array([0, 2, 3, 5], np.int32)
    good = dict(cols=torch.zeros(nnz, dtype=torch.int32), vals=torch.zeros(nnz * 36, dtype=torch.float64),
                b=torch.zeros(6 * n, dtype=torch.float64), x=torch.zeros(6 * n, dtype=torch.float64))
    bad = [("cols", torch.zeros(nnz, dtype=torch.int64), "dtype"),
           ("cols", torch.zeros(nnz - 1, dtype=torch.int32), "elements"),
           ("vals", torch.zeros(nnz * 36, dtype=torch.float32), "dtype"),
           ("vals", torch.zeros(nnz * 35, dtype=torch.float64), "elements"),
           ("b", torch.zeros(6 * n - 1, dtype=torch.float64), "elements"),
           ("x", torch.zeros(6 * n, 2, dtype=torch.float64)[:, 0], "contiguous"),
           ("x", torch.zeros(6 * n, dtype=torch.float64), "CUDA")]
    for name, t, why in bad:
        args = dict(good)
        args[name] = t
        with pytest.raises(B.BAError) as e:
            B.ba_pcg_solve_static(rp, **args)
        assert e.value.status == B.BA_ERR_ARG
        assert why in str(e.value) or name in str(e.value), (name, why, str(e.value))
    with pytest.raises(B.BAError) as e:
        B.ba_pcg_solve_static(rp.astype(np.int64), **good)
    assert e.value.status == B.BA_ERR_ARG
    with pytest.raises(B.BAError) as e:
        B.ba_pcg_solve_static(np.array([0, 2, 2, 5], np.int32), **good)
    assert e.value.status == B.BA_ERR_ARG and "diagonal" in str(e.value)
    P = B.ba_precond_param_count()
    f32 = dict(dtype=torch.float32)      # explicit: another module may change torch's default dtype
    X, E = torch.zeros(4, 32, **f32), torch.zeros(4, 21, **f32)
    m = torch.zeros(4, dtype=torch.uint8)
    zp = lambda k: torch.zeros(k, **f32)
    for args in [(X.double(), E, m, zp(P)), (X, E[:3], m, zp(P)), (X, E, m.int(), zp(P)), (X, E, m, zp(P - 1)),
                 (X, E, m, zp(P))]:
        with pytest.raises(B.BAError) as e:
            B.ba_mlp_grad(*args)
        assert e.value.status == B.BA_ERR_ARG
    with pytest.raises(B.BAError) as e:
        B.ba_precond_train(X, E, m, zp(P), zp(P - 64), zp(P - 66), 0, 1, 4, 1e-3)
    assert e.value.status == B.BA_ERR_ARG and "adam_v" in str(e.value)
