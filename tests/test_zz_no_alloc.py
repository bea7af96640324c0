"""The allocation-free PCG entry point (ba_pcg_solve_static) through the C ABI.

It serves callers that cannot allocate device memory while they run (a fixed arena, a per-frame loop that
may not call cudaMalloc): its scratch is a fixed array inside the library.  The test solves the reduced
system of a seeded scene with it, twice in a row (the second call reuses the array's leftover contents),
and compares each solution with the solution the library's own step (ba_compute_step) gives for the same
system, at the FP64 parity tolerance of the other tests.  This file is collected last.
"""
import numpy as np
import pytest
import torch

from scenegen import config, make_scene
from tests.helpers import counts, gpu_problem, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_04026_b300 import build
    build.build()
    import paper_2609_04026_b300 as B
    return B


def test_static_pcg_matches_library_step(B):
    s = make_scene(config("small"))
    p = gpu_problem(B, s, precision=B.BA_FP64)
    try:
        B.ba_build_reduced(p, 1e-3)
        rp, cols, vals, b = B.ba_export_reduced_system(p)
        ref = B.ba_compute_step(p, counts(s))
    finally:
        B.ba_destroy(p)
    nc, npl, nv = len(s["cams"]["q"]), len(s["planes"]), len(s["vps"])
    x_ref = np.zeros((nc + npl + nv, 6))
    x_ref[:nc] = ref["cam"]
    x_ref[nc:nc + npl, :3] = ref["plane"]
    x_ref[nc + npl:, :2] = ref["vp"]
    dev = torch.device("cuda")
    cols_d = torch.from_numpy(cols).to(dev)
    vals_d = torch.from_numpy(vals).to(dev)
    b_d = torch.from_numpy(b.reshape(-1).copy()).to(dev)
    for call in range(2):
        x_d = torch.full_like(b_d, 7.0 + call)      # garbage that the solve must overwrite
        it, r = B.ba_pcg_solve_static(rp, cols_d, vals_d, b_d, x_d, rel_tol=1e-6, max_iters=1000)
        torch.cuda.synchronize()
        x = x_d.cpu().numpy().reshape(-1, 6)
        assert abs(it - ref["pcg_iters"]) <= 1, (it, ref["pcg_iters"])
        assert r <= 1e-6
        assert rel(x, x_ref) <= 1e-9, (call, rel(x, x_ref))


def test_static_pcg_rejects_oversize(B):
    """More block rows than the fixed scratch array holds: the library refuses the call (BA_ERR_ARG)."""
    n = 5000
    rp = np.arange(n + 1, dtype=np.int32)
    dev = torch.device("cuda")
    cols = torch.arange(n, dtype=torch.int32, device=dev)
    vals = torch.zeros(36 * n, dtype=torch.float64, device=dev)
    v = torch.zeros(6 * n, dtype=torch.float64, device=dev)
    with pytest.raises(B.BAError) as e:
        B.ba_pcg_solve_static(rp, cols, vals, v, v.clone())
    assert e.value.status == B.BA_ERR_ARG and "4096" in str(e.value)


def test_static_pcg_rejects_indefinite_diagonal_block(B):
    """A diagonal block that is not positive definite makes S indefinite: the call says so (BA_ERR_ARG) and
    does not run CG on it."""
    n = 3
    rp = np.array([0, 2, 4, 5], np.int32)
    cols = np.array([0, 1, 0, 1, 2], np.int32)
    vals = np.zeros((5, 6, 6))
    vals[0] = vals[2] = np.eye(6) * 4.0
    vals[1] = vals[3] = np.eye(6) * 0.5
    vals[4] = np.diag([3.0, 2.0, -1.0, 1.0, 1.0, 1.0])    # indefinite
    dev = torch.device("cuda")
    x_d = torch.zeros(6 * n, dtype=torch.float64, device=dev)
    with pytest.raises(B.BAError) as e:
        B.ba_pcg_solve_static(rp, torch.from_numpy(cols).to(dev), torch.from_numpy(vals.reshape(-1)).to(dev),
                              torch.ones(6 * n, dtype=torch.float64, device=dev), x_d)
    assert e.value.status == B.BA_ERR_ARG and "positive definite" in str(e.value)
