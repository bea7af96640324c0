"""Refined intrinsics (cam_dof = 9; Section 3.1, K_c(i)) through the C ABI against the FP64 oracle.

Every camera's (f, k1, k2) is an entity of the reduced system (3 values), one per camera or shared by the
cameras of one camera model (ba_set_intrinsics).  FP64 path at 1e-9 relative: the reduced system S, b with the
intrinsics rows and columns, the step (PCG iterations, every increment including the intrinsics', the predicted
decrease) and an LM run (same decisions, costs, final intrinsics).  The mixed path is compared with the FP64
path on one step (1e-5 relative on S, b, and 1e-3 on the step, as for the rest of the mixed path).
"""
import copy

import numpy as np
import pytest
import torch

from oracle import ba_oracle as O
from scenegen import config, make_scene
from tests.helpers import (counts, gpu_problem, gpu_S_dense, gpu_S_sparse, oracle_delta_split, oracle_setup,
                           padded_to_oracle_index, rel, sparse_rel)

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_04026_b300 import build
    build.build()
    import paper_2609_04026_b300 as B
    return B


_SC = {}


def scene(name, groups, noise=0.01):
    key = (name, groups, noise)
    if key not in _SC:
        _SC[key] = make_scene(config(name, intr_refine=True, intr_groups=groups, intr_noise=noise))
    return _SC[key]


CASES = [("tiny", 0), ("tiny", 3), ("small", 4)]


@pytest.mark.parametrize("name,groups", CASES)
def test_reduced_system_parity_intrinsics(B, name, groups):
    s = scene(name, groups)
    lam = 1e-3
    p = gpu_problem(B, s, cam_dof=9)
    try:
        assert B.ba_intrinsics_count(p) == len(s["intrinsics"]["values"])
        B.ba_build_reduced(p, lam)
        st, lay = oracle_setup(s)
        H, g = O.normal_equations(*O.linearize(st, s["obs"], O.Options(), lay))
        So, bo, *_ = O.reduced_system(H, g, lam, lay)
        if name == "tiny":
            Sg, bg = gpu_S_dense(B, p)
            idx = padded_to_oracle_index(s, lay)
            assert rel(Sg[np.ix_(idx, idx)], So.toarray()) <= FP64_TOL
            assert rel(bg[idx], bo) <= FP64_TOL
        else:
            Sg, bg = gpu_S_sparse(B, p, s, lay)
            assert sparse_rel(Sg, So) <= FP64_TOL
            assert rel(bg, bo) <= FP64_TOL
    finally:
        B.ba_destroy(p)


@pytest.mark.parametrize("name,groups", CASES)
def test_step_parity_intrinsics(B, name, groups):
    """The step at a tight PCG tolerance (1e-10 on both sides): with the intrinsics columns (f in pixels next
    to k1, k2) the reduced system is far less well conditioned than the pose-only one, and two CG runs on the
    same system with different rounding orders part by about the tolerance times its condition; at 1e-6 they
    agreed to 1.3e-6 (same iteration count), at 1e-10 both are the exact step within the parity tolerance."""
    s = scene(name, groups)
    lam = 1e-3
    tol = 1e-10
    p = gpu_problem(B, s, cam_dof=9, pcg_rel_tol=tol)
    try:
        B.ba_build_reduced(p, lam)
        out = B.ba_compute_step(p, counts(s))
        dk = B.ba_get_step_intrinsics(p)
    finally:
        B.ba_destroy(p)
    st, lay = oracle_setup(s)
    delta, info = O.solve_step(st, s["obs"], O.Options(pcg_rel_tol=tol), lam, lay)
    ref = oracle_delta_split(delta, lay)
    assert abs(out["pcg_iters"] - info["pcg_iters"]) <= 2, (out["pcg_iters"], info["pcg_iters"])
    out["intr"] = dk
    keys = ("cam", "plane", "vp", "point", "line", "intr")
    full_g = np.concatenate([out[k].ravel() for k in keys])
    full_o = np.concatenate([ref[k].ravel() for k in keys])
    assert rel(full_g, full_o) <= FP64_TOL, rel(full_g, full_o)
    assert rel(dk, ref["intr"]) <= FP64_TOL, rel(dk, ref["intr"])
    assert abs(out["pred"] - info["pred"]) <= FP64_TOL * abs(info["pred"])


def test_per_camera_default_equals_explicit(B):
    """cam_dof = 9 without ba_set_intrinsics gives every camera its own entity with its own values: the same
    reduced system as the explicit one-entity-per-camera mapping."""
    s = scene("tiny", 0)
    s2 = {k: v for k, v in s.items() if k != "intrinsics"}
    out = []
    for sc in (s, s2):
        p = gpu_problem(B, sc, cam_dof=9)
        try:
            B.ba_build_reduced(p, 1e-3)
            out.append(B.ba_export_reduced_system(p))
        finally:
            B.ba_destroy(p)
    for a, b in zip(out[0], out[1]):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("groups", [0, 3])
def test_lm_trajectory_intrinsics_tiny(B, groups):
    """Twelve LM iterations: the same accept / reject decisions and costs as the oracle, and the same final
    intrinsics of every camera."""
    s = scene("tiny", groups, noise=0.02)
    p = gpu_problem(B, s, cam_dof=9, pcg_rel_tol=1e-10)   # tight CG: see test_step_parity_intrinsics
    reps = []
    try:
        for _ in range(12):
            reps.append(B.ba_lm_step(p).as_dict())
        fk = B.ba_get_intrinsics(p, len(s["cams"]["q"]))
    finally:
        B.ba_destroy(p)
    st, lay = oracle_setup(s)
    opt = O.Options(pcg_rel_tol=1e-10)
    lm = O.LMState(opt.lambda0)
    cur = O.cost(st, s["obs"], opt)
    for i, r in enumerate(reps):
        st, ro = O.lm_step(st, s["obs"], opt, lm, lay, cur)
        assert bool(r["accepted"]) == ro["accepted"], i
        assert abs(r["cost_new"] - ro["E_new"]) <= FP64_TOL * ro["E"], (i, r["cost_new"], ro["E_new"])
        if ro["accepted"]:
            cur = (ro["E_new"], ro["Epx_new"])
    assert sum(r["accepted"] for r in reps) >= 6
    assert rel(fk, st["cams"][:, 7:10]) <= FP64_TOL, rel(fk, st["cams"][:, 7:10])
    # every camera of one model carries its entity's values
    k = s["intrinsics"]["of_cam"]
    assert np.array_equal(fk, st["intr"][k]) or rel(fk, st["intr"][k]) <= FP64_TOL


def test_refined_intrinsics_recover_ground_truth(B):
    """Intrinsics perturbed by 2% in f (k1, k2 by 2e-3, 4e-4) on the small scene (37 cameras in 4 camera models,
    noise and outliers): refining them (cam_dof 9) moves every model's f several times closer to its ground
    truth and ends at a lower cost than holding them (cam_dof 6) from the same start."""
    s = scene("small", 4, noise=0.02)
    res, fk = [], None
    for dof in (6, 9):
        sc = s if dof == 9 else {k: v for k, v in s.items() if k != "intrinsics"}
        p = gpu_problem(B, sc, cam_dof=dof)
        try:
            for _ in range(15):
                B.ba_lm_step(p)
            res.append(B.ba_eval_cost(p)[0])
            if dof == 9:
                fk = B.ba_get_intrinsics(p, len(s["cams"]["q"]))
        finally:
            B.ba_destroy(p)
    gt = s["gt"]["cams"]["intr"]
    e0 = np.abs(s["cams"]["intr"][:, 0] - gt[:, 0]) / gt[:, 0]
    e1 = np.abs(fk[:, 0] - gt[:, 0]) / gt[:, 0]
    print("cost dof6 / dof9", res, "f error before / after", e0.max(), e1.max())
    assert e1.max() < 0.25 * e0.max(), (e0.max(), e1.max())
    assert res[1] < res[0], res


def test_mixed_step_intrinsics_against_fp64(B):
    """The mixed path (float Jacobians, Schur complement and S) on one step with shared intrinsics: S and b
    within 1e-5 of the FP64 path, the step within 1e-3."""
    s = scene("small", 4)
    lam = 1e-3
    outs = []
    for prec in (0, 1):
        p = gpu_problem(B, s, precision=prec, cam_dof=9)
        try:
            B.ba_build_reduced(p, lam)
            rp, cols, vals, b = B.ba_export_reduced_system(p)
            st = B.ba_compute_step(p, counts(s))
            st["intr"] = B.ba_get_step_intrinsics(p)
            outs.append((vals, b, st))
        finally:
            B.ba_destroy(p)
    (v0, b0, s0), (v1, b1, s1) = outs
    assert rel(v1, v0) <= 1e-5, rel(v1, v0)
    assert rel(b1, b0) <= 1e-5, rel(b1, b0)
    for k in ("cam", "intr", "point"):
        assert rel(s1[k], s0[k]) <= 1e-3, (k, rel(s1[k], s0[k]))


def test_batch_rejects_refined_intrinsics(B):
    s = make_scene(config("tiny", intr_refine=True))
    p = gpu_problem(B, s, cam_dof=9)
    try:
        with pytest.raises(B.BAError) as e:
            B.ba_solve_batch([p], 2)
        assert e.value.status == B.BA_ERR_ARG and "intrinsics" in str(e.value)
    finally:
        B.ba_destroy(p)


def test_set_intrinsics_validation(B):
    s = make_scene(config("tiny"))
    p = gpu_problem(B, s)                       # cam_dof 6
    try:
        with pytest.raises(B.BAError) as e:
            B.ba_set_intrinsics(p, np.ones((2, 3)), np.zeros(10, np.int32))
        assert e.value.status == B.BA_ERR_ARG
    finally:
        B.ba_destroy(p)
    s9 = {k: v for k, v in s.items()}
    p = gpu_problem(B, s9, cam_dof=9)
    try:
        with pytest.raises(B.BAError):
            B.ba_set_intrinsics(p, np.ones((2, 3)), np.full(10, 2, np.int32))   # entity out of range
        B.ba_set_intrinsics(p, np.tile([600.0, 0.0, 0.0], (2, 1)), np.zeros(9, np.int32))  # 9 of 10 cameras
        with pytest.raises(B.BAError) as e:
            B.ba_lm_step(p)
        assert e.value.status == B.BA_ERR_ARG and "intr_of_cam" in str(e.value)
    finally:
        B.ba_destroy(p)
