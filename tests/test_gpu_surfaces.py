"""Spheres, cylinders, cones, ellipsoids and cuboids (Appendix B, Table 6) through the C ABI against the FP64
oracle: the group-induced point residual of Eq. 7 with each type's projection, its 4-, 5- and 6-wide group
blocks in the reduced system (a 9-parameter group as two entities, 6 + 3), the log-space radii and semi-axes,
the cone's half-angle, the cuboid's nearest face, and lines on cuboids (Eq. 8 onto the face nearest the line's
point closest to the cuboid's centre).  FP64 path at 1e-9: cost (1e-12), S and b, the
step and the predicted decrease, and an LM run with the oracle's decisions; the mixed step within 1e-5 (S, b)
and 1e-3 (step) of FP64; refusals (batched windows, refined intrinsics, bad parameters)."""
import numpy as np
import pytest
import torch

from oracle import ba_oracle as O
from scenegen import config, make_scene
from tests.helpers import counts, gpu_problem, gpu_S_dense, gpu_S_sparse, oracle_delta_split, oracle_setup, \
    padded_to_oracle_index, rel, sparse_rel

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


def scene(name):
    if name not in _SC:
        kw = dict(n_spheres=2, n_cylinders=2, n_cones=2, n_ellipsoids=2, n_cuboids=2, surf_lines=6) \
            if name == "tiny" else \
            dict(n_spheres=3, n_cylinders=3, n_cones=3, n_ellipsoids=3, n_cuboids=3, surf_points=150, surf_lines=30)
        _SC[name] = make_scene(config(name, **kw))
    return _SC[name]


@pytest.mark.parametrize("name", ["tiny", "small"])
def test_surface_cost_and_reduced_system(B, name):
    s = scene(name)
    lam = 1e-3
    p = gpu_problem(B, s)
    try:
        E, Epx = B.ba_eval_cost(p)
        B.ba_build_reduced(p, lam)
        st, lay = oracle_setup(s)
        Eo, Epxo = O.cost(st, s["obs"], O.Options())
        assert abs(E - Eo) <= 1e-12 * Eo and abs(Epx - Epxo) <= 1e-12 * Epxo, (E, Eo)
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


@pytest.mark.parametrize("name", ["tiny", "small"])
def test_surface_step(B, name):
    s = scene(name)
    lam = 1e-3
    tol = 1e-10
    p = gpu_problem(B, s, pcg_rel_tol=tol)
    try:
        B.ba_build_reduced(p, lam)
        out = B.ba_compute_step(p, counts(s))
        na, _ = B.ba_reduced_size(p)
    finally:
        B.ba_destroy(p)
    st, lay = oracle_setup(s)
    delta, info = O.solve_step(st, s["obs"], O.Options(pcg_rel_tol=tol), lam, lay)
    ref = oracle_delta_split(delta, lay)
    assert abs(out["pcg_iters"] - info["pcg_iters"]) <= 2, (out["pcg_iters"], info["pcg_iters"])
    keys = ("cam", "plane", "vp", "point", "line")
    full_g = np.concatenate([out[k].ravel() for k in keys])
    full_o = np.concatenate([ref[k].ravel() for k in keys])
    assert rel(full_g, full_o) <= FP64_TOL, rel(full_g, full_o)
    assert abs(out["pred"] - info["pred"]) <= FP64_TOL * abs(info["pred"])


def test_surface_lm_trajectory(B):
    """Ten LM iterations with the oracle's decisions and costs; the final spheres, cylinders and cones equal
    the oracle's (radii in log space, the cylinder axis a Pluecker line)."""
    s = scene("tiny")
    opt = O.Options(pcg_rel_tol=1e-10)
    p = gpu_problem(B, s, pcg_rel_tol=1e-10)
    try:
        reps = [B.ba_lm_step(p).as_dict() for _ in range(10)]
        got = {k: B.ba_get_groups(p, kind, len(s[k])) for k, kind in
               (("spheres", B.BA_SPHERE), ("cylinders", B.BA_CYLINDER), ("cones", B.BA_CONE),
                ("ellipsoids", B.BA_ELLIPSOID), ("cuboids", B.BA_CUBOID))}
    finally:
        B.ba_destroy(p)
    st, lay = oracle_setup(s)
    lm = O.LMState(opt.lambda0)
    cur = O.cost(st, s["obs"], opt)
    for i, r in enumerate(reps):
        st, ro = O.lm_step(st, s["obs"], opt, lm, lay, cur)
        assert bool(r["accepted"]) == ro["accepted"], i
        assert abs(r["cost_new"] - ro["E_new"]) <= FP64_TOL * ro["E"], (i, r["cost_new"], ro["E_new"])
        if ro["accepted"]:
            cur = (ro["E_new"], ro["Epx_new"])
    assert sum(r["accepted"] for r in reps) >= 5
    for k in ("spheres", "cylinders", "cones"):
        assert rel(got[k], st[k]) <= FP64_TOL, (k, rel(got[k], st[k]))
    for k in ("ellipsoids", "cuboids"):
        # the library returns (quaternion, 6 values), the oracle keeps (R, 6 values)
        R = O.quat_to_R(torch.from_numpy(got[k][:, :4])).numpy().reshape(-1, 9)
        assert rel(np.concatenate([R, got[k][:, 4:]], 1), st[k]) <= FP64_TOL, k


def test_surface_mixed_step_against_fp64(B):
    s = scene("small")
    lam = 1e-3
    outs = []
    for prec in (0, 1):
        p = gpu_problem(B, s, precision=prec)
        try:
            B.ba_build_reduced(p, lam)
            rp, cols, vals, b = B.ba_export_reduced_system(p)
            outs.append((vals, b, B.ba_compute_step(p, counts(s))))
        finally:
            B.ba_destroy(p)
    (v0, b0, s0), (v1, b1, s1) = outs
    assert rel(v1, v0) <= 1e-5, rel(v1, v0)
    assert rel(b1, b0) <= 1e-5, rel(b1, b0)
    for k in ("cam", "point", "line"):
        assert rel(s1[k], s0[k]) <= 1e-3, (k, rel(s1[k], s0[k]))


def test_surface_refusals(B):
    s = scene("tiny")
    p = gpu_problem(B, s)
    try:
        with pytest.raises(B.BAError) as e:
            B.ba_solve_batch([p], 2)
        assert e.value.status == B.BA_ERR_ARG and "cylinder" in str(e.value)
    finally:
        B.ba_destroy(p)
    p = gpu_problem(B, s, cam_dof=9)
    try:
        with pytest.raises(B.BAError) as e:
            B.ba_lm_step(p)
        assert e.value.status == B.BA_ERR_ARG and "intrinsics" in str(e.value)
    finally:
        B.ba_destroy(p)
    bad = dict(s)
    bad["spheres"] = s["spheres"].copy()
    bad["spheres"][0, 3] = -1.0
    p = gpu_problem(B, bad)
    try:
        with pytest.raises(B.BAError) as e:
            B.ba_lm_step(p)
        assert e.value.status == B.BA_ERR_ARG and "radius" in str(e.value)
    finally:
        B.ba_destroy(p)
