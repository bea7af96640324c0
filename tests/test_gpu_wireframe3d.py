"""The 3D wireframe endpoint distance X x d - m (the form Section 3.3 sets against the projected wireframe
residuals of Eq. 11 / Eq. 12) through the C ABI against the FP64 oracle.  Every point it names is an entity of
the reduced system, so these cases check the coupled points' blocks of S (their own residuals' direct blocks
with cameras and planes, the lines' eliminated couplings with them), b, the step (the coupled points' increments
come out of the reduced solve, the other points' out of the back-substitution) and an LM run with the oracle's
decisions; alone (form "3d"), beside the 2D form ("both") and with the direct 3D plane distances on the same
points, at weights 1 and 100."""
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


def scene(name, form, group_form="2d"):
    key = (name, form, group_form)
    if key not in _SC:
        _SC[key] = make_scene(config(name, wire_form=form, group_form=group_form))
    return _SC[key]


CASES = [("tiny", "3d", "2d", 1.0), ("tiny", "both", "2d", 100.0), ("tiny", "both", "both", 1.0),
         ("small", "3d", "2d", 100.0), ("small", "both", "2d", 1.0)]


@pytest.mark.parametrize("name,form,gform,w", CASES)
def test_wf3d_cost_and_reduced_system(B, name, form, gform, w):
    s = scene(name, form, gform)
    lam = 1e-3
    p = gpu_problem(B, s, w_wire3d=w)
    try:
        E, Epx = B.ba_eval_cost(p)
        B.ba_build_reduced(p, lam)
        st, lay = oracle_setup(s)
        assert len(lay.jpoints) > 0
        opt = O.Options(w_wire3d=w)
        Eo, Epxo = O.cost(st, s["obs"], opt)
        assert abs(E - Eo) <= 1e-12 * Eo and abs(Epx - Epxo) <= 1e-12 * Epxo, (E, Eo, Epx, Epxo)
        H, g = O.normal_equations(*O.linearize(st, s["obs"], opt, lay))
        So, bo, *_ = O.reduced_system(H, g, lam, lay)
        if name == "tiny":
            Sg, bg = gpu_S_dense(B, p)
            idx = padded_to_oracle_index(s, lay)
            assert len(idx) == So.shape[0]
            assert rel(Sg[np.ix_(idx, idx)], So.toarray()) <= FP64_TOL
            assert rel(bg[idx], bo) <= FP64_TOL
        else:
            Sg, bg = gpu_S_sparse(B, p, s, lay)
            assert sparse_rel(Sg, So) <= FP64_TOL
            assert rel(bg, bo) <= FP64_TOL
    finally:
        B.ba_destroy(p)


@pytest.mark.parametrize("name,form,gform,w", CASES)
def test_wf3d_step(B, name, form, gform, w):
    s = scene(name, form, gform)
    lam = 1e-3
    p = gpu_problem(B, s, w_wire3d=w)
    try:
        B.ba_build_reduced(p, lam)
        out = B.ba_compute_step(p, counts(s))
    finally:
        B.ba_destroy(p)
    st, lay = oracle_setup(s)
    delta, info = O.solve_step(st, s["obs"], O.Options(w_wire3d=w), lam, lay)
    ref = oracle_delta_split(delta, lay)
    assert abs(out["pcg_iters"] - info["pcg_iters"]) <= 1, (out["pcg_iters"], info["pcg_iters"])
    keys = ("cam", "plane", "vp", "point", "line")
    full_g = np.concatenate([out[k].ravel() for k in keys])
    full_o = np.concatenate([ref[k].ravel() for k in keys])
    assert rel(full_g, full_o) <= FP64_TOL, rel(full_g, full_o)
    # the coupled points' increments (reduced solve) on their own
    jp = lay.jpoints
    assert rel(out["point"][jp], ref["point"][jp]) <= FP64_TOL
    assert abs(out["pred"] - info["pred"]) <= FP64_TOL * abs(info["pred"])


def test_wf3d_lm_trajectory(B):
    s = scene("tiny", "3d")
    opt = O.Options(w_wire3d=100.0)
    p = gpu_problem(B, s, w_wire3d=100.0)
    try:
        reps = [B.ba_lm_step(p).as_dict() for _ in range(10)]
        pts = B.ba_get_features(p, B.BA_POINT, len(s["points"]))
    finally:
        B.ba_destroy(p)
    st, lay = oracle_setup(s)
    lm = O.LMState(opt.lambda0)
    cur = O.cost(st, s["obs"], opt)
    for i, r in enumerate(reps):
        st, ro = O.lm_step(st, s["obs"], opt, lm, lay, cur)
        assert bool(r["accepted"]) == ro["accepted"], i
        assert abs(r["cost_new"] - ro["E_new"]) <= FP64_TOL * ro["E"], (i, r["cost_new"], ro["E_new"])
        assert abs(r["cost_px_new"] - ro["Epx_new"]) <= FP64_TOL * ro["E"], i
        if ro["accepted"]:
            cur = (ro["E_new"], ro["Epx_new"])
    assert sum(r["accepted"] for r in reps) >= 5
    # the coupled points moved as the oracle's did
    Xo = np.asarray(st["points"])
    assert rel(pts[lay.jpoints], Xo[lay.jpoints]) <= 1e-7


def test_wf3d_mixed_precision_converges(B):
    s = scene("small", "both")
    p = gpu_problem(B, s, precision=B.BA_MIXED, w_wire3d=100.0)
    try:
        rep = B.ba_solve(p).as_dict()
    finally:
        B.ba_destroy(p)
    assert rep["cost"] < 0.5 * rep["cost0"], rep
    assert rep["accepted_steps"] >= 3, rep


def test_wf3d_refused_with_refined_intrinsics(B):
    s = scene("tiny", "3d")
    p = gpu_problem(B, s, cam_dof=9)
    try:
        with pytest.raises(Exception, match="wireframe"):
            B.ba_eval_cost(p)
    finally:
        B.ba_destroy(p)
