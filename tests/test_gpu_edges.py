"""Edge cases of the step through the C ABI against the FP64 oracle: a problem of lines alone (no point feature,
so the point kernels see nothing), most cameras held whole and the others with some pose components held (the
held components' columns absent from the reduced system, their increments zero), an empty observation batch,
and a camera that sees nothing but lines of a VP group (no pixel of a point)."""
import copy

import numpy as np
import pytest
import torch

from oracle import ba_oracle as O
from scenegen import config, make_scene
from tests.helpers import counts, gpu_problem, gpu_S_dense, oracle_delta_split, oracle_setup, padded_to_oracle_index, \
    rel

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


def _step_parity(B, s, lam=1e-3):
    p = gpu_problem(B, s, pcg_rel_tol=1e-10)
    try:
        E, _ = B.ba_eval_cost(p)
        B.ba_build_reduced(p, lam)
        Sg, bg = gpu_S_dense(B, p)
        out = B.ba_compute_step(p, counts(s))
    finally:
        B.ba_destroy(p)
    st, lay = oracle_setup(s)
    opt = O.Options(pcg_rel_tol=1e-10)
    Eo, _ = O.cost(st, s["obs"], opt)
    assert abs(E - Eo) <= 1e-12 * Eo
    H, g = O.normal_equations(*O.linearize(st, s["obs"], opt, lay))
    So, bo, *_ = O.reduced_system(H, g, lam, lay)
    idx = padded_to_oracle_index(s, lay)
    assert rel(Sg[np.ix_(idx, idx)], So.toarray()) <= FP64_TOL
    assert rel(bg[idx], bo) <= FP64_TOL
    delta, info = O.solve_step(st, s["obs"], opt, lam, lay)
    ref = oracle_delta_split(delta, lay)
    keys = ("cam", "plane", "vp", "point", "line")
    full_g = np.concatenate([out[k].ravel() for k in keys])
    full_o = np.concatenate([ref[k].ravel() for k in keys])
    assert rel(full_g, full_o) <= FP64_TOL
    return out, lay


def test_lines_only(B):
    s = copy.deepcopy(make_scene(config("tiny")))
    s["points"] = np.zeros((0, 3))
    s["gt"]["points"] = np.zeros((0, 3))
    for k, o in s["obs"].items():
        if O.FEAT.get(k) == "point" or k in ("l2p", "wf3d"):   # point features, and records naming a point
            s["obs"][k] = {kk: vv[:0] for kk, vv in o.items()}
    assert len(s["obs"]["line"]["feat"]) > 0
    out, _ = _step_parity(B, s)
    assert out["point"].shape[0] == 0


def test_held_cameras(B):
    s = copy.deepcopy(make_scene(config("tiny")))
    nc = len(s["cams"]["q"])
    fixed = np.full(nc, 0x3F, np.uint8)
    fixed[3] = 0
    fixed[5] = 0b000111        # rotation held, translation free
    fixed[7] = 0b101000        # two translation components held
    s["fixed"] = fixed
    out, lay = _step_parity(B, s)
    for c in range(nc):
        held = [k for k in range(6) if (int(fixed[c]) >> k) & 1]
        assert np.all(out["cam"][c][held] == 0), c
    assert np.abs(out["cam"][3]).max() > 0


def test_empty_observation_batch(B):
    s = make_scene(config("tiny"))
    p = gpu_problem(B, s)
    try:
        z = np.zeros(0, np.int32)
        B.ba_add_observations(p, B.OBS_KINDS["point"], z, z, z, np.zeros((0, 2)))
        E, _ = B.ba_eval_cost(p)
    finally:
        B.ba_destroy(p)
    Eo, _ = O.cost(O.state_from_scene(s), s["obs"], O.Options())
    assert abs(E - Eo) <= 1e-12 * Eo
