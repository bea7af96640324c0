"""GPU parity of the inter-group relations (Section 3.2, Inter-Group Relations; Appendix C): orthogonality and
parallelism between plane normals and VP directions, which add only to the group-group blocks of S and to
g_g, to E (not E_px) and to the predicted decrease.  The library against the oracle on the same seeded scenes
with Manhattan relations: cost (1e-12), S and b (1e-9), the step and the predicted decrease (1e-9), and LM
iterations from the same state (same decision, cost 1e-9)."""
import numpy as np
import pytest
import torch

from oracle import ba_oracle as O
from scenegen import config, make_scene
from tests.helpers import counts, gpu_problem, gpu_S_dense, oracle_delta_split, oracle_setup, padded_to_oracle_index, rel

pytestmark = pytest.mark.gpu
TOL = 1e-9


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_04026_b300 import build
    build.build()
    import paper_2609_04026_b300 as B
    return B


def _obs(s):
    return dict(s["obs"], relations=s["relations"])


@pytest.mark.parametrize("name", ["tiny", "small"])
def test_relations_cost_and_reduced_system(B, name):
    s = make_scene(config(name, relations=True))
    assert len(s["relations"]["a"]) > 0
    lam = 1e-3
    p = gpu_problem(B, s)
    try:
        E, Epx = B.ba_eval_cost(p)
        B.ba_build_reduced(p, lam)
        Sg, bg = gpu_S_dense(B, p)
    finally:
        B.ba_destroy(p)
    st, lay = oracle_setup(s)
    opt = O.Options()
    Eo, Epxo = O.cost(st, _obs(s), opt)
    E0, _ = O.cost(st, s["obs"], opt)
    assert Eo > E0
    assert abs(E - Eo) <= 1e-12 * Eo and abs(Epx - Epxo) <= 1e-12 * Epxo, (E, Eo, Epx, Epxo)
    Jt, rt = O.linearize(st, _obs(s), opt, lay)
    H, g = O.normal_equations(Jt, rt)
    So, bo, *_ = O.reduced_system(H, g, lam, lay)
    idx = padded_to_oracle_index(s, lay)
    assert rel(Sg[np.ix_(idx, idx)], So.toarray()) <= TOL
    assert rel(bg[idx], bo) <= TOL


def test_relations_step_parity(B):
    s = make_scene(config("small", relations=True))
    lam = 1e-3
    p = gpu_problem(B, s)
    try:
        B.ba_build_reduced(p, lam)
        out = B.ba_compute_step(p, counts(s))
    finally:
        B.ba_destroy(p)
    st, lay = oracle_setup(s)
    delta, info = O.solve_step(st, _obs(s), O.Options(), lam, lay)
    ref = oracle_delta_split(delta, lay)
    assert out["pcg_iters"] == info["pcg_iters"]
    keys = ("cam", "plane", "vp", "point", "line")
    assert rel(np.concatenate([out[k].ravel() for k in keys]), np.concatenate([ref[k].ravel() for k in keys])) <= TOL
    assert abs(out["pred"] - info["pred"]) <= TOL * abs(info["pred"])


def test_relations_lm_steps_match_oracle(B):
    """Six LM iterations, each compared with the oracle's iteration from the library's state (parameters read
    back, damping set), with PCG run far below its default tolerance on both sides."""
    s = make_scene(config("tiny", relations=True))
    tight = 1e-11
    p = gpu_problem(B, s, pcg_rel_tol=tight, pcg_max_iters=3000)
    try:
        for _ in range(6):
            cams = B.ba_get_cameras(p, len(s["cams"]["q"]))
            st = O.state_from_scene(s)
            st["cams"][:, :7] = cams
            st["points"] = B.ba_get_features(p, B.BA_POINT, len(s["points"]))
            st["lines"] = B.ba_get_features(p, B.BA_LINE, len(s["lines"]))
            st["planes"] = B.ba_get_groups(p, B.BA_PLANE, len(s["planes"]))
            st["vps"] = B.ba_get_groups(p, B.BA_VP, len(s["vps"]))
            lam, nu = B.ba_get_lm_state(p)
            r = B.ba_lm_step(p)
            lay = O.Layout(st, s["fixed"])
            opt = O.Options(pcg_rel_tol=tight, pcg_max_iters=3000)
            _, rep = O.lm_step(st, _obs(s), opt, O.LMState(lam, nu), lay)
            assert bool(r.accepted) == rep["accepted"]
            assert abs(r.cost - rep["E"]) <= TOL * rep["E"]
            assert abs(r.cost_new - rep["E_new"]) <= TOL * rep["E"]
    finally:
        B.ba_destroy(p)


def test_relations_rejected_in_batch_and_invalid_ids(B):
    s = make_scene(config("tiny", relations=True))
    p = gpu_problem(B, s)
    try:
        with pytest.raises(B.BAError) as e:
            B.ba_solve_batch([p], lm_iters=1, autotune=False)
        assert e.value.status == B.BA_ERR_ARG and "relations" in str(e.value)
    finally:
        B.ba_destroy(p)
    q = B.ba_create(B.ba_default_options())
    try:
        B.load_scene(q, make_scene(config("tiny")))
        B.ba_add_relations(q, [B.BA_PLANE], [0], [B.BA_VP], [99], [B.BA_REL_PARALLEL])
        with pytest.raises(B.BAError) as e:
            B.ba_lm_step(q)
        assert e.value.status == B.BA_ERR_ARG
    finally:
        B.ba_destroy(q)
