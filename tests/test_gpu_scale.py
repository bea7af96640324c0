"""GPU parity at the size of the benchmark's reduced system, and the mixed path's error stated per result.

The `pcgprof` scene has the benchmark's cameras and groups -- 2000 cameras, 300 planes and 200 VPs, so the
reduced system has the same 2500 block rows and a pattern of the same density (1.29M stored blocks) -- with a
tenth of its features (2.05M residuals), so that the FP64 oracle builds one LM step in about a minute.  At this
size the library cuts long block rows between the CTAs of the persistent PCG, splits thousands of Schur blocks
over several work units and streams S through L2 with part of it kept resident: paths the small scenes of
tests/test_gpu_parity.py do not reach.

Each stage is checked against the oracle from the same input, at the same damping (1e-4, the initial LM
damping).  FP64 path: cost and candidate cost (1e-12), S and b (1e-9, relative to the largest entry), the
PCG step by its exact residual in the oracle's S (the stopping tolerance 1e-6, with the drift of the
recurrence residual), the back-substituted features and the predicted decrease from the library's own step
(1e-9); with both sides' PCG run to 1e-12 the steps agree to 1e-8.  The step after a fixed number of CG
iterations is not compared at 1e-9: the library runs CG in the Chronopoulos-Gear form and the oracle in the
textbook form, whose iterates agree only up to rounding amplified over ~90 iterations (6e-8 measured).
Mixed path (FP32 Jacobians, Schur complement and SpMV; FP64 landmark inverses, cost and accept test): each
result's relative error against the same oracle values is printed and bounded.
"""
import numpy as np
import pytest
import torch

from oracle import ba_oracle as O
from scenegen import config, make_scene
from tests.helpers import counts, gpu_problem, gpu_S_sparse, oracle_delta_split, oracle_setup, rel, sparse_rel

pytestmark = pytest.mark.gpu

LAM = 1e-4
FP64_TOL = 1e-9
# bounds of the mixed path's per-result error (the benchmark spec's tolerances apply to the final cost and RMS,
# checked in test_gpu_parity.py and by bench.py; these guard the intermediate results)
MIXED_BOUND = dict(S=1e-5, b=1e-5, pcg_true_residual=2e-5, backsub=1e-3, pred=1e-6, cost=1e-12, cost_new=1e-9,
                   delta_vs_same_iterations=1e-2)


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_04026_b300 import build
    build.build()
    import paper_2609_04026_b300 as B
    return B


@pytest.fixture(scope="module")
def ref():
    s = make_scene(config("pcgprof"))
    st, lay = oracle_setup(s)
    opt = O.Options()
    E, Epx = O.cost(st, s["obs"], opt)
    Jt, rt = O.linearize(st, s["obs"], opt, lay)
    H, g = O.normal_equations(Jt, rt)
    S, b, Hffi, Haf, _ = O.reduced_system(H, g, LAM, lay)
    return dict(s=s, st=st, lay=lay, opt=opt, E=E, Epx=Epx, Jt=Jt, g=g, S=S, b=b, Hffi=Hffi, Haf=Haf)


def _oracle_step(ref, iters):
    """The oracle's step after exactly `iters` CG iterations from x0 = 0 (block-Jacobi), back-substituted."""
    lay, g = ref["lay"], ref["g"]
    da, it, _ = O.pcg(ref["S"], ref["b"], lay.a_blocks, 0.0, iters)
    na = lay.na
    df = -(ref["Hffi"] @ (g[na:] + ref["Haf"].T @ da))
    delta = np.concatenate([da, df])
    Jd = ref["Jt"] @ delta
    pred = -float(g @ delta) - 0.5 * float(Jd @ Jd)
    return delta, pred


def _gpu_run(B, ref, precision):
    s = ref["s"]
    p = gpu_problem(B, s, precision=precision)
    try:
        E, Epx = B.ba_eval_cost(p)
        B.ba_build_reduced(p, LAM)
        Sg, bg = gpu_S_sparse(B, p, s, ref["lay"])
        out = B.ba_compute_step(p, counts(s))
        st = B.ba_lm_step(p)          # rebuilds the same system at the initial damping and evaluates the step
    finally:
        B.ba_destroy(p)
    return dict(E=E, Epx=Epx, S=Sg, b=bg, out=out, step=st)


def _errors(ref, g):
    """Each stage against the oracle from the same input: S and b and the cost from the scene; the PCG step
    by its exact residual in the oracle's S (and, for information, against the oracle's iterate after as many
    CG iterations); back-substitution, predicted decrease and candidate cost from the library's own step."""
    lay, opt = ref["lay"], ref["opt"]
    na = lay.na
    keys = ("cam", "plane", "vp", "point", "line")
    out = g["out"]
    # the library's full increment in the oracle's column order
    full = np.zeros(ref["Jt"].shape[1])
    full[lay.cam_cols[lay.cam_cols >= 0]] = out["cam"][lay.cam_cols >= 0]
    if lay.npl:
        full[lay.plane_col[:, None] + np.arange(3)] = out["plane"]
    if lay.nv:
        full[lay.vp_col[:, None] + np.arange(2)] = out["vp"]
    if lay.np_:
        full[lay.point_col[:, None] + np.arange(3)] = out["point"]
    if lay.nl:
        full[lay.line_col[:, None] + np.arange(4)] = out["line"]
    da = full[:na]
    res = np.linalg.norm(ref["b"] - ref["S"] @ da) / np.linalg.norm(ref["b"])
    df_o = -(ref["Hffi"] @ (ref["g"][na:] + ref["Haf"].T @ da))
    Jd = ref["Jt"] @ full
    pred_o = -float(ref["g"] @ full) - 0.5 * float(Jd @ Jd)
    E_new_o = O.cost(O.apply_step(ref["st"], full, lay), ref["s"]["obs"], opt)[0]
    delta_k, _ = _oracle_step(ref, out["pcg_iters"])
    return dict(S=sparse_rel(g["S"], ref["S"]), b=rel(g["b"], ref["b"]), cost=abs(g["E"] - ref["E"]) / ref["E"],
                pcg_true_residual=res, backsub=rel(full[na:], df_o),
                pred=abs(out["pred"] - pred_o) / abs(pred_o),
                cost_new=abs(g["step"].cost_new - E_new_o) / E_new_o,
                delta_vs_same_iterations=rel(full, delta_k))


def test_fp64_parity_at_2000_cameras(B, ref):
    g = _gpu_run(B, ref, B.BA_FP64)
    _, it_o, _ = O.pcg(ref["S"], ref["b"], ref["lay"].a_blocks, 1e-6, 1000)
    assert abs(g["out"]["pcg_iters"] - it_o) <= 1, (g["out"]["pcg_iters"], it_o)
    err = _errors(ref, g)
    print("FP64 path against the oracle at 2000 cameras:", {k: f"{v:.2e}" for k, v in err.items()})
    assert err["cost"] <= 1e-12 and err["cost_new"] <= 1e-12, err
    for k in ("S", "b", "backsub", "pred"):
        assert err[k] <= FP64_TOL, (k, err)
    assert err["pcg_true_residual"] <= 2e-6, err
    # the CG iterate itself: the library runs CG in the Chronopoulos-Gear form, the oracle in the textbook
    # form; both give the same iterates in exact arithmetic, and their rounding differs by ~1e-16 per step
    assert err["delta_vs_same_iterations"] <= 1e-6, err


def test_fp64_step_at_tight_pcg_tolerance(B, ref):
    """Both sides solve the reduced system to a relative residual of 1e-12: the steps then agree to the
    parity tolerance."""
    s = ref["s"]
    p = gpu_problem(B, s, precision=B.BA_FP64, pcg_rel_tol=1e-12, pcg_max_iters=5000)
    try:
        B.ba_build_reduced(p, LAM)
        out = B.ba_compute_step(p, counts(s))
    finally:
        B.ba_destroy(p)
    lay = ref["lay"]
    da, it_o, rel_o = O.pcg(ref["S"], ref["b"], lay.a_blocks, 1e-12, 5000)
    ro = oracle_delta_split(np.concatenate([da, np.zeros(ref["Jt"].shape[1] - lay.na)]), lay)
    keys = ("cam", "plane", "vp")
    dg = np.concatenate([out[k].ravel() for k in keys])
    do = np.concatenate([ro[k].ravel() for k in keys])
    e = rel(dg, do)
    print(f"tight PCG: library {out['pcg_iters']} iterations (rel {out['pcg_rel']:.1e}), oracle {it_o} "
          f"(rel {rel_o:.1e}); step difference {e:.2e}")
    assert e <= FP64_TOL * 10, e


def test_mixed_error_per_result_at_2000_cameras(B, ref):
    g = _gpu_run(B, ref, B.BA_MIXED)
    err = _errors(ref, g)
    print("mixed path against the FP64 oracle at 2000 cameras:", {k: f"{v:.2e}" for k, v in err.items()})
    for k, bound in MIXED_BOUND.items():
        assert err[k] <= bound, (k, err)


def _solve(B, s, precision, **opt):
    p = gpu_problem(B, s, precision=precision, max_lm_iters=400, **opt)
    try:
        r = B.ba_solve(p)
        out = dict(iters=r.iters, converged=r.converged, cost=r.cost, cost_px=r.cost_px,
                   cams=B.ba_get_cameras(p, len(s["cams"]["q"])),
                   points=B.ba_get_features(p, B.BA_POINT, len(s["points"])),
                   lines=B.ba_get_features(p, B.BA_LINE, len(s["lines"])),
                   planes=B.ba_get_groups(p, B.BA_PLANE, len(s["planes"])),
                   vps=B.ba_get_groups(p, B.BA_VP, len(s["vps"])))
    finally:
        B.ba_destroy(p)
    return out


def _state_of(s, sol):
    st = O.state_from_scene(s)
    st["cams"][:, :7] = sol["cams"]   # pose (q, t); the intrinsics are held
    st.update(points=sol["points"], lines=sol["lines"], planes=sol["planes"], vps=sol["vps"])
    return st


def _inlier_rms(s, sol, inl=None):
    """RMS of the point reprojection errors over valid inlier residuals (error below 5 px in the reference
    solution); residuals dropped for a point behind a camera are not counted."""
    r, v = O.residuals(_state_of(s, sol), s["obs"], "point")
    n = np.sqrt((r.numpy() ** 2).sum(1))
    if inl is None:
        inl = (n < 5.0) & v.numpy()
    inl = inl & v.numpy()
    return float(np.sqrt((n[inl] ** 2).mean())), inl


def _scene_from(s, sol):
    """The scene with the solution's parameters as its initial values."""
    s2 = dict(s)
    s2["cams"] = dict(s["cams"], q=sol["cams"][:, :4], t=sol["cams"][:, 4:7])
    s2.update(points=sol["points"], lines=sol["lines"], planes=sol["planes"], vps=sol["vps"])
    return s2


def test_medium_scene_fp64_and_mixed_to_convergence(B):
    """The medium scene (200 cameras, 100k points, 20k lines, 30 planes + 20 VPs, sigma 0.5 px) in FP64 and
    on the mixed path, both run to a relative cost change of 1e-9 (so that they reach a minimum rather than two
    points of plain IRLS's slow linear tail).
    Without outliers: inlier reprojection RMS within 1e-4 px of the FP64 path's (measured 1e-6 px), and final
    costs within 3e-4 relative of each other.  Both paths stop in IRLS's slow tail, where an accepted step of
    relative change below 1e-9 can come early or late with the rounding of the cost sums: the mixed path ended
    1.6e-5 below the FP64 path with one summation order of the FP64 cost pass, 2.2e-5 above it with another, and
    1.3e-4 above it (113 against 379 iterations) with the point and plane-induced records evaluated in pairs
    (measured).
    With its 3% outliers the Cauchy cost has nearby local minima, and which one a path reaches depends on
    rounding (the FP64 and mixed end points differ by 6e-3 px in inlier RMS, measured).  There the mixed end
    point must be a minimum by the FP64 path's standard: FP64 iterations continued from it converge, move the
    inlier RMS by at most 1e-4 px and lower the cost by at most 3e-4 relative (measured: 4 to 24 iterations,
    1e-6 px, 3e-9 to 1e-6 for three builds; 150 iterations of IRLS's slow tail, 0 px and 1.1e-4 for a fourth),
    and its cost is within 1e-3 relative of the FP64 path's own, a nearby minimum (measured 1e-5 below, 3.8e-5,
    2.2e-4 and 2.6e-4 above with four summation orders of the mixed path's products)."""
    clean = make_scene(config("medium", outlier_frac=0.0))
    r64 = _solve(B, clean, B.BA_FP64, rel_cost_tol=1e-9)
    r32 = _solve(B, clean, B.BA_MIXED, rel_cost_tol=1e-9)
    rms64, inl = _inlier_rms(clean, r64)
    rms32, _ = _inlier_rms(clean, r32, inl)
    print(f"medium without outliers: FP64 {r64['iters']} iterations, cost {r64['cost']:.6f}, RMS {rms64:.6f} px; "
          f"mixed {r32['iters']} iterations, cost {r32['cost']:.6f}, RMS {rms32:.6f} px; "
          f"cost rel {abs(r32['cost'] - r64['cost']) / r64['cost']:.2e}")
    assert r64["converged"] and r32["converged"], (r64["iters"], r32["iters"])
    assert abs(r32["cost"] - r64["cost"]) <= 3e-4 * r64["cost"]
    assert abs(rms32 - rms64) <= 1e-4
    s = make_scene(config("medium"))
    m64 = _solve(B, s, B.BA_FP64, rel_cost_tol=1e-9)
    m32 = _solve(B, s, B.BA_MIXED, rel_cost_tol=1e-9)
    p64 = _solve(B, _scene_from(s, m32), B.BA_FP64, rel_cost_tol=1e-9)
    rms_p, inl = _inlier_rms(s, p64)
    rms_m, _ = _inlier_rms(s, m32, inl)
    print(f"medium with outliers: FP64 {m64['iters']} iterations, cost {m64['cost']:.6f}; mixed {m32['iters']} "
          f"iterations, cost {m32['cost']:.6f} (rel {(m32['cost'] - m64['cost']) / m64['cost']:.2e}); FP64 from the "
          f"mixed end point {p64['iters']} iterations, cost {p64['cost']:.6f}, inlier RMS {rms_p:.6f} against "
          f"{rms_m:.6f} px")
    assert m32["converged"] and p64["converged"]
    assert p64["cost"] >= m32["cost"] * (1 - 3e-4)
    assert m32["cost"] <= m64["cost"] * (1 + 1e-3)
    assert abs(rms_p - rms_m) <= 1e-4
