"""Pins of the CPU oracle to things other than itself (no GPU needed).

Each test ties an oracle function to the paper or to mathematics: hand-worked
closed forms (tests/golden/closed_forms.json), finite differences, algebraic
identities from Appendix B, the first-order expansion of Eq. 9, the dense full
normal-equation solve (the Schur step must equal it, Eq. 3 / Eq. 5), an
independent minimiser (scipy's trust-region Newton method), and invariants (monotone accepted
cost, zero residual at noise-free ground truth, similarity invariance).
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.optimize
import scipy.spatial.transform
import torch

from oracle import ba_oracle as O
from scenegen import config, make_scene, noise_free

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


def _case(name):
    return next(c for c in GOLD["cases"] if c["name"] == name)


def _cam_vec(c):
    return torch.tensor(c["q"] + c["t"] + [c["f"], c["k1"], c["k2"]] + c["pp"], dtype=torch.float64)


@pytest.fixture(scope="module")
def tiny():
    s = make_scene(config("tiny"))
    st = O.state_from_scene(s)
    return s, st, s["fixed"]


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("name", ["point_projection_radial", "point_projection_translated"])
def test_point_projection_closed_form(name):
    c = _case(name)
    cam = _cam_vec(c["cam"])
    R = O.quat_to_R(cam[:4])
    x, z = O.pi_point(R, cam[4:7], cam, torch.tensor(c["X"]))
    np.testing.assert_allclose(x.numpy(), c["pi"], rtol=0, atol=1e-10)


def test_line_rho_closed_form():
    c = _case("line_reprojection_rho")
    cam = _cam_vec(c["cam"])
    R = O.quat_to_R(cam[:4])
    l = O.pi_line(R, cam[4:7], cam, torch.tensor(c["line"]))
    r, _ = O.rho(l, torch.tensor(c["seg"]))
    np.testing.assert_allclose(r.numpy(), c["rho"], atol=1e-10)
    # the displacement vectors do not change when the line's sign flips (Eq. 8 difference well defined)
    r2, _ = O.rho(-l, torch.tensor(c["seg"]))
    np.testing.assert_allclose(r2.numpy(), c["rho"], atol=1e-10)


def test_plane_point_closed_form():
    c = _case("plane_point_projection")
    p = O.plane_project_point(torch.tensor(c["plane"]), torch.tensor(c["X"]))
    np.testing.assert_allclose(p.numpy(), c["proj"], atol=1e-14)


@pytest.mark.parametrize("name", ["plane_line_projection", "plane_line_projection_offset"])
def test_plane_line_closed_form(name):
    c = _case(name)
    L = O.plane_project_line(torch.tensor(c["plane"]), torch.tensor(c["line"]))
    np.testing.assert_allclose(L.numpy(), c["proj"], atol=1e-14)


def test_vp_closed_form():
    c = _case("vp_angle")
    r = torch.linalg.cross(torch.tensor(c["d"]), torch.tensor(c["v"]))
    assert abs(float(torch.linalg.norm(r)) - c["abs"]) < 1e-15


# ---------------------------------------------------------------- Appendix B identities
def test_vp_identity_random():
    """|d x v| = |v - (v.d) d| = sin(theta) for unit d, v (Appendix B, VP)."""
    g = np.random.default_rng(0)
    d = g.normal(size=(200, 3)); d /= np.linalg.norm(d, axis=1, keepdims=True)
    v = g.normal(size=(200, 3)); v /= np.linalg.norm(v, axis=1, keepdims=True)
    a = np.linalg.norm(np.cross(d, v), axis=1)
    b = np.linalg.norm(v - (v * d).sum(1, keepdims=True) * d, axis=1)
    th = np.arccos(np.clip((d * v).sum(1), -1, 1))
    np.testing.assert_allclose(a, b, atol=1e-14)
    np.testing.assert_allclose(a, np.sin(th), atol=1e-12)
    r = O.res_vp(torch.zeros(6), torch.zeros(4), torch.zeros(3), torch.zeros(12),
                 torch.tensor(np.concatenate([d[0], np.cross(np.array([0.3, -1.0, 2.0]), d[0])])),
                 torch.tensor(np.concatenate([v[0], [0.0]])), torch.zeros(4))[0]
    assert abs(float(torch.linalg.norm(r)) - a[0]) < 1e-14


def test_plane_line_projection_properties():
    """m'.d' = 0 (Pluecker constraint), n.d' = 0, points of the projected line lie on the plane, and
    m' = p' x d' for the orthogonal projection p' of a point of the line (Appendix B)."""
    g = np.random.default_rng(1)
    for _ in range(100):
        n = g.normal(size=3); n /= np.linalg.norm(n)
        w = g.normal()
        p = g.normal(size=3) * 2
        d = g.normal(size=3) * g.uniform(0.3, 3)
        m = np.cross(p, d)
        Lp = O.plane_project_line(torch.tensor(np.r_[n, w]), torch.tensor(np.r_[d, m])).numpy()
        d2, m2 = Lp[:3], Lp[3:]
        assert abs(m2 @ d2) < 1e-10 * (1 + np.linalg.norm(m2) * np.linalg.norm(d2))
        assert abs(n @ d2) < 1e-12 * np.linalg.norm(d)
        pp = p - (n @ p + w) * n
        np.testing.assert_allclose(m2, np.cross(pp, d2), atol=1e-10 * (1 + np.linalg.norm(m2)))
        # a point of the projected line: p0 = d' x m' / |d'|^2 satisfies the plane equation
        p0 = np.cross(d2, m2) / (d2 @ d2)
        assert abs(n @ p0 + w) < 1e-9 * (1 + abs(w) + np.linalg.norm(p0))


# ---------------------------------------------------------------- residuals vanish on groups
def test_group_residuals_vanish_on_group():
    """Eq. 7 / Eq. 8: a point or line that lies on its plane gives r_g = 0; Eq. 6: an associated
    line parallel to its VP gives 0; Eq. 11 / 12 vanish for exact junction observations."""
    s = noise_free(config("tiny"))
    st = O.state_from_scene(s)
    for k in ("plane_point", "plane_line", "vp", "p2l", "l2p", "point", "line"):
        r, v = O.residuals(st, s["obs"], k)
        assert v.all()
        assert float(r.abs().max()) < 1e-9, k


def test_noise_free_zero_cost_and_zero_step():
    s = noise_free(config("tiny"))
    st = O.state_from_scene(s)
    opt = O.Options()
    E, Epx = O.cost(st, s["obs"], opt)
    assert E <= 1e-18
    fixed = np.zeros(len(st["cams"]), bool); fixed[0] = True
    lay = O.Layout(st, fixed)
    delta, info = O.solve_step(st, s["obs"], opt, 1e-4, lay)
    assert np.abs(delta).max() < 1e-9


# ---------------------------------------------------------------- Jacobians by finite differences
@pytest.fixture(scope="module")
def tiny_both():
    """The tiny scene with both forms of the plane constraints (group-induced 2D and direct 3D) and two spheres,
    cylinders and cones (Appendix B)."""
    s = make_scene(config("tiny", group_form="both", wire_form="both", n_spheres=2, n_cylinders=2, n_cones=2,
                          n_ellipsoids=2, n_cuboids=2, surf_lines=4))
    return s, O.state_from_scene(s), s["fixed"]


@pytest.mark.parametrize("kind", O.KINDS)
def test_jacobian_finite_differences(tiny_both, kind):
    """Central differences through the retraction x (+) delta agree with the oracle's J."""
    s, st, _ = tiny_both
    o = s["obs"][kind]
    assert len(o["feat"]) > 0
    n = min(40, len(o["feat"]))
    sub = {k: {kk: vv[:n] for kk, vv in o.items()} for k, o in s["obs"].items()}
    r, v, Jc, Jf, Jg = O.residuals(st, sub, kind, with_jac=True)
    cam, feat, grp, meas = O._records(st, sub, kind)
    kf = O.FDOF[O.FEAT[kind]]
    fn = O.RES_FN[kind]
    h = 1e-6
    ng = Jg.shape[2]
    for blk, dim, J in ((0, 6, Jc), (1, kf, Jf), (2, ng, Jg)):
        for j in range(dim):
            def ev(sgn):
                out = []
                for i in range(n):
                    d = [torch.zeros(6), torch.zeros(kf), torch.zeros(ng)]
                    d[blk] = d[blk].clone(); d[blk][j] = sgn * h
                    out.append(fn(d[0], d[1], d[2], cam[i], feat[i], grp[i], meas[i])[0])
                return torch.stack(out)
            fd = (ev(1) - ev(-1)) / (2 * h)
            scale = float(J.abs().max()) + 1e-12
            err = float((fd - J[:, :, j]).abs().max())
            assert err <= 2e-6 * scale + 1e-7, (kind, blk, j, err, scale)


def test_first_order_group_residual():
    """Eq. 9: r_g^(p) = J_i delta + O(|delta|^2) with delta = X - Proj(X), J_i = d pi / d X."""
    s = noise_free(config("tiny"))
    st = O.state_from_scene(s)
    o = s["obs"]["plane_point"]
    i = 3
    cam = torch.tensor(st["cams"][o["cam"][i]])
    P = torch.tensor(st["planes"][o["other"][i]])
    X0 = torch.tensor(st["points"][o["feat"][i]])          # on the plane
    R = O.quat_to_R(cam[:4])
    J = torch.func.jacfwd(lambda X: O.pi_point(R, cam[4:7], cam, X)[0])(X0)
    errs = []
    for eps in (1e-1, 1e-2, 1e-3):
        X = X0 + eps * P[:3]                               # move off the plane along the normal
        delta = X - O.plane_project_point(P, X)
        r = O.pi_point(R, cam[4:7], cam, X)[0] - O.pi_point(R, cam[4:7], cam, O.plane_project_point(P, X))[0]
        lin = J @ delta
        errs.append(float(torch.linalg.norm(r - lin) / torch.linalg.norm(lin)))
    # relative error shrinks linearly with |delta|
    assert errs[1] < errs[0] * 0.2 and errs[2] < errs[1] * 0.2, errs


# ---------------------------------------------------------------- the Schur step equals the full solve
@pytest.mark.parametrize("form", ["2d", "both"])
def test_schur_equals_dense_full_solve(tiny, tiny_both, form):
    s, st, fixed = tiny if form == "2d" else tiny_both
    opt = O.Options(solver="dense")
    lay = O.Layout(st, fixed)
    lam = 1e-3
    Jt, rt = O.linearize(st, s["obs"], opt, lay)
    H, g = O.normal_equations(Jt, rt)
    D = O.damping_diag(H)
    full = np.linalg.solve(H.toarray() + np.diag(lam * D), -g)
    delta, info = O.solve_step(st, s["obs"], opt, lam, lay, (Jt, rt))
    rel = np.linalg.norm(delta - full) / np.linalg.norm(full)
    assert rel < 1e-10, rel
    # predicted decrease: -g.d - 1/2 d^T H d computed two ways
    pred2 = -g @ full - 0.5 * full @ (H @ full)
    assert abs(info["pred"] - pred2) <= 1e-9 * abs(pred2)


def test_pcg_matches_dense_cholesky(tiny):
    s, st, fixed = tiny
    lay = O.Layout(st, fixed)
    Jt, rt = O.linearize(st, s["obs"], O.Options(), lay)
    H, g = O.normal_equations(Jt, rt)
    S, b, *_ = O.reduced_system(H, g, 1e-2, lay)
    Sd = S.toarray()
    assert np.allclose(Sd, Sd.T, atol=1e-9 * np.abs(Sd).max())
    L = np.linalg.cholesky(Sd)                      # S is SPD
    x_chol = np.linalg.solve(L.T, np.linalg.solve(L, b))
    x, it, rel = O.pcg(S, b, lay.a_blocks, 1e-12, 5000)
    assert rel <= 1e-12
    assert np.linalg.norm(b - Sd @ x) <= 1e-11 * np.linalg.norm(b)
    np.testing.assert_allclose(x, x_chol, rtol=0, atol=1e-9 * np.abs(x_chol).max())


# ---------------------------------------------------------------- S sparsity (Section 3.3 / 3.4)
def test_schur_pattern_matches_visibility(tiny):
    """A camera-group block of S is non-zero iff the camera sees a feature associated with the group;
    a camera-camera block iff the two cameras share a feature through any residual (Section 3.3, 3.4)."""
    s, st, fixed = tiny
    lay = O.Layout(st, fixed)
    Jt, rt = O.linearize(st, s["obs"], O.Options(), lay)
    H, g = O.normal_equations(Jt, rt)
    S, *_ = O.reduced_system(H, g, 1e-3, lay)
    Sd = np.abs(S.toarray())
    nc, npl = lay.nc, lay.npl
    # entity sets per feature from the raw observation lists (brute force)
    ent = {}
    for k in O.KINDS:
        o = s["obs"][k]
        ft = O.FEAT[k]
        for i in range(len(o["feat"])):
            key = (ft, int(o["feat"][i]))
            e = ent.setdefault(key, set())
            if O.HAS_CAM[k]:
                e.add(("c", int(o["cam"][i])))
            if k in ("plane_point", "plane_line"):
                e.add(("p", int(o["other"][i])))
            if k == "vp":
                e.add(("v", int(o["other"][i])))
    def col(e):
        t, i = e
        if t == "c":
            c = lay.cam_cols[i][lay.cam_cols[i] >= 0]
            return (None, 0) if len(c) == 0 else (int(c[0]), len(c))
        if t == "p":
            return int(lay.plane_col[i]), 3
        return int(lay.vp_col[i]), 2
    expect = set()
    for es in ent.values():
        for a in es:
            for b in es:
                expect.add((a, b))
    ents = [("c", i) for i in range(nc)] + [("p", i) for i in range(npl)] + [("v", i) for i in range(lay.nv)]
    for a in ents:
        ca = col(a)
        if ca[0] is None:
            continue
        for b in ents:
            cb = col(b)
            if cb[0] is None:
                continue
            blk = Sd[ca[0]:ca[0] + ca[1], cb[0]:cb[0] + cb[1]]
            nz = blk.max() > 0
            if a == b:
                continue
            assert nz == ((a, b) in expect), (a, b)


# ---------------------------------------------------------------- invariants of the LM
def test_lm_accepted_cost_monotone(tiny):
    s, st, fixed = tiny
    _, info = O.solve(st, s["obs"], O.Options(), max_iters=8, fixed=fixed)
    E = [r["E"] for r in info["reports"]]
    assert all(b <= a for a, b in zip(E, E[1:]))
    for r in info["reports"]:
        if r["accepted"]:
            assert r["E_new"] < r["E"]


def _similarity(st, s_, Rs, tp):
    """X -> s R X + t' applied to the whole scene; poses (R_i R^T, s t_i - R_i R^T t')."""
    new = {k: v.copy() for k, v in st.items()}
    new["points"] = s_ * st["points"] @ Rs.T + tp
    Rc = O.quat_to_R(torch.tensor(st["cams"][:, :4])).numpy()
    Rn = Rc @ Rs.T
    new["cams"][:, :4] = O.R_to_quat(Rn)
    new["cams"][:, 4:7] = s_ * st["cams"][:, 4:7] - np.einsum("nij,j->ni", Rn, tp)
    d = st["lines"][:, :3] @ Rs.T
    m = s_ * st["lines"][:, 3:] @ Rs.T + np.cross(tp, d)
    new["lines"] = np.concatenate([d, m], 1)
    n = st["planes"][:, :3] @ Rs.T
    new["planes"] = np.concatenate([n, (s_ * st["planes"][:, 3] - n @ tp)[:, None]], 1)
    new["vps"] = st["vps"] @ Rs.T
    return new


def test_cost_similarity_invariant(tiny):
    """Every residual kind is pixel- or angle-based, so E is unchanged by a similarity of the scene
    (Section 1 / Section 3.3: no scale-dependent 3D terms)."""
    s, st, _ = tiny
    opt = O.Options()
    E0 = O.cost(st, s["obs"], opt)
    Rs = scipy.spatial.transform.Rotation.from_rotvec([0.3, -0.7, 0.2]).as_matrix()
    st2 = _similarity(st, 2.7, Rs, np.array([1.0, -3.0, 0.5]))
    E1 = O.cost(st2, s["obs"], opt)
    assert abs(E1[0] - E0[0]) <= 1e-11 * E0[0]
    assert abs(E1[1] - E0[1]) <= 1e-11 * E0[1]


def test_classical_ba_matches_independent_minimiser():
    """Point-only special case (Eq. 1): the LM's converged cost equals the minimum that scipy's
    trust-region Newton method (exact Hessian) finds for the same robust cost, written directly over
    rotation vectors, translations and points.  Two cameras are held fixed in both, so the
    minimum is isolated."""
    cfg = config("tiny", n_cams=5, n_points=40, n_lines=0, n_planes=0, n_vps=0, n_wire_edges=0,
                 outlier_frac=0.0, seed=11)
    s = make_scene(cfg)
    obs = s["obs"]
    st = O.state_from_scene(s)
    fixed = np.zeros(5, bool); fixed[:2] = True
    st_lm, info = O.solve(st, obs, O.Options(rel_cost_tol=1e-13, solver="dense"), max_iters=300, fixed=fixed)
    assert info["converged"]
    o = obs["point"]
    cam = torch.tensor(st["cams"][o["cam"]]); meas = torch.tensor(o["meas"])
    ci = torch.tensor(o["cam"]).long(); fi = torch.tensor(o["feat"]).long()
    R0 = O.quat_to_R(torch.tensor(st["cams"][:, :4]))
    t0 = torch.tensor(st["cams"][:, 4:7])

    def E(x):
        Rf = torch.linalg.matrix_exp(O.skew(x[:9].reshape(3, 3))) @ R0[2:]
        R = torch.cat([R0[:2], Rf]); t = torch.cat([t0[:2], x[9:18].reshape(3, 3)])
        pi, _ = O.pi_point(R[ci], t[ci], cam, x[18:].reshape(-1, 3)[fi])
        return 0.5 * torch.log1p(((pi - meas) ** 2).sum(-1)).sum()     # w = 1, a = 1

    fg = lambda xn: (float(E(torch.tensor(xn))), torch.func.grad(E)(torch.tensor(xn)).numpy())
    hs = lambda xn: torch.func.hessian(E)(torch.tensor(xn)).numpy()
    x0 = np.concatenate([np.zeros(9), st["cams"][2:, 4:7].ravel(), st["points"].ravel()])
    res = scipy.optimize.minimize(fg, x0, jac=True, hess=hs, method="trust-exact",
                                  options=dict(gtol=1e-11, maxiter=500))
    assert abs(info["E"] - res.fun) <= 1e-8 * res.fun, (info["E"], res.fun)


# ---------------------------------------------------------------- the LM rule (hand-worked values)
# Madsen, Nielsen & Tingleff 2004, Sec. 3.2 (Nielsen's damping update): on acceptance
# lambda <- lambda * max(1/3, 1 - (2 rho - 1)^3) and nu <- 2; on rejection lambda <- lambda nu, nu <- 2 nu.
# Each expected value below is worked by hand from that rule; acceptance needs rho > min_gain (1e-3), and
# lambda is clamped to [1e-12, 1e12].
@pytest.mark.parametrize("lam,nu,gain,E_new,acc,lam_exp,nu_exp", [
    (1e-2, 8.0, 0.75, 1.0, True, 8.75e-3, 2.0),          # 2*0.75-1 = 0.5, cube 0.125 -> factor 0.875; nu reset
    (1e-2, 2.0, 0.25, 1.0, True, 1.125e-2, 2.0),         # (-0.5)^3 = -0.125 -> factor 1.125
    (3e-4, 2.0, 1.0, 1.0, True, 1e-4, 2.0),              # 1 - 1 = 0 -> the floor 1/3
    (1e-2, 2.0, 0.9, 1.0, True, 0.488e-2, 2.0),          # 1 - 0.8^3 = 0.488 (above the floor)
    (1e-2, 2.0, 0.95, 1.0, True, 1e-2 / 3.0, 2.0),       # 1 - 0.9^3 = 0.271 -> the floor 1/3
    (1e-2, 2.0, 0.6, 1.0, True, 0.992e-2, 2.0),          # 1 - 0.2^3 = 0.992
    (1.0, 2.0, 0.0011, 1.0, True, 1.993414509352, 2.0),  # 0.9978^3 = 0.99560484 * 0.9978 = 0.993414509352
    (1e-2, 4.0, 1e-3, 1.0, False, 4e-2, 8.0),            # a tie with min_gain rejects
    (1e-2, 2.0, -0.5, 1.0, False, 2e-2, 4.0),            # a cost increase rejects
    (1e-2, 2.0, 0.8, math.inf, False, 2e-2, 4.0),        # a non-finite candidate rejects whatever the gain
    (1e-12, 2.0, 1.0, 1.0, True, 1e-12, 2.0),            # lower clamp
    (6e11, 2.0, 0.0, 1.0, False, 1e12, 4.0),             # upper clamp on rejection
])
def test_lm_update_hand_worked(lam, nu, gain, E_new, acc, lam_exp, nu_exp):
    opt = O.Options()
    lm = O.LMState(lam, nu)
    assert O.lm_update(lm, gain, E_new, opt) is acc
    assert lm.lam == pytest.approx(lam_exp, rel=1e-12)
    assert lm.nu == nu_exp


def test_lm_update_sequence():
    """Two rejections then an acceptance: nu doubles twice, then the accepted factor applies to the
    grown lambda and nu resets (1e-4 -> 2e-4 -> 8e-4 -> 8e-4 * 0.875 = 7e-4)."""
    opt = O.Options()
    lm = O.LMState(1e-4)
    assert not O.lm_update(lm, -1.0, 1.0, opt)
    assert (lm.lam, lm.nu) == (pytest.approx(2e-4), 4.0)
    assert not O.lm_update(lm, 0.0005, 1.0, opt)
    assert (lm.lam, lm.nu) == (pytest.approx(8e-4), 8.0)
    assert O.lm_update(lm, 0.75, 1.0, opt)
    assert (lm.lam, lm.nu) == (pytest.approx(7e-4, rel=1e-12), 2.0)


def test_pixel_cost_excludes_vp_terms(tiny):
    """E_px is E without the angular VP terms (Section 3.5, Appendix C): moving a VP direction changes E
    through its VP residuals only and leaves E_px unchanged, while moving a point changes both."""
    s, st, _ = tiny
    opt = O.Options()
    E0, P0 = O.cost(st, s["obs"], opt)
    vp_only = sum(float(x) for x in _kind_cost(st, s["obs"], opt, "vp"))
    assert vp_only > 0 and abs((E0 - P0) - vp_only) <= 1e-12 * E0
    st2 = {k: v.copy() for k, v in st.items()}
    v = st2["vps"][0] + np.array([0.02, -0.01, 0.015])
    st2["vps"][0] = v / np.linalg.norm(v)
    E1, P1 = O.cost(st2, s["obs"], opt)
    assert abs(E1 - E0) > 1e-6 * E0
    assert P1 == P0
    st3 = {k: v.copy() for k, v in st.items()}
    st3["points"][0] += 0.05
    E2, P2 = O.cost(st3, s["obs"], opt)
    assert P2 != P0 and abs((E2 - P2) - (E0 - P0)) <= 1e-12 * E0


def _kind_cost(st, obs, opt, kind):
    r, v = O.residuals(st, obs, kind)
    a = opt.scale(kind)
    e = 0.5 * opt.weight(kind) * a * a * torch.log1p((r * r).sum(-1) / (a * a))
    return torch.where(v, e, torch.zeros_like(e))


def test_termination_uses_pixel_cost():
    """The stopping test reads the relative change of E_px, not of E: a step that moves only the VP
    terms a lot still stops, and a step that moves E_px by more than the tolerance does not; a rejected
    step never stops."""
    opt = O.Options()
    assert O.step_converged(dict(accepted=True, E=1e3, E_new=5e2, Epx=100.0, Epx_new=100.0 - 5e-5), opt)
    assert not O.step_converged(dict(accepted=True, E=1e3, E_new=1e3 - 1e-6, Epx=100.0, Epx_new=100.0 - 2e-4), opt)
    assert not O.step_converged(dict(accepted=False, E=1e3, E_new=1e3, Epx=100.0, Epx_new=100.0), opt)
    # a relative change of exactly rel_cost_tol does not stop (strict inequality); 2^-20 is exact in binary
    opt2 = O.Options(rel_cost_tol=2.0 ** -20)
    assert not O.step_converged(dict(accepted=True, E=1.0, E_new=1.0, Epx=1.0, Epx_new=1.0 - 2.0 ** -20), opt2)
    assert O.step_converged(dict(accepted=True, E=1.0, E_new=1.0, Epx=1.0, Epx_new=1.0 - 2.0 ** -21), opt2)


# ---------------------------------------------------------------- inter-group relations (Section 3.2)
def _rel_obs(s):
    return dict(s["obs"], relations=s["relations"])


def test_relation_residual_closed_form():
    """Two unit directions at a hand-set angle theta: orthogonality r = cos(theta), parallelism
    r = a x b = (0, 0, sin(theta)) for a = e_x, b = (cos, sin, 0); plane normals and VPs alike."""
    th = 0.3
    z3 = torch.zeros(3)
    a_pl = torch.tensor([1.0, 0.0, 0.0, 2.0])               # plane x = -2 (n, w)
    b_vp = torch.tensor([math.cos(th), math.sin(th), 0.0, 0.0])
    for ka, kb, ga, gb in ((0, 1, a_pl, b_vp), (1, 0, torch.tensor([1.0, 0, 0, 0]), torch.tensor([math.cos(th), math.sin(th), 0, -1.0])),
                           (1, 1, torch.tensor([1.0, 0, 0, 0]), b_vp), (0, 0, a_pl, torch.tensor([math.cos(th), math.sin(th), 0, 0.5]))):
        r_o = O.res_relation(z3, z3, ga, gb, torch.tensor(ka), torch.tensor(kb), torch.tensor(O.REL_ORTH))
        r_p = O.res_relation(z3, z3, ga, gb, torch.tensor(ka), torch.tensor(kb), torch.tensor(O.REL_PAR))
        np.testing.assert_allclose(r_o.numpy(), [math.cos(th), 0, 0], atol=1e-14)
        np.testing.assert_allclose(r_p.numpy(), [0, 0, math.sin(th)], atol=1e-14)


def test_relation_jacobian_finite_differences():
    """Central differences through the group retractions agree with the relation Jacobians, for every pair of
    group kinds and both relation types."""
    s = make_scene(config("small", relations=True))
    st = O.state_from_scene(s)
    rel = s["relations"]
    assert set(zip(rel["ka"].tolist(), rel["kb"].tolist(), rel["type"].tolist())) >= {(0, 0, 0), (0, 0, 1), (1, 1, 0),
                                                                                       (1, 0, 0), (1, 0, 1)}
    r, Ja, Jb = O.relation_residuals(st, rel, with_jac=True)
    ga, gb, ka, kb, ty = O._rel_records(st, rel)
    h = 1e-6
    for side, J in ((0, Ja), (1, Jb)):
        for j in range(3):
            def ev(sgn):
                d = torch.zeros((len(ka), 3))
                d[:, j] = sgn * h
                z = torch.zeros((len(ka), 3))
                args = (d, z) if side == 0 else (z, d)
                return torch.stack([O.res_relation(args[0][i], args[1][i], ga[i], gb[i], ka[i], kb[i], ty[i])
                                    for i in range(len(ka))])
            fd = (ev(1) - ev(-1)) / (2 * h)
            assert float((fd - J[:, :, j]).abs().max()) <= 1e-7, (side, j)


def test_relations_vanish_at_ground_truth_and_change_only_group_blocks():
    """Manhattan relations hold exactly in the noise-free scene (zero residual, zero added cost); in the
    normal equations they add only to group-group blocks (H_gg) -- the camera and feature blocks of H are
    those of the scene without relations (Section 3.2: no effect on H_ff or the Schur structure)."""
    s = noise_free(config("tiny", relations=True))
    st = O.state_from_scene(s)
    r = O.relation_residuals(st, s["relations"])
    assert float(r.abs().max()) < 1e-12
    s2 = make_scene(config("tiny", relations=True))
    st2 = O.state_from_scene(s2)
    lay = O.Layout(st2, s2["fixed"])
    opt = O.Options()
    H0, _ = O.normal_equations(*O.linearize(st2, s2["obs"], opt, lay))
    H1, _ = O.normal_equations(*O.linearize(st2, _rel_obs(s2), opt, lay))
    d = (H1 - H0).tocoo()
    g0 = lay.plane_col[0] if lay.npl else lay.vp_col[0]
    g1 = lay.na
    nz = np.abs(d.data) > 0
    assert nz.any()
    assert ((d.row[nz] >= g0) & (d.row[nz] < g1) & (d.col[nz] >= g0) & (d.col[nz] < g1)).all()
    E0, P0 = O.cost(st2, s2["obs"], opt)
    E1, P1 = O.cost(st2, _rel_obs(s2), opt)
    assert E1 > E0 and P1 == P0     # angular terms: in E, not in E_px


def test_schur_with_relations_equals_dense_full_solve():
    s = make_scene(config("tiny", relations=True))
    st = O.state_from_scene(s)
    obs = _rel_obs(s)
    opt = O.Options(solver="dense")
    lay = O.Layout(st, s["fixed"])
    lam = 1e-3
    Jt, rt = O.linearize(st, obs, opt, lay)
    H, g = O.normal_equations(Jt, rt)
    D = O.damping_diag(H)
    full = np.linalg.solve(H.toarray() + np.diag(lam * D), -g)
    delta, info = O.solve_step(st, obs, opt, lam, lay, (Jt, rt))
    assert np.linalg.norm(delta - full) / np.linalg.norm(full) < 1e-10


def test_relation_cost_rotation_invariant():
    """The relation residuals compare directions only: a rotation of the whole scene leaves them unchanged."""
    s = make_scene(config("small", relations=True))
    st = O.state_from_scene(s)
    Rs = scipy.spatial.transform.Rotation.from_rotvec([0.4, -0.2, 0.9]).as_matrix()
    st2 = _similarity(st, 1.7, Rs, np.array([0.3, 1.0, -2.0]))
    r1 = O.relation_residuals(st, s["relations"]).norm(dim=-1)
    r2 = O.relation_residuals(st2, s["relations"]).norm(dim=-1)
    assert float((r1 - r2).abs().max()) < 1e-12


# ---------------------------------------------------------------- refined intrinsics (Section 3.1, K_c(i))
def test_intrinsics_derivatives_closed_form():
    """d pi / d (f, k1, k2) of the distorted point projection, and d rho / d (f, k1, k2) of the (undistorted)
    line reprojection, against hand-worked values."""
    c = _case("point_projection_intrinsics_derivatives")
    cam = _cam_vec(c["cam"])
    X = torch.tensor(c["X"])
    fk = O.with_intrinsics_increment(O.res_point)
    z6, z3, z4 = torch.zeros(6), torch.zeros(3), torch.zeros(4)
    J = torch.func.jacfwd(lambda dk: fk(z6, z3, z3, dk, cam, torch.cat([X, z3]), torch.zeros(4), z4)[0])(z3)
    np.testing.assert_allclose(J.numpy(), c["dpi_dfk1k2"], rtol=0, atol=1e-10)
    c = _case("line_reprojection_intrinsics_derivatives")
    cam = _cam_vec(c["cam"])
    fk = O.with_intrinsics_increment(O.res_line)
    seg = torch.tensor(c["seg"])
    r = fk(z6, z4, z3, z3, cam, torch.tensor(c["line"]), torch.zeros(4), seg)[0]
    np.testing.assert_allclose(r.numpy(), c["rho"], atol=1e-10)
    J = torch.func.jacfwd(lambda dk: fk(z6, z4, z3, dk, cam, torch.tensor(c["line"]), torch.zeros(4), seg)[0])(z3)
    np.testing.assert_allclose(J.numpy(), c["drho_dfk1k2"], rtol=0, atol=1e-10)


@pytest.mark.parametrize("kind", [k for k in O.KINDS if O.HAS_CAM[k]])
def test_intrinsics_jacobian_finite_differences(kind):
    """Central differences of the residuals in (f, k1, k2) agree with the oracle's intrinsics Jacobian; the
    line kinds and the wireframe kinds do not depend on k1, k2 (undistorted pinhole pixels)."""
    s = make_scene(config("tiny", intr_refine=True, n_spheres=1, n_cylinders=1, n_cones=1, n_ellipsoids=1,
                          n_cuboids=1, surf_lines=4))
    st = O.state_from_scene(s)
    n = min(40, len(s["obs"][kind]["feat"]))
    assert n > 0
    sub = {k: {kk: vv[:n] for kk, vv in o.items()} for k, o in s["obs"].items()}
    r, v, Jc, Jf, Jg, Jk = O.residuals(st, sub, kind, with_jac=True, with_intr=True)
    cam, feat, grp, meas = O._records(st, sub, kind)
    fk = O.with_intrinsics_increment(O.RES_FN[kind])
    kf = O.FDOF[O.FEAT[kind]]
    # the projections are linear in each of f, k1, k2 alone: central differences are exact up to rounding
    for j, h in ((0, 1e-1), (1, 1e-3), (2, 1e-3)):
        def ev(sgn):
            dk = torch.zeros(3); dk[j] = sgn * h
            return torch.stack([fk(torch.zeros(6), torch.zeros(kf), torch.zeros(Jg.shape[2]), dk, cam[i], feat[i],
                                   grp[i], meas[i])[0] for i in range(n)])
        fd = (ev(1) - ev(-1)) / (2 * h)
        scale = float(Jk[:, :, j].abs().max()) + 1e-12
        assert float((fd - Jk[:, :, j]).abs().max()) <= 2e-6 * scale + 1e-7, (kind, j)
    if kind not in ("point", "plane_point", "sphere_point", "cylinder_point", "cone_point", "ellipsoid_point",
                    "cuboid_point"):
        assert float(Jk[:, :, 1:].abs().max()) == 0.0


def test_shared_intrinsics_normal_equations():
    """Sharing one intrinsics entity among cameras is the per-camera system restricted to equal intrinsics:
    with P the matrix that copies an entity's increment to each of its cameras, H_shared = P^T H_cam P and
    g_shared = P^T g_cam (a plain identity of the chain rule)."""
    s = make_scene(config("tiny", intr_refine=True, intr_groups=3))
    st = O.state_from_scene(s)
    lay = O.Layout(st, s["fixed"])
    s1 = dict(s); ik = s["intrinsics"]
    s1["intrinsics"] = dict(of_cam=np.arange(len(ik["of_cam"]), dtype=np.int32), values=ik["values"][ik["of_cam"]])
    st1 = O.state_from_scene(s1)
    lay1 = O.Layout(st1, s["fixed"])
    assert lay.nk == 3 and lay1.nk == 10
    H, g = O.normal_equations(*O.linearize(st, s["obs"], O.Options(), lay))
    H1, g1 = O.normal_equations(*O.linearize(st1, s1["obs"], O.Options(), lay1))
    P = np.zeros((lay1.n, lay.n))
    keep = np.ones(lay1.n, bool); keep[lay1.intr_col[:, None] + np.arange(3)] = False
    other = np.ones(lay.n, bool); other[lay.intr_col[:, None] + np.arange(3)] = False
    P[np.flatnonzero(keep), np.flatnonzero(other)] = 1.0
    for cam, k in enumerate(ik["of_cam"]):
        for j in range(3):
            P[lay1.intr_col[cam] + j, lay.intr_col[k] + j] = 1.0
    Hd, H1d = H.toarray(), H1.toarray()
    np.testing.assert_allclose(Hd, P.T @ H1d @ P, rtol=0, atol=1e-9 * np.abs(Hd).max())
    np.testing.assert_allclose(g, P.T @ g1, rtol=0, atol=1e-9 * np.abs(g).max())


def test_refined_intrinsics_recovered_noise_free():
    """Noise-free scene, intrinsics perturbed (f by 1%, k1, k2 by 5e-3, 1e-3), one entity per group of
    cameras: LM drives the cost to zero and returns the ground-truth intrinsics."""
    s = noise_free(config("tiny", intr_refine=True, intr_groups=3))
    rng = np.random.default_rng(5)
    v = s["intrinsics"]["values"]
    true = v.copy()
    v[:, 0] *= 1 + 0.01 * rng.normal(size=len(v))
    v[:, 1] += 0.005 * rng.normal(size=len(v))
    v[:, 2] += 0.001 * rng.normal(size=len(v))
    st = O.state_from_scene(s)
    E0 = O.cost(st, s["obs"], O.Options())[0]
    st2, info = O.solve(st, s["obs"], O.Options(rel_cost_tol=1e-12), max_iters=12, fixed=s["fixed"])
    assert E0 > 100 and info["E"] < 1e-12 * E0
    np.testing.assert_allclose(st2["intr"], true, rtol=0, atol=1e-7)
    np.testing.assert_allclose(st2["cams"][:, 7:10], true[s["intrinsics"]["of_cam"]], rtol=0, atol=1e-7)


# ---------------------------------------------------------------- direct 3D group distances (Section 3.2, Table 5)
def test_group3d_closed_forms():
    """Point-to-plane distance n.X + w, and for a line its direction's normal component n.d and the distance of
    its foot point d x m: hand-worked values (plane z = 1)."""
    P = torch.tensor([0.0, 0.0, 1.0, -1.0])
    z3 = torch.zeros(3)
    r, _ = O.res_plane_point3d(torch.zeros(6), z3, z3, torch.zeros(12), torch.tensor([1.0, 2.0, 3.0, 0, 0, 0]), P,
                               torch.zeros(4))
    assert abs(float(r[0]) - 2.0) < 1e-15
    # the x axis lifted to z = 5: d = (1,0,0), m = p x d = (0,5,0), foot (0,0,5): r = (0, 4)
    L = torch.tensor([1.0, 0.0, 0.0, 0.0, 5.0, 0.0])
    r, _ = O.res_plane_line3d(torch.zeros(6), torch.zeros(4), z3, torch.zeros(12), L, P, torch.zeros(4))
    np.testing.assert_allclose(r.numpy(), [0.0, 4.0], atol=1e-14)
    # a line through (0,0,1) with d = (0, 0.6, 0.8): foot (0, -0.48, 0.36) (the point of the line nearest the
    # origin): r = (0.8, 0.36 - 1)
    d = torch.tensor([0.0, 0.6, 0.8])
    L = torch.cat([d, torch.linalg.cross(torch.tensor([0.0, 0.0, 1.0]), d)])
    r, _ = O.res_plane_line3d(torch.zeros(6), torch.zeros(4), z3, torch.zeros(12), L, P, torch.zeros(4))
    np.testing.assert_allclose(r.numpy(), [0.8, 0.36 - 1.0], atol=1e-14)


def test_group3d_zero_on_ground_truth_and_outside_pixel_cost():
    """The 3D distances vanish at the noise-free ground truth; they count in E and not in E_px (moving a plane
    in a scene whose planes enter only through them changes E, not E_px); their weight scales their share."""
    s = noise_free(config("tiny", group_form="3d"))
    st = O.state_from_scene(s)
    for k in ("plane_point3d", "plane_line3d"):
        r, v = O.residuals(st, s["obs"], k)
        assert float(r.abs().max()) < 1e-13
    st2 = {k: v.copy() for k, v in st.items()}
    st2["planes"][0, 3] += 0.05
    E1, Epx1 = O.cost(st, s["obs"], O.Options())
    E2, Epx2 = O.cost(st2, s["obs"], O.Options())
    assert E2 > E1 + 1e-6 and Epx2 == Epx1
    E10, _ = O.cost(st2, s["obs"], O.Options(w_group3d=10.0))
    assert abs((E10 - Epx2) - 10 * (E2 - Epx2)) <= 1e-9 * E10


# ---------------------------------------------------------------- sphere, cylinder, cone (Appendix B, Table 6)
@pytest.mark.parametrize("name,kind", [("sphere_projection", "sphere"), ("cylinder_projection", "cylinder"),
                                       ("cone_projection", "cone")])
def test_surface_projection_closed_forms(name, kind):
    c = _case(name)
    out = O.GROUP_PROJECT[kind](torch.tensor(c["group"]), torch.tensor(c["X"]))
    np.testing.assert_allclose(out.numpy(), c["proj"], atol=1e-14)
    # the projection is idempotent (a point of the surface is its own projection)
    again = O.GROUP_PROJECT[kind](torch.tensor(c["group"]), out)
    np.testing.assert_allclose(again.numpy(), c["proj"], atol=1e-13)


def test_surface_groups_zero_on_ground_truth_and_retractions():
    """Points on their spheres, cylinders and cones have zero group-induced residuals at the noise-free
    ground truth; the retractions keep the radius positive (log space), the axes unit and the cylinder axis a
    Pluecker line (d . m = 0)."""
    s = noise_free(config("tiny", n_spheres=2, n_cylinders=2, n_cones=2))
    st = O.state_from_scene(s)
    for k in ("sphere_point", "cylinder_point", "cone_point"):
        r, v = O.residuals(st, s["obs"], k)
        assert len(r) > 100 and bool(v.all()) and float(r.abs().max()) < 1e-10, k
    d = torch.tensor([0.3, -0.2, 0.1, -5.0, 0.2])
    C = O.cylinder_plus(torch.tensor(st["cylinders"][0]), d)
    assert float(C[6]) > 0 and abs(float(torch.linalg.norm(C[:3])) - 1) < 1e-14
    assert abs(float((C[:3] * C[3:6]).sum())) < 1e-14
    S = O.sphere_plus(torch.tensor(st["spheres"][0]), torch.tensor([0.0, 0, 0, -50.0]))
    assert float(S[3]) > 0
    K = O.cone_plus(torch.tensor(st["cones"][0]), torch.tensor([0.1, 0, 0, 0.4, -0.3, 0.01]))
    assert abs(float(torch.linalg.norm(K[3:6])) - 1) < 1e-14


@pytest.mark.parametrize("name,kind", [("ellipsoid_projection", "ellipsoid"), ("cuboid_projection", "cuboid")])
def test_nine_parameter_group_projections(name, kind):
    """Ellipsoid (scaled-radial) and cuboid (nearest face) projections against hand-worked values, and their
    idempotence."""
    c = _case(name)
    G = torch.tensor(c["group"], dtype=torch.float64)
    for X, P in zip(c["X"], c["proj"]):
        out = O.GROUP_PROJECT[kind](G, torch.tensor(X))
        np.testing.assert_allclose(out.numpy(), P, atol=1e-14)
        np.testing.assert_allclose(O.GROUP_PROJECT[kind](G, out).numpy(), P, atol=1e-13)


def test_nine_parameter_groups_ground_truth_and_retractions():
    """Points on their ellipsoids and cuboids have zero residuals at the noise-free ground truth; the
    retractions keep R a rotation and the semi-axes positive; a 9-parameter group is two entities of A (6 + 3
    columns)."""
    s = noise_free(config("tiny", n_ellipsoids=2, n_cuboids=2))
    st = O.state_from_scene(s)
    for k in ("ellipsoid_point", "cuboid_point"):
        r, v = O.residuals(st, s["obs"], k)
        assert len(r) > 100 and bool(v.all()) and float(r.abs().max()) < 1e-10, k
    E = O.ellipsoid_plus(torch.tensor(st["ellipsoids"][0]), torch.tensor([0.3, -0.2, 0.1, 0.1, 0, 0, -9.0, 0.1, 0.2]))
    R = E[:9].reshape(3, 3)
    assert float((R @ R.T - torch.eye(3)).abs().max()) < 1e-14 and float(E[12:15].min()) > 0
    lay = O.Layout(st, s["fixed"])
    assert np.all(np.diff(lay.gcol["ellipsoid"]) == 6) and np.all(np.diff(lay.gcol2["cuboid"]) == 3)
    assert (6, 6) == (lay.gcol2["ellipsoid"][0] - lay.gcol["ellipsoid"][-1], lay.gcol["cuboid"][0] - lay.gcol2["ellipsoid"][-1] + 3)


# ---------------------------------------------------------------- the 3D wireframe endpoint distance (Fig. 3b)
def test_wf3d_closed_form_and_layout():
    """X x d - m: a point at the origin and the line y = 1 along x (d = (1,0,0), m = p x d = (0,0,-1)) are at
    distance 1, r = (0, 0, 1); a point on the line gives 0.  The points it couples with a line feature are
    entities of A (their columns among the reduced system's), the others stay features."""
    L = torch.tensor([1.0, 0.0, 0.0, 0.0, 0.0, -1.0])
    z = torch.zeros(3)
    r, _ = O.res_wf3d(torch.zeros(6), torch.zeros(4), z, torch.zeros(12), L, torch.zeros(8), torch.zeros(4))
    np.testing.assert_allclose(r.numpy(), [0.0, 0.0, 1.0], atol=1e-15)
    r, _ = O.res_wf3d(torch.zeros(6), torch.zeros(4), z, torch.zeros(12), L,
                      torch.tensor([3.0, 1.0, 0.0, 0, 0, 0, 0, 0]), torch.zeros(4))
    assert float(r.abs().max()) < 1e-15
    s = make_scene(config("tiny", wire_form="3d"))
    st = O.state_from_scene(s)
    lay = O.Layout(st, s["fixed"])
    jp = set(s["obs"]["wf3d"]["other"].tolist())
    assert len(jp) > 10 and all(lay.point_col[j] < lay.na for j in jp)
    assert all(lay.point_col[j] >= lay.na for j in range(lay.np_) if j not in jp)
    noise = noise_free(config("tiny", wire_form="3d"))
    r, v = O.residuals(O.state_from_scene(noise), noise["obs"], "wf3d")
    assert float(r.abs().max()) < 1e-13


# ---------------------------------------------------------------- lines on cuboids (Appendix B)
@pytest.mark.parametrize("R,off,d,p,n_exp,w_exp,m_exp", [
    # unit cube at the origin; a line along x through (0, 0.3, 1.2), 0.2 above the top face z = 1: that face
    # (n = e_z, w = -1), and the projected line through (0, 0.3, 1): m' = (0, 0.3, 1) x e_x = (0, 1, -0.3)
    (np.eye(3), [1, 1, 1, 1, 1, 1], [1, 0, 0], [0, 0.3, 1.2], [0, 0, 1], -1, [0, 1, -0.3]),
    # faces x = 2 and x = 0 (d_0 = 2, d_3 = 0): centre (1, 0, 0); a line along y through (2.1, 0, 0.5), whose
    # point nearest the centre is (2.1, 0, 0.5), 0.1 outside face 0: n = e_x, w = -2, m' = (2, 0, 0.5) x e_y
    (np.eye(3), [2, 1, 1, 0, 1, 1], [0, 1, 0], [2.1, 0, 0.5], [1, 0, 0], -2, [-0.5, 0, 2]),
    # the unit cube turned 90 degrees about z (R e_0 = e_y, R e_1 = -e_x): a line along z through
    # (-1.1, 0.2, 0) is nearest face 1, n = R e_1 = -e_x at -x = 1: w = -1, m' = (-1, 0.2, 0) x e_z = (0.2, 1, 0)
    ([[0, -1, 0], [1, 0, 0], [0, 0, 1]], [1, 1, 1, 1, 1, 1], [0, 0, 1], [-1.1, 0.2, 0], [-1, 0, 0], -1, [0.2, 1, 0]),
])
def test_cuboid_line_face_and_projection(R, off, d, p, n_exp, w_exp, m_exp):
    """Hand-worked face choice (the point of the line nearest the cuboid's centre, then the nearest face) and the
    plane projection of the line onto it (Appendix B)."""
    K = torch.tensor(np.concatenate([np.asarray(R, float).ravel(), np.asarray(off, float)]))
    d = torch.tensor(d, dtype=torch.float64)
    L = torch.cat([d, torch.linalg.cross(torch.tensor(p, dtype=torch.float64), d)])
    P = O.cuboid_line_face(K, L)
    np.testing.assert_allclose(P[:3].numpy(), n_exp, atol=1e-15)
    assert abs(float(P[3]) - w_exp) < 1e-15
    Lp = O.plane_project_line(P, L)
    np.testing.assert_allclose(Lp[:3].numpy(), d.numpy(), atol=1e-15)
    np.testing.assert_allclose(Lp[3:].numpy(), m_exp, atol=1e-14)


def test_cuboid_line_zero_at_ground_truth_and_centre():
    """On the noise-free scene every line on a cuboid face has a zero residual (its face is the nearest one), and
    the centre of a generated cuboid is where scenegen put it."""
    cfg = config("tiny", n_cuboids=2, surf_lines=6)
    s = noise_free(cfg)
    r, v = O.residuals(O.state_from_scene(s), s["obs"], "cuboid_line")
    assert r.shape[0] > 10 and bool(v.all())
    assert float(r.abs().max()) < 1e-10
    K = torch.tensor(O.state_from_scene(s)["cuboids"][0])
    faces_n, faces_w = O.cuboid_faces(K)
    c = O.cuboid_centre(K)
    # the centre lies halfway between opposite faces
    for i in range(3):
        a = float((faces_n[i] * c).sum() + faces_w[i])
        b = float((faces_n[i + 3] * c).sum() + faces_w[i + 3])
        assert abs(a - b) < 1e-12 and a < 0
