"""Seeded synthetic holistic-BA scenes (inputs only).

This module draws cameras, points, lines, planes, vanishing points, wireframe
edges and their observation lists, shaped like the synthetic benchmark of the
paper's appendix (A.3): a cube of half-extent 3 with Manhattan-aligned planes,
cameras on a sphere (or a ring) looking inwards, features on planes and free,
wireframe grids on planes, pixel noise, outliers and perturbed initial values.

It is shared by the CPU oracle and the CUDA path as *input* only.  To create
measurements it needs to project ground-truth geometry into the images; it does
so with its own small projection helpers below, which neither the oracle nor
the CUDA library uses.  Nothing here linearises, weights or solves anything.

Conventions (all float64):
  cameras:  q [Nc,4] unit quaternion (w,x,y,z) world->camera, t [Nc,3],
            intr [Nc,3] = (f, k1, k2), pp [Nc,2] principal point (pixels).
            x_cam = R(q) X + t, +z forward.
  points:   [Np,3]
  lines:    [Nl,6] Pluecker (d, m), |d| = 1, m = p x d for any p on the line.
  planes:   [Npl,4] (n, w), |n| = 1, plane n.x + w = 0.
  vps:      [Nv,3] unit directions.
  intrinsics (only with refined intrinsics): of_cam [Nc] int32, the intrinsics entity of every camera, and
            values [Nk,3] the entities' initial (f, k1, k2); cams.intr then equals values[of_cam].
Observation kinds (one record per residual):
  point      (cam, point, -, meas 2 distorted pixels)                 Eq. 1/4
  line       (cam, line,  -, meas 4 undistorted segment endpoints)    Eq. 4
  plane_point(cam, point, plane, no meas)                             Eq. 7
  plane_line (cam, line,  plane, meas 4 segment)                      Eq. 8
  vp         (-1,  line,  vp,    no meas)                             Eq. 6
  p2l        (cam, point, line id of partner, meas 4 partner segment) Eq. 11
  l2p        (cam, line,  point id of partner, meas 2 undistorted pt) Eq. 12
  plane_point3d (-1, point, plane, no meas)  direct 3D distance (Section 3.2's alternative, Table 5)
  plane_line3d  (-1, line,  plane, no meas)  direct 3D distances of a line (direction, foot point)
  wf3d          (-1, line,  point, no meas)  3D wireframe endpoint distance X x d - m (Fig. 3b's form)
  sphere_point .. cuboid_point (cam, point, group, no meas)  Eq. 7 with the other group types (Appendix B)
  cuboid_line   (cam, line, cuboid, meas 4 segment)  Eq. 8 onto the cuboid's face nearest the line
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

IMG_W, IMG_H = 800.0, 600.0
HALF = 3.0

KINDS = ("point", "line", "plane_point", "plane_line", "vp", "p2l", "l2p", "plane_point3d", "plane_line3d",
         "sphere_point", "cylinder_point", "cone_point", "ellipsoid_point", "cuboid_point", "wf3d", "cuboid_line")
MEAS_DIM = {"point": 2, "line": 4, "plane_point": 0, "plane_line": 4, "vp": 0, "p2l": 4, "l2p": 2,
            "plane_point3d": 0, "plane_line3d": 0, "sphere_point": 0, "cylinder_point": 0, "cone_point": 0,
            "ellipsoid_point": 0, "cuboid_point": 0, "wf3d": 0, "cuboid_line": 4}


@dataclasses.dataclass
class SceneConfig:
    name: str = "tiny"
    n_cams: int = 10
    ring: bool = True
    n_points: int = 500
    n_lines: int = 100
    n_planes: int = 4
    n_vps: int = 2
    track_min: int = 3
    track_max: int = 6
    track_mean: float = 0.0          # >0: truncated geometric on [track_min, track_max]
    k_near: int = 64
    frac_points_on_plane: float = 0.5
    frac_lines_on_plane: float = 0.5
    frac_lines_vp: float = 0.6
    n_wire_edges: int = 100
    sigma_px: float = 1.0
    outlier_frac: float = 0.05
    rot_noise_deg: float = 1.0
    trans_noise: float = 0.05
    feat_noise: float = 0.1
    group_rot_noise_deg: float = 2.0
    group_off_noise: float = 0.05
    relations: bool = False          # inter-group orthogonality / parallelism that hold in the ground truth
    # refined intrinsics (f, k1, k2 as entities of the reduced system): intr_groups = 0 gives every camera its
    # own entity; g > 0 makes camera i share entity i % g (its ground-truth intrinsics and principal point are
    # those of camera i % g); intr_noise perturbs the initial values (f relative, k1 and k2 scaled)
    intr_refine: bool = False
    intr_groups: int = 0
    intr_noise: float = 0.0
    # form of the positional group constraints: "2d" the group-induced reprojection residuals (Eq. 7, Eq. 8),
    # "3d" the direct 3D distances to the plane instead (the alternative of Section 3.2, compared in Table 5),
    # "both" all of them; the observations are the same draws in every form
    group_form: str = "2d"
    # form of the wireframe constraints: "2d" the cross-feature reprojection residuals (Eq. 11, Eq. 12), "3d"
    # the 3D endpoint distance of each edge instead (the form Fig. 3b compares; it couples the point with the
    # line), "both"
    wire_form: str = "2d"
    # the other group types of Appendix B (spheres, cylinders, cones), each with surf_points points on its
    # surface, drawn with a generator of their own after everything else (the rest of the scene is unchanged)
    n_spheres: int = 0
    n_cylinders: int = 0
    n_cones: int = 0
    n_ellipsoids: int = 0
    n_cuboids: int = 0
    surf_points: int = 60
    # lines on the cuboids' faces (Appendix B's line projection onto the face nearest the line), per cuboid,
    # drawn with a generator of their own after the surface points
    surf_lines: int = 0
    seed: int = 1


def config(name: str, seed: int | None = None, **over) -> SceneConfig:
    """Named workloads.  Sizes follow the five benchmark configurations."""
    if name == "tiny":         # 10 ring cameras, 500 pts, 100 lines, 4 planes, 2 VPs
        c = SceneConfig(name="tiny", seed=1)
    elif name == "small":      # a parity case a few tiles wide with ragged sizes
        c = SceneConfig(name="small", n_cams=37, ring=False, n_points=5003, n_lines=611,
                        n_planes=7, n_vps=4, track_min=2, track_max=9, track_mean=4.5,
                        k_near=20, n_wire_edges=601, sigma_px=0.7, outlier_frac=0.03, seed=7)
    elif name == "medium":     # 200 cams, 100k pts, 20k lines, 30 planes + 20 VPs
        c = SceneConfig(name="medium", n_cams=200, ring=False, n_points=100_000, n_lines=20_000,
                        n_planes=30, n_vps=20, track_min=2, track_max=12, track_mean=5.0,
                        k_near=40, n_wire_edges=6000, sigma_px=0.5, outlier_frac=0.03, seed=2)
    elif name == "large":      # 2000 cams, 2M pts, 200k lines, 300 planes + 200 VPs
        c = SceneConfig(name="large", n_cams=2000, ring=False, n_points=2_000_000,
                        n_lines=200_000, n_planes=300, n_vps=200, track_min=2, track_max=12,
                        track_mean=6.0, k_near=64, n_wire_edges=68_000, sigma_px=0.5,
                        outlier_frac=0.03, seed=3)
    elif name == "pcgprof":    # the large reduced system (2000 cams, 500 groups) with a tenth of the features
        c = SceneConfig(name="pcgprof", n_cams=2000, ring=False, n_points=200_000, n_lines=20_000,
                        n_planes=300, n_vps=200, track_min=2, track_max=12, track_mean=6.0, k_near=64,
                        n_wire_edges=6800, sigma_px=0.5, outlier_frac=0.03, seed=4)
    else:
        raise ValueError(name)
    if seed is not None:
        c.seed = seed
    for k, v in over.items():
        setattr(c, k, v)
    return c


def window_config(i: int, seed: int = 4000, max_features: int = 20_000) -> SceneConfig:
    """The i-th local-BA window of the batched workload: cameras uniform in 5..40, features log-uniform in
    200..max_features (70 % points, 30 % lines), 0..8 groups split between planes and VPs."""
    rng = np.random.default_rng(seed * 100_003 + i)
    nc = int(rng.integers(5, 41))
    nfeat = int(np.exp(rng.uniform(np.log(200), np.log(max_features))))
    ng = int(rng.integers(0, 9))
    npl = int(rng.integers(0, ng + 1))
    return SceneConfig(name=f"window{i}", n_cams=nc, ring=False, n_points=int(0.7 * nfeat),
                       n_lines=max(nfeat - int(0.7 * nfeat), 1), n_planes=npl, n_vps=ng - npl, track_min=2,
                       track_max=8, track_mean=4.0, k_near=min(12, nc),
                       n_wire_edges=(max(2, nfeat // 40) if npl > 0 else 0), sigma_px=0.7, outlier_frac=0.03,
                       seed=seed * 7919 + i)


# --------------------------------------------------------------------------
# small geometric helpers used only to synthesise data
# --------------------------------------------------------------------------
def _quat_to_mat(q):
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.empty(q.shape[:-1] + (3, 3))
    R[..., 0, 0] = 1 - 2 * (y * y + z * z); R[..., 0, 1] = 2 * (x * y - w * z); R[..., 0, 2] = 2 * (x * z + w * y)
    R[..., 1, 0] = 2 * (x * y + w * z); R[..., 1, 1] = 1 - 2 * (x * x + z * z); R[..., 1, 2] = 2 * (y * z - w * x)
    R[..., 2, 0] = 2 * (x * z - w * y); R[..., 2, 1] = 2 * (y * z + w * x); R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _mat_to_quat(R):
    q = np.empty(R.shape[:-2] + (4,))
    tr = R[..., 0, 0] + R[..., 1, 1] + R[..., 2, 2]
    for i in np.ndindex(R.shape[:-2]):
        M = R[i]
        t = tr[i]
        if t > 0:
            s = math.sqrt(t + 1.0) * 2
            q[i] = ((0.25 * s), (M[2, 1] - M[1, 2]) / s, (M[0, 2] - M[2, 0]) / s, (M[1, 0] - M[0, 1]) / s)
        elif M[0, 0] > M[1, 1] and M[0, 0] > M[2, 2]:
            s = math.sqrt(1.0 + M[0, 0] - M[1, 1] - M[2, 2]) * 2
            q[i] = ((M[2, 1] - M[1, 2]) / s, 0.25 * s, (M[0, 1] + M[1, 0]) / s, (M[0, 2] + M[2, 0]) / s)
        elif M[1, 1] > M[2, 2]:
            s = math.sqrt(1.0 + M[1, 1] - M[0, 0] - M[2, 2]) * 2
            q[i] = ((M[0, 2] - M[2, 0]) / s, (M[0, 1] + M[1, 0]) / s, 0.25 * s, (M[1, 2] + M[2, 1]) / s)
        else:
            s = math.sqrt(1.0 + M[2, 2] - M[0, 0] - M[1, 1]) * 2
            q[i] = ((M[1, 0] - M[0, 1]) / s, (M[0, 2] + M[2, 0]) / s, (M[1, 2] + M[2, 1]) / s, 0.25 * s)
    q *= np.sign(q[..., :1] + 1e-300)
    return q / np.linalg.norm(q, axis=-1, keepdims=True)


def _axis_angle_mat(axis, ang):
    axis = axis / np.linalg.norm(axis, axis=-1, keepdims=True)
    K = np.zeros(axis.shape[:-1] + (3, 3))
    K[..., 0, 1] = -axis[..., 2]; K[..., 0, 2] = axis[..., 1]
    K[..., 1, 0] = axis[..., 2]; K[..., 1, 2] = -axis[..., 0]
    K[..., 2, 0] = -axis[..., 1]; K[..., 2, 1] = axis[..., 0]
    s = np.sin(ang)[..., None, None]
    c = np.cos(ang)[..., None, None]
    return np.eye(3) + s * K + (1 - c) * (K @ K)


def _rand_unit(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _to_cam(R, t, X):
    return np.einsum("...ij,...j->...i", R, X) + t


def _pix_pinhole(f, pp, xc):
    return pp + f[..., None] * xc[..., :2] / xc[..., 2:3]


def _pix_dist(f, k1, k2, pp, xc):
    u = xc[..., :2] / xc[..., 2:3]
    r2 = (u * u).sum(-1)
    s = 1 + k1 * r2 + k2 * r2 * r2
    return pp + (f * s)[..., None] * u


def _visible(xy, z):
    return (z > 0.5) & (xy[..., 0] > 2) & (xy[..., 0] < IMG_W - 2) & (xy[..., 1] > 2) & (xy[..., 1] < IMG_H - 2)


def _track_lengths(rng, cfg: SceneConfig, n):
    lo, hi = cfg.track_min, cfg.track_max
    if cfg.track_mean <= 0:
        return rng.integers(lo, hi + 1, size=n)
    ks = np.arange(lo, hi + 1)
    best = None
    for p in np.linspace(0.01, 0.99, 981):       # pick the geometric rate whose truncated mean fits
        w = p * (1 - p) ** (ks - lo)
        m = (w * ks).sum() / w.sum()
        if best is None or abs(m - cfg.track_mean) < best[0]:
            best = (abs(m - cfg.track_mean), w / w.sum())
    return rng.choice(ks, size=n, p=best[1])


# --------------------------------------------------------------------------
def make_scene(cfg: SceneConfig) -> dict:
    rng = np.random.default_rng(cfg.seed)
    Nc = cfg.n_cams
    # ---- cameras on a ring (horizontal, y up) or a sphere, looking at the origin with 2 deg jitter
    if cfg.ring:
        a = 2 * np.pi * np.arange(Nc) / Nc + rng.uniform(0, 0.1, Nc)
        dirs = np.stack([np.cos(a), 0.15 * rng.normal(size=Nc), np.sin(a)], 1)
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    else:
        dirs = _rand_unit(rng, Nc)
    centers = 8.0 * dirs
    fwd = -dirs
    jit = _axis_angle_mat(_rand_unit(rng, Nc), np.deg2rad(2.0) * rng.normal(size=Nc))
    fwd = np.einsum("nij,nj->ni", jit, fwd)
    up = np.where(np.abs(fwd[:, 1:2]) > 0.99, np.array([[1.0, 0, 0]]), np.array([[0, 1.0, 0]]))
    xax = np.cross(up, fwd); xax /= np.linalg.norm(xax, axis=1, keepdims=True)
    yax = np.cross(fwd, xax)
    Rgt = np.stack([xax, yax, fwd], 1)                 # rows = camera axes in world
    tgt = -np.einsum("nij,nj->ni", Rgt, centers)
    f = rng.uniform(550, 650, Nc)
    k1 = rng.uniform(-0.1, 0.1, Nc)
    k2 = rng.uniform(-0.02, 0.02, Nc)
    pp = np.tile([IMG_W / 2, IMG_H / 2], (Nc, 1)) + rng.uniform(-5, 5, (Nc, 2))
    intr_of_cam = np.arange(Nc, dtype=np.int32)
    if cfg.intr_refine and cfg.intr_groups > 0:
        intr_of_cam = (np.arange(Nc) % cfg.intr_groups).astype(np.int32)
        f, k1, k2, pp = f[intr_of_cam], k1[intr_of_cam], k2[intr_of_cam], pp[intr_of_cam]

    # ---- k nearest cameras (by angle) of each camera, itself included
    K = min(cfg.k_near, Nc)
    near = np.argsort(-(dirs @ dirs.T), axis=1)[:, :K]

    # ---- groups
    npl = cfg.n_planes
    pl_axis = rng.integers(0, 3, npl)
    pl_sign = rng.choice([-1.0, 1.0], npl)
    pl_n = np.zeros((npl, 3)); pl_n[np.arange(npl), pl_axis] = pl_sign
    pl_w = rng.uniform(-2.5, 2.5, npl)
    nv = cfg.n_vps
    vp = np.zeros((nv, 3))
    for i in range(min(nv, 3)):
        vp[i, i] = 1.0
    if nv > 3:
        vp[3:] = _rand_unit(rng, nv - 3)
    vp_axis = np.full(nv, -1); vp_axis[: min(nv, 3)] = np.arange(min(nv, 3))

    def sample_on_plane(pidx):
        n = len(pidx)
        X = rng.uniform(-HALF, HALF, (n, 3))
        ax = pl_axis[pidx]
        X[np.arange(n), ax] = -pl_w[pidx] / pl_sign[pidx]
        return X

    # ---- wireframe grids: junction points on planes joined by row / column lines
    n_edges = cfg.n_wire_edges if npl > 0 else 0
    n_junc = n_edges // 2
    wf_pts, wf_pl, wf_lines_c, wf_lines_d, wf_lines_len, wf_lines_pl, edges = [], [], [], [], [], [], []
    grid_center = {}
    if n_junc > 0:
        per_plane = np.full(npl, n_junc // npl); per_plane[: n_junc % npl] += 1
        lid = 0
        for p in range(npl):
            g = int(math.ceil(math.sqrt(max(per_plane[p], 1))))
            if per_plane[p] == 0:
                continue
            ax = pl_axis[p]; o = [i for i in range(3) if i != ax]
            c0 = rng.uniform(-2.0, 2.0, 2); step = rng.uniform(0.15, 0.3)
            coords = [(i, j) for i in range(g) for j in range(g)][: per_plane[p]]
            gc = np.zeros(3); gc[ax] = -pl_w[p] / pl_sign[p]
            gc[o[0]] = c0[0] + (g - 1) * step / 2; gc[o[1]] = c0[1] + (g - 1) * step / 2
            grid_center[p] = gc
            rows = sorted({i for i, _ in coords}); cols = sorted({j for _, j in coords})
            row_id, col_id = {}, {}
            for i in rows:
                d = np.zeros(3); d[o[1]] = 1.0
                c = np.zeros(3); c[ax] = -pl_w[p] / pl_sign[p]; c[o[0]] = c0[0] + i * step; c[o[1]] = c0[1] + (g - 1) * step / 2
                wf_lines_c.append(c); wf_lines_d.append(d); wf_lines_len.append(max(g - 1, 1) * step + 0.2); wf_lines_pl.append(p)
                row_id[i] = lid; lid += 1
            for j in cols:
                d = np.zeros(3); d[o[0]] = 1.0
                c = np.zeros(3); c[ax] = -pl_w[p] / pl_sign[p]; c[o[0]] = c0[0] + (g - 1) * step / 2; c[o[1]] = c0[1] + j * step
                wf_lines_c.append(c); wf_lines_d.append(d); wf_lines_len.append(max(g - 1, 1) * step + 0.2); wf_lines_pl.append(p)
                col_id[j] = lid; lid += 1
            for i, j in coords:
                X = np.zeros(3); X[ax] = -pl_w[p] / pl_sign[p]; X[o[0]] = c0[0] + i * step; X[o[1]] = c0[1] + j * step
                k = len(wf_pts)
                wf_pts.append(X); wf_pl.append(p)
                edges.append((k, row_id[i])); edges.append((k, col_id[j]))
    n_wf_pts = len(wf_pts)
    n_wf_lines = len(wf_lines_c)

    # ---- points: wireframe junctions first, then plane points, then free points
    Np = max(cfg.n_points, n_wf_pts)
    P = np.empty((Np, 3))
    p_plane = np.full(Np, -1)
    if n_wf_pts:
        P[:n_wf_pts] = np.array(wf_pts); p_plane[:n_wf_pts] = np.array(wf_pl)
    rest = np.arange(n_wf_pts, Np)
    on = rest[rng.random(len(rest)) < cfg.frac_points_on_plane] if npl else rest[:0]
    if len(on):
        p_plane[on] = rng.integers(0, npl, len(on))
        P[on] = sample_on_plane(p_plane[on])
    free = np.setdiff1d(rest, on)
    P[free] = rng.uniform(-HALF, HALF, (len(free), 3))

    # ---- lines: wireframe lines first, then plane lines, then free lines
    Nl = max(cfg.n_lines, n_wf_lines)
    Lc = np.empty((Nl, 3)); Ld = np.empty((Nl, 3)); Llen = rng.uniform(0.5, 2.0, Nl)
    l_plane = np.full(Nl, -1); l_vp = np.full(Nl, -1)
    if n_wf_lines:
        Lc[:n_wf_lines] = np.array(wf_lines_c); Ld[:n_wf_lines] = np.array(wf_lines_d)
        Llen[:n_wf_lines] = np.array(wf_lines_len); l_plane[:n_wf_lines] = np.array(wf_lines_pl)
    rest = np.arange(n_wf_lines, Nl)
    on = rest[rng.random(len(rest)) < cfg.frac_lines_on_plane] if npl else rest[:0]
    if len(on):
        l_plane[on] = rng.integers(0, npl, len(on))
        Lc[on] = sample_on_plane(l_plane[on]) * 0.8
        Lc[on, pl_axis[l_plane[on]]] = -pl_w[l_plane[on]] / pl_sign[l_plane[on]]
        # in-plane direction: an axis (Manhattan) or a random in-plane direction
        for i in on:
            ax = pl_axis[l_plane[i]]
            if rng.random() < 0.7:
                d = np.zeros(3); d[rng.choice([k for k in range(3) if k != ax])] = 1.0
            else:
                d = rng.normal(size=3); d[ax] = 0.0; d /= np.linalg.norm(d)
            Ld[i] = d
    free = np.setdiff1d(rest, on)
    Lc[free] = rng.uniform(-HALF * 0.8, HALF * 0.8, (len(free), 3))
    Ld[free] = _rand_unit(rng, len(free))
    if nv > 0:
        # free lines: a share takes a VP direction
        take = free[rng.random(len(free)) < cfg.frac_lines_vp]
        Ld[take] = vp[rng.integers(0, nv, len(take))]
    # VP associations: a line whose direction is (up to sign) a VP direction
    if nv > 0:
        dots = np.abs(Ld @ vp.T)
        best = dots.argmax(1)
        assoc = dots[np.arange(Nl), best] > 1 - 1e-12
        keep = assoc & (rng.random(Nl) < max(cfg.frac_lines_vp, 0.8))
        l_vp[keep] = best[keep]
    Ld = Ld * np.where(rng.random(Nl) < 0.5, 1.0, -1.0)[:, None]
    E1 = Lc - 0.5 * Llen[:, None] * Ld
    E2 = Lc + 0.5 * Llen[:, None] * Ld

    # ---- tracks: anchor camera uniform, views among its K nearest where the feature is visible
    def draw_tracks(pts_list, n, wf_anchor):
        """Views among the K nearest cameras of an anchor.  Wireframe features (the first len(wf_anchor))
        use their grid's anchor camera and only its K_WIRE nearest cameras, so that the points and lines
        of one junction grid share about half of their views."""
        anchor = rng.integers(0, Nc, n)
        anchor[: len(wf_anchor)] = wf_anchor
        cand = near[anchor]                              # [n, K]
        ok = np.ones((n, K), bool)
        ok[: len(wf_anchor), min(K_WIRE, K):] = False
        for X in pts_list:
            xc = _to_cam(Rgt[cand], tgt[cand], X[:, None, :])
            xy = _pix_pinhole(f[cand], pp[cand], xc)
            ok &= _visible(xy, xc[..., 2])
        L = _track_lengths(rng, cfg, n)
        key = rng.random((n, K)) + np.where(ok, 0.0, 2.0)
        order = np.argsort(key, axis=1)
        nvis = ok.sum(1)
        L = np.minimum(L, nvis)
        sel = np.take_along_axis(cand, order, 1)
        mask = np.arange(K)[None, :] < L[:, None]
        return sel, mask

    # anchor camera of each junction grid: the camera that looks most directly at the grid centre
    K_WIRE = 12
    grid_anchor = {pl: int(np.argmax(dirs @ (c / max(np.linalg.norm(c), 1e-9)))) for pl, c in grid_center.items()}
    p_sel, p_mask = draw_tracks([P], Np, np.array([grid_anchor[q] for q in wf_pl], np.int64))
    l_sel, l_mask = draw_tracks([E1, E2], Nl, np.array([grid_anchor[q] for q in wf_lines_pl], np.int64))

    def pack(sel, mask):
        fid = np.repeat(np.arange(sel.shape[0]), mask.sum(1))
        cam = sel[mask]
        return cam.astype(np.int32), fid.astype(np.int32)

    pc, pf = pack(p_sel, p_mask)
    lc, lf = pack(l_sel, l_mask)
    # drop features seen fewer than 2 times from the observation lists (they keep their params)
    def pt_obs(cam, fid):
        xc = _to_cam(Rgt[cam], tgt[cam], P[fid])
        clean_d = _pix_dist(f[cam], k1[cam], k2[cam], pp[cam], xc)
        clean_u = _pix_pinhole(f[cam], pp[cam], xc)
        n = rng.normal(0, cfg.sigma_px, (len(cam), 2))
        md, mu = clean_d + n, clean_u + n
        out = rng.random(len(cam)) < cfg.outlier_frac
        rnd = np.stack([rng.uniform(0, IMG_W, out.sum()), rng.uniform(0, IMG_H, out.sum())], 1)
        md[out] = rnd; mu[out] = rnd
        return md, mu

    def ln_obs(cam, fid):
        a = _pix_pinhole(f[cam], pp[cam], _to_cam(Rgt[cam], tgt[cam], E1[fid]))
        b = _pix_pinhole(f[cam], pp[cam], _to_cam(Rgt[cam], tgt[cam], E2[fid]))
        m = np.concatenate([a, b], 1) + rng.normal(0, cfg.sigma_px, (len(cam), 4))
        out = rng.random(len(cam)) < cfg.outlier_frac
        m[out] = np.stack([rng.uniform(0, IMG_W, out.sum()), rng.uniform(0, IMG_H, out.sum()),
                           rng.uniform(0, IMG_W, out.sum()), rng.uniform(0, IMG_H, out.sum())], 1)
        return m

    pm_d, pm_u = pt_obs(pc, pf)
    lm = ln_obs(lc, lf)

    obs = {}
    neg = lambda n: np.full(n, -1, np.int32)
    obs["point"] = dict(cam=pc, feat=pf, other=neg(len(pc)), meas=pm_d)
    obs["line"] = dict(cam=lc, feat=lf, other=neg(len(lc)), meas=lm)
    sel = p_plane[pf] >= 0
    obs["plane_point"] = dict(cam=pc[sel], feat=pf[sel], other=p_plane[pf[sel]].astype(np.int32),
                              meas=np.zeros((sel.sum(), 0)))
    sel = l_plane[lf] >= 0
    obs["plane_line"] = dict(cam=lc[sel], feat=lf[sel], other=l_plane[lf[sel]].astype(np.int32), meas=lm[sel])
    # direct 3D group distances: one record per observed feature on a plane (no camera, no measurement)
    pp3 = np.unique(pf[p_plane[pf] >= 0]).astype(np.int32)
    ll3 = np.unique(lf[l_plane[lf] >= 0]).astype(np.int32)
    obs["plane_point3d"] = dict(cam=neg(len(pp3)), feat=pp3, other=p_plane[pp3].astype(np.int32),
                                meas=np.zeros((len(pp3), 0)))
    obs["plane_line3d"] = dict(cam=neg(len(ll3)), feat=ll3, other=l_plane[ll3].astype(np.int32),
                               meas=np.zeros((len(ll3), 0)))
    if cfg.group_form == "2d":
        for k_ in ("plane_point3d", "plane_line3d"):
            obs[k_] = {kk: vv[:0] for kk, vv in obs[k_].items()}
    elif cfg.group_form == "3d":
        for k_ in ("plane_point", "plane_line"):
            obs[k_] = {kk: vv[:0] for kk, vv in obs[k_].items()}
    elif cfg.group_form != "both":
        raise ValueError(cfg.group_form)
    vl = np.nonzero(l_vp >= 0)[0]
    obs["vp"] = dict(cam=neg(len(vl)), feat=vl.astype(np.int32), other=l_vp[vl].astype(np.int32),
                     meas=np.zeros((len(vl), 0)))
    # cross-feature residuals of each wireframe edge (point j on line k)
    p2l = {"cam": [], "feat": [], "other": [], "meas": []}
    l2p = {"cam": [], "feat": [], "other": [], "meas": []}
    if edges:
        # index observation rows by (feature, cam)
        prow = {(int(a), int(b)): i for i, (a, b) in enumerate(zip(pf, pc)) if a < n_wf_pts}
        lrow = {(int(a), int(b)): i for i, (a, b) in enumerate(zip(lf, lc)) if a < n_wf_lines}
        pv = {}
        for (j, c), i in prow.items():
            pv.setdefault(j, []).append(c)
        lv = {}
        for (k, c), i in lrow.items():
            lv.setdefault(k, []).append(c)
        for j, k in edges:
            vp_, vl_ = set(pv.get(j, [])), set(lv.get(k, []))
            for c in sorted(vl_ - vp_):          # line seen, point not: point -> observed line
                p2l["cam"].append(c); p2l["feat"].append(j); p2l["other"].append(k)
                p2l["meas"].append(lm[lrow[(k, c)]])
            for c in sorted(vp_ - vl_):          # point seen, line not: observed point -> line
                l2p["cam"].append(c); l2p["feat"].append(k); l2p["other"].append(j)
                l2p["meas"].append(pm_u[prow[(j, c)]])
    for name, d in (("p2l", p2l), ("l2p", l2p)):
        md = MEAS_DIM[name]
        obs[name] = dict(cam=np.array(d["cam"], np.int32), feat=np.array(d["feat"], np.int32),
                         other=np.array(d["other"], np.int32),
                         meas=np.array(d["meas"], np.float64).reshape(-1, md))
    # the 3D endpoint distance of every edge whose point and line are both observed (line = the feature, point =
    # the other id); no camera, no measurement
    seen_p = set(int(x) for x in pf) if len(pf) else set()
    seen_l = set(int(x) for x in lf) if len(lf) else set()
    e3 = np.array([(k, j) for j, k in edges if j in seen_p and k in seen_l], np.int64).reshape(-1, 2)
    obs["wf3d"] = dict(cam=np.full(len(e3), -1, np.int32), feat=e3[:, 0].astype(np.int32),
                       other=e3[:, 1].astype(np.int32), meas=np.zeros((len(e3), 0)))
    if cfg.wire_form == "2d":
        obs["wf3d"] = {kk: vv[:0] for kk, vv in obs["wf3d"].items()}
    elif cfg.wire_form == "3d":
        for k_ in ("p2l", "l2p"):
            obs[k_] = {kk: vv[:0] for kk, vv in obs[k_].items()}
    elif cfg.wire_form != "both":
        raise ValueError(cfg.wire_form)

    # ---- ground truth and perturbed initial values
    qgt = _mat_to_quat(Rgt)
    gt_lines = np.concatenate([Ld, np.cross(E1, Ld)], 1)
    gt_planes = np.concatenate([pl_n, pl_w[:, None]], 1)
    dR = _axis_angle_mat(_rand_unit(rng, Nc), np.deg2rad(cfg.rot_noise_deg) * rng.normal(size=Nc))
    R0 = dR @ Rgt
    t0 = tgt + rng.normal(0, cfg.trans_noise, (Nc, 3))
    P0 = P + rng.normal(0, cfg.feat_noise, P.shape)
    e1 = E1 + rng.normal(0, cfg.feat_noise, E1.shape)
    e2 = E2 + rng.normal(0, cfg.feat_noise, E2.shape)
    d0 = e2 - e1; d0 /= np.linalg.norm(d0, axis=1, keepdims=True)
    lines0 = np.concatenate([d0, np.cross(e1, d0)], 1)
    if npl:
        n0 = np.einsum("nij,nj->ni", _axis_angle_mat(_rand_unit(rng, npl), np.deg2rad(cfg.group_rot_noise_deg) * rng.normal(size=npl)), pl_n)
        planes0 = np.concatenate([n0, (pl_w + rng.normal(0, cfg.group_off_noise, npl))[:, None]], 1)
    else:
        planes0 = np.zeros((0, 4))
    if nv:
        vps0 = np.einsum("nij,nj->ni", _axis_angle_mat(_rand_unit(rng, nv), np.deg2rad(cfg.group_rot_noise_deg) * rng.normal(size=nv)), vp)
    else:
        vps0 = np.zeros((0, 3))
    intr = np.stack([f, k1, k2], 1)
    intr_gt = intr.copy()
    intrinsics = None
    if cfg.intr_refine:
        # the refined entities: one per camera, or one per group; initial values perturbed with their own
        # generator, so that every other output is the scene without refined intrinsics
        nk = int(intr_of_cam.max()) + 1 if Nc else 0
        vals = intr_gt[:nk].copy() if cfg.intr_groups > 0 else intr_gt.copy()
        if cfg.intr_noise > 0 and nk:
            r2 = np.random.default_rng(cfg.seed * 7 + 12345)
            vals[:, 0] *= 1 + cfg.intr_noise * r2.normal(size=nk)
            vals[:, 1] += 0.1 * cfg.intr_noise * r2.normal(size=nk)
            vals[:, 2] += 0.02 * cfg.intr_noise * r2.normal(size=nk)
        intrinsics = dict(of_cam=intr_of_cam, values=vals)
        intr = vals[intr_of_cam]
    # ---- inter-group relations (no random draws: the other outputs do not change).  Each plane with the
    # next one (parallel on the same axis, orthogonal otherwise); the axis VPs pairwise orthogonal; each axis
    # VP orthogonal to the normal of the first plane of another axis and parallel to that of its own axis.
    # Group kinds: 0 plane, 1 VP; types: 0 orthogonal, 1 parallel.
    rel = dict(ka=[], a=[], kb=[], b=[], type=[])

    def add_rel(ka, a, kb, b, t):
        for k_, v_ in (("ka", ka), ("a", a), ("kb", kb), ("b", b), ("type", t)):
            rel[k_].append(v_)
    if cfg.relations:
        for i in range(npl if npl > 1 else 0):
            j = (i + 1) % npl
            add_rel(0, i, 0, j, 1 if pl_axis[i] == pl_axis[j] else 0)
        na_vp = min(nv, 3)
        for i in range(na_vp):
            for j in range(i + 1, na_vp):
                add_rel(1, i, 1, j, 0)
        for k_ in range(na_vp):
            other = np.flatnonzero(pl_axis != k_)
            same = np.flatnonzero(pl_axis == k_)
            if len(other):
                add_rel(1, k_, 0, int(other[0]), 0)
            if len(same):
                add_rel(1, k_, 0, int(same[0]), 1)
    relations = {k_: np.asarray(v_, np.int8 if k_ in ("ka", "kb", "type") else np.int32) for k_, v_ in rel.items()}
    # gauge (7-DoF similarity): camera 0's pose is held (mask 0x3F) and, for the scale, the translation
    # component of camera 1 that moves most when the scene is scaled about camera 0's centre
    fixed = np.zeros(Nc, np.uint8)
    fixed[0] = 0x3F
    if Nc > 1:
        C0 = -R0[0].T @ t0[0]
        C1 = -R0[1].T @ t0[1]
        j = int(np.argmax(np.abs(R0[1] @ (C1 - C0))))
        fixed[1] = 1 << (3 + j)
    scene = dict(
        name=cfg.name, seed=cfg.seed, fixed=fixed,
        cams=dict(q=_mat_to_quat(R0), t=t0, intr=intr, pp=pp),
        points=P0, lines=lines0, planes=planes0, vps=vps0,
        obs=obs, relations=relations,
        gt=dict(cams=dict(q=qgt, t=tgt.copy(), intr=intr_gt, pp=pp.copy()), points=P.copy(),
                lines=gt_lines, planes=gt_planes, vps=vp.copy()),
        info=dict(n_wf_points=n_wf_pts, n_wf_lines=n_wf_lines, n_edges=len(edges),
                  point_plane=p_plane, line_plane=l_plane, line_vp=l_vp),
    )
    if intrinsics is not None:
        scene["intrinsics"] = intrinsics
    _add_surfaces(scene, cfg, Rgt, tgt, f, k1, k2, pp)
    return scene


def _add_surfaces(scene, cfg, Rgt, tgt, f, k1, k2, pp):
    """Spheres (c, r), cylinders (Pluecker axis d, m with |d| = 1, r) and cones (apex, unit axis, half-angle)
    inside the cube, points on their surfaces appended after the other points, with their point observations
    and one group-induced record per view (kinds sphere_point, cylinder_point, cone_point)."""
    obs = scene["obs"]
    kinds = ("sphere", "cylinder", "cone", "ellipsoid", "cuboid")
    keys = {"sphere": "spheres", "cylinder": "cylinders", "cone": "cones", "ellipsoid": "ellipsoids", "cuboid": "cuboids"}
    for k in kinds:
        obs[k + "_point"] = dict(cam=np.zeros(0, np.int32), feat=np.zeros(0, np.int32), other=np.zeros(0, np.int32),
                                 meas=np.zeros((0, 0)))
    obs["cuboid_line"] = dict(cam=np.zeros(0, np.int32), feat=np.zeros(0, np.int32), other=np.zeros(0, np.int32),
                              meas=np.zeros((0, 4)))
    counts = {"sphere": cfg.n_spheres, "cylinder": cfg.n_cylinders, "cone": cfg.n_cones,
              "ellipsoid": cfg.n_ellipsoids, "cuboid": cfg.n_cuboids}
    gt = {"sphere": np.zeros((0, 4)), "cylinder": np.zeros((0, 7)), "cone": np.zeros((0, 7)),
          "ellipsoid": np.zeros((0, 10)), "cuboid": np.zeros((0, 10))}
    init = {k: v.copy() for k, v in gt.items()}
    if sum(counts.values()) == 0:
        for k in kinds:
            scene[keys[k]] = init[k]
            scene["gt"][keys[k]] = gt[k]
        return
    rng = np.random.default_rng(cfg.seed * 31 + 777)
    Nc = len(Rgt)
    np0 = len(scene["points"])
    new_P, new_gt, recs = [], [], []
    cub_geo = []   # per cuboid (R local -> world, centre, half extents)
    for kind in kinds:
        rows, rows0 = [], []
        for g in range(counts[kind]):
            ctr = rng.uniform(-1.5, 1.5, 3)
            d = _rand_unit(rng, 1)[0]
            e1 = np.cross(d, [1.0, 0, 0] if abs(d[0]) < 0.9 else [0, 1.0, 0]); e1 /= np.linalg.norm(e1)
            e2 = np.cross(d, e1)
            th = rng.uniform(0, 2 * np.pi, cfg.surf_points)
            ring = np.cos(th)[:, None] * e1 + np.sin(th)[:, None] * e2
            if kind == "sphere":
                r = rng.uniform(0.3, 0.8)
                prm = np.concatenate([ctr, [r]])
                X = ctr + r * _rand_unit(rng, cfg.surf_points)
                prm0 = np.concatenate([ctr + rng.normal(0, 0.05, 3), [r * (1 + 0.05 * rng.normal())]])
            elif kind in ("ellipsoid", "cuboid"):
                Rg = _axis_angle_mat(_rand_unit(rng, 1), rng.uniform(0, np.pi, 1))[0]   # local -> world
                q = _mat_to_quat(Rg[None])[0]
                R0g = _axis_angle_mat(_rand_unit(rng, 1), np.deg2rad(2.0) * rng.normal(size=1))[0] @ Rg
                q0 = _mat_to_quat(R0g[None])[0]
                if kind == "ellipsoid":
                    sx = rng.uniform(0.3, 0.9, 3)
                    prm = np.concatenate([q, ctr, sx])
                    X = ctr + (_rand_unit(rng, cfg.surf_points) * sx) @ Rg.T
                    prm0 = np.concatenate([q0, ctr + rng.normal(0, 0.05, 3), sx * (1 + 0.05 * rng.normal(size=3))])
                else:
                    hx = rng.uniform(0.3, 0.8, 3)
                    a_ = Rg.T @ ctr                              # the centre along the face normals R e_i
                    dd = np.concatenate([a_ + hx, hx - a_])      # faces n_i.x = d_i and -n_i.x = d_{i+3}
                    prm = np.concatenate([q, dd])
                    f_ = rng.integers(0, 6, cfg.surf_points)     # a face, then a point inside 90% of it
                    loc = rng.uniform(-0.9, 0.9, (cfg.surf_points, 3)) * hx
                    ax = f_ % 3
                    loc[np.arange(cfg.surf_points), ax] = np.where(f_ < 3, hx[ax], -hx[ax])
                    X = ctr + loc @ Rg.T
                    prm0 = np.concatenate([q0, dd + rng.normal(0, 0.03, 6)])
                    cub_geo.append((Rg, ctr, hx))
            elif kind == "cylinder":
                r = rng.uniform(0.2, 0.5)
                prm = np.concatenate([d, np.cross(ctr, d), [r]])
                X = ctr + rng.uniform(-1, 1, cfg.surf_points)[:, None] * d + r * ring
                d0 = _axis_angle_mat(_rand_unit(rng, 1), np.deg2rad(2.0) * rng.normal(size=1))[0] @ d
                c0 = ctr + rng.normal(0, 0.05, 3)
                prm0 = np.concatenate([d0, np.cross(c0, d0), [r * (1 + 0.05 * rng.normal())]])
            else:
                al = rng.uniform(0.3, 0.7)
                prm = np.concatenate([ctr, d, [al]])
                t_ = rng.uniform(0.5, 1.5, cfg.surf_points)
                X = ctr + t_[:, None] * (np.cos(al) * d + np.sin(al) * ring)
                d0 = _axis_angle_mat(_rand_unit(rng, 1), np.deg2rad(2.0) * rng.normal(size=1))[0] @ d
                prm0 = np.concatenate([ctr + rng.normal(0, 0.05, 3), d0, [al + 0.02 * rng.normal()]])
            rows.append(prm); rows0.append(prm0)
            for x in X:
                new_gt.append(x)
                new_P.append(x + rng.normal(0, cfg.feat_noise, 3))
                recs.append((kind, g))
        if rows:
            gt[kind] = np.array(rows); init[kind] = np.array(rows0)
    new_gt = np.array(new_gt).reshape(-1, 3)
    # views: every camera that sees the point in front and inside the image; a random track of the usual length
    xc = np.einsum("cij,pj->pci", Rgt, new_gt) + tgt[None]
    xy = _pix_dist(f[None], k1[None], k2[None], pp[None], xc)
    vis = _visible(xy, xc[..., 2])
    pc, pf, pm, gk, gc, gf, gg = [], [], [], {k: [] for k in counts}, {k: [] for k in counts}, None, None
    cams_of = {k: [] for k in kinds}
    for i in range(len(new_gt)):
        cs = np.flatnonzero(vis[i])
        if len(cs) < 2:
            continue
        n = int(min(len(cs), rng.integers(cfg.track_min, cfg.track_max + 1)))
        cs = np.sort(rng.choice(cs, size=max(n, 2), replace=False))
        m = xy[i, cs] + rng.normal(0, cfg.sigma_px, (len(cs), 2))
        out = rng.random(len(cs)) < cfg.outlier_frac
        m[out] = np.stack([rng.uniform(0, IMG_W, out.sum()), rng.uniform(0, IMG_H, out.sum())], 1)
        fid = np0 + i
        pc += cs.tolist(); pf += [fid] * len(cs); pm.append(m)
        kind, g = recs[i]
        cams_of[kind] += [(c, fid, g) for c in cs]
    if pc:
        o = obs["point"]
        obs["point"] = dict(cam=np.concatenate([o["cam"], np.array(pc, np.int32)]),
                            feat=np.concatenate([o["feat"], np.array(pf, np.int32)]),
                            other=np.concatenate([o["other"], np.full(len(pc), -1, np.int32)]),
                            meas=np.concatenate([o["meas"], np.concatenate(pm)]))
    for kind in counts:
        t = np.array(cams_of[kind], np.int64).reshape(-1, 3)
        obs[kind + "_point"] = dict(cam=t[:, 0].astype(np.int32), feat=t[:, 1].astype(np.int32),
                                    other=t[:, 2].astype(np.int32), meas=np.zeros((len(t), 0)))
    scene["points"] = np.concatenate([scene["points"], np.array(new_P).reshape(-1, 3)])
    scene["gt"]["points"] = np.concatenate([scene["gt"]["points"], new_gt])
    for k in kinds:
        scene[keys[k]] = init[k]
        scene["gt"][keys[k]] = gt[k]
    if cfg.surf_lines > 0 and cub_geo:
        _add_cuboid_lines(scene, cfg, cub_geo, Rgt, tgt, f, pp)


def _add_cuboid_lines(scene, cfg, cub_geo, Rgt, tgt, f, pp):
    """surf_lines lines on faces of every cuboid (an in-face axis 70% of the time, else a random in-face
    direction, centred inside the middle half of the face), appended after the other lines with their line
    observations (segment endpoints, pinhole pixels) and one cuboid_line record per view."""
    rng = np.random.default_rng(cfg.seed * 37 + 4242)
    obs = scene["obs"]
    E1, E2, gid = [], [], []
    for g, (Rg, ctr, hx) in enumerate(cub_geo):
        for _ in range(cfg.surf_lines):
            fc = int(rng.integers(0, 6))
            a = fc % 3
            b, c = [k for k in range(3) if k != a]
            dl = np.zeros(3)
            if rng.random() < 0.7:
                dl[b if rng.random() < 0.5 else c] = 1.0
            else:
                th = rng.uniform(0, 2 * np.pi)
                dl[b], dl[c] = np.cos(th), np.sin(th)
            loc = np.zeros(3)
            loc[b], loc[c] = rng.uniform(-0.5, 0.5) * hx[b], rng.uniform(-0.5, 0.5) * hx[c]
            loc[a] = hx[a] if fc < 3 else -hx[a]
            ln = rng.uniform(0.5, 0.9) * min(hx[b], hx[c])
            E1.append(ctr + Rg @ (loc - 0.5 * ln * dl))
            E2.append(ctr + Rg @ (loc + 0.5 * ln * dl))
            gid.append(g)
    E1, E2, gid = np.array(E1), np.array(E2), np.array(gid, np.int64)
    nl0 = len(scene["lines"])
    xc1 = np.einsum("cij,pj->pci", Rgt, E1) + tgt[None]
    xc2 = np.einsum("cij,pj->pci", Rgt, E2) + tgt[None]
    a1 = _pix_pinhole(f[None], pp[None], xc1)
    a2 = _pix_pinhole(f[None], pp[None], xc2)
    vis = _visible(a1, xc1[..., 2]) & _visible(a2, xc2[..., 2])
    lc, lf, lm, lg = [], [], [], []
    for i in range(len(E1)):
        cs = np.flatnonzero(vis[i])
        if len(cs) < 2:
            continue
        n = int(min(len(cs), rng.integers(cfg.track_min, cfg.track_max + 1)))
        cs = np.sort(rng.choice(cs, size=max(n, 2), replace=False))
        m = np.concatenate([a1[i, cs], a2[i, cs]], 1) + rng.normal(0, cfg.sigma_px, (len(cs), 4))
        out = rng.random(len(cs)) < cfg.outlier_frac
        m[out] = np.stack([rng.uniform(0, IMG_W, out.sum()), rng.uniform(0, IMG_H, out.sum()),
                           rng.uniform(0, IMG_W, out.sum()), rng.uniform(0, IMG_H, out.sum())], 1)
        lc += cs.tolist(); lf += [nl0 + i] * len(cs); lm.append(m); lg += [int(gid[i])] * len(cs)
    d = E2 - E1
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    gt_l = np.concatenate([d, np.cross(E1, d)], 1)
    e1 = E1 + rng.normal(0, cfg.feat_noise, E1.shape)
    e2 = E2 + rng.normal(0, cfg.feat_noise, E2.shape)
    d0 = e2 - e1
    d0 /= np.linalg.norm(d0, axis=1, keepdims=True)
    init_l = np.concatenate([d0, np.cross(e1, d0)], 1)
    scene["lines"] = np.concatenate([scene["lines"], init_l])
    scene["gt"]["lines"] = np.concatenate([scene["gt"]["lines"], gt_l])
    if lc:
        cam = np.array(lc, np.int32); fid = np.array(lf, np.int32); meas = np.concatenate(lm)
        o = obs["line"]
        obs["line"] = dict(cam=np.concatenate([o["cam"], cam]), feat=np.concatenate([o["feat"], fid]),
                           other=np.concatenate([o["other"], np.full(len(cam), -1, np.int32)]),
                           meas=np.concatenate([o["meas"], meas]))
        obs["cuboid_line"] = dict(cam=cam, feat=fid, other=np.array(lg, np.int32), meas=meas)


def noise_free(cfg: SceneConfig) -> dict:
    """The same scene with zero pixel noise, no outliers, and initial values at ground truth."""
    c = dataclasses.replace(cfg, sigma_px=0.0, outlier_frac=0.0, rot_noise_deg=0.0, trans_noise=0.0,
                            feat_noise=0.0, group_rot_noise_deg=0.0, group_off_noise=0.0)
    s = make_scene(c)
    s["cams"] = {k: v.copy() for k, v in s["gt"]["cams"].items()}
    s["points"] = s["gt"]["points"].copy(); s["lines"] = s["gt"]["lines"].copy()
    s["planes"] = s["gt"]["planes"].copy(); s["vps"] = s["gt"]["vps"].copy()
    for k in ("spheres", "cylinders", "cones", "ellipsoids", "cuboids"):
        s[k] = s["gt"][k].copy()
    if "intrinsics" in s:
        ik = s["intrinsics"]
        nk = len(ik["values"])
        first = np.array([int(np.flatnonzero(ik["of_cam"] == k)[0]) for k in range(nk)], np.int64)
        s["intrinsics"] = dict(of_cam=ik["of_cam"], values=s["gt"]["cams"]["intr"][first].copy())
    return s


def counts(scene: dict) -> dict:
    return {k: int(len(v["cam"])) for k, v in scene["obs"].items()}
