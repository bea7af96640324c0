"""FP64 CPU oracle for one Levenberg-Marquardt step of holistic bundle adjustment.

TEST INFRASTRUCTURE ONLY.  This module exists to check the CUDA library; only the
test-suite, the smoke entry point and the benchmark's CPU-baseline leg may import
it.  It shares no code with the CUDA path: it is written from the paper's
definitions, in plain float64 PyTorch (CPU) / numpy / scipy, and is kept slow and
direct on purpose.  Jacobians are not hand-derived here: each residual is written
as a function of the minimal local increments through the retraction x (+) delta,
and forward-mode automatic differentiation at delta = 0 gives J (the definition
of the derivative); finite differences in the tests pin that.

What follows the paper, and where:
  * cost             Eq. 1 and Eq. 4 (points, lines), Eq. 6 (VP), Eq. 7 / Eq. 8
                     (plane-induced point / line), Eq. 11 / Eq. 12 (wireframe
                     point->line, line->point); weights and Cauchy scales from the
                     cost-balancing paragraph of Appendix C.  Robust cost is
                     E = 1/2 sum_r w_r a_r^2 ln(1 + |r|^2 / a_r^2).
  * plane projection of points and Pluecker lines: Appendix B ("Plane").
  * VP residual: Eq. 6 / Appendix B, as the 3-vector d_hat x v (same squared norm).
  * normal equations, augmented set A = C u G, block-diagonal H_ff and the Schur
    complement S = H_aa - H_af H_ff^-1 H_fa: Eq. 2, Eq. 3, Eq. 5.
  * termination: relative change of the pixel-space cost only (Section 3.5;
    Appendix C excludes the angular VP terms).
Readings where the paper is silent (camera model, the LM rule, PCG, ...) are the
ones listed in the design notes; each function below states the one it uses.

Parity status: every function here is pinned by a CPU test (finite differences,
closed forms, dense full-system solve, an independent trust-region minimiser,
invariants).
"""
from __future__ import annotations

import math
import dataclasses

import numpy as np
import scipy.sparse as sp
import torch
from torch.func import jacfwd, vmap

torch.set_default_dtype(torch.float64)
DT = torch.float64

KINDS = ("point", "line", "plane_point", "plane_line", "vp", "p2l", "l2p", "plane_point3d", "plane_line3d",
         "sphere_point", "cylinder_point", "cone_point", "ellipsoid_point", "cuboid_point", "wf3d", "cuboid_line")
# residual dimension, feature type, group type per kind
RDIM = {"point": 2, "line": 4, "plane_point": 2, "plane_line": 4, "vp": 3, "p2l": 1, "l2p": 1,
        "plane_point3d": 1, "plane_line3d": 2, "sphere_point": 2, "cylinder_point": 2, "cone_point": 2,
        "ellipsoid_point": 2, "cuboid_point": 2, "wf3d": 3, "cuboid_line": 4}
FEAT = {"point": "point", "line": "line", "plane_point": "point", "plane_line": "line",
        "vp": "line", "p2l": "point", "l2p": "line", "plane_point3d": "point", "plane_line3d": "line",
        "sphere_point": "point", "cylinder_point": "point", "cone_point": "point", "ellipsoid_point": "point",
        "cuboid_point": "point", "wf3d": "line", "cuboid_line": "line"}
GROUP = {"plane_point": "plane", "plane_line": "plane", "vp": "vp", "plane_point3d": "plane",
         "plane_line3d": "plane", "sphere_point": "sphere", "cylinder_point": "cylinder", "cone_point": "cone",
         "ellipsoid_point": "ellipsoid", "cuboid_point": "cuboid", "wf3d": "jpoint", "cuboid_line": "cuboid"}
HAS_CAM = {k: k not in ("vp", "plane_point3d", "plane_line3d", "wf3d") for k in KINDS}
# kinds outside the pixel cost E_px: the angular VP term, and the direct 3D distances
NON_PIXEL = ("vp", "plane_point3d", "plane_line3d", "wf3d")
FDOF = {"point": 3, "line": 4}
GDOF = {"plane": 3, "vp": 2, "sphere": 4, "cylinder": 5, "cone": 6, "ellipsoid": 9, "cuboid": 9, "jpoint": 3}
# state key and stored width of every group kind (spheres (c, r); cylinders (d, m, r), the axis a Pluecker line
# with |d| = 1; cones (apex, unit axis, half-angle))
GKEY = {"plane": ("planes", 4), "vp": ("vps", 3), "sphere": ("spheres", 4), "cylinder": ("cylinders", 7),
        "cone": ("cones", 7), "ellipsoid": ("ellipsoids", 15), "cuboid": ("cuboids", 15), "jpoint": ("points", 3)}
SURFACES = ("sphere", "cylinder", "cone")
# the 9-parameter groups: two entities of A each, the first 6 increments (rotation and centre, or rotation and
# three face offsets) and the last 3 (log semi-axes, or the other three offsets)
SPLIT = ("ellipsoid", "cuboid")
CDOF = 6


@dataclasses.dataclass
class Options:
    """Weights and Cauchy scales (Appendix C) and LM / PCG constants."""
    w_point: float = 1.0
    w_line: float = 1.0
    w_group: float = 0.5
    w_wire: float = 0.1
    w_vp: float = 5e3
    w_rel: float = 5e3        # inter-group relations (angular, like the VP term)
    cauchy_rel: float = 0.2
    w_group3d: float = 1.0    # the direct 3D group distances (Section 3.2's alternative; Table 5 weighs it)
    cauchy_3d: float = 1.0
    w_wire3d: float = 1.0     # the 3D wireframe endpoint distance (the form Fig. 3b compares; scale cauchy_3d)
    cauchy_px: float = 1.0
    cauchy_vp: float = 0.2
    lambda0: float = 1e-4
    lambda_min: float = 1e-12
    lambda_max: float = 1e12
    min_gain: float = 1e-3
    rel_cost_tol: float = 1e-6
    pcg_rel_tol: float = 1e-6
    pcg_max_iters: int = 1000
    solver: str = "pcg"           # "pcg" (block-Jacobi PCG) or "dense" (Cholesky of S)

    def weight(self, kind):
        return {"point": self.w_point, "line": self.w_line, "plane_point": self.w_group,
                "plane_line": self.w_group, "vp": self.w_vp, "p2l": self.w_wire,
                "l2p": self.w_wire, "plane_point3d": self.w_group3d, "plane_line3d": self.w_group3d,
                "sphere_point": self.w_group, "cylinder_point": self.w_group, "cone_point": self.w_group,
                "ellipsoid_point": self.w_group, "cuboid_point": self.w_group, "wf3d": self.w_wire3d,
                "cuboid_line": self.w_group}[kind]

    def scale(self, kind):
        if kind in ("plane_point3d", "plane_line3d", "wf3d"):
            return self.cauchy_3d
        return self.cauchy_vp if kind == "vp" else self.cauchy_px


# ===========================================================================
# rotations and manifolds
# ===========================================================================
def skew(v):
    z = torch.zeros_like(v[..., 0])
    return torch.stack([torch.stack([z, -v[..., 2], v[..., 1]], -1),
                        torch.stack([v[..., 2], z, -v[..., 0]], -1),
                        torch.stack([-v[..., 1], v[..., 0], z], -1)], -2)


def so3_exp(w):
    """Rodrigues' formula R = I + A [w]x + B [w]x^2 with a series branch near 0."""
    th2 = (w * w).sum(-1)
    small = th2 < 1e-12
    th2s = torch.where(small, torch.ones_like(th2), th2)
    th = torch.sqrt(th2s)
    A = torch.where(small, 1 - th2 / 6, torch.sin(th) / th)
    B = torch.where(small, 0.5 - th2 / 24, (1 - torch.cos(th)) / th2s)
    K = skew(w)
    eye = torch.eye(3, dtype=w.dtype).expand(K.shape)
    return eye + A[..., None, None] * K + B[..., None, None] * (K @ K)


def quat_to_R(q):
    q = q / torch.linalg.norm(q, dim=-1, keepdim=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)


def R_to_quat(R):
    """Rotation matrix -> unit quaternion (w,x,y,z), w >= 0 (numpy)."""
    R = np.asarray(R)
    q = np.empty(R.shape[:-2] + (4,))
    for i in np.ndindex(R.shape[:-2]):
        M = R[i]
        t = np.trace(M)
        if t > 0:
            s = math.sqrt(t + 1.0) * 2
            v = (0.25 * s, (M[2, 1] - M[1, 2]) / s, (M[0, 2] - M[2, 0]) / s, (M[1, 0] - M[0, 1]) / s)
        elif M[0, 0] > M[1, 1] and M[0, 0] > M[2, 2]:
            s = math.sqrt(1.0 + M[0, 0] - M[1, 1] - M[2, 2]) * 2
            v = ((M[2, 1] - M[1, 2]) / s, 0.25 * s, (M[0, 1] + M[1, 0]) / s, (M[0, 2] + M[2, 0]) / s)
        elif M[1, 1] > M[2, 2]:
            s = math.sqrt(1.0 + M[1, 1] - M[0, 0] - M[2, 2]) * 2
            v = ((M[0, 2] - M[2, 0]) / s, (M[0, 1] + M[1, 0]) / s, 0.25 * s, (M[1, 2] + M[2, 1]) / s)
        else:
            s = math.sqrt(1.0 + M[2, 2] - M[0, 0] - M[1, 1]) * 2
            v = ((M[1, 0] - M[0, 1]) / s, (M[0, 2] + M[2, 0]) / s, (M[1, 2] + M[2, 1]) / s, 0.25 * s)
        q[i] = v
    q *= np.where(q[..., :1] < 0, -1.0, 1.0)
    return q / np.linalg.norm(q, axis=-1, keepdims=True)


def tangent_basis(n):
    """Orthonormal (b1, b2) spanning the tangent plane of the unit vector n:
    a = e_x unless |n_x| >= 0.9 (then e_y); b1 = unit(a - (a.n) n); b2 = n x b1."""
    ex = torch.zeros_like(n); ex[..., 0] = 1.0
    ey = torch.zeros_like(n); ey[..., 1] = 1.0
    a = torch.where((n[..., 0].abs() < 0.9)[..., None], ex, ey)
    b1 = a - (a * n).sum(-1, keepdim=True) * n
    b1 = b1 / torch.linalg.norm(b1, dim=-1, keepdim=True)
    b2 = torch.linalg.cross(n, b1)
    return b1, b2


def s2_exp(n, v):
    """Exponential map of the unit sphere at n along the tangent vector v."""
    th2 = (v * v).sum(-1)
    small = th2 < 1e-12
    th = torch.sqrt(torch.where(small, torch.ones_like(th2), th2))
    c = torch.where(small, 1 - th2 / 2, torch.cos(th))
    s = torch.where(small, 1 - th2 / 6, torch.sin(th) / th)
    return c[..., None] * n + s[..., None] * v


# ---------------------------------------------------------------------------
# retractions x (+) delta (the minimal increments the normal equations use)
# ---------------------------------------------------------------------------
def pose_plus(q, t, dp):
    """R <- Exp(dw) R, t <- t + dt; dp = (dw, dt)."""
    return so3_exp(dp[..., :3]) @ quat_to_R(q), t + dp[..., 3:6]


def line_frame(L):
    """Orthonormal representation (Bartoli-Sturm) of a Pluecker line with |d| = 1:
    U = [m/|m|, d, (m x d)/|m x d|] and the angle phi with (cos, sin) ~ (|m|, |d|)."""
    d, m = L[..., :3], L[..., 3:6]
    dn = torch.linalg.norm(d, dim=-1, keepdim=True)
    d = d / dn
    m = m / dn
    r = torch.linalg.norm(m, dim=-1)
    tiny = r < 1e-12
    b1, _ = tangent_basis(d)
    u1 = torch.where(tiny[..., None], b1, m / torch.where(tiny, torch.ones_like(r), r)[..., None])
    u3 = torch.linalg.cross(u1, d)
    U = torch.stack([u1, d, u3], -1)
    phi = torch.atan2(torch.ones_like(r), r)
    return U, phi


def line_plus(L, dl):
    """U <- U Exp(dl[0:3]), phi <- phi + dl[3]; d = u2, m = cot(phi) u1 (|d| stays 1)."""
    U, phi = line_frame(L)
    U2 = U @ so3_exp(dl[..., :3])
    ph = phi + dl[..., 3]
    return torch.cat([U2[..., :, 1], (torch.cos(ph) / torch.sin(ph))[..., None] * U2[..., :, 0]], -1)


def plane_plus(P, dp):
    """n <- Exp_n(b1 d0 + b2 d1) on S^2, w <- w + d2."""
    n = P[..., :3] / torch.linalg.norm(P[..., :3], dim=-1, keepdim=True)
    b1, b2 = tangent_basis(n)
    v = dp[..., 0:1] * b1 + dp[..., 1:2] * b2
    return torch.cat([s2_exp(n, v), P[..., 3:4] + dp[..., 2:3]], -1)


def vp_plus(v, dv):
    v = v / torch.linalg.norm(v, dim=-1, keepdim=True)
    b1, b2 = tangent_basis(v)
    return s2_exp(v, dv[..., 0:1] * b1 + dv[..., 1:2] * b2)


# ---- the other group types of Appendix B / Table 6 (positives in log space, as the table's parameterisations
# ask for r > 0; the cone's half-angle additive)
def sphere_plus(S, d):
    """centre c <- c + d[0:3], radius r <- r exp(d[3])."""
    return torch.cat([S[..., :3] + d[..., :3], S[..., 3:4] * torch.exp(d[..., 3:4])], -1)


def cylinder_plus(C, d):
    """axis (Pluecker, |d| = 1) by the line update of the features (4), radius r <- r exp(d[4])."""
    return torch.cat([line_plus(C[..., :6], d[..., :4]), C[..., 6:7] * torch.exp(d[..., 4:5])], -1)


def cone_plus(K, d):
    """apex a <- a + d[0:3], axis on S^2 by d[3:5], half-angle alpha <- alpha + d[5]."""
    return torch.cat([K[..., :3] + d[..., :3], vp_plus(K[..., 3:6], d[..., 3:5]), K[..., 6:7] + d[..., 5:6]], -1)


def ellipsoid_plus(E, d):
    """(R, c, s) stored as R row-major (9), c (3), semi-axes s (3): R <- Exp(d[0:3]) R, c <- c + d[3:6],
    s <- s exp(d[6:9])."""
    R = so3_exp(d[..., :3]) @ E[..., :9].reshape(E.shape[:-1] + (3, 3))
    return torch.cat([R.reshape(E.shape[:-1] + (9,)), E[..., 9:12] + d[..., 3:6], E[..., 12:15] * torch.exp(d[..., 6:9])], -1)


def cuboid_plus(K, d):
    """(R, d_0..d_5) stored as R row-major (9) and the six face offsets: R <- Exp(d[0:3]) R, offsets + d[3:9]."""
    R = so3_exp(d[..., :3]) @ K[..., :9].reshape(K.shape[:-1] + (3, 3))
    return torch.cat([R.reshape(K.shape[:-1] + (9,)), K[..., 9:15] + d[..., 3:9]], -1)


GROUP_PLUS = {"sphere": sphere_plus, "cylinder": cylinder_plus, "cone": cone_plus, "ellipsoid": ellipsoid_plus,
              "cuboid": cuboid_plus}


def sphere_project_point(S, X):
    """Appendix B: radial projection c + r (X - c) / |X - c|."""
    u = X - S[..., :3]
    return S[..., :3] + S[..., 3:4] * u / torch.linalg.norm(u, dim=-1, keepdim=True)


def cylinder_project_point(C, X):
    """Appendix B: radially onto the surface, perpendicular to the axis (foot p0 = d x m, direction d)."""
    d, m, r = C[..., :3], C[..., 3:6], C[..., 6:7]
    p0 = torch.linalg.cross(d, m)
    v = X - p0
    h = (v * d).sum(-1, keepdim=True)
    w = v - h * d
    return p0 + h * d + r * w / torch.linalg.norm(w, dim=-1, keepdim=True)


def cone_project_point(K, X):
    """Appendix B: onto the cone surface along the direction perpendicular to its generatrix: with v = X - a,
    the radial unit e of v about the axis and the generatrix g = cos(alpha) d + sin(alpha) e through the apex,
    the projection is a + (v . g) g."""
    a, d, al = K[..., :3], K[..., 3:6], K[..., 6:7]
    v = X - a
    h = (v * d).sum(-1, keepdim=True)
    w = v - h * d
    e = w / torch.linalg.norm(w, dim=-1, keepdim=True)
    g = torch.cos(al) * d + torch.sin(al) * e
    return a + (v * g).sum(-1, keepdim=True) * g


def ellipsoid_project_point(E, X):
    """Appendix B: scaled-radial projection: to the local frame x = R^T (X - c), scaled to the unit sphere,
    normalised, scaled back, and back to the world frame."""
    R = E[..., :9].reshape(E.shape[:-1] + (3, 3))
    c, sx = E[..., 9:12], E[..., 12:15]
    x = (R.transpose(-1, -2) @ (X - c)[..., None])[..., 0]
    y = x / sx
    y = y / torch.linalg.norm(y, dim=-1, keepdim=True)
    return c + (R @ (sx * y)[..., None])[..., 0]


def cuboid_faces(K):
    """The six faces n_f . x + w_f = 0 of a cuboid (R, d): n_i = R e_i with w_i = -d_i, n_{i+3} = -R e_i with
    w_{i+3} = -d_{i+3}; normals pointing out."""
    R = K[..., :9].reshape(K.shape[:-1] + (3, 3))
    Rt = R.transpose(-1, -2)                       # rows: the columns R e_i
    normals = torch.cat([Rt, -Rt], -2)             # [6, 3]
    return normals, -K[..., 9:15]


def cuboid_project_point(K, X):
    """Appendix B: onto the face nearest the point (smallest |signed distance|), along that face's normal."""
    normals, w = cuboid_faces(K)
    dist = (normals @ X[..., None])[..., 0] + w    # signed, outside positive
    ad = dist.abs()
    sel = (ad == ad.min(-1, keepdim=True).values).to(X.dtype)   # the nearest face (a tie is measure zero)
    df = (dist * sel).sum(-1, keepdim=True)
    nf = (normals * sel[..., None]).sum(-2)
    return X - df * nf


def cuboid_centre(K):
    """The centre of a cuboid (R, d): along R e_i its faces lie at d_i and at -d_{i+3}, so the centre is
    sum_i R e_i (d_i - d_{i+3}) / 2."""
    R = K[..., :9].reshape(K.shape[:-1] + (3, 3))
    return (R @ ((K[..., 9:12] - K[..., 12:15]) / 2)[..., None])[..., 0]


def cuboid_line_face(K, L):
    """Appendix B: the face (n, w) a line is projected onto: the point of the infinite line closest to the
    cuboid's centre, then the face nearest that point (smallest |signed distance|).  The choice is piecewise
    constant, so no derivative flows through it."""
    normals, w = cuboid_faces(K)
    d, m = L[..., :3], L[..., 3:6]
    dd = (d * d).sum(-1, keepdim=True)
    p0 = torch.linalg.cross(d, m) / dd                       # the line's point closest to the origin
    c = cuboid_centre(K)
    pc = p0 + (((c - p0) * d).sum(-1, keepdim=True) / dd) * d
    dist = (normals @ pc[..., None])[..., 0] + w
    ad = dist.abs()
    sel = (ad == ad.min(-1, keepdim=True).values).to(L.dtype)   # a tie is measure zero
    return torch.cat([(normals * sel[..., None]).sum(-2), (w * sel).sum(-1, keepdim=True)], -1)


GROUP_PROJECT = {"sphere": sphere_project_point, "cylinder": cylinder_project_point, "cone": cone_project_point,
                 "ellipsoid": ellipsoid_project_point, "cuboid": cuboid_project_point}


# ===========================================================================
# projections (Section 3.1-3.4) and the plane projections (Appendix B)
# ===========================================================================
def to_cam(R, t, X):
    return (R @ X[..., None])[..., 0] + t


def pi_point(R, t, cam, X):
    """Point projection with radial distortion: pp + f (1 + k1 r^2 + k2 r^4) (x/z, y/z)."""
    xc = to_cam(R, t, X)
    u = xc[..., :2] / xc[..., 2:3]
    r2 = (u * u).sum(-1, keepdim=True)
    s = 1 + cam[..., 8:9] * r2 + cam[..., 9:10] * r2 * r2
    return cam[..., 10:12] + cam[..., 7:8] * s * u, xc[..., 2]


def pi_point_pinhole(R, t, cam, X):
    xc = to_cam(R, t, X)
    return cam[..., 10:12] + cam[..., 7:8] * xc[..., :2] / xc[..., 2:3], xc[..., 2]


def pi_line(R, t, cam, L):
    """Image line (homogeneous, pixels) of a Pluecker line: d_c = R d,
    m_c = R m + t x d_c, l = (m_c0, m_c1, f m_c2 - ppx m_c0 - ppy m_c1)."""
    dc = (R @ L[..., :3, None])[..., 0]
    mc = (R @ L[..., 3:6, None])[..., 0] + torch.linalg.cross(t, dc)
    f, px, py = cam[..., 7], cam[..., 10], cam[..., 11]
    return torch.stack([mc[..., 0], mc[..., 1], f * mc[..., 2] - px * mc[..., 0] - py * mc[..., 1]], -1)


def rho(l, seg):
    """Eq. 4: perpendicular displacement vectors of the two observed endpoints to the line l."""
    n12 = torch.sqrt(l[..., 0] ** 2 + l[..., 1] ** 2)
    nrm = l[..., :2] / n12[..., None]
    out = []
    for e in (seg[..., 0:2], seg[..., 2:4]):
        s = (l[..., 0] * e[..., 0] + l[..., 1] * e[..., 1] + l[..., 2]) / n12
        out.append(s[..., None] * nrm)
    return torch.cat(out, -1), n12


def plane_project_point(P, X):
    """Appendix B: p_proj = p - (n.p + w) n."""
    n, w = P[..., :3], P[..., 3]
    return X - ((n * X).sum(-1) + w)[..., None] * n


def plane_project_line(P, L):
    """Appendix B: d' = d - (d.n) n;  m' = (1 - a^2/|d|^2) m + (a g/|d|^2) d + (w - dl/|d|^2)(d x n),
    a = d.n, g = m.n, dl = (d x n).m."""
    n, w = P[..., :3], P[..., 3:4]
    d, m = L[..., :3], L[..., 3:6]
    a = (d * n).sum(-1, keepdim=True)
    g = (m * n).sum(-1, keepdim=True)
    dxn = torch.linalg.cross(d, n)
    dl = (dxn * m).sum(-1, keepdim=True)
    dd = (d * d).sum(-1, keepdim=True)
    return torch.cat([d - a * n, (1 - a * a / dd) * m + (a * g / dd) * d + (w - dl / dd) * dxn], -1)


# ===========================================================================
# residuals as functions of the local increments (one record, vmapped)
#   cam = [q(4) t(3) f k1 k2 ppx ppy] (12), feat = point (3) or line (6),
#   grp = plane (4) or vp (3, padded to 4), meas (4, padded)
# each returns (r, valid)
# ===========================================================================
def _pose(cam, dc):
    return pose_plus(cam[:4], cam[4:7], dc)


def res_point(dc, df, dg, cam, feat, grp, meas):            # Eq. 1 / Eq. 4 (points)
    R, t = _pose(cam, dc)
    x, z = pi_point(R, t, cam, feat[:3] + df)
    return x - meas[:2], z > 1e-6


def res_line(dc, df, dg, cam, feat, grp, meas):             # Eq. 4 (lines)
    R, t = _pose(cam, dc)
    l = pi_line(R, t, cam, line_plus(feat, df))
    r, n12 = rho(l, meas)
    return r, n12 > 1e-12


def res_plane_point(dc, df, dg, cam, feat, grp, meas):      # Eq. 7
    R, t = _pose(cam, dc)
    X = feat[:3] + df
    P = plane_plus(grp, dg)
    x1, z1 = pi_point(R, t, cam, X)
    x2, z2 = pi_point(R, t, cam, plane_project_point(P, X))
    return x1 - x2, (z1 > 1e-6) & (z2 > 1e-6)


def res_plane_line(dc, df, dg, cam, feat, grp, meas):       # Eq. 8
    R, t = _pose(cam, dc)
    L = line_plus(feat, df)
    P = plane_plus(grp, dg)
    r1, n1 = rho(pi_line(R, t, cam, L), meas)
    r2, n2 = rho(pi_line(R, t, cam, plane_project_line(P, L)), meas)
    return r1 - r2, (n1 > 1e-12) & (n2 > 1e-12)


def res_vp(dc, df, dg, cam, feat, grp, meas):               # Eq. 6 as d_hat x v
    L = line_plus(feat, df)
    d = L[:3] / torch.linalg.norm(L[:3])
    v = vp_plus(grp[:3], dg[:2])
    return torch.linalg.cross(d, v), torch.ones((), dtype=torch.bool)


def res_p2l(dc, df, dg, cam, feat, grp, meas):              # Eq. 11
    R, t = _pose(cam, dc)
    x, z = pi_point_pinhole(R, t, cam, feat[:3] + df)
    e1 = torch.cat([meas[0:2], torch.ones(1, dtype=DT)])
    e2 = torch.cat([meas[2:4], torch.ones(1, dtype=DT)])
    lh = torch.linalg.cross(e1, e2)
    lh = lh / torch.sqrt(lh[0] ** 2 + lh[1] ** 2)
    return (lh[:2] * x).sum(-1, keepdim=True) + lh[2:3], z > 1e-6


def res_l2p(dc, df, dg, cam, feat, grp, meas):              # Eq. 12
    R, t = _pose(cam, dc)
    l = pi_line(R, t, cam, line_plus(feat, df))
    n12 = torch.sqrt(l[0] ** 2 + l[1] ** 2)
    return ((l[0] * meas[0] + l[1] * meas[1] + l[2]) / n12)[None], n12 > 1e-12


def res_plane_point3d(dc, df, dg, cam, feat, grp, meas):    # Section 3.2: the direct point-to-plane distance
    X = feat[:3] + df
    P = plane_plus(grp, dg)
    return ((P[:3] * X).sum(-1) + P[3])[None], torch.ones((), dtype=torch.bool)


def res_plane_line3d(dc, df, dg, cam, feat, grp, meas):     # the same for a line: its direction's normal component
    L = line_plus(feat, df)                                  # and the distance of its foot point d x m (|d| = 1)
    P = plane_plus(grp, dg)
    n = P[:3]
    foot = torch.linalg.cross(L[:3], L[3:6])
    return torch.stack([(n * L[:3]).sum(-1), (n * foot).sum(-1) + P[3]]), torch.ones((), dtype=torch.bool)


def res_cuboid_line(dc, df, dg, cam, feat, grp, meas):    # Eq. 8 with the cuboid's face (Appendix B)
    R, t = _pose(cam, dc)
    L = line_plus(feat, df)
    P = cuboid_line_face(cuboid_plus(grp[:15], dg), L)
    r1, n1 = rho(pi_line(R, t, cam, L), meas)
    r2, n2 = rho(pi_line(R, t, cam, plane_project_line(P, L)), meas)
    return r1 - r2, (n1 > 1e-12) & (n2 > 1e-12)


def _res_surface_point(kind):
    """The group-induced point residual of Eq. 7 with the projection of another group type (Appendix B):
    pi(C, X) - pi(C, Proj_g(X))."""
    plus, proj = GROUP_PLUS[kind], GROUP_PROJECT[kind]

    def fn(dc, df, dg, cam, feat, grp, meas):
        R, t = _pose(cam, dc)
        X = feat[:3] + df
        G = plus(grp[:GKEY[kind][1]], dg)
        x1, z1 = pi_point(R, t, cam, X)
        x2, z2 = pi_point(R, t, cam, proj(G, X))
        return x1 - x2, (z1 > 1e-6) & (z2 > 1e-6)
    return fn


res_sphere_point = _res_surface_point("sphere")
res_cylinder_point = _res_surface_point("cylinder")
res_cone_point = _res_surface_point("cone")
res_ellipsoid_point = _res_surface_point("ellipsoid")
res_cuboid_point = _res_surface_point("cuboid")


def res_wf3d(dc, df, dg, cam, feat, grp, meas):   # 3D wireframe endpoint distance: X x d - m (|d| = 1)
    L = line_plus(feat, df)
    X = grp[:3] + dg
    return torch.linalg.cross(X, L[:3]) - L[3:6], torch.ones((), dtype=torch.bool)


RES_FN = {"point": res_point, "line": res_line, "plane_point": res_plane_point,
          "plane_line": res_plane_line, "vp": res_vp, "p2l": res_p2l, "l2p": res_l2p,
          "plane_point3d": res_plane_point3d, "plane_line3d": res_plane_line3d,
          "sphere_point": res_sphere_point, "cylinder_point": res_cylinder_point, "cone_point": res_cone_point,
          "ellipsoid_point": res_ellipsoid_point, "cuboid_point": res_cuboid_point, "wf3d": res_wf3d,
          "cuboid_line": res_cuboid_line}


# ===========================================================================
# problem state
# ===========================================================================
# ---------------------------------------------------------------------------
# inter-group relations (Section 3.2, "Inter-Group Relations"; Appendix C, Manhattan / Atlanta world):
# orthogonality or parallelism between two group directions -- VP directions and plane normals.  They involve
# only kept-set parameters, so they add to H_gg and g_g alone.  Readings (the paper gives no formula): the
# directions are unit vectors a, b; orthogonality r = a . b (the cosine), parallelism r = a x b (the sine, as
# a vector, the form of the VP residual); both are angular and scale-free, so they take the VP term's weight
# and Cauchy scale and stay out of E_px.  Residuals are 3-vectors (an orthogonality residual is padded with
# zeros, which changes neither the cost nor the normal equations).
# ---------------------------------------------------------------------------
REL_ORTH, REL_PAR = 0, 1


def _group_direction(g, kind, d):
    """Unit direction of a group after its increment: a plane's normal (kind 0, d = 3 plane increments;
    the offset increment does not move it) or a VP (kind 1, d[:2])."""
    n_plane = plane_plus(g, d)[:3]
    v = vp_plus(g[:3], d[:2])
    return torch.where(kind == 0, n_plane, v)


def res_relation(da, db, ga, gb, ka, kb, typ):
    a = _group_direction(ga, ka, da)
    b = _group_direction(gb, kb, db)
    orth = torch.stack([(a * b).sum(), torch.zeros((), dtype=a.dtype), torch.zeros((), dtype=a.dtype)])
    par = torch.linalg.cross(a, b)
    return torch.where(typ == REL_ORTH, orth, par)


def _rel_records(state, rel):
    n = len(rel["a"])
    ga = torch.zeros((n, 4)); gb = torch.zeros((n, 4))
    for side, g in (("a", ga), ("b", gb)):
        k = np.asarray(rel["k" + side])
        idx = np.asarray(rel[side])
        pl = k == 0
        if pl.any():
            g[torch.from_numpy(pl)] = torch.from_numpy(state["planes"][idx[pl]])
        if (~pl).any():
            g[torch.from_numpy(~pl), :3] = torch.from_numpy(state["vps"][idx[~pl]])
    to_t = lambda x: torch.from_numpy(np.asarray(x, np.int64))
    return ga, gb, to_t(rel["ka"]), to_t(rel["kb"]), to_t(rel["type"])


def relation_residuals(state, rel, with_jac=False):
    """r [n, 3] and, with with_jac, J w.r.t. the increments of group a and group b (3 each; a VP uses 2)."""
    ga, gb, ka, kb, ty = _rel_records(state, rel)
    n = ga.shape[0]
    da = torch.zeros((n, 3)); db = torch.zeros((n, 3))
    if n == 0:
        z = torch.zeros((0, 3))
        return (z, torch.zeros((0, 3, 3)), torch.zeros((0, 3, 3))) if with_jac else z
    if with_jac:
        def f2(*x):
            r = res_relation(*x)
            return r, r
        jac, r = vmap(jacfwd(f2, argnums=(0, 1), has_aux=True))(da, db, ga, gb, ka, kb, ty)
        return r, jac[0], jac[1]
    return vmap(res_relation)(da, db, ga, gb, ka, kb, ty)


def normalize_lines(L):
    L = np.array(L, dtype=np.float64, copy=True)
    dn = np.linalg.norm(L[:, :3], axis=1, keepdims=True)
    return L / dn


def state_from_scene(scene):
    c = scene["cams"]
    st = dict(
        cams=np.concatenate([c["q"] / np.linalg.norm(c["q"], axis=1, keepdims=True), c["t"],
                             c["intr"], c["pp"]], 1).astype(np.float64),
        points=np.array(scene["points"], np.float64),
        lines=normalize_lines(scene["lines"]) if len(scene["lines"]) else np.zeros((0, 6)),
        planes=np.array(scene["planes"], np.float64).reshape(-1, 4),
        vps=np.array(scene["vps"], np.float64).reshape(-1, 3),
        spheres=np.array(scene.get("spheres", np.zeros((0, 4))), np.float64).reshape(-1, 4),
        cylinders=np.array(scene.get("cylinders", np.zeros((0, 7))), np.float64).reshape(-1, 7),
        cones=np.array(scene.get("cones", np.zeros((0, 7))), np.float64).reshape(-1, 7),
    )
    # ellipsoids (q, c, s) and cuboids (q, d_0..d_5) as given; the state keeps R (row-major) for the quaternion
    for key in ("ellipsoids", "cuboids"):
        g = np.array(scene.get(key, np.zeros((0, 10))), np.float64).reshape(-1, 10)
        q = g[:, :4] / np.linalg.norm(g[:, :4], axis=1, keepdims=True) if len(g) else g[:, :4]
        R = quat_to_R(torch.from_numpy(q)).numpy().reshape(-1, 9)
        st[key] = np.concatenate([R, g[:, 4:]], 1)
    if len(st["cylinders"]):
        # the axis as a Pluecker line with |d| = 1
        st["cylinders"][:, :6] = normalize_lines(st["cylinders"][:, :6])
    if len(st["cones"]):
        st["cones"][:, 3:6] /= np.linalg.norm(st["cones"][:, 3:6], axis=1, keepdims=True)
    if len(st["planes"]):
        # the plane n.x + w = 0 is homogeneous in (n, w): rescale both so that |n| = 1
        st["planes"] /= np.linalg.norm(st["planes"][:, :3], axis=1, keepdims=True)
    if len(st["vps"]):
        st["vps"] /= np.linalg.norm(st["vps"], axis=1, keepdims=True)
    w3 = scene.get("obs", {}).get("wf3d")
    if w3 is not None and len(w3["other"]):
        # the 3D wireframe distance couples a point with a line feature: its points join the reduced system
        st["jpoints"] = np.unique(np.asarray(w3["other"], np.int64))
    ik = scene.get("intrinsics")
    if ik is not None:
        # refined intrinsics (Section 3.1, K_c(i): image i uses the intrinsics of its camera model c(i)): the
        # entities' (f, k1, k2) are parameters, and every camera's copy is the value of its entity
        st["intr"] = np.array(ik["values"], np.float64).reshape(-1, 3)
        st["cam_k"] = np.asarray(ik["of_cam"], np.int64).copy()
        st["cams"][:, 7:10] = st["intr"][st["cam_k"]]
    return st


def _records(state, obs, kind):
    """Gather the per-residual inputs of one kind as float64 tensors."""
    o = obs[kind]
    n = len(o["feat"])
    cam = torch.zeros((n, 12), dtype=DT)
    if HAS_CAM[kind] and n:
        cam = torch.from_numpy(state["cams"][o["cam"]])
    ft = FEAT[kind]
    src = state["points"] if ft == "point" else state["lines"]
    feat = torch.zeros((n, 6), dtype=DT)
    if n:
        feat[:, : src.shape[1]] = torch.from_numpy(src[o["feat"]])
    grp = torch.zeros((n, 16), dtype=DT)
    gk = GROUP.get(kind)
    if gk and n:
        g = state[GKEY[gk][0]]
        grp[:, : g.shape[1]] = torch.from_numpy(g[o["other"]])
    meas = torch.zeros((n, 4), dtype=DT)
    m = np.asarray(o["meas"]).reshape(n, -1)
    if m.shape[1]:
        meas[:, : m.shape[1]] = torch.from_numpy(m)
    return cam, feat, grp, meas


def with_intrinsics_increment(fn):
    """The residual as a function of an additive increment dk of the camera's (f, k1, k2) as well
    (refined intrinsics, Section 3.1): fn(dc, df, dg, dk, cam, ...) = fn(dc, df, dg, cam + [0 dk 0], ...)."""
    def g(dc, df, dg, dk, cam, feat, grp, meas):
        return fn(dc, df, dg, torch.cat([cam[:7], cam[7:10] + dk, cam[10:]]), feat, grp, meas)
    return g


def residuals(state, obs, kind, with_jac=False, chunk=200_000, with_intr=False):
    """r [n, rdim], valid [n] and, with with_jac, J w.r.t. (cam 6, feature k, group 3) increments, and with
    with_intr also J w.r.t. the additive (f, k1, k2) increment of the camera (zero for kinds without one)."""
    cam, feat, grp, meas = _records(state, obs, kind)
    n = cam.shape[0]
    kf = FDOF[FEAT[kind]]
    fn = RES_FN[kind]
    rd = RDIM[kind]
    nj = 4 if with_intr else 3
    if n == 0:
        z = torch.zeros((0, rd))
        out = (z, torch.zeros(0, dtype=torch.bool))
        if with_jac:
            out = out + (torch.zeros((0, rd, 6)), torch.zeros((0, rd, kf)), torch.zeros((0, rd, 3)))
            if with_intr:
                out = out + (torch.zeros((0, rd, 3)),)
        return out
    dc = torch.zeros((n, 6)); df = torch.zeros((n, kf)); dk = torch.zeros((n, 3))
    dg = torch.zeros((n, GDOF[GROUP[kind]] if kind in GROUP else 3))
    rs, vs, Js = [], [], [[] for _ in range(nj)]
    fk = with_intrinsics_increment(fn) if with_intr else fn
    for s in range(0, n, chunk):
        sl = slice(s, s + chunk)
        args = (dc[sl], df[sl], dg[sl]) + ((dk[sl],) if with_intr else ()) + (cam[sl], feat[sl], grp[sl], meas[sl])
        if with_jac:
            def f2(*a):
                r, v = fk(*a)
                return r, (r, v)
            jac, (r, v) = vmap(jacfwd(f2, argnums=tuple(range(nj)), has_aux=True))(*args)
            for i in range(nj):
                Js[i].append(jac[i])
        else:
            r, v = vmap(fk)(*args)
        rs.append(r); vs.append(v)
    out = (torch.cat(rs), torch.cat(vs))
    if with_jac:
        out = out + tuple(torch.cat(J) for J in Js)
    return out


def cost(state, obs, opt: Options):
    """(E, E_px): E = 1/2 sum w a^2 ln(1 + |r|^2/a^2); E_px omits the VP (angular) terms and the direct 3D
    group distances (not pixel terms)."""
    E = 0.0
    Epx = 0.0
    for k in KINDS:
        if k not in obs or len(obs[k]["feat"]) == 0:
            continue
        r, v = residuals(state, obs, k)
        a = opt.scale(k)
        s = (r * r).sum(-1)
        e = 0.5 * opt.weight(k) * a * a * torch.log1p(s / (a * a))
        e = torch.where(v, e, torch.zeros_like(e))
        tot = float(e.sum())
        E += tot
        if k not in NON_PIXEL:
            Epx += tot
    rel = obs.get("relations")
    if rel is not None and len(rel["a"]):
        r = relation_residuals(state, rel)
        a = opt.cauchy_rel
        E += float((0.5 * opt.w_rel * a * a * torch.log1p((r * r).sum(-1) / (a * a))).sum())
    return E, Epx


# ===========================================================================
# the normal equations (Eq. 2 / Eq. 5) and the Schur complement (Eq. 3)
# ===========================================================================
class Layout:
    """Column layout of the full system: [cameras | planes | VPs | intrinsics | points | lines].

    `fixed` holds camera pose components constant (gauge): per camera a bit mask over the six pose
    increments (bits 0-2 rotation, 3-5 translation; 0x3F = the whole pose), or a boolean (True = 0x3F).
    Held components get no column.  With refined intrinsics (state "intr" / "cam_k") every intrinsics
    entity K_c (Section 3.1) takes three columns (f, k1, k2), whatever the pose mask of its cameras."""

    def __init__(self, state, fixed=None):
        self.nc = state["cams"].shape[0]
        self.npl = state["planes"].shape[0]
        self.nv = state["vps"].shape[0]
        self.np_ = state["points"].shape[0]
        self.nl = state["lines"].shape[0]
        mask = np.zeros(self.nc, np.uint8) if fixed is None else np.asarray(fixed)
        if mask.dtype == bool:
            mask = np.where(mask, 0x3F, 0).astype(np.uint8)
        self.held = ((mask.astype(np.int64)[:, None] >> np.arange(6)[None, :]) & 1).astype(bool)
        self.fixed = self.held.all(1)
        self.cam_cols = np.full((self.nc, 6), -1, np.int64)
        free = ~self.held
        self.cam_cols[free] = np.arange(int(free.sum()))
        o = int(free.sum())
        self.plane_col = o + 3 * np.arange(self.npl); o += 3 * self.npl
        self.vp_col = o + 2 * np.arange(self.nv); o += 2 * self.nv
        # the other group types (Appendix B), after the VPs: spheres (4), cylinders (5), cones (6)
        self.ngs = {}
        self.gcol = {"plane": self.plane_col, "vp": self.vp_col}
        for gk in SURFACES:
            ng = state[GKEY[gk][0]].shape[0] if GKEY[gk][0] in state else 0
            self.ngs[gk] = ng
            self.gcol[gk] = o + GDOF[gk] * np.arange(ng); o += GDOF[gk] * ng
        # a 9-parameter group's first 6 increments, then (after all of its kind) its last 3
        self.gcol2 = {}
        for gk in SPLIT:
            ng = state[GKEY[gk][0]].shape[0] if GKEY[gk][0] in state else 0
            self.ngs[gk] = ng
            self.gcol[gk] = o + 6 * np.arange(ng); o += 6 * ng
            self.gcol2[gk] = o + 3 * np.arange(ng); o += 3 * ng
        self.nk = state["intr"].shape[0] if "intr" in state else 0
        self.cam_k = state["cam_k"] if self.nk else np.full(self.nc, -1, np.int64)
        self.intr_col = o + 3 * np.arange(self.nk); o += 3 * self.nk
        # points coupled with a line feature by the 3D wireframe distance: entities of A (after the intrinsics),
        # the other points features
        self.jpoints = np.asarray(state.get("jpoints", np.zeros(0, np.int64)), np.int64)
        self.point_col = np.full(self.np_, -1, np.int64)
        self.point_col[self.jpoints] = o + 3 * np.arange(len(self.jpoints)); o += 3 * len(self.jpoints)
        self.na = o
        rest = np.setdiff1d(np.arange(self.np_), self.jpoints)
        self.point_col[rest] = o + 3 * np.arange(len(rest)); o += 3 * len(rest)
        self.gcol["jpoint"] = self.point_col
        self.line_col = o + 4 * np.arange(self.nl); o += 4 * self.nl
        self.n = o
        # entity blocks of A (for block-Jacobi): (start, size); a camera's free columns are contiguous
        nfree = free.sum(1)
        self.a_blocks = ([(int(self.cam_cols[i][free[i]][0]), int(nfree[i])) for i in range(self.nc) if nfree[i]] +
                         [(int(c), 3) for c in self.plane_col] + [(int(c), 2) for c in self.vp_col] +
                         [(int(c), GDOF[gk]) for gk in SURFACES for c in self.gcol[gk]] +
                         [(int(c), w) for gk in SPLIT for cs, w in ((self.gcol[gk], 6), (self.gcol2[gk], 3))
                          for c in cs] +
                         [(int(c), 3) for c in self.intr_col] +
                         [(int(self.point_col[j]), 3) for j in self.jpoints])
        self.f_blocks = [(int(c), 3) for c in self.point_col[rest]] + [(int(c), 4) for c in self.line_col]


def linearize(state, obs, opt: Options, lay: Layout):
    """Weighted Jacobian J~ = sqrt(w) J (sparse) and r~ = sqrt(w) r with IRLS weights
    w = weight / (1 + |r|^2/a^2) (plain IRLS, no second-order correction)."""
    rows, cols, vals, rt = [], [], [], []
    row0 = 0
    for k in KINDS:
        o = obs.get(k)
        n = len(o["feat"]) if o is not None else 0
        if n == 0:
            continue
        r, v, Jc, Jf, Jg, *Jk = residuals(state, obs, k, with_jac=True, with_intr=lay.nk > 0)
        a = opt.scale(k)
        s = (r * r).sum(-1)
        om = opt.weight(k) / (1 + s / (a * a))
        om = torch.where(v, om, torch.zeros_like(om))
        sq = torch.sqrt(om).numpy()
        rd = RDIM[k]
        ridx = row0 + np.arange(n)[:, None] * rd + np.arange(rd)[None, :]          # [n, rd]
        blocks = []   # (J [n, rd, w], columns [n, w], column present [n, w])
        if HAS_CAM[k]:
            cc = lay.cam_cols[o["cam"]]
            blocks.append((Jc.numpy(), cc, cc >= 0))
            if lay.nk:
                ck = lay.cam_k[o["cam"]]
                kc = np.where(ck >= 0, lay.intr_col[np.maximum(ck, 0)], 0)[:, None] + np.arange(3)[None, :]
                blocks.append((Jk[0].numpy(), kc, np.broadcast_to((ck >= 0)[:, None], (n, 3))))
        ft = FEAT[k]
        fc = (lay.point_col if ft == "point" else lay.line_col)[o["feat"]]
        w = FDOF[ft]
        blocks.append((Jf.numpy(), fc[:, None] + np.arange(w)[None, :], np.ones((n, w), bool)))
        gk = GROUP.get(k)
        if gk in SPLIT:
            for cols_, j0, w in ((lay.gcol[gk], 0, 6), (lay.gcol2[gk], 6, 3)):
                gc = cols_[o["other"]]
                blocks.append((Jg.numpy()[:, :, j0:j0 + w], gc[:, None] + np.arange(w)[None, :], np.ones((n, w), bool)))
        elif gk:
            gc = lay.gcol[gk][o["other"]]
            w = GDOF[gk]
            blocks.append((Jg.numpy()[:, :, :w], gc[:, None] + np.arange(w)[None, :], np.ones((n, w), bool)))
        for J, C0, ok in blocks:
            w = C0.shape[1]
            J = J * sq[:, None, None]
            R_ = np.broadcast_to(ridx[:, :, None], (n, rd, w))
            C_ = np.broadcast_to(C0[:, None, :], (n, rd, w))
            m = np.broadcast_to(ok[:, None, :], (n, rd, w))
            rows.append(R_[m]); cols.append(C_[m]); vals.append(J[m])
        rt.append((r.numpy() * sq[:, None]).reshape(-1))
        row0 += n * rd
    rel = obs.get("relations")
    if rel is not None and len(rel["a"]):
        r, Ja, Jb = relation_residuals(state, rel, with_jac=True)
        n = r.shape[0]
        a = opt.cauchy_rel
        om = opt.w_rel / (1 + (r * r).sum(-1) / (a * a))
        sq = torch.sqrt(om).numpy()
        ridx = row0 + np.arange(n)[:, None] * 3 + np.arange(3)[None, :]
        for side, J in (("a", Ja.numpy()), ("b", Jb.numpy())):
            k = np.asarray(rel["k" + side]); idx = np.asarray(rel[side])
            for kind, colmap, w in ((0, lay.plane_col, 3), (1, lay.vp_col, 2)):
                m = k == kind
                if not m.any():
                    continue
                C0 = colmap[idx[m]][:, None] + np.arange(w)[None, :]
                Jm = J[m][:, :, :w] * sq[m][:, None, None]
                nm = int(m.sum())
                R_ = np.broadcast_to(ridx[m][:, :, None], (nm, 3, w))
                C_ = np.broadcast_to(C0[:, None, :], (nm, 3, w))
                rows.append(R_.ravel()); cols.append(C_.ravel()); vals.append(Jm.ravel())
        rt.append((r.numpy() * sq[:, None]).reshape(-1))
        row0 += 3 * n
    Jt = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(row0, lay.n))
    return Jt, np.concatenate(rt)


def _block_diag_inverse(H, blocks):
    """Inverse of the block-diagonal part of H on the given (start, size) blocks, as sparse."""
    rows, cols, vals = [], [], []
    for size in sorted({s for _, s in blocks}):
        starts = np.array([b for b, s in blocks if s == size], np.int64)
        if len(starts) == 0:
            continue
        idx = starts[:, None] + np.arange(size)[None, :]
        ri = np.broadcast_to(idx[:, :, None], (len(starts), size, size)).ravel()
        ci = np.broadcast_to(idx[:, None, :], (len(starts), size, size)).ravel()
        B = np.asarray(H[ri, ci]).reshape(len(starts), size, size)          # [nb, s, s]
        Bi = np.linalg.inv(B)
        rows.append(np.broadcast_to(idx[:, :, None], Bi.shape).ravel())
        cols.append(np.broadcast_to(idx[:, None, :], Bi.shape).ravel())
        vals.append(Bi.ravel())
    n = H.shape[0]
    if not rows:
        return sp.csr_matrix((n, n))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def normal_equations(Jt, rt):
    """H = J~^T J~ and g = J~^T r~ (Eq. 2 / Eq. 5)."""
    H = (Jt.T @ Jt).tocsr()
    g = Jt.T @ rt
    return H, g


def damping_diag(H):
    """D = clamp(diag H, 1e-6, 1e32)."""
    return np.clip(H.diagonal(), 1e-6, 1e32)


def reduced_system(H, g, lam, lay: Layout):
    """Damp both blocks by lam*D, eliminate the features:
    S = H_aa + lam D_a - H_af (H_ff + lam D_f)^-1 H_fa,  b = -g_a + H_af (H_ff + lam D_f)^-1 g_f (Eq. 3 / Eq. 5)."""
    D = damping_diag(H)
    Hl = (H + sp.diags(lam * D)).tocsr()
    na = lay.na
    Haa = Hl[:na, :na]
    Haf = Hl[:na, na:]
    Hff = Hl[na:, na:]
    fb = [(s - na, k) for s, k in lay.f_blocks]
    Hffi = _block_diag_inverse(Hff, fb)
    S = (Haa - Haf @ Hffi @ Haf.T).tocsr()
    b = -g[:na] + Haf @ (Hffi @ g[na:])
    return S, b, Hffi, Haf, D


def pcg(S, b, blocks, tol, max_iters):
    """Block-Jacobi preconditioned CG from x0 = 0; stops when |r_k| <= tol |b| (recurrence residual)."""
    Minv = _block_diag_inverse(S.tocsr(), blocks)
    x = np.zeros_like(b)
    bn = float(np.sqrt(b @ b))
    if bn == 0.0:
        return x, 0, 0.0
    r = b.copy()
    z = Minv @ r
    p = z.copy()
    rz = float(r @ z)
    it = 0
    rn = bn
    while it < max_iters:
        Ap = S @ p
        alpha = rz / float(p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        it += 1
        rn = float(np.sqrt(r @ r))
        if rn <= tol * bn:
            break
        z = Minv @ r
        rz_new = float(r @ z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return x, it, rn / bn


def apply_step(state, delta, lay: Layout):
    """x (+) delta with the retractions above; returns a new state."""
    new = {k: v.copy() for k, v in state.items()}
    free = np.nonzero(~lay.fixed)[0]
    if len(free):
        cols = lay.cam_cols[free]
        dp = torch.from_numpy(np.where(cols >= 0, delta[np.maximum(cols, 0)], 0.0))
        c = torch.from_numpy(state["cams"][free])
        R, t = pose_plus(c[:, :4], c[:, 4:7], dp)
        new["cams"][free, :4] = R_to_quat(R.numpy())
        new["cams"][free, 4:7] = t.numpy()
    if lay.npl:
        d = delta[lay.plane_col[:, None] + np.arange(3)]
        new["planes"] = plane_plus(torch.from_numpy(state["planes"]), torch.from_numpy(d)).numpy()
    if lay.nv:
        d = delta[lay.vp_col[:, None] + np.arange(2)]
        new["vps"] = vp_plus(torch.from_numpy(state["vps"]), torch.from_numpy(d)).numpy()
    for gk in SURFACES + SPLIT:
        if lay.ngs[gk]:
            key = GKEY[gk][0]
            if gk in SPLIT:
                d = np.concatenate([delta[lay.gcol[gk][:, None] + np.arange(6)],
                                    delta[lay.gcol2[gk][:, None] + np.arange(3)]], 1)
            else:
                d = delta[lay.gcol[gk][:, None] + np.arange(GDOF[gk])]
            new[key] = GROUP_PLUS[gk](torch.from_numpy(state[key]), torch.from_numpy(d)).numpy()
    if lay.nk:
        # intrinsics: additive; every camera's copy follows its entity
        new["intr"] = state["intr"] + delta[lay.intr_col[:, None] + np.arange(3)]
        has = lay.cam_k >= 0
        new["cams"][has, 7:10] = new["intr"][lay.cam_k[has]]
    if lay.np_:
        new["points"] = state["points"] + delta[lay.point_col[:, None] + np.arange(3)]
    if lay.nl:
        d = delta[lay.line_col[:, None] + np.arange(4)]
        new["lines"] = line_plus(torch.from_numpy(state["lines"]), torch.from_numpy(d)).numpy()
    return new


def solve_step(state, obs, opt: Options, lam, lay: Layout, lin=None):
    """The full-system step at damping lam: returns (delta, info)."""
    Jt, rt = lin if lin is not None else linearize(state, obs, opt, lay)
    H, g = normal_equations(Jt, rt)
    S, b, Hffi, Haf, D = reduced_system(H, g, lam, lay)
    if opt.solver == "dense":
        da = np.linalg.solve(S.toarray(), b) if lay.na else np.zeros(0)
        it, rel = 0, 0.0
    else:
        da, it, rel = pcg(S, b, lay.a_blocks, opt.pcg_rel_tol, opt.pcg_max_iters)
    na = lay.na
    df = -(Hffi @ (g[na:] + Haf.T @ da))
    delta = np.concatenate([da, df])
    Jd = Jt @ delta
    pred = -float(g @ delta) - 0.5 * float(Jd @ Jd)
    return delta, dict(pcg_iters=it, pcg_rel=rel, pred=pred, S=S, b=b, g=g, H=H, D=D)


@dataclasses.dataclass
class LMState:
    lam: float
    nu: float = 2.0


def lm_update(lm: LMState, gain, E_new, opt: Options):
    """The accept test and the damping update (Madsen, Nielsen & Tingleff 2004, Sec. 3.2, Nielsen's rule).
    Accept when the candidate cost is finite and the gain ratio exceeds min_gain (a tie rejects); then
    lambda <- lambda * max(1/3, 1 - (2 gain - 1)^3), clamped to [lambda_min, lambda_max], and nu <- 2.
    Otherwise lambda <- min(lambda * nu, lambda_max) and nu <- 2 nu.  Returns the decision."""
    accepted = bool(np.isfinite(E_new) and gain > opt.min_gain)
    if accepted:
        lm.lam = min(max(lm.lam * max(1.0 / 3.0, 1.0 - (2.0 * gain - 1.0) ** 3), opt.lambda_min), opt.lambda_max)
        lm.nu = 2.0
    else:
        lm.lam = min(lm.lam * lm.nu, opt.lambda_max)
        lm.nu *= 2.0
    return accepted


def step_converged(rep, opt: Options):
    """Termination test of Section 3.5: an accepted step whose relative change of the pixel-space cost
    E_px (the VP angular terms excluded, Appendix C) is below rel_cost_tol."""
    if not rep["accepted"]:
        return False
    return abs(rep["Epx"] - rep["Epx_new"]) / max(rep["Epx"], 1e-300) < opt.rel_cost_tol


def lm_step(state, obs, opt: Options, lm: LMState, lay: Layout, cur=None, lin=None):
    """One LM iteration (build, damp, eliminate, solve, back-substitute, evaluate, decide).
    Acceptance: gain ratio > min_gain; lambda update by Nielsen's rule
    (Madsen, Nielsen & Tingleff 2004, Sec. 3.2), lambda clamped to [lambda_min, lambda_max]."""
    E, Epx = cur if cur is not None else cost(state, obs, opt)
    delta, info = solve_step(state, obs, opt, lm.lam, lay, lin)
    cand = apply_step(state, delta, lay)
    E2, Epx2 = cost(cand, obs, opt)
    pred = info["pred"]
    gain = (E - E2) / pred if pred > 0 else -np.inf
    lam_used = lm.lam
    accepted = lm_update(lm, gain, E2, opt)
    rep = dict(E=E, Epx=Epx, E_new=E2, Epx_new=Epx2, gain=gain, accepted=accepted, lam=lam_used,
               pcg_iters=info["pcg_iters"], pcg_rel=info["pcg_rel"], pred=pred, delta=delta)
    return (cand if accepted else state), rep


def solve(scene_or_state, obs, opt: Options = None, max_iters=20, fixed=None, history=False):
    """LM until an accepted step with |dE_px|/E_px < rel_cost_tol (Section 3.5) or max_iters."""
    opt = opt or Options()
    state = scene_or_state if "cams" in scene_or_state and isinstance(scene_or_state["cams"], np.ndarray) \
        else state_from_scene(scene_or_state)
    lay = Layout(state, fixed)
    lm = LMState(opt.lambda0)
    cur = cost(state, obs, opt)
    reps = []
    converged = False
    for _ in range(max_iters):
        state, rep = lm_step(state, obs, opt, lm, lay, cur)
        rep.pop("delta")
        reps.append(rep)
        if rep["accepted"]:
            cur = (rep["E_new"], rep["Epx_new"])
            if step_converged(rep, opt):
                converged = True
                break
    return state, dict(iters=len(reps), converged=converged, reports=reps, E=cur[0], Epx=cur[1])
