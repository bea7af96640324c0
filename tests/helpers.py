"""Shared helpers of the GPU parity tests: run the CUDA library and the oracle on the same scene."""
import numpy as np

from oracle import ba_oracle as O


def gpu_problem(B, scene, precision=0, **opt):
    o = B.ba_default_options(precision=precision, **opt)
    p = B.ba_create(o)
    B.load_scene(p, scene)
    return p


def counts(scene):
    return (len(scene["cams"]["q"]), len(scene["planes"]), len(scene["vps"]), len(scene["points"]),
            len(scene["lines"]))


def gpu_S_dense(B, p):
    """The library's reduced system as a dense matrix over its padded 6-wide entity blocks."""
    rp, cols, vals, b = B.ba_export_reduced_system(p)
    na = len(rp) - 1
    S = np.zeros((6 * na, 6 * na))
    for a in range(na):
        for q in range(rp[a], rp[a + 1]):
            c = cols[q]
            S[6 * a:6 * a + 6, 6 * c:6 * c + 6] = vals[q]
    return S, b.reshape(-1)


def padded_to_oracle_index(scene, lay):
    """Indices into the padded 6-wide layout (cams | planes | VPs) of the oracle's kept-set columns."""
    nc, npl, nv = lay.nc, lay.npl, lay.nv
    idx = []
    for i in range(nc):
        idx += [6 * i + j for j in range(6) if not lay.held[i, j]]
    for g in range(npl):
        idx += list(range(6 * (nc + g), 6 * (nc + g) + 3))
    for v in range(nv):
        idx += list(range(6 * (nc + npl + v), 6 * (nc + npl + v) + 2))
    o = nc + npl + nv
    for gk in O.SURFACES:
        for g in range(lay.ngs.get(gk, 0) if hasattr(lay, "ngs") else 0):
            idx += list(range(6 * o, 6 * o + O.GDOF[gk]))
            o += 1
    for gk in O.SPLIT:   # a 9-parameter kind: all first entities (6), then all second entities (3)
        ng = lay.ngs.get(gk, 0) if hasattr(lay, "ngs") else 0
        for w in (6, 3):
            for g in range(ng):
                idx += list(range(6 * o, 6 * o + w))
                o += 1
    nk = getattr(lay, "nk", 0)
    for k in range(nk):
        idx += list(range(6 * (o + k), 6 * (o + k) + 3))
    for j in range(len(getattr(lay, "jpoints", ()))):   # points that the 3D wireframe distance names
        idx += list(range(6 * (o + nk + j), 6 * (o + nk + j) + 3))
    return np.array(idx, np.int64)


def oracle_delta_split(delta, lay):
    """Split an oracle full increment into the library's per-entity arrays."""
    cols = lay.cam_cols
    cam = np.where(cols >= 0, delta[np.maximum(cols, 0)], 0.0)
    plane = delta[lay.plane_col[:, None] + np.arange(3)] if lay.npl else np.zeros((0, 3))
    vp = delta[lay.vp_col[:, None] + np.arange(2)] if lay.nv else np.zeros((0, 2))
    point = delta[lay.point_col[:, None] + np.arange(3)] if lay.np_ else np.zeros((0, 3))
    line = delta[lay.line_col[:, None] + np.arange(4)] if lay.nl else np.zeros((0, 4))
    intr = delta[lay.intr_col[:, None] + np.arange(3)] if lay.nk else np.zeros((0, 3))
    return dict(cam=cam, plane=plane, vp=vp, point=point, line=line, intr=intr)


def oracle_setup(scene):
    st = O.state_from_scene(scene)
    lay = O.Layout(st, scene.get("fixed"))
    return st, lay


def rel(a, b):
    a = np.asarray(a, float); b = np.asarray(b, float)
    den = max(np.abs(b).max(), 1e-300) if b.size else 1.0
    return float(np.abs(a - b).max() / den) if a.size else 0.0


def gpu_S_sparse(B, p, scene, lay):
    """The library's reduced system in the oracle's column order as a scipy CSR matrix (padding dimensions
    dropped), and b in the same order.  For systems too large to hold densely."""
    import scipy.sparse as sp
    rp, cols, vals, b = B.ba_export_reduced_system(p)
    na = len(rp) - 1
    idx = padded_to_oracle_index(scene, lay)
    inv = np.full(6 * na, -1, np.int64)
    inv[idx] = np.arange(len(idx))
    brow = np.repeat(np.arange(na, dtype=np.int64), np.diff(rp))
    r = (6 * brow[:, None, None] + np.arange(6)[None, :, None]).repeat(6, 2)
    c = (6 * cols.astype(np.int64)[:, None, None] + np.arange(6)[None, None, :]).repeat(6, 1)
    ro, co = inv[r.ravel()], inv[c.ravel()]
    keep = (ro >= 0) & (co >= 0)
    n = len(idx)
    S = sp.csr_matrix((vals.ravel()[keep], (ro[keep], co[keep])), shape=(n, n))
    return S, b.reshape(-1)[idx]


def sparse_rel(A, Bm):
    """max |A - B| / max |B| over sparse matrices."""
    d = (A - Bm).tocsr()
    den = max(abs(Bm).max(), 1e-300)
    return float(abs(d).max() / den) if d.nnz else 0.0
