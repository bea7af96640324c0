"""FP64 CPU oracle of the learned block-Jacobi correction (TEST INFRASTRUCTURE ONLY).

The paper has no learned component; this part follows the specification of the benchmark's fifth
workload: a small per-block MLP, trained on reduced systems that the method itself produces, predicts a
correction of the block-Jacobi inverse of S; blocks whose corrected inverse is not positive definite fall
back to plain block-Jacobi.  The definitions written out here (one per function) are the ones the CUDA
kernels must reproduce:

  features(S)      per block row b of the padded reduced system (6-wide blocks):
                   D_b = diag(S_bb); S^_bb = D_b^-1/2 S_bb D_b^-1/2 (21 upper entries, row-major);
                   over the off-diagonal blocks c of row b, n_bc = || D_b^-1/2 S_bc D_c^-1/2 ||_F:
                   log(1 + count), sum n, max n, sum n^2; the entity type one-hot (camera, plane, VP);
                   zero padding to 32 values.
  mlp(x)           y = W2^T relu(W1^T ((x - mu) / sigma) + b1) + b2, 32 -> 128 -> 21.
  correction       M^_b = inv(S^_bb) + sym(y) with sym filling both triangles from the 21 upper values;
                   entries in padded or held dimensions of a block are not corrected.
  target           T^_b = D_b^1/2 [S^-1]_bb D_b^1/2 (the Jacobi-scaled diagonal block of the exact inverse).
  loss             mean over blocks of || M^_b - T^_b ||_F^2.
  preconditioner   M_b = D_b^-1/2 M^_b D_b^-1/2 if it is positive definite (Cholesky succeeds),
                   else inv(S_bb).
  adam             Kingma & Ba (2015), Algorithm 1, with bias correction.
Pinned by tests/test_precond_oracle.py (finite differences, closed forms, the dense inverse).
"""
from __future__ import annotations

import numpy as np

NF = 32      # input width
NH = 128     # hidden width
NO = 21      # outputs: upper triangle of a symmetric 6x6
IU, JU = np.triu_indices(6)          # row-major upper triangle, the same order as the CUDA code

# parameter blob: mu (32), sigma (32), W1 (32 x 128, row = input), b1 (128), W2 (128 x 21, row = hidden), b2 (21)
SIZES = [("mu", (NF,)), ("sigma", (NF,)), ("W1", (NF, NH)), ("b1", (NH,)), ("W2", (NH, NO)), ("b2", (NO,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)
NTRAIN = NPARAM - 2 * NF           # everything after mu and sigma is trained


def unpack(blob):
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(blob[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in SIZES])


def sym_from_upper(u):
    """[n, 21] upper entries -> [n, 6, 6] symmetric."""
    M = np.zeros(u.shape[:-1] + (6, 6))
    M[..., IU, JU] = u
    M[..., JU, IU] = u
    return M


def real_dims(ent_type, held):
    """[na, 6] bool: dimensions that are real (not padding of a group block, not a held camera component)."""
    nd = np.where(ent_type == 0, 6, np.where(ent_type == 1, 3, 2))
    m = np.arange(6)[None, :] < nd[:, None]
    return m & ~held


def features(row_ptr, cols, vals, ent_type):
    """Inputs of the network for every block row (see module docstring).  vals: [nnzb, 6, 6]."""
    na = len(row_ptr) - 1
    diag = np.zeros((na, 6))
    for a in range(na):
        for q in range(row_ptr[a], row_ptr[a + 1]):
            if cols[q] == a:
                diag[a] = np.diag(vals[q])
    sd = 1.0 / np.sqrt(diag)
    X = np.zeros((na, NF))
    for a in range(na):
        cnt, s1, mx, s2 = 0, 0.0, 0.0, 0.0
        for q in range(row_ptr[a], row_ptr[a + 1]):
            c = cols[q]
            Bs = sd[a][:, None] * vals[q] * sd[c][None, :]
            if c == a:
                X[a, :NO] = Bs[IU, JU]
            else:
                n = float(np.sqrt((Bs * Bs).sum()))
                cnt += 1; s1 += n; mx = max(mx, n); s2 += n * n
        X[a, 21:25] = [np.log1p(cnt), s1, mx, s2]
        X[a, 25 + int(ent_type[a])] = 1.0
    return X, diag


def mlp_forward(p, X):
    Z = (X - p["mu"]) / p["sigma"]
    A = Z @ p["W1"] + p["b1"]
    H = np.maximum(A, 0.0)
    return H @ p["W2"] + p["b2"], (Z, A, H)


def corrected_scaled(Shat_inv, Y, mask):
    """M^ = inv(S^) + sym(Y), with no correction in masked-out (padded / held) dimensions."""
    D = sym_from_upper(Y) * (mask[:, :, None] & mask[:, None, :])
    return Shat_inv + D


def loss_and_grad(p, X, E, mask):
    """loss = mean_b || sym(Y_b) - E_b ||_F^2 restricted to real dims, E_b = T^_b - inv(S^_bb);
    returns (loss, gradient dict over the trained parameters)."""
    n = X.shape[0]
    Y, (Z, A, H) = mlp_forward(p, X)
    mm = (mask[:, :, None] & mask[:, None, :]).astype(np.float64)
    R = (sym_from_upper(Y) - E) * mm                        # residual matrix (masked)
    loss = float((R * R).sum() / n)
    # d loss / d Y (upper entries): diagonal entries appear once, off-diagonal twice
    w = np.where(IU == JU, 1.0, 2.0)
    dY = 2.0 * w[None, :] * R[:, IU, JU] / n
    g = {}
    g["W2"] = H.T @ dY
    g["b2"] = dY.sum(0)
    dH = dY @ p["W2"].T
    dA = dH * (A > 0)
    g["W1"] = Z.T @ dA
    g["b1"] = dA.sum(0)
    return loss, g


def grad_vector(g):
    return np.concatenate([g[k].ravel() for k in ("W1", "b1", "W2", "b2")])


def adam_step(theta, m, v, grad, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015, Algorithm 1) on flat arrays; t is the 1-based step count."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def targets(S_dense, diag):
    """T^_b for every block row: the Jacobi-scaled 6x6 diagonal blocks of inv(S)."""
    na = diag.shape[0]
    Si = np.linalg.inv(S_dense)
    out = np.zeros((na, 6, 6))
    for a in range(na):
        sl = slice(6 * a, 6 * a + 6)
        s = np.sqrt(diag[a])
        out[a] = s[:, None] * Si[sl, sl] * s[None, :]
    return out


def scaled_diag_inverse(row_ptr, cols, vals, diag):
    """inv(S^_bb) for every block row."""
    na = len(row_ptr) - 1
    out = np.zeros((na, 6, 6))
    for a in range(na):
        for q in range(row_ptr[a], row_ptr[a + 1]):
            if cols[q] == a:
                sd = 1.0 / np.sqrt(diag[a])
                out[a] = np.linalg.inv(sd[:, None] * vals[q] * sd[None, :])
    return out


def preconditioner(p, row_ptr, cols, vals, ent_type, held):
    """The learned block preconditioner M_b and a per-block flag (1 = fell back to block-Jacobi)."""
    X, diag = features(row_ptr, cols, vals, ent_type)
    Shi = scaled_diag_inverse(row_ptr, cols, vals, diag)
    mask = real_dims(ent_type, held)
    Y, _ = mlp_forward(p, X)
    Mh = corrected_scaled(Shi, Y, mask)
    sd = 1.0 / np.sqrt(diag)
    M = sd[:, :, None] * Mh * sd[:, None, :]
    fell = np.zeros(len(M), bool)
    for a in range(len(M)):
        try:
            np.linalg.cholesky(M[a])
        except np.linalg.LinAlgError:
            fell[a] = True
            M[a] = sd[a][:, None] * Shi[a] * sd[a][None, :]
    return M, fell
