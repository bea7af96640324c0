"""Pins of the learned-preconditioner oracle (CPU, FP64): finite-difference gradients, Adam's closed-form
first step, the exact-inverse target on decoupled systems, Jacobi-scaling invariance of the features and the
fall-back to block-Jacobi."""
import numpy as np
import pytest

from oracle import precond_oracle as PO


def random_params(rng, scale=0.3):
    p = {"mu": rng.normal(size=PO.NF) * 0.1, "sigma": rng.uniform(0.5, 2.0, PO.NF),
         "W1": rng.normal(size=(PO.NF, PO.NH)) * scale, "b1": rng.normal(size=PO.NH) * 0.1,
         "W2": rng.normal(size=(PO.NH, PO.NO)) * scale / 4, "b2": rng.normal(size=PO.NO) * 0.1}
    return p


def random_system(rng, na=7, ent=None, couple=0.15):
    """A random SPD block system in the padded 6-wide layout, full block-CSR with all blocks stored."""
    ent = np.array(ent if ent is not None else [0, 0, 0, 1, 1, 2, 2][:na])
    n = 6 * na
    A = rng.normal(size=(n, n)) * couple
    S = A @ A.T + np.diag(rng.uniform(1.0, 5.0, n))
    # padded dims of groups: unit diagonal, no coupling
    nd = np.where(ent == 0, 6, np.where(ent == 1, 3, 2))
    for a in range(na):
        for j in range(nd[a], 6):
            k = 6 * a + j
            S[k, :] = 0; S[:, k] = 0; S[k, k] = 1.0
    rp = np.arange(na + 1) * na
    cols = np.tile(np.arange(na), na)
    vals = np.stack([S[6 * a:6 * a + 6, 6 * c:6 * c + 6] for a in range(na) for c in range(na)])
    return S, rp, cols, vals, ent


def test_gradient_finite_differences():
    rng = np.random.default_rng(0)
    p = random_params(rng)
    X = rng.normal(size=(40, PO.NF))
    E = PO.sym_from_upper(rng.normal(size=(40, PO.NO)) * 0.2)
    mask = rng.random((40, 6)) > 0.2
    loss, g = PO.loss_and_grad(p, X, E, mask)
    gv = PO.grad_vector(g)
    blob = PO.pack(p)
    off = 2 * PO.NF
    h = 1e-6
    idx = rng.choice(PO.NTRAIN, 60, replace=False)
    for i in idx:
        bp = blob.copy(); bp[off + i] += h
        bm = blob.copy(); bm[off + i] -= h
        fd = (PO.loss_and_grad(PO.unpack(bp), X, E, mask)[0] - PO.loss_and_grad(PO.unpack(bm), X, E, mask)[0]) / (2 * h)
        assert abs(fd - gv[i]) <= 1e-6 * max(1.0, abs(gv[i])), (i, fd, gv[i])


def test_adam_first_step_closed_form():
    """From zero moments the bias-corrected first Adam step is -lr * g / (|g| + eps)."""
    rng = np.random.default_rng(1)
    g = rng.normal(size=100)
    th = rng.normal(size=100)
    t1, m, v = PO.adam_step(th, np.zeros(100), np.zeros(100), g, 1, lr=1e-3)
    np.testing.assert_allclose(t1, th - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_zero_network_on_decoupled_system_is_block_jacobi():
    """With no coupling the exact inverse's diagonal blocks are the block inverses: target = inv(S^_bb),
    so a zero network has zero loss and the preconditioner equals block-Jacobi."""
    rng = np.random.default_rng(2)
    S, rp, cols, vals, ent = random_system(rng, couple=0.0)
    X, diag = PO.features(rp, cols, vals, ent)
    T = PO.targets(S, diag)
    Shi = PO.scaled_diag_inverse(rp, cols, vals, diag)
    np.testing.assert_allclose(T, Shi, atol=1e-12)
    p = {k: np.zeros(s) for k, s in PO.SIZES}
    p["sigma"] = np.ones(PO.NF)
    held = np.zeros((len(ent), 6), bool)
    mask = PO.real_dims(ent, held)
    loss, _ = PO.loss_and_grad(p, X, T - Shi, mask)
    assert loss < 1e-24
    M, fell = PO.preconditioner(p, rp, cols, vals, ent, held)
    for a in range(len(ent)):
        np.testing.assert_allclose(M[a], np.linalg.inv(S[6 * a:6 * a + 6, 6 * a:6 * a + 6]), atol=1e-12)
    assert not fell.any()


def test_features_jacobi_scaling_invariant():
    """Scaling the system as L S L with positive diagonal L leaves every feature unchanged."""
    rng = np.random.default_rng(3)
    S, rp, cols, vals, ent = random_system(rng)
    X1, _ = PO.features(rp, cols, vals, ent)
    L = rng.uniform(0.1, 10.0, S.shape[0])
    S2 = L[:, None] * S * L[None, :]
    na = len(ent)
    vals2 = np.stack([S2[6 * a:6 * a + 6, 6 * c:6 * c + 6] for a in range(na) for c in range(na)])
    X2, _ = PO.features(rp, cols, vals2, ent)
    np.testing.assert_allclose(X1, X2, atol=1e-10)
    assert (X1[:, 21] == np.log1p(na - 1)).all()
    np.testing.assert_allclose(X1[:, 25:28].sum(1), 1.0)


def test_indefinite_correction_falls_back():
    rng = np.random.default_rng(4)
    S, rp, cols, vals, ent = random_system(rng)
    p = {k: np.zeros(s) for k, s in PO.SIZES}
    p["sigma"] = np.ones(PO.NF)
    p["b2"][0] = -50.0                   # a huge negative correction of entry (0,0): not positive definite
    held = np.zeros((len(ent), 6), bool)
    M, fell = PO.preconditioner(p, rp, cols, vals, ent, held)
    assert fell.all()
    for a in range(len(ent)):
        np.testing.assert_allclose(M[a], np.linalg.inv(S[6 * a:6 * a + 6, 6 * a:6 * a + 6]), atol=1e-10)
