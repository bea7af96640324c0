"""GPU parity of the learned block-Jacobi correction against its CPU oracle (oracle/precond_oracle.py):
features, loss and gradient of the training kernels, the Adam step, and the inference blocks (with the
oracle using the same BF16-rounded weights the inference kernel reads)."""
import numpy as np
import pytest
import torch

from oracle import precond_oracle as PO
from scenegen import config, make_scene
from tests.helpers import gpu_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_04026_b300 import build
    build.build()
    import paper_2609_04026_b300 as B
    return B


@pytest.fixture(scope="module")
def system(B):
    s = make_scene(config("small"))
    p = gpu_problem(B, s, precision=B.BA_FP64, precond=B.BA_PRECOND_LEARNED)
    B.ba_build_reduced(p, 1e-3)
    rp, cols, vals, b = B.ba_export_reduced_system(p)
    na = len(rp) - 1
    ent = np.array([0] * len(s["cams"]["q"]) + [1] * len(s["planes"]) + [2] * len(s["vps"]))
    held = np.zeros((na, 6), bool)
    held[:len(s["fixed"])] = ((s["fixed"].astype(int)[:, None] >> np.arange(6)) & 1).astype(bool)
    yield B, p, s, rp, cols, vals, ent, held
    B.ba_destroy(p)


def bf16_round(a):
    return torch.tensor(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def test_features_match_oracle(system):
    B, p, s, rp, cols, vals, ent, held = system
    X, mask = B.ba_precond_features(p, len(rp) - 1)
    Xo, _ = PO.features(rp, cols, vals, ent)
    np.testing.assert_allclose(X, Xo, rtol=2e-6, atol=2e-6)
    mo = PO.real_dims(ent, held)
    np.testing.assert_array_equal(((mask[:, None].astype(int) >> np.arange(6)) & 1).astype(bool), mo)


def _random_blob(seed):
    rng = np.random.default_rng(seed)
    p = {"mu": rng.normal(size=PO.NF) * 0.1, "sigma": rng.uniform(0.5, 2.0, PO.NF),
         "W1": rng.normal(size=(PO.NF, PO.NH)) * 0.3, "b1": rng.normal(size=PO.NH) * 0.1,
         "W2": rng.normal(size=(PO.NH, PO.NO)) * 0.05, "b2": rng.normal(size=PO.NO) * 0.05}
    return PO.pack(p).astype(np.float32)


def test_gradient_matches_oracle(B):
    rng = np.random.default_rng(5)
    n = 1000
    X = rng.normal(size=(n, PO.NF)).astype(np.float32)
    E = (rng.normal(size=(n, PO.NO)) * 0.2).astype(np.float32)
    mask = rng.integers(0, 64, n).astype(np.uint8)
    blob = _random_blob(6)
    dev = torch.device("cuda")
    loss, grad = B.ba_mlp_grad(torch.from_numpy(X).to(dev), torch.from_numpy(E).to(dev),
                               torch.from_numpy(mask).to(dev), torch.from_numpy(blob).to(dev))
    m = ((mask[:, None].astype(int) >> np.arange(6)) & 1).astype(bool)
    lo, go = PO.loss_and_grad(PO.unpack(blob.astype(np.float64)), X.astype(np.float64),
                              PO.sym_from_upper(E.astype(np.float64)), m)
    gv = PO.grad_vector(go)
    g = grad.cpu().numpy().astype(np.float64)
    assert abs(loss - lo) <= 1e-5 * lo
    assert np.abs(g - gv).max() <= 1e-5 * np.abs(gv).max(), np.abs(g - gv).max() / np.abs(gv).max()


def test_adam_step_matches_oracle(B):
    rng = np.random.default_rng(7)
    n = 256
    X = rng.normal(size=(n, PO.NF)).astype(np.float32)
    E = (rng.normal(size=(n, PO.NO)) * 0.2).astype(np.float32)
    mask = np.full(n, 63, np.uint8)
    blob = _random_blob(8)
    dev = torch.device("cuda")
    Xd, Ed, Md = (torch.from_numpy(a).to(dev) for a in (X, E, mask))
    prm = torch.from_numpy(blob.copy()).to(dev)
    loss, grad = B.ba_mlp_grad(Xd, Ed, Md, prm)
    m = torch.zeros(PO.NTRAIN, dtype=torch.float32, device=dev)
    v = torch.zeros_like(m)
    B.ba_precond_train(Xd, Ed, Md, prm, m, v, 0, 1, n, 1e-3)
    th, _, _ = PO.adam_step(blob[64:].astype(np.float64), np.zeros(PO.NTRAIN), np.zeros(PO.NTRAIN),
                            grad.cpu().numpy().astype(np.float64), 1, 1e-3)
    np.testing.assert_allclose(prm.cpu().numpy()[64:], th, rtol=0, atol=2e-6)


def test_learned_blocks_match_oracle(system):
    B, p, s, rp, cols, vals, ent, held = system
    blob = _random_blob(9)
    B.ba_precond_set_weights(p, blob)
    M, fb = B.ba_precond_blocks(p, len(rp) - 1)
    pr = PO.unpack(blob.astype(np.float64))
    pr["W1"] = bf16_round(pr["W1"]); pr["W2"] = bf16_round(pr["W2"])
    Mo, fell = PO.preconditioner(pr, rp, cols, vals, ent, held)
    assert fb == int(fell.sum())
    scale = np.abs(Mo).max(axis=(1, 2), keepdims=True)
    assert (np.abs(M - Mo) / scale).max() <= 1e-4


def test_trained_correction_gain_on_held_out_scene(B):
    """What the shipped network (trained by precond_train.py, its strength alpha chosen on held-out scenes)
    gains over plain block-Jacobi: PCG iterations on the same reduced systems of a scene outside both sets.
    The learned form must reach the same stopping tolerance; with alpha = 0 it is block-Jacobi exactly, so
    it can take no more iterations.  The unshrunk network (alpha = 1) is reported alongside."""
    import json
    import os
    from paper_2609_04026_b300 import precond_train as PT
    wdir = os.path.join(os.path.dirname(B.__file__), "weights")
    prm = np.load(os.path.join(wdir, "precond_mlp.npy"))
    meta = json.load(open(os.path.join(wdir, "precond_mlp.json")))
    s = make_scene(config("small", seed=77))
    cnt = (len(s["cams"]["q"]), len(s["planes"]), len(s["vps"]), len(s["points"]), len(s["lines"]))
    p = gpu_problem(B, s, precision=B.BA_MIXED, precond=B.BA_PRECOND_LEARNED)
    its = {"jacobi": 0, "learned": 0}
    try:
        for _ in range(4):
            lam, _nu = B.ba_get_lm_state(p)
            B.ba_build_reduced(p, lam)
            oj = B.ba_compute_step(p, cnt)                  # weights not set yet on the first pass: block-Jacobi
            B.ba_precond_set_weights(p, prm)
            ol = B.ba_compute_step(p, cnt)
            B.ba_precond_set_weights(p, PT.shrink(prm, 0.0))
            its["jacobi"] += oj["pcg_iters"]
            its["learned"] += ol["pcg_iters"]
            assert ol["pcg_rel"] <= 1e-6 and oj["pcg_rel"] <= 1e-6
            B.ba_lm_step(p)
    finally:
        B.ba_destroy(p)
    print("held-out PCG iterations", its, "alpha", meta["alpha"], "validation", meta["validation_pcg_iters"])
    if meta["alpha"] == 0.0:
        assert its["learned"] == its["jacobi"]
