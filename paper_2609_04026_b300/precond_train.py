"""Train the learned block-Jacobi correction on reduced systems the solver itself produces.

Data: seeded scene variants (the 200-camera workload with different seeds); for each, the reduced system S is
built at successive LM iterates and logged with the library's own features.  Targets are the Jacobi-scaled
diagonal blocks of the exact inverse of S, computed on the host from the exported system (a dense inverse of
the 6 n x 6 n padded matrix).  Training runs on the GPU in the library's own kernels (FP32 forward / backward,
Adam); the result is the float parameter vector that ba_precond_set_weights takes.  The correction's output is
finally scaled by the alpha in {0, 0.1, 0.25, 0.5, 1} with the fewest PCG iterations on held-out scenes
(alpha = 0 is plain block-Jacobi).

  python -m paper_2609_04026_b300.precond_train --scenes 24 --iters 6 --out weights.npy
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

NF, NH, NO = 32, 128, 21
IU, JU = np.triu_indices(6)


def log_systems(B, scene, iters, precision):
    """(X, E, mask) samples of `iters` reduced systems along the LM path of one scene."""
    o = B.ba_default_options(precision=precision)
    p = B.ba_create(o)
    Xs, Es, Ms = [], [], []
    try:
        B.load_scene(p, scene)
        for _ in range(iters):
            lam, _nu = B.ba_get_lm_state(p)
            B.ba_build_reduced(p, lam)
            rp, cols, vals, _b = B.ba_export_reduced_system(p)
            na = len(rp) - 1
            X, mask = B.ba_precond_features(p, na)
            S = np.zeros((6 * na, 6 * na))
            diag = np.zeros((na, 6))
            for a in range(na):
                for q in range(rp[a], rp[a + 1]):
                    c = cols[q]
                    S[6 * a:6 * a + 6, 6 * c:6 * c + 6] = vals[q]
                    if c == a:
                        diag[a] = np.diag(vals[q])
            Si = np.linalg.inv(S)
            E = np.zeros((na, NO))
            keep = (diag > 0).all(1)
            for a in np.nonzero(keep)[0]:
                sl = slice(6 * a, 6 * a + 6)
                s = np.sqrt(diag[a])
                T = s[:, None] * Si[sl, sl] * s[None, :]
                Shat = S[sl, sl] / s[:, None] / s[None, :]
                E[a] = (T - np.linalg.inv(Shat))[IU, JU]
            # blocks whose float diagonal lost its sign, or whose values are not finite, are not samples
            keep &= np.isfinite(E).all(1) & np.isfinite(X).all(1)
            Xs.append(X[keep]); Es.append(E[keep].astype(np.float32)); Ms.append(mask[keep])
            log_systems.dropped += int((~keep).sum())
            B.ba_lm_step(p)
    finally:
        B.ba_destroy(p)
    return np.concatenate(Xs), np.concatenate(Es), np.concatenate(Ms)


log_systems.dropped = 0


def init_params(X, seed):
    rng = np.random.default_rng(seed)
    mu = X.mean(0)
    sg = X.std(0) + 1e-3
    W1 = rng.normal(0, np.sqrt(2.0 / NF), (NF, NH))
    W2 = rng.normal(0, 1e-3, (NH, NO))
    return np.concatenate([mu, sg, W1.ravel(), np.zeros(NH), W2.ravel(), np.zeros(NO)]).astype(np.float32)


def train(B, X, E, mask, steps=4000, batch=1024, lr=1e-3, seed=0, log_every=500):
    """Train on the GPU; returns (params float32 numpy, list of (step, loss))."""
    import torch
    dev = torch.device("cuda")
    perm = np.random.default_rng(seed).permutation(len(X))
    Xd = torch.from_numpy(np.ascontiguousarray(X[perm])).to(dev)
    Ed = torch.from_numpy(np.ascontiguousarray(E[perm])).to(dev)
    Md = torch.from_numpy(np.ascontiguousarray(mask[perm])).to(dev)
    prm = torch.from_numpy(init_params(X, seed)).to(dev)
    m = torch.zeros(prm.numel() - 2 * NF, dtype=torch.float32, device=dev)
    v = torch.zeros_like(m)
    hist = []
    t = 0
    while t < steps:
        k = min(log_every, steps - t)
        loss = B.ba_precond_train(Xd, Ed, Md, prm, m, v, t, k, batch, lr)
        t += k
        hist.append((t, loss))
    return prm.cpu().numpy(), hist


def shrink(params, alpha):
    """Scale the network's output (W2, b2) by alpha: alpha = 0 gives plain block-Jacobi exactly."""
    q = params.copy()
    o = 2 * NF + NF * NH + NH
    q[o:] *= alpha
    return q


def validate(B, params, scenes, iters, alphas, precision):
    """PCG iterations on the reduced systems of held-out scenes (same systems for every alpha)."""
    tot = {a: 0 for a in alphas}
    for scene in scenes:
        o = B.ba_default_options(precision=precision, precond=B.BA_PRECOND_LEARNED)
        p = B.ba_create(o)
        try:
            B.load_scene(p, scene)
            cnt = (len(scene["cams"]["q"]), len(scene["planes"]), len(scene["vps"]), len(scene["points"]),
                   len(scene["lines"]))
            for _ in range(iters):
                lam, _nu = B.ba_get_lm_state(p)
                B.ba_build_reduced(p, lam)
                for a in alphas:
                    B.ba_precond_set_weights(p, shrink(params, a))
                    tot[a] += B.ba_compute_step(p, cnt)["pcg_iters"]
                B.ba_lm_step(p)
        finally:
            B.ba_destroy(p)
    return tot


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--scenes", type=int, default=24)
    ap.add_argument("--iters", type=int, default=6)
    ap.add_argument("--seed0", type=int, default=10000)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--val-scenes", type=int, default=3)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights",
                                                  "precond_mlp.npy"))
    args = ap.parse_args()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import paper_2609_04026_b300 as B
    from scenegen import config, make_scene
    t0 = time.time()
    parts = [log_systems(B, make_scene(config("medium", seed=args.seed0 + i)), args.iters, B.BA_MIXED)
             for i in range(args.scenes)]
    X = np.concatenate([q[0] for q in parts]); E = np.concatenate([q[1] for q in parts])
    M = np.concatenate([q[2] for q in parts])
    print(f"logged {args.scenes * args.iters} systems, {len(X)} blocks ({log_systems.dropped} dropped) in "
          f"{time.time() - t0:.1f}s", flush=True)
    prm, hist = train(B, X, E, M, steps=args.steps)
    for s, l in hist:
        print(f"step {s}: loss {l:.6g}", flush=True)
    # deployment strength of the correction, chosen on held-out systems by the PCG iteration count
    alphas = (0.0, 0.1, 0.25, 0.5, 1.0)
    val = validate(B, prm, [make_scene(config("medium", seed=args.seed0 + 500 + i)) for i in range(args.val_scenes)],
                   args.iters, alphas, B.BA_MIXED)
    best = min(alphas, key=lambda a: (val[a], a))
    print("validation PCG iterations per alpha:", val, "-> alpha", best, flush=True)
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    np.save(args.out, shrink(prm, best))
    import json
    json.dump({"samples": int(len(X)), "dropped": log_systems.dropped, "systems": args.scenes * args.iters,
               "loss": hist, "alpha": best,
               "validation_pcg_iters": {str(k): int(v) for k, v in val.items()}},
              open(os.path.splitext(args.out)[0] + ".json", "w"), indent=1)
    print("saved", args.out)


if __name__ == "__main__":
    main()
