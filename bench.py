#!/usr/bin/env python
"""Benchmark of the holistic-BA LM step on one B300 (per process; N processes = N independent replicas).

A "step" is one Levenberg-Marquardt iteration of the library: linearise every residual, damp and invert the
landmark blocks, accumulate the Schur complement over cameras and groups, solve it by block-Jacobi PCG,
back-substitute, evaluate the FP64 cost of the candidate and accept or reject.  The one-time structure
build (the analogue of a sparse solver's symbolic analysis) runs before the timed region and is reported
separately.

Workload (default "large"): 2000 cameras, 2M points, 200k lines, 300 planes and 200 VPs, about 20.5M
residuals, mixed precision (FP32 Jacobians / Schur / S storage, FP64 landmark inverses, PCG vectors, cost
and accept test).  Inputs are synthetic and seeded (scenegen), shaped like the paper's synthetic benchmark.

Printed JSON (rank 0, one line): value = LM iterations per second of device time over K timed steps (max
over ranks; N ranks = N replicas, so the value is the sum of their iterations over the slowest rank's time);
e2e = the same metric through the public API with host buffers (problem creation, host->device copies,
structure build, the solve to convergence and the read-back of the parameters inside the timed region);
roofline of the dominant kernel; cpu_baseline = the FP64 oracle on a bounded sample of the same scene.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config large]
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LM iter/s & time-to-converge (cost rel 1e-6) at 2k cams; PCG iters vs Jacobi"
UNIT = "LM iter/s"


# ------------------------------------------------------------------------------------------ helpers
def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi samples of SM clock / power / throttle reasons while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.idx)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def scene_counts(s):
    return {k: int(len(v["feat"])) for k, v in s["obs"].items()}


def workload_desc(s, name):
    c = scene_counts(s)
    return (f"{name}: {len(s['cams']['q'])} cams, {len(s['points'])} points, {len(s['lines'])} lines, "
            f"{len(s['planes'])} planes + {len(s['vps'])} VPs, {sum(c.values())} residuals "
            f"({c['point']} point, {c['line']} line, {c['plane_point']}+{c['plane_line']} plane-induced, "
            f"{c['vp']} VP, {c['p2l'] + c['l2p']} wireframe)")


# per-unit algorithmic FP32 flops of the linearisation (residual + Jacobian + IRLS-weighted accumulation of
# V_f, g_f and the per-slot blocks), counted from the formulas of each residual kind
LIN_FLOPS = {"point": 354, "line": 1100, "plane_point": 660, "plane_line": 2700, "vp": 280, "p2l": 210, "l2p": 440}
# kinds the benchmark scene does not carry (the direct 3D plane distances; sphere ... cuboid points) have no
# flop count here: the linearisation's ALU roofline covers the seven kinds of the benchmark


def s_type_counts(rp, cols, nc, npl):
    """Blocks of the reduced system by storage type: camera-camera (both triangles), camera-plane and
    camera-VP (upper triangle only), group-group (both triangles), and the camera-camera upper triangle."""
    na = len(rp) - 1
    r = np.repeat(np.arange(na), np.diff(rp))
    c = cols.astype(np.int64)
    cam_r = r < nc
    return {"cc": int((cam_r & (c < nc)).sum()), "cp": int((cam_r & (c >= nc) & (c < nc + npl)).sum()),
            "cv": int((cam_r & (c >= nc + npl)).sum()), "gg": int((~cam_r & (c >= nc)).sum()),
            "cc_upper": int((cam_r & (c < nc) & (c >= r)).sum()), "gg_upper": int((~cam_r & (c >= r)).sum())}


# measured DRAM traffic of one PCG iteration of the typed kernel on the 2000-camera workload, mixed path
PCG_DRAM_BYTES_PER_ITER_LARGE = (8.44e9 + 9.38e6) / 121


def pcg_bytes_per_iter(t, T, na):
    """Algorithmic bytes of one PCG iteration on the typed storage: every stored block's values at its real
    width (camera-camera 36, camera-plane 18, camera-VP 12, group-group 36) and its 4-byte column index, and
    the FP64 vectors (~10 reads or writes of 6 doubles per block row).  The symmetric minimum stores the
    camera-camera and group-group blocks once (upper triangle)."""
    vec = na * 6 * 8 * 10
    stored = T * (36 * t["cc"] + 18 * t["cp"] + 12 * t["cv"] + 36 * t["gg"]) + 4 * (t["cc"] + t["cp"] + t["cv"] + t["gg"])
    sym = T * (36 * t["cc_upper"] + 18 * t["cp"] + 12 * t["cv"] + 36 * t["gg_upper"]) + \
        4 * (t["cc_upper"] + t["cp"] + t["cv"] + t["gg_upper"])
    return stored + vec, sym + vec


def roofline_models(n, dims):
    """Algorithmic work per launch of each stage.  n = residual counts per kind; dims from the library."""
    pairs_pt, pairs_ln = dims["pairs_point"], dims["pairs_line"]
    return {
        "linearize": ("alu", sum(LIN_FLOPS[k] * v for k, v in n.items() if k in LIN_FLOPS), "TFLOP/s"),
        # S_ab -= Z_a^T Z_b: 36 k FMA per slot pair (k = 3 point, 4 line)
        "schur_items": ("alu", 2 * 36 * (3 * pairs_pt + 4 * pairs_ln), "TFLOP/s"),
        # PCG: every iteration streams the stored blocks of S and touches the FP64 vectors
        "pcg": ("hbm", dims["pcg_iters_mean"] * dims["pcg_bytes_iter"], "GB/s"),
    }


# ------------------------------------------------------------------------------------------ oracle baseline
def subsample(scene, frac):
    """The scene restricted to the first `frac` of its points and lines (all cameras and groups)."""
    import copy
    s = copy.copy(scene)
    npk = max(1, int(len(scene["points"]) * frac))
    nlk = max(1, int(len(scene["lines"]) * frac))
    obs = {}
    for k, o in scene["obs"].items():
        is_pt = k in ("point", "plane_point", "p2l")
        keep = o["feat"] < (npk if is_pt else nlk)
        obs[k] = {kk: vv[keep] for kk, vv in o.items()}
    s["obs"] = obs
    s["points"] = scene["points"][:npk]
    s["lines"] = scene["lines"][:nlk]
    return s


def oracle_step_time(scene, frac):
    """Seconds of one oracle LM iteration on the sub-sample, and the fraction of residuals it covers."""
    import torch
    from oracle import ba_oracle as O
    sub = subsample(scene, frac)
    n_all = sum(scene_counts(scene).values())
    n_sub = sum(scene_counts(sub).values())
    st = O.state_from_scene(sub)
    lay = O.Layout(st, sub["fixed"])
    opt = O.Options()
    lm = O.LMState(opt.lambda0)
    t = time.perf_counter()
    O.lm_step(st, sub["obs"], opt, lm, lay)
    dt = time.perf_counter() - t
    return dt, n_sub / n_all, torch.get_num_threads()


# ------------------------------------------------------------------------------------------ main
def replica_rate(ms_local, steps, world, dist, device):
    """N independent replicas (one problem per rank, no data-path collective): the slowest rank's time of its
    timed steps (a MAX all-reduce over the ranks) and the whole job's LM iterations per second, every rank's
    steps divided by that time."""
    import torch
    ms = float(ms_local)
    if dist is not None and world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * steps / (ms / 1e3)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="large")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--cpu-frac", type=float, default=0.04)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--max-iters", type=int, default=200, help="LM cap of the end-to-end solve")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-window workload")
    ap.add_argument("--windows", type=int, default=256)
    ap.add_argument("--no-fp64-ttc", action="store_true", help="skip the FP64 block-Jacobi time-to-converge")
    ap.add_argument("--no-mixed-error", action="store_true", help="skip the per-result mixed-vs-FP64 error")
    ap.add_argument("--no-intr", action="store_true", help="skip the refined-intrinsics (cam_dof 9) workload")
    ap.add_argument("--no-group3d", action="store_true", help="skip the direct-3D group-distance workload")
    ap.add_argument("--no-surfaces", action="store_true", help="skip the sphere / cylinder / cone workload")
    ap.add_argument("--no-wire3d", action="store_true", help="skip the 3D wireframe-distance workload")
    ap.add_argument("--intr-models", type=int, default=20,
                    help="camera models sharing refined intrinsics in that workload (0 = one per camera)")
    args = ap.parse_args()
    assert args.warmup >= 3, "at least 3 warm-up steps"

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    from scenegen import config as scfg, make_scene

    if args.impl == "reference":
        if rank != 0:
            return 0
        return run_reference(args, scfg, make_scene)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2609_04026_b300 as B

    scene = make_scene(scfg(args.config, seed=scfg(args.config).seed + rank))
    counts = scene_counts(scene)
    prec = B.BA_MIXED if args.precision == "mixed" else B.BA_FP64
    stream = torch.cuda.Stream()
    opts = B.ba_default_options(precision=prec, cuda_stream=stream.cuda_stream)
    p = B.ba_create(opts)
    B.load_scene(p, scene)
    t0 = time.perf_counter()
    reps = [B.ba_lm_step(p)]                        # first step freezes the structure (built once)
    first_step_s = time.perf_counter() - t0
    for _ in range(args.warmup - 1):
        reps.append(B.ba_lm_step(p))

    smi = ClockSampler(local if "CUDA_VISIBLE_DEVICES" not in os.environ else
                       os.environ["CUDA_VISIBLE_DEVICES"].split(",")[local])
    smi.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    timed = [B.ba_lm_step(p) for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = smi.stop()
    ms, value = replica_rate(ev0.elapsed_time(ev1), args.steps, world, dist, "cuda")
    na, nbf = B.ba_reduced_size(p)
    B.ba_build_reduced(p, float(B.ba_get_lm_state(p)[0]))
    rp_, cols_, _, _ = B.ba_export_reduced_system(p, values=False)
    B.ba_destroy(p)
    tcounts = s_type_counts(rp_, cols_, len(scene["cams"]["q"]), len(scene["planes"]))
    peak32 = B.ba_measure_fma_rate(B.BA_MIXED, stream.cuda_stream)
    peak64 = B.ba_measure_fma_rate(B.BA_FP64, stream.cuda_stream)

    kern = {k: float(np.mean([r.as_dict()["ms_kernel"][k] for r in timed])) for k in timed[0].KERNELS}
    launches = int(sum(r.n_launches for r in timed))
    pcg_iters = [r.pcg_iters for r in timed]
    pcg_rel = [float("%.3g" % r.pcg_rel) for r in timed]
    dims_S = {"block_rows": na, "stored_blocks": nbf, "block_density": round(nbf / max(na * na, 1), 4)}

    # ---------------- roofline of the dominant kernel stage (live CUDA-event times of the timed steps)
    dims = pair_counts(scene)
    dims.update(dims_S)
    dims["pcg_iters_mean"] = float(np.mean(pcg_iters))
    dims["Tbytes"] = 4 if prec == B.BA_MIXED else 8
    dims["pcg_bytes_iter"], sym_iter = pcg_bytes_per_iter(tcounts, dims["Tbytes"], na)
    dims_S["blocks_by_type"] = tcounts
    models = roofline_models(counts, dims)
    pk = measured_peaks()
    hbm_peak = pk["hbm_gbs"] if pk else 6400.0
    hbm_src = "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if pk else "fallback 6.4 TB/s"
    alu_peak = peak32 if prec == B.BA_MIXED else peak64
    alu_src = ("measured FP32 FMA rate of this GPU (ba_measure_fma_rate)" if prec == B.BA_MIXED else
               "measured FP64 FMA rate of this GPU (ba_measure_fma_rate)")

    def stage_roof(stage):
        bound, work, unit = models[stage]
        if bound == "hbm":
            achieved, peak, src = work / (kern[stage] / 1e3) / 1e9, hbm_peak, hbm_src
        else:
            achieved, peak, src = work / (kern[stage] / 1e3) / 1e12, alu_peak, alu_src
        return {"bound": bound, "kernel": stage, "achieved": round(achieved, 3), "peak": round(peak, 2), "unit": unit,
                "frac": round(achieved / peak, 4), "peak_source": src}

    stages = {k: stage_roof(k) for k in models if kern.get(k, 0) > 0}
    stages["pcg"]["work"] = ("algorithmic bytes per launch: PCG iterations x (typed storage of S: camera-camera blocks "
                             "36 values (both triangles), camera-plane 18, camera-VP 12, group-group 36, each with a "
                             "4-byte column index; + block rows x 6 x 8 bytes x 10 vector accesses)")
    stages["pcg"]["frac_of_symmetric_minimum"] = round(
        dims["pcg_iters_mean"] * sym_iter / (kern["pcg"] / 1e3) / 1e9 / hbm_peak, 4)
    # DRAM bytes of the PCG kernel from one ncu capture of the 2000-camera workload (profiles/pcg_dram_large.md:
    # 8.45 GB read + written by a 121-iteration launch), per iteration times this run's mean iterations; only
    # for that workload and precision
    if args.config == "large" and prec == B.BA_MIXED:
        stages["pcg"]["traffic"] = round(PCG_DRAM_BYTES_PER_ITER_LARGE * dims["pcg_iters_mean"])
        stages["pcg"]["traffic_note"] = ("dram__bytes_read.sum + dram__bytes_write.sum per launch, from one ncu "
                                         "capture (8.45 GB over 121 iterations) scaled by the mean iterations; below "
                                         "the algorithmic bytes because ~60 MB of S stays in L2 between iterations")
    else:
        stages["pcg"]["traffic"] = None
    # the dominant kernel: the linearise stage's events span two kernels (points, lines) and, in the timed steps,
    # the candidate's linearisation that shares the SMs with the FP64 cost pass on a second stream, so its time
    # is not one kernel's; the other stages are single kernels (the launch list agrees: k_pcg_typed is the
    # largest share)
    dom = max((k for k in kern if k != "linearize"), key=kern.get)
    roof = dict(stages[dom]) if dom in stages else {
        "bound": None, "kernel": dom, "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None,
        "note": "no algorithmic model for this stage"}
    roof.setdefault("traffic", None)
    roof["dominant"] = ("the largest single-kernel stage by CUDA-event time (the linearise stage spans two kernels "
                        "and the overlapped cost pass)")

    # ---------------- end to end through the public API (host buffers) to convergence
    e2e = None
    ttc = None
    if not args.no_e2e:
        h2d = host_bytes(scene)
        torch.cuda.synchronize()
        t = time.perf_counter()
        o2 = B.ba_default_options(precision=prec, max_lm_iters=args.max_iters, precond=B.BA_PRECOND_LEARNED)
        q = B.ba_create(o2)
        B.load_scene(q, scene)
        torch.cuda.synchronize()
        ts = time.perf_counter()
        B.ba_precond_set_weights(q, shipped_weights())      # freezes the structure: after the inputs
        structure_s = time.perf_counter() - ts
        sr = B.ba_solve(q)
        cams = B.ba_get_cameras(q, len(scene["cams"]["q"]))
        pts = B.ba_get_features(q, B.BA_POINT, len(scene["points"]))
        lns = B.ba_get_features(q, B.BA_LINE, len(scene["lines"]))
        pl = B.ba_get_groups(q, B.BA_PLANE, len(scene["planes"]))
        vp = B.ba_get_groups(q, B.BA_VP, len(scene["vps"]))
        B.ba_destroy(q)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t
        d2h = sum(a.nbytes for a in (cams, pts, lns, pl, vp))
        e2e = {"value": round(sr.iters / wall, 4), "unit": UNIT, "h2d_bytes_per_step": int(h2d / max(sr.iters, 1)),
               "d2h_bytes_per_step": int(d2h / max(sr.iters, 1)),
               "note": "one job = create, host->device inputs, structure build, ba_solve to convergence, "
                       "parameters read back; bytes per step = job bytes / iterations"}
        ttc = {"seconds_wall": round(wall, 3), "seconds_solve": round((sr.ms_total - sr.ms_structure) / 1e3, 3),
               "structure_ms": round(sr.ms_structure + 1e3 * structure_s, 1),
               "structure_note": "structure build (the freeze inside ba_precond_set_weights, timed on the host) "
                                 "plus any part of it inside ba_solve",
               "iters": sr.iters, "converged": bool(sr.converged),
               "accepted": sr.accepted_steps, "pcg_iters_total": sr.total_pcg_iters, "cost0": sr.cost0,
               "cost": sr.cost, "precision": args.precision, "precond": "learned (shipped weights)"}

    # ---------------- time to converge at equal final-cost accuracy: the mixed learned form and the plain FP64
    # block-Jacobi form, each stepped with ba_lm_step (structure built before the clock starts) until its own
    # stopping rule; the target is the lower of the two final costs plus 1e-5 relative, and a form that stopped
    # above it keeps iterating (up to --max-iters) until it reaches it
    ttc64 = None
    equal = None
    if not args.no_fp64_ttc and not args.no_e2e:
        forms = {}
        for name, pr, pc in (("mixed_learned", B.BA_MIXED, B.BA_PRECOND_LEARNED),
                             ("fp64_block_jacobi", B.BA_FP64, B.BA_PRECOND_BLOCK_JACOBI)):
            q = B.ba_create(B.ba_default_options(precision=pr, precond=pc))
            B.load_scene(q, scene)
            if pc == B.BA_PRECOND_LEARNED:
                B.ba_precond_set_weights(q, shipped_weights())
            B.ba_eval_cost(q)                                 # builds the structure
            f = {"q": q, "t": 0.0, "traj": [], "stop": None, "pcg": 0}
            while len(f["traj"]) < args.max_iters:
                t = time.perf_counter()
                r = B.ba_lm_step(q)
                f["t"] += time.perf_counter() - t
                f["pcg"] += r.pcg_iters
                f["traj"].append((f["t"], r.cost_new if r.accepted else r.cost, f["pcg"]))
                if r.converged:
                    f["stop"] = len(f["traj"])
                    break
            forms[name] = f
        target = min(f["traj"][-1][1] for f in forms.values()) * (1 + 1e-5)
        equal = {"target_cost": target, "rule": "lower final cost of the two forms + 1e-5 relative"}
        for name, f in forms.items():
            while f["traj"][-1][1] > target and len(f["traj"]) < args.max_iters:
                t = time.perf_counter()
                r = B.ba_lm_step(f["q"])
                f["t"] += time.perf_counter() - t
                f["pcg"] += r.pcg_iters
                f["traj"].append((f["t"], r.cost_new if r.accepted else r.cost, f["pcg"]))
            hit = next((k for k, row in enumerate(f["traj"]) if row[1] <= target), None)
            B.ba_destroy(f["q"])
            equal[name] = {"seconds": round(f["traj"][hit][0], 3) if hit is not None else None,
                           "lm_iters": hit + 1 if hit is not None else None,
                           "pcg_iters": f["traj"][hit][2] if hit is not None else None,
                           "stopped_at_iter": f["stop"], "final_cost_at_stop": f["traj"][(f["stop"] or 1) - 1][1]}
        if equal["mixed_learned"]["seconds"] and equal["fp64_block_jacobi"]["seconds"]:
            equal["speedup_mixed_learned_over_fp64"] = round(
                equal["fp64_block_jacobi"]["seconds"] / equal["mixed_learned"]["seconds"], 2)
        f64 = equal["fp64_block_jacobi"]
        ttc64 = {"seconds_solve": round(forms["fp64_block_jacobi"]["traj"][(f64["stopped_at_iter"] or 1) - 1][0], 3),
                 "iters": f64["stopped_at_iter"], "cost": f64["final_cost_at_stop"]}

    # ---------------- batched local windows in one persistent launch (CUDA graph), autotuned
    batched = None
    if not args.no_batch:
        from scenegen import window_config
        wins = [make_scene(window_config(i, seed=4 + 1000 * rank)) for i in range(args.windows)]
        ps = []
        for w_ in wins:
            h = B.ba_create(B.ba_default_options(precision=B.BA_MIXED))
            B.load_scene(h, w_)
            ps.append(h)
        B.ba_solve_batch(ps, lm_iters=1, autotune=True)      # freezes the windows and tunes the launch shape
        B.ba_solve_batch(ps, lm_iters=10, autotune=False)     # captures the batch's graph
        reps = B.ba_solve_batch(ps, lm_iters=10, autotune=False)   # launches the kept graph again
        shape = B.ba_batch_launch_shape(ps[0])
        nct, nbig = B.ba_batch_ctas_per_window(ps[0])
        work = [sum(int(len(o["feat"])) for o in w_["obs"].values()) + len(w_["points"]) + len(w_["lines"])
                for w_ in wins]
        big = set(np.argsort(-np.asarray(work), kind="stable")[:nbig].tolist())
        for h in ps:
            B.ba_destroy(h)
        ms_b = reps[0].ms_total
        nres = sum(sum(int(len(o["feat"])) for o in w_["obs"].values()) for w_ in wins)
        batched = {"windows": args.windows, "lm_iters_each": 10, "ms": round(ms_b, 3),
                   "window_lm_iters_per_s": round(args.windows * 10 / (ms_b / 1e3), 1),
                   "residuals_total": nres,
                   "launch_shape": {"threads": shape[0], "ctas": shape[1], "ctas_per_window": nct,
                                    "windows_on_clusters": nbig,
                                    "note": "chosen by the library's autotuner: the largest windows_on_clusters "
                                            "windows on clusters of ctas_per_window CTAs, the rest on single CTAs"},
                   "window_ms": {"max": round(max(r.ms_window for r in reps), 3),
                                 "mean": round(float(np.mean([r.ms_window for r in reps])), 3),
                                 "balanced": round(sum(r.ms_window * (nct if i in big else 1)
                                                       for i, r in enumerate(reps)) / shape[1], 3),
                                 "note": "each window's own device time on its CTAs; balanced = the sum of window x "
                                         "CTA times over the launch's CTAs, the makespan of a perfect balance"},
                   "accepted_steps": int(sum(r.accepted_steps for r in reps)),
                   "cost_decreased": int(sum(r.cost < r.cost0 for r in reps)),
                   "note": "cameras 5-40, features log-uniform 200-20k (70% points), 0-8 groups per window; "
                           "device time of the second launch of the kept graph (10 iterations each, every window "
                           "continuing from the first launch's state)"}

    # ---------------- refined intrinsics (cam_dof 9, Section 3.1 K_c(i)) at the same scale: the scene generated
    # with every camera belonging to one of --intr-models camera models (shared f, k1, k2 in the ground truth),
    # the models' initial intrinsics perturbed by 1%; LM iterations per second of the step with the intrinsics
    # entities in the reduced system, and how far the models' f moved towards the ground truth
    intr = None
    if not args.no_intr:
        si = make_scene(scfg(args.config, seed=scfg(args.config).seed + rank, intr_refine=True,
                             intr_groups=args.intr_models, intr_noise=0.01))
        q = B.ba_create(B.ba_default_options(precision=prec, cam_dof=9, cuda_stream=stream.cuda_stream))
        B.load_scene(q, si)
        for _ in range(3):
            B.ba_lm_step(q)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ti = [B.ba_lm_step(q) for _ in range(5)]
        e1.record(stream)
        torch.cuda.synchronize()
        ms_i = e0.elapsed_time(e1)
        nk = B.ba_intrinsics_count(q)
        na_i, nbf_i = B.ba_reduced_size(q)
        fk = B.ba_get_intrinsics(q, len(si["cams"]["q"]))
        B.ba_destroy(q)
        gt = si["gt"]["cams"]["intr"]
        intr = {"lm_iters_per_s": round(5 / (ms_i / 1e3), 3), "ms_per_step": round(ms_i / 5, 3),
                "intrinsics_entities": nk, "block_rows": na_i, "stored_blocks": nbf_i,
                "pcg_iters": [r.pcg_iters for r in ti],
                "kernels_ms": {k: round(float(np.mean([r.as_dict()["ms_kernel"][k] for r in ti])), 4)
                               for k in ti[0].KERNELS},
                "f_rel_error": {"initial": float(np.abs(si["cams"]["intr"][:, 0] - gt[:, 0]).max() / gt[:, 0].min()),
                                "after_8_steps": float(np.abs(fk[:, 0] - gt[:, 0]).max() / gt[:, 0].min())},
                "note": f"the {args.config} scene with {args.intr_models or 'per-camera'} camera models (seeded), "
                        "intrinsics perturbed by 1%, cam_dof 9, same precision; 5 steps timed after 3 warm-up "
                        "(the typed storage of S when the group and intrinsics values fit, else the full 6 x 6)"}
        del si

    # ---------------- the plane constraints in the direct 3D form (Section 3.2's alternative, Table 5): the same
    # scene with the group-induced residuals replaced by one point-to-plane or line-to-plane distance per feature
    # on a plane (weight 100, Table 5's best on ScanNet++); per-iteration time against the 2D form above
    g3 = None
    if not args.no_group3d:
        s3 = dict(scene)
        ob = dict(scene["obs"])
        for k2, k3 in (("plane_point", "plane_point3d"), ("plane_line", "plane_line3d")):
            f_, i_ = np.unique(ob[k2]["feat"], return_index=True)
            ob[k3] = dict(cam=np.full(len(f_), -1, np.int32), feat=f_.astype(np.int32),
                          other=ob[k2]["other"][i_].astype(np.int32), meas=np.zeros((len(f_), 0)))
            ob[k2] = {kk: vv[:0] for kk, vv in ob[k2].items()}
        s3["obs"] = ob
        q = B.ba_create(B.ba_default_options(precision=prec, w_group3d=100.0, cuda_stream=stream.cuda_stream))
        B.load_scene(q, s3)
        for _ in range(3):
            B.ba_lm_step(q)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t3 = [B.ba_lm_step(q) for _ in range(5)]
        e1.record(stream)
        torch.cuda.synchronize()
        ms3 = e0.elapsed_time(e1)
        na3, nbf3 = B.ba_reduced_size(q)
        B.ba_destroy(q)
        nres3 = sum(int(len(o["feat"])) for o in ob.values())
        g3 = {"lm_iters_per_s": round(5 / (ms3 / 1e3), 3), "ms_per_step": round(ms3 / 5, 3),
              "ms_per_step_2d_form": round(ms / args.steps, 3), "residuals": nres3, "stored_blocks": nbf3,
              "pcg_iters": [r.pcg_iters for r in t3],
              "kernels_ms": {k: round(float(np.mean([r.as_dict()["ms_kernel"][k] for r in t3])), 4)
                             for k in t3[0].KERNELS},
              "note": "the benchmark scene with its plane-induced residuals (Eq. 7, Eq. 8) replaced by the direct "
                      "3D distances, one per feature on a plane, w_group3d = 100; 5 steps timed after 3 warm-up"}
        del s3, ob

    # ---------------- spheres, cylinders, cones, ellipsoids, cuboids (Appendix B, Table 6): the medium scene (200
    # cameras) with 30 of each type, 300 points on each surface; LM iterations per second with the group-induced
    # point residuals of the five types, against the same scene without them
    srf = None
    if not args.no_surfaces:
        res_s = {}
        for label, kw in (("without", {}), ("with", dict(n_spheres=30, n_cylinders=30, n_cones=30, n_ellipsoids=30,
                                                          n_cuboids=30, surf_points=300, surf_lines=100))):
            ss = make_scene(scfg("medium", seed=scfg("medium").seed + rank, **kw))
            q = B.ba_create(B.ba_default_options(precision=prec, cuda_stream=stream.cuda_stream))
            B.load_scene(q, ss)
            E0 = B.ba_eval_cost(q)[0]
            for _ in range(3):
                B.ba_lm_step(q)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ts = [B.ba_lm_step(q) for _ in range(5)]
            e1.record(stream)
            torch.cuda.synchronize()
            ms_s = e0.elapsed_time(e1)
            na_s, nbf_s = B.ba_reduced_size(q)
            E1 = B.ba_eval_cost(q)[0]
            B.ba_destroy(q)
            res_s[label] = {"lm_iters_per_s": round(5 / (ms_s / 1e3), 3), "ms_per_step": round(ms_s / 5, 3),
                            "residuals": sum(int(len(o["feat"])) for o in ss["obs"].values()),
                            "block_rows": na_s, "stored_blocks": nbf_s, "pcg_iters": [r.pcg_iters for r in ts],
                            "cost_after_8_steps_over_initial": round(E1 / E0, 5)}
            if label == "with":
                res_s[label]["surface_residuals"] = {k: int(len(ss["obs"][k]["feat"])) for k in
                                                     ("sphere_point", "cylinder_point", "cone_point",
                                                      "ellipsoid_point", "cuboid_point", "cuboid_line")}
        srf = dict(res_s, note="the medium scene (200 cameras, 100k points, 20k lines) without and with 30 spheres, "
                               "cylinders, cones, ellipsoids and cuboids each, 300 points on each and 100 lines on "
                               "the faces of each cuboid; 5 steps timed after 3 warm-up")

    # ---------------- the wireframe constraints in the 3D form (Section 3.3 / Fig. 3b): the medium scene with its
    # projected wireframe residuals (Eq. 11, Eq. 12), with the 3D endpoint distances instead (the named points
    # become entities of the reduced system), and with both; LM iterations per second and the cost after 8 steps
    wf = None
    if not args.no_wire3d:
        res_w = {}
        for form in ("2d", "3d", "both"):
            sw = make_scene(scfg("medium", seed=scfg("medium").seed + rank, wire_form=form))
            q = B.ba_create(B.ba_default_options(precision=prec, cuda_stream=stream.cuda_stream))
            B.load_scene(q, sw)
            E0 = B.ba_eval_cost(q)[0]
            for _ in range(3):
                B.ba_lm_step(q)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            tw = [B.ba_lm_step(q) for _ in range(5)]
            e1.record(stream)
            torch.cuda.synchronize()
            ms_w = e0.elapsed_time(e1)
            na_w, nbf_w = B.ba_reduced_size(q)
            E1 = B.ba_eval_cost(q)[0]
            B.ba_destroy(q)
            res_w[form] = {"lm_iters_per_s": round(5 / (ms_w / 1e3), 3), "ms_per_step": round(ms_w / 5, 3),
                           "wireframe_residuals": {k: int(len(sw["obs"][k]["feat"])) for k in ("p2l", "l2p", "wf3d")},
                           "block_rows": na_w, "stored_blocks": nbf_w, "pcg_iters": [r.pcg_iters for r in tw],
                           "cost_after_8_steps_over_initial": round(E1 / E0, 5)}
        wf = dict(res_w, note="the medium scene (200 cameras, 100k points, 20k lines) with the projected wireframe "
                              "residuals (2d), the 3D endpoint distances (3d: every named point an entity of the "
                              "reduced system) or both; 5 steps timed after 3 warm-up")

    # ---------------- the mixed path's error per result against the FP64 path, one step from the seeded start
    # at the initial damping (the FP64 path itself is checked against the oracle at 2000 cameras by
    # tests/test_gpu_scale.py)
    mixed_err = None
    if prec == B.BA_MIXED and not args.no_mixed_error:
        res = {}
        for name, pr in (("fp64", B.BA_FP64), ("mixed", B.BA_MIXED)):
            q = B.ba_create(B.ba_default_options(precision=pr))
            B.load_scene(q, scene)
            E0, _ = B.ba_eval_cost(q)
            B.ba_build_reduced(q, 1e-4)
            _, _, vals, bvec = B.ba_export_reduced_system(q)
            out = B.ba_compute_step(q, (len(scene["cams"]["q"]), len(scene["planes"]), len(scene["vps"]),
                                        len(scene["points"]), len(scene["lines"])))
            st1 = B.ba_lm_step(q)
            B.ba_destroy(q)
            res[name] = (E0, vals, bvec, out, st1)
        (E64, S64, b64, o64, s64), (E32, S32, b32, o32, s32) = res["fp64"], res["mixed"]
        rel_ = lambda a, b: float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
        d64 = np.concatenate([o64[k].ravel() for k in ("cam", "plane", "vp", "point", "line")])
        d32 = np.concatenate([o32[k].ravel() for k in ("cam", "plane", "vp", "point", "line")])
        mixed_err = {"S": rel_(S32, S64), "b": rel_(b32, b64), "delta": rel_(d32, d64),
                     "pred": abs(o32["pred"] - o64["pred"]) / abs(o64["pred"]), "cost": abs(E32 - E64) / E64,
                     "cost_new": abs(s32.cost_new - s64.cost_new) / s64.cost_new,
                     "pcg_iters": {"fp64": o64["pcg_iters"], "mixed": o32["pcg_iters"]},
                     "note": "max-norm relative error of the mixed path against the FP64 path, one LM step from "
                             "the seeded start at damping 1e-4, on the benchmark scene"}
        del res, S64, S32

    learned = None
    try:
        meta = json.load(open(os.path.join(ROOT, "paper_2609_04026_b300", "weights", "precond_mlp.json")))
        learned = {"alpha": meta["alpha"], "validation_pcg_iters_by_alpha": meta["validation_pcg_iters"],
                   "training_systems": meta["systems"], "training_blocks": meta["samples"],
                   "note": "alpha = 0 (chosen on held-out systems) makes the learned form plain block-Jacobi"}
    except Exception:
        pass

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        dt, frac, cores = oracle_step_time(scene, args.cpu_frac)
        cpu = {"value": round(frac / dt, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"one FP64 oracle LM iteration on the first {args.cpu_frac:.0%} of the points and lines "
                         f"(all cameras and groups; {frac:.2%} of the residuals) took {dt:.1f} s; "
                         f"scaled to the full scene by residual count"}

    if rank == 0:
        out = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None,
               "dtype": "f32+f64" if prec == B.BA_MIXED else "f64",
               "data": "synthetic, seeded (scenegen): cube scene with Manhattan planes, VPs, wireframes, pixel "
                       "noise and outliers, shaped like the paper's synthetic benchmark (App. A.3)",
               "config": {"workload": workload_desc(scene, args.config), "precision": args.precision,
                          "l2": "inputs larger than L2 (GB-scale working set per step)",
                          "parallelism": "replicas" if world > 1 else "single GPU"},
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": launches,
               "time_to_converge": ttc, "time_to_converge_fp64_block_jacobi": ttc64,
               "time_to_equal_cost": equal,
               "batched_windows": batched, "refined_intrinsics": intr, "group_form_3d": g3, "surface_groups": srf,
               "wireframe_3d": wf, "learned_precond": learned,
               "kernels_ms": {k: round(v, 4) for k, v in kern.items()},
               "stage_rooflines": stages, "measured_fma_tflops": {"fp32": round(peak32, 2), "fp64": round(peak64, 3)},
               "mixed_error": mixed_err,
               "pcg_iters": pcg_iters, "pcg_rel": pcg_rel, "reduced_system": dims_S,
               "first_step_s": round(first_step_s, 3)}
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def shipped_weights():
    return np.load(os.path.join(ROOT, "paper_2609_04026_b300", "weights", "precond_mlp.npy"))


def host_bytes(s):
    n = sum(a.nbytes for a in (s["cams"]["q"], s["cams"]["t"], s["cams"]["intr"], s["cams"]["pp"], s["points"],
                                s["lines"], s["planes"], s["vps"], s["fixed"]))
    for o in s["obs"].values():
        n += sum(np.asarray(v).nbytes for v in o.values())
    return int(n)


def pair_counts(s):
    """Schur slot pairs sum_f n_f (n_f + 1) / 2 split by feature type (n_f = kept entities of feature f)."""
    out = {}
    for ft, kinds in (("point", ("point", "plane_point", "p2l")), ("line", ("line", "plane_line", "vp", "l2p"))):
        nfeat = len(s["points"] if ft == "point" else s["lines"])
        fixed = s["fixed"]
        keys = []
        for k in kinds:
            o = s["obs"][k]
            if len(o["feat"]) == 0:
                continue
            if k != "vp":
                c = o["cam"].astype(np.int64)
                ok = fixed[c] != 0x3F
                keys.append(o["feat"][ok].astype(np.int64) * 1_000_000 + c[ok])
            if k in ("plane_point", "plane_line"):
                keys.append(o["feat"].astype(np.int64) * 1_000_000 + 500_000 + o["other"])
            if k == "vp":
                keys.append(o["feat"].astype(np.int64) * 1_000_000 + 900_000 + o["other"])
        u = np.unique(np.concatenate(keys)) if keys else np.zeros(0, np.int64)
        nf = np.bincount((u // 1_000_000).astype(np.int64), minlength=nfeat)
        out["pairs_" + ft] = int((nf * (nf + 1) // 2).sum())
    return out


def run_reference(args, scfg, make_scene):
    """The oracle (FP64 CPU, as it stands) timed per LM step on a bounded sample of the same workload."""
    scene = make_scene(scfg(args.config))
    times = []
    frac = args.cpu_frac
    for _ in range(args.warmup):
        pass                                          # the oracle has no warm state; warm-up is a no-op
    cores = None
    fr = None
    for _ in range(args.steps):
        dt, fr, cores = oracle_step_time(scene, frac)
        times.append(dt)
    t = float(np.mean(times))
    value = fr / t
    sample = (f"each step: one FP64 oracle LM iteration on the first {frac:.0%} of the points and lines "
              f"({fr:.2%} of the residuals), scaled to the full scene by residual count")
    out = {"metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(t / fr * 1e3, 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "impl": "reference",
           "data": "synthetic, seeded (scenegen)",
           "config": {"workload": workload_desc(scene, args.config), "precision": "fp64",
                      "parallelism": "host cores"},
           "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
