"""Python binding of libba, the B300 library for one LM step of holistic bundle adjustment.

The binding only marshals arguments: every step of the solve runs in the CUDA
kernels of libba.so (built in-tree by ``paper_2609_04026_b300.build``).  The first
call into the library raises ImportError when libba.so is missing; there is no CPU
fallback.

Functions keep the C names (``ba_create``, ``ba_add_cameras``, ... ``ba_lm_step``,
``ba_solve``).  Arrays may be numpy arrays (host memory) or CUDA torch tensors
(device memory); the binding passes BA_MEM_HOST or BA_MEM_DEVICE accordingly.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libba.so")

BA_OK, BA_ERR_ARG, BA_ERR_STATE, BA_ERR_CUDA, BA_ERR_OOM, BA_ERR_NUMERIC, BA_ERR_TIMEOUT = 0, -1, -2, -3, -4, -5, -6
BA_MEM_HOST, BA_MEM_DEVICE = 0, 1
BA_FP64, BA_MIXED = 0, 1
BA_PRECOND_BLOCK_JACOBI, BA_PRECOND_LEARNED = 0, 1
BA_POINT, BA_LINE = 0, 1
BA_PLANE, BA_VP, BA_SPHERE, BA_CYLINDER, BA_CONE, BA_ELLIPSOID, BA_CUBOID = 0, 1, 2, 3, 4, 5, 6
BA_REL_ORTHOGONAL, BA_REL_PARALLEL = 0, 1
OBS_KINDS = {"point": 0, "line": 1, "plane_point": 2, "plane_line": 3, "vp": 4, "p2l": 5, "l2p": 6,
             "plane_point3d": 7, "plane_line3d": 8, "sphere_point": 9, "cylinder_point": 10, "cone_point": 11,
             "ellipsoid_point": 12, "cuboid_point": 13, "wf3d": 14, "cuboid_line": 15}
MEAS_DIM = {0: 2, 1: 4, 2: 0, 3: 4, 4: 0, 5: 4, 6: 2, 7: 0, 8: 0, 9: 0, 10: 0, 11: 0, 12: 0, 13: 0, 14: 0, 15: 4}
NO_CAM = (4, 7, 8, 14)   # kinds without a camera (the VP term, the direct 3D plane and wireframe distances)

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class ba_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("w_point", C.c_double), ("w_line", C.c_double),
                ("w_group", C.c_double), ("w_wire", C.c_double), ("w_vp", C.c_double),
                ("cauchy_px", C.c_double), ("cauchy_vp", C.c_double), ("lambda0", C.c_double),
                ("lambda_min", C.c_double), ("lambda_max", C.c_double), ("min_gain", C.c_double),
                ("rel_cost_tol", C.c_double), ("max_lm_iters", C.c_int), ("pcg_rel_tol", C.c_double),
                ("pcg_max_iters", C.c_int), ("precond", C.c_int), ("cuda_stream", C.c_void_p),
                ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN), ("alloc_ctx", C.c_void_p),
                ("wait_budget_cycles", C.c_longlong), ("mixed_lambda_floor", C.c_double),
                ("w_rel", C.c_double), ("cauchy_rel", C.c_double), ("batch_ctas_per_window", C.c_int),
                ("w_group3d", C.c_double), ("cauchy_3d", C.c_double), ("cam_dof", C.c_int),
                ("w_wire3d", C.c_double)]


class ba_step_report(C.Structure):
    _fields_ = [("cost", C.c_double), ("cost_px", C.c_double), ("cost_new", C.c_double),
                ("cost_px_new", C.c_double), ("pred", C.c_double), ("gain", C.c_double),
                ("lambda_", C.c_double), ("pcg_rel", C.c_double), ("pcg_iters", C.c_int),
                ("accepted", C.c_int), ("converged", C.c_int), ("relinearized", C.c_int),
                ("ms_linearize", C.c_float), ("ms_schur", C.c_float), ("ms_pcg", C.c_float),
                ("ms_update", C.c_float), ("ms_kernel", C.c_float * 10), ("n_launches", C.c_int),
                ("precond_fallbacks", C.c_int)]

    KERNELS = ("linearize", "invert", "schur_items", "schur_blocks", "precond", "pcg", "backsub",
               "candidate", "cost", "decide")

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "ms_kernel"}
        d["ms_kernel"] = dict(zip(self.KERNELS, list(self.ms_kernel)))
        return d


class ba_solve_report(C.Structure):
    _fields_ = [("iters", C.c_int), ("converged", C.c_int), ("accepted_steps", C.c_int),
                ("total_pcg_iters", C.c_int), ("cost0", C.c_double), ("cost", C.c_double),
                ("cost_px", C.c_double), ("ms_structure", C.c_double), ("ms_total", C.c_double),
                ("ms_window", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libba.so not built at {LIB_PATH}: run python -m paper_2609_04026_b300.build")
    lib = C.CDLL(LIB_PATH)
    P, I64, I, D, VP = C.c_void_p, C.c_int64, C.c_int, C.c_double, C.c_void_p
    sig = {
        "ba_default_options": (None, [C.POINTER(ba_options)]),
        "ba_create": (I, [C.POINTER(ba_options), C.POINTER(C.c_void_p)]),
        "ba_destroy": (None, [P]),
        "ba_last_error": (C.c_char_p, [P]),
        "ba_add_cameras": (I, [P, I64, I, VP, VP, VP, VP]),
        "ba_add_features": (I, [P, I, I64, I, VP]),
        "ba_add_groups": (I, [P, I, I64, I, VP]),
        "ba_add_observations": (I, [P, I, I64, I, VP, VP, VP, VP]),
        "ba_add_relations": (I, [P, I64, I, VP, VP, VP, VP, VP]),
        "ba_set_intrinsics": (I, [P, I64, I, VP, VP, I64]),
        "ba_get_intrinsics": (I, [P, I, VP]),
        "ba_get_step_intrinsics": (I, [P, VP]),
        "ba_intrinsics_count": (I, [P, C.POINTER(I64)]),
        "ba_lm_step": (I, [P, C.POINTER(ba_step_report)]),
        "ba_solve": (I, [P, C.POINTER(ba_solve_report)]),
        "ba_get_cameras": (I, [P, I, VP]),
        "ba_get_features": (I, [P, I, I, VP]),
        "ba_get_groups": (I, [P, I, I, VP]),
        "ba_get_lm_state": (I, [P, VP]),
        "ba_set_lm_state": (I, [P, VP]),
        "ba_eval_cost": (I, [P, C.POINTER(D), C.POINTER(D)]),
        "ba_eval_log1p": (I, [I64, VP, VP, VP]),
        "ba_measure_fma_rate": (I, [I, C.POINTER(D), VP]),
        "ba_build_reduced": (I, [P, D]),
        "ba_reduced_size": (I, [P, C.POINTER(I64), C.POINTER(I64)]),
        "ba_export_reduced_system": (I, [P, VP, VP, VP, VP]),
        "ba_compute_step": (I, [P, VP, VP, VP, VP, VP, C.POINTER(I), C.POINTER(D), C.POINTER(D)]),
        "ba_pcg_solve_static": (I, [I64, I64, VP, VP, VP, VP, VP, D, I, VP, C.POINTER(I), C.POINTER(D),
                                    C.c_char_p, C.c_size_t]),
        "ba_solve_batch": (I, [VP, I, I, I, VP]),
        "ba_batch_launch_shape": (I, [P, C.POINTER(I), C.POINTER(I)]),
        "ba_batch_ctas_per_window": (I, [P, C.POINTER(I), C.POINTER(I)]),
        "ba_precond_param_count": (I, []),
        "ba_precond_set_weights": (I, [P, VP, I64]),
        "ba_precond_features": (I, [P, VP, VP]),
        "ba_precond_blocks": (I, [P, VP, C.POINTER(I)]),
        "ba_mlp_work_floats": (I64, [I64]),
        "ba_mlp_grad": (I, [I64, VP, VP, VP, VP, VP, C.POINTER(D), VP, VP]),
        "ba_precond_train": (I, [I64, VP, VP, VP, VP, VP, VP, I, I, I64, C.c_float, VP, C.POINTER(D), VP]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


class _Lazy:
    """libba.so, loaded (and its signatures declared) on first use; a missing library raises ImportError."""
    _h = None

    def __getattr__(self, name):
        if _Lazy._h is None:
            _Lazy._h = _load()
        return getattr(_Lazy._h, name)


_lib = _Lazy()


class BAError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libba status {status}: {msg}")
        self.status = status


def lib():
    _lib.ba_default_options   # force the load
    return _Lazy._h


def _check(p, status):
    if status != BA_OK:
        raise BAError(status, _lib.ba_last_error(p).decode() if p else "")


def _need_dev(*specs):
    """Raw device pointers cross the ABI without lengths, so the binding checks what the C side cannot.
    specs: (tensor, dtype, element count, name) tuples; each must be a contiguous tensor of that dtype and
    count (checked for all first), and all must be CUDA tensors of one device (BA_ERR_ARG otherwise)."""
    for t, dtype, numel, name in specs:
        if getattr(t, "dtype", None) != dtype:
            raise BAError(BA_ERR_ARG, f"{name}: expected dtype {dtype}, got {getattr(t, 'dtype', type(t).__name__)}")
        if t.numel() != numel:
            raise BAError(BA_ERR_ARG, f"{name}: expected {numel} elements, got {t.numel()}")
        if not t.is_contiguous():
            raise BAError(BA_ERR_ARG, f"{name}: must be contiguous")
    for t, _, _, name in specs:
        if not t.is_cuda or t.device != specs[0][0].device:
            raise BAError(BA_ERR_ARG, f"{name}: must be a CUDA tensor on the device of {specs[0][3]}")


def _arr(x, dtype):
    """(pointer, mem, keepalive) for a numpy array (host) or a CUDA torch tensor (device)."""
    if x is None:
        return None, BA_MEM_HOST, None
    if hasattr(x, "is_cuda") and x.is_cuda:
        import torch
        want = {np.float64: torch.float64, np.int32: torch.int32, np.uint8: torch.uint8}[dtype]
        t = x.to(want).contiguous()
        return C.c_void_p(t.data_ptr()), BA_MEM_DEVICE, t
    a = np.ascontiguousarray(np.asarray(x), dtype=dtype)
    return a.ctypes.data_as(C.c_void_p), BA_MEM_HOST, a


# ---------------------------------------------------------------------------- C-named wrappers
def ba_default_options(**kw):
    o = ba_options()
    _lib.ba_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class _TorchAlloc:
    """Device allocator hooks backed by torch's caching allocator on the given stream."""

    def __init__(self, stream_ptr):
        import torch
        self.torch = torch
        self.dev = torch.cuda.current_device()
        self.stream = stream_ptr

        def alloc(n, ctx):
            return self.torch.cuda.caching_allocator_alloc(int(n), self.dev, self.stream)

        def free(p, ctx):
            self.torch.cuda.caching_allocator_delete(p)
        self.alloc = ALLOC_FN(alloc)
        self.free = FREE_FN(free)


def ba_create(opts=None, torch_allocator=False):
    """Returns an opaque handle (int).  torch_allocator=True routes device allocations through
    torch's caching allocator on opts.cuda_stream."""
    opts = opts if opts is not None else ba_default_options()
    keep = None
    if torch_allocator:
        keep = _TorchAlloc(opts.cuda_stream or 0)
        opts.dev_alloc = keep.alloc
        opts.dev_free = keep.free
    h = C.c_void_p()
    st = _lib.ba_create(C.byref(opts), C.byref(h))
    if st != BA_OK:
        raise BAError(st, "ba_create failed (is a CUDA device visible?)")
    _KEEP[h.value] = (opts, keep)
    return h.value


_KEEP = {}


def ba_destroy(p):
    _lib.ba_destroy(p)
    _KEEP.pop(p, None)


def ba_last_error(p):
    return _lib.ba_last_error(p).decode()


def ba_add_cameras(p, quat_t, f_k1_k2, pp, fixed=None):
    a, mem, k1 = _arr(quat_t, np.float64)
    b, _, k2 = _arr(f_k1_k2, np.float64)
    c, _, k3 = _arr(pp, np.float64)
    d, _, k4 = _arr(fixed, np.uint8)
    n = len(k1) if k1 is not None else 0
    _check(p, _lib.ba_add_cameras(p, n, mem, a, b, c, d))


def ba_add_features(p, kind, params):
    a, mem, k = _arr(params, np.float64)
    _check(p, _lib.ba_add_features(p, kind, len(k), mem, a))


def ba_add_groups(p, kind, params):
    a, mem, k = _arr(params, np.float64)
    _check(p, _lib.ba_add_groups(p, kind, len(k), mem, a))


def ba_add_observations(p, kind, cam, feature, other=None, meas=None):
    f, mem, kf = _arr(feature, np.int32)
    c, _, kc = _arr(cam, np.int32)
    o, _, ko = _arr(other, np.int32)
    m, _, km = _arr(meas, np.float64) if MEAS_DIM[kind] else (None, 0, None)
    _check(p, _lib.ba_add_observations(p, kind, len(kf), mem, c, f, o, m))


def ba_add_relations(p, kind_a, a, kind_b, b, type_):
    """Inter-group relations: per relation the kinds (BA_PLANE / BA_VP) and ids of its two groups and its type
    (BA_REL_ORTHOGONAL / BA_REL_PARALLEL)."""
    ka, mem, k1 = _arr(kind_a, np.int32)
    aa, _, k2 = _arr(a, np.int32)
    kb, _, k3 = _arr(kind_b, np.int32)
    bb, _, k4 = _arr(b, np.int32)
    tt, _, k5 = _arr(type_, np.int32)
    _check(p, _lib.ba_add_relations(p, len(k2), mem, ka, aa, kb, bb, tt))


def ba_set_intrinsics(p, values, intr_of_cam):
    """Refined intrinsics shared by camera model (cam_dof = 9): values [n_intr, 3] = (f, k1, k2), intr_of_cam
    [n_cams] the entity of every camera."""
    v, mem, kv = _arr(values, np.float64)
    m, _, km = _arr(intr_of_cam, np.int32)
    _check(p, _lib.ba_set_intrinsics(p, len(kv) if kv is not None else 0, mem, v, m, len(km) if km is not None else 0))


def ba_get_intrinsics(p, n):
    """Current (f, k1, k2) of every camera, [n, 3]."""
    out = np.empty((n, 3))
    _check(p, _lib.ba_get_intrinsics(p, BA_MEM_HOST, out.ctypes.data_as(C.c_void_p)))
    return out


def ba_intrinsics_count(p):
    n = C.c_int64()
    _check(p, _lib.ba_intrinsics_count(p, C.byref(n)))
    return n.value


def ba_get_step_intrinsics(p):
    """The intrinsics part of the last computed step, [n_intr, 3]."""
    n = ba_intrinsics_count(p)
    out = np.empty((n, 3))
    _check(p, _lib.ba_get_step_intrinsics(p, out.ctypes.data_as(C.c_void_p)))
    return out


def ba_lm_step(p):
    r = ba_step_report()
    _check(p, _lib.ba_lm_step(p, C.byref(r)))
    return r


def ba_solve(p):
    r = ba_solve_report()
    _check(p, _lib.ba_solve(p, C.byref(r)))
    return r


def ba_get_cameras(p, n):
    out = np.empty((n, 7))
    _check(p, _lib.ba_get_cameras(p, BA_MEM_HOST, out.ctypes.data_as(C.c_void_p)))
    return out


def ba_get_features(p, kind, n):
    out = np.empty((n, 3 if kind == BA_POINT else 6))
    _check(p, _lib.ba_get_features(p, kind, BA_MEM_HOST, out.ctypes.data_as(C.c_void_p)))
    return out


GROUP_WIDTH = {0: 4, 1: 3, 2: 4, 3: 7, 4: 7, 5: 10, 6: 10}   # BA_PLANE ... BA_CUBOID


def ba_get_groups(p, kind, n):
    out = np.empty((n, GROUP_WIDTH[kind]))
    _check(p, _lib.ba_get_groups(p, kind, BA_MEM_HOST, out.ctypes.data_as(C.c_void_p)))
    return out


def ba_get_lm_state(p):
    out = np.empty(2)
    _check(p, _lib.ba_get_lm_state(p, out.ctypes.data_as(C.c_void_p)))
    return out


def ba_set_lm_state(p, lam, nu):
    a = np.array([lam, nu], np.float64)
    _check(p, _lib.ba_set_lm_state(p, a.ctypes.data_as(C.c_void_p)))


def ba_eval_cost(p):
    e, epx = C.c_double(), C.c_double()
    _check(p, _lib.ba_eval_cost(p, C.byref(e), C.byref(epx)))
    return e.value, epx.value


def ba_build_reduced(p, lam):
    _check(p, _lib.ba_build_reduced(p, float(lam)))


def ba_reduced_size(p):
    a, b = C.c_int64(), C.c_int64()
    _check(p, _lib.ba_reduced_size(p, C.byref(a), C.byref(b)))
    return a.value, b.value


def ba_export_reduced_system(p, values=True):
    """(row_ptr, cols, vals [nb, 6, 6] or None when values=False, b [na, 6])."""
    na, nb = ba_reduced_size(p)
    rp = np.empty(na + 1, np.int32); cols = np.empty(nb, np.int32)
    vals = np.empty((nb, 6, 6)) if values else None
    b = np.empty((na, 6))
    ptr = lambda a: a.ctypes.data_as(C.c_void_p) if a is not None else None
    _check(p, _lib.ba_export_reduced_system(p, ptr(rp), ptr(cols), ptr(vals), ptr(b)))
    return rp, cols, vals, b


def ba_compute_step(p, counts):
    """counts = (nc, npl, nv, np, nl); returns dict of per-entity increments and PCG info."""
    nc, npl, nv, np_, nl = counts
    out = dict(cam=np.empty((nc, 6)), plane=np.empty((npl, 3)), vp=np.empty((nv, 2)),
               point=np.empty((np_, 3)), line=np.empty((nl, 4)))
    it, rel, pred = C.c_int(), C.c_double(), C.c_double()
    ptr = lambda a: a.ctypes.data_as(C.c_void_p)
    _check(p, _lib.ba_compute_step(p, ptr(out["cam"]), ptr(out["plane"]), ptr(out["vp"]), ptr(out["point"]),
                                   ptr(out["line"]), C.byref(it), C.byref(rel), C.byref(pred)))
    out.update(pcg_iters=it.value, pcg_rel=rel.value, pred=pred.value)
    return out


# ---------------------------------------------------------------------------- scene marshalling
def load_scene(p, scene, device_tensors=False):
    """Add every array of a scene dict (cams, points, lines, planes, vps, obs, fixed) to the problem.
    With device_tensors=True the arrays are first placed on the current CUDA device (BA_MEM_DEVICE)."""
    conv = (lambda a: a)
    if device_tensors:
        import torch
        conv = (lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda())
    c = scene["cams"]
    quat_t = np.concatenate([c["q"], c["t"]], 1)
    ba_add_cameras(p, conv(quat_t), conv(c["intr"]), conv(c["pp"]),
                   conv(scene["fixed"].astype(np.uint8)) if "fixed" in scene else None)
    if len(scene["points"]):
        ba_add_features(p, BA_POINT, conv(scene["points"]))
    if len(scene["lines"]):
        ba_add_features(p, BA_LINE, conv(scene["lines"]))
    if len(scene["planes"]):
        ba_add_groups(p, BA_PLANE, conv(scene["planes"]))
    if len(scene["vps"]):
        ba_add_groups(p, BA_VP, conv(scene["vps"]))
    for key, kind in (("spheres", BA_SPHERE), ("cylinders", BA_CYLINDER), ("cones", BA_CONE),
                      ("ellipsoids", BA_ELLIPSOID), ("cuboids", BA_CUBOID)):
        if len(scene.get(key, ())):
            ba_add_groups(p, kind, conv(np.asarray(scene[key], np.float64)))
    ik = scene.get("intrinsics")
    if ik is not None:
        ba_set_intrinsics(p, conv(np.asarray(ik["values"], np.float64)), conv(np.asarray(ik["of_cam"], np.int32)))
    rel = scene.get("relations")
    if rel is not None and len(rel["a"]):
        ba_add_relations(p, conv(rel["ka"].astype(np.int32)), conv(rel["a"]), conv(rel["kb"].astype(np.int32)),
                         conv(rel["b"]), conv(rel["type"].astype(np.int32)))
    for name, k in OBS_KINDS.items():
        o = scene["obs"].get(name)
        if o is None or len(o["feat"]) == 0:
            continue
        meas = o["meas"] if MEAS_DIM[k] else None
        ba_add_observations(p, k, conv(o["cam"]) if k not in NO_CAM else None, conv(o["feat"]), conv(o["other"]),
                            conv(meas) if meas is not None else None)


def ba_pcg_solve_static(row_ptr, cols, vals, b, x, rel_tol=1e-6, max_iters=1000, stream=None):
    """Allocation-free PCG on a reduced system: row_ptr a host int32 array, cols / vals / b / x CUDA tensors
    (int32, float64 [nnz, 6, 6], float64 [6n], float64 [6n] output).  Returns (iterations, relative residual)."""
    import torch
    rp = np.ascontiguousarray(row_ptr)
    if rp.dtype != np.int32 or rp.ndim != 1 or len(rp) < 2:
        raise BAError(BA_ERR_ARG, "row_ptr: expected a 1-D int32 host array of n_block_rows + 1 offsets")
    n, nnz = len(rp) - 1, int(rp[-1])
    if rp[0] != 0 or np.any(np.diff(rp) <= 0):
        raise BAError(BA_ERR_ARG, "row_ptr: must start at 0 and give every block row at least its diagonal block")
    _need_dev((cols, torch.int32, nnz, "cols"), (vals, torch.float64, 36 * nnz, "vals"),
              (b, torch.float64, 6 * n, "b"), (x, torch.float64, 6 * n, "x"))
    it, rel = C.c_int(), C.c_double()
    err = C.create_string_buffer(256)
    st = _lib.ba_pcg_solve_static(n, int(rp[-1]), rp.ctypes.data_as(C.c_void_p), C.c_void_p(cols.data_ptr()),
                                  C.c_void_p(vals.data_ptr()), C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()),
                                  float(rel_tol), int(max_iters), C.c_void_p(stream or 0), C.byref(it), C.byref(rel),
                                  err, 256)
    if st != BA_OK:
        raise BAError(st, err.value.decode())
    return it.value, rel.value


def ba_eval_log1p(x, stream=None):
    """ln(1 + x) of a CUDA float64 tensor as the library's cost pass evaluates it; returns a new tensor."""
    import torch
    _need_dev((x, torch.float64, x.numel(), "x"))
    y = torch.empty_like(x)
    st = _lib.ba_eval_log1p(x.numel(), _dp(x), _dp(y), C.c_void_p(stream or 0))
    if st != BA_OK:
        raise BAError(st, "ba_eval_log1p failed")
    return y


def ba_measure_fma_rate(precision, stream=None):
    """Measured FMA throughput (TFLOP/s, 2 flops per FMA) of the FP32 pipe (BA_MIXED) or FP64 pipe (BA_FP64)."""
    v = C.c_double()
    st = _lib.ba_measure_fma_rate(int(precision), C.byref(v), C.c_void_p(stream or 0))
    if st != BA_OK:
        raise BAError(st, "ba_measure_fma_rate failed")
    return v.value


# ---------------------------------------------------------------------------- learned preconditioner
def ba_precond_param_count():
    return _lib.ba_precond_param_count()


def ba_precond_set_weights(p, params):
    a = np.ascontiguousarray(params, np.float32)
    _check(p, _lib.ba_precond_set_weights(p, a.ctypes.data_as(C.c_void_p), len(a)))


def ba_precond_features(p, na):
    X = np.empty((na, 32), np.float32)
    m = np.empty(na, np.uint8)
    _check(p, _lib.ba_precond_features(p, X.ctypes.data_as(C.c_void_p), m.ctypes.data_as(C.c_void_p)))
    return X, m


def ba_precond_blocks(p, na):
    out = np.empty((na, 6, 6))
    fb = C.c_int()
    _check(p, _lib.ba_precond_blocks(p, out.ctypes.data_as(C.c_void_p), C.byref(fb)))
    return out, fb.value


def _dp(t):
    return C.c_void_p(t.data_ptr())


def ba_mlp_grad(X, E, mask, params, stream=None):
    """X [n,32], E [n,21] float32, mask [n] uint8, params [P] float32: CUDA tensors.  Returns (loss, grad)."""
    import torch
    n = X.shape[0]
    P = ba_precond_param_count()
    _need_dev((X, torch.float32, 32 * n, "X"), (E, torch.float32, 21 * n, "E"), (mask, torch.uint8, n, "mask"),
              (params, torch.float32, P, "params"))
    grad = torch.empty(ba_precond_param_count() - 64, dtype=torch.float32, device=X.device)
    work = torch.empty(int(_lib.ba_mlp_work_floats(n)) + 8, dtype=torch.float32, device=X.device)
    loss = C.c_double()
    st = _lib.ba_mlp_grad(n, _dp(X), _dp(E), _dp(mask), _dp(params), _dp(grad), C.byref(loss), _dp(work),
                          C.c_void_p(stream or 0))
    if st != BA_OK:
        raise BAError(st, "ba_mlp_grad failed")
    return loss.value, grad


def ba_precond_train(X, E, mask, params, adam_m, adam_v, t0, steps, batch, lr, stream=None):
    """In-place Adam training of params (CUDA tensors); returns the last mini-batch loss."""
    import torch
    n = X.shape[0]
    P = ba_precond_param_count()
    _need_dev((X, torch.float32, 32 * n, "X"), (E, torch.float32, 21 * n, "E"), (mask, torch.uint8, n, "mask"),
              (params, torch.float32, P, "params"), (adam_m, torch.float32, P - 64, "adam_m"),
              (adam_v, torch.float32, P - 64, "adam_v"))
    if n < 1 or int(batch) < 1 or int(steps) < 0 or int(t0) < 0:
        raise BAError(BA_ERR_ARG, "need n >= 1, batch >= 1, steps >= 0 and t0 >= 0")
    work = torch.empty(int(_lib.ba_mlp_work_floats(batch)) + 8, dtype=torch.float32, device=X.device)
    loss = C.c_double()
    st = _lib.ba_precond_train(X.shape[0], _dp(X), _dp(E), _dp(mask), _dp(params), _dp(adam_m), _dp(adam_v),
                               int(t0), int(steps), int(batch), float(lr), _dp(work), C.byref(loss),
                               C.c_void_p(stream or 0))
    if st != BA_OK:
        raise BAError(st, "ba_precond_train failed")
    return loss.value


# ---------------------------------------------------------------------------- batched windows
def ba_solve_batch(problems, lm_iters=10, autotune=True):
    """Solve independent problems (handles) in one persistent launch; returns their reports."""
    n = len(problems)
    arr = (C.c_void_p * n)(*problems)
    reps = (ba_solve_report * n)()
    st = _lib.ba_solve_batch(C.cast(arr, C.c_void_p), n, int(lm_iters), 1 if autotune else 0, C.cast(reps, C.c_void_p))
    _check(problems[0], st)
    return list(reps)


def ba_batch_ctas_per_window(p):
    """(CTAs per window, number of the largest windows that ran on clusters) of the last batched solve."""
    c, k = C.c_int(), C.c_int()
    _check(p, _lib.ba_batch_ctas_per_window(p, C.byref(c), C.byref(k)))
    return c.value, k.value


def ba_batch_launch_shape(p):
    t, g = C.c_int(), C.c_int()
    _check(p, _lib.ba_batch_launch_shape(p, C.byref(t), C.byref(g)))
    return t.value, g.value
