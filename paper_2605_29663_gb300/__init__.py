"""EXACT-MPPI hot path on GB300 (sm_103a): thin Python binding of the C ABI.

Every step of the method runs in the CUDA library ``_lib/libexact_mppi.so``
(declared in ``include/exact_mppi.h``).  This module only marshals
arguments: it checks dtypes, devices and shapes of torch tensors, allocates
outputs with torch (device memory is torch's job here) and passes raw
pointers and the current CUDA stream through ctypes.  There is no CPU
fallback: if the library has not been built, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

__all__ = ["load", "Footprint", "Context", "MppiParams", "sdf_batch", "mppi_step", "Batch", "Hybrid", "ExactError", "MLP",
           "polar_hist", "proposal_features", "proposal_prepare", "proposal_select",
           "POLYGON", "RECTS", "DIFF", "ACKERMANN", "OMNI", "SPIN", "PARALLEL", "NU", "EXPORTS"]

POLYGON, RECTS = 0, 1
DIFF, ACKERMANN, OMNI, SPIN, PARALLEL = 0, 1, 2, 3, 4
NU = {DIFF: 2, ACKERMANN: 2, OMNI: 3, SPIN: 1, PARALLEL: 1}

# every symbol declared in include/exact_mppi.h
EXPORTS = ["exact_status_string", "exact_footprint_create", "exact_footprint_destroy",
           "exact_footprint_info", "exact_ctx_create", "exact_ctx_destroy", "exact_ctx_reserve",
           "exact_ctx_reserve_cloud",
           "exact_ctx_get_error", "exact_sdf_batch", "mppi_step", "mppi_step_predicted", "exact_batch_create",
           "exact_batch_destroy",
           "mppi_step_batched", "exact_batch_autotune", "exact_batch_get_tiles", "exact_batch_set_tiles",
           "exact_batch_get_error", "exact_ctx_enable_stats", "exact_ctx_get_stats", "exact_mlp_get_state",
           "exact_mlp_set_state",
           "mppi_step_noalloc", "exact_mlp_create", "exact_mlp_destroy", "exact_mlp_num_params",
           "exact_mlp_set_params", "exact_mlp_get_params", "exact_mlp_forward", "exact_mlp_loss_grad",
           "exact_mlp_train_step", "exact_polar_hist", "exact_proposal_features", "exact_proposal_prepare",
           "exact_proposal_select", "exact_hybrid_create", "exact_hybrid_destroy", "mppi_step_hybrid",
           "exact_hybrid_batch"]

_lock = threading.Lock()
_lib = None


class ExactError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} (status {status})")
        self.status = status


class CycleStats(ctypes.Structure):
    """Mirror of exact_cycle_stats."""
    _fields_ = [("cycles", ctypes.c_longlong), ("validation_failures", ctypes.c_longlong), ("ess", ctypes.c_float),
                ("cost_min", ctypes.c_float), ("cost_mean", ctypes.c_float), ("last_valid", ctypes.c_int)]


def load() -> ctypes.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB_PATH):
            raise RuntimeError(f"{_build.LIB_PATH} is missing: build it with "
                               "`python -m paper_2605_29663_gb300.build` (nvcc, sm_103a)")
        _lib = _bind(ctypes.CDLL(_build.LIB_PATH))
        return _lib


_lib_debug = None


def load_debug() -> ctypes.CDLL:
    """Load the debug variant of the library (device-side index checks;
    built by ``build.build(debug=True)``).  Its objects are its own: pass
    them only to its functions."""
    global _lib_debug
    with _lock:
        if _lib_debug is None:
            if not os.path.exists(_build.LIB_PATH_DEBUG):
                raise RuntimeError(f"{_build.LIB_PATH_DEBUG} is missing: build it with build.build(debug=True)")
            _lib_debug = _bind(ctypes.CDLL(_build.LIB_PATH_DEBUG))
        return _lib_debug


def _bind(lib):
    """Declare the argument and result types of every exported function."""
    P, I, V = ctypes.c_void_p, ctypes.c_int, None
    lib.exact_status_string.restype = ctypes.c_char_p
    lib.exact_status_string.argtypes = [I]
    lib.exact_footprint_create.restype = I
    lib.exact_footprint_create.argtypes = [I, P, I, ctypes.POINTER(P)]
    lib.exact_footprint_destroy.restype = V
    lib.exact_footprint_destroy.argtypes = [P]
    lib.exact_footprint_info.restype = I
    lib.exact_footprint_info.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I)]
    lib.exact_ctx_create.restype = I
    lib.exact_ctx_create.argtypes = [ctypes.POINTER(P)]
    lib.exact_ctx_destroy.restype = V
    lib.exact_ctx_destroy.argtypes = [P]
    lib.exact_ctx_reserve.restype = I
    lib.exact_ctx_reserve.argtypes = [P, I, I, I]
    lib.exact_ctx_reserve_cloud.restype = I
    lib.exact_ctx_reserve_cloud.argtypes = [P, I, I, I, I]
    lib.exact_ctx_get_error.restype = I
    lib.exact_ctx_get_error.argtypes = [P, P]
    lib.exact_batch_get_error.restype = I
    lib.exact_batch_get_error.argtypes = [P, P]
    lib.exact_ctx_enable_stats.restype = I
    lib.exact_ctx_enable_stats.argtypes = [P, I]
    lib.exact_ctx_get_stats.restype = I
    lib.exact_ctx_get_stats.argtypes = [P, ctypes.POINTER(CycleStats), P]
    lib.exact_mlp_get_state.restype = I
    lib.exact_mlp_get_state.argtypes = [P, P, P, P, ctypes.POINTER(ctypes.c_longlong)]
    lib.exact_mlp_set_state.restype = I
    lib.exact_mlp_set_state.argtypes = [P, P, P, P, ctypes.c_longlong]
    lib.exact_sdf_batch.restype = I
    lib.exact_sdf_batch.argtypes = [P, P, P, I, P, I, P, P, P, P, P]
    lib.mppi_step.restype = I
    lib.mppi_step.argtypes = [P, P, P, P, I, P, I, P, P, P, P, P, P, P, P, P, P, P]
    lib.mppi_step_predicted.restype = I
    lib.mppi_step_predicted.argtypes = [P, P, P, P, P, I, P, I, P, P, P, P, P, P, P, P, P, P, P]
    lib.exact_batch_create.restype = I
    lib.exact_batch_create.argtypes = [I, P, ctypes.POINTER(P)]
    lib.exact_batch_destroy.restype = V
    lib.exact_batch_destroy.argtypes = [P]
    lib.mppi_step_batched.restype = I
    lib.mppi_step_batched.argtypes = [P, P]
    lib.exact_batch_autotune.restype = I
    lib.exact_batch_autotune.argtypes = [P, I, ctypes.c_char_p, I, P]
    lib.exact_batch_get_tiles.restype = I
    lib.exact_batch_get_tiles.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I)]
    lib.exact_batch_set_tiles.restype = I
    lib.exact_batch_set_tiles.argtypes = [P, I, I]
    lib.mppi_step_noalloc.restype = I
    lib.mppi_step_noalloc.argtypes = [P, P, P, I, P, I, P, P, P, P, P, P, P, P, P, P, P]
    F, LL = ctypes.c_float, ctypes.c_longlong
    lib.exact_mlp_create.restype = I
    lib.exact_mlp_create.argtypes = [I, I, I, I, ctypes.POINTER(P)]
    lib.exact_mlp_destroy.restype = V
    lib.exact_mlp_destroy.argtypes = [P]
    lib.exact_mlp_num_params.restype = LL
    lib.exact_mlp_num_params.argtypes = [P]
    lib.exact_mlp_set_params.restype = I
    lib.exact_mlp_set_params.argtypes = [P, P]
    lib.exact_mlp_get_params.restype = I
    lib.exact_mlp_get_params.argtypes = [P, P]
    lib.exact_mlp_forward.restype = I
    lib.exact_mlp_forward.argtypes = [P, P, I, P, P]
    lib.exact_mlp_loss_grad.restype = I
    lib.exact_mlp_loss_grad.argtypes = [P, P, P, I, P, P, P]
    lib.exact_mlp_train_step.restype = I
    lib.exact_mlp_train_step.argtypes = [P, P, P, I, F, P, P]
    lib.exact_polar_hist.restype = I
    lib.exact_polar_hist.argtypes = [P, P, I, I, P, I, F, P, P]
    lib.exact_proposal_features.restype = I
    lib.exact_proposal_features.argtypes = [P, I, F, P, P, P, P, I, I, P, P]
    lib.exact_proposal_prepare.restype = I
    lib.exact_proposal_prepare.argtypes = [P, P, LL, P, P, P]
    lib.exact_proposal_select.restype = I
    lib.exact_proposal_select.argtypes = [P, P, I, I, P, P, P, P, I, I, P, P, P, P]
    lib.exact_hybrid_create.restype = I
    lib.exact_hybrid_create.argtypes = [I, P, P, ctypes.POINTER(P)]
    lib.exact_hybrid_destroy.restype = V
    lib.exact_hybrid_destroy.argtypes = [P]
    lib.mppi_step_hybrid.restype = I
    lib.mppi_step_hybrid.argtypes = [P, P, P, P, P]
    lib.exact_hybrid_batch.restype = P
    lib.exact_hybrid_batch.argtypes = [P]
    return lib


def status_string(status: int) -> str:
    return load().exact_status_string(int(status)).decode()


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ExactError(rc, what)


def _torch():
    import torch
    return torch


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dev(t, name, dtype=None, shape=None):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t


def _stream(stream):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class Footprint:
    """Effective footprint (Sec. III-B): a simple polygon (n x 2 vertices) or a
    rectangle cover (n x 4: cx, cy, sx, sy)."""

    def __init__(self, kind: int, data):
        import numpy as np
        arr = np.ascontiguousarray(np.asarray(data, dtype=np.float32))
        per = 2 if kind == POLYGON else 4
        arr = arr.reshape(-1, per)
        h = ctypes.c_void_p()
        _check(load().exact_footprint_create(kind, arr.ctypes.data, arr.shape[0], ctypes.byref(h)),
               "exact_footprint_create")
        self._h = h
        self.kind = kind
        self.n = arr.shape[0]
        self.data = arr.copy()

    @classmethod
    def polygon(cls, verts):
        return cls(POLYGON, verts)

    @classmethod
    def rects(cls, boxes):
        return cls(RECTS, boxes)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            load().exact_footprint_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """Device scratch arena + error word (bound to the current device)."""

    def __init__(self):
        h = ctypes.c_void_p()
        _check(load().exact_ctx_create(ctypes.byref(h)), "exact_ctx_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def reserve(self, max_poses: int = 0, max_K: int = 0, max_T: int = 0, max_points: int = 0):
        """Allocate scratch ahead of time (before a CUDA graph capture): SDF
        batches of max_poses poses, MPPI steps of max_K x max_T, clouds of
        max_points points (their spatially ordered copy)."""
        _check(load().exact_ctx_reserve_cloud(self._h, max_poses, max_K, max_T, max_points),
               "exact_ctx_reserve_cloud")

    def get_error(self, stream=None) -> int:
        """The context's device error word (0 = none), read and cleared in the
        order of `stream` (default: the current stream), which is synchronised."""
        return load().exact_ctx_get_error(self._h, _stream(stream))

    def enable_stats(self, enable: bool = True):
        """Record per-cycle statistics (ESS, J~ min / mean, validation) of the
        MPPI steps run with this context."""
        _check(load().exact_ctx_enable_stats(self._h, int(bool(enable))), "exact_ctx_enable_stats")

    def get_stats(self, stream=None) -> dict:
        """The statistics record (its counters are zeroed by the read)."""
        st = CycleStats()
        _check(load().exact_ctx_get_stats(self._h, ctypes.byref(st), _stream(stream)), "exact_ctx_get_stats")
        return {k: getattr(st, k) for k, _ in CycleStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            load().exact_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sdf_batch(points, poses, footprint: Footprint, mask=None, *, dist=True, dmin=True, argmin=True,
              ctx: Context | None = None, out=None, stream=None):
    """Batched body-frame signed distances (Sec. IV-C/D).  Returns
    (dist [P, N] | None, dmin [P] | None, argmin [P] int32 | None)."""
    torch = _torch()
    points = _dev(points, "points", torch.float32)
    poses = _dev(poses, "poses", torch.float32)
    N = points.shape[0] if points.numel() else 0
    P = poses.shape[0]
    if points.numel() and (points.dim() != 2 or points.shape[1] != 2):
        raise ValueError("points must be N x 2")
    if poses.dim() != 2 or poses.shape[1] != 3:
        raise ValueError("poses must be P x 3")
    if mask is not None:
        mask = _dev(mask, "mask", torch.uint8, (N,))
    o = out or {}
    d = o.get("dist") if dist else None
    if dist and d is None:
        d = torch.empty((P, N), dtype=torch.float32, device=poses.device)
    m = o.get("dmin") if dmin else None
    if dmin and m is None:
        m = torch.empty(P, dtype=torch.float32, device=poses.device)
    a = o.get("argmin") if argmin else None
    if argmin and a is None:
        a = torch.empty(P, dtype=torch.int32, device=poses.device)
    _check(load().exact_sdf_batch(ctx.handle if ctx else None, _ptr(points) if N else None, _ptr(mask), N,
                                  _ptr(poses), P, footprint.handle, _ptr(d), _ptr(m), _ptr(a),
                                  _stream(stream)), "exact_sdf_batch")
    return d, m, a


class MppiParams(ctypes.Structure):
    """Mirror of exact_mppi_params."""
    _fields_ = [("K", ctypes.c_int), ("T", ctypes.c_int), ("n_u", ctypes.c_int), ("model", ctypes.c_int),
                ("dt", ctypes.c_float), ("lam", ctypes.c_float), ("d_safe", ctypes.c_float),
                ("w_coll", ctypes.c_float), ("w_rep", ctypes.c_float), ("w_inf", ctypes.c_float),
                ("w_goal", ctypes.c_float), ("w_term", ctypes.c_float), ("w_ctrl", ctypes.c_float),
                ("wheelbase", ctypes.c_float),
                ("u_min", ctypes.c_float * 3), ("u_max", ctypes.c_float * 3),
                ("clamp", ctypes.c_int), ("state_offset", ctypes.c_int)]

    @classmethod
    def from_dict(cls, d: dict) -> "MppiParams":
        p = cls()
        p.K, p.T, p.n_u, p.model = int(d["K"]), int(d["T"]), int(d["nu"]), int(d["model"])
        for k in ("dt", "d_safe", "w_coll", "w_rep", "w_inf", "w_goal", "w_term", "w_ctrl", "wheelbase"):
            setattr(p, k, float(d[k]))
        p.lam = float(d["lambda"])
        for j in range(3):
            p.u_min[j] = max(float(d["u_min"][j]), -3.0e38)
            p.u_max[j] = min(float(d["u_max"][j]), 3.0e38)
        p.clamp = int(d["clamp"])
        p.state_offset = int(d["state_offset"])
        return p


def mppi_step(ctx: Context, state, cloud, waypoints, U, noise, footprint: Footprint, params, mask=None, *,
              velocity=None, costs=True, weights=True, U_upd=True, dmin=False, out=None, stream=None) -> dict:
    """One EXACT-MPPI control cycle (Algorithm 1).  U is updated in place
    (shifted, or reset to zero when validation fails).  Returns a dict of
    device tensors: u_star, valid, and the requested costs / weights /
    U_upd / dmin.  `velocity` (N x 2, m/s) switches to time-indexed
    obstacle predictions (mppi_step_predicted): step h sees o + t_h v."""
    torch = _torch()
    p = params if isinstance(params, MppiParams) else MppiParams.from_dict(params)
    K, T, nu = p.K, p.T, p.n_u
    state = _dev(state, "state", torch.float32, (3,))
    U = _dev(U, "U", torch.float32, (T, nu))
    noise = _dev(noise, "noise", torch.float32, (K, T, nu))
    waypoints = _dev(waypoints, "waypoints", torch.float32)
    W = waypoints.shape[0]
    cloud = _dev(cloud, "cloud", torch.float32)
    N = cloud.shape[0] if cloud.numel() else 0
    if mask is not None:
        mask = _dev(mask, "mask", torch.uint8, (N,))
    if velocity is not None:
        velocity = _dev(velocity, "velocity", torch.float32, (N, 2) if N else None)
    dev = U.device
    o = dict(out or {})
    if "u_star" not in o:
        o["u_star"] = torch.empty(nu, dtype=torch.float32, device=dev)
    if "valid" not in o:
        o["valid"] = torch.empty(1, dtype=torch.int32, device=dev)
    if costs and "costs" not in o:
        o["costs"] = torch.empty(K, dtype=torch.float32, device=dev)
    if weights and "weights" not in o:
        o["weights"] = torch.empty(K, dtype=torch.float32, device=dev)
    if U_upd and "U_upd" not in o:
        o["U_upd"] = torch.empty((T, nu), dtype=torch.float32, device=dev)
    if dmin and "dmin" not in o:
        o["dmin"] = torch.empty((K, T), dtype=torch.float32, device=dev)
    tail = (_ptr(o["u_star"]), _ptr(o.get("costs")), _ptr(o.get("weights")), _ptr(o["valid"]),
            _ptr(o.get("U_upd")), _ptr(o.get("dmin")), _stream(stream))
    if velocity is None:
        _check(load().mppi_step(ctx.handle, _ptr(state), _ptr(cloud) if N else None, _ptr(mask), N,
                                _ptr(waypoints), W, _ptr(U), _ptr(noise), footprint.handle, ctypes.byref(p), *tail),
               "mppi_step")
    else:
        _check(load().mppi_step_predicted(ctx.handle, _ptr(state), _ptr(cloud) if N else None,
                                          _ptr(velocity) if N else None, _ptr(mask), N, _ptr(waypoints), W, _ptr(U),
                                          _ptr(noise), footprint.handle, ctypes.byref(p), *tail),
               "mppi_step_predicted")
    return o


class ExactScene(ctypes.Structure):
    """Mirror of exact_scene."""
    _fields_ = [("state", ctypes.c_void_p), ("cloud", ctypes.c_void_p), ("mask", ctypes.c_void_p),
                ("n_points", ctypes.c_int), ("waypoints", ctypes.c_void_p), ("n_wp", ctypes.c_int),
                ("U", ctypes.c_void_p), ("noise", ctypes.c_void_p), ("fp", ctypes.c_void_p),
                ("params", MppiParams), ("u_star", ctypes.c_void_p), ("costs", ctypes.c_void_p),
                ("weights", ctypes.c_void_p), ("valid", ctypes.c_void_p), ("U_upd", ctypes.c_void_p),
                ("dmin", ctypes.c_void_p), ("nom_cost", ctypes.c_void_p)]


def scene_class_key(scenes, device: str = "") -> str:
    """Key of a batch's shape class for the tile cache: the sorted multiset of
    (footprint kind, footprint size, N rounded up to a power of two, K, T) of
    its scenes, and the device name.  Batches with the same key are expected
    to prefer the same tile shape."""
    import hashlib
    import json
    items = []
    for sc in scenes:
        fp = sc["fp"]
        p = sc["params"]
        K, T = (p.K, p.T) if isinstance(p, MppiParams) else (int(p["K"]), int(p["T"]))
        N = int(sc["cloud"].shape[0]) if sc["cloud"].numel() else 0
        items.append([int(fp.kind), int(fp.n), 1 << max(N - 1, 0).bit_length(), K, T])
    items.sort()
    blob = json.dumps({"scenes": items, "device": device}, sort_keys=True)
    return hashlib.sha256(blob.encode()).hexdigest()[:24]


def tile_cache_lookup(path: str, key: str):
    """(threads, pairs_per_lane) stored for `key` in the JSON tile cache, or None."""
    import json
    try:
        with open(path) as fh:
            e = json.load(fh).get(key)
    except (OSError, ValueError):
        return None
    if not isinstance(e, dict):
        return None
    try:
        return int(e["threads"]), int(e["pairs_per_lane"])
    except (KeyError, TypeError, ValueError):
        return None


def tile_cache_store(path: str, key: str, threads: int, pairs_per_lane: int, ms: float) -> None:
    """Record the tuned tile shape for `key` (read-modify-write, atomic rename)."""
    import json
    import tempfile
    try:
        with open(path) as fh:
            data = json.load(fh)
        if not isinstance(data, dict):
            data = {}
    except (OSError, ValueError):
        data = {}
    data[key] = {"threads": int(threads), "pairs_per_lane": int(pairs_per_lane), "ms": float(ms)}
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=d, prefix=".tiles-", suffix=".json")
    with os.fdopen(fd, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _scene_array(scenes, dmin, costs, weights, U_upd, nom_cost):
    """exact_scene array for a list of scene dicts (see Batch), the output
    tensors allocated for each scene, and the tensors the array points into."""
    torch = _torch()
    keep = []
    arr = (ExactScene * len(scenes))()
    outputs = []
    for i, sc in enumerate(scenes):
        p = sc["params"] if isinstance(sc["params"], MppiParams) else MppiParams.from_dict(sc["params"])
        K, T, nu = p.K, p.T, p.n_u
        state = _dev(sc["state"], "state", torch.float32, (3,))
        U = _dev(sc["U"], "U", torch.float32, (T, nu))
        noise = _dev(sc["noise"], "noise", torch.float32, (K, T, nu))
        wp = _dev(sc["waypoints"], "waypoints", torch.float32)
        cloud = _dev(sc["cloud"], "cloud", torch.float32)
        N = cloud.shape[0] if cloud.numel() else 0
        mask = sc.get("mask")
        if mask is not None:
            mask = _dev(mask, "mask", torch.uint8, (N,))
        dev = U.device
        o = {"u_star": torch.empty(nu, dtype=torch.float32, device=dev),
             "valid": torch.empty(1, dtype=torch.int32, device=dev)}
        if costs:
            o["costs"] = torch.empty(K, dtype=torch.float32, device=dev)
        if weights:
            o["weights"] = torch.empty(K, dtype=torch.float32, device=dev)
        if U_upd:
            o["U_upd"] = torch.empty((T, nu), dtype=torch.float32, device=dev)
        if dmin:
            o["dmin"] = torch.empty((K, T), dtype=torch.float32, device=dev)
        if nom_cost:
            o["nom_cost"] = torch.empty(1, dtype=torch.float32, device=dev)
        outputs.append(o)
        keep += [state, U, noise, wp, cloud, mask, sc["fp"]]
        e = arr[i]
        e.state, e.cloud, e.mask, e.n_points = state.data_ptr(), cloud.data_ptr() if N else None, \
            None if mask is None else mask.data_ptr(), N
        e.waypoints, e.n_wp, e.U, e.noise = wp.data_ptr(), wp.shape[0], U.data_ptr(), noise.data_ptr()
        e.fp = sc["fp"].handle
        e.params = p
        e.u_star, e.valid = o["u_star"].data_ptr(), o["valid"].data_ptr()
        e.costs = o["costs"].data_ptr() if costs else None
        e.weights = o["weights"].data_ptr() if weights else None
        e.U_upd = o["U_upd"].data_ptr() if U_upd else None
        e.dmin = o["dmin"].data_ptr() if dmin else None
        e.nom_cost = o["nom_cost"].data_ptr() if nom_cost else None
    return arr, outputs, keep


class Batch:
    """Plan + device scratch for advancing many scenes by one control cycle
    each in one persistent launch (mppi_step_batched).

    `scenes` is a list of dicts with device tensors state, cloud, waypoints,
    U (in/out), noise, optional mask, a Footprint `fp` and `params`.  Output
    tensors (u_star, valid, costs, weights, U_upd, and dmin when
    dmin=True) are allocated here and exposed as `outputs[i]`; nom_cost=True
    adds `nom_cost`, the cost J of each scene's updated nominal."""

    def __init__(self, scenes, *, dmin=False, costs=True, weights=True, U_upd=True, nom_cost=False):
        arr, self.outputs, self._keep = _scene_array(scenes, dmin, costs, weights, U_upd, nom_cost)
        torch = _torch()
        self.class_key = scene_class_key(scenes, torch.cuda.get_device_name(self.outputs[0]["u_star"].device))
        h = ctypes.c_void_p()
        _check(load().exact_batch_create(len(scenes), ctypes.cast(arr, ctypes.c_void_p), ctypes.byref(h)),
               "exact_batch_create")
        self._h = h
        self.n = len(scenes)

    def step(self, stream=None):
        _check(load().mppi_step_batched(self._h, _stream(stream)), "mppi_step_batched")

    def get_error(self, stream=None) -> int:
        """The batch's device error word (0 = none), read and cleared in the
        order of `stream`, which is synchronised."""
        return load().exact_batch_get_error(self._h, _stream(stream))

    def autotune(self, iters: int = 3, stream=None, cache: str | None = None) -> dict:
        """Pick the tile shape by timing the candidates (exact_batch_autotune).
        With `cache` (a JSON file path) a shape already tuned for this batch's
        shape class (scene_class_key) is reused without timing, and a new
        result is stored there."""
        import json
        if cache:
            hit = tile_cache_lookup(cache, self.class_key)
            if hit is not None:
                self.set_tiles(*hit)
                return {"cached": True, "key": self.class_key,
                        "best": {"threads": hit[0], "pairs_per_lane": hit[1]}}
        buf = ctypes.create_string_buffer(8192)
        _check(load().exact_batch_autotune(self._h, iters, buf, 8192, _stream(stream)), "exact_batch_autotune")
        rep = json.loads(buf.value.decode())
        if cache:
            b = rep["best"]
            tile_cache_store(cache, self.class_key, b["threads"], b["pairs_per_lane"], b["ms"])
            rep["key"] = self.class_key
        return rep

    @property
    def tiles(self):
        t, p = ctypes.c_int(), ctypes.c_int()
        _check(load().exact_batch_get_tiles(self._h, ctypes.byref(t), ctypes.byref(p)), "exact_batch_get_tiles")
        return t.value, p.value

    def set_tiles(self, threads: int, pairs_per_lane: int):
        _check(load().exact_batch_set_tiles(self._h, threads, pairs_per_lane), "exact_batch_set_tiles")

    def close(self):
        if getattr(self, "_h", None):
            load().exact_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HybridParams(ctypes.Structure):
    """Mirror of exact_hybrid_params."""
    _fields_ = [("lambda_switch", ctypes.c_float), ("cool_max", ctypes.c_int)]


class Hybrid:
    """Hybrid-mode cycle (Algorithm 2, steps 1-2): the modes of one robot as
    scenes (dicts as for Batch, each with its own motion model, U, noise and
    params), advanced together, then the mode selection on the device.

    `mode_state` (int32 [m_prev, tau_cool, stopped]) and `u` (float32 [3])
    live on the device; `Jbar` holds the augmented costs of the last step and
    `outputs[m]` each mode's Algorithm 1 outputs (with nom_cost)."""

    def __init__(self, modes, lambda_switch: float, cool_max: int, *, m_prev: int = -1, costs=True,
                 weights=False, U_upd=True):
        torch = _torch()
        arr, self.outputs, self._keep = _scene_array(modes, False, costs, weights, U_upd, True)
        dev = self.outputs[0]["u_star"].device
        hp = HybridParams(float(lambda_switch), int(cool_max))
        h = ctypes.c_void_p()
        _check(load().exact_hybrid_create(len(modes), ctypes.cast(arr, ctypes.c_void_p), ctypes.byref(hp),
                                          ctypes.byref(h)), "exact_hybrid_create")
        self._h = h
        self.n = len(modes)
        self.mode_state = torch.tensor([int(m_prev), 0, 0], dtype=torch.int32, device=dev)
        self.u = torch.zeros(3, dtype=torch.float32, device=dev)
        self.Jbar = torch.empty(self.n, dtype=torch.float32, device=dev)

    def step(self, stream=None):
        _check(load().mppi_step_hybrid(self._h, self.mode_state.data_ptr(), self.u.data_ptr(),
                                       self.Jbar.data_ptr(), _stream(stream)), "mppi_step_hybrid")

    def autotune(self, iters: int = 3, stream=None) -> dict:
        import json
        buf = ctypes.create_string_buffer(8192)
        b = load().exact_hybrid_batch(self._h)
        _check(load().exact_batch_autotune(b, iters, buf, 8192, _stream(stream)), "exact_batch_autotune")
        return json.loads(buf.value.decode())

    def close(self):
        if getattr(self, "_h", None):
            load().exact_hybrid_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


CKPT_MAGIC = b"EXMLPCK1"


class MLP:
    """Proposal network on the tensor cores (see exact_mlp_* in the C header).
    Parameters are exchanged as one packed float32 vector
    [W1 (H x D), b1, W2 (H x H), b2, W3 (O x H), b3]."""

    def __init__(self, d_in: int, hidden: int, d_out: int, max_batch: int):
        h = ctypes.c_void_p()
        _check(load().exact_mlp_create(d_in, hidden, d_out, max_batch, ctypes.byref(h)), "exact_mlp_create")
        self._h = h
        self.d_in, self.hidden, self.d_out, self.max_batch = d_in, hidden, d_out, max_batch
        self.num_params = int(load().exact_mlp_num_params(h))

    def shapes(self):
        D, H, O = self.d_in, self.hidden, self.d_out
        return [(H, D), (H,), (H, H), (H,), (O, H), (O,)]

    def init_params(self, seed: int = 0):
        """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases (seeded)."""
        import numpy as np
        g = np.random.default_rng(seed)
        parts = []
        for shp in self.shapes():
            fan_in = shp[1] if len(shp) == 2 else (self.d_in if len(parts) == 1 else self.hidden)
            parts.append(g.uniform(-1.0, 1.0, size=shp) / np.sqrt(fan_in))
        self.set_params(np.concatenate([p.reshape(-1) for p in parts]))

    def set_params(self, flat):
        import numpy as np
        a = np.ascontiguousarray(np.asarray(flat, dtype=np.float32).reshape(-1))
        if a.size != self.num_params:
            raise ValueError(f"expected {self.num_params} parameters, got {a.size}")
        _check(load().exact_mlp_set_params(self._h, a.ctypes.data), "exact_mlp_set_params")

    def get_params(self):
        import numpy as np
        a = np.empty(self.num_params, dtype=np.float32)
        _check(load().exact_mlp_get_params(self._h, a.ctypes.data), "exact_mlp_get_params")
        return a

    def get_state(self):
        """(params, Adam first moments, Adam second moments, Adam step)."""
        import numpy as np
        w, m, v = (np.empty(self.num_params, dtype=np.float32) for _ in range(3))
        t = ctypes.c_longlong()
        _check(load().exact_mlp_get_state(self._h, w.ctypes.data, m.ctypes.data, v.ctypes.data, ctypes.byref(t)),
               "exact_mlp_get_state")
        return w, m, v, int(t.value)

    def set_state(self, w, m, v, step: int):
        import numpy as np
        arrs = [np.ascontiguousarray(np.asarray(a, dtype=np.float32).reshape(-1)) for a in (w, m, v)]
        if any(a.size != self.num_params for a in arrs):
            raise ValueError(f"expected {self.num_params} values per array")
        _check(load().exact_mlp_set_state(self._h, arrs[0].ctypes.data, arrs[1].ctypes.data, arrs[2].ctypes.data,
                                          int(step)), "exact_mlp_set_state")

    def save_checkpoint(self, path: str):
        """Flat binary checkpoint: a 64-byte header (CKPT_MAGIC, format
        version, d_in, hidden, d_out, number of parameters, Adam step, all
        little-endian), then the parameters, Adam's first and second moments
        (float32 each, packed like the parameter vector)."""
        import struct
        w, m, v, t = self.get_state()
        head = struct.pack("<8sIIIIqq", CKPT_MAGIC, 1, self.d_in, self.hidden, self.d_out, self.num_params, t)
        tmp = path + ".tmp"
        with open(tmp, "wb") as fh:
            fh.write(head.ljust(64, b"\0"))
            for a in (w, m, v):
                fh.write(a.astype("<f4").tobytes())
        os.replace(tmp, path)

    def load_checkpoint(self, path: str):
        """Restore a checkpoint written by save_checkpoint for this shape."""
        import struct

        import numpy as np
        with open(path, "rb") as fh:
            head = fh.read(64)
            magic, ver, d_in, hidden, d_out, n, t = struct.unpack("<8sIIIIqq", head[:40])
            if magic != CKPT_MAGIC or ver != 1:
                raise ValueError(f"{path}: not a proposal-network checkpoint")
            if (d_in, hidden, d_out, n) != (self.d_in, self.hidden, self.d_out, self.num_params):
                raise ValueError(f"{path}: shape {(d_in, hidden, d_out)} does not match "
                                 f"{(self.d_in, self.hidden, self.d_out)}")
            data = np.frombuffer(fh.read(12 * n), dtype="<f4")
        if data.size != 3 * n:
            raise ValueError(f"{path}: truncated")
        self.set_state(data[:n], data[n:2 * n], data[2 * n:], t)

    def unpack(self, flat):
        out, k = [], 0
        for shp in self.shapes():
            n = 1
            for s in shp:
                n *= s
            out.append(flat[k:k + n].reshape(shp))
            k += n
        return out

    def forward(self, x, out=None, stream=None):
        torch = _torch()
        x = _dev(x, "x", torch.float32)
        B = x.shape[0]
        y = out if out is not None else torch.empty((B, self.d_out), dtype=torch.float32, device=x.device)
        _check(load().exact_mlp_forward(self._h, _ptr(x), B, _ptr(y), _stream(stream)), "exact_mlp_forward")
        return y

    def loss_grad(self, x, target, stream=None):
        torch = _torch()
        x = _dev(x, "x", torch.float32)
        target = _dev(target, "target", torch.float32)
        loss = torch.empty(1, dtype=torch.float32, device=x.device)
        grads = torch.empty(self.num_params, dtype=torch.float32, device=x.device)
        _check(load().exact_mlp_loss_grad(self._h, _ptr(x), _ptr(target), x.shape[0], _ptr(loss), _ptr(grads),
                                          _stream(stream)), "exact_mlp_loss_grad")
        return loss, grads

    def train_step(self, x, target, lr: float, loss=None, stream=None):
        torch = _torch()
        x = _dev(x, "x", torch.float32)
        target = _dev(target, "target", torch.float32)
        if loss is None:
            loss = torch.empty(1, dtype=torch.float32, device=x.device)
        _check(load().exact_mlp_train_step(self._h, _ptr(x), _ptr(target), x.shape[0], float(lr), _ptr(loss),
                                           _stream(stream)), "exact_mlp_train_step")
        return loss

    def close(self):
        if getattr(self, "_h", None):
            load().exact_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def polar_hist(clouds, poses, nbins: int = 64, r_max: float = 10.0, masks=None, out=None, stream=None):
    """Nearest range per angular bin of each robot's points (B x N x 2 clouds, B x 3 poses)."""
    torch = _torch()
    clouds = _dev(clouds, "clouds", torch.float32)
    poses = _dev(poses, "poses", torch.float32)
    B, N = clouds.shape[0], clouds.shape[1]
    if masks is not None:
        masks = _dev(masks, "masks", torch.uint8, (B, N))
    o = out if out is not None else torch.empty((B, nbins), dtype=torch.float32, device=poses.device)
    _check(load().exact_polar_hist(_ptr(clouds), _ptr(masks), B, N, _ptr(poses), nbins, float(r_max), _ptr(o),
                                   _stream(stream)), "exact_polar_hist")
    return o


def proposal_features(hist, poses, goals, prev_cmd, U_prev, r_max: float = 10.0, out=None, stream=None):
    torch = _torch()
    B, nbins = hist.shape
    T = U_prev.shape[1]
    o = out if out is not None else torch.empty((B, nbins + 7 + 2 * T), dtype=torch.float32, device=hist.device)
    _check(load().exact_proposal_features(_ptr(_dev(hist, "hist", torch.float32)), nbins, float(r_max),
                                          _ptr(_dev(poses, "poses", torch.float32)),
                                          _ptr(_dev(goals, "goals", torch.float32)),
                                          _ptr(_dev(prev_cmd, "prev_cmd", torch.float32)),
                                          _ptr(_dev(U_prev, "U_prev", torch.float32)), T, B, _ptr(o), _stream(stream)),
           "exact_proposal_features")
    return o


def proposal_prepare(U_prev, shift, U_prop, U_plain, stream=None):
    _check(load().exact_proposal_prepare(_ptr(U_prev), _ptr(shift), U_prev.numel(), _ptr(U_prop), _ptr(U_plain),
                                         _stream(stream)), "exact_proposal_prepare")


def proposal_select(costs_prop, costs_plain, U_prop, U_plain, u_prop, u_plain, U_out, u_out, chose=None,
                    stream=None):
    B, K = costs_prop.shape
    T, nu = U_prop.shape[1], U_prop.shape[2]
    _check(load().exact_proposal_select(_ptr(costs_prop), _ptr(costs_plain), B, K, _ptr(U_prop), _ptr(U_plain),
                                        _ptr(u_prop), _ptr(u_plain), T, nu, _ptr(U_out), _ptr(u_out), _ptr(chose),
                                        _stream(stream)), "exact_proposal_select")
