"""FP64 CPU oracle for EXACT-MPPI (arXiv 2605.29663) -- test infrastructure.

This package is the parity reference for the CUDA library and nothing else.
Only the test suite, the smoke check and the CPU-baseline leg of the
benchmark may import it; the product path never does.  It shares no code with
the CUDA sources.  ``exact_oracle.c`` holds every function of the method in
plain double precision (each citing its section / equation / algorithm); this
module builds it with gcc and wraps it with ctypes and numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "exact_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

POLYGON, RECTS = 0, 1
DIFF, ACKERMANN, OMNI, SPIN, PARALLEL = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FP contraction) and return the .so path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fopenmp", "-ffp-contract=off",
           "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            D, I, L = ctypes.c_double, ctypes.c_int, ctypes.c_int64
            P = ctypes.c_void_p
            _lib.ox_sdf_box.restype = D
            _lib.ox_sdf_box.argtypes = [D] * 6
            _lib.ox_seg_dist.restype = D
            _lib.ox_seg_dist.argtypes = [D] * 6
            _lib.ox_sdf_points.argtypes = [P, L, I, P, I, P]
            _lib.ox_inside_points.argtypes = [P, L, P, I, P]
            _lib.ox_sdf_batch.argtypes = [P, P, I, P, I, I, P, I, P, P, P]
            _lib.ox_rollout.argtypes = [I, D, P, P, I, I, D, P]
            _lib.ox_mppi_step.restype = I
            _lib.ox_mppi_step.argtypes = [P, P, P, P, P, I, P, I, P, P, I, P, I,
                                          P, P, P, P, P, P, P, P, P, D]
            _lib.ox_hybrid_select.restype = I
            _lib.ox_hybrid_select.argtypes = [I, P, P, D, I, P, P, P]
            _lib.ox_polar_hist.argtypes = [P, P, I, D, D, D, I, D, P]
            _lib.ox_proposal_features.argtypes = [P, I, D, D, D, D, D, D, P, P, I, P]
            _lib.ox_proposal_prepare.argtypes = [P, P, L, P, P]
            _lib.ox_proposal_select.restype = I
            _lib.ox_proposal_select.argtypes = [P, P, I, P, P, P, P, I, I, P, P]
            _lib.ox_mlp_forward.argtypes = [P] * 6 + [I, I, I, P, I, P]
            _lib.ox_mlp_loss_grad.restype = D
            _lib.ox_mlp_loss_grad.argtypes = [P] * 6 + [I, I, I, P, P, I] + [P] * 6
            _lib.ox_adam_step.argtypes = [P, P, P, P, L, I, D, D, D, D]
            _lib.ox_max_threads.restype = I
            _lib.ox_set_threads.argtypes = [I]
            _lib.ox_goal_dist.restype = D
            _lib.ox_goal_dist.argtypes = [D, D, P, I]
            _lib.ox_phi_obs.restype = D
            _lib.ox_phi_obs.argtypes = [D, D, D, D]
        return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _mask(mask, n):
    if mask is None:
        return None
    m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8).reshape(n))
    return m


def max_threads() -> int:
    return lib().ox_max_threads()


def set_threads(n: int) -> None:
    lib().ox_set_threads(int(n))


def sdf_points(pts, kind: int, fp) -> np.ndarray:
    """Signed distance of body-frame points (M x 2) to the footprint (Sec. IV-C)."""
    p = _f64(pts, (-1, 2))
    f = _f64(fp, (-1, 2 if kind == POLYGON else 4))
    out = np.empty(p.shape[0], dtype=np.float64)
    lib().ox_sdf_points(p.ctypes.data, p.shape[0], kind, f.ctypes.data, f.shape[0], out.ctypes.data)
    return out


def inside_points(pts, verts) -> np.ndarray:
    """Ray-casting inside flag (Sec. IV-C.3) of body-frame points."""
    p = _f64(pts, (-1, 2))
    v = _f64(verts, (-1, 2))
    out = np.empty(p.shape[0], dtype=np.int32)
    lib().ox_inside_points(p.ctypes.data, p.shape[0], v.ctypes.data, v.shape[0], out.ctypes.data)
    return out.astype(bool)


def sdf_box(px, py, cx, cy, sx, sy) -> float:
    return lib().ox_sdf_box(px, py, cx, cy, sx, sy)


def seg_dist(px, py, vx, vy, wx, wy) -> float:
    return lib().ox_seg_dist(px, py, vx, vy, wx, wy)


def sdf_batch(points, poses, kind: int, fp, mask=None, want_dist: bool = True):
    """Batched signed distances (Sec. IV-D): returns (dist P x N | None, dmin P, argmin P)."""
    pts = _f64(points, (-1, 2))
    ps = _f64(poses, (-1, 3))
    f = _f64(fp, (-1, 2 if kind == POLYGON else 4))
    N, P = pts.shape[0], ps.shape[0]
    m = _mask(mask, N)
    dist = np.empty((P, N), dtype=np.float64) if want_dist else None
    dmin = np.empty(P, dtype=np.float64)
    arg = np.empty(P, dtype=np.int64)
    lib().ox_sdf_batch(pts.ctypes.data, None if m is None else m.ctypes.data, N,
                       ps.ctypes.data, P, kind, f.ctypes.data, f.shape[0],
                       None if dist is None else dist.ctypes.data, dmin.ctypes.data, arg.ctypes.data)
    return dist, dmin, arg


def rollout(model: int, q0, u, dt: float, wheelbase: float = 1.0) -> np.ndarray:
    """Forward-Euler rollout (Sec. III-D): returns (T+1) x 3 states."""
    uu = _f64(u)
    if uu.ndim == 1:
        uu = uu.reshape(-1, 1)
    T, nu = uu.shape
    q = _f64(q0, (3,))
    out = np.empty((T + 1, 3), dtype=np.float64)
    lib().ox_rollout(model, wheelbase, q.ctypes.data, uu.ctypes.data, T, nu, dt, out.ctypes.data)
    return out


class Params(ctypes.Structure):
    """Algorithm 1 parameters (oracle-side layout)."""
    _fields_ = [("K", ctypes.c_int), ("T", ctypes.c_int), ("nu", ctypes.c_int), ("model", ctypes.c_int),
                ("dt", ctypes.c_double), ("lam", ctypes.c_double), ("d_safe", ctypes.c_double),
                ("w_coll", ctypes.c_double), ("w_rep", ctypes.c_double), ("w_inf", ctypes.c_double),
                ("w_goal", ctypes.c_double), ("w_term", ctypes.c_double), ("w_ctrl", ctypes.c_double),
                ("wheelbase", ctypes.c_double),
                ("u_min", ctypes.c_double * 3), ("u_max", ctypes.c_double * 3),
                ("clamp", ctypes.c_int), ("state_offset", ctypes.c_int)]


def make_params(d: dict) -> Params:
    p = Params()
    for k in ("K", "T", "nu", "model", "clamp", "state_offset"):
        setattr(p, k, int(d[k]))
    for k in ("dt", "d_safe", "w_coll", "w_rep", "w_inf", "w_goal", "w_term", "w_ctrl", "wheelbase"):
        setattr(p, k, float(d[k]))
    p.lam = float(d["lambda"])
    for j in range(3):
        p.u_min[j] = float(d["u_min"][j])
        p.u_max[j] = float(d["u_max"][j])
    return p


def mppi_step(params: dict, q0, cloud, waypoints, U, eps, kind: int, fp, mask=None,
              near_tol: float = 1e-5, vel=None) -> dict:
    """One control cycle of Algorithm 1.  Returns a dict with U (shifted or reset),
    U_upd (updated nominal), u_star, costs (J~), weights (omega), valid,
    dmin (K x T), dmin_nom (T), J_nom (cost of the updated nominal) and n_near
    (threshold-adjacent d_min count).  vel (N x 2): point velocities, each
    step scored against the predicted points o + t_h v."""
    P = make_params(params)
    K, T, nu = P.K, P.T, P.nu
    pts = _f64(cloud, (-1, 2))
    N = pts.shape[0]
    m = _mask(mask, N)
    v = None if vel is None else _f64(vel, (N, 2))
    wp = _f64(waypoints, (-1, 2))
    Uio = _f64(U, (T, nu)).copy()
    e = _f64(eps, (K, T, nu))
    f = _f64(fp, (-1, 2 if kind == POLYGON else 4))
    q = _f64(q0, (3,))
    u_star = np.zeros(nu)
    costs = np.empty(K)
    weights = np.empty(K)
    valid = ctypes.c_int(0)
    U_upd = np.empty((T, nu))
    dmin = np.empty((K, T))
    dmin_nom = np.empty(T)
    J_nom = ctypes.c_double(0.0)
    n_near = ctypes.c_int(0)
    rc = lib().ox_mppi_step(ctypes.byref(P), q.ctypes.data, pts.ctypes.data,
                            None if v is None else v.ctypes.data,
                            None if m is None else m.ctypes.data, N,
                            wp.ctypes.data, wp.shape[0], Uio.ctypes.data, e.ctypes.data,
                            kind, f.ctypes.data, f.shape[0],
                            u_star.ctypes.data, costs.ctypes.data, weights.ctypes.data,
                            ctypes.addressof(valid), U_upd.ctypes.data, dmin.ctypes.data,
                            dmin_nom.ctypes.data, ctypes.addressof(J_nom), ctypes.addressof(n_near), near_tol)
    if rc != 0:
        raise ValueError("oracle mppi_step rejected its arguments")
    return dict(U=Uio, U_upd=U_upd, u_star=u_star, costs=costs, weights=weights,
                valid=bool(valid.value), dmin=dmin, dmin_nom=dmin_nom, J_nom=float(J_nom.value),
                n_near=int(n_near.value))


def hybrid_select(J, valid, lambda_switch: float, tau_max: int, m_prev: int, tau: int):
    """Mode selection of Algorithm 2 (steps 1-2) from per-mode nominal costs and
    validation flags.  Returns (m_star or -1 for a safe stop, m_prev', tau', Jbar)."""
    Jd = _f64(J).reshape(-1)
    M = Jd.size
    v = np.ascontiguousarray(np.asarray(valid, dtype=np.int32).reshape(M))
    mp = ctypes.c_int(int(m_prev))
    tc = ctypes.c_int(int(tau))
    Jbar = np.empty(M)
    ms = lib().ox_hybrid_select(M, Jd.ctypes.data, v.ctypes.data, float(lambda_switch), int(tau_max),
                                ctypes.addressof(mp), ctypes.addressof(tc), Jbar.ctypes.data)
    return int(ms), int(mp.value), int(tc.value), Jbar


def hybrid_step(modes, hp: dict, m_prev: int, tau: int, near_tol: float = 1e-5) -> dict:
    """One hybrid-mode cycle (Algorithm 2, steps 1-2): Algorithm 1 per mode
    (each mode dict holds params, q0, cloud, mask, waypoints, U, eps, kind, fp;
    its U is advanced in place), then the selection.  u is the chosen mode's
    first command (zero padded to 3; zero on a safe stop)."""
    outs = []
    for md in modes:
        o = mppi_step(md["params"], md["q0"], md["cloud"], md["waypoints"], md["U"], md["eps"], md["kind"],
                      md["fp"], mask=md.get("mask"), near_tol=near_tol, vel=md.get("vel"))
        md["U"] = o["U"]
        outs.append(o)
    J = [o["J_nom"] for o in outs]
    valid = [o["valid"] for o in outs]
    ms, mp, tc, Jbar = hybrid_select(J, valid, hp["lambda_switch"], hp["cool_max"], m_prev, tau)
    u = np.zeros(3)
    if ms >= 0:
        us = outs[ms]["u_star"]
        u[:us.size] = us
    return dict(mode=mp, tau=tc, stopped=ms < 0, u=u, Jbar=Jbar, J=np.array(J), valid=np.array(valid),
                modes=outs)


def goal_dist(x, y, waypoints) -> float:
    wp = _f64(waypoints, (-1, 2))
    return lib().ox_goal_dist(x, y, wp.ctypes.data, wp.shape[0])


def phi_obs(d, d_safe, w_coll, w_rep) -> float:
    return lib().ox_phi_obs(d, d_safe, w_coll, w_rep)


def polar_hist(points, pose, nbins: int = 64, r_max: float = 10.0, mask=None) -> np.ndarray:
    """Polar nearest-range histogram in the robot frame (proposal feature)."""
    pts = _f64(points, (-1, 2))
    m = _mask(mask, pts.shape[0])
    out = np.empty(nbins)
    x, y, th = (float(v) for v in pose)
    lib().ox_polar_hist(pts.ctypes.data, None if m is None else m.ctypes.data, pts.shape[0],
                        x, y, th, nbins, r_max, out.ctypes.data)
    return out


def proposal_features(hist, pose, goal, prev_cmd, U_prev, r_max: float = 10.0) -> np.ndarray:
    """Network input of one robot: [hist / r_max, goal in the robot frame /
    r_max, previous command, |goal| / r_max, cos and sin of the goal bearing,
    previous nominal U (T x 2)]."""
    h = _f64(hist, (-1,))
    U = _f64(U_prev, (-1, 2))
    pc = _f64(prev_cmd, (2,))
    out = np.empty(h.size + 7 + 2 * U.shape[0])
    x, y, th = (float(v) for v in pose)
    lib().ox_proposal_features(h.ctypes.data, h.size, r_max, x, y, th, float(goal[0]), float(goal[1]),
                               pc.ctypes.data, U.ctypes.data, U.shape[0], out.ctypes.data)
    return out


def proposal_prepare(U_prev, shift):
    """(U_prev + shift, U_prev) as float64 arrays of U_prev's shape."""
    U = _f64(U_prev)
    sh = _f64(shift, U.shape)
    a, b = np.empty_like(U), np.empty_like(U)
    lib().ox_proposal_prepare(U.ctypes.data, sh.ctypes.data, U.size, a.ctypes.data, b.ctypes.data)
    return a, b


def proposal_select(costs_prop, costs_plain, U_prop, U_plain, u_prop, u_plain):
    """One robot: (kept proposal?, U_out, u_out) -- the proposal candidate is
    kept only when its best cost is strictly lower than plain MPPI's."""
    cp, cq = _f64(costs_prop, (-1,)), _f64(costs_plain, (-1,))
    assert cp.size == cq.size
    Up, Uq = _f64(U_prop), _f64(U_plain, np.shape(U_prop))
    up, uq = _f64(u_prop, (-1,)), _f64(u_plain, (-1,))
    Uo, uo = np.empty_like(Up), np.empty_like(up)
    pick = lib().ox_proposal_select(cp.ctypes.data, cq.ctypes.data, cp.size, Up.ctypes.data, Uq.ctypes.data,
                                    up.ctypes.data, uq.ctypes.data, Up.size, up.size, Uo.ctypes.data,
                                    uo.ctypes.data)
    return bool(pick), Uo, uo


def mlp_forward(W, x) -> np.ndarray:
    """W = (W1, b1, W2, b2, W3, b3) with W1 H x D, W2 H x H, W3 O x H."""
    W = [_f64(w) for w in W]
    H, D = W[0].shape
    O = W[4].shape[0]
    xx = _f64(x, (-1, D))
    y = np.empty((xx.shape[0], O))
    lib().ox_mlp_forward(*[w.ctypes.data for w in W], D, H, O, xx.ctypes.data, xx.shape[0], y.ctypes.data)
    return y


def mlp_loss_grad(W, x, target):
    W = [_f64(w) for w in W]
    H, D = W[0].shape
    O = W[4].shape[0]
    xx = _f64(x, (-1, D))
    t = _f64(target, (-1, O))
    g = [np.empty_like(w) for w in W]
    loss = lib().ox_mlp_loss_grad(*[w.ctypes.data for w in W], D, H, O, xx.ctypes.data,
                                  t.ctypes.data, xx.shape[0], *[a.ctypes.data for a in g])
    return loss, g


def adam_step(w, g, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam step on float64 arrays w, m, v given gradient g."""
    for a in (w, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    gg = _f64(g)
    lib().ox_adam_step(w.ctypes.data, gg.ctypes.data, m.ctypes.data, v.ctypes.data, w.size, t,
                       lr, beta1, beta2, eps)
