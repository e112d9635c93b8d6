"""Seeded synthetic inputs for EXACT-MPPI workloads.

Shared by the CUDA path's tests / benchmark and by the oracle-side tests.
This module only draws geometry, obstacle clouds, noise tensors and
parameter presets; it holds none of the method's arithmetic (no distance,
rollout, cost or weighting).  Every array is float32 (the library's boundary
type); the oracle widens them to float64 exactly.

Workload recipes (sizes follow the five benchmark configurations):
  * sdf_microbench   16,384 poses (xy U[-5,5]^2, heading U[-pi,pi)),
                     8,192 points U[-6,6]^2, random 32-vertex star polygon
                     (sorted angles, radii U(0.3,1.2)).
  * plain_step       diff-drive, L footprint (1.0 x 0.6 body + 0.8 x 0.3 arm),
                     N=512 points U[-4,4]^2 outside a 1.5 m disc, K=256, T=20,
                     sigma=(0.3, 0.6), lambda=1, goal 5 m ahead.
  * forklift         3-rectangle cover (1.8 x 1.0 body + two 1.2 x 0.15 forks),
                     Ackermann L=1.4, |delta|<=0.6, K=2048, T=40, N=4096 points
                     from two jittered aisle walls 1.6 m apart plus 30 boxes.
  * batched          64 heterogeneous scenes (model, polygon 4..64 vertices,
                     N log-uniform 200..20000, K in {256,1024,4096}, T 20..50,
                     10..60 disc/box obstacles edge-sampled every 0.02 m).
"""
from __future__ import annotations

import math

import numpy as np

POLYGON, RECTS = 0, 1
DIFF, ACKERMANN, OMNI, SPIN, PARALLEL = 0, 1, 2, 3, 4
NU = {DIFF: 2, ACKERMANN: 2, OMNI: 3, SPIN: 1, PARALLEL: 1}


def rng(seed) -> np.random.Generator:
    return np.random.default_rng(seed)


# ----------------------------------------------------------------- footprints
def l_footprint() -> np.ndarray:
    """Concave 6-vertex L: 1.0 x 0.6 body with a 0.8 x 0.3 side arm (CCW)."""
    return np.array([(-0.5, -0.3), (0.5, -0.3), (0.5, 1.1), (0.2, 1.1), (0.2, 0.3), (-0.5, 0.3)],
                    dtype=np.float32)


def l_footprint_gap() -> np.ndarray:
    """L shape of the omni gap scenario: 2.0 m x 2.0 m overall, 0.4 m legs (CCW)."""
    return np.array([(0.0, 0.0), (2.0, 0.0), (2.0, 0.4), (0.4, 0.4), (0.4, 2.0), (0.0, 2.0)],
                    dtype=np.float32)


def star_polygon(g: np.random.Generator, n: int, r_lo: float, r_hi: float) -> np.ndarray:
    """Random simple star-shaped polygon around the origin: n sorted distinct
    angles with every gap < pi, radii uniform in (r_lo, r_hi); CCW order."""
    while True:
        ang = np.sort(g.uniform(0.0, 2.0 * math.pi, n))
        gaps = np.diff(np.concatenate([ang, ang[:1] + 2.0 * math.pi]))
        if gaps.max() < math.pi and gaps.min() > 1e-3:
            break
    r = g.uniform(r_lo, r_hi, n)
    return np.stack([r * np.cos(ang), r * np.sin(ang)], axis=1).astype(np.float32)


def forklift_rects() -> np.ndarray:
    """Rectangle cover (cx, cy, sx, sy): 1.8 x 1.0 body and two 1.2 x 0.15 forks."""
    return np.array([(0.0, 0.0, 0.9, 0.5), (1.5, 0.35, 0.6, 0.075), (1.5, -0.35, 0.6, 0.075)],
                    dtype=np.float32)


def rectilinear_shapes() -> dict:
    """The L-, T- and F-shaped rectilinear bodies of the rectangle-cover vs
    polygon comparison (Experiment 1; the paper gives no dimensions, so these
    are readings).  name -> (polygon outline (CCW), rectangle cover (cx, cy,
    sx, sy) of the same set; covering boxes overlap, never just touch), in float64."""
    L_poly = np.array([(-0.5, -0.3), (0.5, -0.3), (0.5, 1.1), (0.2, 1.1), (0.2, 0.3), (-0.5, 0.3)])
    L_rects = np.array([(0.0, 0.0, 0.5, 0.3), (0.35, 0.55, 0.15, 0.55)], dtype=np.float64)
    T_poly = np.array([(-0.15, -0.6), (0.15, -0.6), (0.15, 0.3), (0.6, 0.3), (0.6, 0.6), (-0.6, 0.6),
                       (-0.6, 0.3), (-0.15, 0.3)], dtype=np.float64)
    T_rects = np.array([(0.0, 0.45, 0.6, 0.15), (0.0, -0.075, 0.15, 0.525)], dtype=np.float64)
    F_poly = np.array([(-0.5, -0.6), (-0.2, -0.6), (-0.2, -0.1), (0.2, -0.1), (0.2, 0.15), (-0.2, 0.15),
                       (-0.2, 0.35), (0.4, 0.35), (0.4, 0.6), (-0.5, 0.6)], dtype=np.float64)
    F_rects = np.array([(-0.35, 0.0, 0.15, 0.6), (-0.05, 0.475, 0.45, 0.125), (-0.15, 0.025, 0.35, 0.125)],
                       dtype=np.float64)
    return {"L": (L_poly, L_rects), "T": (T_poly, T_rects), "F": (F_poly, F_rects)}


# ----------------------------------------------------------------- obstacles
def uniform_points(g, n, lo, hi) -> np.ndarray:
    return g.uniform(lo, hi, size=(n, 2)).astype(np.float32)


def ring_excluded_points(g, n, half, r_excl) -> np.ndarray:
    out = np.empty((0, 2))
    while out.shape[0] < n:
        p = g.uniform(-half, half, size=(2 * n, 2))
        p = p[np.hypot(p[:, 0], p[:, 1]) >= r_excl]
        out = np.concatenate([out, p])
    return out[:n].astype(np.float32)


def box_edge_points(cx, cy, w, h, spacing) -> np.ndarray:
    """Points every `spacing` metres along the perimeter of an axis-aligned box."""
    pts = []
    for (x0, y0, x1, y1) in ((cx - w / 2, cy - h / 2, cx + w / 2, cy - h / 2),
                             (cx + w / 2, cy - h / 2, cx + w / 2, cy + h / 2),
                             (cx + w / 2, cy + h / 2, cx - w / 2, cy + h / 2),
                             (cx - w / 2, cy + h / 2, cx - w / 2, cy - h / 2)):
        L = math.hypot(x1 - x0, y1 - y0)
        k = max(1, int(round(L / spacing)))
        t = np.arange(k) / k
        pts.append(np.stack([x0 + t * (x1 - x0), y0 + t * (y1 - y0)], axis=1))
    return np.concatenate(pts)


def disc_edge_points(cx, cy, r, spacing) -> np.ndarray:
    k = max(3, int(round(2 * math.pi * r / spacing)))
    a = np.arange(k) * (2 * math.pi / k)
    return np.stack([cx + r * np.cos(a), cy + r * np.sin(a)], axis=1)


def fit_budget(g, pts, n_budget):
    """Uniform subsample to a fixed budget, or pad (with zeros) plus a validity mask."""
    pts = np.asarray(pts, dtype=np.float64)
    if pts.shape[0] >= n_budget:
        idx = np.sort(g.choice(pts.shape[0], n_budget, replace=False))
        return pts[idx].astype(np.float32), np.ones(n_budget, dtype=np.uint8)
    out = np.zeros((n_budget, 2), dtype=np.float32)
    out[:pts.shape[0]] = pts
    mask = np.zeros(n_budget, dtype=np.uint8)
    mask[:pts.shape[0]] = 1
    return out, mask


# ----------------------------------------------------------------- MPPI params
def mppi_params(K, T, model, **over) -> dict:
    """Algorithm 1 parameters with the default cost weights of the readings."""
    p = dict(K=K, T=T, nu=NU[model], model=model, dt=0.1, d_safe=0.05, w_coll=1000.0,
             w_rep=100.0, w_inf=1.0e4, w_goal=1.0, w_term=5.0, w_ctrl=0.01, wheelbase=1.0,
             u_min=[-1e30, -1e30, -1e30], u_max=[1e30, 1e30, 1e30], clamp=0, state_offset=1)
    p["lambda"] = 1.0
    p.update(over)
    return p


def noise(g, K, T, sigma) -> np.ndarray:
    sigma = np.asarray(sigma, dtype=np.float64)
    return (g.standard_normal((K, T, sigma.size)) * sigma).astype(np.float32)


# ----------------------------------------------------------------- workloads
def sdf_microbench(seed=0, n_poses=16384, n_points=8192, n_vertices=32) -> dict:
    g = rng(seed)
    poses = np.empty((n_poses, 3), dtype=np.float32)
    poses[:, :2] = g.uniform(-5.0, 5.0, size=(n_poses, 2))
    poses[:, 2] = g.uniform(-math.pi, math.pi, size=n_poses)
    return dict(poses=poses, points=uniform_points(g, n_points, -6.0, 6.0),
                kind=POLYGON, fp=star_polygon(g, n_vertices, 0.3, 1.2))


def plain_step(seed=0, K=256, T=20, N=512) -> dict:
    g = rng(seed)
    return dict(q0=np.zeros(3, dtype=np.float32),
                cloud=ring_excluded_points(g, N, 4.0, 1.5), mask=None,
                waypoints=np.array([[5.0, 0.0]], dtype=np.float32),
                U=np.zeros((T, 2), dtype=np.float32),
                eps=noise(g, K, T, (0.3, 0.6)),
                kind=POLYGON, fp=l_footprint(), params=mppi_params(K, T, DIFF))


def paper_budget(seed=0, K=1000, T=50, N=100) -> dict:
    """The paper's navigation sampling budget (Sec. V-A: K = 1000, T = 50,
    dt = 0.1, N = 100 obstacle points) with the 8-vertex T-shaped body of the
    rectangle-cover comparison; diff-drive, points uniform in [-4, 4]^2
    outside a 1.5 m disc, goal 5 m ahead, the plain step's noise."""
    g = rng(seed)
    return dict(q0=np.zeros(3, dtype=np.float32),
                cloud=ring_excluded_points(g, N, 4.0, 1.5), mask=None,
                waypoints=np.array([[5.0, 0.0]], dtype=np.float32),
                U=np.zeros((T, 2), dtype=np.float32),
                eps=noise(g, K, T, (0.3, 0.6)),
                kind=POLYGON, fp=rectilinear_shapes()["T"][0].astype(np.float32), params=mppi_params(K, T, DIFF))


def forklift(seed=0, K=2048, T=40, N=4096) -> dict:
    g = rng(seed)
    xs = np.arange(-2.0, 14.0, 0.01)
    walls = []
    for y in (-0.8, 0.8):
        w = np.stack([xs, np.full_like(xs, y)], axis=1)
        walls.append(w + g.normal(0.0, 0.02, size=w.shape))
    boxes = []
    for _ in range(30):
        side = g.uniform(0.3, 0.8, size=2)
        cx = g.uniform(2.0, 14.0)
        cy = g.choice([-1.0, 1.0]) * (1.2 + side[1] / 2 + g.uniform(0.0, 2.0))
        boxes.append(box_edge_points(cx, cy, side[0], side[1], 0.01))
    cloud, mask = fit_budget(g, np.concatenate(walls + boxes), N)
    p = mppi_params(K, T, ACKERMANN, wheelbase=1.4, clamp=1,
                    u_min=[-1e30, -0.6, -1e30], u_max=[1e30, 0.6, 1e30])
    return dict(q0=np.zeros(3, dtype=np.float32), cloud=cloud, mask=mask,
                waypoints=np.array([[5.0, 0.0]], dtype=np.float32),
                U=np.zeros((T, 2), dtype=np.float32), eps=noise(g, K, T, (0.3, 0.2)),
                kind=RECTS, fp=forklift_rects(), params=p)


def random_scene(g, model, E, N, K, T, n_obst=None) -> dict:
    """One heterogeneous scene: star polygon with E vertices, disc/box obstacles
    edge-sampled every 0.02 m outside a clear disc, fitted to a budget of N."""
    fp = star_polygon(g, E, 0.2, 1.0)
    n_obst = int(g.integers(10, 61)) if n_obst is None else n_obst
    pts = []
    for _ in range(n_obst):
        r = g.uniform(1.5, 8.0)
        a = g.uniform(-math.pi, math.pi)
        cx, cy = r * math.cos(a), r * math.sin(a)
        if g.random() < 0.5:
            pts.append(disc_edge_points(cx, cy, g.uniform(0.1, 0.5), 0.02))
        else:
            pts.append(box_edge_points(cx, cy, g.uniform(0.2, 1.0), g.uniform(0.2, 1.0), 0.02))
    cloud, mask = fit_budget(g, np.concatenate(pts), N)
    sigma = {DIFF: (0.3, 0.6), ACKERMANN: (0.3, 0.2), OMNI: (0.3, 0.3, 0.6)}[model]
    extra = {}
    if model == ACKERMANN:
        extra = dict(wheelbase=1.0, clamp=1, u_min=[-1e30, -0.6, -1e30], u_max=[1e30, 0.6, 1e30])
    goal = np.array([[g.uniform(3.0, 6.0), g.uniform(-2.0, 2.0)]], dtype=np.float32)
    return dict(q0=np.zeros(3, dtype=np.float32), cloud=cloud, mask=mask, waypoints=goal,
                U=np.zeros((T, NU[model]), dtype=np.float32), eps=noise(g, K, T, sigma),
                kind=POLYGON, fp=fp, params=mppi_params(K, T, model, **extra))


def batched(seed=0, n_scenes=64, scale=1.0) -> list:
    """64 heterogeneous scenes; `scale` < 1 shrinks N and K for small test cases."""
    g = rng(seed)
    scenes = []
    for _ in range(n_scenes):
        model = int(g.choice([DIFF, ACKERMANN, OMNI]))
        E = int(g.integers(4, 65))
        N = int(round(math.exp(g.uniform(math.log(200), math.log(20000))) * scale))
        K = int(g.choice([256, 1024, 4096]) * scale)
        T = int(g.integers(20, 51))
        scenes.append(random_scene(g, model, E, max(N, 8), max(K, 4), T))
    return scenes


def ranger_footprint() -> np.ndarray:
    """Hybrid-platform footprint (reading): a 0.74 x 0.50 m chassis with a
    0.30 x 0.20 m payload overhanging the front-left corner, CCW."""
    return np.array([[-0.37, -0.25], [0.37, -0.25], [0.37, 0.25], [0.25, 0.25], [0.25, 0.45],
                     [-0.05, 0.45], [-0.05, 0.25], [-0.37, 0.25]], dtype=np.float32)


def hybrid(seed=0, K=1024, T=20, N=2048) -> list:
    """Hybrid-mode workload: one robot with three motion modes (Ackermann,
    parallel, spin) in a corridor with a side pocket and boxes; the goal lies
    beside the robot so that lateral motion is the short way.  Returns one
    scene dict per mode; they share state, cloud, mask, waypoints, footprint.
    Mode limits follow the platform table of the paper (|v| <= 1.5 m/s,
    |v_para| <= 0.6 m/s, |omega| <= 1 rad/s); the steering limit and the
    noise scales are readings."""
    g = rng(seed)
    xs = np.arange(-4.0, 4.0, 0.02)
    walls = [np.stack([xs, np.full_like(xs, -0.9)], 1), np.stack([xs[np.abs(xs) > 0.8], np.full_like(xs[np.abs(xs) > 0.8], 0.9)], 1)]
    ys = np.arange(0.9, 3.2, 0.02)
    walls += [np.stack([np.full_like(ys, -0.8), ys], 1), np.stack([np.full_like(ys, 0.8), ys], 1)]
    for _ in range(12):
        cx, cy = g.uniform(-4.0, 4.0), g.choice([-1.0, 1.0]) * g.uniform(1.6, 4.0)
        walls.append(box_edge_points(cx, cy, g.uniform(0.2, 0.6), g.uniform(0.2, 0.6), 0.02))
    pts = np.concatenate(walls)
    pts = pts + g.normal(0.0, 0.01, size=pts.shape)
    cloud, mask = fit_budget(g, pts, N)
    common = dict(q0=np.zeros(3, dtype=np.float32), cloud=cloud, mask=mask,
                  waypoints=np.array([[0.0, 2.6]], dtype=np.float32), kind=POLYGON, fp=ranger_footprint())
    modes = []
    for model, sigma, lo, hi in ((ACKERMANN, (0.4, 0.3), (-1.5, -0.6), (1.5, 0.6)),
                                 (PARALLEL, (0.3,), (-0.6,), (0.6,)),
                                 (SPIN, (0.5,), (-1.0,), (1.0,))):
        nu = NU[model]
        u_min = list(lo) + [-1e30] * (3 - nu)
        u_max = list(hi) + [1e30] * (3 - nu)
        p = mppi_params(K, T, model, wheelbase=0.5, clamp=1, u_min=u_min, u_max=u_max)
        modes.append(dict(common, U=np.zeros((T, nu), dtype=np.float32), eps=noise(g, K, T, sigma), params=p))
    return modes


def dynamic_scene(seed=0, K=1024, T=20, N=2048, n_discs=40, speed=0.5) -> dict:
    """Moving-obstacle workload for time-indexed predictions: diff-drive
    robot with the L footprint, goal 6 m ahead, 8 static boxes and n_discs
    discs of radius 0.3 m moving at `speed` m/s in random directions within
    10 m, all sampled every 0.05 m; `vel` gives every point its obstacle's
    velocity (zero for the boxes).  Fitted to N points (subsample, or zero
    padding plus mask; padded points get zero velocity)."""
    g = rng(seed)
    pts, vel = [], []
    for _ in range(8):
        c = (g.uniform(1.5, 6.0), g.uniform(-2.5, 2.5))
        b = box_edge_points(c[0], c[1], g.uniform(0.3, 1.0), g.uniform(0.3, 1.0), 0.05)
        pts.append(b)
        vel.append(np.zeros_like(b))
    for _ in range(n_discs):
        r, a = g.uniform(1.5, 10.0), g.uniform(-math.pi, math.pi)
        d = disc_edge_points(r * math.cos(a), r * math.sin(a), 0.3, 0.05)
        h = g.uniform(-math.pi, math.pi)
        pts.append(d)
        vel.append(np.tile([speed * math.cos(h), speed * math.sin(h)], (d.shape[0], 1)))
    allp, allv = np.concatenate(pts), np.concatenate(vel)
    M = allp.shape[0]
    if M >= N:
        idx = np.sort(g.choice(M, N, replace=False))
        cloud, v, mask = allp[idx], allv[idx], None
    else:
        cloud = np.zeros((N, 2)); v = np.zeros((N, 2))
        cloud[:M], v[:M] = allp, allv
        mask = np.zeros(N, np.uint8); mask[:M] = 1
    return dict(q0=np.zeros(3, dtype=np.float32), cloud=cloud.astype(np.float32), vel=v.astype(np.float32),
                mask=mask, waypoints=np.array([[6.0, 0.0]], dtype=np.float32),
                U=np.zeros((T, 2), dtype=np.float32), eps=noise(g, K, T, (0.3, 0.6)),
                kind=POLYGON, fp=l_footprint(), params=mppi_params(K, T, DIFF))
