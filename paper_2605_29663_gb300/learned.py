"""Learned sampling proposal for EXACT-MPPI (project extension).

A small network (proposal features -> T x 2 mean shift) moves the sampling
mean of MPPI; each cycle evaluates K samples around the shifted nominal and,
with the same noise, K samples around the plain nominal, and keeps the
candidate whose best J~ is lower, so plain MPPI is the fallback whenever the
proposal does worse.  The network is trained on the GPU (exact_mlp_* kernels)
on control sequences that plain MPPI with many samples produced in closed
loop, and compared with plain MPPI in closed-loop episodes.

Everything numeric on the hot path (histogram, features, network, MPPI
cycles, selection, collision checks) runs in the CUDA library; this module
simulates the world (moving obstacles, executing the chosen command) on the
host and orchestrates the calls.

World (one robot per environment): diff-drive robot with the concave L
footprint, goal 8-10 m ahead in a (G + 24) x 30 m arena, 8 static boxes
(0.3-1.0 m) between start and goal and 40 discs of radius 0.3 m moving at
0.5 m/s (bouncing inside
the arena, starting at least 2.5 m from the robot), all sampled as points
every 0.05 m; the robot senses the points within 6 m, fitted to a budget of
N = 2048 (uniform subsample, or zero padding plus mask).  An episode ends at
the goal (0.5 m), at a collision (exact clearance < 0) or after 250 steps.

Controller: T = 20, sampling noise sigma = (0.5 m/s, 1.0 rad/s), temperature
lambda = 0.3 (a sweep of lambda in [0.3, 50], sigma, d_safe and w_ctrl with
plain MPPI found these the settings where both K = 256 and K = 4096 do best
and K = 4096 does better than K = 256).

Guidance (the upstream module the paper assumes): at every reset a shortest
path from start to goal around the static boxes is planned on a 0.25 m grid
(8-connected, cells within 0.8 m of a box blocked); each cycle MPPI's goal
point is the point of that path LOOKAHEAD metres ahead of the path point
nearest the robot (the final goal near the end).  The discs are not planned
around: the local controller has to avoid them.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

import synth

from . import (Batch, Footprint, MLP, POLYGON, proposal_features, proposal_prepare, proposal_select, polar_hist,
               sdf_batch)

T_H = 20
N_BUDGET = 2048
NBINS = 64
R_MAX = 10.0
R_SENSE = 6.0
DT = 0.1
SIGMA = (0.5, 1.0)                   # sampling noise (v, omega)
LAMBDA = 0.3                         # MPPI temperature
U_LO, U_HI = (-1.0, -1.5), (1.5, 1.5)
GOAL_TOL = 0.5
D_IN = NBINS + 7 + 2 * T_H          # 111
GRID = 0.25                          # m, guidance planning grid
INFLATE = 0.8                        # m, blocked margin around boxes
LOOKAHEAD = 3.0                      # m along the planned path


def plan_path(boxes: list, start, goal, lo, hi) -> np.ndarray:
    """Shortest 8-connected grid path (cell centres, start to goal) that keeps
    INFLATE metres from every box (cx, cy, w, h); the straight segment when no
    path exists."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import dijkstra
    nx, ny = int(math.ceil((hi[0] - lo[0]) / GRID)), int(math.ceil((hi[1] - lo[1]) / GRID))
    xs = lo[0] + (np.arange(nx) + 0.5) * GRID
    ys = lo[1] + (np.arange(ny) + 0.5) * GRID
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    free = np.ones((nx, ny), bool)
    for cx, cy, w, h in boxes:
        dx = np.maximum(np.abs(X - cx) - w / 2, 0.0)
        dy = np.maximum(np.abs(Y - cy) - h / 2, 0.0)
        free &= np.hypot(dx, dy) > INFLATE
    cell = lambda p: (min(nx - 1, max(0, int((p[0] - lo[0]) / GRID))), min(ny - 1, max(0, int((p[1] - lo[1]) / GRID))))
    s, gcell = cell(start), cell(goal)
    free[s] = free[gcell] = True
    idx = np.arange(nx * ny).reshape(nx, ny)
    rows, cols, wts = [], [], []
    for di, dj in ((1, 0), (0, 1), (1, 1), (1, -1)):
        a = idx[max(0, -di):nx - max(0, di), max(0, -dj):ny - max(0, dj)]
        b = idx[max(0, di):nx - max(0, -di) if di <= 0 else nx, max(0, dj):ny if dj >= 0 else ny + dj]
        a, b = a.ravel(), b.ravel()
        ok = free.ravel()[a] & free.ravel()[b]
        rows.append(a[ok]); cols.append(b[ok]); wts.append(np.full(ok.sum(), math.hypot(di, dj)))
    r, c, w = np.concatenate(rows), np.concatenate(cols), np.concatenate(wts)
    G = csr_matrix((np.concatenate([w, w]), (np.concatenate([r, c]), np.concatenate([c, r]))), shape=(nx * ny,) * 2)
    _, pred = dijkstra(G, indices=idx[gcell], return_predecessors=True)
    k = idx[s]
    if k != idx[gcell] and pred[k] < 0:
        return np.array([start, goal], float)
    path = [start]
    while k != idx[gcell] and k >= 0:
        k = pred[k]
        path.append((xs[k // ny], ys[k % ny]))
    path.append(goal)
    return np.array(path, float)


def lookahead_point(path: np.ndarray, pos) -> np.ndarray:
    """The point LOOKAHEAD metres along `path` beyond its vertex nearest to pos."""
    k = int(np.argmin(np.hypot(path[:, 0] - pos[0], path[:, 1] - pos[1])))
    left = LOOKAHEAD
    while k + 1 < len(path):
        seg = path[k + 1] - path[k]
        L = math.hypot(*seg)
        if L >= left:
            return path[k] + seg * (left / L)
        left -= L
        k += 1
    return path[-1]


def mppi_params(K: int) -> dict:
    p = synth.mppi_params(K, T_H, synth.DIFF, clamp=1, u_min=[U_LO[0], U_LO[1], 0.0],
                          u_max=[U_HI[0], U_HI[1], 0.0])
    p["lambda"] = LAMBDA
    return p


class World:
    """n independent seeded environments (host-side simulation)."""

    def __init__(self, n: int, seed: int, max_steps: int = 250, n_boxes: int = 8, n_discs: int = 40):
        self.n = n
        self.n_boxes, self.n_discs = n_boxes, n_discs
        self.max_steps = max_steps
        self.seed = seed
        self.next_scene = 0
        self.pose = np.zeros((n, 3))
        self.goal = np.zeros((n, 2))
        self.prev_cmd = np.zeros((n, 2))
        self.steps = np.zeros(n, dtype=int)
        self.static = [None] * n
        self.path = [None] * n
        self.dc = np.zeros((n, n_discs, 2))
        self.dv = np.zeros((n, n_discs, 2))
        self.lo = np.zeros((n, 2))
        self.hi = np.zeros((n, 2))
        ang = np.arange(38) * (2 * math.pi / 38)
        self.disc_off = 0.3 * np.stack([np.cos(ang), np.sin(ang)], 1)
        for i in range(n):
            self.reset(i)

    def reset(self, i: int):
        g = np.random.default_rng((self.seed, self.next_scene))
        self.next_scene += 1
        G = g.uniform(8.0, 10.0)
        self.goal[i] = (G, g.uniform(-2.0, 2.0))
        self.pose[i] = (0.0, 0.0, 0.0)
        self.prev_cmd[i] = 0.0
        self.steps[i] = 0
        self.lo[i] = (-12.0, -15.0)
        self.hi[i] = (G + 12.0, 15.0)
        boxes, rects = [], []
        while len(boxes) < self.n_boxes:
            c = np.array([g.uniform(2.0, G - 0.5), g.uniform(-6.0, 6.0)])
            if np.hypot(*c) < 2.0 or np.hypot(*(c - self.goal[i])) < 1.5:
                continue
            w, h = g.uniform(0.3, 1.0, 2)
            boxes.append(synth.box_edge_points(c[0], c[1], w, h, 0.05))
            rects.append((c[0], c[1], w, h))
        self.static[i] = np.concatenate(boxes) if boxes else np.zeros((0, 2))
        self.path[i] = plan_path(rects, (0.0, 0.0), tuple(self.goal[i]), (-4.0, -9.0), (G + 4.0, 9.0))
        k = 0
        while k < self.n_discs:
            c = g.uniform(self.lo[i], self.hi[i])
            if np.hypot(*c) < 2.5:
                continue
            self.dc[i, k] = c
            a = g.uniform(-math.pi, math.pi)
            self.dv[i, k] = 0.5 * np.array([math.cos(a), math.sin(a)])
            k += 1

    def points(self, i: int, radius: float) -> np.ndarray:
        pts = np.concatenate([self.static[i], (self.dc[i][:, None, :] + self.disc_off[None]).reshape(-1, 2)])
        d = np.hypot(pts[:, 0] - self.pose[i, 0], pts[:, 1] - self.pose[i, 1])
        return pts[d <= radius]

    def clouds(self, rng) -> tuple[np.ndarray, np.ndarray]:
        cl = np.zeros((self.n, N_BUDGET, 2), np.float32)
        mk = np.zeros((self.n, N_BUDGET), np.uint8)
        for i in range(self.n):
            c, m = synth.fit_budget(rng, self.points(i, R_SENSE), N_BUDGET)
            cl[i], mk[i] = c, m
        return cl, mk

    def move(self, u: np.ndarray):
        """Execute the commands (forward Euler, diff-drive) and move the discs."""
        th = self.pose[:, 2].copy()
        self.pose[:, 0] += u[:, 0] * np.cos(th) * DT
        self.pose[:, 1] += u[:, 0] * np.sin(th) * DT
        self.pose[:, 2] += u[:, 1] * DT
        self.prev_cmd[:] = u
        self.steps += 1
        self.dc += self.dv * DT
        for ax in (0, 1):
            low = self.dc[..., ax] < self.lo[:, None, ax]
            high = self.dc[..., ax] > self.hi[:, None, ax]
            self.dv[..., ax] = np.where(low | high, -self.dv[..., ax], self.dv[..., ax])

    def goal_dist(self) -> np.ndarray:
        return np.hypot(self.pose[:, 0] - self.goal[:, 0], self.pose[:, 1] - self.goal[:, 1])

    def guidance(self) -> np.ndarray:
        """Each robot's goal point for this cycle: LOOKAHEAD metres ahead on its planned path."""
        return np.stack([lookahead_point(self.path[i], self.pose[i, :2]) for i in range(self.n)])


def executed_clearance(world: World, fp: Footprint, torch, dev) -> np.ndarray:
    """Exact signed distance of each robot's footprint at its current pose to
    the points within 3 m (exact_sdf_batch, one call per environment)."""
    out = np.empty(world.n)
    for i in range(world.n):
        pts = world.points(i, 3.0).astype(np.float32)
        if pts.shape[0] == 0:
            out[i] = np.inf
            continue
        _, m, _ = sdf_batch(torch.from_numpy(pts).to(dev), torch.from_numpy(world.pose[i:i + 1].astype(np.float32)).to(dev),
                            fp, dist=False, argmin=False)
        out[i] = float(m.item())
    return out


class _Scenes:
    """Device buffers of B scenes that share one footprint and parameter set."""

    def __init__(self, torch, dev, B: int, K: int, fp: Footprint, noise=None):
        self.B, self.K = B, K
        f = dict(dtype=torch.float32, device=dev)
        self.state = torch.zeros((B, 3), **f)
        self.cloud = torch.zeros((B, N_BUDGET, 2), **f)
        self.mask = torch.zeros((B, N_BUDGET), dtype=torch.uint8, device=dev)
        self.goal = torch.zeros((B, 1, 2), **f)
        self.U = torch.zeros((B, T_H, 2), **f)
        self.noise = noise if noise is not None else torch.zeros((B, K, T_H, 2), **f)
        self.params = mppi_params(K)
        self.batch = Batch([dict(state=self.state[b], cloud=self.cloud[b], mask=self.mask[b], waypoints=self.goal[b],
                                 U=self.U[b], noise=self.noise[b], fp=fp, params=self.params) for b in range(B)],
                           costs=True, weights=False, U_upd=True)
        self.costs_view = [o["costs"] for o in self.batch.outputs]

    def gather(self, torch):
        return (torch.stack([o["u_star"] for o in self.batch.outputs]),
                torch.stack([o["U_upd"] for o in self.batch.outputs]),
                torch.stack(self.costs_view))


class PlainController:
    def __init__(self, torch, dev, B: int, K: int, fp: Footprint):
        self.torch, self.dev = torch, dev
        self.S = _Scenes(torch, dev, B, K, fp)

    def load(self, world: World, cl, mk):
        S, t = self.S, self.torch
        S.state.copy_(t.from_numpy(world.pose.astype(np.float32)))
        S.cloud.copy_(t.from_numpy(cl))
        S.mask.copy_(t.from_numpy(mk))
        S.goal.copy_(t.from_numpy(world.guidance().astype(np.float32))[:, None, :])

    def reset_env(self, i: int):
        self.S.U[i].zero_()

    def step(self, world: World, cl, mk, gen):
        S = self.S
        self.load(world, cl, mk)
        S.noise.normal_(generator=gen)
        S.noise.mul_(self.torch.tensor(SIGMA, device=self.dev))
        S.batch.step()
        u, U_upd, costs = S.gather(self.torch)
        return u, U_upd, costs


class ProposalController:
    """K samples around U + shift and K around U (same noise); keep the better."""

    def __init__(self, torch, dev, B: int, K: int, fp: Footprint, mlp: MLP):
        self.torch, self.dev, self.B, self.mlp = torch, dev, B, mlp
        f = dict(dtype=torch.float32, device=dev)
        self.noise = torch.zeros((B, K, T_H, 2), **f)
        self.P = _Scenes(torch, dev, B, K, fp, noise=self.noise)     # proposal candidates
        self.Q = _Scenes(torch, dev, B, K, fp, noise=self.noise)     # plain candidates (fallback)
        self.U_prev = torch.zeros((B, T_H, 2), **f)
        self.prev_cmd = torch.zeros((B, 2), **f)
        self.u_out = torch.zeros((B, 2), **f)
        self.chose = torch.zeros(B, dtype=torch.int32, device=dev)
        self.hist = torch.zeros((B, NBINS), **f)
        self.x = torch.zeros((B, D_IN), **f)
        self.shift = torch.zeros((B, 2 * T_H), **f)

    def reset_env(self, i: int):
        self.U_prev[i].zero_()

    def step(self, world: World, cl, mk, gen):
        t = self.torch
        goal = t.from_numpy(world.guidance().astype(np.float32))[:, None, :]
        for S in (self.P, self.Q):
            S.state.copy_(t.from_numpy(world.pose.astype(np.float32)))
            S.cloud.copy_(t.from_numpy(cl))
            S.mask.copy_(t.from_numpy(mk))
            S.goal.copy_(goal)
        self.prev_cmd.copy_(t.from_numpy(world.prev_cmd.astype(np.float32)))
        polar_hist(self.P.cloud, self.P.state, NBINS, R_MAX, masks=self.P.mask, out=self.hist)
        proposal_features(self.hist, self.P.state, self.P.goal[:, 0, :].contiguous(), self.prev_cmd, self.U_prev,
                          R_MAX, out=self.x)
        self.mlp.forward(self.x, out=self.shift)
        proposal_prepare(self.U_prev, self.shift, self.P.U, self.Q.U)
        self.noise.normal_(generator=gen)
        self.noise.mul_(t.tensor(SIGMA, device=self.dev))
        self.P.batch.step()
        self.Q.batch.step()
        uP, _, cP = self.P.gather(t)
        uQ, _, cQ = self.Q.gather(t)
        proposal_select(cP, cQ, self.P.U, self.Q.U, uP, uQ, self.U_prev, self.u_out, self.chose)
        return self.u_out, cP, cQ


def stage_cost(world: World, u: np.ndarray, d: np.ndarray, p: dict) -> np.ndarray:
    gap = np.maximum(p["d_safe"] - d, 0.0)
    return (p["w_goal"] * world.goal_dist() + p["w_ctrl"] * (u ** 2).sum(1)
            + np.where(d < 0, p["w_coll"], 0.0) + p["w_rep"] * gap ** 2)


def collided_remainder(cost: np.ndarray, collided: np.ndarray, t_coll: np.ndarray, goal_dist: np.ndarray,
                       max_steps: int, w_goal: float) -> np.ndarray:
    """Final trajectory costs: a collided robot stays where it collided and
    pays w_goal * (its distance to the goal) for every step of the episode it
    did not run (max_steps - t_coll); other episodes keep their costs."""
    return cost + np.where(collided, w_goal * goal_dist * (max_steps - t_coll), 0.0)


def generate_dataset(torch, dev, n_samples: int, n_envs: int, K: int, seed: int, log=print):
    """Closed-loop plain MPPI (K samples) in n_envs worlds; returns device
    tensors X (n x D_IN) features and Y (n x 2T) = U_upd - U_prev."""
    fp = Footprint.polygon(synth.l_footprint())
    world = World(n_envs, seed)
    ctl = PlainController(torch, dev, n_envs, K, fp)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    rng = np.random.default_rng(seed + 1)
    f = dict(dtype=torch.float32, device=dev)
    X = torch.empty((n_samples, D_IN), **f)
    Y = torch.empty((n_samples, 2 * T_H), **f)
    hist = torch.zeros((n_envs, NBINS), **f)
    x = torch.zeros((n_envs, D_IN), **f)
    prev = torch.zeros((n_envs, 2), **f)
    k, t0, resets = 0, time.time(), 0
    while k < n_samples:
        cl, mk = world.clouds(rng)
        ctl.load(world, cl, mk)
        prev.copy_(torch.from_numpy(world.prev_cmd.astype(np.float32)))
        polar_hist(ctl.S.cloud, ctl.S.state, NBINS, R_MAX, masks=ctl.S.mask, out=hist)
        U_prev = ctl.S.U.clone()
        proposal_features(hist, ctl.S.state, ctl.S.goal[:, 0, :].contiguous(), prev, U_prev, R_MAX, out=x)
        u, U_upd, _ = ctl.step(world, cl, mk, gen)
        m = min(n_envs, n_samples - k)
        X[k:k + m] = x[:m]
        Y[k:k + m] = (U_upd - U_prev).reshape(n_envs, -1)[:m]
        k += m
        world.move(u.cpu().numpy().astype(np.float64))
        done = (world.goal_dist() < GOAL_TOL) | (world.steps >= world.max_steps)
        for i in np.nonzero(done)[0]:
            world.reset(i)
            ctl.reset_env(i)
            resets += 1
        if log and (k // n_envs) % 200 == 0:
            log(f"dataset {k}/{n_samples} samples, {resets} episodes ended, {time.time() - t0:.0f} s")
    return X, Y


def train(torch, mlp: MLP, X, Y, epochs: int, batch: int, lr: float, seed: int, log=print):
    n = X.shape[0]
    n_val = max(batch, n // 20)
    gen = torch.Generator(device=X.device)
    gen.manual_seed(seed)
    perm = torch.randperm(n, device=X.device, generator=gen)
    Xv, Yv = X[perm[:n_val]].contiguous(), Y[perm[:n_val]].contiguous()
    Xt, Yt = X[perm[n_val:]].contiguous(), Y[perm[n_val:]].contiguous()
    steps = epochs * (Xt.shape[0] // batch)
    hist = []
    loss = torch.empty(1, device=X.device)
    s = 0
    for ep in range(epochs):
        p = torch.randperm(Xt.shape[0], device=X.device, generator=gen)
        for b0 in range(0, Xt.shape[0] - batch + 1, batch):
            idx = p[b0:b0 + batch]
            a = lr * 0.5 * (1 + math.cos(math.pi * s / max(steps, 1)))
            mlp.train_step(Xt[idx].contiguous(), Yt[idx].contiguous(), a, loss=loss)
            s += 1
        vl = []
        for b0 in range(0, n_val - batch + 1, batch):
            l, _ = mlp.loss_grad(Xv[b0:b0 + batch], Yv[b0:b0 + batch])
            vl.append(l.item())
        hist.append({"epoch": ep, "train_loss": loss.item(), "val_loss": float(np.mean(vl)) if vl else None})
        if log:
            log(f"epoch {ep}: train {loss.item():.5f} val {hist[-1]['val_loss']}")
    return hist


def evaluate(torch, dev, method: str, K: int, n_episodes: int, seed: int, mlp: MLP | None = None,
             max_steps: int = 250, log=print, world_kw=None) -> dict:
    """Closed-loop episodes on seeded held-out worlds (the same worlds for
    every method).  Final trajectory cost = sum over executed steps of
    w_goal |p - g| + w_ctrl |u|^2 + phi_obs(d), d the exact clearance of the
    executed pose (a collision step pays w_coll); a collided robot stays put
    and pays the goal term for every step of the episode it did not run."""
    fp = Footprint.polygon(synth.l_footprint())
    world = World(n_episodes, seed, max_steps, **(world_kw or {}))
    if method == "plain":
        ctl = PlainController(torch, dev, n_episodes, K, fp)
    else:
        ctl = ProposalController(torch, dev, n_episodes, K, fp, mlp)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed + 7)
    rng = np.random.default_rng(seed + 8)
    p = mppi_params(K)
    active = np.ones(n_episodes, bool)
    success = np.zeros(n_episodes, bool)
    collided = np.zeros(n_episodes, bool)
    t_goal = np.full(n_episodes, max_steps)
    t_coll = np.full(n_episodes, max_steps)
    cost = np.zeros(n_episodes)
    chose = []
    best_gap = []      # per active step: min J~ of the plain candidate - min J~ of the kept one
    gpu_ms = 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for step in range(max_steps):
        cl, mk = world.clouds(rng)
        e0.record()
        out = ctl.step(world, cl, mk, gen)
        e1.record()
        torch.cuda.synchronize()
        gpu_ms += e0.elapsed_time(e1)
        u = out[0].cpu().numpy().astype(np.float64)
        if method != "plain" and active.any():
            chose.append(ctl.chose.cpu().numpy()[active].mean())
            mp = out[1].min(1).values.cpu().numpy()[active]
            mq = out[2].min(1).values.cpu().numpy()[active]
            best_gap.append(float(np.mean(mq - np.minimum(mp, mq))))
        u[~active] = 0.0
        world.move(u)
        d = executed_clearance(world, fp, torch, dev)
        c = stage_cost(world, u, d, p)
        cost += np.where(active, c, 0.0)
        newly_coll = active & (d < 0)
        collided |= newly_coll
        t_coll = np.where(newly_coll, step + 1, t_coll)
        reached = active & (world.goal_dist() < GOAL_TOL)
        success |= reached
        t_goal = np.where(reached, step + 1, t_goal)
        active &= ~(newly_coll | reached)
        if not active.any():
            break
    cost = collided_remainder(cost, collided, t_coll, world.goal_dist(), max_steps, p["w_goal"])
    ci = 1.96 * cost.std(ddof=1) / math.sqrt(n_episodes)
    progress = np.hypot(world.goal[:, 0], world.goal[:, 1]) - world.goal_dist()
    res = {"method": method, "K": K, "episodes": n_episodes, "cost_mean": float(cost.mean()), "cost_ci95": float(ci),
           "progress_mean_m": float(progress.mean()),
           "success_rate": float(success.mean()), "collision_rate": float(collided.mean()),
           "steps_to_goal_mean": float(t_goal[success].mean()) if success.any() else None,
           "gpu_ms_per_step": gpu_ms / (step + 1), "costs": cost.tolist()}
    if chose:
        res["proposal_chosen_frac"] = float(np.mean(chose))
        res["best_cost_gain_mean"] = float(np.mean(best_gap))
    if log:
        log(f"{method} K={K}: cost {res['cost_mean']:.1f} +- {ci:.1f}, progress {res['progress_mean_m']:.2f} m, "
            f"success {res['success_rate']:.2f}, "
            f"collisions {res['collision_rate']:.2f}, {res['gpu_ms_per_step']:.2f} ms/step")
    return res


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser(description="train and evaluate the learned sampling proposal")
    ap.add_argument("--samples", type=int, default=200000)
    ap.add_argument("--envs", type=int, default=64)
    ap.add_argument("--teacher-k", type=int, default=4096)
    ap.add_argument("--k", type=int, default=256)
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--episodes", type=int, default=100)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default="learned.json")
    a = ap.parse_args(argv)
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    t0 = time.time()
    X, Y = generate_dataset(torch, dev, a.samples, a.envs, a.teacher_k, a.seed)
    t_data = time.time() - t0
    mlp = MLP(D_IN, 256, 2 * T_H, max(a.batch, a.episodes))
    mlp.init_params(a.seed)
    t0 = time.time()
    hist = train(torch, mlp, X, Y, a.epochs, a.batch, a.lr, a.seed)
    t_train = time.time() - t0
    eval_seed = 10_000 + a.seed          # held-out worlds
    res = [evaluate(torch, dev, "plain", a.teacher_k, a.episodes, eval_seed),
           evaluate(torch, dev, "plain", a.k, a.episodes, eval_seed),
           evaluate(torch, dev, "proposal", a.k, a.episodes, eval_seed, mlp=mlp)]
    out = {"dataset": {"samples": a.samples, "envs": a.envs, "teacher_K": a.teacher_k, "seconds": t_data},
           "training": {"epochs": a.epochs, "batch": a.batch, "lr": a.lr, "seconds": t_train, "history": hist},
           "evaluation": [{k: v for k, v in r.items() if k != "costs"} for r in res],
           "costs": {f"{r['method']}_K{r['K']}": r["costs"] for r in res}}
    os.makedirs(os.path.dirname(a.out) or ".", exist_ok=True)
    with open(a.out, "w") as f:
        json.dump(out, f)
    mlp.save_checkpoint(os.path.splitext(a.out)[0] + ".ckpt")   # parameters, Adam moments and step
    print(json.dumps(out["evaluation"]))


if __name__ == "__main__":
    main()
