"""Pins of the FP64 oracle's rollout, cost, weighting, update and validation
(Sec. III-D, III-E, IV-E, Algorithm 1) against closed forms, library
routines and the special cases that the MPPI update reduces to."""
import math
import os

import numpy as np
import pytest
from scipy.special import softmax

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _euler_heading_sum(theta0, a, T):
    """Closed forms of sum_{h<T} cos(theta0 + h a) and sin(...) (geometric series)."""
    if abs(a) < 1e-15:
        return T * math.cos(theta0), T * math.sin(theta0)
    z = complex(math.cos(theta0), math.sin(theta0)) * (1 - complex(math.cos(T * a), math.sin(T * a))) \
        / (1 - complex(math.cos(a), math.sin(a)))
    return z.real, z.imag


# ----------------------------------------------------------------- kinematics
def test_straight_line_and_pure_rotation():
    dt = 0.1
    q = oracle.rollout(oracle.DIFF, [1.0, -2.0, 0.3], np.tile([0.8, 0.0], (20, 1)), dt)
    h = np.arange(21)
    np.testing.assert_allclose(q[:, 0], 1.0 + h * 0.8 * dt * math.cos(0.3), atol=1e-13)
    np.testing.assert_allclose(q[:, 1], -2.0 + h * 0.8 * dt * math.sin(0.3), atol=1e-13)
    np.testing.assert_allclose(q[:, 2], 0.3, atol=0)
    q = oracle.rollout(oracle.DIFF, [0.5, 0.5, 0.0], np.tile([0.0, -0.7], (15, 1)), dt)
    np.testing.assert_allclose(q[:, :2], 0.5, atol=0)
    np.testing.assert_allclose(q[:, 2], -0.7 * dt * np.arange(16), atol=1e-14)


@pytest.mark.parametrize("model", [oracle.DIFF, oracle.ACKERMANN])
def test_constant_turn_matches_geometric_series(model):
    """Euler with the old heading: x_T = x0 + v dt sum_h cos(theta0 + h a)."""
    dt, T, v, theta0 = 0.1, 37, 1.3, -0.4
    if model == oracle.DIFF:
        w = 0.45
        u = np.tile([v, w], (T, 1))
        L = 1.0
        a = w * dt
    else:
        delta, L = 0.33, 1.4
        u = np.tile([v, delta], (T, 1))
        a = v / L * math.tan(delta) * dt
    q = oracle.rollout(model, [0.2, 0.1, theta0], u, dt, wheelbase=L)
    cs, sn = _euler_heading_sum(theta0, a, T)
    np.testing.assert_allclose(q[-1], [0.2 + v * dt * cs, 0.1 + v * dt * sn, theta0 + T * a], atol=1e-12)


def test_omni_spin_parallel():
    dt = 0.1
    q = oracle.rollout(oracle.OMNI, [0, 0, 0], np.tile([0.5, -0.25, 0.0], (10, 1)), dt)
    np.testing.assert_allclose(q[-1], [0.5, -0.25, 0.0], atol=1e-14)
    q = oracle.rollout(oracle.OMNI, [0, 0, math.pi / 2], np.tile([0.5, -0.25, 0.0], (10, 1)), dt)
    np.testing.assert_allclose(q[-1], [0.25, 0.5, math.pi / 2], atol=1e-14)  # body x = world y
    q = oracle.rollout(oracle.SPIN, [1, 2, 0], np.full((8, 1), 0.3), dt)
    np.testing.assert_allclose(q[-1], [1, 2, 0.24], atol=1e-14)
    q = oracle.rollout(oracle.PARALLEL, [0, 0, 0.0], np.full((10, 1), 0.4), dt)
    np.testing.assert_allclose(q[-1], [0.0, 0.4, 0.0], atol=1e-14)  # sideways along body y


# ----------------------------------------------------------------- cost terms
def test_phi_obs_values():
    assert oracle.phi_obs(0.2, 0.05, 1000, 100) == 0.0
    assert oracle.phi_obs(0.05, 0.05, 1000, 100) == 0.0
    assert math.isclose(oracle.phi_obs(0.03, 0.05, 1000, 100), 100 * 0.02 ** 2, rel_tol=1e-12)
    assert math.isclose(oracle.phi_obs(-0.1, 0.05, 1000, 100), 1000 + 100 * 0.15 ** 2, rel_tol=1e-12)
    assert oracle.phi_obs(math.inf, 0.05, 1000, 100) == 0.0


def test_goal_distance_point_and_polyline():
    assert oracle.goal_dist(1.0, 1.0, [[4.0, 5.0]]) == 5.0
    wp = [[0, 0], [2, 0], [2, 2]]
    assert oracle.goal_dist(1.0, -0.5, wp) == 0.5
    assert oracle.goal_dist(3.0, 1.0, wp) == 1.0
    assert math.isclose(oracle.goal_dist(3.0, 3.0, wp), math.sqrt(2))


def _box_scene(X, v=1.0, T=6, K=1, a=0.3, b=0.2, eps=None, **over):
    """Diff-drive box robot driving straight at an obstacle point (X, 0)."""
    p = synth.mppi_params(K, T, synth.DIFF, **over)
    U = np.tile([v, 0.0], (T, 1))
    e = np.zeros((K, T, 2)) if eps is None else eps
    fp = [[0.0, 0.0, a, b]]
    return p, U, e, fp


def test_single_rollout_cost_closed_form():
    """K = 1, zero noise: J from closed-form positions x_{h+1} = (h+1) v dt and
    the box clearance d_h = X - x_{h+1} - a to a point straight ahead."""
    X, v, T, a, dt = 1.2, 1.0, 6, 0.3, 0.1
    p, U, e, fp = _box_scene(X, v, T, a=a)
    res = oracle.mppi_step(p, [0, 0, 0], [[X, 0.0]], [[5.0, 0.0]], U, e, oracle.RECTS, fp)
    x = (np.arange(T) + 1) * v * dt
    d = X - x - a
    stage = 1.0 * np.abs(5.0 - x) + 0.01 * v * v
    obs = 1000.0 * (d < 0) + 100.0 * np.maximum(0.05 - d, 0) ** 2
    J = stage.sum() + obs.sum() + 5.0 * abs(5.0 - x[-1])
    chi = bool(np.any(d < 0.05))
    np.testing.assert_allclose(res["dmin"][0], d, atol=1e-13)
    np.testing.assert_allclose(res["costs"][0], J + 1e4 * chi, rtol=1e-13)
    assert res["weights"][0] == 1.0
    np.testing.assert_allclose(res["U_upd"], U, atol=0)
    # X = 1.2: the box front reaches 0.9 at h = 5 -> d = 0.3 > d_safe: valid, shifted
    assert res["valid"] and not chi
    np.testing.assert_allclose(res["u_star"], [v, 0.0])
    np.testing.assert_allclose(res["U"], U)  # constant sequence is shift-invariant


def test_validation_failure_resets():
    p, U, e, fp = _box_scene(0.75)
    res = oracle.mppi_step(p, [0, 0, 0], [[0.75, 0.0]], [[5.0, 0.0]], U, e, oracle.RECTS, fp)
    assert not res["valid"]
    assert np.all(res["u_star"] == 0) and np.all(res["U"] == 0)
    assert res["dmin_nom"].min() < 0.05
    # the obstacle inside the footprint at q_1 triggers the collision weight
    p, U, e, fp = _box_scene(0.35)
    res = oracle.mppi_step(p, [0, 0, 0], [[0.35, 0.0]], [[5.0, 0.0]], U, e, oracle.RECTS, fp)
    assert res["dmin"][0, 0] < 0 and not res["valid"]


def test_shift_repeats_last_entry():
    T = 5
    p = synth.mppi_params(1, T, synth.DIFF)
    U = np.array([[0.1 * h, -0.05 * h] for h in range(T)])
    res = oracle.mppi_step(p, [0, 0, 0], [[50.0, 50.0]], [[5.0, 0.0]], U, np.zeros((1, T, 2)),
                           oracle.RECTS, [[0, 0, 0.3, 0.2]])
    assert res["valid"]
    np.testing.assert_array_equal(res["u_star"], U[0])
    np.testing.assert_array_equal(res["U"][:-1], U[1:])
    np.testing.assert_array_equal(res["U"][-1], U[-1])


def _plain(seed=0, K=64, T=10, N=128, **over):
    s = synth.plain_step(seed, K=K, T=T, N=N)
    s["params"].update(over)
    return s


def _run(s, **kw):
    return oracle.mppi_step(s["params"], s["q0"], s["cloud"], s["waypoints"], s["U"], s["eps"],
                            s["kind"], s["fp"], mask=s["mask"], **kw)


def test_weights_are_softmax_of_costs_and_update_is_weighted_noise():
    s = _plain(1)
    res = _run(s)
    lam = s["params"]["lambda"]
    np.testing.assert_allclose(res["weights"], softmax(-res["costs"] / lam), rtol=1e-12, atol=1e-300)
    upd = np.einsum("r,rtj->tj", res["weights"], s["eps"].astype(np.float64))
    np.testing.assert_allclose(res["U_upd"] - s["U"], upd, rtol=1e-12, atol=1e-15)
    assert math.isclose(res["weights"].sum(), 1.0, rel_tol=1e-13)


def test_temperature_limits():
    s = _plain(2)
    s["params"]["lambda"] = 1e12
    res = _run(s)
    np.testing.assert_allclose(res["weights"], 1.0 / 64, rtol=1e-9)
    np.testing.assert_allclose(res["U_upd"], s["U"] + s["eps"].astype(np.float64).mean(0), atol=1e-12)
    s["params"]["lambda"] = 1e-6
    res = _run(s)
    best = int(np.argmin(res["costs"]))
    assert res["weights"][best] > 1 - 1e-12
    np.testing.assert_allclose(res["U_upd"], s["U"] + s["eps"][best], atol=1e-12)


def test_k1_and_zero_noise():
    s = _plain(3, K=1)
    res = _run(s)
    assert res["weights"][0] == 1.0
    np.testing.assert_allclose(res["U_upd"], s["U"] + s["eps"][0].astype(np.float64), atol=0)
    s = _plain(4)
    s["eps"] = np.zeros_like(s["eps"])
    res = _run(s)
    np.testing.assert_array_equal(res["U_upd"], s["U"])
    np.testing.assert_allclose(res["weights"], 1.0 / 64, rtol=1e-12)


def test_constant_cost_shift_leaves_weights():
    """Adding the same constant to every J~ leaves omega unchanged: with an
    obstacle point at the robot's origin every rollout is unsafe, so w_inf
    shifts all costs alike (and exp(-1e4) would underflow without beta)."""
    s = _plain(5, K=48, T=8)
    s["cloud"] = np.vstack([s["cloud"], [[0.0, 0.0]]]).astype(np.float32)
    s["params"]["w_inf"] = 1.0e4
    a = _run(s)
    s["params"]["w_inf"] = 0.0
    b = _run(s)
    assert np.all(a["costs"] - b["costs"] == pytest.approx(1e4, abs=1e-9))
    np.testing.assert_allclose(a["weights"], b["weights"], rtol=1e-9, atol=1e-300)
    np.testing.assert_allclose(a["U_upd"], b["U_upd"], rtol=0, atol=1e-12)


def test_unsafe_flag_adds_w_inf():
    s = _plain(6, K=32)
    res = _run(s)
    chi = (res["dmin"] < s["params"]["d_safe"]).any(axis=1)
    s2 = _plain(6, K=32)
    s2["params"]["w_inf"] = 0.0
    r2 = _run(s2)
    np.testing.assert_allclose(res["costs"] - r2["costs"], 1e4 * chi, rtol=0, atol=1e-9)


def test_clamp_limits_and_effective_noise():
    s = synth.forklift(0, K=16, T=8, N=256)
    res = _run(s)
    U = res["U_upd"]
    assert np.all(np.abs(U[:, 1]) <= 0.6 + 1e-12)
    s2 = synth.forklift(0, K=16, T=8, N=256)
    s2["eps"] = s2["eps"] * 20  # saturate steering
    r2 = _run(s2)
    assert np.all(np.abs(r2["U_upd"][:, 1]) <= 0.6 + 1e-12)


def test_state_offset_zero_scores_q0():
    s = _plain(7, K=16, T=6)
    s["params"]["state_offset"] = 0
    res = _run(s)
    assert np.all(res["dmin"][:, 0] == res["dmin"][0, 0])
    s1 = _plain(7, K=16, T=6)
    r1 = _run(s1)
    assert not np.all(r1["dmin"][:, 0] == r1["dmin"][0, 0])


def test_mask_and_empty_cloud():
    s = _plain(8, K=8, T=5, N=16)
    s["mask"] = np.zeros(16, np.uint8)
    res = _run(s)
    assert np.all(np.isinf(res["dmin"])) and res["valid"]


def test_near_threshold_report():
    p, U, e, fp = _box_scene(0.3 + 0.1 + 0.05 + 2e-6, T=1)
    res = oracle.mppi_step(p, [0, 0, 0], [[0.3 + 0.1 + 0.05 + 2e-6, 0.0]], [[5.0, 0.0]], U, e,
                           oracle.RECTS, fp)
    assert res["n_near"] == 2  # the sample and the nominal both sit 2e-6 from d_safe


def test_paper_budget_fixture():
    vals = {}
    with open(os.path.join(GOLDEN, "mppi_budget.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    assert vals["K"] * vals["T"] * vals["N"] == vals["queries"]
    assert vals["T"] * vals["dt"] == pytest.approx(5.0)
