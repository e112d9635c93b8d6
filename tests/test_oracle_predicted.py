"""Pins of the FP64 oracle's time-indexed obstacle prediction (the extension
named in Sec. V-F, constant-velocity reading): each horizon step scores the
points at o + t_h v, t_h the time of the scored state.  Checked against closed
forms of a box robot and a moving point, the static special case and the
literal-indexing switch."""
import numpy as np

import oracle
import synth


def _box(X, v=1.0, T=6, a=0.3, b=0.2, **over):
    p = synth.mppi_params(1, T, synth.DIFF, **over)
    U = np.tile([v, 0.0], (T, 1))
    return p, U, np.zeros((1, T, 2)), [[0.0, 0.0, a, b]]


def _J(x, d, T, v, goal=5.0):
    stage = np.abs(goal - x) + 0.01 * v * v + 1000.0 * (d < 0) + 100.0 * np.maximum(0.05 - d, 0) ** 2
    return stage.sum() + 5.0 * abs(goal - x[-1])


def test_point_moving_with_the_robot_keeps_its_clearance():
    """Robot and point both move at (v, 0): the body-frame point never moves,
    so every step has the initial clearance X - a."""
    X, v, T, a, dt = 1.0, 0.8, 8, 0.3, 0.1
    p, U, e, fp = _box(X, v, T, a)
    o = oracle.mppi_step(p, [0, 0, 0], [[X, 0.0]], [[5.0, 0.0]], U, e, oracle.RECTS, fp, vel=[[v, 0.0]])
    x = (np.arange(T) + 1) * v * dt
    d = np.full(T, X - a)
    np.testing.assert_allclose(o["dmin"][0], d, atol=1e-13)
    np.testing.assert_allclose(o["costs"][0], _J(x, d, T, v), rtol=1e-13)
    assert o["valid"]


def test_point_approaching_a_resting_robot():
    """U = 0: the point at (X, 0) moving at (-w, 0) is at X - w t_h at the
    scored state h (t_h = (h + 1) dt); it enters the box during the horizon."""
    X, w, T, a, dt = 1.0, 3.0, 8, 0.3, 0.1
    p, U, e, fp = _box(X, 0.0, T, a)
    o = oracle.mppi_step(p, [0, 0, 0], [[X, 0.0]], [[5.0, 0.0]], U, e, oracle.RECTS, fp, vel=[[-w, 0.0]])
    t = (np.arange(T) + 1) * dt
    px = X - w * t
    d = np.where(np.abs(px) >= a, np.abs(px) - a, np.maximum(np.abs(px) - a, -0.2))
    np.testing.assert_allclose(o["dmin"][0], d, atol=1e-13)
    np.testing.assert_allclose(o["costs"][0], _J(np.zeros(T), d, T, 0.0) + 1e4, rtol=1e-13)
    assert not o["valid"] and np.all(o["U"] == 0)


def test_literal_indexing_scores_the_current_cloud_first():
    """state_offset = 0 scores q_h at t_h = h dt: step 0 sees the observation."""
    X, w, T, a, dt = 1.0, 1.0, 5, 0.3, 0.1
    p, U, e, fp = _box(X, 0.0, T, a, state_offset=0)
    o = oracle.mppi_step(p, [0, 0, 0], [[X, 0.0]], [[5.0, 0.0]], U, e, oracle.RECTS, fp, vel=[[-w, 0.0]])
    np.testing.assert_allclose(o["dmin"][0], X - a - w * np.arange(T) * dt, atol=1e-13)


def test_zero_velocity_is_the_static_cycle():
    s = synth.dynamic_scene(4, K=48, T=10, N=300)
    args = (s["params"], s["q0"], s["cloud"], s["waypoints"], s["U"], s["eps"], s["kind"], s["fp"])
    a = oracle.mppi_step(*args, mask=s["mask"], vel=np.zeros_like(s["vel"]))
    b = oracle.mppi_step(*args, mask=s["mask"])
    for k in ("costs", "weights", "U", "U_upd", "dmin", "u_star"):
        np.testing.assert_array_equal(a[k], b[k])


def test_prediction_is_a_shift_of_the_cloud_per_step():
    """With one common velocity the prediction at step h equals the static
    cycle run on the cloud shifted by t_h v, evaluated at that step only:
    compare the per-step d_min of a K = 1 zero-noise cycle with the static
    oracle on each shifted cloud."""
    s = synth.dynamic_scene(6, K=1, T=6, N=200)
    vel = np.tile([0.4, -0.3], (s["cloud"].shape[0], 1))
    p = s["params"]
    eps = np.zeros((1, p["T"], 2))
    U = np.tile([0.5, 0.2], (p["T"], 1))
    o = oracle.mppi_step(p, s["q0"], s["cloud"], s["waypoints"], U, eps, s["kind"], s["fp"], mask=s["mask"], vel=vel)
    for h in range(p["T"]):
        t = (h + 1) * p["dt"]
        cl = s["cloud"].astype(np.float64) + t * vel
        st = oracle.mppi_step(p, s["q0"], cl, s["waypoints"], U, eps, s["kind"], s["fp"], mask=s["mask"])
        assert o["dmin"][0, h] == st["dmin"][0, h]
