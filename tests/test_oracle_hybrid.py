"""Pins of the FP64 oracle's hybrid-mode cycle (Sec. IV-F, Algorithm 2,
steps 1-2): the nominal cost J_m that each mode's Algorithm 1 cycle reports,
checked against closed-form positions and clearances, and the mode selection
(switch penalty, validation exclusion, safe stop, cooldown) on hand-made
cost tables whose outcome follows from the algorithm's rules."""
import math

import numpy as np
import pytest

import oracle
import synth


def _box_mode(X, v=1.0, T=6, a=0.3, b=0.2, model=synth.DIFF):
    p = synth.mppi_params(1, T, model)
    nu = p["nu"]
    U = np.zeros((T, nu))
    U[:, 0] = v
    return dict(params=p, q0=[0.0, 0.0, 0.0], cloud=[[X, 0.0]], waypoints=[[5.0, 0.0]], U=U,
                eps=np.zeros((1, T, nu)), kind=oracle.RECTS, fp=[[0.0, 0.0, a, b]])


def test_nominal_cost_closed_form_valid():
    """Zero noise, K = 1: the updated nominal is U itself; its cost is the
    stage sum over x_{h+1} = (h+1) v dt plus the terminal term."""
    X, v, T, a, dt = 1.2, 1.0, 6, 0.3, 0.1
    md = _box_mode(X, v, T, a)
    o = oracle.mppi_step(md["params"], md["q0"], md["cloud"], md["waypoints"], md["U"], md["eps"], md["kind"],
                         md["fp"])
    x = (np.arange(T) + 1) * v * dt
    d = X - x - a
    J = np.sum(np.abs(5.0 - x) + 0.01 * v * v + 100.0 * np.maximum(0.05 - d, 0) ** 2) + 5.0 * abs(5.0 - x[-1])
    assert o["valid"]
    np.testing.assert_allclose(o["J_nom"], J, rtol=1e-13)


def test_nominal_cost_closed_form_collision():
    """A point the box reaches: w_coll for every step with d < 0 and the
    repulsion term for every step with d < d_safe; the nominal fails."""
    X, v, T, a, dt = 0.62, 1.0, 6, 0.3, 0.1
    md = _box_mode(X, v, T, a)
    o = oracle.mppi_step(md["params"], md["q0"], md["cloud"], md["waypoints"], md["U"], md["eps"], md["kind"],
                         md["fp"])
    x = (np.arange(T) + 1) * v * dt
    dx = X - x
    # box SDF to a point on the x axis: outside dx - a, inside max(dx - a, -(b - 0)) = dx - a while |dx| small
    d = np.where(np.abs(dx) >= a, np.abs(dx) - a, np.maximum(np.abs(dx) - a, -0.2))
    J = np.sum(np.abs(5.0 - x) + 0.01 + 1000.0 * (d < 0) + 100.0 * np.maximum(0.05 - d, 0) ** 2) \
        + 5.0 * abs(5.0 - x[-1])
    assert not o["valid"]
    np.testing.assert_allclose(o["dmin_nom"], d, atol=1e-13)
    np.testing.assert_allclose(o["J_nom"], J, rtol=1e-13)


def test_nominal_cost_equals_sample_cost_of_the_same_sequence():
    """With K = 1 and zero noise the single sample is the nominal, so J~ of the
    sample is J_nom (+ w_inf when unsafe): two different code paths agree."""
    s = synth.plain_step(3, K=1, T=12, N=200)
    p = s["params"]
    eps = np.zeros((1, p["T"], p["nu"]))
    U = np.tile([0.4, 0.2], (p["T"], 1))
    o = oracle.mppi_step(p, s["q0"], s["cloud"], s["waypoints"], U, eps, s["kind"], s["fp"])
    chi = bool(np.any(o["dmin"][0] < p["d_safe"]))
    np.testing.assert_allclose(o["costs"][0], o["J_nom"] + p["w_inf"] * chi, rtol=1e-14)


# ----------------------------------------------------------------- selection
def test_switch_penalty_keeps_previous_mode():
    ms, mp, tau, Jbar = oracle.hybrid_select([10.0, 9.5, 12.0], [1, 1, 1], 1.0, 3, m_prev=0, tau=0)
    np.testing.assert_allclose(Jbar, [10.0, 10.5, 13.0])
    assert (ms, mp, tau) == (0, 0, 0)


def test_switch_when_gain_exceeds_penalty():
    ms, mp, tau, Jbar = oracle.hybrid_select([10.0, 8.0, 12.0], [1, 1, 1], 1.0, 3, m_prev=0, tau=0)
    np.testing.assert_allclose(Jbar, [10.0, 9.0, 13.0])
    assert (ms, mp, tau) == (1, 1, 3)


def test_invalid_modes_are_excluded():
    ms, mp, tau, Jbar = oracle.hybrid_select([1.0, 8.0, 12.0], [0, 1, 1], 0.5, 3, m_prev=2, tau=0)
    assert math.isinf(Jbar[0])
    np.testing.assert_allclose(Jbar[1:], [8.5, 12.0])
    assert (ms, mp, tau) == (1, 1, 3)


def test_all_invalid_is_a_safe_stop():
    ms, mp, tau, Jbar = oracle.hybrid_select([1.0, 2.0], [0, 0], 1.0, 3, m_prev=1, tau=2)
    assert ms == -1 and (mp, tau) == (1, 2)
    assert np.all(np.isinf(Jbar))


def test_cooldown_blocks_a_switch_and_counts_down():
    ms, mp, tau, _ = oracle.hybrid_select([5.0, 10.0, 10.0], [1, 1, 1], 1.0, 3, m_prev=1, tau=3)
    assert (ms, mp, tau) == (1, 1, 2)
    ms, mp, tau, _ = oracle.hybrid_select([5.0, 10.0, 10.0], [1, 1, 1], 1.0, 3, m_prev=1, tau=1)
    assert (ms, mp, tau) == (1, 1, 0)
    ms, mp, tau, _ = oracle.hybrid_select([5.0, 10.0, 10.0], [1, 1, 1], 1.0, 3, m_prev=1, tau=0)
    assert (ms, mp, tau) == (0, 0, 3)


def test_cooldown_keeps_an_invalid_previous_mode():
    """Algorithm 2 keeps m_prev during the cooldown even when its candidate
    failed validation; that mode's first command is then the zero command."""
    ms, mp, tau, _ = oracle.hybrid_select([5.0, 1.0, 6.0], [1, 0, 1], 1.0, 3, m_prev=1, tau=2)
    assert (ms, mp, tau) == (1, 1, 1)


def test_first_cycle_has_no_previous_mode():
    ms, mp, tau, Jbar = oracle.hybrid_select([10.0, 10.0], [1, 1], 1.0, 4, m_prev=-1, tau=0)
    np.testing.assert_allclose(Jbar, [11.0, 11.0])
    assert (ms, mp, tau) == (0, 0, 4)       # equal costs: the lowest mode index
    ms, mp, tau, _ = oracle.hybrid_select([10.0, 3.0], [1, 1], 1.0, 4, m_prev=-1, tau=2)
    assert (ms, mp, tau) == (1, 1, 4)       # no mode to keep during a cooldown


def test_hybrid_step_returns_the_chosen_modes_first_command():
    """Three modes of one robot (Ackermann, parallel, spin) facing a wall
    ahead: each mode runs its own cycle; u is the first command of the mode
    with the lowest augmented nominal cost, zero padded."""
    g = np.random.default_rng(5)
    T, K = 10, 64
    pts = np.stack([np.full(60, 1.4), np.linspace(-1.5, 1.5, 60)], 1)
    modes = []
    for model, sig in ((synth.ACKERMANN, [0.3, 0.2]), (synth.PARALLEL, [0.3]), (synth.SPIN, [0.5])):
        p = synth.mppi_params(K, T, model, wheelbase=0.5)
        modes.append(dict(params=p, q0=[0.0, 0.0, 0.0], cloud=pts, waypoints=[[0.0, 3.0]],
                          U=np.zeros((T, p["nu"])), eps=g.standard_normal((K, T, p["nu"])) * sig,
                          kind=oracle.POLYGON, fp=[[-0.3, -0.2], [0.3, -0.2], [0.3, 0.2], [-0.3, 0.2]]))
    r = oracle.hybrid_step(modes, dict(lambda_switch=2.0, cool_max=3), m_prev=-1, tau=0)
    Jb = np.where(r["valid"], r["J"] + 2.0, np.inf)
    np.testing.assert_allclose(r["Jbar"], Jb)
    assert r["mode"] == int(np.argmin(Jb)) and r["tau"] == 3 and not r["stopped"]
    chosen = r["modes"][r["mode"]]["u_star"]
    np.testing.assert_allclose(r["u"][:chosen.size], chosen)
    assert np.all(r["u"][chosen.size:] == 0)
