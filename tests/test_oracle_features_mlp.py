"""Pins of the oracle's learned-proposal pieces: the polar nearest-range
histogram, the GELU MLP forward pass (against torch's CPU fp64 ops), its
analytic gradients (against central finite differences), Adam (against the
closed form of its first step), and the proposal-guided cycle's network input
(hand-derived goals ahead / beside / behind the robot, rigid-motion
invariance), candidate preparation and fallback selection (hand-made cost
tables with ties, numpy's minimum)."""
import math

import numpy as np
import pytest

import oracle


def test_polar_hist_bin_centres_and_empty():
    nb, rmax = 64, 10.0
    bins = np.array([0, 5, 31, 32, 63])
    ranges = np.array([1.0, 2.5, 0.7, 3.0, 9.0])
    ang = (bins + 0.5) / nb * 2 * math.pi - math.pi
    pts = np.stack([ranges * np.cos(ang), ranges * np.sin(ang)], 1)
    far = np.stack([(ranges + 1) * np.cos(ang), (ranges + 1) * np.sin(ang)], 1)  # farther, same bins
    h = oracle.polar_hist(np.vstack([far, pts]), (0.0, 0.0, 0.0), nb, rmax)
    expect = np.full(nb, rmax)
    expect[bins] = ranges
    np.testing.assert_allclose(h, expect, rtol=0, atol=1e-12)


def test_polar_hist_robot_frame_and_mask():
    # robot at (1, 1) facing +y: a world point at (1, 3) is 2 m straight ahead (bin of angle 0)
    h = oracle.polar_hist([[1.0, 3.0], [1.0, 1.5]], (1.0, 1.0, math.pi / 2), 64, 10.0,
                          mask=np.array([1, 0], np.uint8))
    assert h[32] == pytest.approx(2.0, abs=1e-12)
    assert np.sum(h < 10.0) == 1


def _tiny_net(g, D=7, H=5, O=3):
    return [g.normal(0, 0.5, (H, D)), g.normal(0, 0.1, H), g.normal(0, 0.5, (H, H)),
            g.normal(0, 0.1, H), g.normal(0, 0.5, (O, H)), g.normal(0, 0.1, O)]


def test_forward_matches_torch_fp64():
    torch = pytest.importorskip("torch")
    g = np.random.default_rng(0)
    W = _tiny_net(g, 12, 16, 4)
    x = g.normal(size=(9, 12))
    t = [torch.from_numpy(w) for w in W]
    xt = torch.from_numpy(x)
    F = torch.nn.functional
    ref = F.linear(F.gelu(F.linear(F.gelu(F.linear(xt, t[0], t[1])), t[2], t[3])), t[4], t[5])
    np.testing.assert_allclose(oracle.mlp_forward(W, x), ref.numpy(), rtol=1e-13, atol=1e-13)


def test_gradients_match_central_differences():
    g = np.random.default_rng(1)
    W = _tiny_net(g)
    x = g.normal(size=(4, 7))
    tgt = g.normal(size=(4, 3))
    loss, grads = oracle.mlp_loss_grad(W, x, tgt)
    y = oracle.mlp_forward(W, x)
    assert loss == pytest.approx(np.mean((y - tgt) ** 2), rel=1e-13)
    h = 1e-6
    for wi, (w, gw) in enumerate(zip(W, grads)):
        flat = w.reshape(-1)
        num = np.empty(flat.size)
        for k in range(flat.size):
            old = flat[k]
            flat[k] = old + h
            lp, _ = oracle.mlp_loss_grad(W, x, tgt)
            flat[k] = old - h
            lm, _ = oracle.mlp_loss_grad(W, x, tgt)
            flat[k] = old
            num[k] = (lp - lm) / (2 * h)
        np.testing.assert_allclose(gw.reshape(-1), num, rtol=1e-6, atol=1e-9, err_msg=f"tensor {wi}")


def test_adam_first_step_closed_form():
    g = np.random.default_rng(2)
    w = g.normal(size=50)
    grad = g.normal(size=50)
    m = np.zeros(50)
    v = np.zeros(50)
    w0 = w.copy()
    oracle.adam_step(w, grad, m, v, 1, 1e-3)
    # first step: m_hat = g, v_hat = g^2  ->  w -= lr g / (|g| + eps)
    np.testing.assert_allclose(w, w0 - 1e-3 * grad / (np.abs(grad) + 1e-8), rtol=1e-14, atol=1e-16)
    np.testing.assert_allclose(m, 0.1 * grad, rtol=1e-14)
    np.testing.assert_allclose(v, 0.001 * grad ** 2, rtol=1e-14)


# ---------------------------------------------------------------- proposal path
def _feat(pose, goal, T=2, hist=None, prev=(0.25, -0.5), r_max=10.0):
    hist = np.linspace(0.5, 10.0, 64) if hist is None else hist
    U = np.arange(2 * T, dtype=np.float64).reshape(T, 2) * 0.1
    return oracle.proposal_features(hist, pose, goal, prev, U, r_max), hist, U


@pytest.mark.parametrize("pose,goal,expect", [
    # facing +y from (1, 1): a goal at (1, 4) is 3 m straight ahead
    ((1.0, 1.0, math.pi / 2), (1.0, 4.0), (0.3, 0.0, 0.3, 1.0, 0.0)),
    # facing +x from the origin: (0, 2) is 2 m to the left (bearing +90 deg)
    ((0.0, 0.0, 0.0), (0.0, 2.0), (0.0, 0.2, 0.2, 0.0, 1.0)),
    # facing -x from (2, -1): (5, -1) is 3 m behind (bearing 180 deg)
    ((2.0, -1.0, math.pi), (5.0, -1.0), (-0.3, 0.0, 0.3, -1.0, 0.0)),
    # facing +x: the 3-4-5 triangle
    ((0.0, 0.0, 0.0), (3.0, 4.0), (0.3, 0.4, 0.5, 0.6, 0.8)),
    # facing -y from (0, 0): (4, 0) is to the left (rotate the world by +90 deg)
    ((0.0, 0.0, -math.pi / 2), (4.0, 0.0), (0.0, 0.4, 0.4, 0.0, 1.0)),
    # goal at the robot: zero range, bearing 0
    ((1.5, -2.0, 0.7), (1.5, -2.0), (0.0, 0.0, 0.0, 1.0, 0.0)),
])
def test_proposal_features_hand_values(pose, goal, expect):
    x, hist, U = _feat(pose, goal)
    nb = hist.size
    assert x.shape == (nb + 7 + 4,)
    np.testing.assert_allclose(x[:nb], hist / 10.0, rtol=0, atol=1e-15)
    gx, gy, rng, cb, sb = expect
    np.testing.assert_allclose(x[nb:nb + 7], [gx, gy, 0.25, -0.5, rng, cb, sb], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(x[nb + 7:], U.reshape(-1))


def test_proposal_features_rigid_motion():
    """Moving robot and goal by the same rigid motion leaves the features unchanged."""
    g = np.random.default_rng(11)
    for _ in range(20):
        pose = (g.uniform(-3, 3), g.uniform(-3, 3), g.uniform(-math.pi, math.pi))
        goal = (g.uniform(-8, 8), g.uniform(-8, 8))
        a, _, _ = _feat(pose, goal)
        phi, t = g.uniform(-math.pi, math.pi), g.uniform(-5, 5, 2)
        c, s = math.cos(phi), math.sin(phi)
        mv = lambda p: (c * p[0] - s * p[1] + t[0], s * p[0] + c * p[1] + t[1])
        b, _, _ = _feat((*mv(pose[:2]), pose[2] + phi), mv(goal))
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)


def test_proposal_prepare_closed_form():
    U = np.array([[1.0, 2.0], [3.0, 4.0]])
    shift = np.array([[0.5, -1.0], [0.0, 0.25]])
    a, b = oracle.proposal_prepare(U, shift)
    np.testing.assert_array_equal(a, [[1.5, 1.0], [3.0, 4.25]])
    np.testing.assert_array_equal(b, U)


@pytest.mark.parametrize("cp,cq,pick", [
    ([1.0, 7.0], [2.0, 3.0], True),            # proposal's best is lower
    ([3.0, 1.0, 5.0], [1.0, 4.0, 4.0], False),  # equal best costs: plain MPPI is kept
    ([9.0, 9.0, 0.5], [1.0, 1.0, 1.0], True),   # decided by the last sample
    ([4.0], [3.5], False),                      # K = 1
    ([np.inf, np.inf], [np.inf, 2.0], False),   # nothing finite on the proposal side
])
def test_proposal_select_tables(cp, cq, pick):
    Up, Uq = np.full((3, 2), 1.0), np.full((3, 2), -1.0)
    up, uq = np.array([0.5, 0.25]), np.array([-0.5, -0.25])
    got, Uo, uo = oracle.proposal_select(cp, cq, Up, Uq, up, uq)
    assert got == pick
    np.testing.assert_array_equal(Uo, Up if pick else Uq)
    np.testing.assert_array_equal(uo, up if pick else uq)


def test_proposal_select_random_against_numpy_minimum():
    g = np.random.default_rng(12)
    for _ in range(50):
        K = int(g.integers(1, 40))
        cp, cq = g.uniform(0, 10, K), g.uniform(0, 10, K)
        got, _, _ = oracle.proposal_select(cp, cq, np.zeros((2, 2)), np.ones((2, 2)), np.zeros(2), np.ones(2))
        assert got == bool(np.min(cp) < np.min(cq))
