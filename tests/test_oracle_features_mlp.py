"""Pins of the oracle's learned-proposal pieces: the polar nearest-range
histogram, the GELU MLP forward pass (against torch's CPU fp64 ops), its
analytic gradients (against central finite differences) and Adam (against
the closed form of its first step)."""
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
