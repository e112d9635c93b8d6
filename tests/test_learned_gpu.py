"""Parity of the learned-proposal kernels with the FP64 oracle: the polar
histogram (bin-edge ties excluded), the tensor-core MLP forward pass and
gradients (the oracle is fed the same BF16-rounded weights and inputs;
tolerance rel-L2 <= 1e-2 per tensor and cosine >= 0.999, since the GPU also
rounds the hidden activations and gradients to BF16 as GEMM operands), the
Adam step, and the proposal prepare / select kernels."""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ex():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_29663_gb300 import build
    build.build()
    import paper_2605_29663_gb300 as ex
    return ex


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _bf16(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _rel_l2(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def _cos(a, b):
    return float(np.dot(a.ravel(), b.ravel()) / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30))


@pytest.mark.parametrize("D,H,O,B", [(111, 256, 40, 300), (17, 64, 9, 70), (128, 256, 40, 1024)])
def test_forward_and_gradients_match_oracle(ex, D, H, O, B):
    g = np.random.default_rng(D + H + O + B)
    net = ex.MLP(D, H, O, max(B, 64))
    net.init_params(seed=D)
    params = net.get_params()
    W = [_bf16(w) if w.ndim == 2 else w.astype(np.float64) for w in net.unpack(params.astype(np.float64))]
    x = g.normal(0.0, 1.0, size=(B, D)).astype(np.float32)
    tgt = g.normal(0.0, 0.5, size=(B, O)).astype(np.float32)
    y = net.forward(_t(x)).cpu().numpy()
    yo = oracle.mlp_forward(W, _bf16(x))
    assert _rel_l2(y, yo) <= 1e-2 and _cos(y, yo) >= 0.999
    loss, grads = net.loss_grad(_t(x), _t(tgt))
    lo, go = oracle.mlp_loss_grad(W, _bf16(x), tgt.astype(np.float64))
    assert abs(loss.item() - lo) <= 2e-2 * lo
    gg = net.unpack(grads.cpu().numpy())
    for k, (a, b) in enumerate(zip(gg, go)):
        assert _rel_l2(a, b) <= 1e-2, (k, _rel_l2(a, b))
        assert _cos(a, b) >= 0.999, (k, _cos(a, b))


def test_adam_step_matches_oracle_and_training_reduces_loss(ex):
    import torch
    g = np.random.default_rng(3)
    net = ex.MLP(30, 64, 8, 256)
    net.init_params(seed=4)
    x = g.normal(size=(256, 30)).astype(np.float32)
    tgt = np.tanh(x[:, :8] * 0.7).astype(np.float32)
    w0 = net.get_params().astype(np.float64)
    _, grads = net.loss_grad(_t(x), _t(tgt))
    gr = grads.cpu().numpy().astype(np.float64)
    first = net.train_step(_t(x), _t(tgt), 1e-3).item()
    w1 = net.get_params().astype(np.float64)
    m = np.zeros_like(w0)
    v = np.zeros_like(w0)
    wo = w0.copy()
    oracle.adam_step(wo, gr, m, v, 1, 1e-3)
    np.testing.assert_allclose(w1, wo, rtol=0, atol=1e-6)
    for _ in range(300):
        last = net.train_step(_t(x), _t(tgt), 3e-3)
    torch.cuda.synchronize()
    assert last.item() < 0.2 * first


def test_polar_hist_matches_oracle(ex):
    g = np.random.default_rng(5)
    B, N, nb, rmax = 6, 500, 64, 10.0
    clouds = g.uniform(-12, 12, size=(B, N, 2)).astype(np.float32)
    masks = (g.random((B, N)) > 0.2).astype(np.uint8)
    poses = np.column_stack([g.uniform(-2, 2, (B, 2)), g.uniform(-math.pi, math.pi, B)]).astype(np.float32)
    got = ex.polar_hist(_t(clouds), _t(poses), nb, rmax, masks=torch_u8(masks)).cpu().numpy()
    for b in range(B):
        # drop points within 1e-5 rad of a bin edge, where float32 and float64 may bin differently
        c, s = math.cos(poses[b, 2]), math.sin(poses[b, 2])
        d = clouds[b].astype(np.float64) - poses[b, :2]
        px, py = c * d[:, 0] + s * d[:, 1], -s * d[:, 0] + c * d[:, 1]
        u = (np.arctan2(py, px) + math.pi) / (2 * math.pi) * nb
        keep = np.abs(u - np.rint(u)) > 1e-5 * nb / (2 * math.pi)
        ref = oracle.polar_hist(clouds[b][keep], poses[b], nb, rmax, mask=masks[b][keep])
        gk = ex.polar_hist(_t(clouds[b:b + 1][:, keep]), _t(poses[b:b + 1]), nb, rmax,
                           masks=torch_u8(masks[b:b + 1][:, keep])).cpu().numpy()[0]
        np.testing.assert_allclose(gk, ref, rtol=1e-6, atol=1e-6)
    assert got.shape == (B, nb) and np.all(got <= rmax)


def torch_u8(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint8)).cuda()


def test_features_prepare_select(ex):
    """The proposal kernels against the oracle's ox_proposal_features /
    _prepare / _select on the same float32 inputs: the network input within
    float32 rounding (2e-5 relative, 2e-6 absolute), the prepared candidates
    and the selection (decision and copies) bit for bit."""
    import torch
    g = np.random.default_rng(6)
    B, T, nb = 7, 20, 64
    hist = g.uniform(0, 10, (B, nb)).astype(np.float32)
    poses = np.column_stack([g.uniform(-2, 2, (B, 2)), g.uniform(-3, 3, B)]).astype(np.float32)
    goals = g.uniform(-8, 8, (B, 2)).astype(np.float32)
    goals[0] = poses[0, :2]                     # goal at the robot: zero range, bearing 0
    prev = g.normal(size=(B, 2)).astype(np.float32)
    U = g.normal(size=(B, T, 2)).astype(np.float32)
    x = ex.proposal_features(_t(hist), _t(poses), _t(goals), _t(prev), _t(U), 10.0).cpu().numpy()
    assert x.shape == (B, nb + 7 + 2 * T)
    for b in range(B):
        xo = oracle.proposal_features(hist[b], poses[b], goals[b], prev[b], U[b], 10.0)
        np.testing.assert_allclose(x[b], xo, rtol=2e-5, atol=2e-6, err_msg=f"robot {b}")
    shift = g.normal(size=(B, T, 2)).astype(np.float32)
    Up, Uq = torch.empty((B, T, 2), device="cuda"), torch.empty((B, T, 2), device="cuda")
    ex.proposal_prepare(_t(U), _t(shift), Up, Uq)
    po, qo = oracle.proposal_prepare(U, shift)
    np.testing.assert_array_equal(Up.cpu().numpy(), po.astype(np.float32))
    np.testing.assert_array_equal(Uq.cpu().numpy(), qo.astype(np.float32))
    K = 33
    cp = g.uniform(0, 10, (B, K)).astype(np.float32)
    cq = g.uniform(0, 10, (B, K)).astype(np.float32)
    cq[0] = cp[0]                               # equal best costs: plain MPPI is kept
    cq[1, 5] = cp[1].min()                      # a tie through a different sample
    cp[2, -1] = cq[2].min() - 1e-3              # decided by the last sample
    up, uq = g.normal(size=(B, 2)).astype(np.float32), g.normal(size=(B, 2)).astype(np.float32)
    Uo, uo = torch.empty((B, T, 2), device="cuda"), torch.empty((B, 2), device="cuda")
    chose = torch.empty(B, dtype=torch.int32, device="cuda")
    ex.proposal_select(_t(cp), _t(cq), Up, Uq, _t(up), _t(uq), Uo, uo, chose)
    Upn, Uqn = Up.cpu().numpy(), Uq.cpu().numpy()
    for b in range(B):
        pick, Ur, ur = oracle.proposal_select(cp[b], cq[b], Upn[b], Uqn[b], up[b], uq[b])
        assert int(chose[b].item()) == int(pick), b
        np.testing.assert_array_equal(Uo[b].cpu().numpy(), Ur.astype(np.float32))
        np.testing.assert_array_equal(uo[b].cpu().numpy(), ur.astype(np.float32))
    assert not bool(chose[0].item()) and not bool(chose[1].item()) and bool(chose[2].item())


def test_trained_proposal_gains_over_plain(ex):
    """What the trained network gains: trained on closed-loop plain MPPI data
    (reduced scale), the proposal candidate is kept (its best J~ beats plain
    MPPI's on the same noise) more often than with the untrained network, and
    in closed loop the proposal controller at K samples is not worse than
    plain MPPI at the same K on the same worlds (paired; the full-scale run
    shows the gain with significance)."""
    import torch
    from paper_2605_29663_gb300 import learned as L
    dev = torch.device("cuda", 0)
    X, Y = L.generate_dataset(torch, dev, 24576, 64, 1024, seed=101, log=None)
    net = ex.MLP(L.D_IN, 256, 2 * L.T_H, 1024)
    net.init_params(seed=5)
    untrained = ex.MLP(L.D_IN, 256, 2 * L.T_H, 1024)
    untrained.init_params(seed=5)
    hist = L.train(torch, net, X, Y, epochs=8, batch=1024, lr=1e-3, seed=3, log=None)
    assert hist[-1]["val_loss"] < hist[0]["val_loss"]
    kw = dict(max_steps=150, log=None)
    plain = L.evaluate(torch, dev, "plain", 256, 64, 20_001, **kw)
    prop = L.evaluate(torch, dev, "proposal", 256, 64, 20_001, mlp=net, **kw)
    base = L.evaluate(torch, dev, "proposal", 256, 64, 20_001, mlp=untrained, **kw)
    diff = np.array(prop["costs"]) - np.array(plain["costs"])
    ci = 1.96 * diff.std(ddof=1) / np.sqrt(diff.size)
    print(f"plain K=256 cost {plain['cost_mean']:.1f}, proposal {prop['cost_mean']:.1f} "
          f"(paired diff {diff.mean():.1f} +- {ci:.1f}), "
          f"kept: trained {prop['proposal_chosen_frac']:.3f} vs untrained {base['proposal_chosen_frac']:.3f}, "
          f"best-cost gain trained {prop['best_cost_gain_mean']:.2f} vs untrained {base['best_cost_gain_mean']:.2f}")
    assert prop["proposal_chosen_frac"] > base["proposal_chosen_frac"]
    assert prop["best_cost_gain_mean"] > base["best_cost_gain_mean"]
    assert diff.mean() < ci


def test_checkpoint_resume_is_bitwise(ex, tmp_path):
    """Training k Adam steps, saving the flat checkpoint (parameters, both
    moments, step count), and training k more gives the same losses and
    parameters, bit for bit, as a fresh network restored from the checkpoint
    and trained the same k steps."""
    g = np.random.default_rng(21)
    D, H, O, B, k = 40, 128, 12, 512, 6
    xs = [_t(g.normal(size=(B, D))) for _ in range(2 * k)]
    ts = [_t(np.tanh(g.normal(size=(B, O)))) for _ in range(2 * k)]
    a = ex.MLP(D, H, O, B)
    a.init_params(seed=9)
    for i in range(k):
        a.train_step(xs[i], ts[i], 2e-3)
    path = str(tmp_path / "proposal.ckpt")
    a.save_checkpoint(path)
    la = [a.train_step(xs[i], ts[i], 2e-3).item() for i in range(k, 2 * k)]
    b = ex.MLP(D, H, O, B)
    b.init_params(seed=1)                    # different start: everything comes from the checkpoint
    b.load_checkpoint(path)
    lb = [b.train_step(xs[i], ts[i], 2e-3).item() for i in range(k, 2 * k)]
    assert la == lb
    wa, ma, va, sa = a.get_state()
    wb, mb, vb, sb = b.get_state()
    assert sa == sb == 2 * k
    for x, y in ((wa, wb), (ma, mb), (va, vb)):
        np.testing.assert_array_equal(x, y)
    with pytest.raises(ValueError):
        ex.MLP(D, H + 1, O, B).load_checkpoint(path)
