"""Hybrid-mode EXACT-MPPI on the GPU (Sec. IV-F, Algorithm 2, steps 1-2):
the nominal cost J_m that each mode's cycle reports, and the hybrid cycle
(all modes in one batched launch set plus the device-side selection)
against the FP64 oracle over several consecutive cycles, the safe stop and
the cooldown."""
import numpy as np
import pytest

import oracle
import synth
from test_batched_gpu import _dev_scene
from test_mppi_gpu import _t, compare

pytestmark = pytest.mark.gpu

REL_J = 1e-5      # nominal cost of the same sequence: FP32 vs FP64 evaluation
ATOL_J = 5e-3     # d within 2e-5 m moves w_rep (d_safe - d)^2 by at most ~2e-4 per step
TIE = 1e-3        # relative gap below which two augmented costs count as tied


@pytest.fixture(scope="module")
def ex():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_29663_gb300 import build
    build.build()
    import paper_2605_29663_gb300 as ex
    return ex


def _oracle_cost_of(s, U):
    """Oracle cost J of the sequence U itself (K = 1, zero noise: the updated
    nominal is U), with its threshold-adjacency count."""
    p = dict(s["params"], K=1)
    o = oracle.mppi_step(p, s["q0"], s["cloud"], s["waypoints"], U, np.zeros((1,) + U.shape), s["kind"], s["fp"],
                         mask=s["mask"])
    return o["J_nom"], o["n_near"]


def _scenes():
    out = [synth.plain_step(21, K=200, T=16, N=300), synth.forklift(4, K=128, T=20, N=700)]
    out += synth.hybrid(2, K=160, T=14, N=600)
    out += synth.batched(8, n_scenes=3, scale=0.05)
    return out


def test_nominal_cost_matches_oracle(ex):
    import torch
    scenes = _scenes()
    dev = [_dev_scene(ex, s) for s in scenes]
    b = ex.Batch(dev, nom_cost=True)
    b.step()
    torch.cuda.synchronize()
    checked = 0
    for i, (s, d, o) in enumerate(zip(scenes, dev, b.outputs)):
        J_gpu = float(o["nom_cost"].cpu()[0])
        U_upd = o["U_upd"].cpu().numpy().astype(np.float64)
        J_ref, near = _oracle_cost_of(s, U_upd)
        if near:
            continue
        assert abs(J_gpu - J_ref) <= REL_J * abs(J_ref) + ATOL_J, (i, J_gpu, J_ref)
        # end to end: the oracle's own cycle on the same inputs
        full = oracle.mppi_step(s["params"], s["q0"], s["cloud"], s["waypoints"], s["U"], s["eps"], s["kind"],
                                s["fp"], mask=s["mask"])
        if full["n_near"] == 0:
            assert abs(J_gpu - full["J_nom"]) <= 1e-3 * abs(full["J_nom"]) + ATOL_J, (i, J_gpu, full["J_nom"])
        checked += 1
    assert checked >= len(scenes) - 2


def test_nominal_cost_is_repeatable_across_steps(ex):
    """The per-step keys are emptied by each cycle: a second cycle from the same
    inputs reports the same nominal cost bit for bit."""
    import torch
    s = synth.plain_step(5, K=64, T=12, N=400)
    d = _dev_scene(ex, s)
    U0 = d["U"].clone()
    b = ex.Batch([d], nom_cost=True)
    vals = []
    for _ in range(3):
        d["U"].copy_(U0)
        b.step()
        torch.cuda.synchronize()
        vals.append(float(b.outputs[0]["nom_cost"].cpu()[0]))
    assert vals[0] == vals[1] == vals[2]


def _hybrid_dev(ex, modes):
    dev = []
    fp = ex.Footprint(modes[0]["kind"], modes[0]["fp"])
    shared = dict(state=_t(modes[0]["q0"]), cloud=_t(modes[0]["cloud"]), waypoints=_t(modes[0]["waypoints"]),
                  mask=None if modes[0]["mask"] is None else _t(modes[0]["mask"]))
    for m in modes:
        dev.append(dict(shared, U=_t(m["U"]), noise=_t(m["eps"]), fp=fp, params=m["params"]))
    return dev


def _check_selection(g_state, g_u, g_Jbar, o, m_prev, tau, cool_max, modes_gpu):
    """The GPU's choice against the oracle's augmented costs: the same mode, or
    one whose oracle cost ties the minimum; the counters and the command then
    follow Algorithm 2 for the GPU's choice."""
    Jb = o["Jbar"]
    fin = np.isfinite(Jb)
    assert np.array_equal(np.isfinite(g_Jbar), fin)
    if not fin.any():
        assert g_state[2] == 1 and g_state[0] == m_prev and g_state[1] == tau
        assert np.all(g_u == 0)
        return
    assert g_state[2] == 0
    np.testing.assert_allclose(g_Jbar[fin], Jb[fin], rtol=1e-3, atol=ATOL_J)
    best = int(np.argmin(Jb))
    ms = int(g_state[0])
    if ms != o["mode"]:
        # a near-tie at the argmin (or the cooldown keeping m_prev) may pick another valid mode
        am = int(np.argmin(g_Jbar))
        assert abs(Jb[am] - Jb[best]) <= TIE * abs(Jb[best]) + ATOL_J
    expect_tau = cool_max if ms != m_prev else max(tau - 1, 0)
    assert g_state[1] == expect_tau
    us = modes_gpu[ms]["u_star"].cpu().numpy()
    np.testing.assert_array_equal(g_u[:us.size], us)
    assert np.all(g_u[us.size:] == 0)


def test_hybrid_cycles_match_oracle(ex):
    """Four consecutive hybrid cycles: each cycle starts both sides from the
    same inputs (the GPU's U_m and mode state, fresh noise); every mode's
    Algorithm 1 outputs, the augmented costs and the selection are compared."""
    import torch
    g = synth.rng(77)
    modes = synth.hybrid(3, K=256, T=16, N=1500)
    dev = _hybrid_dev(ex, modes)
    hp = dict(lambda_switch=2.0, cool_max=2)
    h = ex.Hybrid(dev, weights=True, **hp)
    compared = 0
    for cycle in range(4):
        if cycle:
            for m, d in zip(modes, dev):
                sig = np.maximum(np.abs(m["eps"]).reshape(-1, m["eps"].shape[-1]).std(axis=0), 1e-3)
                m["eps"] = synth.noise(g, m["params"]["K"], m["params"]["T"], sig)
                d["noise"].copy_(_t(m["eps"]))
        for m, d in zip(modes, dev):
            m["U"] = d["U"].cpu().numpy()
        state0 = h.mode_state.cpu().numpy().copy()
        ins = [dict(m, U=m["U"].astype(np.float64)) for m in modes]
        o = oracle.hybrid_step(ins, hp, int(state0[0]), int(state0[1]))
        h.step()
        torch.cuda.synchronize()
        if any(x["n_near"] for x in o["modes"]):
            continue
        for m, d, out, om in zip(modes, dev, h.outputs, o["modes"]):
            gr = {k: v.cpu().numpy() for k, v in out.items()}
            gr["U"] = d["U"].cpu().numpy()
            gr["valid"] = bool(gr["valid"][0])
            compare(m, gr, om, check_dmin=False)
            assert gr["valid"] == om["valid"]
        _check_selection(h.mode_state.cpu().numpy(), h.u.cpu().numpy(), h.Jbar.cpu().numpy(), o,
                         int(state0[0]), int(state0[1]), hp["cool_max"], h.outputs)
        compared += 1
    assert compared >= 3


def test_hybrid_safe_stop_keeps_mode_state(ex):
    """Obstacle points inside the footprint at q_0: every mode fails
    validation, the command is zero and [m_prev, tau] stay as they were."""
    import torch
    modes = synth.hybrid(4, K=64, T=10, N=400)
    inside = np.array([[0.0, 0.0], [0.1, 0.05], [-0.1, -0.05]], np.float32)
    for m in modes:
        m["cloud"] = np.concatenate([inside, m["cloud"][:-3]])
        if m["mask"] is not None:
            m["mask"] = np.concatenate([np.ones(3, np.uint8), m["mask"][:-3]])
    dev = _hybrid_dev(ex, modes)
    h = ex.Hybrid(dev, lambda_switch=1.0, cool_max=3, m_prev=1)
    h.mode_state.copy_(_t(np.array([1, 2, 0], np.int32)))
    h.step()
    torch.cuda.synchronize()
    st = h.mode_state.cpu().numpy()
    assert list(st) == [1, 2, 1]
    assert np.all(h.u.cpu().numpy() == 0)
    assert np.all(np.isinf(h.Jbar.cpu().numpy()))


def test_hybrid_cooldown_refuses_a_switch(ex):
    """With tau_cool > 0 the previous mode is kept even when another mode's
    augmented cost is lower, and the counter decreases by one."""
    import torch
    modes = synth.hybrid(2, K=256, T=16, N=900)
    dev = _hybrid_dev(ex, modes)
    h = ex.Hybrid(dev, lambda_switch=0.0, cool_max=3)
    h.mode_state.copy_(_t(np.array([2, 2, 0], np.int32)))   # spin-in-place was the previous mode
    ins = [dict(m, U=m["U"].astype(np.float64)) for m in modes]
    o = oracle.hybrid_step(ins, dict(lambda_switch=0.0, cool_max=3), 2, 2)
    h.step()
    torch.cuda.synchronize()
    Jb = h.Jbar.cpu().numpy()
    st = h.mode_state.cpu().numpy()
    assert np.isfinite(Jb[2]) and int(np.argmin(Jb)) != 2       # another mode is cheaper
    assert list(st) == [2, 1, 0] and o["mode"] == 2 and o["tau"] == 1
    us = h.outputs[2]["u_star"].cpu().numpy()
    np.testing.assert_array_equal(h.u.cpu().numpy()[:1], us)
