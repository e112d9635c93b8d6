"""Parity of mppi_step_predicted (time-indexed obstacle predictions: every
horizon step scores the constant-velocity prediction o + t_h v of the cloud)
with the FP64 oracle, at the tolerances of the MPPI parity tests; the zero
velocity case against mppi_step bit for bit."""
import numpy as np
import pytest

import oracle
import synth
from test_mppi_gpu import _t, compare

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


@pytest.fixture(scope="module")
def ctx(ex):
    return ex.Context()


def _run(ex, ctx, s, vel=True):
    import torch
    fp = ex.Footprint(s["kind"], s["fp"])
    U = _t(s["U"].astype(np.float32))
    out = ex.mppi_step(ctx, _t(s["q0"]), _t(s["cloud"]), _t(s["waypoints"]), U, _t(s["eps"]), fp, s["params"],
                       mask=None if s["mask"] is None else _t(s["mask"]),
                       velocity=_t(s["vel"]) if vel else None, dmin=True)
    torch.cuda.synchronize()
    assert ctx.get_error() == 0
    r = {k: v.cpu().numpy() for k, v in out.items()}
    r["U"] = U.cpu().numpy()
    r["valid"] = bool(r["valid"][0])
    return r


def _oracle(s):
    return oracle.mppi_step(s["params"], s["q0"], s["cloud"], s["waypoints"], s["U"], s["eps"], s["kind"], s["fp"],
                            mask=s["mask"], vel=s["vel"])


def _seeded(make, start, tries=6):
    for k in range(tries):
        s = make(start + k)
        o = _oracle(s)
        if o["n_near"] == 0:
            return s, o
    pytest.fail(f"{tries} consecutive seeds had threshold-adjacent d_min values")


def test_dynamic_scene(ex, ctx):
    """Boxes plus discs moving at 0.5 m/s, L footprint, K = 512, N = 2048."""
    s, o = _seeded(lambda k: synth.dynamic_scene(k, K=512, T=20, N=2048), 0)
    compare(s, _run(ex, ctx, s), o)


def test_fast_obstacles_and_padding(ex, ctx):
    """Faster discs (2 m/s), a cloud padded with masked points."""
    s, o = _seeded(lambda k: synth.dynamic_scene(k, K=256, T=24, N=9000, speed=2.0), 10)
    assert s["mask"] is not None
    compare(s, _run(ex, ctx, s), o)


def test_many_points_and_split_horizon(ex, ctx):
    """Few samples (each horizon split over several blocks) and a cloud of
    several shared-memory passes (predicted clouds stage half as many
    points per pass)."""
    def make(k):
        s = synth.dynamic_scene(k, K=24, T=16, N=5000, n_discs=120)
        return s
    s, o = _seeded(make, 20)
    compare(s, _run(ex, ctx, s), o)


@pytest.mark.parametrize("model", [synth.ACKERMANN, synth.OMNI])
def test_other_models_and_rect_cover(ex, ctx, model):
    def make(k):
        s = synth.dynamic_scene(k, K=300, T=18, N=1500)
        nu = synth.NU[model]
        extra = dict(wheelbase=1.4, clamp=1, u_min=[-1e30, -0.6, -1e30], u_max=[1e30, 0.6, 1e30]) \
            if model == synth.ACKERMANN else {}
        s["params"] = synth.mppi_params(300, 18, model, **extra)
        s["U"] = np.zeros((18, nu), np.float32)
        s["eps"] = synth.noise(synth.rng(k + 100), 300, 18, (0.3, 0.2, 0.5)[:nu])
        s["kind"], s["fp"] = synth.RECTS, synth.forklift_rects() * np.float32(0.5)
        return s
    s, o = _seeded(make, 30)
    compare(s, _run(ex, ctx, s), o)


def test_zero_velocity_equals_mppi_step(ex, ctx):
    s = synth.dynamic_scene(3, K=256, T=20, N=2048)
    s["vel"] = np.zeros_like(s["vel"])
    a = _run(ex, ctx, s, vel=True)
    b = _run(ex, ctx, s, vel=False)
    for k in ("dmin", "costs", "weights", "U_upd", "U", "u_star"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def test_missing_velocity_is_rejected(ex, ctx):
    import ctypes
    import torch
    s = synth.dynamic_scene(1, K=8, T=4, N=16)
    fp = ex.Footprint(s["kind"], s["fp"])
    p = ex.MppiParams.from_dict(s["params"])
    d = {k: _t(s[k]) for k in ("q0", "cloud", "waypoints", "U", "eps")}
    u = torch.empty(2, device="cuda")
    rc = ex.load().mppi_step_predicted(ctx.handle, d["q0"].data_ptr(), d["cloud"].data_ptr(), None, None, 16,
                                       d["waypoints"].data_ptr(), 1, d["U"].data_ptr(), d["eps"].data_ptr(),
                                       fp.handle, ctypes.byref(p), u.data_ptr(), None, None, None, None, None,
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 1   # EXACT_EINVAL, before any launch


def test_pruning_with_predictions_changes_no_cost(ex, ctx):
    """Predicted clouds prune with circles grown by t_h * max speed: the run
    without d_min output equals the run with it bit for bit."""
    import torch
    s = synth.dynamic_scene(9, K=384, T=24, N=2048, speed=1.5)
    res = []
    for dmin in (True, False):
        fp = ex.Footprint(s["kind"], s["fp"])
        U = _t(s["U"].astype(np.float32))
        out = ex.mppi_step(ctx, _t(s["q0"]), _t(s["cloud"]), _t(s["waypoints"]), U, _t(s["eps"]), fp, s["params"],
                           mask=None if s["mask"] is None else _t(s["mask"]), velocity=_t(s["vel"]), dmin=dmin)
        torch.cuda.synchronize()
        res.append(dict({k: v.cpu().numpy() for k, v in out.items()}, U=U.cpu().numpy()))
    for k in ("costs", "weights", "U_upd", "U", "u_star", "valid"):
        np.testing.assert_array_equal(res[0][k], res[1][k], err_msg=k)


def test_pruning_with_predictions_rect_cover(ex, ctx):
    """A rectangle cover with predicted points prunes through the fine
    sub-chunks (circles grown by t_h * max speed) and the bounding box: the
    run without a d_min output equals the run with it bit for bit."""
    import torch
    s = synth.dynamic_scene(19, K=320, T=20, N=3000, speed=1.5)
    s["kind"], s["fp"] = synth.RECTS, synth.forklift_rects() * np.float32(0.5)
    res = []
    for dmin in (True, False):
        fp = ex.Footprint(s["kind"], s["fp"])
        U = _t(s["U"].astype(np.float32))
        out = ex.mppi_step(ctx, _t(s["q0"]), _t(s["cloud"]), _t(s["waypoints"]), U, _t(s["eps"]), fp, s["params"],
                           mask=None if s["mask"] is None else _t(s["mask"]), velocity=_t(s["vel"]), dmin=dmin)
        torch.cuda.synchronize()
        res.append(dict({k: v.cpu().numpy() for k, v in out.items()}, U=U.cpu().numpy()))
    for k in ("costs", "weights", "U_upd", "U", "u_star", "valid"):
        np.testing.assert_array_equal(res[0][k], res[1][k], err_msg=k)


def test_predicted_cloud_order_changes_nothing(ex, ctx):
    """Points and velocities shuffled together give the same bits (the cycle
    orders the cloud itself before pruning)."""
    import torch
    s = synth.dynamic_scene(12, K=256, T=20, N=2048)
    perm = synth.rng(13).permutation(2048)
    t = dict(s, cloud=np.ascontiguousarray(s["cloud"][perm]), vel=np.ascontiguousarray(s["vel"][perm]),
             mask=None if s["mask"] is None else np.ascontiguousarray(s["mask"][perm]))
    outs = []
    for sc in (s, t):
        fp = ex.Footprint(sc["kind"], sc["fp"])
        U = _t(sc["U"].astype(np.float32))
        out = ex.mppi_step(ctx, _t(sc["q0"]), _t(sc["cloud"]), _t(sc["waypoints"]), U, _t(sc["eps"]), fp,
                           sc["params"], mask=None if sc["mask"] is None else _t(sc["mask"]), velocity=_t(sc["vel"]))
        torch.cuda.synchronize()
        outs.append(dict({k: v.cpu().numpy() for k, v in out.items()}, U=U.cpu().numpy()))
    for k in ("costs", "weights", "U_upd", "U", "u_star", "valid"):
        np.testing.assert_array_equal(outs[0][k], outs[1][k], err_msg=k)


def test_small_predicted_cloud_point_pruning(ex, ctx):
    """A predicted cloud below 1,024 points without a d_min output is pruned
    point by point at each step's predicted positions; the same bits as the
    run with a d_min output, and the oracle's values."""
    import torch
    s, o = _seeded(lambda k: synth.dynamic_scene(k, K=256, T=20, N=900), 40)
    a = _run(ex, ctx, s)
    fp = ex.Footprint(s["kind"], s["fp"])
    U = _t(s["U"].astype(np.float32))
    out = ex.mppi_step(ctx, _t(s["q0"]), _t(s["cloud"]), _t(s["waypoints"]), U, _t(s["eps"]), fp, s["params"],
                       mask=None if s["mask"] is None else _t(s["mask"]), velocity=_t(s["vel"]), dmin=False)
    torch.cuda.synchronize()
    for k in ("costs", "weights", "U_upd", "u_star"):
        np.testing.assert_array_equal(out[k].cpu().numpy(), a[k], err_msg=k)
    np.testing.assert_array_equal(U.cpu().numpy(), a["U"])
    compare(s, a, o)
