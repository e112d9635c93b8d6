"""The device error word: what kernels record and how the host reads it.

Device data the host never sees (the start state, the nominal U and the noise
of a cycle, the poses of an SDF batch) are checked on the device; a
non-finite value records EXACT_EINVAL in the context's (or batch's) error
word, which exact_ctx_get_error / exact_batch_get_error read and clear in
stream order.  The debug build (-DEXACT_DEBUG_CHECKS) adds index checks; on
valid inputs it records nothing and gives the release build's bits.  Every
case here is small and faults nothing: the bad values are NaN inputs that the
kernels carry through arithmetic only."""
import ctypes

import numpy as np
import pytest

import synth
from test_mppi_gpu import _t

pytestmark = pytest.mark.gpu

EINVAL = 1


@pytest.fixture(scope="module")
def ex():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_29663_gb300 import build
    build.build()
    import paper_2605_29663_gb300 as ex
    return ex


def _cycle(ex, ctx, s, **kw):
    import torch
    fp = ex.Footprint(s["kind"], s["fp"])
    U = _t(s["U"].astype(np.float32))
    out = ex.mppi_step(ctx, _t(s["q0"]), _t(s["cloud"]), _t(s["waypoints"]), U, _t(s["eps"]), fp, s["params"],
                       mask=None if s["mask"] is None else _t(s["mask"]), **kw)
    torch.cuda.synchronize()
    return out, U


@pytest.mark.parametrize("what", ["state", "noise", "U"])
def test_nonfinite_cycle_inputs_are_reported(ex, what):
    ctx = ex.Context()
    s = synth.plain_step(3, K=64, T=10, N=200)
    _cycle(ex, ctx, s)
    assert ctx.get_error() == 0
    bad = dict(s)
    if what == "state":
        bad["q0"] = np.array([0.0, np.nan, 0.0], np.float32)
    elif what == "noise":
        eps = s["eps"].copy()
        eps[17, 3, 1] = np.inf
        bad["eps"] = eps
    else:
        U = s["U"].copy()
        U[4, 0] = np.nan
        bad["U"] = U
    _cycle(ex, ctx, bad)
    assert ctx.get_error() == EINVAL
    assert ctx.get_error() == 0                  # read and cleared
    _cycle(ex, ctx, s)                           # a good cycle records nothing
    assert ctx.get_error() == 0


def test_nonfinite_pose_is_reported(ex):
    import torch
    ctx = ex.Context()
    w = synth.sdf_microbench(seed=2, n_poses=40, n_points=300, n_vertices=8)
    poses = w["poses"].copy()
    fp = ex.Footprint(w["kind"], w["fp"])
    ex.sdf_batch(_t(w["points"]), _t(poses), fp, ctx=ctx)
    assert ctx.get_error() == 0
    poses[7, 2] = np.nan
    ex.sdf_batch(_t(w["points"]), _t(poses), fp, ctx=ctx)
    assert ctx.get_error(torch.cuda.current_stream()) == EINVAL


def test_batch_error_word(ex):
    import torch
    g = synth.rng(5)
    scenes = [synth.random_scene(g, synth.DIFF, 8, 400, 64, 12, n_obst=10) for _ in range(3)]
    dev = []
    for i, s in enumerate(scenes):
        q0 = s["q0"].copy()
        if i == 1:
            q0[0] = np.nan
        dev.append(dict(state=_t(q0), cloud=_t(s["cloud"]), waypoints=_t(s["waypoints"]), U=_t(s["U"]),
                        noise=_t(s["eps"]), fp=ex.Footprint(s["kind"], s["fp"]), params=s["params"],
                        mask=None if s["mask"] is None else _t(s["mask"])))
    b = ex.Batch(dev)
    b.step()
    torch.cuda.synchronize()
    assert b.get_error() == EINVAL
    assert b.get_error() == 0


def _debug_cycle(ex, lib, s, dmin):
    """One mppi_step through the debug library's C ABI."""
    import torch
    p = ex.MppiParams.from_dict(s["params"])
    K, T, nu = p.K, p.T, p.n_u
    fp = ctypes.c_void_p()
    arr = np.ascontiguousarray(np.asarray(s["fp"], np.float32))
    assert lib.exact_footprint_create(s["kind"], arr.ctypes.data, arr.shape[0], ctypes.byref(fp)) == 0
    ctx = ctypes.c_void_p()
    assert lib.exact_ctx_create(ctypes.byref(ctx)) == 0
    f = dict(dtype=torch.float32, device="cuda")
    d = dict(state=_t(s["q0"]), cloud=_t(s["cloud"]), wp=_t(s["waypoints"]), U=_t(s["U"].astype(np.float32)),
             noise=_t(s["eps"]), mask=None if s["mask"] is None else _t(s["mask"]))
    out = {"u_star": torch.empty(nu, **f), "costs": torch.empty(K, **f), "weights": torch.empty(K, **f),
           "valid": torch.empty(1, dtype=torch.int32, device="cuda"), "U_upd": torch.empty((T, nu), **f),
           "dmin": torch.empty((K, T), **f) if dmin else None}
    P = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    N = d["cloud"].shape[0]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.mppi_step(ctx, P(d["state"]), P(d["cloud"]), P(d["mask"]), N, P(d["wp"]), d["wp"].shape[0], P(d["U"]),
                       P(d["noise"]), fp, ctypes.byref(p), P(out["u_star"]), P(out["costs"]), P(out["weights"]),
                       P(out["valid"]), P(out["U_upd"]), P(out["dmin"]), stream)
    assert rc == 0
    err = lib.exact_ctx_get_error(ctx, stream)
    lib.exact_ctx_destroy(ctx)
    lib.exact_footprint_destroy(fp)
    res = {k: v.cpu().numpy() for k, v in out.items() if v is not None}
    res["U"] = d["U"].cpu().numpy()
    return res, err


def test_debug_build_checks_and_bits(ex):
    """The debug library records nothing on valid cycles (point-pruned small
    cloud, sorted and chunk-pruned large cloud, unpruned with d_min, split
    horizon) and gives the release library's bits; a NaN start state is
    reported by it as by the release build."""
    from paper_2605_29663_gb300 import build, load_debug
    build.build(debug=True)
    lib = load_debug()
    ctx = ex.Context()
    cases = [(synth.plain_step(4), False), (synth.plain_step(5, K=24, T=16, N=300), True),
             (synth.forklift(6, K=256, T=24, N=2048), False), (synth.forklift(7, K=128, T=12, N=900), True)]
    for s, dmin in cases:
        got, err = _debug_cycle(ex, lib, s, dmin)
        assert err == 0
        ref, U = _cycle(ex, ctx, s, dmin=dmin)
        assert ctx.get_error() == 0
        for k in ("costs", "weights", "U_upd", "u_star", "valid") + (("dmin",) if dmin else ()):
            np.testing.assert_array_equal(got[k], ref[k].cpu().numpy(), err_msg=k)
        np.testing.assert_array_equal(got["U"], U.cpu().numpy())
    bad = dict(cases[0][0], q0=np.array([np.nan, 0.0, 0.0], np.float32))
    _, err = _debug_cycle(ex, lib, bad, False)
    assert err == EINVAL
