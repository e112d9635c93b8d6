"""mppi_step_noalloc -- the control cycle for callers that cannot allocate
device memory (a real-time loop that must not call cudaMalloc, work inside a
stream capture, memory owned by another allocator).  It keeps its scratch in
a fixed device array inside the library, so these tests check that it
computes what mppi_step computes: the same scenes through both entry points,
two calls in a row (the second starts from the first's shifted U and finds
the array holding the first call's data), compared within the parity
tolerances of the MPPI tests.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

REL = 1e-4
D_TOL = 2e-5


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
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _noalloc_cycle(ex, d, fp, params, out):
    """One call of mppi_step_noalloc through the C ABI (ctypes, no binding helper)."""
    import torch
    lib = ex.load()
    p = ex.MppiParams.from_dict(params)
    N = d["cloud"].shape[0]
    rc = lib.mppi_step_noalloc(_ptr(d["state"]), _ptr(d["cloud"]) if N else None, _ptr(d["mask"]), N,
                               _ptr(d["waypoints"]), d["waypoints"].shape[0], _ptr(d["U"]), _ptr(d["noise"]),
                               fp.handle, ctypes.byref(p), _ptr(out["u_star"]), _ptr(out["costs"]),
                               _ptr(out["weights"]), _ptr(out["valid"]), _ptr(out["U_upd"]), _ptr(out["dmin"]),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, ex.status_string(rc)


def _outputs(K, T, nu):
    import torch
    f = dict(dtype=torch.float32, device="cuda")
    return {"u_star": torch.empty(nu, **f), "costs": torch.empty(K, **f), "weights": torch.empty(K, **f),
            "valid": torch.empty(1, dtype=torch.int32, device="cuda"), "U_upd": torch.empty((T, nu), **f),
            "dmin": torch.empty((K, T), **f)}


def _close(a, b, scale):
    return np.all(np.abs(a - b) <= REL * np.maximum(np.abs(b), scale))


@pytest.mark.parametrize("which", ["plain", "forklift", "few_samples"])
def test_noalloc_matches_mppi_step_two_calls(ex, which):
    import torch
    if which == "plain":
        s = synth.plain_step(11)
    elif which == "forklift":
        s = synth.forklift(2, K=512, T=24, N=900)
    else:
        s = synth.plain_step(12, K=24, T=16, N=300)        # fewer samples than SMs: split horizon
    p = s["params"]
    K, T, nu = p["K"], p["T"], p["nu"]
    fp = ex.Footprint(s["kind"], s["fp"])
    sigma = np.maximum(s["eps"].reshape(-1, nu).std(axis=0), 1e-3)
    ctx = ex.Context()
    dA = dict(state=_t(s["q0"]), cloud=_t(s["cloud"]), waypoints=_t(s["waypoints"]), U=_t(s["U"]),
              noise=_t(s["eps"]), mask=None if s["mask"] is None else _t(s["mask"]))
    dB = dict(dA, U=_t(s["U"]))
    for call in range(2):
        ref = ex.mppi_step(ctx, dA["state"], dA["cloud"], dA["waypoints"], dA["U"], dA["noise"], fp, p,
                           mask=dA["mask"], dmin=True)
        got = _outputs(K, T, nu)
        _noalloc_cycle(ex, dB, fp, p, got)
        torch.cuda.synchronize()
        r = {k: v.cpu().numpy() for k, v in ref.items()}
        g = {k: v.cpu().numpy() for k, v in got.items()}
        assert int(g["valid"][0]) == int(r["valid"][0]), call
        fin = np.isfinite(r["dmin"])
        assert np.array_equal(np.isfinite(g["dmin"]), fin)
        assert np.all(np.abs(g["dmin"][fin] - r["dmin"][fin]) <= D_TOL), call
        big = r["weights"] >= 1e-6 * r["weights"].max()
        assert np.all(np.abs(g["weights"][big] - r["weights"][big]) <= REL * r["weights"][big]), call
        assert _close(g["U_upd"], r["U_upd"], sigma[None, :]), call
        assert _close(g["u_star"], r["u_star"], sigma), call
        assert _close(dB["U"].cpu().numpy(), dA["U"].cpu().numpy(), sigma[None, :]), call
        np.testing.assert_allclose(g["costs"], r["costs"], rtol=1e-5, atol=1e-3)


def test_noalloc_rejects_sizes_beyond_the_array(ex):
    import torch
    s = synth.plain_step(13, K=8, T=8, N=8)
    p = dict(s["params"], K=65536, T=128)
    fp = ex.Footprint(s["kind"], s["fp"])
    d = dict(state=_t(s["q0"]), cloud=_t(s["cloud"]), waypoints=_t(s["waypoints"]),
             U=torch.zeros((128, 2), device="cuda"), noise=torch.zeros((1, 1, 2), device="cuda"), mask=None)
    out = {"u_star": torch.empty(2, device="cuda"), "costs": None, "weights": None, "valid": None, "U_upd": None,
           "dmin": None}
    lib = ex.load()
    prm = ex.MppiParams.from_dict(p)
    rc = lib.mppi_step_noalloc(_ptr(d["state"]), _ptr(d["cloud"]), None, 8, _ptr(d["waypoints"]), 1, _ptr(d["U"]),
                               _ptr(d["noise"]), fp.handle, ctypes.byref(prm), _ptr(out["u_star"]), None, None, None,
                               None, None, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 3   # EXACT_ECAPACITY, checked before any launch
