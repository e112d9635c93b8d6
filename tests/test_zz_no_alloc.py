"""mppi_step_noalloc -- the control cycle for callers that cannot allocate
device memory (a real-time loop that must not call cudaMalloc, work inside a
stream capture, memory owned by another allocator).  It keeps its scratch in
a fixed device array inside the library, so these tests check that it
computes what mppi_step computes: the same scenes through both entry points,
two calls in a row (the second starts from the first's shifted U and finds
the array holding the first call's data), compared bit for bit, with and
without a d_min output (the pruned sample phase).  This file is collected
last on purpose."""
import ctypes

import numpy as np
import pytest

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


def _outputs(K, T, nu, dmin=True):
    import torch
    f = dict(dtype=torch.float32, device="cuda")
    return {"u_star": torch.empty(nu, **f), "costs": torch.empty(K, **f), "weights": torch.empty(K, **f),
            "valid": torch.empty(1, dtype=torch.int32, device="cuda"), "U_upd": torch.empty((T, nu), **f),
            "dmin": torch.empty((K, T), **f) if dmin else None}


def _coherent(seed, K, T, N, mask_tail=0, shuffle=False):
    """Obstacle edge points (spatially coherent runs), optionally shuffled, the
    last mask_tail points masked."""
    g = synth.rng(seed)
    s = synth.random_scene(g, synth.DIFF, 6, N, K, T, n_obst=40)
    s["fp"], s["kind"] = synth.l_footprint(), synth.POLYGON
    m = np.ones(N, np.uint8) if s["mask"] is None else s["mask"].copy()
    if mask_tail:
        m[N - mask_tail:] = 0
    if shuffle:
        perm = synth.rng(seed + 1).permutation(N)
        s["cloud"], m = np.ascontiguousarray(s["cloud"][perm]), np.ascontiguousarray(m[perm])
    s["mask"] = m if (mask_tail or s["mask"] is not None) else None
    return s


CASES = ["plain", "forklift", "few_samples", "pruned_ordered", "pruned_shuffled_masked"]


@pytest.mark.parametrize("which", CASES)
def test_noalloc_matches_mppi_step_two_calls(ex, which):
    """Both entry points run the same kernels in the same order, so their
    outputs are the same bits.  The pruned cases (no d_min output, 1,024 points
    or more) differ in one respect: mppi_step works on a spatially ordered copy
    of the cloud kept in its context, the allocation-free call on the cloud as
    given (its sample blocks bound their own point chunks); the minima over
    points, and so every output, are still the same bits."""
    import torch
    dmin = True
    if which == "plain":
        s = synth.plain_step(11)
    elif which == "forklift":
        s = synth.forklift(2, K=512, T=24, N=900)
    elif which == "few_samples":
        s = synth.plain_step(12, K=24, T=16, N=300)        # fewer samples than SMs: split horizon
    elif which == "pruned_ordered":
        s, dmin = _coherent(14, 384, 20, 3000), False
    else:
        s, dmin = _coherent(15, 256, 16, 2500, mask_tail=37, shuffle=True), False
    p = s["params"]
    K, T, nu = p["K"], p["T"], p["nu"]
    fp = ex.Footprint(s["kind"], s["fp"])
    ctx = ex.Context()
    dA = dict(state=_t(s["q0"]), cloud=_t(s["cloud"]), waypoints=_t(s["waypoints"]), U=_t(s["U"]),
              noise=_t(s["eps"]), mask=None if s["mask"] is None else _t(s["mask"]))
    dB = dict(dA, U=_t(s["U"]))
    for call in range(2):
        ref = ex.mppi_step(ctx, dA["state"], dA["cloud"], dA["waypoints"], dA["U"], dA["noise"], fp, p,
                           mask=dA["mask"], dmin=dmin)
        got = _outputs(K, T, nu, dmin)
        _noalloc_cycle(ex, dB, fp, p, got)
        torch.cuda.synchronize()
        for k in ("costs", "weights", "U_upd", "u_star", "valid") + (("dmin",) if dmin else ()):
            np.testing.assert_array_equal(got[k].cpu().numpy(), ref[k].cpu().numpy(), err_msg=f"call {call} {k}")
        np.testing.assert_array_equal(dB["U"].cpu().numpy(), dA["U"].cpu().numpy(), err_msg=f"call {call} U")


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
