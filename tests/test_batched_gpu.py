"""Parity of mppi_step_batched (one persistent launch over many scenes) with
the single-scene mppi_step path (bit for bit: same device bodies, same
operation order) and with the FP64 oracle (the tolerances of
test_mppi_gpu.py), on heterogeneous seeded scenes."""
import numpy as np
import pytest

import synth
from test_mppi_gpu import _t, compare, run_oracle

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


def _scene_set(seed, n, scale):
    scenes = synth.batched(seed, n_scenes=n, scale=scale)
    # a rectangle-cover forklift and a spin-in-place scene widen the mix
    scenes.append(synth.forklift(seed, K=64, T=12, N=300))
    s = synth.plain_step(seed + 1, K=40, T=9, N=77)
    s["params"] = synth.mppi_params(40, 9, synth.SPIN)
    s["U"] = np.zeros((9, 1), np.float32)
    s["eps"] = synth.noise(synth.rng(seed + 2), 40, 9, (0.5,))
    scenes.append(s)
    return scenes


def _dev_scene(ex, s):
    return dict(state=_t(s["q0"]), cloud=_t(s["cloud"]), waypoints=_t(s["waypoints"]), U=_t(s["U"]),
                noise=_t(s["eps"]), mask=None if s["mask"] is None else _t(s["mask"]),
                fp=ex.Footprint(s["kind"], s["fp"]), params=s["params"])


def _run_batched(ex, scenes, tiles=None, dmin=True):
    import torch
    dev = [_dev_scene(ex, s) for s in scenes]
    b = ex.Batch(dev, dmin=dmin)
    if tiles:
        b.set_tiles(*tiles)
    b.step()
    torch.cuda.synchronize()
    res = []
    for d, o in zip(dev, b.outputs):
        r = {k: v.cpu().numpy() for k, v in o.items()}
        r["U"] = d["U"].cpu().numpy()
        r["valid"] = bool(r["valid"][0])
        res.append(r)
    return res


def _run_single(ex, ctx, s, dmin=True):
    import torch
    d = _dev_scene(ex, s)
    out = ex.mppi_step(ctx, d["state"], d["cloud"], d["waypoints"], d["U"], d["noise"], d["fp"], s["params"],
                       mask=d["mask"], dmin=dmin)
    torch.cuda.synchronize()
    r = {k: v.cpu().numpy() for k, v in out.items()}
    r["U"] = d["U"].cpu().numpy()
    r["valid"] = bool(r["valid"][0])
    return r


@pytest.mark.parametrize("tiles", [None, (128, 1), (512, 8)])
def test_batched_equals_single_scene_bitwise(ex, tiles):
    scenes = _scene_set(3, 10, 0.05)
    got = _run_batched(ex, scenes, tiles)
    ctx = ex.Context()
    for i, s in enumerate(scenes):
        ref = _run_single(ex, ctx, s)
        for key in ("dmin", "costs", "weights", "U_upd", "U", "u_star"):
            np.testing.assert_array_equal(got[i][key], ref[key], err_msg=f"scene {i} {key}")
        assert got[i]["valid"] == ref["valid"]


def test_batched_matches_oracle(ex):
    scenes = [s for s in _scene_set(5, 8, 0.03)]
    got = _run_batched(ex, scenes)
    checked = 0
    for s, g in zip(scenes, got):
        o = run_oracle(s)
        if o["n_near"]:
            continue
        compare(s, g, o)
        checked += 1
    assert checked >= len(scenes) - 3


def test_batched_two_steps_and_autotune(ex):
    """A second step on the same plan (state carried in U) still equals the
    single-scene path; autotuning touches no scene output."""
    import torch
    scenes = _scene_set(7, 6, 0.04)
    dev = [_dev_scene(ex, s) for s in scenes]
    b = ex.Batch(dev, dmin=False)
    U0 = [d["U"].clone() for d in dev]
    report = b.autotune(iters=1)
    assert report["best"]["threads"] in (128, 256, 512) and len(report["candidates"]) >= 6
    for d, u in zip(dev, U0):
        assert torch.equal(d["U"], u)
    b.step()
    b.step()
    torch.cuda.synchronize()
    ctx = ex.Context()
    for i, s in enumerate(scenes):
        d = _dev_scene(ex, s)
        for _ in range(2):
            ex.mppi_step(ctx, d["state"], d["cloud"], d["waypoints"], d["U"], d["noise"], d["fp"], s["params"],
                         mask=d["mask"])
        torch.cuda.synchronize()
        np.testing.assert_array_equal(dev[i]["U"].cpu().numpy(), d["U"].cpu().numpy(), err_msg=f"scene {i}")


def test_batch_rejects_bad_scene(ex):
    s = synth.plain_step(0, K=8, T=4, N=16)
    d = _dev_scene(ex, s)
    d["params"] = dict(s["params"], **{"lambda": 0.0})   # the temperature must be positive
    with pytest.raises(ex.ExactError):
        ex.Batch([d])


def test_batched_pruning_changes_no_cost(ex):
    """A batch without d_min outputs prunes point chunks beyond d_safe: same
    J~, weights and sequences as the batch that outputs d_min, bit for bit."""
    import torch
    scenes = _scene_set(5, 8, 0.05)
    res = []
    for dmin in (True, False):
        dev = [_dev_scene(ex, s) for s in scenes]
        b = ex.Batch(dev, dmin=dmin)
        b.step()
        torch.cuda.synchronize()
        res.append([dict({k: v.cpu().numpy() for k, v in o.items()}, U=d["U"].cpu().numpy())
                    for d, o in zip(dev, b.outputs)])
    for i in range(len(scenes)):
        for k in ("costs", "weights", "U_upd", "U", "u_star", "valid"):
            np.testing.assert_array_equal(res[0][i][k], res[1][i][k], err_msg=f"scene {i} {k}")


def test_autotune_persists_the_tile_shape(ex, tmp_path):
    """Tuning with a cache file stores the winner under the batch's shape key;
    a second batch of the same class reuses it without timing."""
    scenes = _scene_set(6, 4, 0.05)
    cache = str(tmp_path / "tiles.json")
    b1 = ex.Batch([_dev_scene(ex, s) for s in scenes])
    rep = b1.autotune(iters=1, cache=cache)
    assert "candidates" in rep and rep["key"] == b1.class_key
    b2 = ex.Batch([_dev_scene(ex, s) for s in scenes])
    b2.set_tiles(64, 8)
    rep2 = b2.autotune(iters=1, cache=cache)
    assert rep2["cached"] and b2.tiles == b1.tiles


@pytest.mark.parametrize("kind", ["polygon", "rects"])
def test_uniform_footprint_batch_equals_single_scene_bitwise(ex, kind):
    """Scenes that share one footprint run the constant-footprint kernels;
    each still gives the single-scene bits."""
    g = synth.rng(91)
    scenes = []
    for i in range(5):
        model = [synth.DIFF, synth.ACKERMANN, synth.OMNI][i % 3]
        s = synth.random_scene(g, model, 12, int(g.integers(300, 3000)), int(g.choice([64, 200])), int(g.integers(8, 30)))
        if kind == "polygon":
            s["kind"], s["fp"] = synth.POLYGON, synth.l_footprint()
        else:
            s["kind"], s["fp"] = synth.RECTS, synth.forklift_rects() * np.float32(0.4)
        scenes.append(s)
    got = _run_batched(ex, scenes)
    ctx = ex.Context()
    for i, s in enumerate(scenes):
        ref = _run_single(ex, ctx, s)
        for key in ("dmin", "costs", "weights", "U_upd", "U", "u_star"):
            np.testing.assert_array_equal(got[i][key], ref[key], err_msg=f"scene {i} {key}")


def test_batched_ordered_clouds_change_no_cost(ex):
    """Scenes of 1,024 points or more get spatially ordered copies (several
    shared-memory passes for the largest): the batch without d_min outputs
    matches the batch with them bit for bit, shuffled clouds included."""
    import torch
    g = synth.rng(17)
    scenes = []
    for i, N in enumerate([1100, 3000, 9000]):
        s = synth.random_scene(g, [synth.DIFF, synth.ACKERMANN, synth.OMNI][i], 10, N, 160, 16, n_obst=50)
        if i == 1:   # a shuffled cloud
            perm = g.permutation(N)
            s["cloud"] = np.ascontiguousarray(s["cloud"][perm])
            s["mask"] = None if s["mask"] is None else np.ascontiguousarray(s["mask"][perm])
        scenes.append(s)
    res = []
    for dmin in (True, False):
        dev = [_dev_scene(ex, s) for s in scenes]
        b = ex.Batch(dev, dmin=dmin)
        b.step()
        torch.cuda.synchronize()
        res.append([dict({k: v.cpu().numpy() for k, v in o.items()}, U=d["U"].cpu().numpy())
                    for d, o in zip(dev, b.outputs)])
    for i in range(len(scenes)):
        for k in ("costs", "weights", "U_upd", "U", "u_star", "valid"):
            np.testing.assert_array_equal(res[0][i][k], res[1][i][k], err_msg=f"scene {i} {k}")


@pytest.mark.parametrize("shared_fp", [False, True])
@pytest.mark.parametrize("dmin", [True, False])
def test_paired_items_equal_single_scene_bitwise(ex, shared_fp, dmin):
    """A batch of at least 4 samples per SM takes two samples of a scene per
    item (odd K: a lone last sample; T = 64, the longest horizon that pairs;
    T = 65 does not pair).  Each scene alone has fewer samples and runs one
    per block, and still gives the same bits."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    g = synth.rng(123)
    scenes = []
    for i, (K, T) in enumerate([(2 * sms + 1, 64), (sms + 1, 20), (sms + 3, 65)]):
        s = synth.random_scene(g, [synth.DIFF, synth.ACKERMANN, synth.OMNI][i], 10, int(g.integers(400, 2500)), K, T,
                               n_obst=20)
        if shared_fp:
            s["kind"], s["fp"] = synth.POLYGON, synth.l_footprint()
        scenes.append(s)
    got = _run_batched(ex, scenes, dmin=dmin)
    ctx = ex.Context()
    for i, s in enumerate(scenes):
        ref = _run_single(ex, ctx, s, dmin=dmin)
        for key in ("dmin", "costs", "weights", "U_upd", "U", "u_star"):
            if key in ref:
                np.testing.assert_array_equal(got[i][key], ref[key], err_msg=f"scene {i} {key}")
        assert got[i]["valid"] == ref["valid"]


@pytest.mark.parametrize("shared_fp", [False, True])
def test_batched_step_captured_in_a_cuda_graph(ex, shared_fp):
    """The whole batched control step (memset, ordering, persistent sample
    kernel, update, validation) captured once in a CUDA graph and replayed
    for three consecutive cycles gives, after every cycle, the bits of three
    eager steps of an identical batch: outputs and the shifted nominals."""
    import torch
    scenes = synth.batched(31, n_scenes=10, scale=0.3)
    if shared_fp:
        for s in scenes:
            s["kind"], s["fp"] = synth.POLYGON, synth.l_footprint()
    eager = [_dev_scene(ex, s) for s in scenes]
    graph = [_dev_scene(ex, s) for s in scenes]
    be, bg = ex.Batch(eager), ex.Batch(graph)
    st = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            bg.step()
    torch.cuda.synchronize()
    for cycle in range(3):
        be.step()
        g.replay()
        torch.cuda.synchronize()
        for i, (de, dg, oe, og) in enumerate(zip(eager, graph, be.outputs, bg.outputs)):
            for k in oe:
                np.testing.assert_array_equal(og[k].cpu().numpy(), oe[k].cpu().numpy(),
                                              err_msg=f"cycle {cycle} scene {i} {k}")
            np.testing.assert_array_equal(dg["U"].cpu().numpy(), de["U"].cpu().numpy(),
                                          err_msg=f"cycle {cycle} scene {i} U")
    assert be.get_error() == 0 and bg.get_error() == 0
