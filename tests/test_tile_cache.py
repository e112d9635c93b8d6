"""Host logic of the batch tile cache: the shape-class key and the JSON store
(no GPU needed)."""
import json
import types

import torch

import synth
from paper_2605_29663_gb300 import scene_class_key, tile_cache_lookup, tile_cache_store


def _scene(kind, n, N, K, T):
    return {"fp": types.SimpleNamespace(kind=kind, n=n), "cloud": torch.zeros((N, 2)),
            "params": synth.mppi_params(K, T, synth.DIFF)}


def test_key_ignores_scene_order_and_small_size_changes():
    a = [_scene(0, 6, 500, 256, 20), _scene(1, 3, 3000, 1024, 30)]
    b = [a[1], a[0]]
    c = [_scene(0, 6, 510, 256, 20), _scene(1, 3, 2900, 1024, 30)]   # same powers of two
    assert scene_class_key(a, "gpu") == scene_class_key(b, "gpu") == scene_class_key(c, "gpu")


def test_key_separates_shape_classes_and_devices():
    a = [_scene(0, 6, 500, 256, 20)]
    assert scene_class_key(a, "gpu") != scene_class_key([_scene(0, 6, 600, 256, 20)], "gpu")
    assert scene_class_key(a, "gpu") != scene_class_key([_scene(0, 8, 500, 256, 20)], "gpu")
    assert scene_class_key(a, "gpu") != scene_class_key([_scene(0, 6, 500, 512, 20)], "gpu")
    assert scene_class_key(a, "gpu") != scene_class_key(a, "other gpu")


def test_store_and_lookup(tmp_path):
    path = str(tmp_path / "sub" / "tiles.json")
    assert tile_cache_lookup(path, "k1") is None
    tile_cache_store(path, "k1", 256, 1, 3.5)
    tile_cache_store(path, "k2", 512, 2, 4.0)
    assert tile_cache_lookup(path, "k1") == (256, 1)
    assert tile_cache_lookup(path, "k2") == (512, 2)
    tile_cache_store(path, "k1", 128, 4, 3.0)            # overwrite
    assert tile_cache_lookup(path, "k1") == (128, 4)
    data = json.load(open(path))
    assert set(data) == {"k1", "k2"}


def test_corrupt_cache_is_ignored_and_rewritten(tmp_path):
    path = str(tmp_path / "tiles.json")
    open(path, "w").write("{not json")
    assert tile_cache_lookup(path, "k") is None
    tile_cache_store(path, "k", 256, 1, 1.0)
    assert tile_cache_lookup(path, "k") == (256, 1)
    open(path, "w").write(json.dumps({"k": {"threads": "x"}}))
    assert tile_cache_lookup(path, "k") is None
