"""Host-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every function that include/exact_mppi.h declares; footprint
validation (a host-only path) accepts simple polygons and rejects the rest."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "exact_mppi.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2605_29663_gb300 import build, load
    build.build()
    return load()


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:(?:unsigned|long|short)\s+)*[A-Za-z_][A-Za-z0-9_]*(?:\s+|\s*\*+\s*)"
                       r"([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declarations_are_exported(lib):
    from paper_2605_29663_gb300 import EXPORTS, build
    declared = _declared_functions()
    assert declared, "no declarations parsed"
    assert sorted(EXPORTS) == declared
    nm = subprocess.run(["nm", "-D", "--defined-only", build.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in nm.splitlines() if " T " in line}
    for name in declared:
        assert name in exported, name
        assert hasattr(lib, name)


def test_library_targets_sm103a():
    from paper_2605_29663_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_status_strings(lib):
    from paper_2605_29663_gb300 import status_string
    assert status_string(0) == "ok"
    assert "simple" in status_string(2)
    assert status_string(99) == "unknown status"


def _create(lib, kind, data, n=None):
    arr = np.ascontiguousarray(np.asarray(data, dtype=np.float32))
    h = ctypes.c_void_p()
    rc = lib.exact_footprint_create(kind, arr.ctypes.data, arr.shape[0] if n is None else n, ctypes.byref(h))
    if rc == 0:
        k, m = ctypes.c_int(), ctypes.c_int()
        assert lib.exact_footprint_info(h, ctypes.byref(k), ctypes.byref(m)) == 0
        assert k.value == kind and m.value == (arr.shape[0] if n is None else n)
        lib.exact_footprint_destroy(h)
    return rc


def test_footprint_accepts_simple_polygons(lib):
    g = np.random.default_rng(0)
    assert _create(lib, 0, synth.l_footprint()) == 0
    assert _create(lib, 0, synth.l_footprint()[::-1].copy()) == 0      # clockwise
    assert _create(lib, 0, synth.l_footprint_gap()) == 0
    for n in (3, 4, 7, 32, 64):
        assert _create(lib, 0, synth.star_polygon(g, n, 0.3, 1.2)) == 0
    assert _create(lib, 1, synth.forklift_rects()) == 0


def test_footprint_rejections(lib):
    bowtie = [(0, 0), (1, 1), (1, 0), (0, 1)]
    assert _create(lib, 0, bowtie) == 2                                  # self-intersecting
    assert _create(lib, 0, [(0, 0), (1, 0), (1, 0), (1, 1)]) == 2        # repeated vertex
    assert _create(lib, 0, [(0, 0), (1, 0), (2, 0)]) == 2                # zero area
    assert _create(lib, 0, [(0, 0), (2, 0), (1, 0), (1, 1)]) == 2        # edge folds back
    assert _create(lib, 0, [(0, 0), (1, 0)]) == 1                        # too few vertices
    assert _create(lib, 0, [(0, 0), (1, np.nan), (0, 1)]) == 1           # non-finite
    big = synth.star_polygon(np.random.default_rng(1), 65, 0.3, 1.2)
    assert _create(lib, 0, big) == 3                                     # capacity
    assert _create(lib, 1, [(0, 0, 1, 0)]) == 1                          # zero half-extent
    assert _create(lib, 1, np.tile([0, 0, 1, 1], (9, 1))) == 3           # more than 8 boxes
    assert _create(lib, 7, [(0, 0), (1, 0), (0, 1)]) == 1                # unknown kind


def test_python_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2605_29663_gb300 as pkg
    monkeypatch.setattr(pkg, "_lib", None)
    monkeypatch.setattr(pkg._build, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        pkg.load()
