"""The seeded scene generators (the inputs of every test and of the bench) and
bench.py's guard on its recorded DRAM traffic, on the CPU.

Scenes: valid indices and materials, finite vertices, the documented sizes,
and the same arrays for the same seed.  Traffic guard: the recorded figure is
reported only for the workload it was captured on and only while the kernel
sources hash to the recorded values."""
import hashlib
import os
import sys

import numpy as np
import pytest

from paper_2409_07148_gb300 import scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _valid(sc):
    assert sc.verts.ndim == 2 and sc.verts.shape[1] == 3 and np.all(np.isfinite(sc.verts))
    assert sc.tris.ndim == 2 and sc.tris.shape[1] == 3
    assert sc.tris.size == 0 or (sc.tris.min() >= 0 and sc.tris.max() < len(sc.verts))
    assert len(sc.tri_mat) == len(sc.tris)
    assert sc.tri_mat.size == 0 or sc.tri_mat.max() < len(sc.mats)
    assert np.asarray(sc.camera).size == 12 and np.all(np.isfinite(sc.camera))
    assert sc.D == 2 + 2 * sc.depth


CASES = [
    ("cornell", dict()),
    ("cornell_spheres", dict(width=64, height=64, depth=5, n_lon=30, n_lat=16)),
    ("furnace", dict()),
    ("glass_furnace", dict()),
    ("random_boxes", dict(seed=3, n_tris=5000, width=32, height=32, depth=4)),
    ("caustic_slit", dict(width=64, height=64, depth=6, n_lon=40, n_lat=21)),
    ("terrain", dict(width=64, height=64, depth=4, n_grid=60, n_lights=8)),
]


@pytest.mark.parametrize("name,kw", CASES)
def test_scene_is_valid_and_seeded(name, kw):
    a = scenes.by_name(name, **kw)
    _valid(a)
    b = scenes.by_name(name, **kw)
    assert np.array_equal(a.verts, b.verts) and np.array_equal(a.tris, b.tris)
    assert np.array_equal(a.tri_mat, b.tri_mat) and np.array_equal(a.mats, b.mats)


def test_documented_sizes():
    assert scenes.cornell_spheres().n_tris == 40024        # the bench scene
    assert scenes.cornell().n_tris > 0 and scenes.cornell().D == 8
    t = scenes.terrain(width=64, height=64, depth=12, n_grid=60, n_lights=8)
    assert t.D == 26
    r = scenes.random_boxes(3, 5000, 32, 32, 4)
    assert abs(r.n_tris - 5000) / 5000 < 0.25                # log-uniform counts are approximate targets


def test_seeds_differ():
    a = scenes.random_boxes(3, 5000, 32, 32, 4)
    b = scenes.random_boxes(4, 5000, 32, 32, 4)
    assert a.verts.shape != b.verts.shape or not np.array_equal(a.verts, b.verts)


def test_bench_traffic_guard(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    src = os.path.join(ROOT, "paper_2409_07148_gb300", "csrc")
    now = {f: hashlib.sha256(open(os.path.join(src, f), "rb").read()).hexdigest()[:16]
           for f in bench.PATH_TRAFFIC["sources"]}
    rec = dict(bench.PATH_TRAFFIC, sources=now, bytes_per_launch=123.0)
    monkeypatch.setattr(bench, "PATH_TRAFFIC", rec)
    assert bench.path_traffic("cornell_spheres", 1 << 20) == 123.0
    assert bench.path_traffic("cornell_spheres", 1 << 18) is None          # another size
    assert bench.path_traffic("caustic_slit", 1 << 20) is None             # another workload
    stale = dict(rec, sources={f: "0" * 16 for f in now})
    monkeypatch.setattr(bench, "PATH_TRAFFIC", stale)
    assert bench.path_traffic("cornell_spheres", 1 << 20) is None          # the kernel changed
