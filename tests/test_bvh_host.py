"""The host BVH builder (csrc/bvh_build.cpp) on the CPU: tests/bvh_check.cpp
is compiled with the host compiler against the builder and checks the tree of
seeded scenes -- every triangle in exactly one leaf, its record exact, every
child box containing its subtree, refs in range, empty slots empty, the stack
bound, and two builds byte-identical (the top subtrees are built on separate
threads).  Damaged trees must fail the checks, so they are not vacuous.  Two
trees merged as a batch merges its scenes (refs moved by rebase_ref, the same
function the GPU's merge kernel applies) keep both scenes' trees intact."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2409_07148_gb300 import scenes

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx or not os.path.exists(os.path.join(CUDA_INC, "vector_types.h")):
        pytest.skip("no host C++ compiler or CUDA headers")
    out = str(tmp_path_factory.mktemp("bvh") / "bvh_check")
    cmd = [cxx, "-std=c++17", "-O2", "-pthread", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(ROOT, "paper_2409_07148_gb300", "csrc"), "-I", CUDA_INC,
           os.path.join(HERE, "bvh_check.cpp"), os.path.join(ROOT, "paper_2409_07148_gb300", "csrc", "bvh_build.cpp"),
           "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


def _write(path, verts, tris, mats):
    with open(path, "wb") as f:
        f.write(np.array([len(verts), len(tris)], np.uint32).tobytes())
        f.write(np.ascontiguousarray(verts, np.float32).tobytes())
        f.write(np.ascontiguousarray(tris, np.uint32).tobytes())
        f.write(np.ascontiguousarray(mats, np.uint32).tobytes())


def _run(checker, path, mode=None, other=None):
    r = subprocess.run([checker, path] + ([mode] if mode else []) + ([other] if other else []), capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    return dict(kv.split("=", 1) for kv in r.stdout.split())


def _scene_cases():
    rng = np.random.default_rng(7)
    cases = {}
    for name, sc in (("cornell", scenes.cornell()),
                     ("cornell_spheres", scenes.cornell_spheres()),          # 40k: threaded top levels
                     ("random_boxes", scenes.random_boxes(3, 20000, 64, 64, 4))):
        cases[name] = (sc.verts, sc.tris, sc.tri_mat)
    # all centroids coincide: the split falls back to positions
    v = rng.normal(0.0, 1.0, (300, 3)).astype(np.float32)
    v[1::3] = -v[0::3]
    v[2::3] = 0.0
    cases["same_centroid"] = (v, np.arange(300, dtype=np.uint32).reshape(100, 3), np.zeros(100, np.uint32))
    cases["one_triangle"] = (np.eye(3, dtype=np.float32), np.array([[0, 1, 2]], np.uint32), np.zeros(1, np.uint32))
    return cases


@pytest.mark.parametrize("name", ["cornell", "cornell_spheres", "random_boxes", "same_centroid", "one_triangle"])
def test_bvh_invariants(checker, tmp_path, name):
    verts, tris, mats = _scene_cases()[name]
    path = str(tmp_path / f"{name}.bin")
    _write(path, verts, tris, mats)
    res = _run(checker, path)
    assert res["ok"] == "1", res
    for k in ("same", "cover", "records", "refs", "empty", "contain", "stack"):
        assert res[k] == "1", (k, res)
    assert int(res["tris"]) == len(tris)


def test_bvh_checks_catch_damage(checker, tmp_path):
    sc = scenes.random_boxes(5, 3000, 32, 32, 4)
    path = str(tmp_path / "rb.bin")
    _write(path, sc.verts, sc.tris, sc.tri_mat)
    assert _run(checker, path, "shrink")["contain"] == "0"
    assert _run(checker, path, "drop")["cover"] == "0"


def test_bvh_merge_as_in_a_batch(checker, tmp_path):
    a = scenes.cornell_spheres(width=32, height=32, depth=4, n_lon=24, n_lat=13)
    b = scenes.random_boxes(8, 6000, 32, 32, 4)
    pa, pb = str(tmp_path / "a.bin"), str(tmp_path / "b.bin")
    _write(pa, a.verts, a.tris, a.tri_mat)
    _write(pb, b.verts, b.tris, b.tri_mat)
    for x, y in ((pa, pb), (pb, pa)):
        res = _run(checker, x, "merge", y)
        assert res["merge_a"] == "1" and res["merge_b"] == "1", res
    res = _run(checker, pa, "merge_off_by_one", pb)
    assert res["merge_a"] == "1" and res["merge_b"] == "0", res


@pytest.mark.parametrize("bad", ["index", "nan", "inf", "both"])
def test_bvh_rejects_a_bad_triangle_in_a_late_chunk(checker, tmp_path, bad):
    """The 40k-triangle scene is set up in chunks on several threads; a bad
    triangle deep in the last chunk is still found, and with two bad triangles
    the error of the earlier one (in triangle order) is the one reported."""
    sc = scenes.cornell_spheres()
    verts, tris = sc.verts.copy(), sc.tris.copy()
    late = 37_000
    if bad in ("index", "both"):
        tris[late if bad == "index" else 100, 2] = len(verts)
    if bad in ("nan", "inf", "both"):
        verts[tris[late, 1], 0] = np.inf if bad == "inf" else np.nan
    path = str(tmp_path / f"bad_{bad}.bin")
    _write(path, verts, tris, sc.tri_mat)
    r = subprocess.run([checker, path], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok=0"), r.stdout
    assert ("out of range" if bad in ("index", "both") else "not finite") in r.stdout, r.stdout
