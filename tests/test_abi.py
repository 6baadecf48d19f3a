"""The C-ABI library loads and exports every symbol include/jr.h declares, and
rejects bad arguments with a status code before any device work (CPU only)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2409_07148_gb300 import build, jr
    build.build()
    return jr


def _declared(header):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:jr_status|void|const char\s*\*)\s+(jr_\w+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(L):
    lib = L.lib()
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            names += _declared(h)
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_error_string(L):
    assert "sm_103a" in L.version()
    assert isinstance(L.lib().jr_last_error(), bytes)


def _desc(L, sc, mats=None, tri_mat=None):
    mats = np.ascontiguousarray(sc.mats if mats is None else mats, np.float32)
    tm = np.ascontiguousarray(sc.tri_mat if tri_mat is None else tri_mat, np.uint32)
    v = np.ascontiguousarray(sc.verts, np.float32)
    t = np.ascontiguousarray(sc.tris, np.uint32)
    keep = (mats, tm, v, t)
    d = L.SceneDesc(v.ctypes.data, v.shape[0], t.ctypes.data, t.shape[0], tm.ctypes.data, mats.ctypes.data,
                    mats.shape[0], (ctypes.c_float * 12)(*[float(c) for c in sc.camera]))
    return d, keep


def test_invalid_scene_arguments(L):
    from paper_2409_07148_gb300 import scenes
    lib = L.lib()
    sc = scenes.cornell()
    h = ctypes.c_void_p()
    assert lib.jr_scene_create(None, None, ctypes.byref(h)) == L.JR_ERR_INVALID_ARG
    assert b"null" in lib.jr_last_error()
    bad = sc.tri_mat.copy()
    bad[3] = 99
    d, keep = _desc(L, sc, tri_mat=bad)
    assert lib.jr_scene_create(ctypes.byref(d), None, ctypes.byref(h)) == L.JR_ERR_INVALID_ARG
    assert b"material index" in lib.jr_last_error()
    m = sc.mats.copy()
    m[0, 0] = 7
    d, keep = _desc(L, sc, mats=m)
    assert lib.jr_scene_create(ctypes.byref(d), None, ctypes.byref(h)) == L.JR_ERR_INVALID_ARG
    assert b"material type" in lib.jr_last_error()
    t = sc.tris.copy()
    t[0, 0] = 10**6
    sc2 = scenes.SceneArrays("bad", sc.verts, t, sc.tri_mat, sc.mats, sc.camera, 8, 8, 1)
    d, keep = _desc(L, sc2)
    assert lib.jr_scene_create(ctypes.byref(d), None, ctypes.byref(h)) == L.JR_ERR_INVALID_ARG
    assert b"out of range" in lib.jr_last_error()
    for bad_value in (np.nan, np.inf, -np.inf):  # a triangle's vertex must be finite
        v = sc.verts.copy()
        v[sc.tris[5, 1], 2] = bad_value
        sc3 = scenes.SceneArrays("bad", v, sc.tris, sc.tri_mat, sc.mats, sc.camera, 8, 8, 1)
        d, keep = _desc(L, sc3)
        assert lib.jr_scene_create(ctypes.byref(d), None, ctypes.byref(h)) == L.JR_ERR_INVALID_ARG
        assert b"not finite" in lib.jr_last_error()


def test_invalid_chain_arguments(L):
    lib = L.lib()
    h = ctypes.c_void_p()
    p = L.make_params(8, 8, 3, n_chains=4)
    assert lib.jr_chains_create(None, ctypes.byref(p), None, ctypes.byref(h)) == L.JR_ERR_INVALID_ARG
    assert lib.jr_advance(None, 5, None) == L.JR_ERR_INVALID_ARG
    assert lib.jr_resolve(None, None, 0, None) == L.JR_ERR_INVALID_ARG
    assert lib.jr_get_stats(None, None, None) == L.JR_ERR_INVALID_ARG
    assert lib.jr_eval_states(None, None, None, 0, None, None, None, None, None, None) == L.JR_ERR_INVALID_ARG


def test_no_device_is_a_status_not_a_crash(L):
    """Without a GPU the first device call fails cleanly with JR_ERR_CUDA."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2409_07148_gb300 import scenes
    lib = L.lib()
    sc = scenes.cornell()
    d, keep = _desc(L, sc)
    h = ctypes.c_void_p()
    rc = lib.jr_scene_create(ctypes.byref(d), None, ctypes.byref(h))
    assert rc in (L.JR_ERR_CUDA, L.JR_ERR_OOM)
    assert lib.jr_last_error()


def test_failure_hooks_reject_bad_arguments(L):
    """The traversal-limit and testing-hook entry points check their arguments
    before touching the device."""
    lib = L.lib()
    assert lib.jr_chains_set_limits(None, 5, 5) == L.JR_ERR_INVALID_ARG
    assert lib.jr_debug_flow_wait(None, 1) == L.JR_ERR_INVALID_ARG
    assert lib.jr_debug_fail_alloc(-1) == L.JR_OK
    assert lib.jr_fp32_peak(None, None, None) == L.JR_ERR_INVALID_ARG
