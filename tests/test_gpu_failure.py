"""Failure detection through the C ABI (needs a GB300), each failure provoked
from the host without faulting the device.

* Traversal watchdog: a per-set node-visit budget or stack bound too small for
  the scene stops the affected rays (they count as misses), sets
  JR_STATUS_TRAVERSAL / JR_STATUS_STACK, and jr_get_stats returns
  JR_ERR_WATCHDOG with the counters filled in; in the megakernel, the
  wavefront and a batch.  The default limits never trip on the test scenes.
* Non-finite integrand: a scene whose light emits +inf gives non-finite path
  contributions; they are treated as 0, JR_STATUS_NONFINITE is set and
  jr_get_stats returns JR_ERR_NUMERIC.
* Device out of memory: the n-th allocation of a call fails (hook); the call
  returns JR_ERR_OOM, leaves its outputs untouched, frees what it had taken
  (free device memory unchanged) and the library stays usable.
* The flow kernel's bounded barrier wait: armed for more bytes than its copy
  delivers (hook), the wait runs out after its 2 s limit; the kernel sets
  JR_STATUS_FLOW_WAIT, writes no output and returns; the next launch works.
"""
import ctypes

import numpy as np
import pytest

from paper_2409_07148_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def J():
    import torch
    assert torch.cuda.is_available()
    from paper_2409_07148_gb300 import jr
    jr.lib()
    return jr


def _stats_rc(J, ch):
    lib = J.lib()
    s = J.Stats()
    rc = lib.jr_get_stats(ch.h, ctypes.byref(s), None)
    return rc, s.as_dict()


@pytest.mark.parametrize("mode", ["mega", "wave"])
def test_node_visit_budget_trips_the_watchdog(J, mode):
    sc = scenes.cornell_spheres(width=32, height=32, depth=4, n_lon=40, n_lat=21)
    g = J.Scene(sc)
    ok = J.Chains(g, 32, 32, sc.depth, 1 << 16, seed=1)
    ok.set_execution(mode)
    ok.advance(3)
    assert _stats_rc(J, ok)[0] == J.JR_OK
    ch = J.Chains(g, 32, 32, sc.depth, 1 << 16, seed=1)
    ch.set_execution(mode)
    ch.set_limits(node_visit_budget=2)
    ch.advance(3)
    rc, st = _stats_rc(J, ch)
    assert rc == J.JR_ERR_WATCHDOG, rc
    assert st["status_word"] & J.JR_STATUS_TRAVERSAL
    assert st["regenerations"] + st["local_steps"] == 3 * (1 << 16)   # the counters are still filled in
    assert b"budget" in J.lib().jr_last_error()
    img = ch.resolve()
    assert np.all(np.isfinite(img))       # stopped rays are misses, not garbage
    # a budget that the scene never needs leaves the set clean
    ch2 = J.Chains(g, 32, 32, sc.depth, 1 << 16, seed=1)
    ch2.set_execution(mode)
    ch2.set_limits(node_visit_budget=10_000)
    ch2.advance(3)
    assert _stats_rc(J, ch2)[0] == J.JR_OK


def test_stack_bound_trips_the_watchdog(J):
    sc = scenes.cornell_spheres(width=32, height=32, depth=3, n_lon=40, n_lat=21)
    g = J.Scene(sc)
    assert g.info()["bvh_depth"] > 2
    ch = J.Chains(g, 32, 32, sc.depth, 4096, seed=2)
    ch.set_limits(stack_entries=1)
    ch.advance(2)
    rc, st = _stats_rc(J, ch)
    assert rc == J.JR_ERR_WATCHDOG and st["status_word"] & J.JR_STATUS_STACK
    lib = J.lib()
    assert lib.jr_chains_set_limits(ch.h, 0, 97) == J.JR_ERR_INVALID_ARG


def test_batch_reports_each_sets_watchdog(J):
    sc = scenes.cornell_spheres(width=24, height=24, depth=3, n_lon=30, n_lat=16)
    g = J.Scene(sc)
    a = J.Chains(g, 24, 24, sc.depth, 1000, seed=3)
    b = J.Chains(g, 24, 24, sc.depth, 1000, seed=4)
    b.set_limits(node_visit_budget=2)
    bt = J.Batch([a, b])
    bt.set_block(64)
    bt.advance(2)
    assert _stats_rc(J, a)[0] == J.JR_OK
    rc, st = _stats_rc(J, b)
    assert rc == J.JR_ERR_WATCHDOG and st["status_word"] & J.JR_STATUS_TRAVERSAL


def test_non_finite_emission_is_reported(J):
    sc = scenes.cornell(width=16, height=16)
    mats = sc.mats.copy()
    lit = np.nonzero(np.any(mats[:, 4:7] > 0, axis=1))[0]
    assert len(lit) == 1
    mats[lit[0], 4:7] = np.inf
    bad = scenes.SceneArrays("cornell_inf", sc.verts, sc.tris, sc.tri_mat, mats, sc.camera, 16, 16, sc.depth)
    g = J.Scene(bad)
    for mode in ("mega", "wave"):
        ch = J.Chains(g, 16, 16, sc.depth, 1 << 16, seed=5)
        ch.set_execution(mode)
        ch.advance(4)
        rc, st = _stats_rc(J, ch)
        assert rc == J.JR_ERR_NUMERIC and st["status_word"] & J.JR_STATUS_NONFINITE, (mode, rc, st)
        x, fpu = ch.get_state()
        assert np.all(np.isfinite(fpu))           # treated as F = 0
        assert np.all(np.isfinite(ch.resolve()))


def _free():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_out_of_memory_in_every_allocation(J):
    import torch
    lib = J.lib()
    sc = scenes.cornell(width=16, height=16)
    g = J.Scene(sc)
    try:
        # jr_chains_create: 6 device allocations
        p = J.make_params(16, 16, sc.depth, n_chains=1 << 18, seed=1)
        for k in range(6):
            f0 = _free()
            h = ctypes.c_void_p(12345)
            lib.jr_debug_fail_alloc(k)
            rc = lib.jr_chains_create(g.h, ctypes.byref(p), None, ctypes.byref(h))
            lib.jr_debug_fail_alloc(-1)
            assert rc == J.JR_ERR_OOM and h.value == 12345, (k, rc)
            assert b"jr_chains_create" in lib.jr_last_error()
            assert _free() == f0, k
        # jr_scene_create: 3
        for k in range(3):
            f0 = _free()
            lib.jr_debug_fail_alloc(k)
            with pytest.raises(J.JRError) as ei:
                J.Scene(sc)
            lib.jr_debug_fail_alloc(-1)
            assert ei.value.status == J.JR_ERR_OOM
            assert _free() == f0, k
        # the wavefront buffers of a first wavefront advance: 9; the chains are untouched
        ch = J.Chains(g, 16, 16, sc.depth, 1 << 18, seed=1)
        ch.set_execution("wave")
        x0, f0s = ch.get_state()
        for k in range(9):
            m0 = _free()
            lib.jr_debug_fail_alloc(k)
            assert lib.jr_advance(ch.h, 3, None) == J.JR_ERR_OOM, k
            lib.jr_debug_fail_alloc(-1)
            assert _free() == m0, k
            x1, f1 = ch.get_state()
            assert np.array_equal(x0, x1) and np.array_equal(f0s, f1) and ch.stats()["steps_per_chain"] == 0
        ch.advance(3)                              # and then it works
        assert ch.stats()["steps_per_chain"] == 3
        # jr_flow_create: 6
        from paper_2409_07148_gb300.flowinit import init_flow_params
        perm, w = init_flow_params(8, 0)
        for k in range(6):
            m0 = _free()
            lib.jr_debug_fail_alloc(k)
            with pytest.raises(J.JRError) as ei:
                J.Flow(8, perm, w)
            lib.jr_debug_fail_alloc(-1)
            assert ei.value.status == J.JR_ERR_OOM
            assert _free() == m0, k
    finally:
        lib.jr_debug_fail_alloc(-1)
    torch.cuda.synchronize()


def test_flow_wait_runs_out_and_is_reported(J):
    import torch
    from paper_2409_07148_gb300.flowinit import init_flow_params
    lib = J.lib()
    D = 8
    perm, w = init_flow_params(D, 1)
    f = J.Flow(D, perm, w)
    x = torch.rand((D, 100), device="cuda")
    lq = torch.full((100,), float("nan"), device="cuda")
    assert lib.jr_debug_flow_wait(f.h, 1) == J.JR_OK
    try:
        rc = lib.jr_flow_log_density(f.h, ctypes.c_void_p(x.data_ptr()), 100, ctypes.c_void_p(lq.data_ptr()), None)
        assert rc == J.JR_OK
        torch.cuda.synchronize()
    finally:
        lib.jr_debug_flow_wait(f.h, 0)
    assert torch.isnan(lq).all()                  # no output written
    assert f.status() & 8                         # JR_STATUS_FLOW_WAIT
    lq2 = f.log_density(x)                        # the context is still usable
    torch.cuda.synchronize()
    assert torch.isfinite(lq2).all()
