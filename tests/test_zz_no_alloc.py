"""jr_advance_static: the advance for callers that may not allocate device memory.

Some callers cannot call cudaMalloc when they advance the chains: a host
framework that owns all device memory and forbids allocation in its execute
step, or a loop that cannot afford cudaMalloc/cudaFree (allocator locks, and
a device-wide synchronisation for cudaFree).  jr_advance_static serves them:
the wavefront launches of jr_advance with their scratch in a fixed array
inside the library.  These tests call it through the C ABI and check it
against jr_advance (wavefront mode) on the same chains, two calls in a row,
with the tolerances the other parity tests use.  The file is named so that
pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

REL = 1e-5


def _compare(a, b):
    """jr_advance_static runs the wavefront kernels of jr_advance on the same
    Philox counters, so states, cached F/p/u and counters are bit-identical.
    Only the framebuffer is summed by float atomics in an order that varies from
    run to run, so the accumulator and the image agree to rounding."""
    (xa, fa), (xb, fb) = a.get_state(), b.get_state()
    assert np.array_equal(xa, xb)
    assert np.array_equal(fa, fb)
    sa, sb = a.stats(), b.stats()
    for k in ("steps_per_chain", "regenerations", "local_steps", "accepted", "status_word"):
        assert sa[k] == sb[k], (k, sa[k], sb[k])
    acc_a, acc_b = a.accumulator(), b.accumulator()
    assert np.allclose(acc_a, acc_b, rtol=REL, atol=1e-6 * np.abs(acc_a).max())
    ia, ib = a.resolve(), b.resolve()
    assert np.allclose(ia, ib, rtol=REL, atol=1e-6 * np.abs(ia).max())


@pytest.mark.parametrize("name,kw,n", [("cornell", {}, 4099),
                                       ("cornell_spheres", dict(width=64, height=64, depth=6, n_lon=40, n_lat=21),
                                        65536)])
def test_advance_static_matches_advance_two_calls(name, kw, n):
    import torch
    assert torch.cuda.is_available()
    from paper_2409_07148_gb300 import jr, scenes
    lib = jr.lib()
    sc = scenes.by_name(name, **kw)
    g = jr.Scene(sc)
    ref = jr.Chains(g, sc.width, sc.height, sc.depth, n, seed=21, sigma=0.02)
    ref.set_execution("wave")
    fixed = jr.Chains(g, sc.width, sc.height, sc.depth, n, seed=21, sigma=0.02)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        ref.advance(9)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        rc = lib.jr_advance_static(fixed.h, 9, ctypes.c_void_p(stream.cuda_stream))
        assert rc == jr.JR_OK, lib.jr_last_error()
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        # the call allocated nothing on the device (on the first call too: the
        # scratch array was set up when the chain sets were created)
        assert free1 == free0, (free0, free1)
        _compare(ref, fixed)


def test_advance_static_rejects_more_chains_than_its_scratch():
    import torch
    assert torch.cuda.is_available()
    from paper_2409_07148_gb300 import jr, scenes
    lib = jr.lib()
    sc = scenes.cornell(width=8, height=8)
    ch = jr.Chains(jr.Scene(sc), 8, 8, sc.depth, jr.STATIC_MAX_CHAINS + 1, seed=1)
    x0, _ = ch.get_state()
    rc = lib.jr_advance_static(ch.h, 3, None)
    assert rc == jr.JR_ERR_INVALID_ARG
    msg = lib.jr_last_error().decode()
    assert "65536" in msg and "jr_advance" in msg
    x1, _ = ch.get_state()
    assert np.array_equal(x0, x1) and ch.stats()["steps_per_chain"] == 0   # nothing was launched
