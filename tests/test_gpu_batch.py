"""Batched advance (one persistent launch over many chain sets, optionally
replayed from a CUDA graph, with the autotuner) against per-set advances
through the C ABI (needs a GB300)."""
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


SETS = [("cornell", dict(width=16, height=16), 100, 1),
        ("cornell_spheres", dict(width=32, height=24, depth=5, n_lon=30, n_lat=16), 513, 2),
        ("glass_furnace", {}, 1000, 3),
        ("random_boxes", dict(seed=4, n_tris=2500, width=48, height=48, depth=6), 2047, 4),
        ("furnace", dict(depth=0), 64, 5),
        ("random_boxes", dict(seed=9, n_tris=9000, width=40, height=40, depth=9), 33, 6)]


def _make(J, sets=SETS):
    out = []
    for name, kw, n, seed in sets:
        sc = scenes.by_name(name, **kw)
        g = J.Scene(sc)
        out.append((sc, g, J.Chains(g, sc.width, sc.height, sc.depth, n, seed=seed, sigma=0.03)))
    return out


def _compare(a, b):
    (xa, fa), (xb, fb) = a.get_state(), b.get_state()
    same = np.all(xa == xb, axis=0)
    assert np.mean(same) >= 0.999
    assert np.allclose(fa[:, same], fb[:, same], rtol=1e-5, atol=0)
    sa, sb = a.stats(), b.stats()
    for k in ("steps_per_chain", "regenerations", "local_steps", "accepted", "status_word"):
        assert abs(sa[k] - sb[k]) <= int(1e-3 * a.n * sa["steps_per_chain"]) + 1, (k, sa[k], sb[k])
    ia, ib = a.accumulator(), b.accumulator()
    assert np.allclose(ia, ib, rtol=1e-4, atol=1e-6 * max(np.abs(ia).max(), 1e-30))


def test_batch_equals_individual_advances(J):
    ref = _make(J)
    bat = _make(J)
    for _, _, c in ref:
        c.set_execution("mega")
        c.advance(17)
    b = J.Batch([c for _, _, c in bat])
    b.set_block(64)
    b.advance(5)
    b.advance_graph(6)
    b.advance_graph(6)   # a replay continues the chains
    for (_, _, r), (_, _, c) in zip(ref, bat):
        _compare(r, c)


def test_autotune_and_interleaved_individual_advance(J):
    ref = _make(J)
    bat = _make(J)
    for _, _, c in ref:
        c.set_execution("mega")
        c.advance(5 * 2 + 3 + 2)
    b = J.Batch([c for _, _, c in bat])
    rep = b.autotune(2)                     # 5 candidates (4 block sizes, the wavefront) x 2 real steps
    assert rep["best_block"] in (0, 32, 64, 128, 256) and len(rep["ns_per_chain_step"]) == 5
    assert all(v > 0 for v in rep["ns_per_chain_step"].values())
    bat[2][2].advance(3)                    # one set moves on its own ...
    for k, (_, _, c) in enumerate(bat):     # ... the others catch up individually
        if k != 2:
            c.advance(3)
    b.advance_graph(2)                      # the batch picks up every set's step index
    for (_, _, r), (_, _, c) in zip(ref, bat):
        _compare(r, c)


def _make_shared(J):
    """SETS plus two more chain sets on the scenes of the first two (a
    distinct scene is merged once and shared)."""
    out = _make(J)
    for k, seed in ((0, 11), (1, 12)):
        sc, g, _ = out[k]
        out.append((sc, g, J.Chains(g, sc.width, sc.height, sc.depth, 300, seed=seed, sigma=0.03)))
    return out


def test_batch_wavefront_equals_individual_wavefronts(J):
    """The batched wavefront (every set in the same step and path launches,
    over the merged scene) runs each set's chains as that set's own wavefront
    advance does: the same states, and F, p, counters and images up to the
    rounding of separately compiled kernels (a contraction into an FMA may
    differ) and the order of the framebuffer's atomic sums."""
    ref = _make_shared(J)
    bat = _make_shared(J)
    for _, _, c in ref:
        c.set_execution("wave")
        c.advance(5)
        c.advance(6)
        c.advance(6)
    b = J.Batch([c for _, _, c in bat])
    b.set_block(0)
    b.advance(5)
    b.advance_graph(6)
    b.advance_graph(6)   # a replay continues the chains
    for (_, _, r), (_, _, c) in zip(ref, bat):
        _compare(r, c)


def test_batch_images_are_estimates(J):
    """Resolved images of a batched run are finite and non-negative and the
    counters add up (regenerations + local steps = chains x steps)."""
    bat = _make(J)
    b = J.Batch([c for _, _, c in bat])
    b.advance_graph(20)
    for sc, _, c in bat:
        img = c.resolve()
        st = c.stats()
        assert np.all(np.isfinite(img)) and np.all(img >= 0)
        assert st["regenerations"] + st["local_steps"] == c.n * 20


# --------------------------------------------------------------------------
# Batched chains replayed by the FP64 oracle (Alg. 2 per chain): every set of a
# batch, after a batched advance, hands a contiguous sample of its chains to
# the oracle, which takes the next step on the same Philox counters; the
# batch's next states must match except at the rounding ties and FP32 topology
# differences the single-set replay tests allow (0.5 % of the sample).
def _oracle_replay_sets(J, sets, before, after, step, m=256):
    from oracle import oracle as O
    from tests.gpu_util import oracle_state_from_gpu, rel_err, torus_diff
    worst = 1.0
    for (sc, _, c), (x, fpu), (x2, fpu2) in zip(sets, before, after):
        mm = min(m, c.n)
        first = (c.n - mm) // 2
        oc = O.Chains(O.Scene(sc, bvh=sc.n_tris > 64), sc.D, sc.width, sc.height, sigma=float(c.params.sigma),
                      seed=int(c.params.seed), chain_begin=first, n_chains=mm)
        oc.state[:] = oracle_state_from_gpu(x[:, first:first + mm], fpu[:, first:first + mm])
        oc.step = step
        oc.advance(1)
        dx = torus_diff(x2[:, first:first + mm].T, oc.state[:, :sc.D]).max(axis=1)
        ref = oc.state[:, sc.D:sc.D + 4]
        gf = fpu2[:4, first:first + mm].T
        eF = rel_err(gf, ref)
        ok = (dx <= 2e-6) & np.all((eF <= 1e-5) | ((ref == 0) & (gf == 0)), axis=1)
        worst = min(worst, float(np.mean(ok)))
        assert np.mean(ok) >= 0.995 or (mm < 200 and np.sum(~ok) <= 1), (sc.name, np.mean(ok))
    return worst


@pytest.mark.parametrize("block", [64, 0])
def test_batched_chains_replayed_by_oracle(J, block):
    """Megakernel batch (64-chain work items) and batched wavefront (block 0)."""
    bat = _make_shared(J)
    b = J.Batch([c for _, _, c in bat])
    b.set_block(block)
    b.advance(4)
    b.advance_graph(3)
    before = [c.get_state() for _, _, c in bat]
    b.advance(1)
    after = [c.get_state() for _, _, c in bat]
    _oracle_replay_sets(J, bat, before, after, step=7)


def test_batched64_workload_replayed_by_oracle(J):
    """The 64-scene workload (1k-200k triangles, 128^2-1024^2, depths 4-10, one
    chain per pixel) in the launch form the autotuner picks for it (the batched
    wavefront, replayed from a CUDA graph): after 3 graph-replayed steps every
    set's next step is replayed by the oracle on 256 sampled chains."""
    scs = scenes.batched_workload(seed=0)
    sets = []
    for sc in scs:
        g = J.Scene(sc)
        sets.append((sc, g, J.Chains(g, sc.width, sc.height, sc.depth, sc.width * sc.height, seed=0)))
    b = J.Batch([c for _, _, c in sets])
    b.set_block(0)
    b.advance_graph(3)
    before = [c.get_state() for _, _, c in sets]
    b.advance_graph(1)
    after = [c.get_state() for _, _, c in sets]
    assert all(c.stats()["status_word"] == 0 for _, _, c in sets)
    _oracle_replay_sets(J, sets, before, after, step=3)
