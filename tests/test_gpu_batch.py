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


# --------------------------------------------------------------------------
# Sets with a learned regeneration flow in the batched wavefront (the learned +
# batched configuration): the batch advances each set as the set's own
# wavefront advance with the same flow does.
def _flow_params(D, seed, sd=0.1):
    from paper_2409_07148_gb300.flowinit import init_flow_params
    perm, w = init_flow_params(D, seed)
    A = D // 2
    tail = A * 16 * 64 + A * 16
    w[:, -tail:] = np.random.default_rng(seed + 100).normal(0.0, sd, (w.shape[0], tail)).astype(np.float32)
    return perm, w


# (scene, arguments, chains, seed, beta, flow dimension: None = all D; the
# spheres set's flow models the leading 6 of its 12 coordinates)
FLOW_SETS = [("cornell", dict(width=16, height=16), 3000, 1, 0.6, None),
             ("random_boxes", dict(seed=4, n_tris=2500, width=48, height=48, depth=6), 2047, 4, None, None),
             ("cornell_spheres", dict(width=32, height=24, depth=5, n_lon=30, n_lat=16), 2500, 2, 0.3, 6),
             ("furnace", dict(depth=2), 700, 5, None, None)]


def _make_flow_sets(J):
    out = []
    for name, kw, n, seed, beta, flow_dim in FLOW_SETS:
        sc = scenes.by_name(name, **kw)
        g = J.Scene(sc)
        c = J.Chains(g, sc.width, sc.height, sc.depth, n, seed=seed, sigma=0.03)
        c.set_execution("wave")
        f = None
        if beta is not None:
            Df = flow_dim or sc.D
            perm, w = _flow_params(Df, seed)
            f = J.Flow(Df, perm, w)
            J.set_flow(c, f, beta)
        out.append((sc, g, c, f))
    return out


def test_batched_wavefront_with_flows_equals_individual_advances(J):
    ref = _make_flow_sets(J)
    bat = _make_flow_sets(J)
    for _, _, c, _ in ref:
        c.advance(4)
        c.advance(5)
        c.advance(5)
    b = J.Batch([c for _, _, c, _ in bat])
    lib = J.lib()
    assert lib.jr_batch_set_block(b.h, 64) == J.JR_ERR_STATE       # flows run in the batched wavefront only
    b.advance(4)
    b.advance_graph(5)
    b.advance_graph(5)
    for (_, _, r, _), (_, _, c, _) in zip(ref, bat):
        _compare(r, c)
        assert c.stats()["status_word"] == 0


def test_flow_attached_after_the_batch_was_built(J):
    """A set gets its flow after jr_batch_create: the batch picks the new
    regeneration density up (its descriptor and graph are renewed)."""
    sets = [("cornell", dict(width=16, height=16), 3000, 1, 0.6),
            ("random_boxes", dict(seed=4, n_tris=2500, width=48, height=48, depth=6), 2047, 4, None)]
    mk = []
    for name, kw, n, seed, beta in sets:
        sc = scenes.by_name(name, **kw)
        g = J.Scene(sc)
        mk.append((sc, g, J.Chains(g, sc.width, sc.height, sc.depth, n, seed=seed, sigma=0.03),
                   J.Chains(g, sc.width, sc.height, sc.depth, n, seed=seed, sigma=0.03)))
    for sc, _, r, c in mk:
        r.set_execution("wave")
        c.set_execution("wave")
    b = J.Batch([c for _, _, _, c in mk])
    b.set_block(0)
    b.advance_graph(3)
    for _, _, r, _ in mk:
        r.advance(3)
    sc0 = mk[0][0]
    perm, w = _flow_params(sc0.D, 1)
    fr, fc = J.Flow(sc0.D, perm, w), J.Flow(sc0.D, perm, w)
    J.set_flow(mk[0][2], fr, 0.6)
    J.set_flow(mk[0][3], fc, 0.6)
    b.advance_graph(3)             # the old graph had no flow launches
    for _, _, r, c in mk:          # each reference catches up with its batched twin
        r.advance(c.stats()["steps_per_chain"] - r.stats()["steps_per_chain"])
    for _, _, r, c in mk:
        _compare(r, c)


def test_batched_flow_set_replayed_by_oracle(J):
    """One batched step of the flow set, replayed by the oracle's Alg. 2 with
    the FP64 flow (u = beta q + 1 - beta) from the GPU's state."""
    from oracle import learned as LR
    from oracle import oracle as O
    bat = _make_flow_sets(J)
    b = J.Batch([c for _, _, c, _ in bat])
    b.advance_graph(4)
    sc, _, ch, f = bat[0]
    x, fpu = ch.get_state()
    st = ch.stats()
    b.advance_graph(1)
    x2, fpu2 = ch.get_state()
    perm, w = _flow_params(sc.D, 1)
    osc = O.Scene(sc)
    F_of = lambda xx: O.eval_states(osc, xx)[0]
    oc = LR.LearnedChains(F_of, sc.D, sc.width, sc.height, perm, w, beta=0.6, sigma=float(ch.params.sigma), seed=1,
                          n_chains=ch.n)
    oc.x = x.T.astype(np.float64)
    oc.F = fpu[:3].T.astype(np.float64)
    oc.p = fpu[3].astype(np.float64)
    oc.u = fpu[4].astype(np.float64)
    oc.step = st["steps_per_chain"]
    oc.advance(1)
    dx = np.abs(x2.T - oc.x)
    dx = np.minimum(dx, 1 - dx).max(axis=1)
    assert np.mean(dx <= 1e-4) >= 0.97, np.mean(dx <= 1e-4)
    same = (dx <= 1e-4) & (fpu2[3] > 0)
    assert np.mean(np.abs(fpu2[4][same] - oc.u[same]) <= 3e-3 * oc.u[same]) >= 0.98
