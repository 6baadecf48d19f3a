"""The regeneration flow on the GPU (tensor-core MLP) against the FP64 flow
oracle, and Jump Restore chains with a learned mixture mu (needs a GB300).

Tolerance (derived from the arithmetic): the MLP operands are bf16 on both
sides, but the GPU accumulates in FP32 and runs the couplings in FP32 while the
oracle works exactly, so the two agree to FP32 rounding -- |log q_gpu -
log q_oracle| <= 1e-5 (1.5e-5 at D = 32, whose 96 per-coordinate log terms add
their roundings) -- except where the rounding decides a discrete step: the bf16
rounding of an activation (a 2^-8 relative step) or the bin of a coordinate
(the density jumps there).  The oracle reports, per row, the distance of every
such value to its edge in units of the GPU's FP32 error (oracle.flow's rounding
margins); every row that differs by more than the tolerance must have a margin
below 1, and such rows must be rare.
"""
TOL = {2: 1e-5, 8: 1e-5, 18: 1e-5, 22: 1e-5, 26: 1e-5, 32: 1.5e-5}
FLIP_BUDGET = 0.02   # share of rows allowed to take the other side of an edge


def _check_rows(d, margin, tol):
    """d: per-row disagreement; margin: the oracle's rounding margin."""
    off = d > tol
    assert np.all(margin[off] < 1.0), (np.sort(d[off & (margin >= 1.0)])[-5:], np.sort(margin[off])[-5:])
    assert np.mean(off) <= FLIP_BUDGET, np.mean(off)
    return float(np.mean(off)), float(np.mean(margin < 1.0))
import numpy as np
import pytest

from oracle import flow as FL
from oracle import learned as LR
from oracle import oracle as O
from paper_2409_07148_gb300 import scenes
from paper_2409_07148_gb300.flowinit import init_flow_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def J():
    import torch
    assert torch.cuda.is_available()
    from paper_2409_07148_gb300 import jr
    jr.lib()
    return jr


def _flow(D, seed, sd):
    perm, w = init_flow_params(D, seed)
    A = D // 2
    tail = A * 16 * 64 + A * 16
    w[:, -tail:] = np.random.default_rng(seed + 100).normal(0.0, sd, (w.shape[0], tail)).astype(np.float32)
    return perm, w


@pytest.mark.parametrize("D,n", [(2, 100), (8, 10007), (18, 4096), (22, 5000), (32, 3000)])
def test_log_density_matches_oracle(J, D, n):
    import torch
    perm, w = _flow(D, D, 0.1)
    f = J.Flow(D, perm, w)
    x = np.random.default_rng(D).random((n, D)).astype(np.float32)
    lq = f.log_density(torch.from_numpy(np.ascontiguousarray(x.T)).cuda()).cpu().numpy()
    lo, _ = FL.log_density(perm, w, x.astype(np.float64))
    d = np.abs(lq.astype(np.float64) - lo)
    assert np.isfinite(lq).all()
    _check_rows(d, FL.log_density_margin(perm, w, x.astype(np.float64)), TOL[D])


@pytest.mark.parametrize("D,n", [(8, 4099), (22, 5000)])
def test_sampling_matches_oracle_and_inverts(J, D, n):
    import torch
    perm, w = _flow(D, D + 1, 0.1)
    f = J.Flow(D, perm, w)
    z = np.random.default_rng(D + 7).random((n, D)).astype(np.float32)
    t = torch.from_numpy(np.ascontiguousarray(z.T)).cuda()
    lq = f.sample(t).cpu().numpy()
    x = t.cpu().numpy().T
    xo, lqo = FL.sample(perm, w, z.astype(np.float64))
    d = np.maximum(np.abs(x.astype(np.float64) - xo).max(axis=1), np.abs(lq.astype(np.float64) - lqo))
    _check_rows(d, FL.sample_margin(perm, w, z.astype(np.float64)), TOL[D])
    # GPU round trip: the density direction gives back the sampling log-density
    lq2 = f.log_density(torch.from_numpy(np.ascontiguousarray(x.T)).cuda()).cpu().numpy()
    d2 = np.abs(lq2.astype(np.float64) - lq)
    m2 = np.minimum(FL.log_density_margin(perm, w, x.astype(np.float64)), FL.sample_margin(perm, w, z.astype(np.float64)))
    _check_rows(d2, m2, 2 * TOL[D])


def test_params_round_trip(J):
    perm, w = _flow(10, 3, 0.2)
    f = J.Flow(10, perm, w)
    assert np.array_equal(f.get_params(), w.ravel())
    w2 = w * 0.5
    f.set_params(w2)
    assert np.array_equal(f.get_params(), w2.ravel())


@pytest.mark.parametrize("flow_dim", [None, 4])
def test_chains_with_flow_step_replay(J, flow_dim):
    """One step of chains with u = beta q + 1 - beta, replayed by the oracle's
    Alg. 2 with the FP64 flow from the GPU's own state.  flow_dim = 4: the flow
    models coordinates 0..3 of the 8 (the rest uniform), u = beta q(x[:4]) +
    1 - beta."""
    sc = scenes.cornell(width=16, height=16, depth=3)
    Df = flow_dim or sc.D
    perm, w = _flow(Df, 5, 0.1)
    g = J.Scene(sc)
    f = J.Flow(Df, perm, w)
    ch = J.Chains(g, 16, 16, sc.depth, 512, seed=3, sigma=0.02)
    J.set_flow(ch, f, 0.6)
    ch.advance(4)
    x, fpu = ch.get_state()
    st = ch.stats()
    osc = O.Scene(sc)
    F_of = lambda xx: O.eval_states(osc, xx)[0]
    oc = LR.LearnedChains(F_of, sc.D, 16, 16, perm, w, beta=0.6, sigma=0.02, seed=3, n_chains=512)
    oc.x = x.T.astype(np.float64)
    oc.F = fpu[:3].T.astype(np.float64)
    oc.p = fpu[3].astype(np.float64)
    oc.u = fpu[4].astype(np.float64)
    oc.step = st["steps_per_chain"]
    # u of the GPU state is the flow's density (up to the tolerance above)
    # wherever p > 0; at p = 0 the killing rate is +inf whatever u is, and the
    # chains keep u = 1 there without evaluating the flow
    u_o = FL.regen_density(perm, w, oc.x[:, :Df], 0.6)
    pos = fpu[3] > 0
    assert pos.sum() >= 20
    # u = beta q + 1 - beta at each state with p > 0, to 1e-5 relative off the edges
    du = np.abs(fpu[4][pos] - u_o[pos]) / u_o[pos]
    _check_rows(du, FL.log_density_margin(perm, w, oc.x[pos][:, :Df]), 1e-5)
    assert np.all(fpu[4][~pos] == 1.0)
    oc.advance(1)
    ch.advance(1)
    x2, fpu2 = ch.get_state()
    dx = np.abs(x2.T - oc.x)
    dx = np.minimum(dx, 1 - dx).max(axis=1)
    assert np.mean(dx <= 1e-4) >= 0.97       # decisions and flow draws agree except near ties / bin edges
    # u at every new state with p > 0, against the oracle's density of the GPU's own state
    pos2 = fpu2[3] > 0
    xs2 = x2.T[pos2].astype(np.float64)[:, :Df]
    u2 = FL.regen_density(perm, w, xs2, 0.6)
    _check_rows(np.abs(fpu2[4][pos2] - u2) / u2, FL.log_density_margin(perm, w, xs2), 1e-5)


@pytest.mark.parametrize("flow_dim", [None, 4])
def test_learned_mixture_image_is_unbiased(J, flow_dim):
    """With a non-trivial flow (beta = 0.7) the Jump Restore image converges to
    the same pixels as with uniform regeneration (per-pixel z over batches);
    flow_dim = 4: a flow over the leading 4 of the 8 coordinates."""
    from scipy import stats
    import torch
    sc = scenes.cornell(width=32, height=32, depth=3)
    Df = flow_dim or sc.D
    perm, w = _flow(Df, 9, 0.1)
    g = J.Scene(sc)
    f = J.Flow(Df, perm, w)
    a, b = [], []
    for k in range(16):
        c1 = J.Chains(g, 32, 32, sc.depth, 16384, seed=1, chain_offset=16384 * k)
        J.set_flow(c1, f, 0.7)
        c1.advance(300)
        assert J.complete_tours(c1) == 0     # no open tour left: the completed-tour estimator
        a.append(c1.resolve())
        c2 = J.Chains(g, 32, 32, sc.depth, 16384, seed=2, chain_offset=16384 * k)
        c2.set_execution("wave")
        c2.advance(300)
        assert J.complete_tours(c2) == 0
        b.append(c2.resolve())
        assert c1.stats()["status_word"] == 0
    a, b = np.array(a, np.float64), np.array(b, np.float64)
    va, vb = a.var(0, ddof=1) / len(a), b.var(0, ddof=1) / len(b)
    ok = (va + vb) > 0
    t = (a.mean(0) - b.mean(0))[ok] / np.sqrt((va + vb)[ok])
    z = np.sign(t) * stats.norm.isf(stats.t.sf(np.abs(t), 2 * len(a) - 2))
    assert np.mean(np.abs(z) > 4) <= 2e-3
    assert 0.6 < np.mean(z ** 2) < 1.6


@pytest.mark.parametrize("beta,flow_dim", [(0.0, None), (0.6, None), (0.6, 4)])
def test_complete_tours_paired_with_oracle(J, beta, flow_dim):
    """Identical Philox streams: GPU chains (wavefront, learned mixture or
    uniform) advanced, drained until every tour ends, and restarted, against
    the oracle's Alg. 2 doing the same from the same initial states."""
    sc = scenes.cornell(width=8, height=8, depth=3)
    Df = flow_dim or sc.D
    perm, w = _flow(Df, 13, 0.1)
    g = J.Scene(sc)
    ch = J.Chains(g, 8, 8, sc.depth, 2048, seed=4, sigma=0.02)
    ch.set_execution("wave")
    osc = O.Scene(sc)
    F_of = lambda xx: O.eval_states(osc, xx)[0]
    oc = LR.LearnedChains(F_of, sc.D, 8, 8, beta=0.0, sigma=0.02, seed=4, n_chains=2048)
    if beta:
        f = J.Flow(Df, perm, w)
        J.set_flow(ch, f, beta)
        oc.set_flow(perm, w, beta)
    ch.advance(6)
    oc.advance(6)
    s_gpu, s_orc = ch.stats()["steps_per_chain"], oc.step
    assert J.complete_tours(ch) == 0 and oc.complete_tours() == 0
    st = ch.stats()
    # the drain runs in groups of launches, but counts the steps a drain checked after
    # every step takes (the oracle's); only a rare tie can change the longest tour
    assert abs((st["steps_per_chain"] - s_gpu) - (oc.step - s_orc)) <= 2
    assert abs(st["regenerations"] - oc.J) <= 0.01 * oc.J
    ga, oa = ch.accumulator(), oc.accum
    rel = np.abs(ga - oa).sum() / np.abs(oa).sum()
    assert rel < 0.02, rel                 # identical streams; only rare ties and FP32/bf16 differences diverge
    x, fpu = ch.get_state()                # the restart drew the same new states
    same = np.all(np.abs(x.T - oc.x) <= 1e-4, axis=1)
    assert np.mean(same) >= 0.98


@pytest.mark.parametrize("flow_dim", [None, 8])
def test_full_size_learned_step_sampled(J, flow_dim):
    """The learned-regeneration workload at full size: the slit caustic
    (80k triangles, glass, 1024^2, depth 10, D = 22), 2^20 chains in the
    wavefront with a non-trivial flow (beta = 0.3).  A contiguous sample of
    2048 chains is handed to the oracle's Alg. 2 with the same flow before a
    step; the next states agree except near ties and bin edges (the
    tolerance of the small replay above).  flow_dim = 8: the flow over the
    leading 8 of the 22 coordinates that the time-to-relMSE harness uses."""
    sc = scenes.caustic_slit()
    Df = flow_dim or sc.D
    perm, w = _flow(Df, 17, 0.1)
    g = J.Scene(sc)
    f = J.Flow(Df, perm, w)
    n, first, m = 1 << 20, 700_000, 2048
    ch = J.Chains(g, sc.width, sc.height, sc.depth, n, seed=2)
    J.set_flow(ch, f, 0.3)
    ch.advance(3)
    x, fpu = ch.get_state()
    step = ch.stats()["steps_per_chain"]
    ch.advance(1)
    x2, fpu2 = ch.get_state()
    osc = O.Scene(sc, bvh=True)
    F_of = lambda xx: O.eval_states(osc, xx)[0]
    oc = LR.LearnedChains(F_of, sc.D, sc.width, sc.height, perm, w, beta=0.3, seed=2, chain_begin=first,
                          n_chains=m)
    sl = slice(first, first + m)
    oc.x = x[:, sl].T.astype(np.float64)
    oc.F = fpu[:3, sl].T.astype(np.float64)
    oc.p = fpu[3, sl].astype(np.float64)
    oc.u = fpu[4, sl].astype(np.float64)
    oc.step = step
    oc.advance(1)
    dx = np.abs(x2[:, sl].T - oc.x)
    dx = np.minimum(dx, 1 - dx).max(axis=1)
    assert np.mean(dx <= 1e-4) >= 0.97, np.mean(dx <= 1e-4)
    # u at the new lit states (rare here: all of the 2^20 chains' are checked), against
    # the oracle's density of the GPU's own state, to 1e-5 off the rounding edges
    pos2 = fpu2[3] > 0
    if pos2.any():
        xs2 = x2.T[pos2].astype(np.float64)[:, :Df]
        u2 = FL.regen_density(perm, w, xs2, 0.3)
        _check_rows(np.abs(fpu2[4][pos2] - u2) / u2, FL.log_density_margin(perm, w, xs2), 1e-5)
    assert ch.stats()["status_word"] == 0


def test_flow_dimension_is_checked(J):
    """A flow covers all D coordinates or a leading block of at least 4 (the
    path's start record); anything else is an argument error."""
    sc = scenes.cornell(width=8, height=8, depth=3)     # D = 8
    g = J.Scene(sc)
    ch = J.Chains(g, 8, 8, sc.depth, 64, seed=1)
    for Df in (2, 10):
        perm, w = _flow(Df, 3, 0.1)
        f = J.Flow(Df, perm, w)
        with pytest.raises(J.JRError) as e:
            J.set_flow(ch, f, 0.5)
        assert "dimension" in str(e.value)
    perm, w = _flow(6, 3, 0.1)
    f6 = J.Flow(6, perm, w)
    J.set_flow(ch, f6, 0.5)
    ch.advance(2)
    assert ch.stats()["status_word"] == 0
