"""GPU parity of the MH baseline "Metropolis" (JR_FLAG_MH) against the FP64
oracle's MH chains, through the C ABI (needs a GB300).

The baseline is the paper's reference algorithm (Section 8, practical
pairing): Alg. 1 with the mixture proposal l mu + (1 - l) zeta of Section 5,
l = 0.3, estimation after a burn-in (Section 9).  Tolerances are the Restore
parity tests': on identical Philox counters the large-step choice and the splat
pixel agree exactly (up to a pixel boundary within FP32 rounding), the MH
decision agrees except where U_a p(x) and p(y) tie to FP32 rounding or the FP32
path hits another triangle than the FP64 one, and accepted next states agree
to 2e-6 in x and 1e-5 relative in F and p.
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_07148_gb300 import scenes
from tests.gpu_util import oracle_state_from_gpu, rel_err, torus_diff

pytestmark = pytest.mark.gpu

REL = 1e-5
ELL = float(np.float32(0.3))   # the library holds l in float32; the oracle compares U_s with the same value
EPS = 1e-2


@pytest.fixture(scope="module")
def J():
    import torch
    assert torch.cuda.is_available()
    from paper_2409_07148_gb300 import jr
    jr.lib()
    return jr


def _mh(J, g, sc, n, seed, burn_in, sigma=0.01, mode=None, chain_offset=0, stream=None):
    ch = J.Chains(g, sc.width, sc.height, sc.depth, n, seed=seed, sigma=sigma, flags=J.JR_FLAG_MH, large_step=ELL,
                  burn_in=burn_in, chain_offset=chain_offset, stream=stream)
    if mode:
        ch.set_execution(mode)
    return ch


def _replay_mh(J, sc, osc, n, n_steps, seed, burn_in, sigma=0.01):
    """One GPU step at a time (megakernel, traced); before each step the
    oracle gets the GPU's state and takes the same step on the same counters."""
    import torch
    g = J.Scene(sc)
    ch = _mh(J, g, sc, n, seed, burn_in, sigma)
    oc = O.MHChains(osc, sc.D, sc.width, sc.height, sigma=sigma, ell=ELL, burn_in=burn_in, seed=seed, n_chains=n)
    fl = torch.empty(n, dtype=torch.uint8, device="cuda")
    dt = torch.empty(n, dtype=torch.float32, device="cuda")
    px = torch.empty(n, dtype=torch.int32, device="cuda")
    summ = dict(steps=0, checked=0, accept_flip=0, topo=0, pix_flip=0)
    x, fpu = ch.get_state()
    for s in range(n_steps):
        oc.state[:] = oracle_state_from_gpu(x, fpu)
        oc.step = s
        tr = oc.advance(1, trace=True, margins=True)
        ch.advance_traced(1, fl, dt, px)
        x2, fpu2 = ch.get_state()
        gf, gdt, gpx = fl.cpu().numpy(), dt.cpu().numpy(), px.cpu().numpy()
        of, opx, om = tr["flags"][:, 0], tr["pix"][:, 0], tr["margin"][:, 0]
        assert np.array_equal(gf & 1, of & 1), "large-step choice differs"
        # the splat: the held state's pixel once the burn-in is over, nothing before
        if s < burn_in:
            assert np.all(gpx == -1) and np.all(gdt == 0) and np.all(opx == -1)
        else:
            assert np.array_equal(gpx >= 0, opx >= 0)
            assert np.all(gdt[gpx >= 0] == 1.0)
            pflip = gpx != opx
            summ["pix_flip"] += int(pflip.sum())
            if pflip.any():
                xw = x[0, pflip].astype(np.float64) * sc.width
                yh = x[1, pflip].astype(np.float64) * sc.height
                assert np.all((np.abs(xw - np.round(xw)) < 1e-4) | (np.abs(yh - np.round(yh)) < 1e-4))
        same = (gf & 2) == (of & 2)
        flip = ~same
        if flip.any():
            near = np.abs(om[flip]) <= 1e-4 * (fpu[3, flip].astype(np.float64) + 1e-30)
            summ["accept_flip"] += int(flip.sum())
            summ["topo"] += int((~near).sum())
        dx = torus_diff(x2[:, same].T, oc.state[same, :sc.D]).max(axis=1)
        assert np.all(dx <= 2e-6), dx.max()
        ref = oc.state[same, sc.D:sc.D + 4]
        eF = rel_err(fpu2[:4, same].T, ref)
        nz = ref != 0
        bad = np.any((eF > REL) & nz, axis=1) | np.any((fpu2[:4, same].T != 0) & ~nz, axis=1)
        summ["topo"] += int(bad.sum())
        summ["checked"] += int(same.sum())
        summ["steps"] += n
        x, fpu = x2, fpu2
    return summ, ch, oc


@pytest.mark.parametrize("name,kw,bvh,n,steps,burn", [("cornell", {}, False, 512, 40, 12),
                                                      ("cornell_spheres", dict(width=64, height=64, depth=4,
                                                                               n_lon=32, n_lat=17), True, 256, 24, 5)])
def test_mh_step_replay(J, name, kw, bvh, n, steps, burn):
    sc = scenes.by_name(name, **kw)
    s, ch, oc = _replay_mh(J, sc, O.Scene(sc, bvh=bvh), n, steps, seed=4, burn_in=burn)
    assert s["checked"] >= 0.99 * s["steps"], s
    assert s["topo"] <= 5e-3 * s["steps"], s
    assert s["accept_flip"] <= 5e-3 * s["steps"], s
    st = ch.stats()
    # the large-step proposals are the same uniform draws on both sides: their
    # count is exact and the sum of their p agrees to FP32 accuracy
    assert st["regenerations"] == oc.n_large and st["local_steps"] == oc.n_small
    assert abs(st["p_sum_large"] - oc.p_sum_large) <= 1e-4 * oc.p_sum_large
    assert abs(st["accepted"] - oc.accepts) <= s["accept_flip"]


@pytest.mark.parametrize("name,kw,n", [("cornell", {}, 4099),
                                       ("cornell_spheres", dict(width=128, height=128, depth=6, n_lon=40, n_lat=21),
                                        8192)])
def test_mh_wavefront_equals_megakernel(J, name, kw, n):
    sc = scenes.by_name(name, **kw)
    g = J.Scene(sc)
    out = []
    for mode in ("mega", "wave"):
        ch = _mh(J, g, sc, n, 13, burn_in=4, sigma=0.02, mode=mode)
        ch.advance(7)
        ch.advance(5)
        out.append((ch.get_state(), ch.stats(), ch.accumulator(), ch.resolve()))
    (xa, fa), sa, aa, ia = out[0]
    (xb, fb), sb, ab, ib = out[1]
    same = np.all(xa == xb, axis=0)
    assert np.mean(same) >= 0.999, np.mean(same)
    assert np.allclose(fa[:, same], fb[:, same], rtol=1e-6, atol=0)
    assert sa["regenerations"] == sb["regenerations"] and sa["local_steps"] == sb["local_steps"]
    assert abs(sa["accepted"] - sb["accepted"]) <= max(2, int(1e-3 * n * 12))
    assert abs(sa["p_sum_large"] - sb["p_sum_large"]) <= 1e-3 * abs(sa["p_sum_large"])
    assert abs(aa[..., 3].sum() - ab[..., 3].sum()) <= 1e-3 * aa[..., 3].sum()
    assert np.allclose(ia.sum(), ib.sum(), rtol=1e-2)


def test_mh_static_advance_equals_wavefront(J):
    """jr_advance_static runs the MH chains of jr_advance's wavefront bit for bit."""
    import torch
    sc = scenes.cornell()
    g = J.Scene(sc)
    a = _mh(J, g, sc, 5000, 3, burn_in=2, mode="wave")
    b = _mh(J, g, sc, 5000, 3, burn_in=2)
    for _ in range(2):
        a.advance(6)
        b.advance_static(6)
        torch.cuda.synchronize()
        (xa, fa), (xb, fb) = a.get_state(), b.get_state()
        assert np.array_equal(xa, xb) and np.array_equal(fa, fb)
        sa, sb = a.stats(), b.stats()
        for k in ("regenerations", "local_steps", "accepted"):
            assert sa[k] == sb[k]


def test_mh_full_size_wavefront_step_sampled(J):
    """The 40k-triangle scene at 512^2, depth 8, 2^20 MH chains in the
    wavefront (the bench's launch configuration): after 3 steps a contiguous
    sample of 2048 chains goes to the oracle, which takes the 4th step on the
    same counters."""
    sc = scenes.cornell_spheres()
    n, k, first, m = 1 << 20, 3, 654_321, 2048
    ch = _mh(J, J.Scene(sc), sc, n, 0, burn_in=2)
    ch.advance(k)
    x, fpu = ch.get_state()
    ch.advance(1)
    x2, fpu2 = ch.get_state()
    oc = O.MHChains(O.Scene(sc, bvh=True), sc.D, sc.width, sc.height, ell=ELL, burn_in=2, seed=0, chain_begin=first,
                    n_chains=m)
    oc.state[:] = oracle_state_from_gpu(x[:, first:first + m], fpu[:, first:first + m])
    oc.step = k
    oc.advance(1)
    dx = torus_diff(x2[:, first:first + m].T, oc.state[:, :sc.D]).max(axis=1)
    ref = oc.state[:, sc.D:sc.D + 4]
    gf = fpu2[:4, first:first + m].T
    eF = rel_err(gf, ref)
    ok = (dx <= 2e-6) & np.all((eF <= REL) | ((ref == 0) & (gf == 0)), axis=1)
    assert np.mean(ok) >= 0.995, np.mean(ok)
    assert ch.stats()["status_word"] == 0


def _gpu_mh_batches(J, sc, n_batches, chains, steps, seed, burn_in, first_chain=0):
    import torch
    g = J.Scene(sc)
    sets, streams = [], []
    for b in range(n_batches):
        s = torch.cuda.Stream()
        c = _mh(J, g, sc, chains, seed, burn_in, chain_offset=first_chain + b * chains, stream=s)
        c.advance(steps, stream=s)
        sets.append(c)
        streams.append(s)
    torch.cuda.synchronize()
    imgs = np.array([c.resolve(stream=s) for c, s in zip(sets, streams)], np.float64)
    for c, s in zip(sets, streams):
        assert c.stats(stream=s)["status_word"] == 0
    return imgs


def test_mh_cornell_paired_streams_match_oracle(J):
    """Identical Philox streams: the GPU's MH images equal the oracle's up to
    FP32 rounding, except where a chain diverged at a tie (an accepted large
    step brings the two copies together again)."""
    sc = scenes.cornell()
    osc = O.Scene(sc)
    g = _gpu_mh_batches(J, sc, 8, 256, 1500, seed=3, burn_in=200)
    o = []
    for b in range(8):
        oc = O.MHChains(osc, sc.D, sc.width, sc.height, ell=ELL, burn_in=200, seed=3, chain_begin=256 * b,
                        n_chains=256)
        oc.advance(1500)
        o.append(oc.image())
    o = np.array(o)
    se = np.sqrt(o.var(0, ddof=1) / len(o))
    d = np.abs(g.mean(0) - o.mean(0))
    ok = se > 0
    assert np.all(d[~ok] < 1e-6)
    r = d[ok] / se[ok]
    assert np.median(r) < 2e-2
    assert np.max(r) < 4.0


@pytest.fixture(scope="module")
def reference(J):
    """Converged plain path tracing of the 64x64 Cornell box on the GPU
    (2^32 samples), the reference of the Restore image tests."""
    import torch
    sc = scenes.cornell()
    acc = torch.zeros((sc.height, sc.width, 4), dtype=torch.float64, device="cuda")
    n, chunk = 1 << 32, 1 << 28
    g = J.Scene(sc)
    for s0 in range(0, n, chunk):
        J.render_pt(g, sc.width, sc.height, sc.depth, chunk, seed=123, sample_begin=s0, accum=acc)
    torch.cuda.synchronize()
    return sc, (acc[..., :3] / n).cpu().numpy()


def test_mh_cornell_per_pixel_vs_converged_reference(J, reference):
    """Independent MH batches (burn-in 10^4 as in Section 9) scatter about the
    converged reference as their standard errors say: per pixel within 4 sigma
    (0.1 % budget), and the pooled image's relMSE is small."""
    from scipy import stats
    sc, ref = reference
    imgs = _gpu_mh_batches(J, sc, 32, 2048, 16_000, seed=17, burn_in=10_000, first_chain=1 << 22)
    img = imgs.mean(0)
    se = imgs.std(0, ddof=1) / np.sqrt(len(imgs))
    ok = se > 0
    t = (img - ref)[ok] / se[ok]
    z = np.sign(t) * stats.norm.isf(stats.t.sf(np.abs(t), len(imgs) - 1))
    assert np.mean(np.abs(z) > 4) <= 1e-3, np.sort(np.abs(z))[-8:]
    assert 0.6 < np.mean(z ** 2) < 1.6, np.mean(z ** 2)
    e = float(np.mean((img - ref) ** 2 / (ref ** 2 + EPS)))
    assert e <= 2e-3, e


def test_mh_api_refusals(J):
    sc = scenes.cornell(width=8, height=8)
    g = J.Scene(sc)
    lib = J.lib()
    h = ctypes.c_void_p()
    p = J.make_params(8, 8, sc.depth, n_chains=4, flags=J.JR_FLAG_MH | J.JR_FLAG_RAO_BLACKWELL, large_step=0.3)
    assert lib.jr_chains_create(g.h, ctypes.byref(p), None, ctypes.byref(h)) == J.JR_ERR_INVALID_ARG
    p = J.make_params(8, 8, sc.depth, n_chains=4, flags=J.JR_FLAG_MH, large_step=1.5)
    assert lib.jr_chains_create(g.h, ctypes.byref(p), None, ctypes.byref(h)) == J.JR_ERR_INVALID_ARG
    p = J.make_params(8, 8, sc.depth, n_chains=4, flags=8)
    assert lib.jr_chains_create(g.h, ctypes.byref(p), None, ctypes.byref(h)) == J.JR_ERR_INVALID_ARG
    ch = _mh(J, g, sc, 64, 1, burn_in=0)
    assert lib.jr_complete_tours(ch.h, 10, None, None) == J.JR_ERR_STATE
    assert lib.jr_chains_set_flow(ch.h, None, ctypes.c_float(0.0), 10, None, None) == J.JR_ERR_STATE
    # before the burn-in ends the image is zero; the counters still move
    ch2 = _mh(J, g, sc, 64, 1, burn_in=50)
    ch2.advance(10)
    assert np.all(ch2.resolve() == 0) and ch2.accumulator()[..., 3].sum() == 0
    st = ch2.stats()
    assert st["regenerations"] + st["local_steps"] == 640
