"""Image-level parity of the GPU Jump Restore estimator (needs a GB300).

Two kinds of comparison:

* paired -- the GPU and the oracle draw identical Philox streams (same seed,
  same chain / sample ids), so their images agree sample for sample up to
  FP32 rounding, decision ties and rare FP32-vs-FP64 topology flips;
* independent -- different seeds, per-pixel Welch t statistics over batches
  with disjoint chain ids, turned into equal-tail normal scores (so the few
  batches' degrees of freedom do not inflate the tails); the 4-sigma budget is
  0.1 % of pixel-channels (Bonferroni-style; ~0.006 % expected).

The converged references are plain path tracing on the GPU (2^32 to 2^35
samples; for the Cornell box, the 40k-triangle Cornell + spheres scene, the
glass slit caustic and the many-emitter fBm terrain), each path tracer checked
against the oracle's on identical samples.
relMSE = mean over pixels and channels of (I - R)^2 / (R^2 + 1e-2).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_07148_gb300 import scenes

pytestmark = pytest.mark.gpu
EPS = 1e-2


@pytest.fixture(scope="module")
def J():
    import torch
    assert torch.cuda.is_available()
    from paper_2409_07148_gb300 import jr
    jr.lib()
    return jr


def relmse(img, ref):
    return float(np.mean((img - ref) ** 2 / (ref ** 2 + EPS)))


def welch_z(a, b):
    """Per-pixel Welch t of mean(a) - mean(b) over batches, mapped to the
    normal score with the same two-sided tail probability."""
    from scipy import stats
    na, nb = len(a), len(b)
    va, vb = a.var(0, ddof=1) / na, b.var(0, ddof=1) / nb
    d = a.mean(0) - b.mean(0)
    se2 = va + vb
    ok = se2 > 0
    assert np.all(d[~ok] == 0)
    t = d[ok] / np.sqrt(se2[ok])
    df = se2[ok] ** 2 / (va[ok] ** 2 / (na - 1) + vb[ok] ** 2 / (nb - 1))
    p = 2 * stats.t.sf(np.abs(t), df)
    return np.sign(t) * stats.norm.isf(np.maximum(p, 1e-300) / 2)


def _gpu_batches(J, sc, n_batches, chains, steps, seed, first_chain=0):
    import torch
    g = J.Scene(sc)
    sets, streams = [], []
    for b in range(n_batches):
        s = torch.cuda.Stream()
        c = J.Chains(g, sc.width, sc.height, sc.depth, chains, seed=seed, chain_offset=first_chain + b * chains,
                     stream=s)
        c.advance(steps, stream=s)
        sets.append(c)
        streams.append(s)
    torch.cuda.synchronize()
    imgs = np.array([c.resolve(stream=s) for c, s in zip(sets, streams)], np.float64)
    for c, s in zip(sets, streams):
        assert c.stats(stream=s)["status_word"] == 0
    return imgs


def _oracle_batches(sc, n_batches, chains, steps, seed, first_chain=0):
    osc = O.Scene(sc)
    out = []
    for b in range(n_batches):
        ch = O.Chains(osc, sc.D, sc.width, sc.height, seed=seed, chain_begin=first_chain + b * chains,
                      n_chains=chains)
        ch.advance(steps)
        out.append(ch.image())
    return np.array(out)


def test_cornell_paired_streams_match_oracle(J):
    """Identical Philox streams: 16 batches of 256 chains x 2000 steps on both
    sides.  The image difference per pixel is far below one standard error."""
    sc = scenes.cornell()
    g = _gpu_batches(J, sc, 16, 256, 2000, seed=3)
    o = _oracle_batches(sc, 16, 256, 2000, seed=3)
    se = np.sqrt(o.var(0, ddof=1) / len(o))
    d = np.abs(g.mean(0) - o.mean(0))
    ok = se > 0
    assert np.all(d[~ok] < 1e-6)
    r = d[ok] / se[ok]
    assert np.median(r) < 1e-2          # most pixels: identical trajectories, FP32 rounding only
    assert np.mean(r > 1.0) < 0.01      # a few pixels touched by a chain that diverged at a tie
    assert np.max(r) < 4.0


def test_cornell_per_pixel_vs_oracle(J):
    """Independent seeds: 64 GPU batches vs 32 oracle batches, each batch the
    256-chain x 10^4-step Cornell workload (equal batch shapes keep the
    batch-mean distributions alike on both sides)."""
    sc = scenes.cornell()
    g = _gpu_batches(J, sc, 64, 256, 10_000, seed=0)
    o = _oracle_batches(sc, 32, 256, 10_000, seed=1, first_chain=1 << 20)
    z = welch_z(g, o)
    assert np.mean(np.abs(z) > 4) <= 1e-3, np.sort(np.abs(z))[-10:]
    assert 0.75 < np.mean(z ** 2) < 1.35, np.mean(z ** 2)


@pytest.fixture(scope="module")
def reference(J):
    """Converged plain path tracing of the 64x64 Cornell box on the GPU
    (2^32 samples = 2^20 per pixel)."""
    import torch
    sc = scenes.cornell()
    g = J.Scene(sc)
    acc = torch.zeros((sc.height, sc.width, 4), dtype=torch.float64, device="cuda")
    n = 1 << 32
    chunk = 1 << 28
    for s0 in range(0, n, chunk):
        J.render_pt(g, sc.width, sc.height, sc.depth, chunk, seed=123, sample_begin=s0, accum=acc)
    torch.cuda.synchronize()
    return sc, (acc[..., :3] / n).cpu().numpy()


def test_plain_path_tracer_matches_oracle_paired(J):
    """Same seed and sample ids on both sides: identical samples, so pixel sums
    agree to FP32 rounding except for rare topology flips."""
    import torch
    sc = scenes.cornell()
    n = 1 << 22
    acc = J.render_pt(J.Scene(sc), sc.width, sc.height, sc.depth, n, seed=5)
    torch.cuda.synchronize()
    g = (acc[..., :3] / n).cpu().numpy()
    o, _ = O.render_pt(O.Scene(sc), sc.D, sc.width, sc.height, n, seed=5)
    nz = o != 0
    assert np.all(g[~nz] == 0) or np.mean(g[~nz] != 0) < 1e-3
    rel = np.abs(g - o)[nz] / o[nz]
    assert np.mean(rel > 1e-4) < 5e-3, np.sort(rel)[-5:]
    assert relmse(g, o) < 1e-6


def test_cornell_relmse_vs_converged_reference(J, reference):
    sc, ref = reference
    imgs = _gpu_batches(J, sc, 32, 4096, 4000, seed=11, first_chain=1 << 22)
    img = imgs.mean(0)
    e = relmse(img, ref)
    assert e <= 1e-3, e
    # the batches scatter about the reference as their standard errors say
    from scipy import stats
    se = imgs.std(0, ddof=1) / np.sqrt(len(imgs))
    ok = se > 0
    t = (img - ref)[ok] / se[ok]
    z = np.sign(t) * stats.norm.isf(stats.t.sf(np.abs(t), len(imgs) - 1))
    assert np.mean(np.abs(z) > 4) <= 1e-3
    assert 0.7 < np.mean(z ** 2) < 1.5


def test_furnace_image_is_flat(J):
    sc = scenes.furnace(width=8, height=8, depth=6, albedo=0.5, emission=1.0)
    imgs = _gpu_batches(J, sc, 8, 1024, 200, seed=2)
    expect = (1 - 0.5 ** 7) / 0.5
    m = imgs.mean(axis=(1, 2, 3))
    se = m.std(ddof=1) / np.sqrt(len(m))
    assert abs(m.mean() - expect) < 4 * se + 1e-6


@pytest.fixture(scope="module")
def spheres_reference(J):
    """Converged plain path tracing of the full 40k-triangle Cornell + spheres
    scene (Phong n = 50 and diffuse spheres, 0.05-wide light, depth 8) at
    128^2: 2^35 samples in two independent halves, whose disagreement bounds
    the reference's own noise."""
    import torch
    sc = scenes.cornell_spheres(width=128, height=128, depth=8)
    g = J.Scene(sc)
    halves = []
    n, chunk = 1 << 34, 1 << 28
    for h in range(2):
        acc = torch.zeros((sc.height, sc.width, 4), dtype=torch.float64, device="cuda")
        for s0 in range(0, n, chunk):
            J.render_pt(g, sc.width, sc.height, sc.depth, chunk, seed=500 + h, sample_begin=s0, accum=acc)
        halves.append((acc[..., :3] / n).cpu().numpy())
    torch.cuda.synchronize()
    return sc, 0.5 * (halves[0] + halves[1]), relmse(halves[0], halves[1]) / 4.0


def test_spheres_plain_path_tracer_matches_oracle_paired(J):
    """The full scene's GPU path tracer against the oracle's (with its own BVH)
    on identical samples: pixel sums agree to FP32 rounding except for rare
    FP32-vs-FP64 topology flips."""
    import torch
    sc = scenes.cornell_spheres(width=128, height=128, depth=8)
    n = 1 << 20
    acc = J.render_pt(J.Scene(sc), sc.width, sc.height, sc.depth, n, seed=9)
    torch.cuda.synchronize()
    g = (acc[..., :3] / n).cpu().numpy()
    o, _ = O.render_pt(O.Scene(sc, bvh=True), sc.D, sc.width, sc.height, n, seed=9)
    nz = o != 0
    rel = np.abs(g - o)[nz] / o[nz]
    assert np.mean(rel > 1e-4) < 1e-2, np.sort(rel)[-5:]
    assert relmse(g, o) < 1e-5


def test_spheres_relmse_and_per_pixel_vs_converged_reference(J, spheres_reference):
    """Jump Restore on the full 40k-triangle scene at 128^2, depth 8: 32
    independent batches of 2^16 chains x 1500 steps, each stopped with every
    tour completed (the completed-tour estimator of Section 7.4, which has no
    open-tour bias; with 2^16 open tours against J ~ 10^8 that bias reaches
    several standard errors in the bright pixels, where tours are long), scatter
    about the converged reference within 4 sigma per pixel (0.1 % budget), and
    the pooled image reaches relMSE <= 1e-3."""
    import torch
    from scipy import stats
    sc, ref, ref_noise = spheres_reference
    assert ref_noise < 2e-4, ref_noise
    g = J.Scene(sc)
    imgs = []
    for b in range(32):
        c = J.Chains(g, sc.width, sc.height, sc.depth, 1 << 16, seed=31, chain_offset=(1 << 24) + b * (1 << 16))
        c.advance(1500)
        assert J.complete_tours(c) == 0
        imgs.append(c.resolve())
        assert c.stats()["status_word"] == 0
    torch.cuda.synchronize()
    imgs = np.array(imgs, np.float64)
    img = imgs.mean(0)
    e = relmse(img, ref)
    assert e <= 1e-3, e
    # Per-pixel 4 sigma where the batch means are in the central-limit regime: at
    # least 24 of the 32 batches saw light in the pixel-channel.  Pixels lit
    # only by rare paths (glossy reflections of the 0.05-wide light) have batch
    # values that are mostly exactly 0 with a rare large one; there the batch
    # standard error underestimates and a z-score means nothing, so they are
    # checked in 8x8 tiles below (and by the relMSE above).
    def zscores(a, r):
        se = a.std(0, ddof=1) / np.sqrt(len(a))
        ok = se > 0
        t = (a.mean(0) - r)[ok] / se[ok]
        return np.sign(t) * stats.norm.isf(stats.t.sf(np.abs(t), len(a) - 1)), ok
    z, ok = zscores(imgs, ref)
    dense = (np.count_nonzero(imgs, axis=0) >= 24)[ok]
    assert dense.mean() > 0.8, dense.mean()
    zd = z[dense]
    bad = np.abs(zd) > 4
    msg = dict(frac=float(np.mean(bad)), worst=np.sort(np.abs(zd))[-8:].tolist())
    assert np.mean(bad) <= 1e-3, msg
    assert 0.7 < np.mean(zd ** 2) < 1.5, np.mean(zd ** 2)
    tiles = imgs.reshape(len(imgs), 16, 8, 16, 8, 3).mean(axis=(2, 4))
    zt, _ = zscores(tiles, ref.reshape(16, 8, 16, 8, 3).mean(axis=(1, 3)))
    assert np.abs(zt).max() < 4.5, np.sort(np.abs(zt))[-5:]


def _big_scene(name):
    """64^2 versions of the two large benchmark scenes: the slit caustic (a glass
    sphere of 80k triangles, IOR 1.5, lit only through a 0.02-wide slit;
    depth 10, D = 22) and the fBm terrain (79k triangles, lit only by 256 small
    emitters with L_e log-uniform in [1, 100], open sky; depth 12, D = 26)."""
    if name == "caustic":
        return scenes.caustic_slit(width=64, height=64, depth=10)
    return scenes.terrain(width=64, height=64, n_grid=200)


@pytest.fixture(scope="module", params=["caustic", "terrain"])
def big_reference(J, request):
    """Converged plain path tracing of a large scene at 64^2: 16 independent
    chunks of 2^30 samples, so that a test can carry the reference's own
    per-pixel error."""
    import torch
    sc = _big_scene(request.param)
    g = J.Scene(sc)
    chunks = []
    n, chunk = 1 << 30, 1 << 28
    for h in range(16):
        acc = torch.zeros((sc.height, sc.width, 4), dtype=torch.float64, device="cuda")
        for s0 in range(0, n, chunk):
            J.render_pt(g, sc.width, sc.height, sc.depth, chunk, seed=700 + h, sample_begin=s0, accum=acc)
        chunks.append((acc[..., :3] / n).cpu().numpy())
    torch.cuda.synchronize()
    return request.param, sc, np.array(chunks)


@pytest.mark.parametrize("name", ["caustic", "terrain"])
def test_big_scene_plain_path_tracer_matches_oracle_paired(J, name):
    """The GPU path tracer against the oracle's, with its own BVH, on
    identical samples (the caustic's dielectric Fresnel choices and
    refractions; the terrain's 256 emitters and open sky): pixel sums agree to
    FP32 rounding except for rare FP32-vs-FP64 topology flips."""
    import torch
    sc = _big_scene(name)
    n = 1 << 21
    acc = J.render_pt(J.Scene(sc), sc.width, sc.height, sc.depth, n, seed=9)
    torch.cuda.synchronize()
    g = (acc[..., :3] / n).cpu().numpy()
    o, _ = O.render_pt(O.Scene(sc, bvh=True), sc.D, sc.width, sc.height, n, seed=9)
    nz = o != 0
    assert nz.sum() > 1000            # enough light reaches the film for the comparison to mean something
    rel = np.abs(g - o)[nz] / o[nz]
    assert np.mean(rel > 1e-4) < 1e-2, np.sort(rel)[-5:]
    assert relmse(g, o) < 1e-5


def test_big_scene_relmse_and_per_pixel_vs_converged_reference(J, big_reference):
    """Jump Restore on a large scene at 64^2: 32 independent batches of 2^16
    chains x 1500 steps, each stopped with every tour completed, against the
    16 reference chunks.  The pooled image reaches relMSE <= 1e-3; per
    pixel-channel, Welch's t between the batches and the chunks (so the
    reference's own error is carried) stays within 4 sigma (0.1 % budget) where
    both are in the central-limit regime (lit in at least 24 of 32 batches and
    12 of 16 chunks); the rest, pixels lit by rare paths, is checked in 8x8
    tiles and by the relMSE."""
    import torch
    from scipy import stats
    name, sc, chunks = big_reference
    ref = chunks.mean(0)
    g = J.Scene(sc)
    imgs = []
    for b in range(32):
        c = J.Chains(g, sc.width, sc.height, sc.depth, 1 << 16, seed=41, chain_offset=(1 << 24) + b * (1 << 16))
        c.advance(1500)
        assert J.complete_tours(c) == 0
        imgs.append(c.resolve())
        assert c.stats()["status_word"] == 0
    torch.cuda.synchronize()
    imgs = np.array(imgs, np.float64)
    e = relmse(imgs.mean(0), ref)
    assert e <= 1e-3, (name, e)

    def welch(a, b):
        na, nb = len(a), len(b)
        va, vb = a.var(0, ddof=1) / na, b.var(0, ddof=1) / nb
        se2 = va + vb
        ok = se2 > 0
        t = (a.mean(0) - b.mean(0))[ok] / np.sqrt(se2[ok])
        df = se2[ok] ** 2 / (va[ok] ** 2 / (na - 1) + vb[ok] ** 2 / (nb - 1))
        p = 2 * stats.t.sf(np.abs(t), df)
        return np.sign(t) * stats.norm.isf(np.maximum(p, 1e-300) / 2), ok

    z, ok = welch(imgs, chunks)
    dense = ((np.count_nonzero(imgs, axis=0) >= 24) & (np.count_nonzero(chunks, axis=0) >= 12))[ok]
    assert dense.mean() > 0.5, (name, dense.mean())
    zd = z[dense]
    msg = dict(scene=name, frac=float(np.mean(np.abs(zd) > 4)), worst=np.sort(np.abs(zd))[-8:].tolist())
    assert np.mean(np.abs(zd) > 4) <= 1e-3, msg
    assert 0.7 < np.mean(zd ** 2) < 1.5, (name, np.mean(zd ** 2))
    tiles = imgs.reshape(32, 8, 8, 8, 8, 3).mean(axis=(2, 4))
    rtiles = chunks.reshape(16, 8, 8, 8, 8, 3).mean(axis=(2, 4))
    zt, _ = welch(tiles, rtiles)
    assert np.abs(zt).max() < 4.5, (name, np.sort(np.abs(zt))[-5:])
