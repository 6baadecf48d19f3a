"""Image-level parity of the GPU Jump Restore estimator (needs a GB300).

* per pixel: the GPU image of the 64x64 depth-3 Cornell workload (256 chains
  x 10^4 steps per batch, 32 batches with disjoint chain ids) against the
  oracle's image (16 independent batches), z-scores from batch standard
  errors: at most 0.1% of pixel-channels beyond 4 sigma;
* a converged plain path-tracing reference (GPU kernel, itself compared
  pixel by pixel with the oracle's path tracer) and the GPU Jump Restore
  image against it: relMSE <= 1e-3 (relMSE = mean (I - R)^2 / (R^2 + 1e-2));
* the furnace image is flat at the closed form L_e (1 - rho^(d+1)) / (1 - rho).
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


def _z(a, b):
    d = a.mean(0) - b.mean(0)
    se = np.sqrt(a.var(0, ddof=1) / len(a) + b.var(0, ddof=1) / len(b))
    ok = se > 0
    assert np.all(d[~ok] == 0)
    return d[ok] / se[ok]


def test_cornell_per_pixel_vs_oracle(J):
    sc = scenes.cornell()
    gimgs = _gpu_batches(J, sc, 32, 256, 10_000, seed=0)
    osc = O.Scene(sc)
    oimgs = []
    for b in range(16):
        ch = O.Chains(osc, sc.D, sc.width, sc.height, seed=1, chain_begin=b * 256, n_chains=256)
        ch.advance(2500)
        oimgs.append(ch.image())
    z = _z(gimgs, np.array(oimgs))
    assert np.mean(np.abs(z) > 4) <= 1e-3, np.sort(np.abs(z))[-10:]
    assert 0.7 < np.mean(z ** 2) < 1.4


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


def test_plain_path_tracer_matches_oracle(J, reference):
    import torch
    sc, _ = reference
    g = J.Scene(sc)
    gb, ob = [], []
    osc = O.Scene(sc)
    for b in range(16):
        acc = J.render_pt(g, sc.width, sc.height, sc.depth, 1 << 22, seed=5, sample_begin=b << 22)
        torch.cuda.synchronize()
        gb.append((acc[..., :3] / (1 << 22)).cpu().numpy())
        img, _ = O.render_pt(osc, sc.D, sc.width, sc.height, 1 << 20, seed=6, sample_begin=b << 20)
        ob.append(img)
    z = _z(np.array(gb), np.array(ob))
    assert np.mean(np.abs(z) > 4) <= 1e-3
    assert 0.7 < np.mean(z ** 2) < 1.4


def test_cornell_relmse_vs_converged_reference(J, reference):
    sc, ref = reference
    imgs = _gpu_batches(J, sc, 8, 1 << 14, 4000, seed=11, first_chain=1 << 20)
    img = imgs.mean(0)
    e = relmse(img, ref)
    assert e <= 1e-3, e
    # and the batches scatter around the reference as their standard errors say
    se = imgs.std(0, ddof=1) / np.sqrt(len(imgs))
    ok = se > 0
    z = (img - ref)[ok] / se[ok]
    assert np.mean(np.abs(z) > 4.5) <= 2e-3


def test_furnace_image_is_flat(J):
    sc = scenes.furnace(width=8, height=8, depth=6, albedo=0.5, emission=1.0)
    imgs = _gpu_batches(J, sc, 8, 1024, 200, seed=2)
    expect = (1 - 0.5 ** 7) / 0.5
    m = imgs.mean(axis=(1, 2, 3))
    se = m.std(ddof=1) / np.sqrt(len(m))
    assert abs(m.mean() - expect) < 4 * se + 1e-6
