"""Stochastic pins of the oracle's Alg. 2 on tiny analytic targets (CPU only).

The oracle runs the full Jump Restore loop (clocks, branch, splat, MH local
move, regeneration) on analytic targets whose integrals are known by
brute-force quadrature.  Closed forms checked, each within 4 standard errors
from independent chain batches:

* regeneration fraction J/N -> c~ / (p_lambda + c~)   (jump-chain law p + c~u)
* mean holding time per step -> p_lambda / (p_lambda + c~)
* time-weighted occupancy of a pixel -> pi(pixel)     (Section 7.4, "approx")
* normalisation-free estimate (c~/J) sum dt g/p -> lambda(g) (Section 6.3)
* mean tour length sum dt / J -> 1/c = p_lambda / c~  (Section 6.2; the
  worked example of Section 7.3 uses c = 1/4, tour length 4).
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MODES = [(1.0, 0.25, 0.3, 0.06), (0.6, 0.7, 0.7, 0.08), (0.3, 0.8, 0.2, 0.04)]
BAND = (0.45, 0.5)


def _quadrature(target, D, W, H, n=1024):
    """Midpoint rule on an n x n grid: returns (p_lambda, pixel means of F [H,W,3],
    pixel masses of p [H,W])."""
    g = (np.arange(n) + 0.5) / n
    X0, X1 = np.meshgrid(g, g, indexing="xy")      # X1 rows, X0 columns
    x = np.stack([X0.ravel(), X1.ravel()], 1)
    if D == 1:
        x = x[:, :1]
    F = target.eval(x).reshape(n, n, 3)
    p = 0.2126 * F[..., 0] + 0.7152 * F[..., 1] + 0.0722 * F[..., 2]
    p_lambda = p.mean()
    pix = F.reshape(H, n // H, W, n // W, 3).mean(axis=(1, 3))
    pm = p.reshape(H, n // H, W, n // W).mean(axis=(1, 3)) / (W * H)
    return p_lambda, pix, pm


def _run_batches(target, D, W, H, c_tilde, sigma, n_batches, chains, steps, rb=False, seed=11):
    out = []
    for b in range(n_batches):
        ch = O.Chains(target, D, W, H, c_tilde=c_tilde, sigma=sigma, seed=seed, chain_begin=b * chains,
                      n_chains=chains, rao_blackwell=rb)
        ch.advance(steps)
        out.append(ch)
    return out


def _z(vals, expect):
    vals = np.asarray(vals, dtype=np.float64)
    se = vals.std(ddof=1, axis=0) / np.sqrt(len(vals))
    return (vals.mean(0) - expect) / np.maximum(se, 1e-300)


@pytest.fixture(scope="module")
def target2d():
    return O.Analytic(MODES, BAND)


@pytest.fixture(scope="module")
def quad2d(target2d):
    return _quadrature(target2d, 2, 4, 4)


@pytest.fixture(scope="module")
def runs2d(target2d):
    return _run_batches(target2d, 2, 4, 4, c_tilde=1.0, sigma=0.05, n_batches=16, chains=256, steps=2000)


def test_regeneration_fraction_and_mean_holding_time(runs2d, quad2d):
    p_lambda = quad2d[0]
    c = 1.0
    N = np.array([r.n * r.step for r in runs2d], dtype=np.float64)
    frac = np.array([r.J for r in runs2d]) / N
    mean_dt = np.array([r.accum[..., 3].sum() for r in runs2d]) / N
    assert abs(_z(frac, c / (p_lambda + c))) < 4
    assert abs(_z(mean_dt, p_lambda / (p_lambda + c))) < 4
    # and the normalisation-constant estimate of Section 6.3 (c~/j) sum tau
    est = np.array([r.accum[..., 3].sum() / r.J for r in runs2d]) * c
    assert abs(_z(est, p_lambda)) < 4


def test_time_weighted_occupancy_is_pi(runs2d, quad2d):
    _, _, pm = quad2d
    p_lambda = quad2d[0]
    occ = np.array([r.accum[..., 3] / r.accum[..., 3].sum() for r in runs2d])
    expect = pm / pm.sum()                      # pi(pixel) = mass of p in the pixel / p_lambda
    z = _z(occ, expect)
    assert np.abs(z).max() < 4.5


def test_normalisation_free_estimator_matches_quadrature(runs2d, quad2d):
    _, pix, _ = quad2d
    imgs = np.array([r.image() for r in runs2d])
    z = _z(imgs, pix)
    assert np.abs(z).max() < 4.5
    pooled = sum(r.accum[..., :3] for r in runs2d) / sum(r.J for r in runs2d)
    assert np.abs(pooled - pix).max() / pix.max() < 0.03


def test_rao_blackwell_holding_time_same_limit(target2d, quad2d):
    """Replacing dt by its conditional mean 1/(1+k) keeps the estimator's limit."""
    _, pix, _ = quad2d
    runs = _run_batches(target2d, 2, 4, 4, 1.0, 0.05, 12, 256, 1500, rb=True, seed=12)
    z = _z(np.array([r.image() for r in runs]), pix)
    assert np.abs(z).max() < 4.5


def test_large_c_tilde_reduces_to_plain_monte_carlo(target2d, quad2d):
    """c~ -> inf: every step regenerates and dt ~ p/c~, so the estimator is the
    plain Monte Carlo average of W H F (Section 6.3 with k -> inf)."""
    _, pix, _ = quad2d
    runs = _run_batches(target2d, 2, 4, 4, 1e6, 0.05, 12, 256, 1500, seed=13)
    for r in runs:
        assert r.J >= 0.999 * r.n * r.step
    z = _z(np.array([r.image() for r in runs]), pix)
    assert np.abs(z).max() < 4.5


def test_paper_example_tour_length():
    """Section 7.3: three-mode 1-D mixture, uniform mu, c = 1/4 -> mean tour
    length 4 (in process time)."""
    gold = json.load(open(os.path.join(GOLDEN, "paper_example_tour_length.json")))
    t1 = O.Analytic([(1.0, 0.2, 0.0, 0.04), (1.6, 0.5, 0.0, 0.05), (0.8, 0.82, 0.0, 0.04)])
    p_lambda = _quadrature(t1, 1, 1, 1, n=4096)[0]
    c_tilde = gold["c"] * p_lambda
    lengths = []
    for b in range(16):
        ch = O.Chains(t1, 1, 1, 1, c_tilde=c_tilde, sigma=0.02, seed=5, chain_begin=256 * b, n_chains=256)
        ch.advance(1000)
        lengths.append(ch.accum[..., 3].sum() / ch.J)
    assert abs(_z(lengths, gold["expected_tour_length"])) < 4
    assert abs(np.mean(lengths) - gold["expected_tour_length"]) < 0.1


def test_zero_density_start_is_killed_immediately(target2d):
    """Where p = 0 the killing rate is infinite: t2 = 0, the step regenerates
    with dt = 0 and splats nothing."""
    ch = O.Chains(target2d, 2, 4, 4, c_tilde=1.0, sigma=0.05, seed=1, n_chains=64)
    ch.state[:, 0] = 0.47          # inside the zero band
    ch.state[:, 1] = 0.5
    ch.state[:, 2:] = 0.0          # F = p = 0, u would be reset below
    ch.state[:, 6] = 1.0           # u
    tr = ch.advance(1, trace=True)
    assert np.all(tr["flags"][:, 0] & 1)
    assert np.all(tr["dt"][:, 0] == 0.0)
    assert np.all(tr["pix"][:, 0] == -1)
    assert ch.J == 64
