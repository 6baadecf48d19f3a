"""Pins of the oracle's MH baseline "Metropolis" (CPU only).

The paper's reference algorithm (Section 8, practical pairing) is an MH chain
with the mixture proposal of Section 5, Q_l = l mu + (1 - l) zeta, with l = 0.3
and estimation after a burn-in (Section 9).  Pinned here:

* exact, finite state space: the mixture MH kernel built from the oracle's own
  acceptance function leaves pi invariant (pi K = pi to 1e-12) and is
  pi-reversible, for several l; negative controls (the inverted acceptance
  ratio; a non-uniform mu without the Hastings correction) must break it;
* the C oracle's chains on an analytic 2-D target whose integrals are known by
  quadrature: the normalisation b_hat -> p_lambda, the occupancy of each
  pixel -> pi(pixel), and the image -> the pixel means, within 4.5 standard
  errors of independent chain batches, for l = 0.3 and the independence
  sampler l = 1; the large-step share -> l; the burn-in iterations splat
  nothing.
"""
import numpy as np
import pytest

from oracle import finite_state as FS
from oracle import oracle as O

MODES = [(1.0, 0.25, 0.3, 0.06), (0.6, 0.7, 0.7, 0.08), (0.3, 0.8, 0.2, 0.04)]
BAND = (0.45, 0.5)


def _target(M=48, seed=0):
    rng = np.random.default_rng(seed)
    p = rng.random(M) ** 3 + 1e-6
    p[::7] *= 1e-4
    return p


@pytest.mark.parametrize("ell", [0.0, 0.3, 1.0])
def test_mixture_mh_kernel_leaves_pi_invariant(ell):
    p = _target()
    M = len(p)
    mu = np.full(M, 1.0 / M)
    K = FS.mh_mixture_kernel(p, mu, ell)
    pi = p / p.sum()
    assert np.all(K >= -1e-15) and np.allclose(K.sum(1), 1.0, atol=1e-14)
    assert np.abs(pi @ K - pi).max() < 1e-12 * pi.max()
    F = pi[:, None] * K
    assert np.abs(F - F.T).max() < 1e-15          # detailed balance


def test_mixture_mh_negative_controls():
    p = _target(seed=1)
    M = len(p)
    pi = p / p.sum()
    mu = np.full(M, 1.0 / M)
    K = FS.mh_mixture_kernel(p, mu, 0.3, accept=lambda px, py: min(1.0, px / py) if py > 0 else 1.0)
    assert np.abs(pi @ K - pi).max() > 1e-4
    rng = np.random.default_rng(3)
    mu2 = rng.random(M) + 0.05
    mu2 /= mu2.sum()
    K = FS.mh_mixture_kernel(p, mu2, 0.3)         # symmetric acceptance, asymmetric proposal
    assert np.abs(pi @ K - pi).max() > 1e-4


def _quadrature(target, W, H, n=1024):
    g = (np.arange(n) + 0.5) / n
    X0, X1 = np.meshgrid(g, g, indexing="xy")
    x = np.stack([X0.ravel(), X1.ravel()], 1)
    F = target.eval(x).reshape(n, n, 3)
    p = 0.2126 * F[..., 0] + 0.7152 * F[..., 1] + 0.0722 * F[..., 2]
    pix = F.reshape(H, n // H, W, n // W, 3).mean(axis=(1, 3))
    pm = p.reshape(H, n // H, W, n // W).mean(axis=(1, 3))
    return p.mean(), pix, pm / pm.sum()


def _z(vals, expect):
    vals = np.asarray(vals, dtype=np.float64)
    se = vals.std(ddof=1, axis=0) / np.sqrt(len(vals))
    return (vals.mean(0) - expect) / np.maximum(se, 1e-300)


@pytest.fixture(scope="module")
def target2d():
    return O.Analytic(MODES, BAND)


@pytest.fixture(scope="module")
def quad2d(target2d):
    return _quadrature(target2d, 4, 4)


def _runs(target, ell, burn_in, n_batches=16, chains=256, steps=2500, seed=21):
    out = []
    for b in range(n_batches):
        ch = O.MHChains(target, 2, 4, 4, sigma=0.05, ell=ell, burn_in=burn_in, seed=seed, chain_begin=b * chains,
                        n_chains=chains)
        ch.advance(steps)
        out.append(ch)
    return out


@pytest.mark.parametrize("ell", [0.3, 1.0])
def test_mh_estimator_matches_quadrature(target2d, quad2d, ell):
    p_lambda, pix, occ_pi = quad2d
    runs = _runs(target2d, ell, burn_in=500)
    for r in runs:
        assert r.splats == r.n * (r.step - 500)
        assert r.n_large + r.n_small == r.n * r.step
    share = np.array([r.n_large / (r.n * r.step) for r in runs])
    assert abs(_z(share, ell)) < 4 or ell == 1.0 and np.all(share == 1.0)
    assert abs(_z([r.b_hat() for r in runs], p_lambda)) < 4
    occ = np.array([r.accum[..., 3] / r.splats for r in runs])
    live = occ_pi > 1e-6                         # pixels with mass a run can see
    assert np.abs(_z(occ, occ_pi)[live]).max() < 4.5
    assert occ[:, ~live].max(initial=0) < 1e-4
    imgs = np.array([r.image() for r in runs])
    assert np.abs(_z(imgs, pix)[live]).max() < 4.5
    assert imgs[:, ~live].max(initial=0) < 1e-3 * pix.max()


def test_mh_burn_in_splats_nothing(target2d):
    ch = O.MHChains(target2d, 2, 4, 4, sigma=0.05, ell=0.3, burn_in=7, seed=3, n_chains=64)
    tr = ch.advance(10, trace=True)
    assert np.all(tr["flags"][:, :7] & 4 == 0) and np.all(tr["pix"][:, :7] == -1)
    assert np.all(tr["flags"][:, 7:] & 4 == 4)
    assert ch.splats == 64 * 3
    # a rejected proposal leaves the state; an accepted one moves it (same stream, one step at a time)
    a = O.MHChains(target2d, 2, 4, 4, sigma=0.05, ell=0.3, burn_in=0, seed=5, n_chains=256)
    for _ in range(5):
        x0 = a.x.copy()
        t = a.advance(1, trace=True)
        acc = (t["flags"][:, 0] & 2) != 0
        assert np.array_equal(a.x[~acc], x0[~acc])
        assert np.all(np.any(a.x[acc] != x0[acc], axis=1))


def test_mh_zero_density_start_accepts_any_proposal(target2d):
    """Section 4: alpha = 1 when p(x) = 0, so a chain started in the zero band
    takes its first proposal whatever it is."""
    ch = O.MHChains(target2d, 2, 4, 4, sigma=0.05, ell=0.3, burn_in=0, seed=1, n_chains=64)
    ch.state[:, 0] = 0.47
    ch.state[:, 1] = 0.5
    ch.state[:, 2:] = 0.0
    tr = ch.advance(1, trace=True)
    assert np.all(tr["flags"][:, 0] & 2)
    assert np.all(tr["pix"][:, 0] == -1)          # nothing splatted at p = 0
