"""Pins of two oracle functions that no invariant of the method can see (CPU only).

* The modified Phong sampler (Lafortune & Willems 1994).  Its mean weight over
  the sampler's own measure must equal the directional albedo of the BRDF
  f = rho (n+2)/(2 pi) max(0, cos alpha)^n, i.e. the hemisphere integral of
  f cos theta_i, computed here by brute-force quadrature from the BRDF's
  definition, not from the sampler.  At normal incidence the mirror direction
  is the normal, so cos alpha = cos theta_i and a weight that uses the lobe
  cosine instead of cos theta_i goes unseen; oblique incidences (30, 60, 80
  degrees) separate the two, and at 80 degrees part of the lobe lies below
  the surface, where the sampler must return no path.
* The small-step kernel zeta of the local move (Section 5, the Gaussian small
  step of the MH baseline): y = (x + N(0, sigma^2)) mod 1 per coordinate.  Any
  symmetric proposal leaves pi invariant, so the quadrature pins of Alg. 2 cannot
  see a wrong scale.  Here the oracle's own accepted local moves on a target
  that depends on (x0, x1) only give unbiased draws of zeta in the other
  coordinates (acceptance does not look at them): mean 0, variance sigma^2,
  kurtosis 3, independent coordinates, and for a large sigma the wrapped
  normal's closed form E[cos 2 pi k dx] = exp(-2 pi^2 k^2 sigma^2).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_07148_gb300 import scenes


# ------------------------------------------------------------------ Phong
def _frame(theta_deg):
    """Geometric normal +z and an incoming direction at theta from the normal."""
    th = math.radians(theta_deg)
    ng = np.array([0.0, 0.0, 1.0])
    d = np.array([math.sin(th), 0.0, -math.cos(th)])
    return ng, d


def _albedo_quadrature(theta_deg, nexp, rho, n_mu=2000, n_phi=2000):
    """Directional albedo of the modified Phong BRDF by the midpoint rule over
    the hemisphere above the normal, in (mu = cos theta_i, phi): d omega = d mu d phi.
    Also the lobe mass (n+1)/(2 pi) cos^n alpha that lies below the surface."""
    ng, d = _frame(theta_deg)
    r = d - 2.0 * np.dot(d, ng) * ng                     # mirror direction
    mu = (np.arange(n_mu) + 0.5) / n_mu
    phi = (np.arange(n_phi) + 0.5) / n_phi * 2 * math.pi
    MU, PHI = np.meshgrid(mu, phi, indexing="ij")
    s = np.sqrt(1 - MU * MU)
    wx, wy, wz = s * np.cos(PHI), s * np.sin(PHI), MU
    cos_a = np.maximum(wx * r[0] + wy * r[1] + wz * r[2], 0.0)
    f = rho * (nexp + 2) / (2 * math.pi) * cos_a ** nexp
    dA = (1.0 / n_mu) * (2 * math.pi / n_phi)
    albedo = float((f * MU).sum() * dA)
    # lobe mass below the surface: integrate the lobe pdf over the lower hemisphere
    wz_lo = -MU
    cos_lo = np.maximum(wx * r[0] + wy * r[1] + wz_lo * r[2], 0.0)
    below = float(((nexp + 1) / (2 * math.pi) * cos_lo ** nexp).sum() * dA)
    return albedo, below, r


def _sampler_grid(theta_deg, nexp, rho, n1=256, n2=64):
    """The oracle's Phong sampler on a stratified (u1, u2) grid: its weights,
    directions and the 'path ends' flags."""
    m = scenes.material(scenes.PHONG, (rho, rho, rho), phong_n=nexp)
    ng, d = _frame(theta_deg)
    W, WI, OK = [], [], []
    for a in (np.arange(n1) + 0.5) / n1:
        for b in (np.arange(n2) + 0.5) / n2:
            ok, wi, w = O.scatter(m, d, ng, a, b)
            W.append(w[0])
            WI.append(wi)
            OK.append(ok)
    return np.array(W), np.array(WI), np.array(OK, bool), ng


@pytest.mark.parametrize("theta", [0.0, 30.0, 60.0, 80.0])
@pytest.mark.parametrize("nexp", [1.0, 10.0, 50.0])
def test_phong_mean_weight_is_the_directional_albedo(theta, nexp):
    rho = float(np.float32(0.7))
    tol = 2e-4   # quadrature and stratified-grid error, measured at <= 5e-5
    albedo, below, r = _albedo_quadrature(theta, nexp, rho)
    w, wi, ok, ng = _sampler_grid(theta, nexp, rho)
    cos_i = wi @ ng
    # below-surface cut: exactly the samples under the surface end the path, with weight 0
    assert np.all(ok == (cos_i > 0))
    assert np.all(w[~ok] == 0)
    assert abs((~ok).mean() - below) < 2e-3 + 0.02 * below
    # the sampler's mean weight is the BRDF's directional albedo
    assert abs(w.mean() - albedo) < tol, (w.mean(), albedo)
    # negative control: a weight that uses the lobe cosine cos(alpha) in place of
    # cos(theta_i) (identical at normal incidence) misses the albedo at oblique
    # incidence by far more than the tolerance
    cos_a = wi @ r
    wrong = np.where(ok, rho * (nexp + 2) / (nexp + 1) * cos_a, 0.0)
    if theta >= 30.0:
        assert abs(wrong.mean() - albedo) > 10 * tol, (wrong.mean(), albedo)
    else:
        assert abs(wrong.mean() - albedo) < tol
    # negative control: the lobe normalisation (n+1)/(n+2) in place of (n+2)/(n+1)
    wrong2 = w * ((nexp + 1) / (nexp + 2)) ** 2
    assert abs(wrong2.mean() - albedo) > 10 * tol


def test_phong_albedo_quadrature_reduces_to_rho_at_normal_incidence():
    """The quadrature itself: at normal incidence the whole lobe is above the
    surface and the normalised lobe integrates to rho (closed form)."""
    for nexp in (1.0, 10.0, 50.0):
        a, below, _ = _albedo_quadrature(0.0, nexp, 0.7)
        assert abs(a - 0.7) < 1e-4 * (1 + nexp / 10) and below < 1e-12


# ------------------------------------------------------------------ zeta
def _flat_target():
    """p depends on (x0, x1) only and varies by < 30 %: acceptance is high and
    independent of the other coordinates' displacements."""
    return O.Analytic([(1.0, 0.5, 0.5, 1.0e3)], band=(0.0, 0.0))


def _zeta_draws(sigma, n_chains=1 << 15, D=6, seed=11):
    """Displacements of coordinates 2..D-1 in the oracle's accepted local moves
    (signed, on the torus), one step per chain; c~ is tiny, so the local branch
    is always taken."""
    tgt = _flat_target()
    ch = O.Chains(tgt, D, 4, 4, c_tilde=1e-12, sigma=sigma, seed=seed, n_chains=n_chains)
    x0 = ch.x.copy()
    tr = ch.advance(1, trace=True)
    flags = tr["flags"][:, 0]
    assert np.all(flags & 1 == 0)                     # never the killing branch
    acc = (flags & 2) != 0
    assert acc.mean() > 0.5
    dx = ch.x[acc, 2:] - x0[acc, 2:]
    dx = (dx + 0.5) % 1.0 - 0.5                       # signed torus difference
    return dx, acc, x0


@pytest.mark.parametrize("sigma", [0.01, 0.03])
def test_zeta_moments_small_sigma(sigma):
    dx, _, _ = _zeta_draws(sigma)
    z = dx / sigma
    N = z.shape[0]
    se = 1 / math.sqrt(N)
    assert np.all(np.abs(z.mean(axis=0)) < 4 * se)                              # mean 0
    assert np.all(np.abs((z ** 2).mean(axis=0) - 1) < 4 * math.sqrt(2) * se)    # variance sigma^2
    assert np.all(np.abs((z ** 4).mean(axis=0) - 3) < 4 * math.sqrt(96) * se)  # Gaussian kurtosis
    c = np.corrcoef(z.T)
    assert np.all(np.abs(c[np.triu_indices(z.shape[1], 1)]) < 4 * se)           # uncorrelated
    # the two coordinates of one Box-Muller pair are independent, not only uncorrelated
    assert abs((z[:, 0] ** 2 * z[:, 1] ** 2).mean() - 1) < 4 * math.sqrt(8) * se


@pytest.mark.parametrize("sigma", [0.15, 0.3])
def test_zeta_is_the_wrapped_normal(sigma):
    """(x + N(0, sigma^2)) mod 1 has E[cos 2 pi k dx] = exp(-2 pi^2 k^2 sigma^2)
    and E[sin 2 pi k dx] = 0 (the wrapped normal's characteristic function)."""
    dx, _, _ = _zeta_draws(sigma)
    N = dx.size
    for k in (1, 2):
        c = np.cos(2 * math.pi * k * dx).mean()
        s = np.sin(2 * math.pi * k * dx).mean()
        assert abs(c - math.exp(-2 * math.pi ** 2 * k * k * sigma ** 2)) < 4 / math.sqrt(2 * N)
        assert abs(s) < 4 / math.sqrt(2 * N)


def test_zeta_negative_control_catches_a_missing_square_root():
    """The same Philox uniforms through Box-Muller with R = -2 ln(1 - a) (the
    square root dropped) give a variance the moment test rejects; with the
    square root they reproduce the oracle's displacements."""
    sigma, D, seed, n = 0.01, 6, 11, 1 << 15
    dx, acc, x0 = _zeta_draws(sigma, n_chains=n, D=D, seed=seed)
    blk1 = O.draw_uniforms_many(seed, 0, 1, 0, n, 0)   # coordinates 0..3
    blk2 = O.draw_uniforms_many(seed, 0, 2, 0, n, 0)   # coordinates 4..5
    a = np.stack([blk1[:, 2], blk2[:, 0]], 1)           # pair (2, 3) and pair (4, 5)
    b = np.stack([blk1[:, 3], blk2[:, 1]], 1)
    R = np.sqrt(-2 * np.log(1 - a))
    good = np.stack([R[:, 0] * np.cos(2 * math.pi * b[:, 0]), R[:, 0] * np.sin(2 * math.pi * b[:, 0]),
                     R[:, 1] * np.cos(2 * math.pi * b[:, 1]), R[:, 1] * np.sin(2 * math.pi * b[:, 1])], 1)
    assert np.abs(sigma * good[acc] - dx).max() < 1e-12
    Rw = -2 * np.log(1 - a)
    wrong = np.stack([Rw[:, 0] * np.cos(2 * math.pi * b[:, 0]), Rw[:, 0] * np.sin(2 * math.pi * b[:, 0]),
                      Rw[:, 1] * np.cos(2 * math.pi * b[:, 1]), Rw[:, 1] * np.sin(2 * math.pi * b[:, 1])], 1)
    se = 1 / math.sqrt(acc.sum())
    assert np.all(np.abs((wrong[acc] ** 2).mean(axis=0) - 1) > 40 * math.sqrt(2) * se)
