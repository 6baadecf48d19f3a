"""Pins of the oracle's Langevin local dynamics (MALA; the paper's "MALA" and
"MALA Restore", Section 9) (CPU only).

* The integrand's gradient (forward mode) equals central finite differences of
  the oracle's own F at every lit state of a glossy box whose hit sequence does
  not change within the difference step (brute force); it is exactly zero for
  the Lambertian Cornell box and the dielectric furnace, whose path weights do
  not depend on x.
* The analytic target's closed-form gradient equals central finite differences.
* pi-invariance of the MALA kernel, as the definition states it, on the
  analytic target (where the drift is large): exact samples of pi (rejection
  sampling) pushed through MALA steps keep the mean of every test function
  (paired differences within 4.5 standard errors), while the same steps with
  the Hastings ratio dropped move them by far more.  On the glossy box the
  drift is about 1 % of sigma (a PSS gradient through Phong weights is small),
  so there MALA is close to the random-walk small step.
* MALA Restore and the MALA baseline (large steps l = 0.3) give the pixel
  means of the quadrature (analytic target) and of the plain path tracer
  (glossy box) within 4.5 standard errors of independent batches.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_07148_gb300 import scenes


def glossy_box(width=8, height=8, depth=3, n=10.0):
    """The Cornell box with every non-emitting surface made modified Phong."""
    sc = scenes.cornell(width=width, height=height, depth=depth)
    mats = sc.mats.copy()
    dull = ~np.any(mats[:, 4:7] > 0, axis=1)
    mats[dull, 0] = scenes.PHONG
    mats[dull, 7] = n
    return scenes.SceneArrays("glossy_box", sc.verts, sc.tris, sc.tri_mat, mats, sc.camera, width, height, depth)


@pytest.fixture(scope="module")
def box():
    sc = glossy_box()
    return sc, O.Scene(sc)


def test_gradient_equals_finite_differences(box):
    sc, S = box
    x = np.random.default_rng(0).random((40_000, sc.D))
    F0, p0, _, _, ids0 = O.eval_states(S, x, hit_ids=True)
    x = x[p0 > 0][:400]
    assert len(x) == 400
    F0, p0, _, _, ids0 = O.eval_states(S, x, hit_ids=True)
    F, dF = O.eval_grad(S, x)
    assert np.allclose(F, F0, rtol=1e-12, atol=0)   # the same path (rounding order aside)
    assert np.count_nonzero(dF) > 0.15 * dF.size
    h = 1e-7
    checked = 0
    for d in range(sc.D):
        xp, xm = x.copy(), x.copy()
        xp[:, d] += h
        xm[:, d] -= h
        Fp, _, _, _, idp = O.eval_states(S, xp, hit_ids=True)
        Fm, _, _, _, idm = O.eval_states(S, xm, hit_ids=True)
        same = np.all(idp == ids0, axis=1) & np.all(idm == ids0, axis=1)
        fd = (Fp - Fm) / (2 * h)
        err = np.abs(fd - dF[:, :, d])[same]
        assert np.all(err <= 1e-5 * (np.abs(dF[:, :, d])[same] + np.abs(F[same])) + 1e-9), err.max()
        checked += int(same.sum())
    assert checked >= 0.9 * len(x) * sc.D


def test_gradient_is_zero_where_the_weights_are_constant():
    for sc in (scenes.cornell(), scenes.glass_furnace()):
        S = O.Scene(sc)
        x = np.random.default_rng(1).random((500, sc.D))
        F, dF = O.eval_grad(S, x)
        assert np.count_nonzero(F) > 0 and np.all(dF == 0)


MODES = [(1.0, 0.25, 0.3, 0.06), (0.6, 0.7, 0.7, 0.08), (0.3, 0.8, 0.2, 0.04)]
LUM = np.array([0.2126, 0.7152, 0.0722])
SIG = 0.05


@pytest.fixture(scope="module")
def target2d():
    return O.Analytic(MODES, band=(0.45, 0.5))


def test_analytic_gradient_equals_finite_differences(target2d):
    x = np.random.default_rng(2).random((2000, 2))
    x = x[(x[:, 0] < 0.449) | (x[:, 0] > 0.501)]          # off the band's edges
    F, dF = O.eval_grad(target2d, x)
    h = 1e-7
    for d in range(2):
        xp, xm = x.copy(), x.copy()
        xp[:, d] += h
        xm[:, d] -= h
        fd = (target2d.eval(xp) - target2d.eval(xm)) / (2 * h)
        assert np.allclose(fd, dF[:, :, d], rtol=1e-6, atol=1e-9)


def _pi_samples(target, n, seed):
    """Exact samples of pi = p / p_lambda by rejection from uniform, with the
    bound p <= (sum of the mode weights) x lum(1.5, 1, 1.5)."""
    bound = sum(m[0] for m in MODES) * (LUM @ np.array([1.5, 1.0, 1.5]))
    rng = np.random.default_rng(seed)
    out = []
    while sum(len(o) for o in out) < n:
        x = rng.random((1 << 18, 2))
        p = target.eval(x) @ LUM
        assert p.max() <= bound
        out.append(x[rng.random(len(x)) * bound < p])
    return np.concatenate(out)[:n]


def _mala_steps(target, x0, method, seed, k):
    """k MALA steps (no large steps) from the states x0."""
    ch = O.MALAChains(target, 2, 4, 4, sigma=SIG, method=method, ell=0.0, burn_in=1 << 40, seed=seed,
                      n_chains=len(x0))
    F, dF = O.eval_grad(target, x0)
    p = F @ LUM
    g = np.einsum("c,ncd->nd", LUM, dF) / p[:, None]
    ch.state[:, :2] = x0
    ch.state[:, 2:5] = F
    ch.state[:, 5] = p
    ch.state[:, 6] = 1.0
    ch.state[:, 7:] = np.clip(0.5 * SIG ** 2 * g, -2 * SIG, 2 * SIG)
    ch.advance(k)
    return ch.x.copy(), ch.accepts / (k * len(x0))


def test_mala_steps_leave_pi_invariant(target2d):
    """E[f(X4)] = E[f(X0)] for X0 ~ pi (exact samples) and X4 four MALA steps
    on, for f = sin, cos(2 pi x_d) and p itself; the same steps with the
    Hastings ratio dropped drift away from pi (the negative control).  The
    drift here is large (|m| reaches 2 sigma), so the correction matters."""
    x0 = _pi_samples(target2d, 40_000, seed=3)

    def stats(x):
        return np.concatenate([np.sin(2 * np.pi * x), np.cos(2 * np.pi * x), (target2d.eval(x) @ LUM)[:, None]],
                              axis=1)
    z = {}
    for method in ("mh", "mh_uncorrected"):
        x1, acc = _mala_steps(target2d, x0, method, seed=5, k=4)
        assert acc > 0.3
        d = stats(x1) - stats(x0)
        z[method] = np.abs(d.mean(0)) / (d.std(0, ddof=1) / np.sqrt(len(d)))
    assert np.max(z["mh"]) < 4.5, z["mh"]
    assert np.max(z["mh_uncorrected"]) > 8.0, z["mh_uncorrected"]


def _quad(target, W, H, n=1024):
    g = (np.arange(n) + 0.5) / n
    X0, X1 = np.meshgrid(g, g, indexing="xy")
    F = target.eval(np.stack([X0.ravel(), X1.ravel()], 1)).reshape(n, n, 3)
    return F.reshape(H, n // H, W, n // W, 3).mean(axis=(1, 3))


@pytest.mark.parametrize("method", ["restore", "mh"])
def test_mala_estimators_match_quadrature(target2d, method):
    """MALA Restore (Alg. 2 with MALA local moves, k = c~ u / p) and the MALA
    baseline (l = 0.3) on the analytic target: pixel means of 16 independent
    batches within 4.5 standard errors of the quadrature."""
    pix = _quad(target2d, 4, 4)
    imgs = []
    for b in range(16):
        ch = O.MALAChains(target2d, 2, 4, 4, sigma=SIG, method=method, ell=0.3, burn_in=100, seed=7,
                          chain_begin=256 * b, n_chains=256)
        ch.advance(1500)
        imgs.append(ch.image())
    z = _z(imgs, pix)
    live = pix.max(axis=2) > 1e-6
    assert np.abs(z[live]).max() < 4.5, np.abs(z[live]).max()


def _z(vals, expect):
    vals = np.asarray(vals, np.float64)
    se = vals.std(ddof=1, axis=0) / np.sqrt(len(vals))
    return (vals.mean(0) - expect) / np.maximum(se, 1e-300)


@pytest.mark.parametrize("method", ["restore", "mh"])
def test_mala_images_on_the_glossy_box_match_path_tracing(box, method):
    sc, S = box
    ref, _ = O.render_pt(S, sc.D, sc.width, sc.height, 1 << 22, seed=11)
    imgs = []
    for b in range(16):
        # MH chains start uniform and the directly seen light attracts them: the
        # burn-in must cover their mixing (MALA Restore needs none)
        burn = 1500 if method == "mh" else 0
        ch = O.MALAChains(S, sc.D, sc.width, sc.height, sigma=SIG, method=method, ell=0.3, burn_in=burn, seed=13,
                          chain_begin=128 * b, n_chains=128)
        ch.advance(burn + 1500)
        imgs.append(ch.image())
    imgs = np.array(imgs)
    # per pixel where the batch means are in the central-limit regime (at least
    # 12 of 16 batches saw the pixel-channel lit); pixels of small pi mass, which
    # the chains visit rarely and then stay in, are checked in 2x2 tiles
    dense = np.count_nonzero(imgs, axis=0) >= 12
    assert dense.mean() > 0.4, dense.mean()
    z = _z(imgs, ref)
    if method == "restore":    # the MH chains stay where they are: their per-pixel batch values are too heavy-tailed
        assert np.abs(z[dense]).max() < 4.5, np.abs(z[dense]).max()
    tiles = imgs.reshape(16, 4, 2, 4, 2, 3).mean(axis=(2, 4))
    zt = _z(tiles, ref.reshape(4, 2, 4, 2, 3).mean(axis=(1, 3)))
    tdense = np.count_nonzero(tiles, axis=0) >= 12
    assert np.abs(zt[tdense]).max() < 4.5, np.abs(zt[tdense]).max()
