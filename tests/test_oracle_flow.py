"""Pins of the regeneration-flow oracle and of Alg. 2 with a learned mixture mu
(CPU only).  The flow is the library's addition (not in the paper); what the
paper fixes is that Alg. 2 with k = c~ u / p is exact for any regeneration
density u (Section 6.2, Theorem A) -- checked here with u = beta q + 1 - beta."""
import numpy as np
import pytest

from oracle import flow as FL
from oracle import learned as LR
from oracle import oracle as O
from paper_2409_07148_gb300.flowinit import init_flow_params, layer_size


def _flow(D, seed, sd):
    perm, w = init_flow_params(D, seed)
    A = D // 2
    tail = A * 16 * 64 + A * 16
    w[:, -tail:] = np.random.default_rng(seed + 100).normal(0.0, sd, (w.shape[0], tail)).astype(np.float32)
    return perm, w


def test_initial_flow_is_identity():
    perm, w = init_flow_params(12, 3)
    x = np.random.default_rng(0).random((500, 12))
    lq, z = FL.log_density(perm, w, x)
    assert np.all(lq == 0.0) and np.array_equal(z, x)
    xs, lqs = FL.sample(perm, w, x)
    assert np.abs(xs - x).max() < 1e-12 and np.all(lqs == 0.0)


def test_density_integrates_to_one_2d():
    perm, w = _flow(2, 1, 0.05)      # q varies 25x; the midpoint rule's error at bin edges stays < 1e-4
    n = 768
    g = (np.arange(n) + 0.5) / n
    X0, X1 = np.meshgrid(g, g)
    q = np.exp(FL.log_density(perm, w, np.stack([X0.ravel(), X1.ravel()], 1))[0])
    assert q.max() / q.min() > 5            # a non-trivial density
    assert abs(q.mean() - 1.0) < 5e-4


def test_density_normalised_in_8d():
    perm, w = _flow(8, 2, 0.03)
    x = np.random.default_rng(1).random((200_000, 8))
    q = np.exp(FL.log_density(perm, w, x)[0])
    assert abs(q.mean() - 1.0) < 4 * q.std() / np.sqrt(len(q))


def test_sampling_inverts_density_direction():
    perm, w = _flow(10, 3, 0.1)
    z = np.random.default_rng(2).random((5000, 10))
    x, lq_s = FL.sample(perm, w, z)
    lq_d, zb = FL.log_density(perm, w, x)
    assert np.abs(zb - z).max() < 1e-9
    assert np.abs(lq_s - lq_d).max() < 1e-9


def test_samples_follow_the_density():
    """2-D histogram of T^{-1}(uniform) against the cell integrals of q."""
    perm, w = _flow(2, 4, 0.08)
    x, _ = FL.sample(perm, w, np.random.default_rng(3).random((200_000, 2)))
    h, _, _ = np.histogram2d(x[:, 1], x[:, 0], bins=16, range=[[0, 1], [0, 1]])
    n = 256
    g = (np.arange(n) + 0.5) / n
    X0, X1 = np.meshgrid(g, g)
    q = np.exp(FL.log_density(perm, w, np.stack([X0.ravel(), X1.ravel()], 1))[0]).reshape(n, n)
    expect = q.reshape(16, n // 16, 16, n // 16).mean(axis=(1, 3)) / 256 * len(x)
    chi2 = ((h - expect) ** 2 / expect).sum()
    assert chi2 < 256 + 5 * np.sqrt(2 * 256)


def test_nll_gradient_matches_finite_differences():
    """Autograd gradient of -sum w log q / sum w against central differences
    (bf16 rounding off, so the loss is differentiable)."""
    import torch  # noqa: F401
    perm, w = _flow(6, 5, 0.1)
    rng = np.random.default_rng(4)
    x = rng.random((64, 6))
    wt = rng.random(64) + 0.1
    orig = FL.bf16
    FL.bf16 = lambda a: np.asarray(a, np.float64)
    try:
        _, g = FL.nll_and_grad_torch(perm, w.astype(np.float64), x, wt)
        S = layer_size(6)
        picks = [(0, 5), (1, 64 * 16 + 3), (2, 64 * 16 + 64 + 100), (3, S - 50), (5, S - 3), (4, S - 3 * 16 * 64)]
        for (l, k) in picks:
            e = 1e-6
            wp = w.astype(np.float64).copy()
            wm = wp.copy()
            wp[l, k] += e
            wm[l, k] -= e
            fp = -(wt * FL.log_density(perm, wp, x)[0]).sum() / wt.sum()
            fm = -(wt * FL.log_density(perm, wm, x)[0]).sum() / wt.sum()
            fd = (fp - fm) / (2 * e)
            assert abs(fd - g[l, k]) <= 1e-5 * max(1.0, abs(fd)), (l, k, fd, g[l, k])
    finally:
        FL.bf16 = orig


def test_learned_oracle_with_beta_zero_is_the_c_oracle():
    """The Python Alg. 2 with beta = 0 follows the C oracle chain for chain."""
    an = O.Analytic([(1.0, 0.3, 0.4, 0.08), (0.5, 0.7, 0.6, 0.1)], (0.45, 0.5))
    F_of = an.eval
    pl = LR.LearnedChains(F_of, 2, 4, 4, beta=0.0, sigma=0.05, seed=7, n_chains=64)
    pl.advance(50)
    oc = O.Chains(an, 2, 4, 4, sigma=0.05, seed=7, n_chains=64)
    oc.advance(50)
    assert pl.J == oc.J
    assert np.allclose(pl.x, oc.x, atol=1e-12)
    assert np.allclose(pl.accum, oc.accum, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("beta", [0.5, 0.9])
def test_learned_mixture_keeps_the_estimator_exact(beta):
    """Alg. 2 with u = beta q + 1 - beta (a non-trivial flow): the image still
    converges to the pixel means (quadrature), and J/N to c~/(p_lambda + c~)."""
    an = O.Analytic([(1.0, 0.3, 0.4, 0.08), (0.5, 0.7, 0.6, 0.1)], (0.45, 0.5))
    perm, w = _flow(2, 8, 0.1)
    n = 1024
    g = (np.arange(n) + 0.5) / n
    X0, X1 = np.meshgrid(g, g)
    F = an.eval(np.stack([X0.ravel(), X1.ravel()], 1)).reshape(n, n, 3)
    pix = F.reshape(4, n // 4, 4, n // 4, 3).mean(axis=(1, 3))
    p_lambda = (F @ LR.LUM).mean()
    imgs, fr = [], []
    for b in range(10):
        ch = LR.LearnedChains(an.eval, 2, 4, 4, perm, w, beta=beta, sigma=0.05, seed=11, chain_begin=384 * b,
                              n_chains=384)
        ch.advance(250)
        imgs.append(ch.image())
        fr.append(ch.J / (384 * 250))
    imgs = np.array(imgs)
    se = imgs.std(0, ddof=1) / np.sqrt(len(imgs))
    z = (imgs.mean(0) - pix) / se
    assert np.abs(z).max() < 4.5
    fr = np.array(fr)
    assert abs(fr.mean() - 1.0 / (p_lambda + 1.0)) < 4 * fr.std(ddof=1) / np.sqrt(len(fr)) + 1e-3


def test_completed_tours_remove_the_finite_run_bias():
    """Short runs (10 steps per chain): stopping at a fixed step leaves one open
    tour per chain, a bias of order chains / J; completing every tour (drain)
    gives the pixel means again (quadrature), for uniform and learned mu."""
    an = O.Analytic([(1.0, 0.3, 0.4, 0.08), (0.5, 0.7, 0.6, 0.1)], (0.45, 0.5))
    n = 1024
    g = (np.arange(n) + 0.5) / n
    X0, X1 = np.meshgrid(g, g)
    F = an.eval(np.stack([X0.ravel(), X1.ravel()], 1)).reshape(n, n, 3)
    pix = F.reshape(2, n // 2, 2, n // 2, 3).mean(axis=(1, 3))
    perm, w = _flow(2, 8, 0.1)
    for beta in (0.0, 0.7):
        open_, done_ = [], []
        for b in range(10):
            ch = LR.LearnedChains(an.eval, 2, 2, 2, perm, w, beta=beta, c_tilde=0.2, sigma=0.05, seed=21,
                                  chain_begin=4096 * b, n_chains=4096)
            if beta:
                ch.set_flow(perm, w, beta)
            ch.advance(10)
            open_.append(ch.image())
            assert ch.complete_tours() == 0
            done_.append(ch.image())
        done_ = np.array(done_)
        z = (done_.mean(0) - pix) / (done_.std(0, ddof=1) / np.sqrt(len(done_)))
        assert np.abs(z).max() < 4.5, (beta, z)
        open_ = np.array(open_)
        zo = (open_.mean(0) - pix) / (open_.std(0, ddof=1) / np.sqrt(len(open_)))
        assert np.abs(zo).max() > 4.5     # the open-tour bias is real at this run length


def _product_target(an):
    """F(x) = F_an(x0, x1) g(x2, x3) h(x4, x5) on [0,1)^6 with g and h of
    integral 1, so the pixel means are the 2-D target's."""
    def F_of(x):
        g = (1.0 + 0.6 * np.cos(2 * np.pi * x[:, 2])) * (1.0 + 0.5 * np.sin(2 * np.pi * x[:, 3]))
        h = (1.0 + 0.6 * np.cos(2 * np.pi * x[:, 4])) * (1.0 + 0.5 * np.sin(2 * np.pi * x[:, 5]))
        return an.eval(x[:, :2]) * (g * h)[:, None]
    return F_of


def _prefix_run(F_of, perm, w, planted=False):
    imgs = []
    for b in range(8):
        ch = LR.LearnedChains(F_of, 6, 4, 4, perm, w, beta=0.7, sigma=0.05, seed=31, chain_begin=256 * b,
                              n_chains=256)
        if planted:   # a flow draw that forgets its density: u = 1 whatever T^{-1} did
            draw = ch._flow_draw
            ch._flow_draw = lambda v, draw=draw: (draw(v)[0], np.ones(len(v)))
        ch.advance(150)
        imgs.append(ch.image())
    return np.array(imgs)


def test_prefix_flow_mixture_keeps_the_estimator_exact():
    """A flow over the leading 4 of 6 coordinates (the rest uniform):
    mu = beta (q x uniform) + (1 - beta) uniform has density
    u = beta q(x[:4]) + 1 - beta, and Alg. 2 with k = c~ u / p stays exact
    (Section 6.2) on a target that varies in all six coordinates.  Planted
    mistake: flow draws that keep u = 1 bias the image, so the check is not
    vacuous."""
    an = O.Analytic([(1.0, 0.3, 0.4, 0.08), (0.5, 0.7, 0.6, 0.1)], (0.45, 0.5))
    F_of = _product_target(an)
    n = 1024
    g = (np.arange(n) + 0.5) / n
    X0, X1 = np.meshgrid(g, g)
    F = an.eval(np.stack([X0.ravel(), X1.ravel()], 1)).reshape(n, n, 3)
    pix = F.reshape(4, n // 4, 4, n // 4, 3).mean(axis=(1, 3))
    perm, w = _flow(4, 41, 0.3)
    q = np.exp(FL.log_density(perm, w, np.random.default_rng(5).random((4096, 4)))[0])
    assert q.max() / q.min() > 5            # the flow is far from uniform
    imgs = _prefix_run(F_of, perm, w)
    z = (imgs.mean(0) - pix) / (imgs.std(0, ddof=1) / np.sqrt(len(imgs)))
    assert np.abs(z).max() < 4.5, z
    bad = _prefix_run(F_of, perm, w, planted=True)
    zb = (bad.mean(0) - pix) / (bad.std(0, ddof=1) / np.sqrt(len(bad)))
    assert np.abs(zb).max() > 4.5
