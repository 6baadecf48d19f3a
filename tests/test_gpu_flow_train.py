"""Training of the regeneration flow on the GPU (hand-written tensor-core
forward/backward, Adam) against the FP64 oracle's autograd (needs a GB300).

Tolerance: both sides round the forward GEMM operands to bf16 and pass
gradients straight through; the GPU's backward GEMMs also take bf16 operands
(relative 2^-9 per operand), so gradients agree to about 1e-2 in norm and in
direction (cosine > 0.99); the loss agrees to 1e-3 relative.
"""
import numpy as np
import pytest

from oracle import flow as FL
from paper_2409_07148_gb300.flowinit import init_flow_params, layer_size

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


@pytest.mark.parametrize("D,rows", [(4, 256), (8, 320), (22, 192)])
def test_gradient_matches_oracle_autograd(J, D, rows):
    import torch
    perm, w = _flow(D, 40 + D, 0.1)
    f = J.Flow(D, perm, w)
    rng = np.random.default_rng(D)
    x = rng.random((rows, D)).astype(np.float32)
    wt = (rng.random(rows) + 0.05).astype(np.float32)
    loss, g = f.gradient(torch.from_numpy(np.ascontiguousarray(x.T)).cuda(), torch.from_numpy(wt).cuda())
    lo, go = FL.nll_and_grad_torch(perm, w, x.astype(np.float64), wt.astype(np.float64))
    assert abs(loss - lo) <= 1e-3 * max(1.0, abs(lo)), (loss, lo)
    g = g.reshape(w.shape)
    S = layer_size(D)
    for l in range(w.shape[0]):
        a, b = g[l].astype(np.float64), go[l]
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30)
        assert cos > 0.99, (l, cos)
        assert np.linalg.norm(a - b) <= 3e-2 * np.linalg.norm(b), (l, np.linalg.norm(a - b) / np.linalg.norm(b))
    assert g.shape[1] == S


def test_training_fits_a_known_density(J):
    """Weighted samples of a 2-D mixture (weights = the density itself on
    uniform points): Adam lowers the loss and the learned q correlates with the
    target density."""
    import torch
    D = 2
    perm, w = init_flow_params(D, 7)
    f = J.Flow(D, perm, w)
    rng = np.random.default_rng(3)
    x = rng.random((65536, D)).astype(np.float32)

    def target(p):
        return (np.exp(-((p[:, 0] - 0.3) ** 2 + (p[:, 1] - 0.6) ** 2) / (2 * 0.05 ** 2))
                + 0.5 * np.exp(-((p[:, 0] - 0.75) ** 2 + (p[:, 1] - 0.25) ** 2) / (2 * 0.08 ** 2)))

    wt = target(x).astype(np.float32)
    xd = torch.from_numpy(np.ascontiguousarray(x.T)).cuda()
    wd = torch.from_numpy(wt).cuda()
    losses = f.train(xd, wd, iters=600, batch=4096, lr=3e-3, seed=1)
    assert losses[-50:].mean() < losses[:10].mean() - 0.5
    g = (np.arange(64) + 0.5) / 64
    G = np.stack(np.meshgrid(g, g), -1).reshape(-1, 2).astype(np.float32)
    lq = f.log_density(torch.from_numpy(np.ascontiguousarray(G.T)).cuda()).cpu().numpy()
    t = target(G.astype(np.float64))
    assert np.corrcoef(np.exp(lq), t)[0, 1] > 0.8
    # the trained parameters still satisfy the oracle's normalisation
    p = f.get_params().reshape(w.shape)
    q = np.exp(FL.log_density(perm, p, G.astype(np.float64))[0])
    assert abs(q.mean() - 1.0) < 0.05
