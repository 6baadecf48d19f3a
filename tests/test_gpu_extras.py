"""GPU checks of the library's instrumentation and training-data entry
points: jr_advance_timed, jr_chains_snapshot_append (ring of training rows),
jr_flow_train_rows and jr_flow_get_status (needs a GB300)."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("execution,n", [("wave", 1 << 16), ("mega", 300)])
def test_advance_timed_is_advance(J, execution, n):
    """The timed advance runs the same steps: identical states, the same
    estimate, and one timed launch per kernel of the step sequence."""
    sc = scenes.cornell(width=32, height=32, depth=3)
    g = J.Scene(sc)
    a = J.Chains(g, 32, 32, sc.depth, n, seed=7)
    b = J.Chains(g, 32, 32, sc.depth, n, seed=7)
    a.set_execution(execution)
    b.set_execution(execution)
    a.advance(8)
    split = b.advance_timed(8)
    xa, fa = a.get_state()
    xb, fb = b.get_state()
    assert np.array_equal(xa, xb) and np.array_equal(fa, fb)
    assert a.stats() == b.stats()
    assert np.allclose(a.accumulator(), b.accumulator(), rtol=1e-6, atol=1e-9)
    if execution == "wave":
        assert split["step"]["launches"] == 9 and split["path"]["launches"] == 8
    else:
        assert split["step"]["launches"] == 1 and split["path"]["launches"] == 0
    assert split["flow"]["launches"] == 0 and split["reserved"]["launches"] == 0
    assert all(v["ms"] >= 0.0 for v in split.values()) and split["step"]["ms"] > 0.0


def test_snapshot_append_keeps_the_rows_of_positive_weight(J):
    sc = scenes.cornell(width=16, height=16, depth=3)
    g = J.Scene(sc)
    ch = J.Chains(g, 16, 16, sc.depth, 4096, seed=3)
    ch.set_execution("wave")
    ch.advance(6)
    x, w = J.snapshot(ch)
    x, w = x.cpu().numpy(), w.cpu().numpy()
    keep = w > 0
    k = int(keep.sum())
    assert 0 < k < len(w)
    cap = k + k // 2
    buf = J.ReplayBuffer(sc.D, cap)
    buf.append(ch)
    assert buf.rows() == k and int(buf.total.item()) == k
    rows = np.concatenate([buf.x[:, :k].cpu().numpy(), buf.w[None, :k].cpu().numpy()], 0).T
    want = np.concatenate([x[:, keep], w[None, keep]], 0).T
    order = lambda r: r[np.lexsort(r.T[::-1])]
    assert np.array_equal(order(rows), order(want))
    buf.append(ch)  # the same rows again: they wrap around the ring
    assert int(buf.total.item()) == 2 * k and buf.rows() == cap
    assert np.all(buf.w.cpu().numpy() > 0)


def test_train_rows_reads_only_the_filled_rows(J):
    """Training on the first n_rows of a wider ring follows training on a
    compact copy of those rows (same minibatch windows); the unfilled slots
    hold NaN and must not be read.  Gradients are summed with atomics, so two
    runs differ by rounding; Adam's normalised steps turn that into small
    parameter differences, hence the norm tolerance."""
    import torch
    D, n_rows, stride = 8, 4096, 6000
    perm, w0 = init_flow_params(D, 5)
    rng = np.random.default_rng(2)
    x = rng.random((D, n_rows)).astype(np.float32)
    wt = (rng.random(n_rows) + 0.1).astype(np.float32)
    ring_x = np.full((D, stride), np.nan, np.float32)
    ring_w = np.full(stride, np.nan, np.float32)
    ring_x[:, :n_rows], ring_w[:n_rows] = x, wt

    class Ring:
        pass

    r = Ring()
    r.x, r.w, r.capacity = torch.from_numpy(ring_x).cuda(), torch.from_numpy(ring_w).cuda(), stride
    r.rows = lambda: n_rows
    fa, fb = J.Flow(D, perm, w0), J.Flow(D, perm, w0)
    la = fa.train_replay(r, iters=20, batch=1024, lr=2e-3, seed=9)
    lb = fb.train(torch.from_numpy(x).cuda(), torch.from_numpy(wt).cuda(), iters=20, batch=1024, lr=2e-3, seed=9)
    assert np.isfinite(la).all()
    # the loss before any update and after the first one agree to rounding; from
    # the second Adam step on, the atomics' summation order (which varies from run
    # to run) reaches the losses through Adam's normalisation of near-zero gradients
    assert np.allclose(la[:2], lb[:2], rtol=1e-5, atol=1e-6)
    assert np.abs(la - lb).max() <= 3e-3
    pa, pb = fa.get_params().astype(np.float64), fb.get_params().astype(np.float64)
    assert np.isfinite(pa).all()
    assert np.linalg.norm(pa - pb) <= 0.1 * np.linalg.norm(pb - w0.ravel())
    assert fa.status() == 0 and fb.status() == 0


def test_drain_stopped_by_its_step_limit(J):
    """A drain cut off after max_steps reports the tours still open and
    advances the step counter by exactly max_steps; an unlimited drain of the
    same chains finishes every tour and takes more steps."""
    sc = scenes.cornell(width=16, height=16, depth=3)
    g = J.Scene(sc)
    a = J.Chains(g, 16, 16, sc.depth, 1 << 16, seed=21, sigma=0.02)
    b = J.Chains(g, 16, 16, sc.depth, 1 << 16, seed=21, sigma=0.02)
    for ch in (a, b):
        ch.set_execution("wave")
        ch.advance(5)
    s0 = a.stats()["steps_per_chain"]
    assert J.complete_tours(a, max_steps=3) > 0
    assert a.stats()["steps_per_chain"] == s0 + 3
    assert J.complete_tours(b) == 0
    assert b.stats()["steps_per_chain"] - s0 > 3
    assert b.stats()["regenerations"] > a.stats()["regenerations"]
