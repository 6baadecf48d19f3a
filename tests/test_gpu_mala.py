"""Langevin local dynamics (JR_FLAG_MALA) on the GPU against the FP64 oracle,
through the C ABI (needs a GB300).

* The gradient of the path contribution (jr_eval_grad, forward mode in FP32)
  against the oracle's FP64 forward mode on identical states: every component
  within 1e-4 of the gradient's scale (|dF| + 1e-2 |F|; FP32 propagates the
  derivatives through up to depth products of Jacobians), on states whose hit
  sequence agrees.
* One MALA step at a time from the GPU's state (megakernel, traced), replayed
  by the oracle on the same counters: MALA Restore and the MALA baseline
  (large steps l = 0.3).  The oracle takes the drift from its own FP64 gradient
  at the GPU's state, so proposals agree to FP32 rounding; decisions must agree
  except at ties of the acceptance ratio and FP32 topology differences.
* MALA Restore on a glossy box: independent batches against a converged
  path-traced reference (per pixel where the batch means are in the
  central-limit regime, and in tiles).
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from paper_2409_07148_gb300 import scenes
from tests.gpu_util import rel_err, torus_diff

pytestmark = pytest.mark.gpu
SIG = 0.02
ELL = float(np.float32(0.3))
LUM = np.array([0.2126, 0.7152, 0.0722])


@pytest.fixture(scope="module")
def J():
    import torch
    assert torch.cuda.is_available()
    from paper_2409_07148_gb300 import jr
    jr.lib()
    return jr


def glossy_box(width=16, height=16, depth=3, n=10.0):
    sc = scenes.cornell(width=width, height=height, depth=depth)
    mats = sc.mats.copy()
    dull = ~np.any(mats[:, 4:7] > 0, axis=1)
    mats[dull, 0] = scenes.PHONG
    mats[dull, 7] = n
    return scenes.SceneArrays("glossy_box", sc.verts, sc.tris, sc.tri_mat, mats, sc.camera, width, height, depth)


@pytest.mark.parametrize("which", ["glossy_box", "spheres"])
def test_gradient_matches_oracle(J, which):
    import torch
    if which == "glossy_box":
        sc, bvh = glossy_box(), False
    else:
        sc, bvh = scenes.cornell_spheres(width=32, height=32, depth=4, n_lon=40, n_lat=21), True
    osc = O.Scene(sc, bvh=bvh)
    x = np.random.default_rng(1).random((60_000 if which == "glossy_box" else 800_000, sc.D)).astype(np.float32)
    _, p0, _, _ = O.eval_states(osc, x.astype(np.float64))
    x = x[p0 > 0][:3000]
    assert len(x) >= 500
    F, dF = J.eval_grad(J.Scene(sc), torch.from_numpy(np.ascontiguousarray(x.T)).cuda(), sc.depth)
    torch.cuda.synchronize()
    Fg = F.cpu().numpy().T                       # [n, 3]
    dFg = dF.cpu().numpy().transpose(2, 0, 1)    # [n, 3, D]
    Fo, dFo = O.eval_grad(osc, x.astype(np.float64))
    _, _, _, _, io = O.eval_states(osc, x.astype(np.float64), hit_ids=True)
    gid = J.eval_states(J.Scene(sc), torch.from_numpy(np.ascontiguousarray(x.T)).cuda(), sc.depth, hit_ids=True)[4]
    same = np.all(gid.cpu().numpy().T == io, axis=1)
    assert np.mean(same) > 0.99
    # diffuse bounces make F piecewise constant in x (cosine sampling cancels the
    # BSDF's cosine), so only paths through a Phong surface carry a gradient: most
    # entries on the glossy box, a few percent on the spheres scene (one glossy sphere)
    floor = 0.1 if which == "glossy_box" else 0.01
    assert np.count_nonzero(dFo[same]) > floor * dFo[same].size
    scale = np.abs(dFo[same]) + 1e-2 * np.abs(Fo[same])[:, :, None] + 1e-6
    err = np.abs(dFg[same] - dFo[same]) / scale
    assert np.mean(err > 1e-4) < 1e-3, np.sort(err.ravel())[-5:]
    # F to 1e-5 (up to 0.5 % of entries to 1e-4: a grazing Phong bounce, cos theta_i
    # near 0, is ill-conditioned in FP32 through up to three such bounces)
    rf = rel_err(Fg[same][Fo[same] > 0], Fo[same][Fo[same] > 0])
    assert np.mean(rf > 1e-5) <= 5e-3 and rf.max() <= 1e-4, np.sort(rf)[-5:]


def _replay(J, sc, osc, n, steps, seed, method):
    import torch
    g = J.Scene(sc)
    flags = J.JR_FLAG_MALA | (J.JR_FLAG_MH if method == "mh" else 0)
    ch = J.Chains(g, sc.width, sc.height, sc.depth, n, seed=seed, sigma=SIG, flags=flags, large_step=ELL, burn_in=2)
    oc = O.MALAChains(osc, sc.D, sc.width, sc.height, sigma=SIG, method=method, ell=ELL, burn_in=2, seed=seed,
                      n_chains=n)
    fl = torch.empty(n, dtype=torch.uint8, device="cuda")
    dt = torch.empty(n, dtype=torch.float32, device="cuda")
    px = torch.empty(n, dtype=torch.int32, device="cuda")
    summ = dict(steps=0, checked=0, flips=0, topo=0)
    x, fpu = ch.get_state()
    for s in range(steps):
        xs = x.T.astype(np.float64)
        F, dF = O.eval_grad(osc, xs)
        p = F @ LUM
        gr = np.where(p[:, None] > 0, np.einsum("c,ncd->nd", LUM, dF) / np.where(p > 0, p, 1)[:, None], 0.0)
        oc.state[:, :sc.D] = xs
        oc.state[:, sc.D:sc.D + 3] = fpu[:3].T
        oc.state[:, sc.D + 3] = fpu[3]
        oc.state[:, sc.D + 4] = fpu[4]
        oc.state[:, sc.D + 5:] = np.clip(0.5 * SIG ** 2 * gr, -2 * SIG, 2 * SIG)
        oc.step = s
        tr = oc.advance(1, trace=True, margins=True)
        ch.advance_traced(1, fl, dt, px)
        x2, fpu2 = ch.get_state()
        gf, of, om = fl.cpu().numpy(), tr["flags"][:, 0], tr["margin"][:, 0]
        if method == "mh":
            assert np.array_equal(gf & 1, of & 1)          # the large-step choice
        same_branch = (gf & 1) == (of & 1)
        same = same_branch & ((gf & 2) == (of & 2))
        flip = ~same
        summ["flips"] += int(flip.sum())
        # a decision flip needs a near-tie (in log space for MALA moves) or a topology difference
        near = np.abs(om[flip]) <= 1e-3 * (1 + np.abs(om[flip]))
        summ["topo"] += int((~near).sum())
        dx = torus_diff(x2[:, same].T, oc.state[same, :sc.D]).max(axis=1)
        ref = oc.state[same, sc.D:sc.D + 4]
        eF = rel_err(fpu2[:4, same].T, ref)
        ok = (dx <= 2e-6) & np.all((eF <= 1e-5) | ((ref == 0) & (fpu2[:4, same].T == 0)), axis=1)
        summ["topo"] += int((~ok).sum())
        summ["checked"] += int(same.sum())
        summ["steps"] += n
        x, fpu = x2, fpu2
    return summ, ch


@pytest.mark.parametrize("method", ["restore", "mh"])
def test_mala_step_replay(J, method):
    sc = glossy_box()
    s, ch = _replay(J, sc, O.Scene(sc), 512, 20, seed=3, method=method)
    assert s["checked"] >= 0.98 * s["steps"], s
    assert s["topo"] <= 1e-2 * s["steps"], s
    assert ch.stats()["status_word"] == 0


def test_mala_restore_image_matches_path_tracing(J):
    import torch
    from scipy import stats
    sc = glossy_box(width=16, height=16)
    g = J.Scene(sc)
    acc = torch.zeros((sc.height, sc.width, 4), dtype=torch.float64, device="cuda")
    n, chunk = 1 << 32, 1 << 28
    for s0 in range(0, n, chunk):
        J.render_pt(g, sc.width, sc.height, sc.depth, chunk, seed=77, sample_begin=s0, accum=acc)
    torch.cuda.synchronize()
    ref = (acc[..., :3] / n).cpu().numpy()
    # 32 batches of 512 chains x 20 000 steps: a run stopped at a fixed step
    # carries an open-tour bias of order chains / J (MALA sets have no drain, which
    # runs in the wavefront), here about 5e-5, far below the batch noise
    sets, streams = [], []
    for b in range(32):
        st = torch.cuda.Stream()
        c = J.Chains(g, sc.width, sc.height, sc.depth, 512, seed=9, sigma=SIG, flags=J.JR_FLAG_MALA,
                     chain_offset=512 * b, stream=st)
        c.advance(20_000, stream=st)
        sets.append(c)
        streams.append(st)
    torch.cuda.synchronize()
    imgs = []
    for c, st in zip(sets, streams):
        imgs.append(c.resolve(stream=st))
        assert c.stats(stream=st)["status_word"] == 0
    imgs = np.array(imgs, np.float64)
    img = imgs.mean(0)
    se = imgs.std(0, ddof=1) / np.sqrt(len(imgs))
    dense = (np.count_nonzero(imgs, axis=0) >= 24) & (se > 0)
    t = (img - ref)[dense] / se[dense]
    z = np.sign(t) * stats.norm.isf(stats.t.sf(np.abs(t), len(imgs) - 1))
    assert np.mean(np.abs(z) > 4) <= 1e-3 and np.abs(z).max() < 6, np.sort(np.abs(z))[-5:]
    assert float(np.mean((img - ref) ** 2 / (ref ** 2 + 1e-2))) < 2e-3


def test_mala_api_refusals(J):
    sc = glossy_box(width=8, height=8)
    g = J.Scene(sc)
    lib = J.lib()
    h = ctypes.c_void_p()
    p = J.make_params(8, 8, sc.depth, n_chains=4, flags=J.JR_FLAG_MALA | J.JR_FLAG_RAO_BLACKWELL)
    assert lib.jr_chains_create(g.h, ctypes.byref(p), None, ctypes.byref(h)) == J.JR_ERR_INVALID_ARG
    ch = J.Chains(g, 8, 8, sc.depth, 64, seed=1, sigma=SIG, flags=J.JR_FLAG_MALA)
    assert lib.jr_advance_static(ch.h, 2, None) == J.JR_ERR_STATE
    assert lib.jr_complete_tours(ch.h, 5, None, None) == J.JR_ERR_STATE
    with pytest.raises(J.JRError):
        J.Batch([ch])
    ch.advance(3)
    st = ch.stats()
    assert st["regenerations"] + st["local_steps"] == 3 * 64
