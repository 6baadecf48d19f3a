"""FP64 oracle of the regeneration flow -- TEST INFRASTRUCTURE ONLY.

The paper has no learned regeneration; this is the library's own addition
(a defensive mixture mu = beta mu_flow + (1 - beta) uniform keeps the density
u = beta q + (1 - beta) exact, so the killing rate k = c~ u / p of Section 6.2
stays exact).  The flow, as the CUDA library defines it:

* L coupling layers; layer l conditions on x[perm[l][:A]] and transforms
  x[perm[l][A:]], A = D/2;
* MLP per layer: h1 = relu(W1 bf16(x_A) + b1), h2 = relu(W2 bf16(h1) + b2),
  o = W3 bf16(h2) + b3 with bf16 weights (products accumulated exactly here,
  in FP32 on the GPU) -- bf16() rounds to nearest even at the GEMM inputs;
* per transformed coordinate j: Q_j = (1 - E) softmax(o[jK:(j+1)K]) + E/K
  (K bins on [0,1), E = 1e-3), a piecewise-constant density K Q_j[bin];
  density direction t -> CDF_j(t), log q += log(K Q_j[bin(t)]);
* sampling direction: layers in reverse order, t = CDF_j^{-1}(c).

Functions take the parameter arrays of paper_2409_07148_gb300.flowinit's
layout (perm [L][D] int32, w [L][S] float32).  The bf16 rounding is written out
(round to nearest even of the float32 value).
"""
from __future__ import annotations

import numpy as np

H, K, AP, E = 64, 16, 16, 1e-3


def bf16(a):
    """Round to bfloat16 (nearest even) via float32; returned as float64."""
    f = np.ascontiguousarray(np.asarray(a, np.float64).astype(np.float32)).view(np.uint32).astype(np.uint64)
    r = ((f + 0x7FFF + ((f >> 16) & 1)) >> 16) << 16
    return (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(w_layer, D):
    A = D // 2
    o = 0
    W1 = w_layer[o:o + H * AP].reshape(H, AP)[:, :A].astype(np.float64)
    o += H * AP
    b1 = w_layer[o:o + H].astype(np.float64)
    o += H
    W2 = w_layer[o:o + H * H].reshape(H, H).astype(np.float64)
    o += H * H
    b2 = w_layer[o:o + H].astype(np.float64)
    o += H
    W3 = w_layer[o:o + A * K * H].reshape(A * K, H).astype(np.float64)
    o += A * K * H
    b3 = w_layer[o:o + A * K].astype(np.float64)
    return W1, b1, W2, b2, W3, b3


def bins(w_layer, xa, D):
    """Bin masses Q [n, A, K] of one layer for conditioner values xa [n, A]."""
    W1, b1, W2, b2, W3, b3 = unpack(w_layer, D)
    h1 = np.maximum(bf16(xa) @ bf16(W1).T + b1, 0.0)
    h2 = np.maximum(bf16(h1) @ bf16(W2).T + b2, 0.0)
    o = bf16(h2) @ bf16(W3).T + b3
    o = o.reshape(len(xa), D // 2, K)
    o = o - o.max(axis=2, keepdims=True)
    e = np.exp(o)
    return (1.0 - E) * e / e.sum(axis=2, keepdims=True) + E / K


def log_density(perm, w, x):
    """log q(x) for rows x [n, D] (density direction).  Also returns z = T(x)."""
    x = np.array(x, np.float64, copy=True)
    n, D = x.shape
    A = D // 2
    lq = np.zeros(n)
    for l in range(len(perm)):
        ca, cb = perm[l][:A], perm[l][A:]
        Q = bins(w[l], x[:, ca], D)
        t = x[:, cb]
        b = np.minimum(np.floor(t * K), K - 1).astype(np.int64)
        cum = np.concatenate([np.zeros((n, A, 1)), np.cumsum(Q, axis=2)], axis=2)
        qb = np.take_along_axis(Q, b[..., None], axis=2)[..., 0]
        cb_lo = np.take_along_axis(cum, b[..., None], axis=2)[..., 0]
        x[:, cb] = cb_lo + (t * K - b) * qb
        lq += np.log(K * qb).sum(axis=1)
    return lq, x


def sample(perm, w, z):
    """x = T^{-1}(z) for rows z [n, D] in [0,1)^D; returns (x, log q(x))."""
    x = np.array(z, np.float64, copy=True)
    n, D = x.shape
    A = D // 2
    lq = np.zeros(n)
    for l in reversed(range(len(perm))):
        ca, cb = perm[l][:A], perm[l][A:]
        Q = bins(w[l], x[:, ca], D)
        c = x[:, cb]
        cum = np.cumsum(Q, axis=2)                       # right edges
        b = np.minimum((cum <= c[..., None]).sum(axis=2), K - 1)
        lo = np.concatenate([np.zeros((n, A, 1)), cum], axis=2)
        clo = np.take_along_axis(lo, b[..., None], axis=2)[..., 0]
        qb = np.take_along_axis(Q, b[..., None], axis=2)[..., 0]
        x[:, cb] = np.clip((b + (c - clo) / qb) / K, 0.0, 1.0 - 2.0 ** -24)
        lq += np.log(K * qb).sum(axis=1)
    return x, lq


def regen_density(perm, w, x, beta):
    """u(x) = beta q(x) + (1 - beta)."""
    lq, _ = log_density(perm, w, x)
    return beta * np.exp(lq) + (1.0 - beta)


def nll_and_grad_torch(perm, w, x, wt):
    """Time-weighted negative log-likelihood -sum wt log q / sum wt and its
    gradient w.r.t. the float32 parameters, by PyTorch CPU float64 autograd.
    bf16 rounding passes gradients straight through (as the GPU backward does)."""
    import torch
    D = x.shape[1]
    A = D // 2
    wt_ = torch.tensor(wt, dtype=torch.float64)
    params = torch.tensor(np.asarray(w, np.float64), requires_grad=True)

    def rb(t):  # straight-through bf16 rounding
        return t + (torch.tensor(bf16(t.detach().numpy())) - t).detach()

    xx = torch.tensor(np.asarray(x, np.float64))
    lq = torch.zeros(len(x), dtype=torch.float64)
    for l in range(len(perm)):
        p = params[l]
        o = 0
        W1 = p[o:o + H * AP].reshape(H, AP)[:, :A]
        o += H * AP
        b1 = p[o:o + H]
        o += H
        W2 = p[o:o + H * H].reshape(H, H)
        o += H * H
        b2 = p[o:o + H]
        o += H
        W3 = p[o:o + A * K * H].reshape(A * K, H)
        o += A * K * H
        b3 = p[o:o + A * K]
        ca = torch.tensor(perm[l][:A].astype(np.int64))
        cbi = torch.tensor(perm[l][A:].astype(np.int64))
        xa = xx[:, ca]
        h1 = torch.relu(rb(xa) @ rb(W1).T + b1)
        h2 = torch.relu(rb(h1) @ rb(W2).T + b2)
        out = (rb(h2) @ rb(W3).T + b3).reshape(len(x), A, K)
        Q = (1.0 - E) * torch.softmax(out, dim=2) + E / K
        t = xx[:, cbi]
        b = torch.clamp(torch.floor(t * K), max=K - 1).long()
        cum = torch.cat([torch.zeros(len(x), A, 1, dtype=torch.float64), torch.cumsum(Q, dim=2)], dim=2)
        qb = torch.gather(Q, 2, b[..., None])[..., 0]
        clo = torch.gather(cum, 2, b[..., None])[..., 0]
        newb = clo + (t * K - b) * qb
        xx = xx.clone()
        xx[:, cbi] = newb
        lq = lq + torch.log(K * qb).sum(dim=1)
    loss = -(wt_ * lq).sum() / wt_.sum()
    loss.backward()
    return float(loss.detach()), params.grad.numpy()


# --------------------------------------------------------------------------
# Rounding margins.  The GPU accumulates the GEMMs in FP32 and runs the
# couplings in FP32, the oracle exactly; the two agree to FP32 rounding except
# where that rounding decides a discrete step: the bf16 rounding of an
# activation (h1, h2, or a conditioner coordinate transformed by an earlier
# layer) or the bin of a coordinate (density: floor(t K); sampling: the CDF
# edge below c).  These functions give, per row, the smallest distance of any
# such value to its decision edge, in units of the FP32 error the GPU can make
# there: ACC_ERR times the sum of the magnitudes that formed an activation, or
# COORD_ERR for a coordinate.  A row with margin < 1 may legitimately take the
# other side on the GPU; every other row must agree to FP32 accuracy.
# The units: FP32 accumulation of <= 64 exact bf16 products plus a bias is
# within 2^-23 (one unit in the last place at 1.0) of the exact sum, relative to
# the sum of the magnitudes; a coordinate in [0, 1) after up to 6 FP32 coupling
# transforms is within 2^-20 of the exact value.
ACC_ERR = 2.0 ** -23
COORD_ERR = 2.0 ** -20


def _bf16_edge_distance(v):
    """Distance of v to the nearest bf16 rounding edge (the midpoint between
    the two bf16 neighbours of float32(v))."""
    v = np.asarray(v, np.float64)
    u = np.ascontiguousarray(v.astype(np.float32)).view(np.uint32).astype(np.uint64)
    lo = (((u >> 16) << 16) & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    hi = ((((u >> 16) + 1) << 16) & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    return np.abs(v - 0.5 * (lo + hi))


def _layer_margin(w_layer, xa, D, first, acc_err, coord_err):
    """Per-row margin (in units of the GPU's error) of one layer's bf16
    roundings: the conditioner coordinates (exact inputs in the first layer)
    and the positive pre-activations of h1 and h2."""
    W1, b1, W2, b2, W3, b3 = unpack(w_layer, D)
    n = len(xa)
    m = np.full(n, np.inf)
    if not first:
        m = np.minimum(m, (_bf16_edge_distance(xa) / coord_err).min(axis=1))
    xb = bf16(xa)
    pre1 = xb @ bf16(W1).T + b1
    s1 = np.abs(xb) @ np.abs(bf16(W1)).T + np.abs(b1)
    m1 = np.where(pre1 > 0, _bf16_edge_distance(pre1) / (acc_err * np.maximum(s1, 1e-300)), np.inf)
    h1 = bf16(np.maximum(pre1, 0.0))
    pre2 = h1 @ bf16(W2).T + b2
    s2 = np.abs(h1) @ np.abs(bf16(W2)).T + np.abs(b2)
    m2 = np.where(pre2 > 0, _bf16_edge_distance(pre2) / (acc_err * np.maximum(s2, 1e-300)), np.inf)
    return np.minimum(m, np.minimum(m1.min(axis=1), m2.min(axis=1)))


def log_density_margin(perm, w, x, acc_err=ACC_ERR, coord_err=COORD_ERR):
    """Per-row rounding margin of log_density (see above)."""
    x = np.array(x, np.float64, copy=True)
    n, D = x.shape
    A = D // 2
    m = np.full(n, np.inf)
    for l in range(len(perm)):
        ca, cb = perm[l][:A], perm[l][A:]
        m = np.minimum(m, _layer_margin(w[l], x[:, ca], D, l == 0, acc_err, coord_err))
        t = x[:, cb]
        tk = t * K
        edge = np.abs(tk - np.round(tk)) / K
        m = np.minimum(m, (edge / coord_err).min(axis=1))
        Q = bins(w[l], x[:, ca], D)
        b = np.minimum(np.floor(tk), K - 1).astype(np.int64)
        cum = np.concatenate([np.zeros((n, A, 1)), np.cumsum(Q, axis=2)], axis=2)
        qb = np.take_along_axis(Q, b[..., None], axis=2)[..., 0]
        x[:, cb] = np.take_along_axis(cum, b[..., None], axis=2)[..., 0] + (tk - b) * qb
    return m


def sample_margin(perm, w, z, acc_err=ACC_ERR, coord_err=COORD_ERR):
    """Per-row rounding margin of sample (see above)."""
    x = np.array(z, np.float64, copy=True)
    n, D = x.shape
    A = D // 2
    m = np.full(n, np.inf)
    L = len(perm)
    for l in reversed(range(L)):
        ca, cb = perm[l][:A], perm[l][A:]
        m = np.minimum(m, _layer_margin(w[l], x[:, ca], D, l == L - 1, acc_err, coord_err))
        Q = bins(w[l], x[:, ca], D)
        c = x[:, cb]
        cum = np.cumsum(Q, axis=2)
        m = np.minimum(m, (np.abs(cum[..., :-1] - c[..., None]) / coord_err).min(axis=(1, 2)))
        b = np.minimum((cum <= c[..., None]).sum(axis=2), K - 1)
        lo = np.concatenate([np.zeros((n, A, 1)), cum], axis=2)
        clo = np.take_along_axis(lo, b[..., None], axis=2)[..., 0]
        qb = np.take_along_axis(Q, b[..., None], axis=2)[..., 0]
        x[:, cb] = np.clip((b + (c - clo) / qb) / K, 0.0, 1.0 - 2.0 ** -24)
    return m
