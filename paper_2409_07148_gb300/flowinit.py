"""Seeded initial parameters of the regeneration flow (inputs only).

Layout (the interface documented in include/jr.h, jr_flow_*): D even, A = D/2,
AP = 16 (padded conditioner width), L = 6 layers, H = 64, K = 16 bins.

* perm  int32 [L][D]   -- layer l conditions on coordinates perm[l][:A] and
                          transforms perm[l][A:]
* w     float32 [L][S] -- per layer, in order: W1 [H][AP] (columns >= A are 0),
                          b1 [H], W2 [H][H], b2 [H], W3 [A*K][H], b3 [A*K];
                          S = H*AP + H + H*H + H + A*K*H + A*K

W3 and b3 start at zero, so the initial flow is the identity (uniform density).
This module draws random numbers and lays them out; it computes nothing of the
method.
"""
import numpy as np

L, H, K, AP = 6, 64, 16, 16


def layer_size(D: int) -> int:
    A = D // 2
    return H * AP + H + H * H + H + A * K * H + A * K


def init_flow_params(D: int, seed: int = 0):
    if D % 2 or not 2 <= D <= 32:
        raise ValueError("D must be even, 2..32")
    A = D // 2
    rng = np.random.default_rng(seed)
    perm = np.stack([rng.permutation(D) for _ in range(L)]).astype(np.int32)
    w = np.zeros((L, layer_size(D)), np.float32)
    for l in range(L):
        o = 0
        W1 = np.zeros((H, AP), np.float32)
        W1[:, :A] = rng.normal(0.0, np.sqrt(2.0 / A), (H, A))
        w[l, o:o + H * AP] = W1.ravel()
        o += H * AP
        w[l, o:o + H] = rng.normal(0.0, 0.1, H)
        o += H
        w[l, o:o + H * H] = rng.normal(0.0, np.sqrt(2.0 / H), (H, H)).ravel()
        o += H * H
        w[l, o:o + H] = rng.normal(0.0, 0.1, H)
        o += H
        o += A * K * H + A * K      # W3, b3 = 0: identity flow
        assert o == layer_size(D)
    return perm, w
