"""Finite-state Jump Restore generator -- TEST INFRASTRUCTURE ONLY (oracle).

On a finite state space {0..M-1} with counting reference measure lambda, the
Jump Restore process of Section 7 (local dynamics = the continuous-time
embedding, rate 1, of an MH chain; global dynamics = a state-independent
distribution mu with density u; killing rate k) has the generator

    A = (K - I) + diag(k) (1 mu^T - I),

the jump-process form of Section 7.2 ("pure-jump-type transition rule") and of
the rate-kernel generator in supplement A.  Theorem A states that pi A = 0 when
k = c~ u / p and the local chain is pi-invariant (Section 6.2,
"killing-rate-simplified").  The killing rate and the MH acceptance are taken
from the C oracle itself, so these matrices pin those two functions.
"""
from __future__ import annotations

import numpy as np

from . import oracle as _o


def mh_ring_kernel(p: np.ndarray) -> np.ndarray:
    """MH transition matrix (Alg. 1, Section 4) on a ring of M states.

    The proposal moves to one of the two neighbours with probability 1/2 each
    (symmetric, so the acceptance is min(1, p(y)/p(x)))."""
    M = len(p)
    K = np.zeros((M, M))
    for i in range(M):
        for j in ((i - 1) % M, (i + 1) % M):
            K[i, j] += 0.5 * _o.mh_accept_prob(p[i], p[j])
        K[i, i] = 1.0 - K[i].sum()
    return K


def jump_restore_generator(p: np.ndarray, mu: np.ndarray, c_tilde: float, k: np.ndarray | None = None):
    """Generator of the continuous-time Jump Restore process on {0..M-1}.

    mu is the regeneration distribution (its density w.r.t. counting measure is
    u = mu).  If k is None the oracle's killing rate c~ u / p is used."""
    M = len(p)
    K = mh_ring_kernel(p)
    if k is None:
        k = np.array([_o.killing_rate(p[i], mu[i], c_tilde) for i in range(M)])
    A = (K - np.eye(M)) + np.diag(k) @ (np.outer(np.ones(M), mu) - np.eye(M))
    return A, k


def jump_chain_matrix(p: np.ndarray, mu: np.ndarray, c_tilde: float) -> np.ndarray:
    """Embedded jump chain of Section 7.2: (1/(1+k)) K + (k/(1+k)) 1 mu^T."""
    M = len(p)
    K = mh_ring_kernel(p)
    k = np.array([_o.killing_rate(p[i], mu[i], c_tilde) for i in range(M)])
    a = 1.0 / (1.0 + k)
    return a[:, None] * K + (1.0 - a)[:, None] * np.outer(np.ones(M), mu)


def mh_mixture_kernel(p: np.ndarray, mu: np.ndarray, ell: float, accept=None) -> np.ndarray:
    """MH transition matrix of the baseline "Metropolis" (Alg. 1 with the
    mixture proposal of Section 5, Q_l(x, .) = l mu + (1 - l) zeta(x, .)) on a
    ring of M states, zeta = one step to either neighbour with probability 1/2.

    With mu uniform Q_l is symmetric, so the acceptance is the oracle's
    min(1, p(y)/p(x)); `accept(px, py)` replaces it (negative controls)."""
    M = len(p)
    acc = accept if accept is not None else _o.mh_accept_prob
    Q = ell * np.outer(np.ones(M), mu)
    for i in range(M):
        Q[i, (i - 1) % M] += 0.5 * (1.0 - ell)
        Q[i, (i + 1) % M] += 0.5 * (1.0 - ell)
    K = np.zeros((M, M))
    for i in range(M):
        for j in range(M):
            if j != i and Q[i, j] > 0.0:
                K[i, j] = Q[i, j] * acc(p[i], p[j])
        K[i, i] = 1.0 - K[i].sum()
    return K


def restore_generator_general(p: np.ndarray, K: np.ndarray, M: np.ndarray, kappa: float, k: np.ndarray | None = None):
    """Generator of the Restore process with general local dynamics and transfer
    kernel (Section 6.1, eq. "killing-rate"; supplement, Theorem A) on
    {0..M-1} with counting reference measure:

        A = (K - I) + diag(k) (M - I),

    local dynamics = rate-1 jumps by the Markov matrix K (not necessarily
    pi-invariant), transfer rule mu(exit, .) = row `exit` of M, and
    k_x = ((L* + kappa mu*) p)_x / p_x with L = K - I, (L* p)_x = (p K)_x - p_x
    and (mu* p)_x = (p M)_x, formed by the oracle's killing_rate_general.
    Returns (A, k); k may come out negative when kappa is too small."""
    n = len(p)
    ls = p @ K - p
    ms = p @ M
    if k is None:
        k = np.array([_o.killing_rate_general(p[i], ls[i], kappa * ms[i]) for i in range(n)])
    A = (K - np.eye(n)) + np.diag(k) @ (M - np.eye(n))
    return A, k
