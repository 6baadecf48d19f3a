"""Exact finite-state pins of the killing rate and the MH step (CPU only).

Theorem A (supplement) with pi-invariant local dynamics and state-independent
mu: the Jump Restore generator A = (K - I) + diag(k)(1 mu^T - I) satisfies
pi A = 0 iff the killing rate is the one of Section 6.2.  The oracle's own
killing-rate and acceptance functions build A, so a wrong sign, a swapped
p/u, or a wrong acceptance ratio breaks these identities.
"""
import json
import os

import numpy as np

from oracle import finite_state as FS
from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _target(M=64, seed=0):
    rng = np.random.default_rng(seed)
    p = rng.random(M) ** 3 + 1e-6          # spread over six orders of magnitude
    p[::9] *= 1e-4                         # near-zero states
    return p


def test_pi_stationary_uniform_mu():
    p = _target()
    M = len(p)
    mu = np.full(M, 1.0 / M)
    for c_tilde in (1.0, 0.05, 17.0):
        A, _ = FS.jump_restore_generator(p, mu, c_tilde)
        pi = p / p.sum()
        assert np.allclose(A.sum(1), 0.0, atol=1e-9)        # rows of a generator sum to 0
        res = pi @ A
        assert np.abs(res).max() < 1e-12 * np.abs(A).max()


def test_pi_stationary_nonuniform_mu():
    p = _target(seed=1)
    M = len(p)
    rng = np.random.default_rng(2)
    mu = rng.random(M) + 0.1
    mu /= mu.sum()
    A, _ = FS.jump_restore_generator(p, mu, 1.0)
    pi = p / p.sum()
    assert np.abs(pi @ A).max() < 1e-12 * np.abs(A).max()


def test_negative_controls_break_invariance():
    """A constant killing rate, or u/p replaced by p/u, must NOT leave pi
    stationary (guards against a test that cannot fail)."""
    p = _target(seed=3)
    M = len(p)
    mu = np.full(M, 1.0 / M)
    pi = p / p.sum()
    A, _ = FS.jump_restore_generator(p, mu, 1.0, k=np.full(M, 1.0))
    assert np.abs(pi @ A).max() > 1e-4
    A, _ = FS.jump_restore_generator(p, mu, 1.0, k=p / mu)
    assert np.abs(pi @ A).max() > 1e-4


def test_mh_kernel_is_pi_reversible():
    p = _target(seed=4)
    K = FS.mh_ring_kernel(p)
    pi = p / p.sum()
    F = pi[:, None] * K
    assert np.abs(F - F.T).max() < 1e-15
    assert np.all(K >= -1e-15)


def test_embedded_jump_chain_law():
    """The jump chain of Section 7.2 has stationary law proportional to
    p (1 + k) = p + c~ u (derived from pi A = 0 and the holding rate 1 + k)."""
    p = _target(seed=5)
    M = len(p)
    mu = np.full(M, 1.0 / M)
    c_tilde = 0.7
    Pj = FS.jump_chain_matrix(p, mu, c_tilde)
    w, V = np.linalg.eig(Pj.T)
    v = np.real(V[:, np.argmin(np.abs(w - 1.0))])
    v /= v.sum()
    expect = (p + c_tilde * mu) / (p.sum() + c_tilde)
    assert np.abs(v - expect).max() < 1e-10


def test_expected_lifetime_matches_paper_identity():
    """Section 6.2: E_mu[tau] = 1/c = p_lambda / c~.  Computed exactly from
    the killed sub-generator: E[tau] = mu^T (-(K - I - diag k))^{-1} 1."""
    gold = json.load(open(os.path.join(GOLDEN, "paper_example_tour_length.json")))
    p = _target(seed=6)
    M = len(p)
    mu = np.full(M, 1.0 / M)
    p_lambda = p.sum()                     # counting reference measure
    c = gold["c"]
    c_tilde = c * p_lambda
    K = FS.mh_ring_kernel(p)
    k = np.array([O.killing_rate(p[i], mu[i], c_tilde) for i in range(M)])
    sub = K - np.eye(M) - np.diag(k)
    tau = mu @ np.linalg.solve(-sub, np.ones(M))
    assert abs(tau - gold["expected_tour_length"]) < 1e-9


def test_killing_rate_special_values():
    assert O.killing_rate(0.0, 1.0, 1.0) == float("inf")
    assert O.killing_rate(2.0, 1.0, 1.0) == 0.5
    assert O.killing_rate(2.0, 3.0, 4.0) == 6.0
    assert O.mh_accept_prob(0.0, 0.3) == 1.0
    assert O.mh_accept_prob(2.0, 1.0) == 0.5
    assert O.mh_accept_prob(1.0, 2.0) == 1.0
