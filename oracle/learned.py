"""Alg. 2 with a learned regeneration mixture -- TEST INFRASTRUCTURE ONLY.

Jump Restore (Section 7.2, Alg. 2) with mu = beta mu_flow + (1 - beta) uniform
and the killing rate k = c~ u / p of Section 6.2, u = beta q + (1 - beta) the
density of mu (exact: q is the flow's change-of-variables density).  The
steps follow the C oracle's Alg. 2 (oracle/jr_oracle.c) one for one, vectorised
over chains in FP64; the integrand F(x) comes from a callable (the C oracle's
path integrand or an analytic target) and q from oracle/flow.py.

Random numbers: the Philox layout of the C oracle.  Block 0 of a step gives
(U1, U2, Ua, Ub); a regeneration draws from the flow when Ub < beta (then
y = T^{-1}(v) for the step's D uniforms v), else y = v.

A flow of dimension D' < D (perm [L][D']) models the leading D' coordinates
only: mu_flow = q on [0,1)^D' times the uniform density on the other D - D'
coordinates, so u(x) = beta q(x[:D']) + (1 - beta), and a flow draw maps the
first D' uniforms through T^{-1} and keeps the rest.
"""
from __future__ import annotations

import numpy as np

from . import flow as FL
from . import oracle as O

LUM = np.array([0.2126, 0.7152, 0.0722])
TAG_STEP, TAG_INIT, TAG_RESTART = 0, 1, 3


def _coords(seed, tag, chain_begin, n, step, D):
    nblk = (D + 3) // 4
    v = np.concatenate([O.draw_uniforms_many(seed, tag, b + 1, chain_begin, n, step) for b in range(nblk)], axis=1)
    return v[:, :D]


class LearnedChains:
    def __init__(self, F_of, D, width, height, perm=None, w=None, beta=0.0, c_tilde=1.0, sigma=0.01, seed=0,
                 chain_begin=0, n_chains=1, init_from_mu=False):
        self.F_of, self.D, self.W, self.H = F_of, int(D), int(width), int(height)
        self.perm, self.w, self.beta = perm, w, float(beta)
        self.c, self.sigma, self.seed = float(c_tilde), float(sigma), int(seed)
        self.cb, self.n = int(chain_begin), int(n_chains)
        self.step = 0
        self.J = 0
        self.accum = np.zeros((self.H, self.W, 4))
        x = _coords(self.seed, TAG_INIT, self.cb, self.n, 0, self.D)   # x0 ~ uniform (tag 1)
        self._set(x, self.u_of(x))

    def flow_dim(self):
        return len(self.perm[0]) if self.w is not None else self.D

    def u_of(self, x):
        if self.w is None or self.beta == 0.0:
            return np.ones(len(x))
        return FL.regen_density(self.perm, self.w, x[:, :self.flow_dim()], self.beta)

    def _flow_draw(self, v):
        """y = (T^{-1}(v[:, :D']), v[:, D':]) and u(y)."""
        Df = self.flow_dim()
        y = v.copy()
        xf, lq = FL.sample(self.perm, self.w, v[:, :Df])
        y[:, :Df] = xf
        return y, self.beta * np.exp(lq) + (1.0 - self.beta)

    def _set(self, x, u):
        self.x = x
        self.F = self.F_of(x)
        self.p = self.F @ LUM
        self.u = u

    def advance(self, n_steps):
        WH = self.W * self.H
        for _ in range(n_steps):
            s = self.step
            U = O.draw_uniforms_many(self.seed, TAG_STEP, 0, self.cb, self.n, s)
            E1, E2 = -np.log(1.0 - U[:, 0]), -np.log(1.0 - U[:, 1])
            t2 = np.where(self.p > 0, E2 * self.p / (self.c * self.u), 0.0)   # Exp(k), k = c~ u / p
            local = E1 < t2
            dt = np.where(local, E1, t2)
            ok = (dt > 0) & (self.p > 0)
            px = np.minimum(np.floor(self.x[:, 0] * self.W), self.W - 1).astype(int)
            py = np.minimum(np.floor(self.x[:, 1] * self.H), self.H - 1).astype(int)
            wgt = np.where(ok, self.c * dt * WH / np.where(self.p > 0, self.p, 1.0), 0.0)
            np.add.at(self.accum, (py[ok], px[ok], slice(0, 3)), (wgt[ok, None] * self.F[ok]))
            np.add.at(self.accum, (py[ok], px[ok], 3), dt[ok])
            v = _coords(self.seed, TAG_STEP, self.cb, self.n, s, self.D)
            y = np.empty_like(self.x)
            uy = np.ones(self.n)
            # local move: Gaussian small step wrapped on the torus
            R = np.sqrt(-2.0 * np.log(1.0 - v[:, 0::2]))
            ang = 2.0 * np.pi * v[:, 1::2]
            step_xy = np.empty_like(self.x)
            step_xy[:, 0::2] = R * np.cos(ang)
            step_xy[:, 1::2] = R * np.sin(ang)
            yl = self.x + self.sigma * step_xy
            yl = yl - np.floor(yl)
            yl[yl >= 1.0] = 0.0
            y[local] = yl[local]
            # regeneration: flow draw with probability beta, else uniform
            regen = ~local
            use_flow = regen & (U[:, 3] < self.beta) & (self.w is not None)
            uni = regen & ~use_flow
            y[uni] = v[uni]
            if use_flow.any():
                y[use_flow], uy[use_flow] = self._flow_draw(v[use_flow])
            dens = ~use_flow
            if dens.any():
                uy[dens] = self.u_of(y[dens])
            Fy = self.F_of(y)
            py_ = Fy @ LUM
            accept = np.where(local, U[:, 2] * self.p < py_, True)
            self.J += int(regen.sum())
            self.x = np.where(accept[:, None], y, self.x)
            self.F = np.where(accept[:, None], Fy, self.F)
            self.p = np.where(accept, py_, self.p)
            self.u = np.where(accept, uy, self.u)
            self.step += 1

    def image(self):
        return self.accum[:, :, :3] / max(self.J, 1)

    def _draw_candidates(self, tag, key, regen_mask, U, v):
        """Candidates of a regeneration (uniform or flow draw); returns (y, u(y))."""
        y = v.copy()
        uy = np.ones(len(v))
        use_flow = regen_mask & (U[:, 3] < self.beta) & (self.w is not None)
        if use_flow.any():
            y[use_flow], uy[use_flow] = self._flow_draw(v[use_flow])
        dens = ~use_flow
        if dens.any():
            uy[dens] = self.u_of(y[dens])
        return y, uy

    def complete_tours(self, max_steps=1 << 20):
        """Drain, then restart every chain from mu.  Returns the open tours."""
        remaining = self.drain(max_steps)
        self.restart()
        return remaining

    def set_flow(self, perm, w, beta, max_steps=1 << 20):
        """Complete the tours under the old mu, switch mu, restart."""
        remaining = self.drain(max_steps)
        self.perm, self.w, self.beta = perm, w, float(beta)
        self.restart()
        return remaining

    def drain(self, max_steps=1 << 20):
        """Chains inside a tour keep stepping (Alg. 2); a kill ends the tour
        (J += 1) and the chain.  Returns the chains whose tour was still open
        after max_steps."""
        done = np.zeros(self.n, bool)
        WH = self.W * self.H
        k = 0
        while (~done).any() and k < max_steps:
            s = self.step
            act = ~done
            U = O.draw_uniforms_many(self.seed, TAG_STEP, 0, self.cb, self.n, s)
            E1, E2 = -np.log(1.0 - U[:, 0]), -np.log(1.0 - U[:, 1])
            t2 = np.where(self.p > 0, E2 * self.p / (self.c * self.u), 0.0)
            local = (E1 < t2) & act
            kill = act & ~local
            dt = np.where(local, E1, t2)
            ok = act & (dt > 0) & (self.p > 0)
            px = np.minimum(np.floor(self.x[:, 0] * self.W), self.W - 1).astype(int)
            py = np.minimum(np.floor(self.x[:, 1] * self.H), self.H - 1).astype(int)
            wgt = np.where(ok, self.c * dt * WH / np.where(self.p > 0, self.p, 1.0), 0.0)
            np.add.at(self.accum, (py[ok], px[ok], slice(0, 3)), (wgt[ok, None] * self.F[ok]))
            np.add.at(self.accum, (py[ok], px[ok], 3), dt[ok])
            self.J += int(kill.sum())
            done |= kill
            if local.any():
                v = _coords(self.seed, TAG_STEP, self.cb, self.n, s, self.D)
                R = np.sqrt(-2.0 * np.log(1.0 - v[:, 0::2]))
                ang = 2.0 * np.pi * v[:, 1::2]
                st = np.empty_like(self.x)
                st[:, 0::2] = R * np.cos(ang)
                st[:, 1::2] = R * np.sin(ang)
                yl = self.x + self.sigma * st
                yl = yl - np.floor(yl)
                yl[yl >= 1.0] = 0.0
                Fy = self.F_of(yl[local])
                pyv = Fy @ LUM
                acc = U[local, 2] * self.p[local] < pyv
                idx = np.nonzero(local)[0][acc]
                self.x[idx] = yl[idx]
                self.F[idx] = Fy[acc]
                self.p[idx] = pyv[acc]
                self.u[idx] = self.u_of(yl[idx])
            self.step += 1
            k += 1
        return int((~done).sum())

    def restart(self):
        """Every chain starts a new tour from mu (tag 3, the restart count)."""
        self.epochs = getattr(self, "epochs", 0) + 1
        U = O.draw_uniforms_many(self.seed, TAG_RESTART, 0, self.cb, self.n, self.epochs)
        v = _coords(self.seed, TAG_RESTART, self.cb, self.n, self.epochs, self.D)
        y, uy = self._draw_candidates(TAG_RESTART, self.epochs, np.ones(self.n, bool), U, v)
        self._set(y, uy)
