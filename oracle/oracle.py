"""FP64 CPU oracle for Jump Restore light transport -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this module.  It shares no code with the CUDA library; it compiles
``jr_oracle.c`` with the host C compiler into ``oracle/_build/liboracle.so`` and
marshals numpy arrays through ctypes.

Every numerical step lives in ``jr_oracle.c`` (Alg. 2 of Section 7.2, the
killing rate of Section 6.2, the MH step of Section 4, the estimator of
Sections 6.3/7.4, the PSS path integrand).  Functions here only convert arrays.

Parity status: every function is pinned (see tests/test_oracle_*.py), except
the Philox stream layout itself, which is a reading (the paper fixes no RNG);
the Philox permutation is pinned against an independent implementation.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

MAT_FLOATS = 12
TAG_STEP, TAG_INIT, TAG_PT = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, -O2, no machine-specific flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-pthread",
               "-fvisibility=hidden", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            P, D, U64, I, U32 = ctypes.c_void_p, ctypes.c_double, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32
            L.orc_philox4x32_10.argtypes = [P, P, P]
            L.orc_draw_uniforms.argtypes = [U64, U32, U32, U32, U64, P]
            L.orc_draw_uniforms_many.argtypes = [U64, U32, U32, U32, U64, U64, P]
            L.orc_scene_create.argtypes = [P, I, P, I, P, P, I, P]
            L.orc_scene_create.restype = P
            L.orc_scene_destroy.argtypes = [P]
            L.orc_scene_build_bvh.argtypes = [P]
            L.orc_scene_build_bvh.restype = I
            L.orc_intersect_triangle.argtypes = [P, P, P, P, P]
            L.orc_intersect_triangle.restype = D
            L.orc_closest_hit.argtypes = [P, P, P, I, P]
            L.orc_closest_hit.restype = I
            L.orc_fresnel.argtypes = [D, D, D]
            L.orc_fresnel.restype = D
            L.orc_scatter.argtypes = [P, P, P, D, D, P, P]
            L.orc_scatter.restype = I
            L.orc_analytic_create.argtypes = [P]
            L.orc_analytic_create.restype = P
            L.orc_analytic_destroy.argtypes = [P]
            L.orc_analytic_eval.argtypes = [P, I, I, P, P]
            L.orc_killing_rate.argtypes = [D, D, D]
            L.orc_killing_rate.restype = D
            L.orc_mh_accept_prob.argtypes = [D, D]
            L.orc_mh_accept_prob.restype = D
            L.orc_chains_init.argtypes = [I, P, P, I, I, I, I, D, D, U64, U64, U64, P]
            L.orc_chains_advance.argtypes = [I, P, P, I, I, I, I, D, D, U64, I, U64, U64, U64, U64,
                                             P, P, P, P, P, P, P, I]
            L.orc_chains_advance.restype = I
            L.orc_mh_advance.argtypes = [I, P, P, I, I, I, I, D, D, U64, U64, U64, U64, U64, U64, P, P, P, P,
                                         P, P, P, I]
            L.orc_mh_advance.restype = I
            L.orc_eval_grad.argtypes = [P, I, I, U64, P, P, P]
            L.orc_analytic_grad.argtypes = [P, I, U64, P, P, P]
            L.orc_mala_init.argtypes = [I, P, P, I, I, D, U64, U64, U64, P]
            L.orc_mala_advance.argtypes = [I, P, P, I, I, I, I, D, D, I, D, U64, U64, U64, U64, U64, U64, P, P, P,
                                           P, P, P, P, I]
            L.orc_mala_advance.restype = I
            L.orc_killing_rate_general.argtypes = [D, D, D]
            L.orc_killing_rate_general.restype = D
            L.orc_lstar_p_1d.argtypes = [P, I, P, D, I, P]
            L.orc_general_init.argtypes = [P, D, D, I, I, U64, U64, U64, P]
            L.orc_general_advance.argtypes = [P, I, D, D, I, I, U64, U64, U64, U64, U64, P, P, I]
            L.orc_general_advance.restype = U64
            L.orc_eval_states.argtypes = [I, P, P, I, I, D, U64, P, P, P, P, P, P]
            L.orc_render_pt.argtypes = [I, P, P, I, I, I, I, U64, U64, U64, P, I]
            L.orc_threads_default.restype = I
            L.orc_state_stride.argtypes = [I]
            L.orc_state_stride.restype = I
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------- primitives
def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def draw_uniforms(seed, tag, block, chain, step):
    o = np.zeros(4, dtype=np.float64)
    lib().orc_draw_uniforms(seed, tag, block, chain, step, _ptr(o))
    return o


def draw_uniforms_many(seed, tag, block, chain_begin, n, step):
    """Philox block `block` of chains chain_begin .. +n at one step: [n, 4] uniforms."""
    o = np.zeros((int(n), 4), dtype=np.float64)
    lib().orc_draw_uniforms_many(int(seed), int(tag), int(block), int(chain_begin), int(n), int(step), _ptr(o))
    return o


def killing_rate(p, u, c_tilde):
    return lib().orc_killing_rate(float(p), float(u), float(c_tilde))


def mh_accept_prob(px, py):
    return lib().orc_mh_accept_prob(float(px), float(py))


def intersect_triangle(o, d, v0, v1, v2):
    a = [np.ascontiguousarray(np.asarray(v, dtype=np.float64)) for v in (o, d, v0, v1, v2)]
    return lib().orc_intersect_triangle(*[_ptr(v) for v in a])


def fresnel(cos_i, eta_i, eta_t):
    return lib().orc_fresnel(cos_i, eta_i, eta_t)


def scatter(mat12, d, ng, u1, u2):
    m = np.ascontiguousarray(np.asarray(mat12, dtype=np.float32))
    dd = np.ascontiguousarray(np.asarray(d, dtype=np.float64))
    nn = np.ascontiguousarray(np.asarray(ng, dtype=np.float64))
    wi = np.zeros(3)
    w = np.zeros(3)
    ok = lib().orc_scatter(_ptr(m), _ptr(dd), _ptr(nn), float(u1), float(u2), _ptr(wi), _ptr(w))
    return ok, wi, w


# ---------------------------------------------------------------- targets
class Scene:
    """Oracle copy (FP64) of a scene made by the seeded scene generator."""

    def __init__(self, sc, bvh: bool = False):
        self.sc = sc
        self._keep = [np.ascontiguousarray(sc.verts, dtype=np.float32),
                      np.ascontiguousarray(sc.tris, dtype=np.uint32),
                      np.ascontiguousarray(sc.tri_mat, dtype=np.uint32),
                      np.ascontiguousarray(sc.mats, dtype=np.float32),
                      np.ascontiguousarray(sc.camera, dtype=np.float32)]
        v, t, tm, m, cam = self._keep
        self.h = lib().orc_scene_create(_ptr(v), v.shape[0], _ptr(t), t.shape[0], _ptr(tm), _ptr(m), m.shape[0],
                                        _ptr(cam))
        if not self.h:
            raise ValueError("oracle: invalid scene arrays")
        self.n_nodes = lib().orc_scene_build_bvh(self.h) if bvh else 0
        self.kind, self.analytic = 0, None

    def closest_hit(self, o, d, use_bvh=False):
        oo = np.ascontiguousarray(o, dtype=np.float64)
        dd = np.ascontiguousarray(d, dtype=np.float64)
        t = ctypes.c_double(0.0)
        i = lib().orc_closest_hit(self.h, _ptr(oo), _ptr(dd), int(use_bvh), ctypes.byref(t))
        return i, t.value

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_scene_destroy(self.h)
            self.h = None


class Analytic:
    """Analytic target on [0,1)^D: Gaussian bumps in (x0, x1), a zero band in x0."""

    def __init__(self, modes, band=(0.0, 0.0)):
        prm = [len(modes), band[0], band[1]]
        for (w, m0, m1, s) in modes:
            prm += [w, m0, m1, s]
        self._prm = np.ascontiguousarray(prm, dtype=np.float64)
        self.h = lib().orc_analytic_create(_ptr(self._prm))

    def eval(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        n, D = x.shape
        F = np.zeros((n, 3))
        lib().orc_analytic_eval(self.h, D, n, _ptr(x), _ptr(F))
        return F

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_analytic_destroy(self.h)
            self.h = None


def _target(t):
    if isinstance(t, Scene):
        return 0, t.h, None
    return 1, None, t.h


class Chains:
    """A set of Jump Restore chains run by the oracle (Alg. 2)."""

    def __init__(self, target, D, width, height, c_tilde=1.0, sigma=0.01, seed=0, depth=None, chain_begin=0,
                 n_chains=1, rao_blackwell=False):
        self.target = target
        self.kind, self.sh, self.ah = _target(target)
        self.D = int(D)
        self.depth = int(depth) if depth is not None else (self.D - 2) // 2
        self.W, self.H = int(width), int(height)
        self.c_tilde, self.sigma, self.seed = float(c_tilde), float(sigma), int(seed)
        self.rb = int(bool(rao_blackwell))
        self.chain_begin, self.n = int(chain_begin), int(n_chains)
        self.S = lib().orc_state_stride(self.D)
        self.state = np.zeros((self.n, self.S))
        lib().orc_chains_init(self.kind, self.sh, self.ah, self.D, self.depth, self.W, self.H, self.c_tilde,
                              self.sigma, self.seed, self.chain_begin, self.n, _ptr(self.state))
        self.accum = np.zeros((self.H, self.W, 4))
        self.step = 0
        self.J = 0
        self.accepts = 0
        self.locals = 0

    @property
    def x(self):
        return self.state[:, :self.D]

    @property
    def F(self):
        return self.state[:, self.D:self.D + 3]

    @property
    def p(self):
        return self.state[:, self.D + 3]

    def advance(self, n_steps, trace=False, margins=False, n_threads=0):
        out = np.zeros(3, dtype=np.uint64)
        tr = None
        if trace:
            tr = dict(flags=np.zeros((self.n, n_steps), np.uint8), dt=np.zeros((self.n, n_steps)),
                      pix=np.zeros((self.n, n_steps), np.int32),
                      margin=np.zeros((self.n, n_steps, 2)) if margins else None)
        rc = lib().orc_chains_advance(
            self.kind, self.sh, self.ah, self.D, self.depth, self.W, self.H, self.c_tilde, self.sigma, self.seed,
            self.rb, self.chain_begin, self.n, self.step, n_steps, _ptr(self.state), _ptr(self.accum), _ptr(out),
            _ptr(tr["flags"]) if tr else None, _ptr(tr["dt"]) if tr else None, _ptr(tr["pix"]) if tr else None,
            _ptr(tr["margin"]) if tr and margins else None, int(n_threads))
        if rc != 0:
            raise ValueError("oracle: invalid dimension")
        self.step += n_steps
        self.J += int(out[0])
        self.accepts += int(out[1])
        self.locals += int(out[2])
        return tr

    def image(self):
        """Normalisation-free estimate (Section 6.3): accum / J."""
        return self.accum[:, :, :3] / max(self.J, 1)


class MHChains:
    """MH chains with the mixture proposal l mu + (1 - l) zeta (the baseline
    "Metropolis" of Section 8) run by the oracle; x0 ~ mu as for Restore."""

    def __init__(self, target, D, width, height, sigma=0.01, ell=0.3, burn_in=10_000, seed=0, depth=None,
                 chain_begin=0, n_chains=1):
        self.target = target
        self.kind, self.sh, self.ah = _target(target)
        self.D = int(D)
        self.depth = int(depth) if depth is not None else (self.D - 2) // 2
        self.W, self.H = int(width), int(height)
        self.sigma, self.ell, self.burn_in, self.seed = float(sigma), float(ell), int(burn_in), int(seed)
        self.chain_begin, self.n = int(chain_begin), int(n_chains)
        self.S = lib().orc_state_stride(self.D)
        self.state = np.zeros((self.n, self.S))
        lib().orc_chains_init(self.kind, self.sh, self.ah, self.D, self.depth, self.W, self.H, 1.0, self.sigma,
                              self.seed, self.chain_begin, self.n, _ptr(self.state))
        self.accum = np.zeros((self.H, self.W, 4))
        self.step = 0
        self.n_large = self.n_small = self.accepts = self.splats = 0
        self.p_sum_large = 0.0

    x = Chains.x
    F = Chains.F
    p = Chains.p

    def advance(self, n_steps, trace=False, margins=False, n_threads=0):
        out = np.zeros(4, dtype=np.uint64)
        ps = np.zeros(1)
        tr = None
        if trace:
            tr = dict(flags=np.zeros((self.n, n_steps), np.uint8), pix=np.zeros((self.n, n_steps), np.int32),
                      margin=np.zeros((self.n, n_steps)) if margins else None)
        rc = lib().orc_mh_advance(
            self.kind, self.sh, self.ah, self.D, self.depth, self.W, self.H, self.sigma, self.ell, self.burn_in,
            self.seed, self.chain_begin, self.n, self.step, n_steps, _ptr(self.state), _ptr(self.accum), _ptr(out),
            _ptr(ps), _ptr(tr["flags"]) if tr else None, _ptr(tr["pix"]) if tr else None,
            _ptr(tr["margin"]) if tr and margins else None, int(n_threads))
        if rc != 0:
            raise ValueError("oracle: invalid dimension or large-step probability")
        self.step += n_steps
        self.n_large += int(out[0])
        self.n_small += int(out[1])
        self.accepts += int(out[2])
        self.splats += int(out[3])
        self.p_sum_large += float(ps[0])
        return tr

    def b_hat(self):
        """Estimate of b = integral of p from the large-step proposals."""
        return self.p_sum_large / max(self.n_large, 1)

    def image(self):
        """MH ergodic-average estimate: b_hat * accum / N."""
        return self.b_hat() * self.accum[:, :, :3] / max(self.splats, 1)


def eval_grad(target, x, depth=None):
    """F [n, 3] and dF/dx [n, 3, D] of a scene integrand (forward mode) or of
    an analytic target (closed form)."""
    x = np.ascontiguousarray(x, np.float64)
    n, D = x.shape
    dep = int(depth) if depth is not None else (D - 2) // 2
    F = np.zeros((n, 3))
    dF = np.zeros((n, 3, D))
    if isinstance(target, Scene):
        lib().orc_eval_grad(target.h, D, dep, n, _ptr(x), _ptr(F), _ptr(dF))
    else:
        lib().orc_analytic_grad(target.h, D, n, _ptr(x), _ptr(F), _ptr(dF))
    return F, dF


class MALAChains:
    """Chains with Langevin (MALA) local moves on a scene target: method
    "restore" (MALA Restore: Jump Restore, k = c~ u / p) or "mh" (the MALA
    baseline: large steps with probability l, MALA small steps)."""

    def __init__(self, target, D, width, height, sigma=0.01, c_tilde=1.0, method="restore", ell=0.3, burn_in=0,
                 seed=0, chain_begin=0, n_chains=1, depth=None):
        self.target, self.D = target, int(D)
        self.kind, self.sh, self.ah = _target(target)
        self.depth = int(depth) if depth is not None else (self.D - 2) // 2
        self.W, self.H = int(width), int(height)
        self.sigma, self.c_tilde, self.ell, self.burn_in = float(sigma), float(c_tilde), float(ell), int(burn_in)
        self.method = {"restore": 0, "mh": 1, "mh_uncorrected": 2}[method]
        self.seed, self.cb, self.n = int(seed), int(chain_begin), int(n_chains)
        self.state = np.zeros((self.n, 2 * self.D + 5))
        lib().orc_mala_init(self.kind, self.sh, self.ah, self.D, self.depth, self.sigma, self.seed, self.cb, self.n,
                            _ptr(self.state))
        self.accum = np.zeros((self.H, self.W, 4))
        self.step = 0
        self.J = self.locals = self.accepts = self.splats = 0
        self.p_sum_large = 0.0

    @property
    def x(self):
        return self.state[:, :self.D]

    def advance(self, n_steps, trace=False, margins=False, n_threads=0):
        out = np.zeros(4, np.uint64)
        ps = np.zeros(1)
        tr = None
        if trace:
            tr = dict(flags=np.zeros((self.n, n_steps), np.uint8), pix=np.zeros((self.n, n_steps), np.int32),
                      margin=np.zeros((self.n, n_steps)) if margins else None)
        rc = lib().orc_mala_advance(self.kind, self.sh, self.ah, self.D, self.depth, self.W, self.H, self.sigma,
                                    self.c_tilde,
                                    self.method, self.ell, self.burn_in, self.seed, self.cb, self.n, self.step,
                                    n_steps, _ptr(self.state), _ptr(self.accum), _ptr(out), _ptr(ps),
                                    _ptr(tr["flags"]) if tr else None, _ptr(tr["pix"]) if tr else None,
                                    _ptr(tr["margin"]) if tr and margins else None, int(n_threads))
        if rc != 0:
            raise ValueError("oracle: invalid dimension")
        self.step += n_steps
        self.J += int(out[0])
        self.locals += int(out[1])
        self.accepts += int(out[2])
        self.splats += int(out[3])
        self.p_sum_large += float(ps[0])
        return tr

    def image(self):
        if self.method == 0:
            return self.accum[:, :, :3] / max(self.J, 1)
        return (self.p_sum_large / max(self.J, 1)) * self.accum[:, :, :3] / max(self.splats, 1)


def killing_rate_general(p, lstar_p, kappa_mustar_p):
    """((L* + kappa mu*) p) / p (Section 6.1), +inf at p = 0."""
    return lib().orc_killing_rate_general(float(p), float(lstar_p), float(kappa_mustar_p))


def lstar_p_1d(target, x, sigma, n_quad=4096):
    """(L* p)(x) of the unadjusted wrapped-Gaussian random walk on a 1-D analytic target."""
    x = np.ascontiguousarray(x, np.float64)
    out = np.zeros(len(x))
    lib().orc_lstar_p_1d(target.h, len(x), _ptr(x), float(sigma), int(n_quad), _ptr(out))
    return out


class GeneralChains:
    """General Restore (Section 6.1) on a 1-D analytic target: local dynamics =
    the unadjusted Gaussian random walk (not pi-invariant), mu uniform,
    k = (L* p + c~) / p; simplified=True drops L* p (a wrong rate here)."""

    def __init__(self, target, width, sigma, c_tilde, seed=0, chain_begin=0, n_chains=1, n_quad=4096,
                 simplified=False):
        self.target, self.W, self.sigma, self.c_tilde = target, int(width), float(sigma), float(c_tilde)
        self.seed, self.cb, self.n, self.nq, self.simp = int(seed), int(chain_begin), int(n_chains), int(n_quad), \
            int(bool(simplified))
        self.state = np.zeros((self.n, 3))
        lib().orc_general_init(target.h, self.sigma, self.c_tilde, self.nq, self.simp, self.seed, self.cb, self.n,
                               _ptr(self.state))
        self.accum = np.zeros((self.W, 4))
        self.step = 0
        self.J = 0

    def advance(self, n_steps, n_threads=0):
        self.J += int(lib().orc_general_advance(self.target.h, self.W, self.sigma, self.c_tilde, self.nq, self.simp,
                                                self.seed, self.cb, self.n, self.step, n_steps, _ptr(self.state),
                                                _ptr(self.accum), int(n_threads)))
        self.step += n_steps

    def image(self):
        return self.accum[:, :3] / max(self.J, 1)


def eval_states(target, x, c_tilde=1.0, depth=None, hit_ids=False):
    kind, sh, ah = _target(target)
    x = np.ascontiguousarray(x, dtype=np.float64)
    n, D = x.shape
    dep = int(depth) if depth is not None else (D - 2) // 2
    F = np.zeros((n, 3))
    p = np.zeros(n)
    u = np.zeros(n)
    k = np.zeros(n)
    ids = np.zeros((n, dep + 1), np.int32) if hit_ids else None
    lib().orc_eval_states(kind, sh, ah, D, dep, float(c_tilde), n, _ptr(x), _ptr(F), _ptr(p), _ptr(u), _ptr(k),
                          _ptr(ids))
    return (F, p, u, k, ids) if hit_ids else (F, p, u, k)


def render_pt(target, D, width, height, n_samples, seed=0, sample_begin=0, depth=None, n_threads=0):
    """Plain Monte Carlo estimate of every pixel; returns (image HxWx3, accum)."""
    kind, sh, ah = _target(target)
    dep = int(depth) if depth is not None else (D - 2) // 2
    accum = np.zeros((height, width, 4))
    lib().orc_render_pt(kind, sh, ah, int(D), dep, int(width), int(height), int(seed), int(sample_begin),
                        int(n_samples), _ptr(accum), int(n_threads))
    return accum[:, :, :3] / max(n_samples, 1), accum


def threads_default():
    return lib().orc_threads_default()
