"""Python binding of the C ABI in include/jr.h (argument marshalling only).

Every step of the method runs in the CUDA library ``_lib/libjr_gb300.so``;
this module converts numpy arrays and torch tensors to pointers and status
codes to exceptions.  There is no fallback: if the library is missing the
import of :func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libjr_gb300.so")

JR_OK, JR_ERR_INVALID_ARG, JR_ERR_CUDA, JR_ERR_OOM, JR_ERR_WATCHDOG, JR_ERR_NUMERIC, JR_ERR_STATE = range(7)
JR_FLAG_RAO_BLACKWELL = 1
JR_FLAG_MH = 2
JR_FLAG_MALA = 4
JR_EXEC_AUTO, JR_EXEC_MEGAKERNEL, JR_EXEC_WAVEFRONT, JR_EXEC_WARP = 0, 1, 2, 3
JR_STATUS_NONFINITE, JR_STATUS_TRAVERSAL, JR_STATUS_STACK, JR_STATUS_FLOW_WAIT = 1, 2, 4, 8
JR_BATCH_WAVEFRONT = 0
MATERIAL_FLOATS = 12
MAX_DEPTH = 15
STATIC_MAX_CHAINS = 65536


class JRError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"jr status {status}: {msg}")
        self.status = status


class SceneDesc(ctypes.Structure):
    _fields_ = [("verts", ctypes.c_void_p), ("n_verts", ctypes.c_uint32), ("tris", ctypes.c_void_p),
                ("n_tris", ctypes.c_uint32), ("tri_material", ctypes.c_void_p), ("materials", ctypes.c_void_p),
                ("n_materials", ctypes.c_uint32), ("camera", ctypes.c_float * 12)]


class Params(ctypes.Structure):
    _fields_ = [("width", ctypes.c_uint32), ("height", ctypes.c_uint32), ("max_depth", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("n_chains", ctypes.c_uint64), ("chain_offset", ctypes.c_uint64),
                ("seed", ctypes.c_uint64), ("c_tilde", ctypes.c_float), ("sigma", ctypes.c_float),
                ("large_step", ctypes.c_float), ("burn_in", ctypes.c_uint32)]


class Stats(ctypes.Structure):
    _fields_ = [("steps_per_chain", ctypes.c_uint64), ("regenerations", ctypes.c_uint64),
                ("local_steps", ctypes.c_uint64), ("accepted", ctypes.c_uint64), ("status_word", ctypes.c_uint32),
                ("dim", ctypes.c_uint32), ("p_sum_large", ctypes.c_double)]

    def as_dict(self):
        return {k: (float(getattr(self, k)) if k == "p_sum_large" else int(getattr(self, k)))
                for k, _ in self._fields_}


class SceneInfo(ctypes.Structure):
    _fields_ = [("n_tris", ctypes.c_uint32), ("n_nodes", ctypes.c_uint32), ("bvh_depth", ctypes.c_uint32),
                ("n_materials", ctypes.c_uint32), ("device_bytes", ctypes.c_uint64)]


_lib = None
_lock = threading.Lock()

_P, _U32, _U64, _I, _F = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_float
_SIGS = {
    "jr_scene_create": [ctypes.POINTER(SceneDesc), _P, ctypes.POINTER(_P)],
    "jr_scene_get_info": [_P, ctypes.POINTER(SceneInfo)],
    "jr_scene_destroy": [_P],
    "jr_chains_create": [_P, ctypes.POINTER(Params), _P, ctypes.POINTER(_P)],
    "jr_chains_destroy": [_P],
    "jr_advance": [_P, _U32, _P],
    "jr_advance_traced": [_P, _U32, _P, _P, _P, _P],
    "jr_advance_counted": [_P, _U32, _P, _P],
    "jr_advance_timed": [_P, _U32, _P, _P, _P],
    "jr_set_block_size": [_P, _U32],
    "jr_set_execution": [_P, _U32],
    "jr_advance_static": [_P, _U32, _P],
    "jr_resolve": [_P, _P, _I, _P],
    "jr_get_accumulator": [_P, _P, _I, _P],
    "jr_get_stats": [_P, ctypes.POINTER(Stats), _P],
    "jr_get_state": [_P, _P, _P, _P],
    "jr_set_state": [_P, _P, _P, _P],
    "jr_set_counters": [_P, ctypes.POINTER(Stats), _P, _P],
    "jr_eval_states": [_P, ctypes.POINTER(Params), _P, _U64, _P, _P, _P, _P, _P, _P],
    "jr_render_pt": [_P, ctypes.POINTER(Params), _U64, _U64, _P, _P],
    "jr_philox": [_U64, _U32, _U32, _U64, _U64, _U64, _P, _P],
    "jr_fp32_peak": [_P, _P, _P],
    "jr_eval_grad": [_P, _P, _P, _U64, _P, _P, _P],
    "jr_chains_set_limits": [_P, _U32, _U32],
    "jr_debug_fail_alloc": [ctypes.c_int64],
    "jr_debug_flow_wait": [_P, ctypes.c_int],
    "jr_batch_create": [_P, _U32, _P, ctypes.POINTER(_P)],
    "jr_batch_destroy": [_P],
    "jr_batch_set_block": [_P, _U32],
    "jr_batch_advance": [_P, _U32, _P],
    "jr_batch_advance_graph": [_P, _U32, _P],
    "jr_batch_autotune": [_P, _U32, _P, _P],
    "jr_flow_param_count": [_U32],
    "jr_flow_create": [_U32, _P, _P, _P, ctypes.POINTER(_P)],
    "jr_flow_destroy": [_P],
    "jr_flow_set_params": [_P, _P, _P],
    "jr_flow_get_params": [_P, _P, _P],
    "jr_flow_get_status": [_P, _P, _P],
    "jr_flow_log_density": [_P, _P, _U64, _P, _P],
    "jr_flow_sample": [_P, _P, _U64, _P, _P],
    "jr_chains_set_flow": [_P, _P, ctypes.c_float, _U32, _P, _P],
    "jr_complete_tours": [_P, _U32, _P, _P],
    "jr_flow_copy_params": [_P, _P, _P],
    "jr_chains_snapshot": [_P, _P, _P, _P],
    "jr_chains_snapshot_append": [_P, _P, _P, _U64, _P, _P],
    "jr_flow_gradient": [_P, _P, _P, _U64, _U64, _U32, _P, _P, _P],
    "jr_flow_train": [_P, _P, _P, _U64, _U32, _U32, ctypes.c_float, _U64, _P, _P],
    "jr_flow_train_rows": [_P, _P, _P, _U64, _U64, _U32, _U32, ctypes.c_float, _U64, _P, _P],
    "jr_last_error": [],
    "jr_version": [],
}


class TuneReport(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("block", ctypes.c_uint32 * 8), ("ns_per_chain_step", ctypes.c_double * 8),
                ("best_block", ctypes.c_uint32)]


def lib():
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"CUDA library missing at {LIB_PATH}: run paper_2409_07148_gb300.build.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, args in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = ctypes.c_char_p if name in ("jr_last_error", "jr_version") else ctypes.c_int
            L.jr_scene_destroy.restype = None
            L.jr_chains_destroy.restype = None
            L.jr_batch_destroy.restype = None
            L.jr_flow_destroy.restype = None
            L.jr_flow_param_count.restype = ctypes.c_uint64
            _lib = L
    return _lib


def _check(rc):
    if rc != JR_OK:
        raise JRError(rc, lib().jr_last_error().decode())


def _stream(stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _hptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def make_params(width, height, depth, n_chains=1, seed=0, c_tilde=1.0, sigma=0.01, chain_offset=0, flags=0,
                large_step=0.0, burn_in=0):
    return Params(int(width), int(height), int(depth), int(flags), int(n_chains), int(chain_offset), int(seed),
                  float(c_tilde), float(sigma), float(large_step), int(burn_in))


class Scene:
    """A scene uploaded to the GPU (BVH built by the library)."""

    def __init__(self, sc, stream=None):
        self.sc = sc
        self._keep = [np.ascontiguousarray(sc.verts, np.float32), np.ascontiguousarray(sc.tris, np.uint32),
                      np.ascontiguousarray(sc.tri_mat, np.uint32), np.ascontiguousarray(sc.mats, np.float32)]
        v, t, tm, m = self._keep
        d = SceneDesc(_hptr(v), v.shape[0], _hptr(t), t.shape[0], _hptr(tm), _hptr(m), m.shape[0],
                      (ctypes.c_float * 12)(*[float(c) for c in sc.camera]))
        h = ctypes.c_void_p()
        _check(lib().jr_scene_create(ctypes.byref(d), _stream(stream), ctypes.byref(h)))
        self.h = h

    def info(self):
        i = SceneInfo()
        _check(lib().jr_scene_get_info(self.h, ctypes.byref(i)))
        return {k: int(getattr(i, k)) for k, _ in i._fields_}

    def close(self):
        if getattr(self, "h", None):
            lib().jr_scene_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Chains:
    """A set of Jump Restore chains on the GPU (state, framebuffer, counters)."""

    def __init__(self, scene: Scene, width, height, depth, n_chains, seed=0, c_tilde=1.0, sigma=0.01,
                 chain_offset=0, flags=0, large_step=0.3, burn_in=10_000, stream=None):
        """flags may include JR_FLAG_MH: the MH baseline with large-step
        probability `large_step` and `burn_in` (both ignored otherwise)."""
        self.scene = scene
        self.params = make_params(width, height, depth, n_chains, seed, c_tilde, sigma, chain_offset, flags,
                                  large_step, burn_in)
        self.W, self.H, self.depth, self.n = int(width), int(height), int(depth), int(n_chains)
        self.D = 2 + 2 * self.depth
        h = ctypes.c_void_p()
        _check(lib().jr_chains_create(scene.h, ctypes.byref(self.params), _stream(stream), ctypes.byref(h)))
        self.h = h

    def advance(self, n_steps, stream=None):
        _check(lib().jr_advance(self.h, int(n_steps), _stream(stream)))

    def advance_traced(self, n_steps, flags=None, dt=None, pix=None, stream=None):
        _check(lib().jr_advance_traced(self.h, int(n_steps), _dptr(flags), _dptr(dt), _dptr(pix), _stream(stream)))

    def advance_static(self, n_steps, stream=None):
        """jr_advance_static: the wavefront advance with no device allocation
        (fixed in-library scratch, at most STATIC_MAX_CHAINS chains)."""
        _check(lib().jr_advance_static(self.h, int(n_steps), _stream(stream)))

    def advance_timed(self, n_steps, stream=None):
        """Advance with device time per kernel class (step, path, reserved, flow)."""
        ms = (ctypes.c_double * 4)()
        nl = (ctypes.c_uint64 * 4)()
        _check(lib().jr_advance_timed(self.h, int(n_steps), ms, nl, _stream(stream)))
        names = ("step", "path", "reserved", "flow")
        return {k: {"ms": ms[i], "launches": int(nl[i])} for i, k in enumerate(names)}

    def advance_counted(self, n_steps, stream=None):
        """Advance and return {rays, nodes, tris} counted by the instrumented kernel."""
        w = (ctypes.c_uint64 * 3)()
        _check(lib().jr_advance_counted(self.h, int(n_steps), w, _stream(stream)))
        return {"rays": int(w[0]), "nodes": int(w[1]), "tris": int(w[2])}

    def set_limits(self, node_visit_budget=0, stack_entries=0):
        """Traversal watchdog limits of this set's launches (0 = default)."""
        _check(lib().jr_chains_set_limits(self.h, int(node_visit_budget), int(stack_entries)))

    def set_block_size(self, block):
        _check(lib().jr_set_block_size(self.h, int(block)))

    def set_execution(self, mode):
        """JR_EXEC_AUTO, _MEGAKERNEL, _WAVEFRONT or _WARP (or 'auto'/'mega'/'wave'/'warp')."""
        m = {"auto": 0, "mega": 1, "megakernel": 1, "wave": 2, "wavefront": 2, "warp": 3}.get(mode, mode)
        _check(lib().jr_set_execution(self.h, int(m)))

    def resolve(self, out=None, stream=None):
        """Into a device tensor (async) if given, else into a new host array."""
        if out is not None:
            _check(lib().jr_resolve(self.h, _dptr(out), 1, _stream(stream)))
            return out
        img = np.zeros((self.H, self.W, 3), np.float32)
        _check(lib().jr_resolve(self.h, _hptr(img), 0, _stream(stream)))
        return img

    def accumulator(self, out=None, stream=None):
        if out is not None:
            _check(lib().jr_get_accumulator(self.h, _dptr(out), 1, _stream(stream)))
            return out
        a = np.zeros((self.H, self.W, 4), np.float64)
        _check(lib().jr_get_accumulator(self.h, _hptr(a), 0, _stream(stream)))
        return a

    def stats(self, stream=None, check=True):
        s = Stats()
        rc = lib().jr_get_stats(self.h, ctypes.byref(s), _stream(stream))
        if check:
            _check(rc)
        return s.as_dict()

    def get_state(self, stream=None):
        x = np.zeros((self.D, self.n), np.float32)
        fpu = np.zeros((5, self.n), np.float32)
        _check(lib().jr_get_state(self.h, _hptr(x), _hptr(fpu), _stream(stream)))
        return x, fpu

    def set_state(self, x, fpu=None, stream=None):
        x = np.ascontiguousarray(x, np.float32)
        f = None if fpu is None else np.ascontiguousarray(fpu, np.float32)
        _check(lib().jr_set_state(self.h, _hptr(x), _hptr(f), _stream(stream)))

    def set_counters(self, stats: dict, accumulator=None, stream=None):
        s = Stats(*[(float(stats.get(k, 0.0)) if k == "p_sum_large" else int(stats[k])) for k, _ in Stats._fields_])
        a = None if accumulator is None else np.ascontiguousarray(accumulator, np.float64)
        _check(lib().jr_set_counters(self.h, ctypes.byref(s), _hptr(a), _stream(stream)))

    def close(self):
        if getattr(self, "h", None):
            lib().jr_chains_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Flow:
    """The learned regeneration flow (parameters in the layout of include/jr.h)."""

    def __init__(self, D, perm, params, stream=None):
        self.D = int(D)
        self._perm = np.ascontiguousarray(perm, np.int32)
        p = np.ascontiguousarray(params, np.float32)
        assert p.size == lib().jr_flow_param_count(self.D), "parameter count does not match the layout"
        h = ctypes.c_void_p()
        _check(lib().jr_flow_create(self.D, _hptr(self._perm), _hptr(p), _stream(stream), ctypes.byref(h)))
        self.h = h

    def set_params(self, params, stream=None):
        p = np.ascontiguousarray(params, np.float32)
        _check(lib().jr_flow_set_params(self.h, _hptr(p), _stream(stream)))

    def get_params(self, stream=None):
        p = np.zeros(int(lib().jr_flow_param_count(self.D)), np.float32)
        _check(lib().jr_flow_get_params(self.h, _hptr(p), _stream(stream)))
        return p

    def log_density(self, x, stream=None):
        """x: CUDA float32 [D, n] -> log q [n]."""
        import torch
        lq = torch.empty(x.shape[1], dtype=torch.float32, device=x.device)
        _check(lib().jr_flow_log_density(self.h, _dptr(x), int(x.shape[1]), _dptr(lq), _stream(stream)))
        return lq

    def sample(self, z, stream=None):
        """z: CUDA float32 [D, n], replaced in place by T^{-1}(z); returns log q [n]."""
        import torch
        lq = torch.empty(z.shape[1], dtype=torch.float32, device=z.device)
        _check(lib().jr_flow_sample(self.h, _dptr(z), int(z.shape[1]), _dptr(lq), _stream(stream)))
        return lq

    def copy_params_from(self, other, stream=None):
        _check(lib().jr_flow_copy_params(self.h, other.h, _stream(stream)))

    def gradient(self, x, w, off=0, batch=None, stream=None):
        """Loss and gradient of rows [off, off + batch) of x [D, n], w [n] (CUDA)."""
        n = x.shape[1]
        batch = n - off if batch is None else batch
        g = np.zeros(int(lib().jr_flow_param_count(self.D)), np.float32)
        loss = ctypes.c_float(0.0)
        _check(lib().jr_flow_gradient(self.h, _dptr(x), _dptr(w), int(n), int(off), int(batch), _hptr(g),
                                      ctypes.byref(loss), _stream(stream)))
        return float(loss.value), g

    def train(self, x, w, iters, batch, lr=1e-3, seed=0, stream=None):
        """iters Adam steps on x [D, n], w [n] (CUDA); returns the per-step losses."""
        losses = np.zeros(max(int(iters), 1), np.float32)
        _check(lib().jr_flow_train(self.h, _dptr(x), _dptr(w), int(x.shape[1]), int(iters), int(batch), float(lr),
                                   int(seed), _hptr(losses), _stream(stream)))
        return losses[:int(iters)]

    def status(self, stream=None):
        v = ctypes.c_uint32(0)
        _check(lib().jr_flow_get_status(self.h, ctypes.byref(v), _stream(stream)))
        return int(v.value)

    def train_replay(self, buf, iters, batch, lr=1e-3, seed=0, stream=None):
        """iters Adam steps on the valid rows of a ReplayBuffer; returns the
        per-step losses (empty when the buffer holds fewer than `batch` rows)."""
        n = buf.rows()
        batch = min(int(batch), n // 64 * 64)
        if batch < 64:
            return np.zeros(0, np.float32)
        losses = np.zeros(max(int(iters), 1), np.float32)
        _check(lib().jr_flow_train_rows(self.h, _dptr(buf.x), _dptr(buf.w), buf.capacity, n, int(iters), batch,
                                        float(lr), int(seed), _hptr(losses), _stream(stream)))
        return losses[:int(iters)]

    def close(self):
        if getattr(self, "h", None):
            lib().jr_flow_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_flow(chains, flow, beta, max_drain_steps=1 << 20, stream=None):
    """Complete the current tours, attach `flow` (or None) with mixture weight
    beta, restart every chain.  Returns the tours left open by the drain."""
    rem = ctypes.c_uint64(0)
    _check(lib().jr_chains_set_flow(chains.h, None if flow is None else flow.h, float(beta), int(max_drain_steps),
                                    ctypes.byref(rem), _stream(stream)))
    chains._flow = flow   # the device keeps using the flow's weights: hold it as long as the chains
    return int(rem.value)


def snapshot(chains, stream=None):
    """Training rows from the chains' states: (x [D, n], w [n]) CUDA tensors."""
    import torch
    x = torch.empty((chains.D, chains.n), dtype=torch.float32, device="cuda")
    w = torch.empty(chains.n, dtype=torch.float32, device="cuda")
    _check(lib().jr_chains_snapshot(chains.h, _dptr(x), _dptr(w), _stream(stream)))
    return x, w


class ReplayBuffer:
    """Device ring of training rows (states with p > 0 and their weights)."""

    def __init__(self, D, capacity):
        import torch
        self.D, self.capacity = int(D), int(capacity)
        self.x = torch.empty((self.D, self.capacity), dtype=torch.float32, device="cuda")
        self.w = torch.empty(self.capacity, dtype=torch.float32, device="cuda")
        self.total = torch.zeros(1, dtype=torch.int64, device="cuda")

    def append(self, chains, stream=None):
        _check(lib().jr_chains_snapshot_append(chains.h, _dptr(self.x), _dptr(self.w), self.capacity,
                                               _dptr(self.total), _stream(stream)))

    def rows(self):
        """Number of valid rows (synchronises)."""
        return min(int(self.total.item()), self.capacity)


def complete_tours(chains, max_steps=1 << 20, stream=None):
    """Finish every chain's current tour, then start new tours.  Returns the
    tours still open after max_steps (0: the image is the completed-tour
    estimator)."""
    rem = ctypes.c_uint64(0)
    _check(lib().jr_complete_tours(chains.h, int(max_steps), ctypes.byref(rem), _stream(stream)))
    return int(rem.value)


class Batch:
    """Many chain sets advanced by one persistent launch (optionally a CUDA graph)."""

    def __init__(self, sets, stream=None):
        self.sets = list(sets)
        arr = (ctypes.c_void_p * len(self.sets))(*[c.h.value for c in self.sets])
        h = ctypes.c_void_p()
        _check(lib().jr_batch_create(arr, len(self.sets), _stream(stream), ctypes.byref(h)))
        self.h = h

    def set_block(self, block):
        """Chains per megakernel work item (a multiple of 32 in [32, 256]), or
        JR_BATCH_WAVEFRONT (0): every set in shared wavefront launches over a
        merged copy of the sets' scenes."""
        _check(lib().jr_batch_set_block(self.h, int(block)))

    def advance(self, n_steps, stream=None):
        _check(lib().jr_batch_advance(self.h, int(n_steps), _stream(stream)))

    def advance_graph(self, n_steps, stream=None):
        _check(lib().jr_batch_advance_graph(self.h, int(n_steps), _stream(stream)))

    def autotune(self, probe_steps, stream=None):
        """Time probe_steps real steps for each megakernel item size and for the
        batched wavefront, keep the fastest; returns {"best_block", "ns_per_chain_step"}
        (block 0 is the batched wavefront)."""
        r = TuneReport()
        _check(lib().jr_batch_autotune(self.h, int(probe_steps), _stream(stream), ctypes.byref(r)))
        return {"best_block": int(r.best_block),
                "ns_per_chain_step": {int(r.block[k]): float(r.ns_per_chain_step[k]) for k in range(r.n)}}

    def close(self):
        if getattr(self, "h", None):
            lib().jr_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def eval_states(scene: Scene, x, depth, c_tilde=1.0, hit_ids=False, stream=None):
    """x: CUDA float32 tensor [D, n] (SoA).  Returns F [3, n], p, u, k [n] (and ids)."""
    import torch
    n = x.shape[1]
    dev = x.device
    F = torch.empty((3, n), dtype=torch.float32, device=dev)
    p = torch.empty(n, dtype=torch.float32, device=dev)
    u = torch.empty(n, dtype=torch.float32, device=dev)
    k = torch.empty(n, dtype=torch.float32, device=dev)
    ids = torch.empty((depth + 1, n), dtype=torch.int32, device=dev) if hit_ids else None
    prm = make_params(1, 1, depth, c_tilde=c_tilde)
    _check(lib().jr_eval_states(scene.h, ctypes.byref(prm), _dptr(x), int(n), _dptr(F), _dptr(p), _dptr(u),
                                _dptr(k), _dptr(ids), _stream(stream)))
    return (F, p, u, k, ids) if hit_ids else (F, p, u, k)


def eval_grad(scene: Scene, x, depth, stream=None):
    """F [3, n] and dF/dx [3, D, n] (device tensors) for states x (CUDA float32 [D, n])."""
    import torch
    n = x.shape[1]
    D = 2 + 2 * int(depth)
    F = torch.empty((3, n), dtype=torch.float32, device=x.device)
    dF = torch.empty((3, D, n), dtype=torch.float32, device=x.device)
    p = make_params(1, 1, depth)
    _check(lib().jr_eval_grad(scene.h, ctypes.byref(p), _dptr(x), int(n), _dptr(F), _dptr(dF), _stream(stream)))
    return F, dF


def render_pt(scene: Scene, width, height, depth, n_samples, seed=0, sample_begin=0, accum=None, stream=None):
    """Plain Monte Carlo path tracing into a CUDA float64 accum [H, W, 4]."""
    import torch
    if accum is None:
        accum = torch.zeros((height, width, 4), dtype=torch.float64, device="cuda")
    prm = make_params(width, height, depth, seed=seed)
    _check(lib().jr_render_pt(scene.h, ctypes.byref(prm), int(sample_begin), int(n_samples), _dptr(accum),
                              _stream(stream)))
    return accum


def philox(seed, tag, block, chain_begin, step, n, stream=None):
    import torch
    out = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    _check(lib().jr_philox(int(seed), int(tag), int(block), int(chain_begin), int(step), int(n), _dptr(out),
                           _stream(stream)))
    return out


def fp32_peak(stream=None):
    """Measured FP32 FMA throughput of the device: (TFLOP/s, ms of one launch)."""
    t = ctypes.c_double()
    ms = ctypes.c_double()
    _check(lib().jr_fp32_peak(ctypes.byref(t), ctypes.byref(ms), _stream(stream)))
    return t.value, ms.value


def version():
    return lib().jr_version().decode()
