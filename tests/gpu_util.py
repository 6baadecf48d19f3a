"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np


def rel_err(a, b, floor=1e-30):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), floor)


def torus_diff(a, b):
    """Distance on the unit torus (coordinates wrap at 1)."""
    d = np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64))
    return np.minimum(d, 1.0 - d)


def oracle_state_from_gpu(x_soa, fpu_soa):
    """GPU SoA state (x [D][n], fpu [5][n]) -> oracle rows [n][D+5] in float64."""
    return np.concatenate([x_soa.T.astype(np.float64), fpu_soa.T.astype(np.float64)], axis=1)
