"""Comparison helpers for GPU-vs-oracle parity (pure numpy/scipy)."""
import numpy as np
from scipy.optimize import linear_sum_assignment


def matched_agreement(a, b):
    """Fraction of foreground pixels (a >= 0) with equal labels after the
    optimal one-to-one matching of a's clusters to b's (Hungarian method on
    the contingency table)."""
    a = np.asarray(a); b = np.asarray(b)
    fg = a >= 0
    a, b = a[fg], b[fg]
    if a.size == 0:
        return 1.0
    ua, ia = np.unique(a, return_inverse=True)
    ub, ib = np.unique(b, return_inverse=True)
    C = np.zeros((ua.size, ub.size), dtype=np.int64)
    np.add.at(C, (ia, ib), 1)
    r, c = linear_sum_assignment(-C)
    return C[r, c].sum() / a.size


def mode_errors(gpu_modes, ref_modes):
    """1 - cos between every GPU mode and its nearest oracle mode."""
    g = np.asarray(gpu_modes, dtype=np.float64)
    r = np.asarray(ref_modes, dtype=np.float64)
    g = g / np.linalg.norm(g, axis=1, keepdims=True)
    r = r / np.linalg.norm(r, axis=1, keepdims=True)
    return 1.0 - (g @ r.T).max(axis=1)


def same_order_errors(gpu_modes, ref_modes):
    g = np.asarray(gpu_modes, dtype=np.float64)
    r = np.asarray(ref_modes, dtype=np.float64)
    return 1.0 - (g * r).sum(1) / (np.linalg.norm(g, axis=1) * np.linalg.norm(r, axis=1))
