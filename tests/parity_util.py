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


def labels_equal_oracle(ref_labels, ref_margin, labels, ref_modes, modes, margin=1e-5):
    """Element-by-element parity of a label map with the oracle's: both sides
    keep the same modes in the same order (1 - cos <= 1e-5), labels agree on
    every pixel whose oracle top-two margin exceeds `margin` (and twice the
    modes' direction error), on >= 99.9% of foreground pixels, and background
    is -1 on both. Returns the largest mode error."""
    ref_labels = np.asarray(ref_labels); labels = np.asarray(labels)
    assert np.asarray(modes).shape == np.asarray(ref_modes).shape, (np.shape(modes), np.shape(ref_modes))
    err = same_order_errors(modes, ref_modes) if len(modes) else np.zeros(1)
    assert err.max() <= 1e-5, err.max()
    delta = float(np.sqrt(2.0 * max(err.max(), 0.0)))
    fg = ref_labels >= 0
    assert np.array_equal(labels[~fg], ref_labels[~fg])
    safe = fg & (np.nan_to_num(np.asarray(ref_margin), nan=-1.0) > max(margin, 2 * delta))
    assert np.array_equal(labels[safe], ref_labels[safe])
    assert (labels[fg] == ref_labels[fg]).mean() >= 0.999
    return float(err.max())
