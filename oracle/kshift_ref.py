"""FP64 reference for mean-shift with other distances and kernel profiles -- TEST INFRASTRUCTURE.

Eq. 2 estimates the density with a kernel k and a distance d; Eq. 5-6 turn
its gradient into the mean-shift vector, whose update moves a seed x to the
k-weighted mean of the vectors:

    t_i = (d(x, p_i) / h)^2,   w_i = k(t_i),   x' = sum_i w_i p_i / sum_i w_i.

Distances: Euclidean d = ||x - p|| (Eq. 4) on the vectors as given, and the
cosine distance d = 1 - cos(x, p) (Eq. 9), for which the vectors are
normalised and x' is renormalised to the unit sphere (cosine distance ignores
scale; the flat cosine case is the library's main method). Profiles k(t):
flat [t <= 1] (Eq. 3), Epanechnikov max(0, 1 - t), Gaussian exp(-t / 2).
Every seed moves T times against all vectors (the dense update of
Sec. 3.2.1); a seed whose weights are all zero stays where it is.

Plain numpy float64, one step at a time, nothing fused.
"""
from __future__ import annotations

import numpy as np

COSINE, EUCLID = 0, 1
FLAT, EPANECHNIKOV, GAUSSIAN = 0, 1, 2


def profile(t: np.ndarray, kind: int) -> np.ndarray:
    if kind == FLAT:
        return (t <= 1.0).astype(np.float64)
    if kind == EPANECHNIKOV:
        return np.maximum(0.0, 1.0 - t)
    if kind == GAUSSIAN:
        return np.exp(-t / 2.0)
    raise ValueError(kind)


def sq_scaled_distance(X: np.ndarray, P: np.ndarray, distance: int, h: float) -> np.ndarray:
    """t[m, i] = (d(x_m, p_i) / h)^2."""
    if distance == EUCLID:
        D2 = ((X[:, None, :] - P[None, :, :]) ** 2).sum(axis=2)
        return D2 / (h * h)
    if distance == COSINE:
        Xn = X / np.linalg.norm(X, axis=1, keepdims=True)
        Pn = P / np.linalg.norm(P, axis=1, keepdims=True)
        return ((1.0 - Xn @ Pn.T) / h) ** 2
    raise ValueError(distance)


def step(X: np.ndarray, P: np.ndarray, distance: int, kind: int, h: float):
    """One update of every seed; returns (X', weight sums, nonzero-weight counts)."""
    X = np.asarray(X, dtype=np.float64)
    P = np.asarray(P, dtype=np.float64)
    Pw = P / np.linalg.norm(P, axis=1, keepdims=True) if distance == COSINE else P
    W = profile(sq_scaled_distance(X, P, distance, h), kind)
    s = W.sum(axis=1)
    Y = W @ Pw
    Xn = X.copy()
    ok = s > 0
    if distance == COSINE:
        Xn[ok] = Y[ok] / np.linalg.norm(Y[ok], axis=1, keepdims=True)
    else:
        Xn[ok] = Y[ok] / s[ok, None]
    return Xn, s, (W > 0).sum(axis=1)


def run(P, X0, distance: int, kind: int, h: float, T: int):
    """x_T for every seed, and the smallest |t - 1| met by a flat-profile
    decision on the way (how close a pair came to the window's edge)."""
    X = np.asarray(X0, dtype=np.float64)
    if distance == COSINE:
        X = X / np.linalg.norm(X, axis=1, keepdims=True)
    margin = np.inf
    for _ in range(T):
        if kind == FLAT:
            margin = min(margin, float(np.abs(sq_scaled_distance(X, np.asarray(P, np.float64), distance, h)
                                              - 1.0).min()))
        X, _, _ = step(X, P, distance, kind, h)
    return X, margin


def density(X, P, distance: int, kind: int, h: float) -> np.ndarray:
    """sum_i k(t_i) per seed: the unnormalised density of Eq. 2."""
    return profile(sq_scaled_distance(np.asarray(X, np.float64), np.asarray(P, np.float64), distance, h),
                   kind).sum(axis=1)
