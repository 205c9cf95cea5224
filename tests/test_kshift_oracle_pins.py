"""Pins for the FP64 reference of the distance/profile variants (Eq. 2-6 with
Eq. 3/4/9 and the Epanechnikov and Gaussian profiles), each against something
other than the reference itself: hand-worked steps, closed forms, the C
oracle's flat cosine window, and the density ascent that mean-shift guarantees
for these profiles."""
import math

import numpy as np
import pytest

import oracle
from oracle import kshift_ref as K


def test_euclid_flat_hand_worked_1d():
    # points 0, 0.5, 1, 3 on a line, h = 1.2: from x = 0.4 the window is
    # {0, 0.5, 1} (|3 - 0.4| = 2.6 > 1.2), mean 0.5; from 0.5 the same window
    P = np.array([[0.0], [0.5], [1.0], [3.0]])
    X, s, n = K.step(np.array([[0.4]]), P, K.EUCLID, K.FLAT, 1.2)
    assert X[0, 0] == pytest.approx(0.5, abs=1e-15) and s[0] == 3 and n[0] == 3
    XT, margin = K.run(P, np.array([[0.4]]), K.EUCLID, K.FLAT, 1.2, 5)
    assert XT[0, 0] == pytest.approx(0.5, abs=1e-15)
    # the decision nearest the window's edge: d = 0.6 in the first step, t = 1/4
    assert margin == pytest.approx(0.75, abs=1e-15)


def test_epanechnikov_hand_worked_1d():
    # points 0 and 1, h = 1, x = 0.25: t = 1/16 and 9/16, w = 15/16 and 7/16,
    # x' = (7/16) / (22/16) = 7/22
    X, s, n = K.step(np.array([[0.25]]), np.array([[0.0], [1.0]]), K.EUCLID, K.EPANECHNIKOV, 1.0)
    assert X[0, 0] == pytest.approx(7.0 / 22.0, abs=1e-15)
    assert s[0] == pytest.approx(22.0 / 16.0, abs=1e-15) and n[0] == 2


def test_gaussian_hand_worked_and_wide_bandwidth_limit():
    # points 0 and 2, h = 1, x = 0.5: w = exp(-1/8) and exp(-9/8),
    # x' = 2 exp(-9/8) / (exp(-1/8) + exp(-9/8)) = 2 / (1 + e)
    X, _, _ = K.step(np.array([[0.5]]), np.array([[0.0], [2.0]]), K.EUCLID, K.GAUSSIAN, 1.0)
    assert X[0, 0] == pytest.approx(2.0 / (1.0 + math.e), abs=1e-14)
    # h -> infinity: every weight -> 1, one step lands on the plain mean
    rng = np.random.default_rng(0)
    P = rng.standard_normal((50, 3))
    X, _, _ = K.step(rng.standard_normal((4, 3)), P, K.EUCLID, K.GAUSSIAN, 1e8)
    assert np.allclose(X, P.mean(axis=0), rtol=0, atol=1e-12)


def test_symmetric_configuration_is_a_fixed_point():
    # vectors symmetric about c: every profile keeps x = c
    P = np.array([[1.0, 0.0], [-1.0, 0.0], [0.0, 0.7], [0.0, -0.7]]) + np.array([3.0, -2.0])
    for kind in (K.FLAT, K.EPANECHNIKOV, K.GAUSSIAN):
        X, _, _ = K.step(np.array([[3.0, -2.0]]), P, K.EUCLID, kind, 1.5)
        assert np.allclose(X, [[3.0, -2.0]], rtol=0, atol=1e-15), kind


def test_flat_cosine_equals_the_c_oracle_window_mean():
    # the flat cosine variant is the main method's update: the C oracle's
    # or_shift_step (its own pins fix the window and the mean)
    rng = np.random.default_rng(1)
    P = rng.standard_normal((400, 16))
    Pn, pn, _ = oracle.normalize(P.astype(np.float32))
    X0 = Pn[rng.choice(400, 20, replace=False)] + 0.05 * rng.standard_normal((20, 16))
    h = 0.1
    X, s, n = K.step(X0, Pn, K.COSINE, K.FLAT, h)
    for m in range(20):
        xn, cnt, margin = oracle.shift_step(Pn, pn, X0[m], 1.0 - h)
        if margin < 1e-9:
            continue
        assert n[m] == cnt
        if cnt:
            assert np.allclose(X[m], xn, rtol=0, atol=1e-12)


# Shadow profiles: weights g = k are the derivative -k_s' of the profile
# k_s(t) below, and mean-shift with weights g never decreases sum_i k_s(t_i)
# (Cheng 1995; the convergence argument the paper cites): Gaussian is its own
# shadow, Epanechnikov weights rise the biweight density, flat weights the
# Epanechnikov density.
SHADOW = {0: lambda t: np.maximum(0.0, 1.0 - t), 1: lambda t: np.maximum(0.0, 1.0 - t) ** 2,
          2: lambda t: np.exp(-t / 2.0)}


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_euclidean_steps_ascend_the_shadow_density(kind):
    rng = np.random.default_rng(2)
    C = 3.0 * rng.standard_normal((4, 8))
    P = np.concatenate([c + 0.6 * rng.standard_normal((60, 8)) for c in C])
    X = P[rng.choice(len(P), 12, replace=False)] + 0.5 * rng.standard_normal((12, 8))
    h = 3.0

    def f(X):
        return SHADOW[kind](K.sq_scaled_distance(X, P, K.EUCLID, h)).sum(axis=1)
    f0 = f(X)
    for _ in range(6):
        X, _, _ = K.step(X, P, K.EUCLID, kind, h)
        f1 = f(X)
        assert np.all(f1 >= f0 - 1e-12)
        f0 = f1


def test_empty_window_keeps_the_seed():
    X, s, n = K.step(np.array([[10.0, 10.0]]), np.array([[0.0, 0.0], [1.0, 0.0]]), K.EUCLID, K.FLAT, 1.0)
    assert np.array_equal(X, [[10.0, 10.0]]) and s[0] == 0 and n[0] == 0


def test_flat_window_includes_its_boundary():
    # Eq. 3's flat kernel counts t <= 1: from x = 0 with h = 1 the vector at
    # distance exactly 1 is in the window (dyadic values, t = 1 exactly)
    X, s, n = K.step(np.array([[0.0]]), np.array([[-0.5], [1.0], [1.5]]), K.EUCLID, K.FLAT, 1.0)
    assert n[0] == 2 and X[0, 0] == 0.25


def test_cosine_epanechnikov_hand_worked_2d():
    # directions e1 and e2 given at lengths 2 and 3 (the cosine form
    # normalises them), x = e1, h = 2: 1 - cos = 0 and 1, t = 0 and 1/4,
    # w = 1 and 3/4, y = e1 + (3/4) e2, x' = (4, 3) / 5
    P = np.array([[2.0, 0.0], [0.0, 3.0]])
    X, s, n = K.step(np.array([[1.0, 0.0]]), P, K.COSINE, K.EPANECHNIKOV, 2.0)
    assert np.allclose(X, [[0.8, 0.6]], rtol=0, atol=1e-15) and s[0] == pytest.approx(1.75, abs=1e-15)


def test_run_takes_exactly_T_steps():
    # Epanechnikov on 0 and 1 from 0.25 (h = 1): one step gives 7/22 (above);
    # a second gives, with t = (7/22)^2 and (15/22)^2,
    # x'' = w1 / (w0 + w1), w0 = 1 - 49/484, w1 = 1 - 225/484
    P = np.array([[0.0], [1.0]])
    x1, _ = K.run(P, np.array([[0.25]]), K.EUCLID, K.EPANECHNIKOV, 1.0, 1)
    x2, _ = K.run(P, np.array([[0.25]]), K.EUCLID, K.EPANECHNIKOV, 1.0, 2)
    assert x1[0, 0] == pytest.approx(7.0 / 22.0, abs=1e-15)
    assert x2[0, 0] == pytest.approx((259.0 / 484.0) / (435.0 / 484.0 + 259.0 / 484.0), abs=1e-15)
    # T = 0 returns the seeds, normalised for the cosine distance
    x0, _ = K.run(np.array([[1.0, 0.0]]), np.array([[3.0, 4.0]]), K.COSINE, K.FLAT, 0.5, 0)
    assert np.allclose(x0, [[0.6, 0.8]], rtol=0, atol=1e-15)
