"""Other distances and kernel profiles on the GPU (ms_kernel_shift) against
the FP64 reference (oracle/kshift_ref.py): Euclidean (Eq. 4) and cosine
(Eq. 9) distance, flat (Eq. 3), Epanechnikov and Gaussian profiles, T dense
steps of Eq. 6. Seeds must agree within 1e-5 (FP32 weights and sums); with
the flat and Epanechnikov profiles the windows must agree exactly, which the
inputs guarantee: no pair comes within 1e-4 of the window's edge on the
reference trajectory (asserted)."""
import numpy as np
import pytest
import torch

import synth
from oracle import kshift_ref as K

pytestmark = pytest.mark.gpu


def _ball(rng, n, dim, radius):
    """n points uniform in a ball of the given radius around 0."""
    v = rng.standard_normal((n, dim))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v * radius * rng.uniform(0.0, 1.0, size=(n, 1)) ** (1.0 / dim)


def _data(distance, dim, seed, bounded):
    """Clusters of 500 vectors. Bounded (for the flat profile, whose windows
    jump at t = 1): each cluster fits well inside one window and lies far from
    every other, so no pair comes near the edge. Otherwise Gaussian (Euclidean)
    or vMF (cosine) clusters whose pairs spread across the whole profile."""
    rng = np.random.default_rng(seed)
    if distance == K.EUCLID:
        if bounded:
            C = 20.0 * np.eye(dim)[:6]
            P = np.concatenate([c + _ball(rng, 500, dim, 0.5) for c in C])
        else:
            C = 3.0 * rng.standard_normal((6, dim))
            P = np.concatenate([c + 0.5 * rng.standard_normal((500, dim)) for c in C])
        h = 2.5
    else:
        if bounded:
            means = np.eye(dim)[:6]  # 90 degrees apart
            P = np.concatenate([m + _ball(rng, 500, dim, 0.08) for m in means])
        else:
            means = synth.uniform_sphere(rng, 6, dim)
            P = np.concatenate([synth.sample_vmf(rng, m, 300.0, 500) for m in means])
        P *= rng.uniform(0.5, 2.0, size=(len(P), 1))
        h = 0.1
    X0 = P[rng.choice(len(P), 96, replace=False)]
    return P.astype(np.float32), X0.astype(np.float32), h


@pytest.mark.parametrize("dim", [16, 18])
@pytest.mark.parametrize("profile", [0, 1, 2])
@pytest.mark.parametrize("distance", [0, 1])
def test_kernel_shift_matches_fp64(ms_lib, distance, profile, dim):
    P, X0, h = _data(distance, dim, seed=10 * distance + dim, bounded=profile == K.FLAT)
    T = 5
    ref, margin = K.run(P.astype(np.float64), X0.astype(np.float64), distance, profile, h, T)
    XT, counts = ms_lib.ms_kernel_shift(torch.from_numpy(P).cuda(), torch.from_numpy(X0).cuda(), distance,
                                        profile, h, T)
    XT = XT.cpu().numpy().astype(np.float64)
    if profile == K.FLAT:
        assert margin > 1e-4, margin
    assert np.abs(XT - ref).max() <= 1e-5, np.abs(XT - ref).max()
    # the last step's nonzero-weight counts: from the reference's step T-1
    Xp, _ = K.run(P.astype(np.float64), X0.astype(np.float64), distance, profile, h, T - 1)
    _, _, n_ref = K.step(Xp, P.astype(np.float64), distance, profile, h)
    if profile != K.GAUSSIAN:
        tt = K.sq_scaled_distance(Xp, P.astype(np.float64), distance, h)
        if np.abs(tt - 1.0).min() > 1e-4:
            assert np.array_equal(counts.cpu().numpy(), n_ref)
    else:
        # exp(-t/2) is nonzero in FP64 for every pair; in FP32 it underflows to
        # 0 once t exceeds about 206 (2^-149), so only the pairs well below
        # that are sure to count
        tt = K.sq_scaled_distance(Xp, P.astype(np.float64), distance, h)
        got = counts.cpu().numpy()
        assert np.all(got <= len(P)) and np.all(got >= (tt < 150.0).sum(axis=1))


def test_kernel_shift_rejects_bad_input(ms_lib):
    P = torch.zeros((10, 4), device="cuda")
    X = torch.ones((2, 4), device="cuda")
    with pytest.raises(ms_lib.MsError) as e:
        ms_lib.ms_kernel_shift(P, X, ms_lib.MS_DIST_COSINE, ms_lib.MS_PROFILE_FLAT, 0.1, 1)
    assert e.value.status == ms_lib.MS_ERR_INVALID_ARG
    with pytest.raises(ms_lib.MsError):
        ms_lib.ms_kernel_shift(P + 1, X, ms_lib.MS_DIST_EUCLID, 7, 0.1, 1)
    XT, counts = ms_lib.ms_kernel_shift(P + 1, X, ms_lib.MS_DIST_EUCLID, ms_lib.MS_PROFILE_FLAT, 0.5, 0)
    assert torch.equal(XT, X) and int(counts.sum()) == 0
