"""ms_window_sums_static: window sums from an entry point that allocates nothing.

Callers that cannot allocate device memory (a pool or arena that owns the
device, no cudaMalloc while a stream is captured, a plugin handed only its
input and output buffers) use this entry point; its scratch is a fixed static
device array. It must agree with ms_tc_selftest, the existing entry point that
returns the same per-seed window sums and window sizes, on two calls in a row
(the second with other inputs and sizes, so stale scratch would show).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _inputs(seed, n):
    rng = np.random.default_rng(seed)
    centres = synth.uniform_sphere(rng, 5, 16)
    P = np.concatenate([synth.sample_vmf(rng, centres[i % 5], 80.0, 1) for i in range(n)]).astype(np.float32)
    P *= rng.uniform(0.5, 2.0, size=(n, 1)).astype(np.float32)  # not unit: normalised inside
    X = P[rng.choice(n, 128, replace=False)]
    X = (X / np.linalg.norm(X, axis=1, keepdims=True)).astype(np.float32)
    return np.ascontiguousarray(X), np.ascontiguousarray(P)


def test_static_window_sums_match_existing_entry_point_twice(ms_lib):
    import torch
    for seed, n in [(1, 640), (2, 300)]:
        X, P = _inputs(seed, n)
        Xd, Pd = torch.from_numpy(X).cuda(), torch.from_numpy(P).cuda()
        out = torch.full((128, 17), -7, dtype=torch.int64, device="cuda")
        ms_lib.ms_window_sums_static(Xd, Pd, out, 0.9)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        _, ref = ms_lib.ms_tc_selftest(Xd, Pd, 0.9)
        cnt = ref[:, 16]
        assert (cnt > 0).all()
        assert np.array_equal(got[:, 16], cnt)
        err = np.abs(got[:, :16] - ref[:, :16]).astype(np.float64) * 2.0 ** -36
        assert (err.max(axis=1) <= 1e-4 * np.maximum(1, cnt)).all(), err.max()


def test_static_window_sums_reject_sizes_beyond_the_scratch(ms_lib):
    import torch
    X = torch.zeros((1025, 16), dtype=torch.float32, device="cuda")
    P = torch.ones((16, 16), dtype=torch.float32, device="cuda")
    out = torch.zeros((1025, 17), dtype=torch.int64, device="cuda")
    with pytest.raises(ms_lib.MsError) as e:
        ms_lib.ms_window_sums_static(X, P, out)
    assert e.value.status == ms_lib.MS_ERR_INVALID_ARG
    P = torch.ones((16385, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(ms_lib.MsError) as e:
        ms_lib.ms_window_sums_static(X[:4], P, out[:4])
    assert e.value.status == ms_lib.MS_ERR_INVALID_ARG
