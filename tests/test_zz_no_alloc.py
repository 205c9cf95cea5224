"""ms_window_sums_static: window sums from an entry point that allocates nothing.

Callers that cannot allocate device memory (a pool or arena that owns the
device, no cudaMalloc while a stream is captured, a plugin handed only its
input and output buffers) use this entry point; its scratch is a fixed static
device array. It must agree with ms_tc_selftest, the existing entry point that
returns the same per-seed window sums and window sizes, on two calls in a row
(the second with other inputs and sizes, so stale scratch would show), and
its window sizes and sum directions must equal the FP64 oracle's window
(Eq. 11) and update (Eq. 8) for every seed whose window has no pixel within
1e-5 of the bandwidth. A pixel of zero norm must show in the output (count
-1 on every row) without leaving the shared scratch in an error state.
"""
import numpy as np
import pytest

import oracle
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


def test_static_window_sums_match_the_oracle(ms_lib):
    import torch
    X, P = _inputs(3, 1000)
    out = torch.empty((128, 17), dtype=torch.int64, device="cuda")
    ms_lib.ms_window_sums_static(torch.from_numpy(X).cuda(), torch.from_numpy(P).cuda(), out, 0.9)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    Pn, pn, _ = oracle.normalize(P)
    checked = 0
    for r in range(128):
        xn, cnt, margin = oracle.shift_step(Pn, pn, X[r].astype(np.float64), 0.9)
        if margin <= 1e-5:
            continue
        checked += 1
        assert got[r, 16] == cnt, r
        y = got[r, :16].astype(np.float64)
        assert 1.0 - float(y @ xn) / np.linalg.norm(y) <= 1e-6, r
    assert checked >= 100


def test_static_window_sums_flag_a_zero_norm_pixel_then_recover(ms_lib):
    import torch
    X, P = _inputs(4, 400)
    Xd = torch.from_numpy(X).cuda()
    bad = P.copy()
    bad[123] = 0.0
    out = torch.zeros((128, 17), dtype=torch.int64, device="cuda")
    ms_lib.ms_window_sums_static(Xd, torch.from_numpy(bad).cuda(), out, 0.9)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.all(got[:, 16] == -1) and np.all(got[:, :16] == 0)
    Pd = torch.from_numpy(P).cuda()
    ms_lib.ms_window_sums_static(Xd, Pd, out, 0.9)
    torch.cuda.synchronize()
    _, ref = ms_lib.ms_tc_selftest(Xd, Pd, 0.9)
    assert np.array_equal(out.cpu().numpy()[:, 16], ref[:, 16])
