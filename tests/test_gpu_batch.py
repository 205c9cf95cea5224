"""Batched form: B uneven frames in one CUDA graph with the OSOP control on the
device. Each frame of a batch must reproduce, bit for bit, the single-frame
path on that frame (same seed order with frame_id = base + f, same rounds,
modes, supports and labels): the two share the per-seed arithmetic and the
window sums are order-independent fixed point. The single-frame path is
itself parity-tested against the FP64 oracle; the batch is also checked
against the oracle directly on small frames."""
import numpy as np
import pytest

import oracle
import synth
from parity_util import matched_agreement, mode_errors, same_order_errors

pytestmark = pytest.mark.gpu

MODE_TOL = 1e-5


def _frames_mixed(d=16):
    frames = synth.batch_c4(seed=5, B=6, d=d, n_lo=500, n_hi=20000)
    out = [(f.emb, f.mask) for f in frames]
    rng = np.random.default_rng(9)
    one = rng.standard_normal((1, d)).astype(np.float32)
    bg = rng.standard_normal((300, d)).astype(np.float32)
    out.insert(2, (one, None))                                    # a single pixel
    out.insert(4, (bg, np.zeros(300, dtype=np.uint8)))            # all background
    out.append((np.zeros((0, d), dtype=np.float32), None))        # no pixels at all
    return out


def _to_dev(frames):
    import torch
    embs = [torch.from_numpy(np.ascontiguousarray(e)).cuda() for e, _ in frames]
    masks = [None if m is None else torch.from_numpy(np.ascontiguousarray(m)).cuda() for _, m in frames]
    return embs, masks


def _single(ms, emb, mask, frame_id, **cfg):
    import torch
    if emb.shape[0] == 0:
        return np.zeros(0, np.int32), np.zeros((0, emb.shape[1]), np.float32), None
    res = ms.cluster(emb, mask, frame_id=frame_id, **cfg)
    torch.cuda.synchronize()
    return res.labels.cpu().numpy(), res.modes.cpu().numpy(), res.stats


def _batch(ms, embs, masks, **cfg):
    c = ms.ms_config_default(dim=int(embs[0].shape[1]), **cfg)
    b = ms.ms_batch_create(c, embs, masks if any(m is not None for m in masks) else None)
    ms.ms_batch_run(b)
    return b


def _compare_to_single(ms, frames, **cfg):
    embs, masks = _to_dev(frames)
    b = _batch(ms, embs, masks, **cfg)
    try:
        for f in range(len(frames)):
            lab_b = b.labels[f].cpu().numpy()
            modes_b = ms.ms_batch_modes(b, f)
            st_b = ms.ms_batch_stats(b, f)
            lab_s, modes_s, st_s = _single(ms, embs[f], masks[f], f, **cfg)
            assert np.array_equal(modes_b, modes_s), f
            assert np.array_equal(lab_b, lab_s), f
            if st_s is not None:
                for k in ("rounds", "n_modes", "seeds", "seed_iters", "candidates", "dropped", "n_fg",
                          "iters_total", "uncovered"):
                    assert st_b[k] == st_s[k], (f, k, st_b[k], st_s[k])
            else:
                assert st_b["n_fg"] == 0 and st_b["n_modes"] == 0
        tot = ms.ms_batch_stats(b, -1)
        assert tot["n_fg"] == sum(ms.ms_batch_stats(b, f)["n_fg"] for f in range(len(frames)))
    finally:
        b.close()


def test_batch_equals_single_frames_fp32(ms_lib):
    _compare_to_single(ms_lib, _frames_mixed())


def test_batch_equals_single_frames_bf16(ms_lib):
    _compare_to_single(ms_lib, _frames_mixed(), precision=ms_lib.MS_BF16)


@pytest.mark.parametrize("bf16", [False, True])
def test_batch_equals_single_frames_d32(ms_lib, bf16):
    frames = [(f.emb, f.mask) for f in synth.batch_c4(seed=6, B=3, d=32, n_lo=800, n_hi=6000)]
    _compare_to_single(ms_lib, frames, precision=ms_lib.MS_BF16 if bf16 else ms_lib.MS_FP32)


def test_batch_all_seeds_algorithm1(ms_lib):
    frames = [(synth.frame_c1_separable(seed=s).emb, None) for s in (1, 2)]
    _compare_to_single(ms_lib, frames, all_seeds=1)


@pytest.mark.parametrize("split,bf16", [(0, False), (1, False), (1, True)])
def test_batch_matches_oracle(ms_lib, split, bf16):
    # batch_split = 1 shares work items across frames by load, so window sums
    # are cut differently from a single-frame run: held to the oracle bar only
    fs = synth.batch_c4(seed=7, B=3, n_lo=600, n_hi=4000)
    embs, masks = _to_dev([(f.emb, f.mask) for f in fs])
    b = _batch(ms_lib, embs, masks, batch_split=split,
               precision=ms_lib.MS_BF16 if bf16 else ms_lib.MS_FP32)
    try:
        for i, f in enumerate(fs):
            ref = oracle.run(f.emb, f.mask, frame_id=i)
            labels = b.labels[i].cpu().numpy()
            modes = ms_lib.ms_batch_modes(b, i)
            st = ms_lib.ms_batch_stats(b, i)
            assert modes.shape[0] > 0
            assert mode_errors(modes, ref.modes).max() <= MODE_TOL
            assert matched_agreement(ref.labels, labels) >= 0.999
            assert ((labels == -1) == (ref.labels == -1)).all()
            if modes.shape[0] == ref.modes.shape[0] and same_order_errors(modes, ref.modes).max() <= MODE_TOL:
                safe = ref.label_margin > 1e-5
                assert np.array_equal(labels[safe], ref.labels[safe])
                assert st["seeds"] == ref.stats["seeds"] and st["rounds"] == ref.stats["rounds"]
    finally:
        b.close()


def test_batch_rerun_and_new_inputs(ms_lib):
    import torch
    fs = synth.batch_c4(seed=8, B=4, n_lo=1000, n_hi=8000)
    embs, masks = _to_dev([(f.emb, f.mask) for f in fs])
    b = _batch(ms_lib, embs, masks)
    try:
        first = [t.clone() for t in b.labels]
        ms_lib.ms_batch_run(b)
        for a, c in zip(first, b.labels):
            assert torch.equal(a, c)
        # new embeddings in the same buffers: the graph reads them at launch
        g = torch.Generator().manual_seed(3)
        for t in embs:
            t.copy_(torch.randn(t.shape, generator=g))
        ms_lib.ms_batch_run(b)
        for f in range(len(fs)):
            lab_s, modes_s, _ = _single(ms_lib, embs[f], masks[f], f)
            assert np.array_equal(ms_lib.ms_batch_modes(b, f), modes_s)
            assert np.array_equal(b.labels[f].cpu().numpy(), lab_s)
    finally:
        b.close()


def test_batch_rejects_bad_frames(ms_lib):
    import torch
    c = ms_lib.ms_config_default(dim=16)
    e = torch.zeros((10, 16), device="cuda")
    e[3, 0] = 1.0  # nine foreground vectors of zero norm
    b = ms_lib.ms_batch_create(c, [e])
    with pytest.raises(ms_lib.MsError) as err:
        ms_lib.ms_batch_run(b)
    assert err.value.status == ms_lib.MS_ERR_INVALID_ARG
    b.close()
    bad = ms_lib.ms_config_default(dim=33, precision=ms_lib.MS_BF16)
    with pytest.raises(ms_lib.MsError):
        ms_lib.ms_batch_create(bad, [torch.zeros((4, 33), device="cuda")])


def test_batch_host_buffers_and_profile(ms_lib):
    import torch
    fs = synth.batch_c4(seed=10, B=3, n_lo=1000, n_hi=5000)
    embs, masks = _to_dev([(f.emb, f.mask) for f in fs])
    b = _batch(ms_lib, embs, masks, precision=ms_lib.MS_BF16)
    try:
        ref = [t.cpu().clone() for t in b.labels]
        st0 = ms_lib.ms_batch_stats(b, -1)
        assert st0["shift_launches"] == 0 and st0["launches"] > 0
        ms_lib.ms_batch_profile(b, True)
        h_e = [torch.from_numpy(f.emb).pin_memory() for f in fs]
        h_m = [torch.from_numpy(f.mask).pin_memory() for f in fs]
        h_l = [torch.full((f.emb.shape[0],), 7, dtype=torch.int32).pin_memory() for f in fs]
        for t in embs:
            t.zero_()  # the host call must copy the inputs in again
        ms_lib.ms_batch_run_host(b, h_e, h_m, h_l)
        for a, c in zip(ref, h_l):
            assert torch.equal(a, c)
        st = ms_lib.ms_batch_stats(b, -1)
        assert st["shift_launches"] > 0 and st["shift_ms"] > 0.0
        assert st["seed_iters"] == st0["seed_iters"] and st["n_modes"] == st0["n_modes"]
        assert st["launches"] > st0["launches"]  # two timer kernels per pass
    finally:
        b.close()


def test_batch_phase_timers(ms_lib):
    """Profiling level 2 adds phase timers between the graph's phases: the
    labels and counters do not change, every phase sum is positive, and the
    phases account for the run's time (within the launch gaps around them)."""
    import time

    import torch
    fs = synth.batch_c4(seed=12, B=3, n_lo=1000, n_hi=5000)
    embs, masks = _to_dev([(f.emb, f.mask) for f in fs])
    b = _batch(ms_lib, embs, masks, precision=ms_lib.MS_BF16)
    try:
        ref = [t.cpu().clone() for t in b.labels]
        st0 = ms_lib.ms_batch_stats(b, -1)
        assert all(v == 0.0 for v in ms_lib.ms_batch_phase_ms(b).values())
        ms_lib.ms_batch_profile(b, 2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ms_lib.ms_batch_run(b)
        wall_ms = 1e3 * (time.perf_counter() - t0)
        for a, c in zip(ref, b.labels):
            assert torch.equal(a, c.cpu())
        st = ms_lib.ms_batch_stats(b, -1)
        assert st["seed_iters"] == st0["seed_iters"] and st["n_modes"] == st0["n_modes"]
        ph = ms_lib.ms_batch_phase_ms(b)
        assert set(ph) == set(ms_lib.MS_BATCH_PHASES)
        assert all(v > 0.0 for v in ph.values()), ph
        assert 0.5 * wall_ms <= sum(ph.values()) <= wall_ms, (ph, wall_ms)
        assert ph["shift"] >= 0.9 * st["shift_ms"]  # the phase spans the shift timers' own span
        with pytest.raises(ms_lib.MsError):
            ms_lib.ms_batch_profile(b, 3)
    finally:
        b.close()


def test_batch_eager_launches_equal_graph(ms_lib):
    import torch
    fs = synth.batch_c4(seed=11, B=3, n_lo=800, n_hi=6000)
    embs, masks = _to_dev([(f.emb, f.mask) for f in fs])
    b = _batch(ms_lib, embs, masks, precision=ms_lib.MS_BF16)
    try:
        ref = [t.clone() for t in b.labels]
        passes = ms_lib.ms_batch_stats(b, -1)["reserved0"]
        st_ref = [ms_lib.ms_batch_stats(b, f) for f in range(3)]
        for t in b.labels:
            t.fill_(7)
        ms_lib.ms_batch_run_eager(b, passes + 2)
        for a, c in zip(ref, b.labels):
            assert torch.equal(a, c)
        for f in range(3):
            assert ms_lib.ms_batch_stats(b, f)["seed_iters"] == st_ref[f]["seed_iters"]
        with pytest.raises(ms_lib.MsError):
            ms_lib.ms_batch_run_eager(b, 1)  # too few passes to finish
    finally:
        b.close()


def test_batch_autotune_picks_a_candidate_and_keeps_results_valid(ms_lib):
    fs = synth.batch_c4(seed=12, B=4, n_lo=1000, n_hi=8000)
    embs, masks = _to_dev([(f.emb, f.mask) for f in fs])
    b = _batch(ms_lib, embs, masks, precision=ms_lib.MS_BF16)
    try:
        res = ms_lib.ms_batch_autotune(b, reps=2)
        splits = [(0, 2), (1, 1), (1, 2), (1, 4), (1, 8)]
        assert [(r["batch_split"], r["target_mult"], r["tc_shape"]) for r in res[:5]] == [s + (0,) for s in splits]
        # phase 2: the other tile shapes on phase 1's fastest split
        best = min(res[:5], key=lambda r: r["ms"])
        assert [(r["batch_split"], r["target_mult"], r["tc_shape"]) for r in res[5:]] == \
            [(best["batch_split"], best["target_mult"], sh) for sh in (1, 2, 3, 4, 5, 6, 7)]
        assert all(r["ms"] > 0 for r in res)
        # the batch now holds the fastest candidate's outputs: still within the oracle bar
        for i, f in enumerate(fs[:2]):
            ref = oracle.run(f.emb, f.mask, frame_id=i)
            modes = ms_lib.ms_batch_modes(b, i)
            assert mode_errors(modes, ref.modes).max() <= MODE_TOL
            assert matched_agreement(ref.labels, b.labels[i].cpu().numpy()) >= 0.999
        # configuring the canonical split again reproduces single-frame results
        # exactly, on every tile shape
        lab_s, modes_s, _ = _single(ms_lib, embs[0], masks[0], 0, precision=ms_lib.MS_BF16)
        for sh in range(8):
            ms_lib.ms_batch_configure(b, 0, 2, sh)
            ms_lib.ms_batch_run(b)
            assert np.array_equal(ms_lib.ms_batch_modes(b, 0), modes_s), sh
            assert np.array_equal(b.labels[0].cpu().numpy(), lab_s), sh
        with pytest.raises(ms_lib.MsError):
            ms_lib.ms_batch_configure(b, 0, 2, 8)
    finally:
        b.close()
