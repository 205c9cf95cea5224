"""Video form (Sec. 3.2.4; Sec. 4.3 and Table 3): consecutive frames of one
drifting sequence clustered in order, the OSOP seed count N carried from each
frame into the next, frame t+1 bound on a second stream while frame t runs.

Each frame must equal the FP64 oracle run on that frame with n_initial set to
the carried N and frame_id = t: the same modes in keep order within
1 - cos <= 1e-5, identical labels wherever the oracle's top-two margin exceeds
1e-5 (and >= 99.9% of pixels), and the carried N must be the oracle's
n_carry of the previous frame exactly (an integer schedule). Each frame must
also equal the single-frame API (ms_create + ms_set_state + ms_run) bit for
bit, and a video split over two calls must equal one call.
"""
import numpy as np
import pytest

import oracle
import synth
from parity_util import same_order_errors

pytestmark = pytest.mark.gpu


def _frames(T=5, seed=3):
    return synth.video_sequence(seed=seed, T=T, n_fg=6000, H=96, W=96, n_cells=9, drift=0.05,
                                kappa_lo=80.0, kappa_hi=200.0)


def _dev(fs):
    import torch
    return ([torch.from_numpy(f.emb).cuda() for f in fs],
            [torch.from_numpy(f.mask).cuda() if f.mask is not None else None for f in fs])


@pytest.mark.parametrize("bf16", [False, True])
def test_video_frames_equal_oracle_with_carried_n(ms_lib, bf16):
    fs = _frames()
    embs, masks = _dev(fs)
    cfg = ms_lib.ms_config_default(dim=16, precision=ms_lib.MS_BF16 if bf16 else ms_lib.MS_FP32)
    with ms_lib.ms_video_create(cfg, max(f.emb.shape[0] for f in fs)) as v:
        labels, n_start, n_modes = ms_lib.ms_video_run(v, embs, masks)
        carry_after, frames = ms_lib.ms_video_state(v)
    assert frames == len(fs) and n_start[0] == cfg.n_initial
    carry = cfg.n_initial
    for t, f in enumerate(fs):
        ref = oracle.run(f.emb, f.mask, frame_id=t, n_initial=carry)
        assert n_start[t] == carry, (t, n_start[t], carry)
        got_lab = labels[t].cpu().numpy()
        assert n_modes[t] == ref.modes.shape[0]
        # the modes themselves, through the single-frame API (bit for bit)
        c1 = ms_lib.ms_config_default(dim=16, precision=cfg.precision, frame_id=t)
        ctx = ms_lib.ms_create(c1, embs[t], masks[t])
        try:
            ms_lib.ms_set_state(ctx, n_start[t])
            import torch
            lab1 = torch.empty(f.emb.shape[0], dtype=torch.int32, device="cuda")
            ms_lib.ms_run(ctx, lab1)
            modes1 = ms_lib.ms_inspect(ctx, ms_lib.MS_INSPECT_MODES)
            assert ms_lib.ms_get_state(ctx) == ref.stats["n_carry"]
        finally:
            ctx.close()
        assert np.array_equal(lab1.cpu().numpy(), got_lab), t
        assert same_order_errors(modes1, ref.modes).max() <= 1e-5
        safe = np.nan_to_num(ref.label_margin, nan=-1.0) > 1e-5
        fg = ref.labels >= 0
        assert np.all(got_lab[~fg] == -1)
        assert np.array_equal(got_lab[safe], ref.labels[safe]), t
        assert (got_lab[fg] == ref.labels[fg]).mean() >= 0.999
        carry = ref.stats["n_carry"]
    assert carry_after == carry
    # the carried N grows past N_initial once the scene's mode count is known
    assert max(n_start) > cfg.n_initial


def test_video_split_over_calls_equals_one_call(ms_lib):
    fs = _frames(T=4, seed=5)
    embs, masks = _dev(fs)
    cfg = ms_lib.ms_config_default(dim=16, precision=ms_lib.MS_BF16)
    n = max(f.emb.shape[0] for f in fs)
    with ms_lib.ms_video_create(cfg, n) as v:
        a, sa, ka = ms_lib.ms_video_run(v, embs, masks)
    with ms_lib.ms_video_create(cfg, n) as v:
        b1, sb1, kb1 = ms_lib.ms_video_run(v, embs[:1], masks[:1])
        b2, sb2, kb2 = ms_lib.ms_video_run(v, embs[1:], masks[1:])
    assert sa == sb1 + sb2 and ka == kb1 + kb2
    for x, y in zip(a, b1 + b2):
        assert np.array_equal(x.cpu().numpy(), y.cpu().numpy())


def test_video_rejects_oversized_frames_and_continues(ms_lib):
    import torch
    fs = _frames(T=2, seed=7)
    embs, masks = _dev(fs)
    cfg = ms_lib.ms_config_default(dim=16, precision=ms_lib.MS_FP32)
    with ms_lib.ms_video_create(cfg, 1000) as v:
        with pytest.raises(ms_lib.MsError) as e:
            ms_lib.ms_video_run(v, embs, masks)
        assert e.value.status == ms_lib.MS_ERR_INVALID_ARG
        assert ms_lib.ms_video_state(v) == (cfg.n_initial, 0)
    bad = fs[0].emb.copy()
    bad[np.flatnonzero(fs[0].mask)[10]] = 0.0  # a foreground vector of zero norm
    with ms_lib.ms_video_create(cfg, fs[0].emb.shape[0]) as v:
        with pytest.raises(ms_lib.MsError) as e:
            ms_lib.ms_video_run(v, [torch.from_numpy(bad).cuda()] + embs[1:], masks)
        assert e.value.status == ms_lib.MS_ERR_INVALID_ARG
        # the video is still usable
        labels, _, _ = ms_lib.ms_video_run(v, embs, masks)
        assert (labels[0].cpu().numpy() >= -1).all()


def test_video_restart_equals_independent_frames(ms_lib):
    import torch
    fs = _frames(T=3, seed=9)
    embs, masks = _dev(fs)
    cfg = ms_lib.ms_config_default(dim=16, precision=ms_lib.MS_BF16, video_restart=1)
    with ms_lib.ms_video_create(cfg, max(f.emb.shape[0] for f in fs)) as v:
        labels, n_start, _ = ms_lib.ms_video_run(v, embs, masks)
    assert n_start == [cfg.n_initial] * len(fs)
    for t in range(len(fs)):
        res = ms_lib.cluster(embs[t], masks[t], precision=ms_lib.MS_BF16, frame_id=t)
        assert torch.equal(res.labels, labels[t])
