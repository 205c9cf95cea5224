"""GPU parity: the CUDA library against the FP64 oracle through the C ABI.

Tolerances:
  * modes: 1 - cos(gpu, oracle) <= 1e-5 (the GPU keeps seeds in FP32 and
    tests convergence in FP64; a direction error delta costs delta^2 / 2)
  * labels: >= 99.9% identical after optimal cluster matching; bit-identical
    integer maps when both sides kept the same modes in the same order, on
    every pixel whose oracle top-1/top-2 margin exceeds 1e-5
  * integer work (seed order, counts, coverage bookkeeping): exact
"""
import numpy as np
import pytest

import oracle
import synth
from parity_util import matched_agreement, mode_errors, same_order_errors

pytestmark = pytest.mark.gpu

MODE_TOL = 1e-5
LABEL_AGREE = 0.999
MARGIN = 1e-5


def _run_gpu(ms, emb, mask=None, **cfg):
    import torch
    e = torch.from_numpy(np.ascontiguousarray(emb)).cuda()
    m = None if mask is None else torch.from_numpy(np.ascontiguousarray(mask)).cuda()
    res = ms.cluster(e, m, **cfg)
    torch.cuda.synchronize()
    return res.labels.cpu().numpy(), res.modes.cpu().numpy(), res.stats


def _check_parity(labels, modes, stats, ref, exact_ok=True):
    assert modes.shape[0] > 0
    err = mode_errors(modes, ref.modes)
    assert err.max() <= MODE_TOL, err.max()
    assert matched_agreement(ref.labels, labels) >= LABEL_AGREE
    assert ((labels == -1) == (ref.labels == -1)).all()
    if exact_ok and modes.shape[0] == ref.modes.shape[0] and same_order_errors(modes, ref.modes).max() <= MODE_TOL:
        safe = ref.label_margin > MARGIN
        assert np.array_equal(labels[safe], ref.labels[safe])


def test_c1_separable_exact(ms_lib):
    f = synth.frame_c1_separable(seed=0)
    ref = oracle.run(f.emb)
    labels, modes, st = _run_gpu(ms_lib, f.emb)
    assert modes.shape[0] == ref.modes.shape[0] == 8
    assert same_order_errors(modes, ref.modes).max() <= MODE_TOL
    assert np.array_equal(labels, ref.labels)
    assert np.array_equal(st["seed_log"], ref.seed_log)
    assert np.array_equal(st["round_log"], ref.round_log)
    assert np.array_equal(st["support"], ref.support)
    assert st["seeds"] == ref.stats["seeds"] and st["rounds"] == ref.stats["rounds"]


@pytest.mark.parametrize("seed", [0, 1])
def test_c1_fragmented(ms_lib, seed):
    # 64x64, K = 8, kappa = 50: hundreds of modes; the literal config.
    f = synth.frame_c1(seed=seed)
    ref = oracle.run(f.emb)
    labels, modes, st = _run_gpu(ms_lib, f.emb)
    _check_parity(labels, modes, st, ref)
    assert abs(modes.shape[0] - ref.modes.shape[0]) <= max(2, ref.modes.shape[0] // 500)


def test_all_pixels_as_seeds_algorithm1(ms_lib):
    f = synth.frame_c1_separable(seed=3)
    ref = oracle.run(f.emb, all_seeds=1)
    labels, modes, st = _run_gpu(ms_lib, f.emb, all_seeds=1)
    assert st["rounds"] == 1 and st["seeds"] == 4096
    assert modes.shape[0] == ref.modes.shape[0]
    assert same_order_errors(modes, ref.modes).max() <= MODE_TOL
    assert np.array_equal(labels, ref.labels)


def test_masked_ragged_frame(ms_lib):
    # 1237 foreground pixels of 50x50: not a multiple of any tile
    f = synth.make_frame(21, 50, 50, 16, 1237, 5, 240.0, 0.3, 150.0, 200.0, 0.02)
    ref = oracle.run(f.emb, f.mask)
    labels, modes, st = _run_gpu(ms_lib, f.emb, f.mask)
    assert (labels[f.mask == 0] == -1).all()
    assert np.array_equal(st["seed_log"][: ref.round_log[0, 1]], ref.seed_log[: ref.round_log[0, 1]])
    _check_parity(labels, modes, st, ref)


def test_dim18_orthogonal_blobs_padded_path(ms_lib):
    # Sec. 4.2 design at d = 18 (padded to 32 inside the library)
    emb, truth = synth.orthogonal_blobs(seed=5, n=3000)
    ref = oracle.run(emb, dim=18)
    labels, modes, st = _run_gpu(ms_lib, emb)
    assert modes.shape == (10, 18)
    assert np.array_equal(labels, ref.labels)
    assert same_order_errors(modes, ref.modes).max() <= 1e-6


def test_dim32(ms_lib):
    f = synth.make_frame(8, 64, 64, 32, 3000, 6, 480.0, 0.2, 400.0, 600.0, 0.0)
    ref = oracle.run(f.emb, f.mask)
    labels, modes, st = _run_gpu(ms_lib, f.emb, f.mask)
    _check_parity(labels, modes, st, ref)


def test_normalised_pixels_and_compaction(ms_lib):
    import torch
    f = synth.make_frame(2, 40, 40, 16, 900, 3, 280.0, 0.2, 100.0, 100.0, 0.05)
    P, _, idx = oracle.normalize(f.emb, f.mask)
    ctx = ms_lib.ms_create(ms_lib.ms_config_default(), torch.from_numpy(f.emb).cuda(),
                           torch.from_numpy(f.mask).cuda())
    got = ms_lib.ms_inspect(ctx, ms_lib.MS_INSPECT_PIXELS)
    assert got.shape == P.shape
    assert np.abs(got - P).max() <= 2e-7
    ctx.close()


def test_step_api_and_state_errors(ms_lib):
    import torch
    f = synth.frame_c1_separable(seed=4)
    ref = oracle.run(f.emb)
    ctx = ms_lib.ms_create(ms_lib.ms_config_default(), torch.from_numpy(f.emb).cuda())
    with pytest.raises(ms_lib.MsError) as e:
        ms_lib.ms_iterate(ctx)
    assert e.value.status == ms_lib.MS_ERR_STATE
    m = ms_lib.ms_seed_batch(ctx)
    assert m == 128
    with pytest.raises(ms_lib.MsError) as e:
        ms_lib.ms_seed_batch(ctx)
    assert e.value.status == ms_lib.MS_ERR_STATE
    conv, iters = ms_lib.ms_iterate(ctx)
    assert 0.9 * m < conv <= m
    k, unc = ms_lib.ms_merge_modes(ctx)
    assert (k, unc) == (ref.round_log[0, 2], ref.round_log[0, 3])
    # the seed count a next frame would start from: the unclamped schedule,
    # bounded by the largest batch drawn so far (128)
    assert ms_lib.ms_get_state(ctx) == min(oracle.next_n(128, int(k), uncovered=10 ** 12), m)
    with pytest.raises(ms_lib.MsError) as e:
        ms_lib.ms_set_state(ctx, 64)  # only before the frame's first round
    assert e.value.status == ms_lib.MS_ERR_STATE
    while unc > 0:
        assert ms_lib.ms_seed_batch(ctx) > 0
        ms_lib.ms_iterate(ctx)
        k, unc = ms_lib.ms_merge_modes(ctx)
    assert ms_lib.ms_get_state(ctx) == ref.stats["n_carry"]
    labels = torch.empty(4096, dtype=torch.int32, device="cuda")
    modes = torch.empty((k, 16), dtype=torch.float32, device="cuda")
    assert ms_lib.ms_label(ctx, labels, modes) == k
    assert np.array_equal(labels.cpu().numpy(), ref.labels)
    small = torch.empty((max(k - 1, 0), 16), dtype=torch.float32, device="cuda")
    with pytest.raises(ms_lib.MsError) as e:
        ms_lib.ms_label(ctx, labels, small)
    assert e.value.status == ms_lib.MS_ERR_INVALID_ARG
    ctx.close()


def test_not_converged_status(ms_lib):
    import torch
    # one dense cluster: no seed can converge in a single iteration
    rng = np.random.default_rng(0)
    P = synth.sample_vmf(rng, np.eye(16)[0], 300.0, 500).astype(np.float32)
    ctx = ms_lib.ms_create(ms_lib.ms_config_default(), torch.from_numpy(P).cuda())
    ms_lib.ms_seed_batch(ctx, 64)
    with pytest.raises(ms_lib.MsError) as e:
        ms_lib.ms_iterate(ctx, 1)
    assert e.value.status == ms_lib.MS_ERR_NOT_CONVERGED
    k, unc = ms_lib.ms_merge_modes(ctx)
    assert k == 0 and unc == 500 - 64
    ctx.close()


def test_invalid_inputs_rejected(ms_lib):
    import torch
    emb = np.random.default_rng(1).standard_normal((100, 16)).astype(np.float32)
    emb[17] = 0.0
    with pytest.raises(ms_lib.MsError) as e:
        ms_lib.ms_create(ms_lib.ms_config_default(), torch.from_numpy(emb).cuda())
    assert e.value.status == ms_lib.MS_ERR_INVALID_ARG
    emb[17] = np.nan
    with pytest.raises(ms_lib.MsError):
        ms_lib.ms_create(ms_lib.ms_config_default(), torch.from_numpy(emb).cuda())
    # masked-out zero vectors are fine
    mask = np.ones(100, np.uint8); mask[17] = 0
    emb[17] = 0.0
    labels, modes, st = _run_gpu(ms_lib, emb, mask)
    assert labels[17] == -1


def test_empty_inputs(ms_lib):
    import torch
    emb = np.zeros((0, 16), np.float32)
    labels, modes, st = _run_gpu(ms_lib, np.ones((10, 16), np.float32), np.zeros(10, np.uint8))
    assert (labels == -1).all() and st["n_fg"] == 0 and modes.shape[0] == 0
    ctx = ms_lib.ms_create(ms_lib.ms_config_default(), torch.from_numpy(emb).cuda())
    out = torch.empty(0, dtype=torch.int32, device="cuda")
    assert ms_lib.ms_run(ctx, out) == 0
    ctx.close()


def test_single_pixel(ms_lib):
    emb = np.array([[0.3, -2.0] + [0.0] * 14], np.float32)
    labels, modes, st = _run_gpu(ms_lib, emb)
    assert labels.tolist() == [0] and modes.shape[0] == 1
    # normalised in FP32 at ingest and again by the shift: a few units in the last place
    assert np.allclose(modes[0], emb[0] / np.linalg.norm(emb[0]), rtol=0, atol=5e-7)


def test_deterministic_repeat(ms_lib):
    f = synth.frame_c1(seed=7)
    a = _run_gpu(ms_lib, f.emb)
    b = _run_gpu(ms_lib, f.emb)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
