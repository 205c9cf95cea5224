"""The BF16 tensor-core shift tile (tcgen05 GEMM1 -> mask -> tcgen05 GEMM2)
against a numpy reconstruction of the same split arithmetic, and the BF16
form of the whole method against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from parity_util import matched_agreement, mode_errors, same_order_errors

pytestmark = pytest.mark.gpu


def bf16(a):
    """Round float32 to bfloat16 (nearest even), returned as float32."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def unit(rng, n, d=16):
    v = rng.standard_normal((n, d))
    return (v / np.linalg.norm(v, axis=1, keepdims=True)).astype(np.float32)


@pytest.mark.parametrize("n_pix", [128, 200, 640])
def test_tc_tile_products_and_sums(ms_lib, n_pix):
    import torch
    rng = np.random.default_rng(n_pix)
    # pixels in a few tight clusters so windows are non-trivial
    centres = unit(rng, 4)
    P = np.concatenate([synth.sample_vmf(rng, centres[i % 4], 60.0, 1) for i in range(n_pix)]).astype(np.float32)
    X = P[rng.choice(n_pix, 128, replace=n_pix < 128)].copy()
    X[:7] = unit(rng, 7)  # a few seeds with tiny windows
    c = 0.9
    S, acc = ms_lib.ms_tc_selftest(torch.from_numpy(X).cuda(), torch.from_numpy(P).cuda(), c)
    # the library normalises pixels in FP32; rebuild exactly that input
    Pn = (P / np.sqrt((P.astype(np.float32) ** 2).sum(1, dtype=np.float32))[:, None]).astype(np.float32)
    Xh = bf16(X); Xl = bf16(X - Xh)
    Ph = bf16(Pn); Pm = bf16(Pn - Ph); Pl = bf16((Pn - Ph) - Pm)
    S_ref = (Xh.astype(np.float64) @ Ph.T.astype(np.float64) + Xh.astype(np.float64) @ Pm.T.astype(np.float64)
             + Xl.astype(np.float64) @ Ph.T.astype(np.float64))
    c_f = float(np.nextafter(np.float32(c), np.float32(2))) if float(np.float32(c)) < c else float(np.float32(c))
    got = S[:, :n_pix].astype(np.float64) + c_f
    # tensor-core FP32 accumulation error, measured: <= 6e-6 (the mask's recheck band is 2^-14)
    assert np.abs(got - S_ref).max() <= 1e-5, np.abs(got - S_ref).max()
    # padded pixels score exactly -c and never enter a window
    assert np.all(np.abs(S[:, n_pix:] + c_f) <= 1e-6)
    # window decisions equal the exact ones away from the boundary
    exact = X.astype(np.float64) @ Pn.T.astype(np.float64)
    inw = exact >= c
    safe = np.abs(exact - c) > 1e-5
    cnt = acc[:, 16]
    Y = acc[:, :16].astype(np.float64) * 2.0 ** -36
    split = (Ph.astype(np.float64) + Pm + Pl)
    for r in range(128):
        if not safe[r].all():
            continue
        assert cnt[r] == inw[r].sum(), r
        assert np.abs(Y[r] - split[inw[r]].sum(0)).max() <= 1e-4 * max(1, cnt[r])
    assert (cnt > 0).sum() >= 100


def _run(ms, emb, mask=None, **cfg):
    import torch
    e = torch.from_numpy(np.ascontiguousarray(emb)).cuda()
    m = None if mask is None else torch.from_numpy(np.ascontiguousarray(mask)).cuda()
    res = ms.cluster(e, m, **cfg)
    torch.cuda.synchronize()
    return res.labels.cpu().numpy(), res.modes.cpu().numpy(), res.stats


def assert_labels_are_fp64_argmax(emb, mask, labels, modes):
    """Every foreground label is the FP64 argmax of the raw embedding's cosine
    over the given modes (lowest index on ties); pixels whose top two differ by
    less than 1e-12 accept either."""
    fg = np.ones(emb.shape[0], bool) if mask is None else mask.astype(bool)
    E = emb[fg].astype(np.float64)
    M = modes.astype(np.float64)
    C = (E @ M.T) / np.linalg.norm(E, axis=1)[:, None] / np.linalg.norm(M, axis=1)[None, :]
    best = np.argmax(C, axis=1)
    top = np.sort(C, axis=1)[:, -2:] if C.shape[1] > 1 else np.concatenate([C, C - 1], 1)
    clear = top[:, 1] - top[:, 0] > 1e-12
    got = labels[fg]
    assert np.array_equal(got[clear], best[clear]), int((got[clear] != best[clear]).sum())
    assert np.all(C[np.arange(len(got)), got] >= top[:, 1] - 1e-12)


def test_bf16_c1_separable_exact(ms_lib):
    f = synth.frame_c1_separable(seed=0)
    ref = oracle.run(f.emb)
    labels, modes, st = _run(ms_lib, f.emb, precision=ms_lib.MS_BF16)
    assert modes.shape[0] == ref.modes.shape[0] == 8
    assert same_order_errors(modes, ref.modes).max() <= 1e-5
    assert np.array_equal(labels, ref.labels)
    assert np.array_equal(st["seed_log"], ref.seed_log)
    assert np.array_equal(st["round_log"], ref.round_log)


@pytest.mark.parametrize("seed", [0, 1])
def test_bf16_c1_fragmented(ms_lib, seed):
    f = synth.frame_c1(seed=seed)
    ref = oracle.run(f.emb)
    labels, modes, st = _run(ms_lib, f.emb, precision=ms_lib.MS_BF16)
    assert mode_errors(modes, ref.modes).max() <= 1e-5
    assert matched_agreement(ref.labels, labels) >= 0.999
    assert st["band_pairs"] > 0


def test_bf16_equals_fp32_form(ms_lib):
    # identical window decisions: same seeds, rounds, modes count and labels
    f = synth.make_frame(4, 96, 96, 16, 6000, 9, 600.0, 0.3, 40.0, 200.0, 0.02)
    a = _run(ms_lib, f.emb, f.mask, precision=ms_lib.MS_FP32)
    b = _run(ms_lib, f.emb, f.mask, precision=ms_lib.MS_BF16)
    assert np.array_equal(a[2]["round_log"], b[2]["round_log"])
    assert a[1].shape == b[1].shape
    assert same_order_errors(a[1], b[1]).max() <= 1e-6
    assert matched_agreement(a[0], b[0]) >= 0.999


def test_bf16_masked_ragged(ms_lib):
    f = synth.make_frame(21, 50, 50, 16, 1237, 5, 240.0, 0.3, 150.0, 200.0, 0.02)
    ref = oracle.run(f.emb, f.mask)
    labels, modes, st = _run(ms_lib, f.emb, f.mask, precision=ms_lib.MS_BF16)
    assert (labels[f.mask == 0] == -1).all()
    assert mode_errors(modes, ref.modes).max() <= 1e-5
    assert matched_agreement(ref.labels, labels) >= 0.999


@pytest.mark.parametrize("shape", [1, 2, 3, 4, 5, 6, 7])
def test_tile_shapes_are_bit_identical(ms_lib, shape):
    # every warp arrangement runs the same arithmetic in the same order: the
    # same windows, band re-decisions, sums and therefore identical outputs
    for f in (synth.make_frame(4, 96, 96, 16, 6000, 9, 600.0, 0.3, 40.0, 200.0, 0.02), synth.frame_c1(seed=1)):
        a = _run(ms_lib, f.emb, f.mask, precision=ms_lib.MS_BF16)
        b = _run(ms_lib, f.emb, f.mask, precision=ms_lib.MS_BF16, tc_shape=shape)
        assert np.array_equal(a[0], b[0])
        assert np.array_equal(a[1], b[1])
        for k in ("seed_log", "round_log"):
            assert np.array_equal(a[2][k], b[2][k])
        assert a[2]["band_pairs"] == b[2]["band_pairs"]


def test_tile_shape_out_of_range_is_rejected(ms_lib):
    f = synth.frame_c1_separable(seed=0)
    with pytest.raises(ms_lib.MsError) as e:
        _run(ms_lib, f.emb, precision=ms_lib.MS_BF16, tc_shape=8)
    assert e.value.status == ms_lib.MS_ERR_INVALID_ARG


# ---------------------------------------------------------------- d = 32
# The tensor-core form for 17 <= d <= 32: two 16-dimensional halves, each with
# its own BF16 split operand tiles (seven GEMM1 products per tile, two Y
# blocks in GEMM2), the same FP32 re-decision band; labelling and coverage
# score both halves on the tensor cores (six products per mode tile).


@pytest.mark.parametrize("d", [32, 18])
def test_bf16_d32_equals_fp32_form_and_oracle(ms_lib, d):
    f = synth.make_frame(11, 96, 96, d, 6000, 9, 600.0, 0.3, 40.0, 200.0, 0.02)
    a = _run(ms_lib, f.emb, f.mask, precision=ms_lib.MS_FP32)
    b = _run(ms_lib, f.emb, f.mask, precision=ms_lib.MS_BF16)
    # identical window decisions: the same rounds, seeds and modes
    assert np.array_equal(a[2]["round_log"], b[2]["round_log"])
    assert np.array_equal(a[2]["seed_log"], b[2]["seed_log"])
    assert a[1].shape == b[1].shape
    assert same_order_errors(a[1], b[1]).max() <= 1e-6
    assert matched_agreement(a[0], b[0]) >= 0.999
    ref = oracle.run(f.emb, f.mask)
    assert mode_errors(b[1], ref.modes).max() <= 1e-5
    assert matched_agreement(ref.labels, b[0]) >= 0.999
    assert (b[0][f.mask == 0] == -1).all()
    # the tensor-core labelling (both 16-dimensional halves for d > 16) gives
    # the exact FP64 argmax over its own modes
    assert_labels_are_fp64_argmax(f.emb, f.mask, b[0], b[1])


@pytest.mark.parametrize("shape", [2, 4, 6])
def test_bf16_d32_tile_shapes_are_bit_identical(ms_lib, shape):
    f = synth.make_frame(12, 64, 64, 32, 3000, 6, 400.0, 0.3, 60.0, 200.0, 0.02)
    a = _run(ms_lib, f.emb, f.mask, precision=ms_lib.MS_BF16)
    b = _run(ms_lib, f.emb, f.mask, precision=ms_lib.MS_BF16, tc_shape=shape)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(a[2]["round_log"], b[2]["round_log"])
