"""Parity at the full configuration sizes, in the launch configurations the
benchmark times.

C2 (one 512x512 frame, 131072 foreground pixels): the oracle needs about a
minute per frame, so its counters for synth.frame_c2(seed=0) are stored in
tests/golden/c2_oracle_stats.json and its kept modes, label map and seed log
in tests/golden/c2_oracle_result.npz (both written by committed scripts that
call only oracle/ and synth/). The GPU's modes must equal the oracle's in
count and keep order, each within 1 - cos <= 1e-5; its labels must equal the
oracle's on every pixel whose oracle top-two margin clears both 1e-5 and
twice the modes' largest direction error, and on at least 99.9% of all
pixels; the seed log must be the oracle's. This holds for the FP32 form, the
BF16 form and the BF16-batched graph with the work split its autotuner picks
(the benchmark's launch configuration), and for the C3 stack. Every integer counter of the GPU run -- rounds, kept
modes, seeds, seed-iterations, candidates, dropped seeds, iterations -- must
equal the oracle's where the method fixes it: rounds, kept modes and seeds
(which follow from the modes through coverage) exactly -- seeds within 0.01%
when the oracle saw a pixel within tol of the coverage boundary, because the
modes themselves agree only within the convergence tolerance. The counters that
count iterations (seed-iterations, candidates, dropped seeds, iterations) also
depend on the iteration at which a seed's FP32 step first falls below tol,
which can differ by one from the FP64 oracle's for a seed whose last moves are
near tol: they agree within 0.01% (seed-iterations), two seeds per round plus
0.1% (candidates, dropped; their sum is exact) and one iteration per round. Sampled outputs are then
checked one by one in FP64: labels are the FP64 argmax over the GPU's modes
(pixels whose top-two margin exceeds 1e-5), every foreground pixel is covered
(seeded or within c of a mode) and modes are fixed points of the FP64 update;
then every pixel's label is checked against the FP64 argmax over the GPU's
modes (top-two margin above 1e-12).

C4 (64 frames of uneven size, 2k-260k foreground pixels, one graph): each
frame of the batch equals a single-frame run of that frame bit for bit, and
the single-frame path is the one held to the oracle above.

C3 (three frames clustered jointly, ~393k pixels): counters against
tests/golden/c3_oracle_stats.json when that file is present."""
import json
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
COUNTERS = ("rounds", "n_modes", "seeds", "seed_iters", "candidates", "dropped", "iters_total")
EXACT = ("rounds", "n_modes", "seeds")


def _counters_match_oracle(st, ref, tol=1e-6):
    for k in EXACT:
        if k == "seeds" and ref["min_cover_margin"] <= tol:
            # the modes agree with the oracle's only within the convergence
            # tolerance, so a pixel whose FP64 cosine to a kept mode lies
            # within tol of c may be covered on one side and seeded on the
            # other; the oracle records that such a pixel exists
            assert abs(st[k] - ref[k]) <= max(2, 1e-4 * ref[k]), (k, st[k], ref[k])
            continue
        assert st[k] == ref[k], (k, st[k], ref[k])
    assert abs(st["seed_iters"] - ref["seed_iters"]) <= 1e-4 * ref["seed_iters"], (st["seed_iters"], ref["seed_iters"])
    # every seed ends as a candidate or a dropped seed; a seed converging one
    # iteration earlier or later moves between the two only at a round's early stop
    assert st["candidates"] + st["dropped"] == st["seeds"]
    for k in ("candidates", "dropped"):
        assert abs(st[k] - ref[k]) <= 2 * ref["rounds"] + 1e-3 * ref[k], (k, st[k], ref[k])
    assert abs(st["iters_total"] - ref["iters_total"]) <= ref["rounds"], (st["iters_total"], ref["iters_total"])


def _golden(name):
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        pytest.skip(f"{name} not present")
    return json.load(open(path))


def _dev(f):
    import torch
    e = torch.from_numpy(np.ascontiguousarray(f.emb)).cuda()
    m = None if f.mask is None else torch.from_numpy(np.ascontiguousarray(f.mask)).cuda()
    return e, m


def _sampled_checks(f, labels, modes, seed_pixels, c=0.9, n_samples=3000, seed=0):
    fg = np.flatnonzero(f.mask) if f.mask is not None else np.arange(f.emb.shape[0])
    P = f.emb[fg].astype(np.float64)
    P /= np.linalg.norm(P, axis=1, keepdims=True)
    M = modes.astype(np.float64)
    M /= np.linalg.norm(M, axis=1, keepdims=True)
    rng = np.random.default_rng(seed)
    idx = rng.choice(len(fg), size=min(n_samples, len(fg)), replace=False)
    S = P[idx] @ M.T
    top = np.sort(S, axis=1)
    safe = top[:, -1] - top[:, -2] > 1e-5
    # labels are the FP64 argmax over the kept modes
    assert np.array_equal(np.argmax(S, axis=1)[safe], labels[fg[idx]][safe])
    assert safe.mean() > 0.99
    # coverage: every sampled pixel was seeded or lies within c of a mode
    seeded = np.zeros(len(fg), dtype=bool)
    seeded[seed_pixels] = True
    assert np.all((top[:, -1] >= c - 1e-6) | seeded[idx])
    # modes are fixed points of the FP64 update over their FP64 window, to the
    # modes' 1e-5 bar; excused only is a mode whose window has a pixel within
    # FP32 rounding of the boundary (such a pixel can fall on either side)
    errs, excused = [], 0
    for j in rng.choice(len(M), size=min(64, len(M)), replace=False):
        s = P @ M[j]
        if np.any(np.abs(s - c) < 2e-6):
            excused += 1
            continue
        y = P[s >= c].sum(0)
        errs.append(1.0 - float(y @ M[j]) / np.linalg.norm(y))
    errs = np.array(errs)
    assert excused <= 8 and errs.max() <= 1e-5, (excused, errs.max())


def _full_label_check(f, labels, modes, margin=1e-12):
    """Every foreground pixel's label is the FP64 argmax of its cosine over the
    GPU's modes (lowest index on ties), except where the top two lie within
    `margin` (FP64 rounding decides those). Covers the labelling's near-tie
    re-decision, which the sampled check rarely reaches."""
    fg = np.flatnonzero(f.mask) if f.mask is not None else np.arange(f.emb.shape[0])
    P = f.emb[fg].astype(np.float64)
    P /= np.linalg.norm(P, axis=1, keepdims=True)
    M = modes.astype(np.float64)
    M /= np.linalg.norm(M, axis=1, keepdims=True)
    lab = labels[fg]
    for a in range(0, len(fg), 16384):
        S = P[a:a + 16384] @ M.T
        want = np.argmax(S, axis=1)
        top = np.partition(S, -2, axis=1)[:, -2:] if S.shape[1] > 1 else np.concatenate([S, S - 1], axis=1)
        clear = (top[:, 1] - top[:, 0]) > margin if S.shape[1] > 1 else np.ones(len(S), bool)
        assert np.array_equal(want[clear], lab[a:a + 16384][clear]), a
    assert np.all(labels[np.setdiff1d(np.arange(labels.size), fg)] == -1)


def _oracle_result(name):
    path = os.path.join(GOLDEN, f"{name}_oracle_result.npz")
    if not os.path.exists(path):
        pytest.skip(f"{name}_oracle_result.npz not present")
    return dict(np.load(path))


def _fg_unit(f):
    fg = np.flatnonzero(f.mask) if f.mask is not None else np.arange(f.emb.shape[0])
    P = f.emb[fg].astype(np.float64)
    return fg, P / np.linalg.norm(P, axis=1, keepdims=True)


def _top_two_margin(P, M):
    """Per pixel, FP64 top-1 minus top-2 cosine over the modes M."""
    Mn = M / np.linalg.norm(M, axis=1, keepdims=True)
    out = np.empty(P.shape[0])
    for a in range(0, P.shape[0], 16384):
        S = P[a:a + 16384] @ Mn.T
        top = np.partition(S, -2, axis=1)[:, -2:] if S.shape[1] > 1 else np.concatenate([S - 2, S], axis=1)
        out[a:a + 16384] = top[:, 1] - top[:, 0]
    return out


def _equal_to_oracle(f, ref, labels, modes, seed_log=None, exact_seeds=True):
    """Element-by-element parity with the oracle's stored result (the labelling
    step of Algorithm 2: every vector labelled by its nearest kept mode)."""
    from parity_util import same_order_errors
    K = ref["modes"].shape[0]
    assert modes.shape[0] == K, (modes.shape[0], K)
    err = same_order_errors(modes, ref["modes"])
    assert err.max() <= 1e-5, err.max()
    # a direction error delta moves any cosine by at most delta, and 1 - cos = delta^2 / 2
    delta = float(np.sqrt(2.0 * max(err.max(), 0.0)))
    fg, P = _fg_unit(f)
    bg = np.setdiff1d(np.arange(labels.size), fg)
    assert np.all(labels[bg] == -1) and np.all(ref["labels"][bg] == -1)
    want, got = ref["labels"][fg], labels[fg]
    if 2 * delta <= ref["safe_margin"]:
        safe = np.unpackbits(ref["margin_gt"])[: ref["labels"].size].astype(bool)[fg]
    else:
        safe = _top_two_margin(P, ref["modes"]) > 2 * delta
    assert safe.mean() > 0.99, safe.mean()
    bad = np.flatnonzero(safe & (want != got))
    assert bad.size == 0, (bad.size, bad[:10])
    assert (want == got).mean() >= 0.999, (want == got).mean()
    if seed_log is not None:
        if exact_seeds:
            assert np.array_equal(np.asarray(seed_log), ref["seed_log"])
        else:
            # a pixel within tol of the coverage boundary may be covered on one
            # side and drawn as a seed on the other: apart from those few seeds
            # the two logs are the same sequence
            a, b = np.asarray(seed_log), np.asarray(ref["seed_log"])
            odd = np.setxor1d(a, b)
            assert odd.size <= max(2, b.size // 10000), odd.size
            assert np.array_equal(a[~np.isin(a, odd)], b[~np.isin(b, odd)])
    return err.max()


def _label_agreement(a, b, modes_a, modes_b):
    """Share of foreground pixels with equal labels: index by index when both
    mode lists agree in order, else a greedy overlap matching (a lower bound of
    the optimal matching, which is too large to solve for 10^4 clusters)."""
    fg = a >= 0
    a, b = a[fg], b[fg]
    if modes_a.shape == modes_b.shape:
        ga = modes_a.astype(np.float64); gb = modes_b.astype(np.float64)
        err = 1.0 - (ga * gb).sum(1) / (np.linalg.norm(ga, axis=1) * np.linalg.norm(gb, axis=1))
        if err.max() <= 1e-5:
            return float((a == b).mean())
    nb = int(b.max()) + 1
    key, cnt = np.unique(a.astype(np.int64) * nb + b, return_counts=True)
    used_a, used_b, hit = set(), set(), 0
    order = np.argsort(-cnt, kind="stable")
    for k, n in zip(key[order], cnt[order]):
        ia, ib = int(k // nb), int(k % nb)
        if ia not in used_a and ib not in used_b:
            used_a.add(ia); used_b.add(ib); hit += int(n)
    return hit / max(1, a.size)


@pytest.mark.parametrize("bf16", [False, True])
def test_c2_full_frame_counters_equal_oracle(ms_lib, bf16):
    ref = _golden("c2_oracle_stats.json")
    f = synth.frame_c2(seed=0)
    e, m = _dev(f)
    prec = ms_lib.MS_BF16 if bf16 else ms_lib.MS_FP32
    res = ms_lib.cluster(e, m, precision=prec)
    _counters_match_oracle(res.stats, ref)
    _sampled_checks(f, res.labels.cpu().numpy(), res.modes.cpu().numpy(), res.stats["seed_log"])
    _full_label_check(f, res.labels.cpu().numpy(), res.modes.cpu().numpy())


def test_c2_frames_batched_as_benchmarked(ms_lib):
    """The benchmark's launch configuration: C2 frames in one graph, BF16, the
    work split chosen by the autotuner. With the canonical split frame 0's
    counters match the oracle's; a load-shared split cuts the FP32 partial sums
    differently, so it is held to the parity bar against the canonical run."""
    ref = _golden("c2_oracle_stats.json")
    import torch
    from parity_util import mode_errors
    fs = [synth.frame_c2(seed=i) for i in range(4)]
    embs = [torch.from_numpy(f.emb).cuda() for f in fs]
    masks = [torch.from_numpy(f.mask).cuda() for f in fs]
    c = ms_lib.ms_config_default(dim=16, precision=ms_lib.MS_BF16)
    b = ms_lib.ms_batch_create(c, embs, masks)
    try:
        ms_lib.ms_batch_run(b)  # canonical split
        _counters_match_oracle(ms_lib.ms_batch_stats(b, 0), ref)
        canon_labels = b.labels[0].cpu().numpy()
        canon_modes = ms_lib.ms_batch_modes(b, 0)
        single = ms_lib.cluster(embs[0], masks[0], precision=ms_lib.MS_BF16)
        _sampled_checks(fs[0], canon_labels, canon_modes, single.stats["seed_log"])
        res = ms_lib.ms_batch_autotune(b, reps=1)
        assert len(res) == 12
        modes = ms_lib.ms_batch_modes(b, 0)
        assert abs(modes.shape[0] - ref["n_modes"]) <= ref["n_modes"] // 1000
        assert mode_errors(modes, canon_modes).max() <= 1e-5
        assert _label_agreement(canon_labels, b.labels[0].cpu().numpy(), canon_modes, modes) >= 0.999
    finally:
        b.close()


@pytest.mark.parametrize("d,bf16,n_single", [(16, True, 64), (32, False, 6), (32, True, 6)])
def test_c4_batch_equals_single_frames(ms_lib, d, bf16, n_single):
    import torch
    fs = synth.batch_c4(seed=0, B=64, d=d)
    embs = [torch.from_numpy(f.emb).cuda() for f in fs]
    masks = [torch.from_numpy(f.mask).cuda() for f in fs]
    prec = ms_lib.MS_BF16 if bf16 else ms_lib.MS_FP32
    c = ms_lib.ms_config_default(dim=d, precision=prec)
    b = ms_lib.ms_batch_create(c, embs, masks)
    try:
        ms_lib.ms_batch_run(b)
        # a spread of frames, always including the smallest and the largest
        sizes = np.array([int(f.mask.sum()) for f in fs])
        order = list(np.argsort(sizes))
        pick = sorted(set([order[0], order[-1]] + list(np.linspace(0, 63, n_single).astype(int))))
        for i in pick[:n_single]:
            res = ms_lib.cluster(embs[i], masks[i], precision=prec, frame_id=i)
            assert np.array_equal(ms_lib.ms_batch_modes(b, i), res.modes.cpu().numpy()), i
            assert np.array_equal(b.labels[i].cpu().numpy(), res.labels.cpu().numpy()), i
            st = ms_lib.ms_batch_stats(b, i)
            for k in COUNTERS:
                assert st[k] == res.stats[k], (i, k)
    finally:
        b.close()


def test_c3_tracking_stack_counters_equal_oracle(ms_lib):
    ref = _golden("c3_oracle_stats.json")
    f = synth.stack_c3(seed=0)
    e, m = _dev(f)
    res = ms_lib.cluster(e, m, precision=ms_lib.MS_BF16)
    _counters_match_oracle(res.stats, ref)
    _sampled_checks(f, res.labels.cpu().numpy(), res.modes.cpu().numpy(), res.stats["seed_log"])


@pytest.mark.parametrize("bf16", [False, True])
def test_c2_full_frame_modes_and_labels_equal_oracle(ms_lib, bf16):
    ref = _oracle_result("c2")
    st = _golden("c2_oracle_stats.json")
    f = synth.frame_c2(seed=0)
    e, m = _dev(f)
    res = ms_lib.cluster(e, m, precision=ms_lib.MS_BF16 if bf16 else ms_lib.MS_FP32)
    _equal_to_oracle(f, ref, res.labels.cpu().numpy(), res.modes.cpu().numpy(), res.stats["seed_log"],
                     exact_seeds=st["min_cover_margin"] > 1e-6)
    assert np.array_equal(res.stats["round_log"], ref["round_log"])


def test_c2_batched_autotuned_modes_and_labels_equal_oracle(ms_lib):
    """The benchmark's launch configuration (BF16, C2 frames in one graph, the
    work split the autotuner keeps), frame 0 against the oracle."""
    import torch
    ref = _oracle_result("c2")
    fs = [synth.frame_c2(seed=i) for i in range(4)]
    embs = [torch.from_numpy(f.emb).cuda() for f in fs]
    masks = [torch.from_numpy(f.mask).cuda() for f in fs]
    c = ms_lib.ms_config_default(dim=16, precision=ms_lib.MS_BF16)
    b = ms_lib.ms_batch_create(c, embs, masks)
    try:
        ms_lib.ms_batch_autotune(b, reps=1)
        _equal_to_oracle(fs[0], ref, b.labels[0].cpu().numpy(), ms_lib.ms_batch_modes(b, 0))
        st = ms_lib.ms_batch_stats(b, 0)
        assert st["n_modes"] == ref["modes"].shape[0] and st["rounds"] == ref["round_log"].shape[0]
    finally:
        b.close()


def test_c3_stack_modes_and_labels_equal_oracle(ms_lib):
    ref = _oracle_result("c3")
    st = _golden("c3_oracle_stats.json")
    f = synth.stack_c3(seed=0)
    e, m = _dev(f)
    res = ms_lib.cluster(e, m, precision=ms_lib.MS_BF16)
    # the oracle saw a pixel within tol of the coverage boundary, so the seed
    # log may differ by a seed where the FP32 modes cover it and FP64's do not
    _equal_to_oracle(f, ref, res.labels.cpu().numpy(), res.modes.cpu().numpy(), res.stats["seed_log"],
                     exact_seeds=st["min_cover_margin"] > 1e-6)
