"""Pins for the FP64 oracle: each check ties it to something other than itself.

Sources of truth: hand-placed geometry with windows listed by hand, closed
forms, published generator outputs, the paper's own simulation design
(Sec. 4.2: orthogonal/opposite blob centres), the inverse relation between
Eq. 14 and Eq. 19, the exact inclusion-exclusion probability, Monte Carlo,
and the per-seed trajectory function checked against the lockstep round.
"""
import math
import os

import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def matched_agreement(a, b):
    """Fraction of foreground pixels with equal labels after optimal matching."""
    fg = a >= 0
    a, b = a[fg], b[fg]
    ua, ia = np.unique(a, return_inverse=True)
    ub, ib = np.unique(b, return_inverse=True)
    C = np.zeros((ua.size, ub.size), dtype=np.int64)
    np.add.at(C, (ia, ib), 1)
    r, c = linear_sum_assignment(-C)
    return C[r, c].sum() / max(fg.sum(), 1)


# ------------------------------------------------------------------ seeding
def test_splitmix64_published_outputs():
    lines = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64.txt")) if l.strip() and not l.startswith("#")]
    state = int(lines[0][1])
    want = [int(l[0], 16) for l in lines[1:]]
    assert oracle.splitmix64(state, len(want)) == want


@pytest.mark.parametrize("n", [1, 2, 3, 10, 97, 4096, 65537])
def test_affine_permutation_is_bijection(n):
    a, b = oracle.perm_params(n, seed=7, frame_id=3)
    p = oracle.perm(n, seed=7, frame_id=3)
    assert sorted(p.tolist()) == list(range(n))
    if n > 1:
        assert math.gcd(a, n) == 1 and 1 <= a <= n - 1
        # nearest coprime to round(0.618 n): nothing closer is coprime
        a0 = math.floor(0.6180339887 * n + 0.5)
        for k in range(abs(a - a0)):
            for cand in (a0 - k, a0 + k):
                assert not (1 <= cand <= n - 1 and math.gcd(cand, n) == 1)
        # b is the first SplitMix64 output of seed ^ frame_id, mod n
        assert b == oracle.splitmix64(7 ^ 3)[0] % n
        assert p[0] == b


def test_affine_step_tie_takes_the_lower_candidate():
    # n = 16: round(0.618 * 16) = 10 shares the factor 2 with 16; at distance
    # one both 9 and 11 are coprime, and the lower one is taken
    assert oracle.perm_params(16)[0] == 9
    # n = 10: 6 and 5 share a factor with 10, 7 does not
    assert oracle.perm_params(10)[0] == 7


# ------------------------------------------------------------ normalisation
def test_normalize_compacts_and_unit_norms():
    rng = np.random.default_rng(0)
    emb = rng.standard_normal((50, 5)).astype(np.float32) * 3
    mask = (rng.uniform(size=50) < 0.5).astype(np.uint8)
    P, pn, idx = oracle.normalize(emb, mask)
    assert idx.tolist() == np.flatnonzero(mask).tolist()
    assert np.allclose(np.linalg.norm(P, axis=1), 1.0, rtol=0, atol=1e-15)
    assert np.allclose(pn, 1.0, rtol=0, atol=1e-15)
    # direction preserved
    e = emb[idx].astype(np.float64)
    assert np.allclose(P * np.linalg.norm(e, axis=1, keepdims=True), e, rtol=1e-14, atol=1e-14)
    bad = emb.copy(); bad[np.flatnonzero(mask)[0]] = 0
    with pytest.raises(ValueError):
        oracle.normalize(bad, mask)


def test_cosine_eq1_values():
    assert oracle.cos([1, 0], [1, 1]) == pytest.approx(1 / math.sqrt(2), abs=1e-15)
    assert oracle.cos([1, 0, 0], [-2, 0, 0]) == pytest.approx(-1.0, abs=1e-15)
    assert oracle.cos([1, 0, 0], [0, 5, 0]) == 0.0
    assert oracle.cos([3, 4], [6, 8]) == pytest.approx(1.0, abs=1e-15)  # scale invariant


# ------------------------------------------------------- window and update
def _ring(angles_deg):
    a = np.deg2rad(np.asarray(angles_deg, dtype=np.float64))
    return np.stack([np.cos(a), np.sin(a)], axis=1)


def test_window_listed_by_hand_d2():
    # Points on the unit circle; c = cos(25 deg). From x at 0 deg the window is
    # exactly the points within 25 degrees: -20, -5, 10, 24 (not 26, 90, 180).
    ang = [-20, -5, 10, 24, 26, 90, 180, -60]
    P = _ring(ang)
    pn = np.ones(len(ang))
    c = math.cos(math.radians(25))
    xn, cnt, margin = oracle.shift_step(P, pn, [1.0, 0.0], c)
    assert cnt == 4
    # the decision closest to the edge: the point at 24 degrees
    assert margin == pytest.approx(math.cos(math.radians(24)) - c, rel=0, abs=1e-15)
    s = P[[0, 1, 2, 3]].sum(axis=0)
    assert np.allclose(xn, s / np.linalg.norm(s), rtol=0, atol=1e-15)


def test_window_boundary_is_inclusive_eq11():
    # d = 4 dyadic unit vectors: cos((1,0,0,0), (1/2,1/2,1/2,1/2)) = 1/2 exactly.
    P = np.array([[0.5, 0.5, 0.5, 0.5], [1.0, 0.0, 0.0, 0.0]])
    pn = np.ones(2)
    x = np.array([1.0, 0.0, 0.0, 0.0])
    _, cnt_at, _ = oracle.shift_step(P, pn, x, 0.5)
    _, cnt_above, _ = oracle.shift_step(P, pn, x, np.nextafter(0.5, 1.0))
    assert cnt_at == 2 and cnt_above == 1


def test_symmetric_window_mean_closed_form():
    # Pairs at +/- alpha around 0 deg: the normalised mean is exactly (1, 0).
    P = _ring([-15, 15, -7, 7, 0])
    xn, cnt, _ = oracle.shift_step(P, np.ones(5), [math.cos(0.01), math.sin(0.01)], 0.9)
    assert cnt == 5
    assert abs(xn[1]) < 1e-15 and xn[0] == pytest.approx(1.0, abs=1e-15)


def test_one_cluster_single_step_fixed_point():
    # All pairwise cosines >= c: the window is the whole set from any seed, so
    # one step reaches normalise(sum p), and the next step does not move.
    rng = np.random.default_rng(1)
    mu = np.array([1.0, 0, 0, 0])
    P = synth.sample_vmf(rng, mu, 5000.0, 40)
    assert (P @ P.T).min() >= 0.9
    want = P.sum(axis=0) / np.linalg.norm(P.sum(axis=0))
    for s in (0, 17, 39):
        traj, counts, T = oracle.trajectory(P, np.linalg.norm(P, axis=1), P[s], 0.9)
        assert T == 2 and counts.tolist() == [40, 40]
        assert np.allclose(traj[1], want, rtol=0, atol=1e-15)
        assert np.array_equal(traj[2], traj[1])


# ------------------------------------------------- trajectories and rounds
def _F(P, x, c):
    return np.maximum(0.0, P @ x - c).sum()


def test_objective_monotone_along_trajectories():
    # F(x) = sum_i max(0, x.p_i - c) cannot decrease under the flat-kernel
    # update (x' maximises y.x on the sphere for y = sum of the window).
    f = synth.frame_c1(seed=3)
    P, pn, _ = oracle.normalize(f.emb)
    rng = np.random.default_rng(2)
    for s in rng.choice(P.shape[0], 40, replace=False):
        traj, counts, T = oracle.trajectory(P, pn, P[s], 0.9)
        F = [_F(P, x, 0.9) for x in traj]
        assert all(F[i + 1] >= F[i] - 1e-12 for i in range(len(F) - 1))
        assert np.allclose(np.linalg.norm(traj[1:], axis=1), 1.0, rtol=0, atol=1e-12)


def test_round_early_stop_matches_trajectories():
    # The lockstep round must stop at the first sweep t with
    # #{seeds converged by t} > gamma * m ("more than gamma", Sec. 3.2.3),
    # where each seed's convergence sweep comes from its own trajectory.
    # m = 64 and gamma = count/64 make gamma*m exact, so thresholds that are
    # met with equality are exercised.
    f = synth.frame_c1(seed=4)
    P, pn, _ = oracle.normalize(f.emb)
    rng = np.random.default_rng(3)
    m = 64
    seeds = rng.choice(P.shape[0], m, replace=False)
    T = np.array([oracle.trajectory(P, pn, P[s], 0.9)[2] for s in seeds])
    assert (T > 0).all()
    counts = sorted(set(int((T <= t).sum()) for t in range(1, T.max() + 1)))
    gammas = [0.0, 0.9, 1.0] + [cnt / m for cnt in counts if 0 < cnt < m][:6]
    for gamma in gammas:
        r = oracle.shift_round(P, pn, P[seeds], gamma=gamma)
        t_stop = next(t for t in range(1, 301) if (T <= t).sum() > gamma * m or (T <= t).sum() == m)
        assert r["sweeps"] == t_stop, gamma
        # one seed-iteration per seed and sweep while it is active: a seed is
        # shifted until it converges or the round stops
        assert r["seed_iters"] == int(np.minimum(T, t_stop).sum()), gamma
        conv = r["state"] == 1
        assert np.array_equal(conv, T <= t_stop)
        assert np.array_equal(r["conv_iter"][conv], T[conv])
        # the converged positions equal the trajectories' end points
        for j in np.flatnonzero(conv)[:10]:
            traj, _, _ = oracle.trajectory(P, pn, P[seeds[j]], 0.9)
            assert np.array_equal(r["X"][j], traj[-1])


# ---------------------------------------------------------------- merge
def test_merge_order_and_threshold_by_hand():
    # Candidates at 0, 10, 30 and 80 degrees with supports 5, 9, 1, 1.
    # Order: 10 (9), 0 (5), then 30 and 80 (support 1, seed order 2 < 3).
    # 10 kept; 0 has cos 10deg = 0.985 >= 0.9 -> merged; 30 has cos 20deg =
    # 0.940 to 10 -> merged; 80 has cos 70deg to 10 -> kept.
    cand = _ring([0, 10, 30, 80])
    kept, src, _ = oracle.merge(cand, [5, 9, 1, 1], [0, 1, 2, 3], 0.9)
    assert src.tolist() == [1, 3]
    assert np.array_equal(kept, cand[[1, 3]])
    # equal supports: earlier seed order wins
    kept, src, _ = oracle.merge(_ring([0, 5]), [4, 4], [7, 3], 0.9)
    assert src.tolist() == [1]
    # previously kept modes persist and suppress new candidates
    kept, src, _ = oracle.merge(_ring([2, 60]), [1, 1], [0, 1], 0.9, kept=_ring([0]))
    assert kept.shape[0] == 2 and src.tolist() == [1]


def test_merge_threshold_is_strict():
    # a candidate is kept only when its cosine to every kept mode is below
    # merge_cos: (1,1,1,1) and (1,1,1,-1) have cosine 2/4 = 1/2 exactly, so at
    # merge_cos = 1/2 the second merges, and just above 1/2 it is kept
    cand = np.array([[1.0, 1.0, 1.0, 1.0], [1.0, 1.0, 1.0, -1.0]])
    _, src, _ = oracle.merge(cand, [2, 1], [0, 1], 0.5)
    assert src.tolist() == [0]
    _, src, _ = oracle.merge(cand, [2, 1], [0, 1], np.nextafter(0.5, 1.0))
    assert src.tolist() == [0, 1]


def test_cover_by_hand():
    P = _ring([0, 20, 40, 100])
    cov, left, margin = oracle.cover(P, np.ones(4), _ring([30]), np.zeros(4, np.uint8), c=math.cos(math.radians(12)))
    assert cov.tolist() == [0, 1, 1, 0] and left == 2
    # closest to the edge: the pixels 10 degrees from the mode
    assert margin == pytest.approx(math.cos(math.radians(10)) - math.cos(math.radians(12)), rel=0, abs=1e-15)
    cov2, left2, _ = oracle.cover(P, np.ones(4), _ring([30]), np.array([1, 0, 0, 0], np.uint8),
                                  c=math.cos(math.radians(12)))
    assert cov2.tolist() == [1, 1, 1, 0] and left2 == 1
    # inclusive boundary: cos = 1/2 exactly with c = 1/2 covers the pixel
    Pd = np.array([[0.5, 0.5, 0.5, 0.5], [0.0, 1.0, 0.0, 0.0]])
    cov3, left3, _ = oracle.cover(Pd, np.ones(2), np.array([[1.0, 0, 0, 0]]), np.zeros(2, np.uint8), c=0.5)
    assert cov3.tolist() == [1, 0] and left3 == 1


def test_label_argmax_ties_lowest_and_background():
    P = _ring([0, 44, 46, 90])
    modes = _ring([0, 90, 0])  # mode 2 duplicates mode 0
    labels, margin = oracle.label(P, np.ones(4), np.array([0, 2, 3, 5]), modes, 6)
    assert labels.tolist() == [0, -1, 0, 1, -1, 1]
    assert margin[0] == 0.0  # exact tie between modes 0 and 2
    # top-two margin when the best mode comes last: 1 - cos 45 degrees
    _, margin = oracle.label(_ring([0]), np.ones(1), np.array([0]), _ring([90, 45, 0]), 1)
    assert margin[0] == pytest.approx(1.0 - math.sqrt(0.5), rel=0, abs=1e-15)


# ----------------------------------------------------------- OSOP theory
def _exact_all_hit(N, I):
    # inclusion-exclusion for I equal clusters, in exact rationals (the float
    # sum cancels catastrophically for large I)
    from fractions import Fraction
    return float(sum((-1) ** j * math.comb(I, j) * Fraction(I - j, I) ** N for j in range(I + 1)))


@pytest.mark.parametrize("I", [1, 2, 5, 10, 40])
def test_eq14_against_exact_and_special_values(I):
    for N in (0, 1, 5, 20, 100, 400):
        eq14 = oracle.p_all_seeded(N, I)
        exact = _exact_all_hit(N, I)
        # hitting events are negatively correlated: product of marginals >= joint
        assert eq14 >= exact - 1e-12
        if I == 1:
            assert eq14 == (0.0 if N == 0 else 1.0)
        if I == 2 and N >= 1:
            assert eq14 - exact == pytest.approx(0.25 ** N, abs=1e-15)
    assert abs(oracle.p_all_seeded(2000, I) - _exact_all_hit(2000, I)) < 1e-6


def test_eq14_monte_carlo():
    rng = np.random.default_rng(5)
    I, N, trials = 8, 40, 20000
    hits = rng.integers(0, I, size=(trials, N))
    allhit = np.mean([len(np.unique(h)) == I for h in hits])
    exact = _exact_all_hit(N, I)
    assert abs(allhit - exact) < 4 * math.sqrt(exact * (1 - exact) / trials)
    assert oracle.p_all_seeded(N, I) >= allhit - 0.02


@pytest.mark.parametrize("I,r,P", [(2, 1.0, 0.99), (10, 1.0, 0.99), (60, 1.0, 0.99), (8, 0.5, 0.95),
                                   (2500, 1.0, 0.99), (3, 0.3, 0.9)])
def test_eq19_inverts_eq14(I, r, P):
    nmin = oracle.nmin(I, r, P)
    assert nmin > 0
    assert oracle.p_all_seeded(nmin, I, r) == pytest.approx(P, rel=1e-9)
    assert oracle.p_all_seeded(math.ceil(nmin), I, r) >= P - 1e-12
    assert oracle.nmin(I, r, min(P + 0.005, 0.999)) > nmin
    assert oracle.nmin(I + 1, r, P) > nmin


def test_schedule_hand_worked_rows():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "eq19_schedule.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) >= 10
    for N, I, unc, want in rows:
        assert oracle.next_n(int(N), int(I), int(unc)) == int(want), (N, I, unc)


def test_schedule_bounds_are_strict():
    # Eq. 21 doubles N only when it is below L N_min and subtracts N_min only
    # when it is above H N_min: at N = L N_min (or H N_min) exactly, N stays.
    # L is chosen as N / N_min where that product rounds back to N exactly.
    I = 10
    nm = oracle.nmin(I)
    N = next(N for N in range(int(nm) + 2, int(nm) + 400) if (N / nm) * nm == N)
    edge = N / nm
    assert oracle.next_n(N, I, 10 ** 6, L=edge, H=1e9) == N
    assert oracle.next_n(N, I, 10 ** 6, L=0.5, H=edge) == N
    # one unit in the last place inside the band's edge, the rule acts
    assert oracle.next_n(N, I, 10 ** 6, L=np.nextafter(edge, 2 * edge), H=1e9) == 2 * N
    assert oracle.next_n(N, I, 10 ** 6, L=0.5, H=np.nextafter(edge, 0.0)) == N - math.ceil(nm)
    # N never drops below one seed: with P = 0.001 and I = 2, N_min = 0.046, so
    # N = 1 lies above H N_min and 1 - ceil(N_min) = 0 is clamped to 1
    assert oracle.nmin(2, P=0.001) < 1.0 / 8.0
    assert oracle.next_n(1, 2, 100, P=0.001) == 1


# ------------------------------------------------------- whole method
def test_paper_orthogonal_blob_design_modes_are_cluster_means():
    # Sec. 4.2 design: 10 clusters, 18-d, noise 0.01, centres orthogonal or
    # opposite. Every cluster fits one window, so each mode is exactly the
    # normalised sum of its cluster's unit vectors and labels equal the truth.
    emb, truth = synth.orthogonal_blobs(seed=11, n=2000)
    r = oracle.run(emb, dim=18)
    assert r.modes.shape[0] == 10
    assert matched_agreement(truth, r.labels) == 1.0
    P, _, _ = oracle.normalize(emb)
    for k in range(10):
        members = r.labels == k
        s = P[members].sum(axis=0)
        assert np.allclose(r.modes[k], s / np.linalg.norm(s), rtol=0, atol=1e-13)
        assert r.support[k] == members.sum()


def test_separable_clusters_recovered_and_modes_fixed_points():
    f = synth.frame_c1_separable()
    r = oracle.run(f.emb)
    assert r.modes.shape[0] == 8
    assert matched_agreement(f.truth, r.labels) == 1.0
    P, pn, _ = oracle.normalize(f.emb)
    for k in range(8):
        assert abs(np.linalg.norm(r.modes[k]) - 1.0) <= 1e-12
        xn, cnt, _ = oracle.shift_step(P, pn, r.modes[k], 0.9)
        assert np.abs(xn - r.modes[k]).max() <= 1e-12
        assert cnt == r.support[k]
        # close to the generating direction
        assert np.max(f.means @ r.modes[k]) > 0.99


def test_fixed_points_on_fragmented_frame():
    f = synth.frame_c1(seed=0)
    r = oracle.run(f.emb)
    P, pn, _ = oracle.normalize(f.emb)
    S = r.modes @ P.T
    margin = np.abs(S - 0.9).min(axis=1)
    checked = 0
    for k in np.flatnonzero(margin > 1e-6):
        xn, cnt, _ = oracle.shift_step(P, pn, r.modes[k], 0.9)
        assert np.abs(xn - r.modes[k]).max() <= 1e-12
        checked += 1
    assert checked > 0.95 * r.modes.shape[0]
    assert np.allclose(np.linalg.norm(r.modes, axis=1), 1.0, rtol=0, atol=1e-12)
    # kept modes are pairwise farther apart than the merge threshold
    G = r.modes @ r.modes.T
    np.fill_diagonal(G, -1)
    assert G.max() < 0.9


def test_osop_labels_equal_all_seeds_labels_when_separable():
    f = synth.frame_c1_separable(seed=2)
    r_osop = oracle.run(f.emb)
    r_all = oracle.run(f.emb, all_seeds=1)
    assert r_all.stats["rounds"] == 1 and r_all.stats["seeds"] == 4096
    # Algorithm 1 has no early stop: every seed is shifted to its mode
    assert r_all.stats["dropped"] == 0 and r_all.stats["candidates"] == 4096
    assert r_osop.stats["seeds"] < 1000
    assert matched_agreement(r_all.labels, r_osop.labels) == 1.0


@pytest.mark.parametrize("separable,n_initial", [(False, 128), (True, 1)])
def test_run_covers_every_pixel_and_schedule_follows_rule(separable, n_initial):
    # Eq. 19-21 with I = every mode kept so far. The separable frame started
    # from one seed keeps 1, 2, 4, 8 modes over its rounds: after round two,
    # I = 2 doubles N where the single mode of that round alone would not.
    f = synth.frame_c1_separable(seed=0) if separable else synth.frame_c1(seed=5)
    r = oracle.run(f.emb, n_initial=n_initial)
    log = r.round_log
    assert log[-1, 3] == 0
    assert log[0, 0] == n_initial
    for i in range(1, log.shape[0]):
        want = oracle.next_n(log[i - 1, 0], log[i - 1, 2], log[i - 1, 3])
        assert log[i, 0] == want
        assert log[i, 1] == min(log[i, 0], log[i - 1, 3])
    assert log[:, 1].sum() == r.stats["seeds"]
    # every pixel is a seed or within c of a mode
    P, _, _ = oracle.normalize(f.emb)
    within = (P @ r.modes.T).max(axis=1) >= 0.9
    seeded = np.zeros(P.shape[0], bool); seeded[r.seed_log] = True
    assert (within | seeded).all()
    assert np.unique(r.seed_log).size == r.seed_log.size


def test_seed_selection_is_next_uncovered_positions():
    # Re-derive every round's seeds from the permutation and the coverage
    # implied by the modes kept so far (the seed-selection step of Algorithm 2 with OSOP rounds).
    f = synth.frame_c1(seed=6)
    r = oracle.run(f.emb)
    P, _, _ = oracle.normalize(f.emb)
    n = P.shape[0]
    perm = oracle.perm(n)
    covered = np.zeros(n, bool)
    cursor = 0
    drawn = 0
    S = P @ r.modes.T
    for rnd, (want, got, kept, left) in enumerate(r.round_log):
        take = []
        while len(take) < want and cursor < n:
            i = perm[cursor]; cursor += 1
            if not covered[i]:
                covered[i] = True
                take.append(i)
        assert take == r.seed_log[drawn:drawn + got].tolist(), rnd
        drawn += got
        covered |= (S[:, :kept] >= 0.9).any(axis=1)
        assert n - covered.sum() == left


def test_masked_frame_background_is_minus_one():
    f = synth.make_frame(9, 48, 48, 16, 1200, 4, 300.0, 0.2, 200.0, 200.0, 0.0)
    r = oracle.run(f.emb, f.mask)
    assert (r.labels[f.mask == 0] == -1).all()
    assert (r.labels[f.mask == 1] >= 0).all()
    assert matched_agreement(np.where(f.mask == 1, f.truth, -1), r.labels) == 1.0


def test_video_carry_follows_the_schedule_bounded_by_the_largest_draw():
    """The seed count a video carries into its next frame (Sec. 3.2.4;
    Sec. 4.3, Table 3): the Eq. 19-21 update applied round by round from
    n_initial with each round's kept-mode count, without the clamp to the
    frame's uncovered pixels, then bounded by the largest batch the frame
    drew. Hand-worked on the separable C1 frame: 8 modes give
    N_min = ln(1 - 0.99^(1/8)) / ln(7/8) = 50.03, so N = 128 lies in
    [2 N_min, 8 N_min] and stays 128, the frame's largest draw; its own N
    was clamped to 3 for the last round."""
    f = synth.frame_c1_separable(seed=0)
    r = oracle.run(f.emb)
    assert r.round_log[:, 0].tolist() == [128, 3]
    nmin = math.log(1 - 0.99 ** (1 / 8)) / math.log(7 / 8)
    assert 100 < 2 * nmin < 128 < 8 * nmin
    assert r.stats["n_carry"] == 128
    # a frame whose modes keep N doubling: the unclamped updates outgrow the
    # frame, and its largest draw bounds the carry
    g = synth.frame_c1(seed=0)
    q = oracle.run(g.emb)
    n = 128
    for kept in q.round_log[:, 2]:
        n = oracle.next_n(n, int(kept), uncovered=10 ** 12)
    assert n > q.round_log[:, 1].max()
    assert q.stats["n_carry"] == q.round_log[:, 1].max()
