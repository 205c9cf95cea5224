"""Error bounds of the BF16-split scores on the tensor cores, emulated in numpy.

Labelling and coverage (BF16 form) score a pixel p against a mode m as
    S = Ph.Mh + Ph.Mm + Pm.Mh      (per 16-dimensional half)
with p = Ph + Pm + Pl and m = Mh + Mm + Ml the round-to-nearest BF16 splits of
the FP32 unit vectors. Labelling keeps the best mode only when it leads the
second by more than 2 * eps, coverage decides only scores more than eps from
c, so |S - p.m| <= eps must hold for any summation order of the 3d products
in FP32: eps = 6e-5 for d = 16 and 7e-5 for d = 32. The dropped products
ph.ml + pm.(mm + ml) + pl.m are at most 2^-16 (1 + 2^-8) |p_k||m_k| each (a
round-to-nearest BF16 residual is at most 2^-8 of the value it splits), so at
most 3.04 * 2^-16 = 4.64e-5 over a unit pair; the accumulation adds at most
2^-22 per addition. The worst case is built explicitly: every component at the
rounding pattern that maximises the dropped terms. The shift scores a seed x against
p as S' = Xh.Ph + Xh.Pm + Xl.Ph - c (the -c enters as three BF16 terms
against a ones column) and re-decides pairs with |S'| < 2^-14, so
|S' - (x.p - c)| must stay well below 2^-14, and every pair outside the band
must be settled the way the exact score and the FP32 form's dot product
(within 1e-6 of it) settle it.

Each BF16 x BF16 product has at most 16 significant bits and is exact in
FP32. The tensor cores' FP32 accumulation order and rounding are not
specified, so the emulation sums the products in two ways: sequentially with
one round-to-nearest per addition, and with a pessimistic truncating adder
that first cuts both addends to the grid of the larger one's last FP32 bit and
then rounds the sum toward zero (at most two units in the last place lost per
addition, where round to nearest loses half of one). The dropped terms are
checked in exact float64 arithmetic."""
import numpy as np

EPS_TC = {16: 6e-5, 32: 7e-5}
DROPPED = 3.04 * 2.0 ** -16
BAND = 2.0 ** -14


def bf16_rn(x):
    """FP32 -> nearest BF16 (ties to even), returned as FP32."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def split3(v):
    v = np.asarray(v, dtype=np.float32)
    h = bf16_rn(v)
    m = bf16_rn((v - h).astype(np.float32))
    l = bf16_rn(((v - h).astype(np.float32) - m).astype(np.float32))
    return h, m, l


def unit_rows(rng, n, d=16):
    v = rng.standard_normal((n, d))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    v = v.astype(np.float32)
    # components below 2^-100 are stored as 0 by the library
    v[np.abs(v) < 2.0 ** -100] = 0.0
    return v


def adversarial_pairs(rng, n, d=16):
    """Pairs with cosines near 0.9 and near 1 (close directions), components
    straddling BF16 rounding boundaries."""
    a = unit_rows(rng, n, d).astype(np.float64)
    t = rng.standard_normal((n, d))
    t -= (t * a).sum(1, keepdims=True) * a
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    ang = np.where(rng.random(n) < 0.5, np.arccos(0.9) + rng.normal(0, 1e-4, n), rng.uniform(0, 0.05, n))
    b = np.cos(ang)[:, None] * a + np.sin(ang)[:, None] * t
    b /= np.linalg.norm(b, axis=1, keepdims=True)
    # nudge components onto BF16 half-way points (rounding ties)
    b32 = b.astype(np.float32)
    k = rng.integers(0, d, n)
    bits = b32[np.arange(n), k].view(np.uint32)
    b32[np.arange(n), k] = ((bits & 0xFFFF0000) | 0x8000).view(np.float32)
    b32 /= np.linalg.norm(b32.astype(np.float64), axis=1, keepdims=True).astype(np.float32)
    return a.astype(np.float32), b32


def fp32_sequential_sum(terms):
    """terms: [n, T] float64 holding exact FP32 products; returns the FP32 sum
    taken left to right."""
    acc = np.zeros(terms.shape[0], dtype=np.float32)
    for j in range(terms.shape[1]):
        acc = (acc + terms[:, j].astype(np.float32)).astype(np.float32)
    return acc.astype(np.float64)


def _ulp32(x):
    """Spacing of FP32 values at |x| (the normal range is all that occurs here)."""
    e = np.floor(np.log2(np.maximum(np.abs(x), 2.0 ** -126)))
    return 2.0 ** (e - 23)


def _trunc(x, q):
    return np.trunc(x / q) * q


def fp32_truncating_sum(terms):
    """The same sum with a truncating adder: both addends cut toward zero to the
    last-bit grid of the larger one, the exact sum of the cut values then cut
    toward zero to FP32. Every value stays an FP32 number (float64 holds it
    exactly)."""
    acc = np.zeros(terms.shape[0])
    for j in range(terms.shape[1]):
        t = terms[:, j]
        q = _ulp32(np.maximum(np.abs(acc), np.abs(t)))
        s = _trunc(acc, q) + _trunc(t, q)
        acc = _trunc(s, _ulp32(s))
    return acc


def worst_pairs(d, n=256, seed=3):
    """Pairs of near-unit vectors whose components all sit at the BF16
    rounding pattern with the largest dropped terms: candidate values
    0.25 (1 + a) with the first residual near 2^-8 of the value, searched pair
    by pair; the best few pairs are repeated over all d components (norms
    within 1% of 1)."""
    rng = np.random.default_rng(seed)
    a = np.concatenate([s * (2.0 ** -8 - rng.uniform(0, 2.0 ** -14, 1500)) + rng.uniform(-2.0 ** -16, 2.0 ** -16, 1500)
                        for s in (-1, 1)])
    x = (0.25 * (1 + a)).astype(np.float32)
    h, m, _ = split3(x)
    X = x.astype(np.float64)
    E = np.abs(np.outer(h, h.astype(np.float64)) + np.outer(h, m.astype(np.float64))
               + np.outer(m, h.astype(np.float64)) - np.outer(X, X)) / np.outer(X, X)
    flat = np.argsort(E, axis=None)[::-1][:n]
    i, j = np.unravel_index(flat, E.shape)
    return np.repeat(x[i][:, None], d, 1) * 4 / np.sqrt(d), np.repeat(x[j][:, None], d, 1) * 4 / np.sqrt(d)


def _pairs(d=16):
    rng = np.random.default_rng(7)
    p1, m1 = unit_rows(rng, 60000, d), unit_rows(rng, 60000, d)
    p2, m2 = adversarial_pairs(rng, 60000, d)
    p3, m3 = worst_pairs(d)
    return (np.concatenate([p1, p2, p3.astype(np.float32)]), np.concatenate([m1, m2, m3.astype(np.float32)]))


def _label_terms(p, m, d):
    """The 3d products of S, half by half."""
    ph, pm, _ = split3(p)
    mh, mm, _ = split3(m)
    out = []
    for h0 in range(0, d, 16):
        sl = slice(h0, h0 + 16)
        out += [ph[:, sl].astype(np.float64) * mh[:, sl], ph[:, sl].astype(np.float64) * mm[:, sl],
                pm[:, sl].astype(np.float64) * mh[:, sl]]
    return np.concatenate(out, axis=1)


def test_worst_pairs_reach_the_dropped_term_regime():
    """The constructed pairs drop more than 2^-16 per unit pair, the old
    2.5e-5 allowance is not a bound, and none drops more than the derived
    3.04 * 2^-16."""
    p, m = worst_pairs(16)
    exact = (p * m).sum(1)
    dropped = np.abs(_label_terms(p.astype(np.float32), m.astype(np.float32), 16).sum(1) - exact)
    scale = np.linalg.norm(p, axis=1) * np.linalg.norm(m, axis=1)
    assert dropped.max() > 2.5e-5
    assert np.all(dropped <= DROPPED * scale)


def test_label_score_error_within_eps():
    for d in (16, 32):
        p, m = _pairs(d)
        exact = (p.astype(np.float64) * m.astype(np.float64)).sum(1)
        scale = np.linalg.norm(p.astype(np.float64), axis=1) * np.linalg.norm(m.astype(np.float64), axis=1)
        terms = _label_terms(p, m, d)
        # every product of two BF16 values is exact in FP32
        assert np.array_equal(terms.astype(np.float32).astype(np.float64), terms)
        dropped = np.abs(terms.sum(1) - exact)
        assert np.all(dropped <= DROPPED * scale)
        for total in (fp32_sequential_sum(terms), fp32_truncating_sum(terms)):
            assert np.all(np.abs(total - exact) <= EPS_TC[d] * scale), d


def test_shift_score_error_inside_band():
    c = np.float32(0.9)
    c_f = float(c) if float(c) >= 0.9 else float(np.nextafter(c, np.float32(2)))  # c rounded up to FP32
    x, p = _pairs()
    xh = bf16_rn(x)
    xl = bf16_rn((x - xh).astype(np.float32))
    ph, pm, _ = split3(p)
    ch = bf16_rn(np.float32(c_f))
    cm = bf16_rn(np.float32(c_f - ch))
    cl = np.float32((np.float32(c_f) - ch) - cm)
    assert float(ch) + float(cm) + float(cl) == c_f  # the three-term split of c is exact
    exact = (x.astype(np.float64) * p.astype(np.float64)).sum(1) - c_f
    n = x.shape[0]
    cterm = np.tile(np.array([-ch, -cm, -cl], dtype=np.float64), (n, 1))
    terms = np.concatenate([xh.astype(np.float64) * ph, xh.astype(np.float64) * pm,
                            xl.astype(np.float64) * ph, cterm], axis=1)
    assert np.array_equal(terms.astype(np.float32).astype(np.float64), terms)
    for S in (fp32_sequential_sum(terms), fp32_truncating_sum(terms)):
        err = np.abs(S - exact)
        # the dropped terms (Xh.Pl, Xl.Pm, Xl.Pl and x - (Xh + Xl)): at most
        # 3.04 * 2^-16; the FP32 accumulation of 51 terms: at most 51 * 2^-22
        assert err.max() <= DROPPED + 51 * 2.0 ** -22
        assert DROPPED + 51 * 2.0 ** -22 + 1e-6 < BAND
        # outside the band the sign of S' is the exact decision, with room for
        # the FP32 form's 1e-6
        out = np.abs(S) >= BAND
        assert np.all((S[out] >= 0) == (exact[out] >= 0))
        assert np.all(np.abs(exact[out]) > BAND - err.max() - 1e-7)
        assert (~out).sum() > 100  # the adversarial pairs reach the band
