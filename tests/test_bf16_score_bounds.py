"""Error bounds of the BF16-split scores on the tensor cores, emulated in numpy.

Labelling (BF16 form) scores a pixel p against a mode m as
    S = Ph.Mh + Ph.Mm + Pm.Mh
with p = Ph + Pm + Pl and m = Mh + Mm + Ml the round-to-nearest BF16 splits of
the FP32 unit vectors (d = 16). It keeps the best mode only when it leads the
second by more than 2 * 2.5e-5, so |S - p.m| <= 2.5e-5 must hold for any
summation order of the 48 products in FP32. The shift scores a seed x against
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

EPS_TC = 2.5e-5
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


def _pairs():
    rng = np.random.default_rng(7)
    p1, m1 = unit_rows(rng, 60000), unit_rows(rng, 60000)
    p2, m2 = adversarial_pairs(rng, 60000)
    return np.concatenate([p1, p2]), np.concatenate([m1, m2])


def test_label_score_error_within_eps():
    p, m = _pairs()
    ph, pm, _ = split3(p)
    mh, mm, _ = split3(m)
    exact = (p.astype(np.float64) * m.astype(np.float64)).sum(1)
    terms = np.concatenate([ph.astype(np.float64) * mh, ph.astype(np.float64) * mm,
                            pm.astype(np.float64) * mh], axis=1)
    # every product of two BF16 values is exact in FP32
    assert np.array_equal(terms.astype(np.float32).astype(np.float64), terms)
    dropped = np.abs(terms.sum(1) - exact)
    assert dropped.max() <= 3 * 2.0 ** -18
    for total in (fp32_sequential_sum(terms), fp32_truncating_sum(terms)):
        assert np.abs(total - exact).max() <= EPS_TC


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
        # the dropped terms (Xh.Pl, Xl.Pm, Xl.Pl and x - (Xh + Xl)) and FP32 accumulation
        assert err.max() <= 2.4e-5
        assert err.max() + 1e-6 < BAND / 2
        # outside the band the sign of S' is the exact decision, with room for
        # the FP32 form's 1e-6
        out = np.abs(S) >= BAND
        assert np.all((S[out] >= 0) == (exact[out] >= 0))
        assert np.all(np.abs(exact[out]) > BAND - err.max() - 1e-7)
        assert (~out).sum() > 100  # the adversarial pairs reach the band
