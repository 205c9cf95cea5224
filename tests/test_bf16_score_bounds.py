"""Error bounds of the BF16-split scores on the tensor cores, emulated in numpy.

Labelling (BF16 form) scores a pixel p against a mode m as
    S = Ph.Mh + Ph.Mm + Pm.Mh
with p = Ph + Pm + Pl and m = Mh + Mm + Ml the round-to-nearest BF16 splits of
the FP32 unit vectors (d = 16). It keeps the best mode only when it leads the
second by more than 2 * 2.5e-5, so |S - p.m| <= 2.5e-5 must hold for any
summation order of the 48 products in FP32. The shift scores a seed x against
p as S' = Xh.Ph + Xh.Pm + Xl.Ph - c (the -c enters as three BF16 terms
against a ones column) and re-decides pairs with |S'| < 2^-14, so
|S' - (x.p - c)| must stay well below 2^-14.

Each BF16 x BF16 product has at most 16 significant bits and is exact in
FP32; the emulation sums them in FP32 sequentially (the worst common order,
one rounding per addition) and also checks the dropped terms in exact float64
arithmetic."""
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
    s32 = fp32_sequential_sum(terms)
    assert np.abs(s32 - exact).max() <= EPS_TC


def test_shift_score_error_inside_band():
    c = np.float32(0.9)
    x, p = _pairs()
    xh = bf16_rn(x)
    xl = bf16_rn((x - xh).astype(np.float32))
    ph, pm, _ = split3(p)
    ch = bf16_rn(c)
    cm = bf16_rn(np.float32(c - ch))
    cl = np.float32((c - ch) - cm)
    exact = (x.astype(np.float64) * p.astype(np.float64)).sum(1) - float(c)
    n = x.shape[0]
    cterm = np.tile(np.array([-ch, -cm, -cl], dtype=np.float64), (n, 1))
    terms = np.concatenate([xh.astype(np.float64) * ph, xh.astype(np.float64) * pm,
                            xl.astype(np.float64) * ph, cterm], axis=1)
    s32 = fp32_sequential_sum(terms)
    err = np.abs(s32 - exact)
    # the dropped terms (Xh.Pl, Xl.Pm, Xl.Pl and x - (Xh + Xl)) and FP32 accumulation
    assert err.max() <= 2e-5
    assert err.max() < BAND / 2
