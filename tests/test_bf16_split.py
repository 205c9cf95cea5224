"""The BF16 tensor-core form re-decides near-boundary pairs against the
pixel's FP32 value rebuilt from its three BF16 parts (h, m, l) in shared
memory. That relies on two facts about round-to-nearest-even BF16 splitting
of an FP32 value p, checked here with an independent numpy emulation:
  1. l = RN_bf16((p - h) - m) loses nothing: l == (p - h) - m exactly;
  2. the rebuild (h + m) + l, evaluated in FP32, returns p bit for bit.
(p - h has at most 17 significant bits, (p - h) - m at most 8.) Both hold
while the residuals stay above BF16's subnormal range, i.e. for |p| >= 2^-100;
the library stores smaller normalised components as 0 (flush_tiny)."""
import numpy as np


def bf16_rn(x):
    """FP32 -> nearest BF16 (ties to even), returned as FP32."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def _split_and_rebuild(p):
    p = np.asarray(p, dtype=np.float32)
    h = bf16_rn(p)
    r1 = (p - h).astype(np.float32)
    m = bf16_rn(r1)
    r2 = (r1 - m).astype(np.float32)
    l = bf16_rn(r2)
    rebuilt = ((h + m).astype(np.float32) + l).astype(np.float32)
    return r2, l, rebuilt


def _cases():
    rng = np.random.default_rng(0)
    u = rng.uniform(-1, 1, 2_000_000).astype(np.float32)
    g = rng.standard_normal((200_000, 16)).astype(np.float32)
    g = (g / np.linalg.norm(g, axis=1, keepdims=True)).astype(np.float32).ravel()
    e = np.arange(-126, 1, dtype=np.float64)
    pw = (2.0 ** e).astype(np.float32)
    near = np.concatenate([np.nextafter(pw, np.float32(0)), pw, np.nextafter(pw, np.float32(2))])
    tiny = np.array([2.0 ** -100, -(2.0 ** -99), 1e-29, 0.0, -0.0], dtype=np.float32)
    # every FP32 bit pattern whose top bits are those of values in [0.5, 1)
    dense = (np.uint32(0x3F000000) + np.arange(0, 1 << 23, 7, dtype=np.uint32)).view(np.float32)
    p = np.concatenate([u, g, near, -near, tiny, dense, -dense])
    return p[(np.abs(p) >= 2.0 ** -100) | (p == 0)]


def test_bf16_emulation_rounds_to_nearest_even():
    # BF16 keeps 7 fraction bits: 1 + 2^-7 is exact, 1 + 2^-8 ties to even
    # (1), 1 + 3*2^-8 ties to even (1 + 2^-6), 1 + 3*2^-9 rounds up to 1 + 2^-7
    x = np.array([1.0078125, 1.00390625, 1.01171875, 1.005859375, -1.00390625], dtype=np.float32)
    assert bf16_rn(x).tolist() == [1.0078125, 1.0, 1.015625, 1.0078125, -1.0]


def test_third_term_is_exact():
    r2, l, _ = _split_and_rebuild(_cases())
    assert np.array_equal(r2, l)


def test_rebuild_is_bit_exact():
    p = _cases()
    _, _, rebuilt = _split_and_rebuild(p)
    nz = p != 0
    assert np.array_equal(rebuilt[nz].view(np.uint32), p[nz].view(np.uint32))
    assert np.array_equal(rebuilt[~nz], p[~nz])
