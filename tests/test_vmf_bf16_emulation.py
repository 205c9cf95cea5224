"""The BF16 arithmetic of the smooth-kernel (vMF) tensor-core kernels, emulated
in numpy on the CPU and held to float64.

One forward step and one reverse step of x' = normalise(sum_i w_i p_i),
w_i = exp(kappa (x . p_i - 1)) (the vMF kernel of the paper's Sec. 3), are
rebuilt term by term in the form the kernels compute them:
- scores: three-term round-to-nearest BF16 splits of both operands and the six
  products hh, hm, mh, hl, mm, lh summed in FP32; in the adjoint the constant
  -kappa log2(e) enters the same accumulator as a split against ones;
- weights: w = 2^E (ex2.approx, modelled as a relative error of up to 2^-22),
  split into two BF16 terms;
- sums: the high weight term against three data terms, the low one against
  two, accumulated in FP32;
- pass A (seeds as rows): dL/dx = sum_i ds_i p_i with ds = w (kappa gy . p);
- pass B (pixels as rows): dL/dp = sum_m w gy_m + ds'_m V_m, with ds' =
  ln(2) w (gy . p) and V = kappa log2(e) x, so ds' V = ds x.
A step must stay within 2e-5 of the float64 step (forward: every component;
each gradient: relative norm); the GPU tests chain T = 10 steps to 1e-4. Two
plausible simplifications (dropping a low BF16 term) must miss that bar, so
the emulation is sharp enough to justify the terms the kernels keep.
"""
import numpy as np

import synth
from test_bf16_score_bounds import bf16_rn, split3 as _split3

LOG2E = 1.4426950408889634
BAR = 2e-5


def split3(v):
    return tuple(t.astype(np.float64) for t in _split3(v))


def split2(v):
    v = np.asarray(v, dtype=np.float32)
    h = bf16_rn(v)
    lo = bf16_rn((v - h).astype(np.float32))
    return h.astype(np.float64), lo.astype(np.float64)


def f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def scores(a, b, const=None):
    """[rows(a), rows(b)] FP32 scores from the six split products, plus the
    split constant when given. Each product's sum is taken in float64 and
    rounded once: the FP32 accumulation error of the kernels (2^-24 per
    addition, a few hundred additions) is far below the bar."""
    ah, am, al = split3(a)
    bh, bm, bl = split3(b)
    s = ah @ bh.T + ah @ bm.T + am @ bh.T + ah @ bl.T + am @ bm.T + al @ bh.T
    if const is not None:
        s = s + sum(split3(np.float32(const)))
    return f32(s)


def ex2(e, rng):
    """2^e with the approximate unit's relative error, up to 2^-22."""
    return f32(np.exp2(e) * (1.0 + rng.uniform(-1.0, 1.0, np.shape(e)) * 2.0 ** -22))


def problem(seed, N=3000, M=48):
    prob = synth.vmf_problem_c5(seed=seed, N=N, M=M, K=8)
    return prob["P"].astype(np.float32), prob["X0"].astype(np.float32)


def forward(P, X, kappa, rng, keep_wl=True):
    k2 = np.float32(kappa * LOG2E)
    E = scores((X * k2).astype(np.float32), P)
    w = ex2(f32(E - k2), rng)
    wh, wl = split2(w)
    ph, pm, pl = split3(P)
    Y = wh @ (ph + pm + pl) + (wl @ (ph + pm) if keep_wl else 0.0)
    Y = f32(Y)
    return Y / np.linalg.norm(Y, axis=1, keepdims=True)


def forward64(P, X, kappa):
    P64, X64 = P.astype(np.float64), X.astype(np.float64)
    Y = np.exp(kappa * (X64 @ P64.T - 1.0)) @ P64
    return Y / np.linalg.norm(Y, axis=1, keepdims=True)


def adjoint64(P, X, G, kappa):
    """Exact reverse pass of one float64 step: (dL/dx, dL/dp, gy, W, A)."""
    P64, X64 = P.astype(np.float64), X.astype(np.float64)
    W = np.exp(kappa * (X64 @ P64.T - 1.0))
    Y = W @ P64
    yn = np.linalg.norm(Y, axis=1, keepdims=True)
    xn = Y / yn
    gy = (G - xn * (xn * G).sum(1, keepdims=True)) / yn
    A = gy @ P64.T
    DS = kappa * W * A
    return DS @ P64, W.T @ gy + DS.T @ X64, gy, W, A


def adjoint(P, X, gy, kappa, rng, keep_dl_b=True):
    k2 = np.float32(kappa * LOG2E)
    gy32 = gy.astype(np.float32)
    V = (X * k2).astype(np.float32)
    w = ex2(scores(V, P, const=-k2), rng)                           # 2^(kappa log2(e) (x . p - 1))
    ph, pm, pl = split3(P)
    dh, dl = split2(f32(w * scores((np.float32(kappa) * gy32).astype(np.float32), P)))
    dX = f32(dh @ (ph + pm + pl) + dl @ (ph + pm))                  # pass A
    wh, wl = split2(w)
    d2h, d2l = split2(f32(np.log(2.0) * f32(w * scores(gy32, P))))
    gh, gm, gl = split3(gy32)
    vh, vm, vl = split3(V)
    dP = wh.T @ (gh + gm + gl) + wl.T @ (gh + gm) + d2h.T @ (vh + vm + vl)
    if keep_dl_b:
        dP = dP + d2l.T @ (vh + vm)
    return dX, f32(dP)                                              # pass B


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_forward_step_emulation():
    rng = np.random.default_rng(1)
    for seed, kappa in ((3, 20.0), (7, 60.0)):
        P, X = problem(seed)
        err = np.abs(forward(P, X, kappa, rng) - forward64(P, X, kappa)).max()
        assert err <= BAR, (seed, kappa, err)


def test_adjoint_step_emulation():
    rng = np.random.default_rng(2)
    for seed, kappa in ((4, 20.0), (8, 60.0)):
        P, X = problem(seed)
        G = np.random.default_rng(seed + 100).standard_normal(X.shape)
        dX_ref, dP_ref, gy, _, _ = adjoint64(P, X, G, kappa)
        dX, dP = adjoint(P, X, gy, kappa, rng)
        assert rel(dX, dX_ref) <= BAR, (seed, kappa, rel(dX, dX_ref))
        assert rel(dP, dP_ref) <= BAR, (seed, kappa, rel(dP, dP_ref))


def test_pass_b_rescaling_is_ds_x():
    """ln(2) w a against V = kappa log2(e) x equals ds x = kappa w a x, up to
    the FP32 rounding of kappa log2(e)."""
    P, X = problem(5)
    kappa = 20.0
    G = np.random.default_rng(6).standard_normal(X.shape)
    _, _, _, W, A = adjoint64(P, X, G, kappa)
    k2 = float(np.float32(kappa * LOG2E))
    lhs = (np.log(2.0) * W * A).T @ (k2 * X.astype(np.float64))
    rhs = (kappa * W * A).T @ X.astype(np.float64)
    assert rel(lhs, rhs) <= 2.0 ** -23


def test_dropping_the_low_weight_term_is_visible():
    P, X = problem(6)
    rng = np.random.default_rng(3)
    err = np.abs(forward(P, X, 20.0, rng, keep_wl=False) - forward64(P, X, 20.0)).max()
    assert err > BAR, err


def test_dropping_pass_b_low_term_is_visible():
    P, X = problem(9)
    kappa = 20.0
    G = np.random.default_rng(10).standard_normal(X.shape)
    _, dP_ref, gy, _, _ = adjoint64(P, X, G, kappa)
    _, dP = adjoint(P, X, gy, kappa, np.random.default_rng(4), keep_dl_b=False)
    assert rel(dP, dP_ref) > BAR, rel(dP, dP_ref)
