"""FP64 CPU oracle (ctypes wrapper over oracle.c) -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package. The CUDA library never calls it, and it shares
no code with the CUDA library.

Every function follows a passage of "Faster Mean-shift" (Zhao et al.):
Eq. 1/9 cosine, Eq. 6-8 and 11 the flat-kernel update, Algorithm 2 the
seed/shift/prune/cluster loop, Eq. 14 and 19 the OSOP probability and
seed bound, Sec. 3.2.3-3.2.4 early stopping and the N schedule.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (OpenMP when gcc has it)."""
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler found for the oracle")
    tmp = _SO + f".tmp{os.getpid()}"
    base = [cc, "-std=c11", "-O3", "-ffp-contract=off", "-fPIC", "-shared", src, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:4] + ["-fopenmp"] + base[4:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    """The loaded oracle. MS_ORACLE_SO overrides the library path; the mutation
    tests use it to load deliberately broken copies of the oracle."""
    global _lib
    if _lib is None:
        path = os.environ.get("MS_ORACLE_SO") or build()
        _lib = _bind(ctypes.CDLL(path))
    return _lib


P_d = ctypes.POINTER(ctypes.c_double)
P_f = ctypes.POINTER(ctypes.c_float)
P_i64 = ctypes.POINTER(ctypes.c_int64)
P_i32 = ctypes.POINTER(ctypes.c_int32)
P_u8 = ctypes.POINTER(ctypes.c_uint8)
P_u64 = ctypes.POINTER(ctypes.c_uint64)


class OrConfig(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32), ("bandwidth_cos", ctypes.c_double), ("tol", ctypes.c_double),
        ("max_iter", ctypes.c_int32), ("gamma", ctypes.c_double), ("n_initial", ctypes.c_int32),
        ("L", ctypes.c_double), ("H", ctypes.c_double), ("P_target", ctypes.c_double),
        ("alpha", ctypes.c_double), ("merge_cos", ctypes.c_double), ("seed", ctypes.c_uint64),
        ("frame_id", ctypes.c_uint64), ("max_rounds", ctypes.c_int32), ("all_seeds", ctypes.c_int32),
    ]


class OrStats(ctypes.Structure):
    _fields_ = [
        ("rounds", ctypes.c_int32), ("n_modes", ctypes.c_int32), ("iters_total", ctypes.c_int32),
        ("pad_", ctypes.c_int32), ("seeds", ctypes.c_int64), ("seed_iters", ctypes.c_int64),
        ("candidates", ctypes.c_int64), ("dropped", ctypes.c_int64),
        ("min_window_margin", ctypes.c_double), ("min_cover_margin", ctypes.c_double),
        ("min_merge_margin", ctypes.c_double), ("n_carry", ctypes.c_int64),
    ]


def _bind(L):
    sig = {
        "or_splitmix64_next": (ctypes.c_uint64, [P_u64]),
        "or_perm_params": (None, [ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64, P_i64, P_i64]),
        "or_perm_at": (ctypes.c_int64, [ctypes.c_int64] * 4),
        "or_normalize": (ctypes.c_int64, [P_f, P_u8, ctypes.c_int64, ctypes.c_int32, P_d, P_d, P_i64]),
        "or_cos": (ctypes.c_double, [P_d, ctypes.c_double, P_d, ctypes.c_double, ctypes.c_int32]),
        "or_shift_step": (ctypes.c_int64, [P_d, P_d, ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                           P_d, P_d, P_d]),
        "or_trajectory": (ctypes.c_int32, [P_d, P_d, ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int32, P_d, P_d, P_i64]),
        "or_shift_round": (ctypes.c_int32, [P_d, P_d, ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_int32, ctypes.c_double, P_d,
                                            ctypes.c_int32, P_u8, P_i64, P_i32, P_i64, P_d]),
        "or_merge": (ctypes.c_int32, [P_d, P_i64, P_i64, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                      P_d, ctypes.c_int32, ctypes.c_int32, P_i32, P_d]),
        "or_cover": (ctypes.c_int64, [P_d, P_d, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, P_d,
                                      ctypes.c_int32, ctypes.c_int32, P_u8, P_d]),
        "or_nmin": (ctypes.c_double, [ctypes.c_double] * 3),
        "or_p_all_seeded": (ctypes.c_double, [ctypes.c_double] * 3),
        "or_next_n": (ctypes.c_int64, [ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_int64]),
        "or_label": (None, [P_d, P_d, P_i64, ctypes.c_int64, ctypes.c_int32, P_d, ctypes.c_int32,
                            ctypes.c_int64, P_i32, P_d]),
        "or_run": (ctypes.c_int32, [ctypes.POINTER(OrConfig), P_f, P_u8, ctypes.c_int64, P_i32, P_d,
                                    ctypes.c_int32, P_i32, P_i64, P_d, P_i64, P_i64,
                                    ctypes.POINTER(OrStats)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def _p(a, t):
    if a is None:
        return None
    return a.ctypes.data_as(t)


DEFAULTS = dict(dim=16, bandwidth_cos=0.9, tol=1e-6, max_iter=300, gamma=0.9, n_initial=128,
                L=2.0, H=8.0, P_target=0.99, alpha=1.0, merge_cos=0.9, seed=0, frame_id=0,
                max_rounds=100000, all_seeds=0)


def make_config(**kw) -> OrConfig:
    cfg = dict(DEFAULTS)
    unknown = set(kw) - set(cfg)
    if unknown:
        raise KeyError(f"unknown oracle config keys {sorted(unknown)}")
    cfg.update(kw)
    return OrConfig(**cfg)


# ---------------------------------------------------------------- primitives
def splitmix64(state: int, count: int = 1):
    """Outputs of SplitMix64 starting from `state`."""
    st = ctypes.c_uint64(state)
    return [lib().or_splitmix64_next(ctypes.byref(st)) for _ in range(count)]


def perm_params(n: int, seed: int = 0, frame_id: int = 0):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    lib().or_perm_params(n, seed, frame_id, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def perm(n: int, seed: int = 0, frame_id: int = 0) -> np.ndarray:
    a, b = perm_params(n, seed, frame_id)
    return np.array([lib().or_perm_at(j, n, a, b) for j in range(n)], dtype=np.int64)


def normalize(emb: np.ndarray, mask=None):
    """(P [n,d] float64, pnorm [n], idx [n]) of the compacted, normalised foreground."""
    emb = np.ascontiguousarray(emb, dtype=np.float32)
    npix, d = emb.shape
    mask = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    P = np.empty((npix, d)); pn = np.empty(npix); idx = np.empty(npix, dtype=np.int64)
    n = lib().or_normalize(_p(emb, P_f), _p(mask, P_u8), npix, d, _p(P, P_d), _p(pn, P_d), _p(idx, P_i64))
    if n < 0:
        raise ValueError("invalid embedding (zero or non-finite norm)")
    return P[:n].copy(), pn[:n].copy(), idx[:n].copy()


def cos(a, b) -> float:
    a = np.ascontiguousarray(a, dtype=np.float64); b = np.ascontiguousarray(b, dtype=np.float64)
    return lib().or_cos(_p(a, P_d), float(np.sqrt(a @ a)), _p(b, P_d), float(np.sqrt(b @ b)), a.size)


def shift_step(P, pn, x, c=0.9):
    P = np.ascontiguousarray(P, dtype=np.float64); pn = np.ascontiguousarray(pn, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64); xn = x.copy()
    mm = ctypes.c_double(np.inf)
    cnt = lib().or_shift_step(_p(P, P_d), _p(pn, P_d), P.shape[0], P.shape[1], c, _p(x, P_d),
                              _p(xn, P_d), ctypes.byref(mm))
    return xn, int(cnt), mm.value


def trajectory(P, pn, x0, c=0.9, tol=1e-6, max_iter=300):
    P = np.ascontiguousarray(P, dtype=np.float64); pn = np.ascontiguousarray(pn, dtype=np.float64)
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    d = P.shape[1]
    traj = np.zeros((max_iter + 1, d)); counts = np.zeros(max_iter, dtype=np.int64)
    T = lib().or_trajectory(_p(P, P_d), _p(pn, P_d), P.shape[0], d, c, tol, max_iter, _p(x0, P_d),
                            _p(traj, P_d), _p(counts, P_i64))
    t = abs(T)
    return traj[: t + 1].copy(), counts[:t].copy(), T


def shift_round(P, pn, X0, c=0.9, tol=1e-6, max_iter=300, gamma=0.9):
    P = np.ascontiguousarray(P, dtype=np.float64); pn = np.ascontiguousarray(pn, dtype=np.float64)
    X = np.ascontiguousarray(X0, dtype=np.float64).copy()
    m = X.shape[0]
    state = np.zeros(m, dtype=np.uint8); sup = np.zeros(m, dtype=np.int64)
    it = np.zeros(m, dtype=np.int32); si = ctypes.c_int64(0); mm = ctypes.c_double(np.inf)
    sweeps = lib().or_shift_round(_p(P, P_d), _p(pn, P_d), P.shape[0], P.shape[1], c, tol, max_iter,
                                  gamma, _p(X, P_d), m, _p(state, P_u8), _p(sup, P_i64),
                                  _p(it, P_i32), ctypes.byref(si), ctypes.byref(mm))
    return dict(X=X, state=state, support=sup, conv_iter=it, sweeps=sweeps, seed_iters=si.value,
                min_margin=mm.value)


def merge(cand, support, order, merge_cos=0.9, kept=None):
    cand = np.ascontiguousarray(cand, dtype=np.float64)
    k, d = cand.shape
    n0 = 0 if kept is None else kept.shape[0]
    buf = np.zeros((n0 + k, d))
    if n0:
        buf[:n0] = kept
    src = np.zeros(max(k, 1), dtype=np.int32)
    mm = ctypes.c_double(np.inf)
    sup = np.ascontiguousarray(support, dtype=np.int64); ordr = np.ascontiguousarray(order, dtype=np.int64)
    nk = lib().or_merge(_p(cand, P_d), _p(sup, P_i64), _p(ordr, P_i64), k, d, merge_cos, _p(buf, P_d),
                        n0, n0 + k, _p(src, P_i32), ctypes.byref(mm))
    if nk < 0:
        raise RuntimeError(f"or_merge failed: {nk}")
    return buf[:nk].copy(), src[: nk - n0].copy(), mm.value


def cover(P, pn, modes, covered, c=0.9, k0=0, k1=None):
    P = np.ascontiguousarray(P, dtype=np.float64); pn = np.ascontiguousarray(pn, dtype=np.float64)
    modes = np.ascontiguousarray(modes, dtype=np.float64)
    k1 = modes.shape[0] if k1 is None else k1
    cov = np.ascontiguousarray(covered, dtype=np.uint8).copy()
    mm = ctypes.c_double(np.inf)
    left = lib().or_cover(_p(P, P_d), _p(pn, P_d), P.shape[0], P.shape[1], c, _p(modes, P_d), k0, k1,
                          _p(cov, P_u8), ctypes.byref(mm))
    return cov, int(left), mm.value


def nmin(I, r=1.0, P=0.99) -> float:
    return lib().or_nmin(float(I), float(r), float(P))


def p_all_seeded(N, I, r=1.0) -> float:
    return lib().or_p_all_seeded(float(N), float(I), float(r))


def next_n(N, I, uncovered, r=1.0, P=0.99, L=2.0, H=8.0) -> int:
    return int(lib().or_next_n(int(N), int(I), float(r), float(P), float(L), float(H), int(uncovered)))


def label(P, pn, idx, modes, n_pixels):
    P = np.ascontiguousarray(P, dtype=np.float64); pn = np.ascontiguousarray(pn, dtype=np.float64)
    idx = np.ascontiguousarray(idx, dtype=np.int64); modes = np.ascontiguousarray(modes, dtype=np.float64)
    labels = np.empty(n_pixels, dtype=np.int32); margin = np.empty(max(P.shape[0], 1))
    lib().or_label(_p(P, P_d), _p(pn, P_d), _p(idx, P_i64), P.shape[0], P.shape[1], _p(modes, P_d),
                   modes.shape[0], n_pixels, _p(labels, P_i32), _p(margin, P_d))
    return labels, margin[: P.shape[0]].copy()


@dataclass
class OracleResult:
    labels: np.ndarray        # int32 [n_pixels], -1 background
    modes: np.ndarray         # float64 [K, d] in keep order
    support: np.ndarray       # int64 [K]
    label_margin: np.ndarray  # float64 [n_pixels] top1 - top2 (NaN background)
    round_log: np.ndarray     # int64 [rounds, 4]: N requested, seeds drawn, modes kept, uncovered
    seed_log: np.ndarray      # int64 [seeds]: foreground index of each seed in draw order
    stats: dict


def run(emb: np.ndarray, mask=None, **cfg) -> OracleResult:
    """The whole method on one frame (Algorithm 2 driven by OSOP)."""
    emb = np.ascontiguousarray(emb, dtype=np.float32)
    npix, d = emb.shape
    cfg.setdefault("dim", d)
    c = make_config(**cfg)
    mask = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    n_fg = npix if mask is None else int(np.count_nonzero(mask))
    cap = max(n_fg, 1)
    labels = np.empty(npix, dtype=np.int32)
    modes = np.empty((cap, d)); sup = np.empty(cap, dtype=np.int64); marg = np.empty(max(npix, 1))
    max_rounds = min(c.max_rounds, max(n_fg, 1) + 1)
    c.max_rounds = max_rounds
    rlog = np.zeros((max_rounds, 4), dtype=np.int64)
    slog = np.zeros(max(n_fg, 1), dtype=np.int64)
    nm = ctypes.c_int32(0); st = OrStats()
    rc = lib().or_run(ctypes.byref(c), _p(emb, P_f), _p(mask, P_u8), npix, _p(labels, P_i32),
                      _p(modes, P_d), cap, ctypes.byref(nm), _p(sup, P_i64), _p(marg, P_d),
                      _p(rlog, P_i64), _p(slog, P_i64), ctypes.byref(st))
    if rc != 0:
        raise RuntimeError(f"or_run failed with {rc}")
    k = nm.value
    stats = {f: getattr(st, f) for f, _ in OrStats._fields_ if f != "pad_"}
    return OracleResult(labels=labels, modes=modes[:k].copy(), support=sup[:k].copy(),
                        label_margin=marg[:npix].copy(), round_log=rlog[: st.rounds].copy(),
                        seed_log=slog[: st.seeds].copy(), stats=stats)
