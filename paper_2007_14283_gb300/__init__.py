"""Python binding of libms, cosine mean-shift with OSOP on one GPU (sm_103a).

The functions below carry the names of the C ABI in include/ms.h and only
marshal arguments: tensors become device pointers, the current torch stream
becomes the library's stream. Every step of the method runs in libms's CUDA
kernels; there is no Python or CPU fallback. If libms.so has not been built
the first call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libms.so")

MS_OK, MS_ERR_INVALID_ARG, MS_ERR_CUDA, MS_ERR_OOM = 0, 1, 2, 3
MS_ERR_NOT_CONVERGED, MS_ERR_STATE, MS_ERR_TIMEOUT = 4, 5, 6
MS_FLAT, MS_VMF = 0, 1
MS_FP32, MS_BF16 = 0, 1
MS_DIST_COSINE, MS_DIST_EUCLID = 0, 1
MS_PROFILE_FLAT, MS_PROFILE_EPANECHNIKOV, MS_PROFILE_GAUSSIAN = 0, 1, 2
MS_INSPECT_SEED_LOG, MS_INSPECT_MODES, MS_INSPECT_SUPPORT = 1, 2, 3
MS_INSPECT_COVERED, MS_INSPECT_ROUND_LOG, MS_INSPECT_PIXELS = 4, 5, 6

_STATUS = {0: "MS_OK", 1: "MS_ERR_INVALID_ARG", 2: "MS_ERR_CUDA", 3: "MS_ERR_OOM",
           4: "MS_ERR_NOT_CONVERGED", 5: "MS_ERR_STATE", 6: "MS_ERR_TIMEOUT"}


class MsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class ms_config(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32), ("kernel", ctypes.c_int32), ("bandwidth_cos", ctypes.c_double),
        ("kappa", ctypes.c_double), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
        ("n_initial", ctypes.c_int32), ("gamma", ctypes.c_double), ("L", ctypes.c_double),
        ("H", ctypes.c_double), ("P_target", ctypes.c_double), ("alpha", ctypes.c_double),
        ("merge_cos", ctypes.c_double), ("seed", ctypes.c_uint64), ("frame_id", ctypes.c_uint64),
        ("precision", ctypes.c_int32), ("max_rounds", ctypes.c_int32), ("eps_band", ctypes.c_double),
        ("all_seeds", ctypes.c_int32), ("batch_split", ctypes.c_int32), ("batch_max_passes", ctypes.c_int32),
        ("video_restart", ctypes.c_int32), ("tc_shape", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3),
    ]


class ms_stats(ctypes.Structure):
    _fields_ = [
        ("rounds", ctypes.c_int32), ("n_modes", ctypes.c_int32), ("iters_total", ctypes.c_int32),
        ("reserved0", ctypes.c_int32), ("n_fg", ctypes.c_int64), ("seeds", ctypes.c_int64),
        ("seed_iters", ctypes.c_int64), ("candidates", ctypes.c_int64), ("dropped", ctypes.c_int64),
        ("band_pairs", ctypes.c_int64), ("uncovered", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64),
        ("launches", ctypes.c_int64), ("shift_launches", ctypes.c_int64), ("shift_ms", ctypes.c_double),
    ]


class ms_tune_result(ctypes.Structure):
    _fields_ = [("batch_split", ctypes.c_int32), ("target_mult", ctypes.c_int32), ("tc_shape", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("ms", ctypes.c_double)]


_lib = None
_vp = ctypes.c_void_p
_i32, _i64 = ctypes.c_int32, ctypes.c_int64
_pi32, _pi64 = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)

_SIGNATURES = {
    "ms_config_default": (None, [ctypes.POINTER(ms_config)]),
    "ms_last_error": (ctypes.c_char_p, []),
    "ms_workspace_bytes": (_i32, [ctypes.POINTER(ms_config), _i64, _pi64]),
    "ms_create": (_i32, [ctypes.POINTER(ms_config), _vp, _vp, _i64, _vp, ctypes.POINTER(_vp)]),
    "ms_seed_batch": (_i32, [_vp, _i32, _pi32]),
    "ms_iterate": (_i32, [_vp, _i32, _pi32, _pi32]),
    "ms_merge_modes": (_i32, [_vp, _pi32, _pi64]),
    "ms_label": (_i32, [_vp, _vp, _vp, _i32, _pi32]),
    "ms_destroy": (None, [_vp]),
    "ms_run": (_i32, [_vp, _vp, _vp, _i32, _pi32]),
    "ms_stats_get": (_i32, [_vp, ctypes.POINTER(ms_stats)]),
    "ms_get_state": (_i32, [_vp, _pi64]),
    "ms_set_state": (_i32, [_vp, _i64]),
    "ms_inspect": (_i32, [_vp, _i32, _vp, _i64, _pi64]),
    "ms_profile": (_i32, [_vp, _i32]),
    "ms_tc_selftest": (_i32, [_vp, _vp, _i32, ctypes.c_double, _vp, _vp]),
    "ms_window_sums_static": (_i32, [_vp, _i32, _vp, _i32, ctypes.c_double, _vp, _vp]),
    "ms_vmf_forward": (_i32, [_vp, _i64, _vp, _i32, _i32, ctypes.c_double, _i32, _vp, _vp]),
    "ms_vmf_backward": (_i32, [_vp, _i64, _vp, _i32, _i32, ctypes.c_double, _i32, _vp, _vp, _vp, _vp]),
    "ms_vmf_forward_ex": (_i32, [_vp, _i64, _vp, _i32, _i32, ctypes.c_double, _i32, _i32, _vp, _vp]),
    "ms_vmf_backward_ex": (_i32, [_vp, _i64, _vp, _i32, _i32, ctypes.c_double, _i32, _i32, _vp, _vp, _vp, _vp]),
    "ms_run_host": (_i32, [ctypes.POINTER(ms_config), _vp, _vp, _i64, _vp, _vp, _vp, _i32, _pi32,
                           ctypes.POINTER(ms_stats)]),
    "ms_batch_create": (_i32, [ctypes.POINTER(ms_config), _i32, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                               _pi64, ctypes.POINTER(_vp), _vp, ctypes.POINTER(_vp)]),
    "ms_batch_run": (_i32, [_vp, _i32]),
    "ms_batch_run_host": (_i32, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp)]),
    "ms_batch_stats": (_i32, [_vp, _i32, ctypes.POINTER(ms_stats)]),
    "ms_batch_profile": (_i32, [_vp, _i32]),
    "ms_batch_phase_ms": (_i32, [_vp, ctypes.POINTER(ctypes.c_double), _i32, _pi32]),
    "ms_batch_run_eager": (_i32, [_vp, _i32]),
    "ms_batch_configure": (_i32, [_vp, _i32, _i32, _i32]),
    "ms_batch_autotune": (_i32, [_vp, _i32, ctypes.POINTER(ms_tune_result), _i32, _pi32]),
    "ms_batch_modes": (_i32, [_vp, _i32, _vp, _i32, _pi32]),
    "ms_batch_destroy": (None, [_vp]),
    "ms_inject_alloc_failure": (None, [_i32]),
    "ms_video_create": (_i32, [ctypes.POINTER(ms_config), _i64, _vp, ctypes.POINTER(_vp)]),
    "ms_video_run": (_i32, [_vp, _i32, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _pi64, ctypes.POINTER(_vp),
                            _pi64, _pi32]),
    "ms_video_state": (_i32, [_vp, _pi64, _pi64]),
    "ms_video_stats": (_i32, [_vp, _i32, ctypes.POINTER(ms_stats)]),
    "ms_video_destroy": (None, [_vp]),
    "ms_kernel_shift": (_i32, [_vp, _i64, _vp, _i32, _i32, _i32, _i32, ctypes.c_double, _i32, _vp, _vp, _vp]),
}


def load(path: Optional[str] = None):
    """Load libms.so (built in-tree by __graft_entry__.build()). Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libms.so is not built ({p}); run __graft_entry__.build() first")
    lib = ctypes.CDLL(p)
    for name, (res, args) in _SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != MS_OK:
        raise MsError(status, load().ms_last_error().decode())


def _stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t, dtype, what):
    import torch
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{what} must be a contiguous CUDA tensor of {dtype}")
    return ctypes.c_void_p(t.data_ptr())


# ------------------------------------------------------------------ C ABI
def ms_config_default(**overrides) -> ms_config:
    cfg = ms_config()
    load().ms_config_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        if not hasattr(cfg, k):
            raise KeyError(k)
        setattr(cfg, k, v)
    return cfg


def ms_inject_alloc_failure(count: int) -> None:
    """Testing hook: the next `count` workspace allocations fail with MS_ERR_OOM."""
    load().ms_inject_alloc_failure(int(count))


def ms_last_error() -> str:
    return load().ms_last_error().decode()


def ms_workspace_bytes(cfg: ms_config, n_pixels: int) -> int:
    out = ctypes.c_int64()
    _check(load().ms_workspace_bytes(ctypes.byref(cfg), n_pixels, ctypes.byref(out)))
    return out.value


class Context:
    """Owns an ms_ctx and keeps the borrowed input tensors alive."""

    def __init__(self, handle, emb, mask):
        self.handle = handle
        self._keep = (emb, mask)

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "handle", None):
            load().ms_destroy(self.handle)
            self.handle = None


def ms_create(cfg: ms_config, emb, mask=None, stream=None) -> Context:
    """emb: CUDA float32 [n_pixels, dim]; mask: CUDA uint8 [n_pixels] or None."""
    import torch
    n_pixels = emb.shape[0] if emb.dim() == 2 else 0
    h = ctypes.c_void_p()
    _check(load().ms_create(ctypes.byref(cfg), _dptr(emb, torch.float32, "emb"),
                            _dptr(mask, torch.uint8, "mask"), n_pixels, _stream_handle(stream),
                            ctypes.byref(h)))
    return Context(h, emb, mask)


def ms_seed_batch(ctx: Context, n_requested: int = 0) -> int:
    m = ctypes.c_int32()
    _check(load().ms_seed_batch(ctx.handle, n_requested, ctypes.byref(m)))
    return m.value


def ms_iterate(ctx: Context, max_iter: int = 0):
    """(n_converged, n_iters); MS_ERR_NOT_CONVERGED raises MsError."""
    c, it = ctypes.c_int32(), ctypes.c_int32()
    _check(load().ms_iterate(ctx.handle, max_iter, ctypes.byref(c), ctypes.byref(it)))
    return c.value, it.value


def ms_merge_modes(ctx: Context):
    """(n_modes, n_uncovered)."""
    k, u = ctypes.c_int32(), ctypes.c_int64()
    _check(load().ms_merge_modes(ctx.handle, ctypes.byref(k), ctypes.byref(u)))
    return k.value, u.value


def ms_label(ctx: Context, labels, modes=None) -> int:
    import torch
    k = ctypes.c_int32()
    cap = modes.shape[0] if modes is not None else 0
    _check(load().ms_label(ctx.handle, _dptr(labels, torch.int32, "labels"),
                           _dptr(modes, torch.float32, "modes"), cap, ctypes.byref(k)))
    return k.value


def ms_run(ctx: Context, labels, modes=None) -> int:
    import torch
    k = ctypes.c_int32()
    cap = modes.shape[0] if modes is not None else 0
    _check(load().ms_run(ctx.handle, _dptr(labels, torch.int32, "labels"),
                         _dptr(modes, torch.float32, "modes"), cap, ctypes.byref(k)))
    return k.value


def ms_destroy(ctx: Context):
    ctx.close()


def ms_stats_get(ctx: Context) -> dict:
    st = ms_stats()
    _check(load().ms_stats_get(ctx.handle, ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in ms_stats._fields_ if not f.startswith("reserved")}


def ms_profile(ctx: Context, enable: bool = True):
    _check(load().ms_profile(ctx.handle, 1 if enable else 0))


def ms_run_host(cfg: ms_config, emb, mask, labels, modes=None, stream=None):
    """Whole method on host (ideally pinned) tensors: emb float32 [n, d],
    mask uint8 [n] or None, labels int32 [n] written in place, modes float32
    [cap, d] or None. Returns (n_modes, stats dict)."""
    import torch

    def hp(t, dtype, what):
        if t is None:
            return None
        if t.is_cuda or t.dtype != dtype or not t.is_contiguous():
            raise ValueError(f"{what} must be a contiguous host tensor of {dtype}")
        return ctypes.c_void_p(t.data_ptr())
    k = ctypes.c_int32()
    st = ms_stats()
    cap = modes.shape[0] if modes is not None else 0
    _check(load().ms_run_host(ctypes.byref(cfg), hp(emb, torch.float32, "emb"), hp(mask, torch.uint8, "mask"),
                              emb.shape[0], _stream_handle(stream), hp(labels, torch.int32, "labels"),
                              hp(modes, torch.float32, "modes"), cap, ctypes.byref(k), ctypes.byref(st)))
    return k.value, {f: getattr(st, f) for f, _ in ms_stats._fields_ if not f.startswith("reserved")}


def ms_tc_selftest(X, P, c: float = 0.9):
    """Run the BF16 tensor-core tile once: X CUDA float32 [128, 16] seeds, P
    CUDA float32 [n_pix, 16] pixels. Returns (S [128, n_pad] float32 numpy,
    acc [128, 17] int64 numpy)."""
    import numpy as np
    import torch
    n = P.shape[0]
    n_pad = (n + 127) // 128 * 128
    S = np.zeros((128, n_pad), dtype=np.float32)
    acc = np.zeros((128, 17), dtype=np.int64)
    _check(load().ms_tc_selftest(_dptr(X, torch.float32, "X"), _dptr(P, torch.float32, "P"), n, c,
                                 S.ctypes.data_as(ctypes.c_void_p), acc.ctypes.data_as(ctypes.c_void_p)))
    return S, acc


def ms_window_sums_static(X, P, acc_out, c: float = 0.9, stream=None):
    """Window sums and sizes without device allocation (see ms.h): X CUDA
    float32 [m, 16], P CUDA float32 [n, 16], acc_out CUDA int64 [m, 17] written
    in place. Asynchronous on the stream."""
    import torch
    _check(load().ms_window_sums_static(_dptr(X, torch.float32, "X"), X.shape[0], _dptr(P, torch.float32, "P"),
                                        P.shape[0], c, _dptr(acc_out, torch.int64, "acc_out"),
                                        _stream_handle(stream)))


def ms_kernel_shift(P, X0, distance: int, profile: int, h: float, T: int, stream=None):
    """T dense mean-shift steps with the given distance (MS_DIST_*) and kernel
    profile (MS_PROFILE_*). P CUDA float32 [N, dim], X0 [M, dim]. Returns
    (x_T [M, dim], counts [M] of nonzero weights in the last step)."""
    import torch
    XT = torch.empty_like(X0)
    counts = torch.empty(X0.shape[0], dtype=torch.int32, device=X0.device)
    _check(load().ms_kernel_shift(_dptr(P, torch.float32, "P"), P.shape[0], _dptr(X0, torch.float32, "X0"),
                                  X0.shape[0], X0.shape[1], int(distance), int(profile), float(h), int(T),
                                  _dptr(XT, torch.float32, "XT"), _dptr(counts, torch.int32, "counts"),
                                  _stream_handle(stream)))
    return XT, counts


def ms_vmf_forward(P, X0, kappa: float, T: int, stream=None, precision: int = MS_FP32):
    """x_T of T smooth-kernel steps. P CUDA float32 [N, 16], X0 [M, 16].
    precision MS_BF16 runs the steps on the tensor cores."""
    import torch
    XT = torch.empty_like(X0)
    _check(load().ms_vmf_forward_ex(_dptr(P, torch.float32, "P"), P.shape[0], _dptr(X0, torch.float32, "X0"),
                                    X0.shape[0], X0.shape[1], float(kappa), int(T), int(precision),
                                    _dptr(XT, torch.float32, "XT"), _stream_handle(stream)))
    return XT


def ms_vmf_backward(P, X0, kappa: float, T: int, GT, stream=None, precision: int = MS_FP32):
    """(dL/dP, dL/dX0) for upstream gradient GT = dL/dx_T (the iterates are
    recomputed and the adjoint passes run in `precision`)."""
    import torch
    dP = torch.empty_like(P)
    dX0 = torch.empty_like(X0)
    _check(load().ms_vmf_backward_ex(_dptr(P, torch.float32, "P"), P.shape[0], _dptr(X0, torch.float32, "X0"),
                                     X0.shape[0], X0.shape[1], float(kappa), int(T), int(precision),
                                     _dptr(GT.contiguous(), torch.float32, "GT"), _dptr(dP, torch.float32, "dP"),
                                     _dptr(dX0, torch.float32, "dX0"), _stream_handle(stream)))
    return dP, dX0


def ms_vmf_forward_ex(P, X0, kappa: float, T: int, precision: int, stream=None):
    return ms_vmf_forward(P, X0, kappa, T, stream, precision)


def ms_vmf_backward_ex(P, X0, kappa: float, T: int, precision: int, GT, stream=None):
    return ms_vmf_backward(P, X0, kappa, T, GT, stream, precision)


def ms_get_state(ctx: Context) -> int:
    v = ctypes.c_int64()
    _check(load().ms_get_state(ctx.handle, ctypes.byref(v)))
    return v.value


def ms_set_state(ctx: Context, n_next: int):
    _check(load().ms_set_state(ctx.handle, n_next))


def ms_inspect(ctx: Context, what: int, dim: int = 16):
    """A copy of an internal array as a numpy array (see MS_INSPECT_* in ms.h)."""
    import numpy as np
    dtype, width = {MS_INSPECT_SEED_LOG: (np.int32, 1), MS_INSPECT_MODES: (np.float32, dim),
                    MS_INSPECT_SUPPORT: (np.int32, 1), MS_INSPECT_COVERED: (np.uint8, 1),
                    MS_INSPECT_ROUND_LOG: (np.int64, 4), MS_INSPECT_PIXELS: (np.float32, dim)}[what]
    cnt = ctypes.c_int64()
    _check(load().ms_inspect(ctx.handle, what, None, 0, ctypes.byref(cnt)))
    out = np.zeros((cnt.value, width), dtype=dtype)
    if cnt.value:
        _check(load().ms_inspect(ctx.handle, what, out.ctypes.data_as(ctypes.c_void_p), cnt.value,
                                 ctypes.byref(cnt)))
    return out if width > 1 else out[:, 0]


class Batch:
    """Owns an ms_batch; keeps the borrowed embeddings, masks and label buffers alive."""

    def __init__(self, handle, embs, masks, labels, dim):
        self.handle = handle
        self.labels = labels
        self.dim = dim
        self._keep = (embs, masks)

    def __del__(self):
        self.close()

    def close(self):
        if getattr(self, "handle", None):
            load().ms_batch_destroy(self.handle)
            self.handle = None


class Video:
    """Owns an ms_video (two workspaces and a side stream)."""

    def __init__(self, handle):
        self.handle = handle

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def close(self):
        if getattr(self, "handle", None):
            load().ms_video_destroy(self.handle)
            self.handle = None


def ms_video_create(cfg: ms_config, max_pixels: int, stream=None) -> Video:
    h = ctypes.c_void_p()
    _check(load().ms_video_create(ctypes.byref(cfg), int(max_pixels), _stream_handle(stream), ctypes.byref(h)))
    return Video(h)


def ms_video_destroy(v: Video):
    v.close()


def ms_video_run(v: Video, embs, masks=None, labels=None):
    """Cluster the next frames of the video. embs: list of CUDA float32
    [n_t, dim]; masks: None or a list (entries may be None) of CUDA uint8
    [n_t]; labels: None (allocated here) or a list of CUDA int32 [n_t].
    Returns (labels, n_start per frame, mode count per frame)."""
    import torch
    T = len(embs)
    arr = _vp * max(T, 1)
    e = arr(*[_dptr(t, torch.float32, "emb") for t in embs])
    m = None if masks is None else arr(*[_dptr(t, torch.uint8, "mask") if t is not None else None for t in masks])
    if labels is None:
        labels = [torch.empty(t.shape[0], dtype=torch.int32, device=t.device) for t in embs]
    lab = arr(*[_dptr(t, torch.int32, "labels") for t in labels])
    n = (ctypes.c_int64 * max(T, 1))(*[int(t.shape[0]) for t in embs])
    n_start = (ctypes.c_int64 * max(T, 1))()
    n_modes = (ctypes.c_int32 * max(T, 1))()
    _check(load().ms_video_run(v.handle, T, e, m, n, lab, n_start, n_modes))
    return labels, [int(x) for x in n_start[:T]], [int(x) for x in n_modes[:T]]


def ms_video_state(v: Video):
    """(N the next frame starts from, frames clustered so far)."""
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(load().ms_video_state(v.handle, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def ms_video_stats(v: Video, which: int = 0) -> dict:
    st = ms_stats()
    _check(load().ms_video_stats(v.handle, int(which), ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in ms_stats._fields_ if not f.startswith("reserved")}


def ms_batch_create(cfg: ms_config, embs, masks=None, stream=None) -> Batch:
    """embs: list of CUDA float32 [n_pixels_f, dim]; masks: None or a list of
    CUDA uint8 [n_pixels_f] (entries may be None). Label buffers (CUDA int32
    [n_pixels_f]) are allocated here and exposed as Batch.labels."""
    import torch
    B = len(embs)
    ptr_arr = _vp * max(B, 1)
    e = ptr_arr(*[_dptr(t, torch.float32, "emb") for t in embs])
    m = None
    if masks is not None:
        m = ptr_arr(*[_dptr(t, torch.uint8, "mask") if t is not None else None for t in masks])
    labels = [torch.empty(t.shape[0], dtype=torch.int32, device=t.device) for t in embs]
    lab = ptr_arr(*[ctypes.c_void_p(t.data_ptr()) for t in labels])
    n = (ctypes.c_int64 * max(B, 1))(*[int(t.shape[0]) for t in embs])
    h = ctypes.c_void_p()
    _check(load().ms_batch_create(ctypes.byref(cfg), B, e, m, n, lab, _stream_handle(stream),
                                  ctypes.byref(h)))
    return Batch(h, list(embs), masks, labels, cfg.dim)


def ms_batch_run(b: Batch, sync: bool = True):
    _check(load().ms_batch_run(b.handle, 1 if sync else 0))


def ms_batch_run_host(b: Batch, h_embs, h_masks, h_labels):
    """Host tensors (CPU, ideally pinned): h_embs float32 [n_f, dim], h_masks
    uint8 [n_f] or None, h_labels int32 [n_f] (written)."""
    import torch

    def hp(t, dtype, what):
        if t is None:
            return None
        if t.is_cuda or t.dtype != dtype or not t.is_contiguous():
            raise ValueError(f"{what} must be a contiguous CPU tensor of {dtype}")
        return ctypes.c_void_p(t.data_ptr())
    B = len(h_embs)
    arr = _vp * max(B, 1)
    e = arr(*[hp(t, torch.float32, "emb") for t in h_embs])
    m = None if h_masks is None else arr(*[hp(t, torch.uint8, "mask") for t in h_masks])
    lab = arr(*[hp(t, torch.int32, "labels") for t in h_labels])
    _check(load().ms_batch_run_host(b.handle, e, m, lab))


def ms_batch_stats(b: Batch, frame: int = -1) -> dict:
    st = ms_stats()
    _check(load().ms_batch_stats(b.handle, frame, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in ms_stats._fields_}


def ms_batch_run_eager(b: Batch, passes: int):
    _check(load().ms_batch_run_eager(b.handle, passes))


def ms_batch_configure(b: Batch, batch_split: int, target_mult: int = 2, tc_shape: int = 0):
    _check(load().ms_batch_configure(b.handle, batch_split, target_mult, tc_shape))


def ms_batch_autotune(b: Batch, reps: int = 3) -> list:
    """Time the work-split candidates, then (BF16) the tile shapes on the best
    split, on the batch's frames and keep the fastest; returns
    [{batch_split, target_mult, tc_shape, ms}] in the order timed."""
    res = (ms_tune_result * 16)()
    n = ctypes.c_int32()
    _check(load().ms_batch_autotune(b.handle, reps, res, 16, ctypes.byref(n)))
    return [{"batch_split": r.batch_split, "target_mult": r.target_mult, "tc_shape": r.tc_shape, "ms": r.ms}
            for r in res[:n.value]]


def ms_batch_profile(b: Batch, enable=True):
    """enable: False/0 off, True/1 shift timers, 2 shift and phase timers."""
    _check(load().ms_batch_profile(b.handle, int(enable)))


MS_BATCH_PHASES = ("setup", "seed_plan", "shift", "finalize_check", "merge", "cover", "schedule", "label")


def ms_batch_phase_ms(b: Batch) -> dict:
    """Per-phase time of the last synchronised run (profiling level 2), ms."""
    out = (ctypes.c_double * len(MS_BATCH_PHASES))()
    n = ctypes.c_int32()
    _check(load().ms_batch_phase_ms(b.handle, out, len(MS_BATCH_PHASES), ctypes.byref(n)))
    return {k: out[i] for i, k in enumerate(MS_BATCH_PHASES)}


def ms_batch_modes(b: Batch, frame: int):
    """Frame `frame`'s kept modes as a numpy float32 [K, dim] array (last synchronised run)."""
    import numpy as np
    k = ctypes.c_int32()
    _check(load().ms_batch_modes(b.handle, frame, None, 0, ctypes.byref(k)))
    out = np.zeros((k.value, b.dim), dtype=np.float32)
    if k.value:
        _check(load().ms_batch_modes(b.handle, frame, out.ctypes.data_as(ctypes.c_void_p), k.value,
                                     ctypes.byref(k)))
    return out


def ms_batch_destroy(b: Batch):
    b.close()


# ------------------------------------------------------------ convenience
@dataclass
class Result:
    labels: "object"   # torch int32 [n_pixels] on the device, -1 background
    modes: "object"    # torch float32 [K, dim] on the device
    stats: dict


def cluster(emb, mask=None, stream=None, **cfg) -> Result:
    """Run the whole method on one frame already on the GPU."""
    import torch
    c = ms_config_default(dim=int(emb.shape[1]), **cfg)
    ctx = ms_create(c, emb, mask, stream)
    try:
        labels = torch.empty(emb.shape[0], dtype=torch.int32, device=emb.device)
        n_fg = emb.shape[0] if mask is None else None
        cap = n_fg if n_fg is not None else int(mask.sum().item())
        modes = torch.empty((max(cap, 1), emb.shape[1]), dtype=torch.float32, device=emb.device)
        k = ms_run(ctx, labels, modes)
        stats = ms_stats_get(ctx)
        stats["round_log"] = ms_inspect(ctx, MS_INSPECT_ROUND_LOG)
        stats["seed_log"] = ms_inspect(ctx, MS_INSPECT_SEED_LOG)
        stats["support"] = ms_inspect(ctx, MS_INSPECT_SUPPORT)
        return Result(labels=labels, modes=modes[:k], stats=stats)
    finally:
        ctx.close()
