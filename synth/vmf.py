"""Seeded von Mises-Fisher frames shaped like the paper's microscopy workloads.

Everything here is input generation: it draws embeddings, masks and
ground-truth cell ids. No mean-shift step is computed here.

* vMF sampling follows Wood (1994), "Simulation of the von Mises-Fisher
  distribution": draw the cosine w to the mean direction by rejection from a
  Beta proposal, then a uniform direction in the tangent space.
* A frame is an H x W grid. Each cell is an elliptical blob of an exact pixel
  count (log-normal sizes), carved from the free pixels nearest its centre.
  Cell pixels get that cell's vMF samples, outliers (scattered foreground
  pixels) get uniform-sphere vectors, background pixels are masked out.
* Embedding norms are scaled by U[0.5, 2] where stated, because a network's
  raw output is not unit length (the method normalises it, Eq. 9).

The frame shapes follow the paper's cohorts (512x512 DIC-C2DH-HeLa, Sec. 4.3)
and its simulation designs (Sec. 4.2). Datasets and trained embeddings are
not available, so these synthetic frames stand in for them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

__all__ = [
    "Frame", "sample_vmf", "uniform_sphere", "make_frame", "frame_c1",
    "frame_c1_separable", "frame_c2", "stack_c3", "batch_c4", "vmf_problem_c5",
    "orthogonal_blobs",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def uniform_sphere(rng: np.random.Generator, n: int, d: int) -> np.ndarray:
    """n directions uniform on S^(d-1), float64 [n, d]."""
    v = rng.standard_normal((n, d))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v


def sample_vmf(rng: np.random.Generator, mu: np.ndarray, kappa: float, n: int) -> np.ndarray:
    """n samples of vMF(mu, kappa) on S^(d-1) by Wood's (1994) rejection scheme.

    Returns float64 [n, d], unit rows.
    """
    mu = np.asarray(mu, dtype=np.float64)
    mu = mu / np.linalg.norm(mu)
    d = mu.shape[0]
    if n == 0:
        return np.zeros((0, d))
    if kappa <= 0.0:
        return uniform_sphere(rng, n, d)
    m1 = d - 1.0
    # b = (-2k + sqrt(4k^2 + (d-1)^2)) / (d-1), written in the cancellation-free form.
    b = m1 / (2.0 * kappa + math.sqrt(4.0 * kappa * kappa + m1 * m1))
    x0 = (1.0 - b) / (1.0 + b)
    c = kappa * x0 + m1 * math.log(1.0 - x0 * x0)
    w = np.empty(n)
    filled = 0
    while filled < n:
        m = 2 * (n - filled) + 16
        z = rng.beta(m1 / 2.0, m1 / 2.0, size=m)
        ww = (1.0 - (1.0 + b) * z) / (1.0 - (1.0 - b) * z)
        u = rng.uniform(size=m)
        ok = kappa * ww + m1 * np.log(1.0 - x0 * ww) - c >= np.log(u)
        take = ww[ok][: n - filled]
        w[filled:filled + take.size] = take
        filled += take.size
    v = rng.standard_normal((n, d))
    v -= (v @ mu)[:, None] * mu[None, :]
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return w[:, None] * mu[None, :] + np.sqrt(np.maximum(0.0, 1.0 - w * w))[:, None] * v


@dataclass
class Frame:
    """One synthetic frame.

    emb   : float32 [H*W, d], row-major pixels (not necessarily unit length)
    mask  : uint8 [H*W] (1 = foreground) or None when every pixel is foreground
    truth : int32 [H*W]; cell id >= 0, -1 background, -2 outlier
    means : float64 [K, d] cell mean directions; kappas : float64 [K]
    """
    emb: np.ndarray
    mask: Optional[np.ndarray]
    truth: np.ndarray
    means: np.ndarray
    kappas: np.ndarray
    H: int
    W: int
    info: dict = field(default_factory=dict)

    @property
    def n_pixels(self) -> int:
        return self.emb.shape[0]

    @property
    def dim(self) -> int:
        return self.emb.shape[1]

    @property
    def n_fg(self) -> int:
        return self.n_pixels if self.mask is None else int(self.mask.sum())


def _split_sizes(rng, total: int, k: int, median: float, sigma: float) -> np.ndarray:
    """k log-normal sizes rescaled to sum exactly to total (largest remainder)."""
    raw = np.exp(rng.normal(math.log(median), sigma, size=k))
    share = raw / raw.sum() * total
    base = np.floor(share).astype(np.int64)
    base = np.maximum(base, 1)
    rem = total - int(base.sum())
    if rem > 0:
        order = np.argsort(-(share - np.floor(share)), kind="stable")
        base[order[:rem]] += 1
    elif rem < 0:
        order = np.argsort(-base, kind="stable")
        i = 0
        while rem < 0:
            j = order[i % k]
            if base[j] > 1:
                base[j] -= 1
                rem += 1
            i += 1
    return base


def _carve_cells(rng, H: int, W: int, sizes: np.ndarray) -> np.ndarray:
    """Assign each cell its exact pixel count as an elliptical blob.

    Returns owner int32 [H*W] (-1 = free). Cells are placed largest first; each
    takes the free pixels nearest its centre in its own ellipse metric.
    """
    owner = np.full(H * W, -1, dtype=np.int32)
    yy_all, xx_all = np.divmod(np.arange(H * W), W)
    order = np.argsort(-sizes, kind="stable")
    for k in order:
        area = int(sizes[k])
        free = np.flatnonzero(owner < 0)
        if free.size < area:
            raise ValueError("frame too small for the requested cells")
        centre = free[rng.integers(free.size)]
        cy, cx = yy_all[centre], xx_all[centre]
        aspect = rng.uniform(1.0, 1.6)
        theta = rng.uniform(0.0, math.pi)
        r1 = math.sqrt(area * aspect / math.pi)
        r2 = math.sqrt(area / (aspect * math.pi))
        ct, st = math.cos(theta), math.sin(theta)
        R = int(math.ceil(2.0 * r1)) + 2
        while True:
            y0, y1 = max(0, cy - R), min(H, cy + R + 1)
            x0, x1 = max(0, cx - R), min(W, cx + R + 1)
            ys, xs = np.meshgrid(np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
            idx = (ys * W + xs).ravel()
            keep = owner[idx] < 0
            if keep.sum() >= area or (y0 == 0 and x0 == 0 and y1 == H and x1 == W):
                break
            R *= 2
        idx = idx[keep]
        dy = (idx // W - cy).astype(np.float64)
        dx = (idx % W - cx).astype(np.float64)
        u = (dx * ct + dy * st) / r1
        v = (-dx * st + dy * ct) / r2
        metric = u * u + v * v
        pick = idx[np.argsort(metric, kind="stable")[:area]]
        owner[pick] = k
    return owner


def make_frame(seed: int, H: int, W: int, d: int, n_fg: int, n_cells: int,
               size_median: float, size_sigma: float, kappa_lo: float,
               kappa_hi: float, outlier_frac: float, scale: Optional[tuple] = (0.5, 2.0),
               equal_sizes: bool = False) -> Frame:
    """A frame of n_fg foreground pixels: n_cells vMF cells plus outliers.

    The outlier count is floor(outlier_frac * n_fg); the cells share the rest.
    kappa per cell ~ U[kappa_lo, kappa_hi]; mean directions uniform on S^(d-1).
    When n_fg == H*W the mask is None (all foreground).
    """
    rng = _rng(seed)
    n_pix = H * W
    if not (0 < n_fg <= n_pix):
        raise ValueError("n_fg out of range")
    n_out = int(math.floor(outlier_frac * n_fg))
    n_cell_px = n_fg - n_out
    if equal_sizes:
        sizes = np.full(n_cells, n_cell_px // n_cells, dtype=np.int64)
        sizes[: n_cell_px - int(sizes.sum())] += 1
    else:
        sizes = _split_sizes(rng, n_cell_px, n_cells, size_median, size_sigma)
    owner = _carve_cells(rng, H, W, sizes)
    truth = owner.copy()
    if n_out > 0:
        free = np.flatnonzero(owner < 0)
        out_idx = rng.choice(free, size=n_out, replace=False)
        truth[out_idx] = -2
    means = uniform_sphere(rng, n_cells, d)
    kappas = rng.uniform(kappa_lo, kappa_hi, size=n_cells)
    emb = rng.standard_normal((n_pix, d))  # background: never clustered
    for k in range(n_cells):
        idx = np.flatnonzero(truth == k)
        emb[idx] = sample_vmf(rng, means[k], float(kappas[k]), idx.size)
    out_idx = np.flatnonzero(truth == -2)
    if out_idx.size:
        emb[out_idx] = uniform_sphere(rng, out_idx.size, d)
    fg = truth != -1
    if scale is not None:
        s = rng.uniform(scale[0], scale[1], size=n_pix)
        emb[fg] *= s[fg, None]
    mask = None if n_fg == n_pix else fg.astype(np.uint8)
    return Frame(emb=np.ascontiguousarray(emb, dtype=np.float32), mask=mask,
                 truth=truth.astype(np.int32), means=means, kappas=kappas, H=H, W=W,
                 info=dict(seed=seed, n_fg=n_fg, n_cells=n_cells, n_outliers=n_out))


def frame_c1(seed: int = 0, kappa: float = 50.0) -> Frame:
    """64x64 frame, every pixel foreground: 8 equal vMF clusters of 512 unit
    vectors, d = 16, one kappa for all cells."""
    return make_frame(seed, 64, 64, 16, 4096, 8, 512.0, 0.0, kappa, kappa, 0.0,
                      scale=None, equal_sizes=True)


def frame_c1_separable(seed: int = 0) -> Frame:
    """The 64x64 frame with kappa = 200, where each cluster fits one window."""
    return frame_c1(seed, kappa=200.0)


def frame_c2(seed: int = 0, d: int = 16) -> Frame:
    """512x512 frame with 131072 foreground pixels: 60 cells with log-normal
    sizes (median 2000 px, sigma 0.37) holding 98% of them, kappa ~ U[20, 200],
    and 2% uniform-sphere outliers; embedding norms ~ U[0.5, 2]."""
    return make_frame(seed, 512, 512, d, 131072, 60, 2000.0, 0.37, 20.0, 200.0, 0.02)


def _rotate_toward(mu: np.ndarray, tangent: np.ndarray, angle: float) -> np.ndarray:
    t = tangent - (tangent @ mu) * mu
    t /= np.linalg.norm(t)
    return math.cos(angle) * mu + math.sin(angle) * t


def stack_c3(seed: int = 0, d: int = 16, n_fg: int = 131072, H: int = 512, W: int = 512,
             n_cells: int = 60, drift: float = 0.02, split_frac: float = 0.05,
             split_angle: float = 0.5) -> Frame:
    """Three consecutive frames clustered as one set (tracking stack).

    Each cell's mean direction drifts by `drift` radians along a random tangent
    per frame. In the third frame split_frac of the cells split into two
    children at +/- split_angle along a random tangent. truth holds track ids:
    0..n_cells-1 for cells, n_cells.. for the children.
    """
    rng = _rng(seed)
    n_out = int(math.floor(0.02 * n_fg))
    sizes = _split_sizes(rng, n_fg - n_out, n_cells, 2000.0, 0.37)
    owner = _carve_cells(rng, H, W, sizes)
    means0 = uniform_sphere(rng, n_cells, d)
    kappas = rng.uniform(20.0, 200.0, size=n_cells)
    n_split = int(round(split_frac * n_cells))
    split_cells = rng.choice(n_cells, size=n_split, replace=False)
    embs, masks, truths = [], [], []
    means = means0.copy()
    child_means = []
    for f in range(3):
        if f > 0:
            for k in range(n_cells):
                means[k] = _rotate_toward(means[k], rng.standard_normal(d), drift)
        truth = owner.copy()
        free = np.flatnonzero(owner < 0)
        out_idx = rng.choice(free, size=n_out, replace=False)
        truth[out_idx] = -2
        emb = rng.standard_normal((H * W, d))
        for k in range(n_cells):
            idx = np.flatnonzero(owner == k)
            if f == 2 and k in split_cells:
                j = int(np.flatnonzero(split_cells == k)[0])
                tang = rng.standard_normal(d)
                ma = _rotate_toward(means[k], tang, split_angle)
                mb = _rotate_toward(means[k], -tang, split_angle)
                half = idx.size // 2
                emb[idx[:half]] = sample_vmf(rng, ma, float(kappas[k]), half)
                emb[idx[half:]] = sample_vmf(rng, mb, float(kappas[k]), idx.size - half)
                truth[idx[:half]] = n_cells + 2 * j
                truth[idx[half:]] = n_cells + 2 * j + 1
                child_means += [ma, mb]
            else:
                emb[idx] = sample_vmf(rng, means[k], float(kappas[k]), idx.size)
        emb[out_idx] = uniform_sphere(rng, n_out, d)
        fg = truth != -1
        s = rng.uniform(0.5, 2.0, size=H * W)
        emb[fg] *= s[fg, None]
        embs.append(emb)
        masks.append(fg.astype(np.uint8))
        truths.append(truth)
    all_means = np.concatenate([means, np.array(child_means).reshape(-1, d)], axis=0)
    return Frame(emb=np.ascontiguousarray(np.concatenate(embs), dtype=np.float32),
                 mask=np.concatenate(masks), truth=np.concatenate(truths).astype(np.int32),
                 means=all_means, kappas=kappas, H=3 * H, W=W,
                 info=dict(seed=seed, frames=3, split_cells=split_cells.tolist()))


def video_sequence(seed: int = 0, T: int = 8, d: int = 16, n_fg: int = 131072, H: int = 512, W: int = 512,
                   n_cells: int = 60, drift: float = 0.02, kappa_lo: float = 20.0,
                   kappa_hi: float = 200.0) -> List[Frame]:
    """T consecutive frames of one time-lapse sequence, each a Frame of its own:
    the cells keep their pixels and sizes (log-normal, median 0.98 n_fg /
    n_cells, sigma 0.37), their mean directions drift by `drift` radians along
    a random tangent per frame, every frame draws fresh vMF samples and 2%
    uniform outliers; embedding norms ~ U[0.5, 2]. truth holds cell ids (-2
    outliers, -1 background)."""
    rng = _rng(seed)
    n_out = int(math.floor(0.02 * n_fg))
    sizes = _split_sizes(rng, n_fg - n_out, n_cells, 0.98 * n_fg / n_cells, 0.37)
    owner = _carve_cells(rng, H, W, sizes)
    means = uniform_sphere(rng, n_cells, d)
    kappas = rng.uniform(kappa_lo, kappa_hi, size=n_cells)
    frames = []
    for f in range(T):
        if f > 0:
            for k in range(n_cells):
                means[k] = _rotate_toward(means[k], rng.standard_normal(d), drift)
        truth = owner.copy()
        out_idx = rng.choice(np.flatnonzero(owner < 0), size=n_out, replace=False)
        truth[out_idx] = -2
        emb = rng.standard_normal((H * W, d))
        for k in range(n_cells):
            idx = np.flatnonzero(owner == k)
            emb[idx] = sample_vmf(rng, means[k], float(kappas[k]), idx.size)
        emb[out_idx] = uniform_sphere(rng, n_out, d)
        fg = truth != -1
        sc = rng.uniform(0.5, 2.0, size=H * W)
        emb[fg] *= sc[fg, None]
        mask = None if n_fg == H * W else fg.astype(np.uint8)
        frames.append(Frame(emb=np.ascontiguousarray(emb, dtype=np.float32), mask=mask,
                            truth=truth.astype(np.int32), means=means.copy(), kappas=kappas, H=H, W=W,
                            info=dict(seed=seed, frame=f, n_fg=n_fg, n_cells=n_cells)))
    return frames


def overlap_discs(seed: int = 0, H: int = 1000, W: int = 1000, d: int = 18, n_discs: int = 8,
                  diameter: int = 250, overlap: float = 0.0) -> Frame:
    """The paper's overlap study (Appendix A): n_discs discs of the given
    diameter on an H x W canvas, their centres on a ring around the canvas
    centre, adjacent centres diameter * (1 - overlap) apart, so adjacent discs
    intersect over `overlap` of a diameter (a later disc owns the shared
    pixels). Disc k's pixels all hold the same unit vector +/- e_j, orthogonal
    or opposite to every other disc's; no noise. Background is masked."""
    rng = _rng(seed)
    if n_discs > 2 * d:
        raise ValueError("at most 2*d orthogonal/opposite directions")
    spacing = diameter * (1.0 - overlap)
    ring = spacing / (2.0 * math.sin(math.pi / n_discs))
    phase = rng.uniform(0.0, 2.0 * math.pi)
    yy, xx = np.divmod(np.arange(H * W), W)
    owner = np.full(H * W, -1, dtype=np.int32)
    for k in range(n_discs):
        cy = H / 2.0 + ring * math.sin(phase + 2.0 * math.pi * k / n_discs)
        cx = W / 2.0 + ring * math.cos(phase + 2.0 * math.pi * k / n_discs)
        owner[(yy - cy) ** 2 + (xx - cx) ** 2 <= (diameter / 2.0) ** 2] = k
    dirs = np.zeros((n_discs, d))
    for k in range(n_discs):
        dirs[k, k // 2] = 1.0 if k % 2 == 0 else -1.0
    emb = np.zeros((H * W, d))
    fg = owner >= 0
    emb[fg] = dirs[owner[fg]]
    emb[~fg] = rng.standard_normal((int((~fg).sum()), d))  # masked: never clustered
    return Frame(emb=np.ascontiguousarray(emb, dtype=np.float32), mask=fg.astype(np.uint8),
                 truth=owner, means=dirs, kappas=np.full(n_discs, np.inf), H=H, W=W,
                 info=dict(seed=seed, overlap=overlap, n_fg=int(fg.sum()), fg_fraction=float(fg.mean())))


def volume(seed: int = 0, D: int = 128, H: int = 256, W: int = 256, d: int = 16, n_cells: int = 400,
           fg_fraction: float = 0.5, kappa_lo: float = 20.0, kappa_hi: float = 200.0,
           outlier_frac: float = 0.02) -> Frame:
    """A 3D volume of D x H x W voxels (the paper's 2D-only limitation, Sec. 5.3,
    lifted): n_cells ellipsoidal vMF cells filling fg_fraction of the voxels,
    sizes log-normal (sigma 0.37), kappa ~ U[kappa_lo, kappa_hi], plus
    outlier_frac uniform-sphere voxels; norms ~ U[0.5, 2]. Voxels are listed in
    z-major order; truth as for frames."""
    rng = _rng(seed)
    n_vox = D * H * W
    n_fg = int(round(fg_fraction * n_vox))
    n_out = int(math.floor(outlier_frac * n_fg))
    sizes = _split_sizes(rng, n_fg - n_out, n_cells, (n_fg - n_out) / n_cells, 0.37)
    # each cell takes the free voxels nearest its centre in its own ellipsoid metric
    owner = np.full(n_vox, -1, dtype=np.int32)
    zz, rem = np.divmod(np.arange(n_vox), H * W)
    yy, xx = np.divmod(rem, W)
    for k in np.argsort(-sizes, kind="stable"):
        area = int(sizes[k])
        free = np.flatnonzero(owner < 0)
        c = free[rng.integers(free.size)]
        cz, cy, cx = zz[c], yy[c], xx[c]
        axes = rng.uniform(1.0, 1.6, size=3)
        axes /= axes.prod() ** (1.0 / 3.0)
        r = (3.0 * area / (4.0 * math.pi)) ** (1.0 / 3.0)
        R = int(math.ceil(2.0 * r * axes.max())) + 2
        while True:
            z0, z1 = max(0, cz - R), min(D, cz + R + 1)
            y0, y1 = max(0, cy - R), min(H, cy + R + 1)
            x0, x1 = max(0, cx - R), min(W, cx + R + 1)
            gz, gy, gx = np.meshgrid(np.arange(z0, z1), np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
            idx = (gz * H * W + gy * W + gx).ravel()
            keep = owner[idx] < 0
            if keep.sum() >= area or (z1 - z0 == D and y1 - y0 == H and x1 - x0 == W):
                break
            R *= 2
        idx = idx[keep]
        m = (((idx // (H * W) - cz) / axes[0]) ** 2 + (((idx // W) % H - cy) / axes[1]) ** 2
             + ((idx % W - cx) / axes[2]) ** 2)
        owner[idx[np.argsort(m, kind="stable")[:area]]] = k
    truth = owner.copy()
    out_idx = rng.choice(np.flatnonzero(owner < 0), size=n_out, replace=False)
    truth[out_idx] = -2
    means = uniform_sphere(rng, n_cells, d)
    kappas = rng.uniform(kappa_lo, kappa_hi, size=n_cells)
    emb = np.zeros((n_vox, d), dtype=np.float32)
    for k in range(n_cells):
        idx = np.flatnonzero(truth == k)
        emb[idx] = sample_vmf(rng, means[k], float(kappas[k]), idx.size)
    emb[out_idx] = uniform_sphere(rng, n_out, d)
    fg = truth != -1
    emb[~fg] = rng.standard_normal((int((~fg).sum()), d))
    emb[fg] *= rng.uniform(0.5, 2.0, size=int(fg.sum()))[:, None].astype(np.float32)
    return Frame(emb=np.ascontiguousarray(emb, dtype=np.float32), mask=fg.astype(np.uint8),
                 truth=truth.astype(np.int32), means=means, kappas=kappas, H=D * H, W=W,
                 info=dict(seed=seed, shape=(D, H, W), n_fg=int(fg.sum()), n_cells=n_cells))


def batch_c4(seed: int = 0, B: int = 64, d: int = 16, n_lo: int = 2000,
             n_hi: int = 260000) -> List[Frame]:
    """B frames of uneven foreground size, log-uniform in [n_lo, n_hi], with
    5..120 cells each (kappa ~ U[20, 200], 2% outliers). A frame is the
    smallest square (side a multiple of 16, at most 512) holding twice its
    foreground, or 512x512."""
    rng = _rng(seed)
    ns = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=B)).round().astype(np.int64)
    ks = rng.integers(5, 121, size=B)
    frames = []
    for f in range(B):
        n = int(ns[f])
        side = int(math.ceil(math.sqrt(2 * n) / 16.0)) * 16
        side = min(max(side, 16), 512)
        k = int(ks[f])
        median = 0.98 * n / k
        frames.append(make_frame(seed * 1000003 + f + 1, side, side, d, n, k, median, 0.37,
                                 20.0, 200.0, 0.02))
    return frames


def vmf_problem_c5(seed: int = 0, N: int = 65536, M: int = 1024, d: int = 16, K: int = 32):
    """Differentiable-form inputs: N unit pixels from K vMF cells
    (kappa ~ U[20, 200], equal sizes), M seeds drawn among the pixels, and each
    seed's target = its cell's mean direction.

    Returns dict(P float32 [N,d], X0 float32 [M,d], target float32 [M,d],
    seed_idx int64 [M], truth int32 [N]).
    """
    rng = _rng(seed)
    means = uniform_sphere(rng, K, d)
    kappas = rng.uniform(20.0, 200.0, size=K)
    truth = np.repeat(np.arange(K), int(math.ceil(N / K)))[:N]
    rng.shuffle(truth)
    P = np.empty((N, d))
    for k in range(K):
        idx = np.flatnonzero(truth == k)
        P[idx] = sample_vmf(rng, means[k], float(kappas[k]), idx.size)
    seed_idx = rng.choice(N, size=M, replace=False)
    X0 = P[seed_idx]
    target = means[truth[seed_idx]]
    return dict(P=np.ascontiguousarray(P, dtype=np.float32),
                X0=np.ascontiguousarray(X0, dtype=np.float32),
                target=np.ascontiguousarray(target, dtype=np.float32),
                seed_idx=seed_idx.astype(np.int64), truth=truth.astype(np.int32))


def orthogonal_blobs(seed: int, n: int, d: int = 18, K: int = 10, sigma: float = 0.01):
    """The paper's speed/memory simulation design (Sec. 4.2): K blob clusters in
    d dimensions whose centres are orthogonal or opposite (+/- e_j), with
    Gaussian noise of standard deviation sigma. Not normalised.

    Returns (emb float32 [n, d], truth int32 [n]).
    """
    if K > 2 * d:
        raise ValueError("at most 2*d orthogonal/opposite centres")
    rng = _rng(seed)
    centres = np.zeros((K, d))
    for k in range(K):
        centres[k, k // 2] = 1.0 if k % 2 == 0 else -1.0
    truth = np.arange(n) % K
    rng.shuffle(truth)
    emb = centres[truth] + sigma * rng.standard_normal((n, d))
    return np.ascontiguousarray(emb, dtype=np.float32), truth.astype(np.int32)
