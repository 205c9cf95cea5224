"""The seeded input generators that the oracle tests, the GPU tests and the
bench share (no GPU): the 512x512 frame holds exactly the foreground count the
bench's flop count assumes, for the seeds every rank draws; embeddings have
the stated norms; the same seed gives the same arrays; the smooth-kernel
problem has its stated shapes and unit vectors."""
import sys
import os

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("seed", [0, 63, 1000, 7063])   # first and last frame of ranks 0 and 7
def test_c2_frame_matches_the_bench_workload(seed):
    f = synth.frame_c2(seed=seed)
    assert f.emb.shape == (512 * 512, bench.DIM) and f.emb.dtype == np.float32
    fg = f.mask.astype(bool)
    assert int(fg.sum()) == bench.N_FG == 131072
    nrm = np.linalg.norm(f.emb[fg], axis=1)
    assert nrm.min() >= 0.5 * (1 - 1e-6) and nrm.max() <= 2.0 * (1 + 1e-6)
    # 60 cells and the outlier class
    assert np.unique(f.truth[fg]).size == 61


def test_generators_are_deterministic():
    a, b = synth.frame_c2(seed=5), synth.frame_c2(seed=5)
    assert np.array_equal(a.emb, b.emb) and np.array_equal(a.mask, b.mask)
    c = synth.frame_c2(seed=6)
    assert not np.array_equal(a.emb, c.emb)
    p, q = synth.vmf_problem_c5(seed=2, N=512, M=32, K=4), synth.vmf_problem_c5(seed=2, N=512, M=32, K=4)
    assert all(np.array_equal(p[k], q[k]) for k in p)


def test_vmf_problem_shapes_and_unit_vectors():
    p = synth.vmf_problem_c5(seed=0, N=2048, M=64, K=8)
    assert p["P"].shape == (2048, 16) and p["X0"].shape == (64, 16) and p["target"].shape == (64, 16)
    for k in ("P", "X0", "target"):
        assert np.abs(np.linalg.norm(p[k].astype(np.float64), axis=1) - 1.0).max() <= 1e-6
    # the seeds start on pixels
    assert np.array_equal(p["X0"], p["P"][p["seed_idx"]])
