"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This package draws inputs only: von Mises-Fisher embeddings laid out like
microscopy frames, masks and ground-truth cell ids. It holds none of the
mean-shift arithmetic, so the oracle and the CUDA path stay independent.
"""
from .vmf import (  # noqa: F401
    Frame,
    sample_vmf,
    uniform_sphere,
    make_frame,
    frame_c1,
    frame_c1_separable,
    frame_c2,
    stack_c3,
    batch_c4,
    video_sequence,
    overlap_discs,
    volume,
    vmf_problem_c5,
    orthogonal_blobs,
)
