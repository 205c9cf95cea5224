"""Failure paths, made to happen on the host or by a device-side limit that
runs out (no GPU fault, trap or hang):

- the batched graph's loop guard (ms_config.batch_max_passes) set below what a
  frame needs: the run must stop with MS_ERR_TIMEOUT, the graph returning
  normally, and the CUDA context must stay usable;
- a workspace allocation that fails (ms_inject_alloc_failure makes the next
  one return MS_ERR_OOM without calling cudaMalloc): the create call must
  report MS_ERR_OOM, leave nothing allocated, and the next create must work.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_batch_pass_limit_reports_timeout_and_context_survives(ms_lib):
    import torch
    f = synth.frame_c1(seed=0)
    e = torch.from_numpy(f.emb).cuda()
    c = ms_lib.ms_config_default(dim=16, precision=ms_lib.MS_FP32, batch_max_passes=2)
    b = ms_lib.ms_batch_create(c, [e], [None])
    try:
        with pytest.raises(ms_lib.MsError) as err:
            ms_lib.ms_batch_run(b)
        assert err.value.status == ms_lib.MS_ERR_TIMEOUT
        assert ms_lib.ms_batch_stats(b, -1)["reserved0"] == 2  # passes run before the guard stopped it
    finally:
        b.close()
    # the context is intact: the same frame clusters normally afterwards
    ref = oracle.run(f.emb)
    c = ms_lib.ms_config_default(dim=16, precision=ms_lib.MS_FP32)
    b = ms_lib.ms_batch_create(c, [e], [None])
    try:
        ms_lib.ms_batch_run(b)
        assert ms_lib.ms_batch_modes(b, 0).shape[0] == ref.modes.shape[0]
        assert np.array_equal(b.labels[0].cpu().numpy(), ref.labels)
    finally:
        b.close()


def test_injected_allocation_failure_reports_oom_and_leaks_nothing(ms_lib):
    import torch
    f = synth.frame_c1_separable(seed=0)
    e = torch.from_numpy(f.emb).cuda()
    cfg = ms_lib.ms_config_default(dim=16, precision=ms_lib.MS_BF16)
    # the binding allocates the batch's label buffers through torch's caching
    # allocator before the library runs: warm that cache so they come from it
    tmp = torch.empty(f.emb.shape[0], dtype=torch.int32, device="cuda")
    del tmp
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    ms_lib.ms_inject_alloc_failure(2)
    try:
        with pytest.raises(ms_lib.MsError) as err:
            ms_lib.ms_create(cfg, e, None)
        assert err.value.status == ms_lib.MS_ERR_OOM
        with pytest.raises(ms_lib.MsError) as err:
            ms_lib.ms_batch_create(cfg, [e], [None])
        assert err.value.status == ms_lib.MS_ERR_OOM
    finally:
        ms_lib.ms_inject_alloc_failure(0)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    # the hook is spent: the next create allocates and runs
    res = ms_lib.cluster(e, None, precision=ms_lib.MS_BF16)
    assert np.array_equal(res.labels.cpu().numpy(), oracle.run(f.emb).labels)
