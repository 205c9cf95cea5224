"""Host logic of the multi-GPU form (replicas: each rank clusters its own
frames, no collective on the data path) on two gloo ranks on the CPU: the
barrier, the max and sum over ranks, the whole-job rate (units of all ranks
over the slowest rank's time), disjoint frame shards, and the reference arm
doing no work on ranks other than 0."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        bench.barrier(ws)
        assert bench.reduce_over_ranks(float(rank), ws, "max") == ws - 1
        assert bench.reduce_over_ranks(float(rank + 1), ws, "sum") == ws * (ws + 1) / 2
        # rank r processed 10 (r + 1) frames in 1 + r seconds
        rate, t = bench.whole_job_rate(10 * (rank + 1), 1.0 + rank, ws)
        assert t == ws and rate == 10 * ws * (ws + 1) / 2 / ws
        shards = [None] * ws
        dist.all_gather_object(shards, bench.frame_seeds(rank, 64))
        seen = [s for shard in shards for s in shard]
        assert len(seen) == len(set(seen)) == 64 * ws
        if rank != 0:
            assert bench.run_reference(None, rank) is None   # returns before touching its arguments
        bench.barrier(ws)
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_replicas_host_logic_two_gloo_ranks():
    mp.spawn(_rank, args=(2, _free_port()), nprocs=2, join=True)


def test_world_size_one_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    assert bench.reduce_over_ranks(3.5, 1, "max") == 3.5
    assert bench.whole_job_rate(64, 0.5, 1) == (128.0, 0.5)
    bench.barrier(1)


def test_frame_shards_stay_disjoint_or_refuse():
    sys.path.insert(0, ROOT)
    import bench
    seeds = [s for r in range(8) for s in bench.frame_seeds(r, 1000)]
    assert len(seeds) == len(set(seeds))
    with pytest.raises(ValueError):
        bench.frame_seeds(0, 1001)
