"""The benchmark's multi-rank host logic on CPU: two gloo ranks, each with
its own independent replica (no data-path collective), take the slowest
rank's time and report whole-job throughput from rank 0."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_setup() == (world, rank, rank)
        bench.rank_barrier(dist, cuda=False)
        seconds = 1.0 + rank                     # rank 1 is the slowest
        slowest = bench.ranks_max(dist, seconds)
        rate = bench.job_rate(world, 1000.0, slowest)
        bench.rank_barrier(dist, cuda=False)
        out[rank] = (slowest, rate)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    assert out[0] == out[1] == (2.0, 1000.0)


def test_single_rank_needs_no_process_group():
    assert bench.ranks_max(None, 3.5) == 3.5
    assert bench.job_rate(1, 10.0, 2.0) == pytest.approx(5.0)


def test_bench_helpers_run_without_a_gpu():
    """The pieces of bench.py that need no GPU: the kernel-source hash that
    keys recorded ncu traffic, and the measured-peak lookup."""
    h = bench.kernel_hash()
    assert len(h) == 12 and int(h, 16) >= 0
    peak, kind = bench.load_peaks()
    assert peak > 0 and kind in ("measured", "fallback")
