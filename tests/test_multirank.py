"""The multi-rank plumbing of bench.py, on CPU with the gloo backend.

randUTV of one matrix has no data-parallel split without an exchange every
block step, so more GPUs run independent replicas (one matrix per rank): the
only cross-rank operations are the barrier around the timed region and the
maximum of the per-rank times.  These run here as two gloo ranks.
"""
import os
import socket

import pytest
import torch
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_setup(None)
    assert (w, r) == (world, rank)
    bench.barrier(w)
    t = bench.max_over_ranks(10.0 + rank, w)   # per-rank "times"
    out[rank] = t
    dist.destroy_process_group()


@pytest.mark.timeout(120) if hasattr(pytest.mark, "timeout") else (lambda f: f)
def test_two_gloo_ranks_barrier_and_max():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn",
                       join=True)
    assert dict(out) == {0: 11.0, 1: 11.0}


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    bench.barrier(1)   # no-op
    assert not torch.distributed.is_initialized()
