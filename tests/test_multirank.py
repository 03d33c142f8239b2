"""The benchmark's multi-rank bookkeeping on CPU with the gloo backend (world size 2): the
timed region's maximum over ranks and the whole-job throughput of independent replica sets."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 + 25.0 * rank          # rank 1 is the slow one
    m = bench.max_over_ranks(local_ms, world, device="cpu")
    out[rank] = (m, bench.job_throughput(20, world, m))
    dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_throughput():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (125.0, 2 * 20 / 0.125)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(7.5, 1) == 7.5
    assert bench.job_throughput(10, 1, 20.0) == 500.0
