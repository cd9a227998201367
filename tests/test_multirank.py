"""Host logic of the multi-GPU bench path on CPU: two gloo ranks, each with
its own replica, combine to whole-job throughput (time = max over ranks,
units = sum over ranks)."""
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
    ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
    units = 1.0e9 * (rank + 1)
    t, u = bench.combine_ranks(ms, units, dist, "cpu")
    out[rank] = (t, u)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_to_whole_job_figures():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        t, u = out[r]
        assert t == 150.0 and u == 3.0e9


def test_single_rank_is_identity():
    import bench
    assert bench.combine_ranks(12.5, 7.0, None) == (12.5, 7.0)

