"""Multi-GPU runs are independent replicas (one process per GPU, no
data-path collective): the bench's whole-job totals are the slowest rank's
time and the work summed over ranks.  Two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, work = bench.replica_totals(10.0 + 5.0 * rank, 100.0 * (rank + 1), dist, "cpu")
    out[rank] = (ms, work)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_max_time_and_summed_work():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == (15.0, 300.0) and out[1] == (15.0, 300.0)


def test_single_process_is_identity():
    import bench
    assert bench.replica_totals(3.0, 7.0, None, "cpu") == (3.0, 7.0)
