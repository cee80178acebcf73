"""The N>1 path of the benchmark is N independent replicas (the candidates of a
poll are independent problems): no data-path collective, the job time is the
slowest rank's, and the whole-job rate counts every rank's work.  Checked with
two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # rank r "took" 1 + r seconds for its replica of 1000 units
        t = bench.max_over_ranks_of(1.0 + rank, world, "cpu")
        out[rank] = (t, bench.replica_throughput(1000.0, t, world))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (2.0, 1000.0)


def test_one_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks_of(3.5, 1, "cpu") == 3.5
    assert bench.replica_throughput(10.0, 2.0, 1) == 5.0
