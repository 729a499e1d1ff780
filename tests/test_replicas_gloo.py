"""Multi-process replica timing on CPU (gloo, world size 2).

The build does not shard: N GPUs run N independent replicas of the same
workload (weak scaling) and the slowest rank's time decides the whole-job
throughput.  This checks that reduction with two gloo ranks on the host."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 180.0][rank]
    q.put((rank,) + bench.replica_throughput(local_ms, 10, 8000, world, "cpu"))
    dist.destroy_process_group()


def test_replica_throughput_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    positions = 8000 * 8001 / 2
    for rank, max_ms, value in out:
        assert max_ms == 180.0
        assert value == pytest.approx(2 * 10 * positions / 0.180, rel=1e-12)


def test_replica_throughput_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    max_ms, value = bench.replica_throughput(50.0, 4, 100, 1, "cpu")
    assert max_ms == 50.0
    assert value == pytest.approx(4 * 5050 / 0.05)


def test_reference_arm_other_ranks_do_no_work(capsys):
    sys.path.insert(0, ROOT)
    import argparse

    import bench
    args = argparse.Namespace(config="c2", warmup=3, steps=2, gpus=2)
    assert bench.run_reference(args, 1, 2) is None
    assert capsys.readouterr().out == ""
