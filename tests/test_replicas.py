"""The N > 1 path of bench.py (independent replicas, one process per GPU) on CPU:
two gloo ranks with different step times agree on the slowest rank's time, and the
whole-job throughput counts every rank's units."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
    out[rank] = (t, bench.replica_throughput(6_000_000, world, 4, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        assert out[0] == out[1]
        t, value = out[0]
        assert t == 15.0
        assert value == pytest.approx(6e6 * 2 * 4 / 15e-3 / 1e6)


def test_single_rank_is_unchanged():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.replica_throughput(1000, 1, 10, 2.0) == pytest.approx(1000 * 10 / 2e-3 / 1e6)
