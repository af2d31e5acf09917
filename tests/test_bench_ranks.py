"""The N > 1 path of bench.py (independent replicas, one per rank): the time
is the maximum over ranks and the value aggregates every rank's cells.
Checked with two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank  # the second replica is slower
    m = bench.max_over_ranks(ms, dist, device="cpu")
    out[rank] = (m, bench.aggregate_rate(1000, 4, m, world))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_time_is_max_over_ranks_and_value_aggregates():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        m, v = res[r]
        assert m == 15.0
        assert v == pytest.approx(world * 1000 * 4 / 15e-3)


def test_single_process_is_unchanged():
    assert bench.max_over_ranks(3.5) == 3.5
