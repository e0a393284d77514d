"""The multi-GPU path of bench.py runs independent replicas (one grid lives
on one GPU, so no rank exchanges data with another): every rank advances its own
grid, the job time is the slowest rank's, and the whole-job value counts the
units of every rank.  Exercised here with two gloo ranks on the CPU."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, _ = bench._dist()
    dt = bench.replica_time(1.0 + 0.5 * rank)  # rank 1 is the slow one
    value = bench.replica_value(ws, 1000, 10, dt)
    out.put((r, ws, dt, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_sum_the_units():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert all(r[2] == 1.5 for r in res)  # max over ranks
    assert all(abs(r[3] - 2 * 1000 * 10 / 1.5 / 1e6) < 1e-15 for r in res)


def test_single_process_time_is_its_own():
    import bench
    assert bench.replica_time(0.25) == 0.25
    assert bench.replica_value(1, 500, 4, 0.5) == 500 * 4 / 0.5 / 1e6
