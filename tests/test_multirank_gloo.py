"""The N > 1 path of bench.py on CPU: two gloo ranks (independent replicas,
weak scaling) agree on the whole-job time, the maximum over ranks, and on
the job's seconds per trajectory; the replicas draw different seeds."""
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
    import bench

    ms = 100.0 * (rank + 1)  # rank 1 is the slow one
    total, value = bench.job_time(ms, 5, dist, "cpu")
    seed = bench.WL["seed"] + rank
    gathered = [None] * world
    dist.all_gather_object(gathered, seed)
    out[rank] = (total, value, len(set(gathered)))
    dist.destroy_process_group()


def test_job_time_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        total, value, nseeds = res[r]
        assert total == 200.0
        assert abs(value - 200.0 / 1e3 / (5 * world)) < 1e-15
        assert nseeds == world


def test_job_time_single_rank():
    import bench

    total, value = bench.job_time(300.0, 3)
    assert total == 300.0 and abs(value - 0.1) < 1e-15
