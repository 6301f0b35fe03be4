"""The multi-process path of bench.py on CPU: two gloo ranks, each timing
its own replica; the job's time is the slowest rank's and its throughput the
units of all ranks over that time (replicas exchange no data)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [12.5, 40.0, 7.0][rank]
    dist.barrier()
    t = bench.max_over_ranks(local_ms, dist, "cpu")
    out[rank] = (t, bench.whole_job_rate(20, world, t / 1000.0))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_max_over_ranks_and_whole_job_rate(world):
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
    slowest = max([12.5, 40.0, 7.0][:world])
    for r in range(world):
        t, v = res[r]
        assert t == slowest
        assert v == pytest.approx(world * 20 / (slowest / 1000.0))


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
    assert bench.whole_job_rate(10, 1, 0.5) == 20.0
