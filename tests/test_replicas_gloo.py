"""The multi-process path of bench.py on CPU ranks (gloo, world size 2): the
barrier, the max over ranks of the timed region and the whole-job rate.  The
time stepper is not sharded across GPUs (replicas only), so these helpers are
the whole N > 1 path."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    bench.barrier(world)
    seconds = 1.0 + rank  # rank 1 is the slowest replica
    t = bench.max_over_ranks(world, seconds)
    rate = bench.whole_job_rate(20, world, t)
    q.put((rank, t, rate))
    bench.barrier(world)
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_time_and_the_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2.0, 2.0]
    assert [o[2] for o in out] == [20.0, 20.0]  # 2 x 20 steps over 2 s
