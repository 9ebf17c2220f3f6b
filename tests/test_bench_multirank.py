"""The benchmark's multi-process path on the CPU: two gloo ranks, launched as
torchrun would (RANK / WORLD_SIZE / MASTER_* in the environment). Replicas
only: every rank solves its own system; the job time is the slowest rank's,
the job's throughput counts every rank's unknowns, and the reference arm runs
on rank 0 alone."""
import contextlib
import io
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import argparse

    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier()
    ms = bench.max_over_ranks(10.0 + 5.0 * rank)
    value = bench.job_value(1000, world, ms)
    out = ""
    if rank != 0:
        # the reference arm: ranks other than 0 return at once, without output
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            bench.run_reference(argparse.Namespace(workload="C1", warmup=0, steps=1))
        out = buf.getvalue()
    bench.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, value, out))


def test_two_gloo_ranks_report_the_slowest_rank():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(2))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]           # max over ranks
    assert res[0][2] == res[1][2] == 1000 * 2 / 0.015    # both ranks' unknowns / job time
    assert res[1][3] == ""                               # rank 1 ran no reference work
