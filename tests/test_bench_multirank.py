"""Host logic of bench.py's N-GPU run on CPU ranks (gloo, world size 2).

The PIC path does not shard on one box (one GPU per box), so N GPUs run N
independent replicas: each rank draws its own seed, the slowest rank's time
sets the job time (max over ranks), the value is every rank's particles over
that time, and only rank 0 prints; the reference arm runs on rank 0 alone.
"""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # the max over ranks is what every rank sees
        t = bench._barrier_max(world, 1.0 + rank)
        bench._barrier(world)
        wl = bench.replica_workload("thermal2d_64", rank, world)
        # the reference arm prints on rank 0 only; other ranks do no work
        buf = io.StringIO()
        if rank != 0:
            with redirect_stdout(buf):
                bench.run_reference(type("A", (), {"workload": "thermal2d_64", "steps": 1, "warmup": 0})(), rank, world)
        out.put((rank, t, wl.seed, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_and_max_time():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, s0, o0), (r1, t1, s1, o1) = res
    assert t0 == t1 == 2.0          # max of 1.0 and 2.0 on both ranks
    assert s0 != s1                 # independent replicas
    assert o1 == ""                 # rank 1 prints nothing in the reference arm


def test_aggregate_rate_counts_every_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_rate(4, 1000, 10, 2.0) == 4 * 1000 * 10 / 2.0
    assert bench.replica_workload("thermal2d_64", 0, 1).seed == bench.replica_workload("thermal2d_64", 3, 1).seed
