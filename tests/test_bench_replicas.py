"""The N > 1 path of bench.py on CPU: two gloo ranks on 127.0.0.1.

Each rank is an independent replica; the job's time is the slowest rank's
(max over ranks), its value counts every rank's cell updates, and the
reference arm does its work on rank 0 only.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 25.0 * rank  # the replicas' own times differ
        bench.barrier_sync(world, cuda=False)
        worst = bench.max_over_ranks(ms, world, device="cpu")
        val = bench.job_value(world, 16384 * 4000, 5, worst * 5)
        rc = bench.run_reference(type("A", (), {"steps": 1, "warmup": 0, "gpus": world})()) \
            if rank != 0 else 0
        out.put((rank, worst, val, rc))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(q.get(timeout=5) for _ in range(world))
    worst = 100.0 + 25.0 * (world - 1)
    for rank, w, val, rc in res:
        assert w == worst
        # 2 replicas x 16384 cells x 4000 steps x 5 runs over 5 x 125 ms
        assert val == pytest.approx(world * 16384 * 4000 * 5 / (worst * 5 * 1e-3))
        assert rc == 0
