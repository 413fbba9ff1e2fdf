"""The bench's multi-rank logic (independent replicas, job time = slowest rank) on two gloo ranks on the CPU."""
import os
import socket
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    sys.path.insert(0, ROOT)
    import bench
    from paper_2405_12913_gb300.configs import COSMO_1024 as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank  # rank 1 is the slower replica
        job_ms = bench.max_over_ranks(ms, world, "cpu")
        out.put((rank, bench.replica_seed(W, rank), job_ms, bench.replica_rate(8, job_ms, world)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_distinct_seeds():
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
    (r0, s0, t0, v0), (r1, s1, t1, v1) = res
    assert s0 != s1
    assert t0 == t1 == 150.0
    assert v0 == v1 == 2 * 8 / 0.150
