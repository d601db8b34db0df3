"""Multi-rank host logic of the benchmark (replicas, one pair per rank), on CPU
with two gloo ranks: distinct phantoms per rank, the slowest rank's time and
the summed Gauss-Newton products define the whole-job throughput."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank                  # rank 1 is the slow one
        mv = 30 * (rank + 1)
        out = bench.aggregate_ranks(ms, mv, dist)
        q.put((rank, bench.replica_seed(rank), out))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_benchmark():
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
    seeds = {r[1] for r in res}
    assert len(seeds) == 2                        # a different phantom pair per rank
    for _, _, (ms_max, mv_total, value) in res:   # every rank sees the job totals
        assert ms_max == 150.0 and mv_total == 90.0
        assert value == pytest.approx(90.0 / 0.15)


def test_single_rank_aggregate_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(200.0, 30) == (200.0, 30.0, 150.0)
