"""bench.py --gpus N runs N independent replicas (no data-path collective): rank r
uses seed + r, and the whole-job figures are the slowest rank's time and the sum
of the edges.  Exercised here with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, _ = bench.dist_env()
        elapsed, edges = bench.combine_ranks(10.0 + 5.0 * rank, 1000 * (rank + 1), w, "cpu")
        out.put((r, w, bench.replica_seed(3, r), elapsed, edges))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_combine():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[0] for g in got] == [0, 1] and all(g[1] == 2 for g in got)
    assert [g[2] for g in got] == [3, 4]  # distinct seeds, one graph per replica
    assert all(g[3] == 15.0 for g in got)  # slowest rank's time on every rank
    assert all(g[4] == 3000 for g in got)  # edges summed over the replicas


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(7.5, 42, 1, "cpu") == (7.5, 42)
