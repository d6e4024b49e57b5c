"""The N > 1 path of bench.py (replicas: one Jacobian per GPU, the step time is
the max over ranks), exercised with world_size 2 on the gloo backend."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench.dist_setup()
        step_ms = 10.0 + 5.0 * r                      # rank 1 is the slow one
        m = bench.max_over_ranks(step_ms)
        q.put((r, w, m, bench.job_seconds_per_solve(m, w), bench.replica_seeds(r, 5)))
    finally:
        dist.destroy_process_group()


def test_replica_timing_with_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert all(r[2] == 15.0 for r in res)                  # max over ranks on every rank
    assert all(abs(r[3] - 15.0 / 1e3 / 2) < 1e-15 for r in res)
    seeds = [set(r[4]) for r in res]
    assert not (seeds[0] & seeds[1]) and len(seeds[0]) == 5  # disjoint replicas


def test_single_rank_defaults(monkeypatch):
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_setup() == (1, 0, 0)
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.replica_seeds(0, 5) == [0, 1, 2, 3, 4]
