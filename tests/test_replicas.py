"""The multi-rank path of bench.py on CPU: two gloo ranks on 127.0.0.1, each
timing its own replica; the reported time is the slowest rank's, every rank
builds the same seeded workload, and one rank alone skips the group."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench
    from paper_1703_01325_gb300.reservoir import reservoir_system
    dist, w, r, local = bench.replica_group("gloo")
    ms = bench.max_over_ranks(10.0 + 5.0 * r, dist)  # rank 1 is the slower replica
    S = reservoir_system(4, 3, 2, 3, seed=9)  # each replica builds the same workload
    q.put((r, w, ms, float(S.vals.sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_replica():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[2] == 15.0 for o in out)
    assert out[0][3] == out[1][3]


def test_single_rank_has_no_group(monkeypatch):
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    dist, w, r, local = bench.replica_group("gloo")
    assert dist is None and (w, r) == (1, 0)
    assert bench.max_over_ranks(3.5, None) == 3.5
