"""The benchmark's multi-rank logic on CPU with two gloo ranks: the whole-job
aggregate (maximum time, summed iterations), one distinct instance per rank,
and the reference arm running on rank 0 only."""
import argparse
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE="2", LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    import bench
    ws, r, _ = bench._dist()
    t, it = bench._aggregate(1.0 + rank, 100 * (rank + 1), ws)
    args = argparse.Namespace(workload="portfolio", n=200, k=5, limits=2, precision="fp64")
    prob, _ = bench._workload(args, r)
    dist.destroy_process_group()
    out.put((rank, t, it, float(prob["c"][0])))


def test_two_gloo_ranks_aggregate_and_distinct_instances():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.0, 2.0]       # max over ranks
    assert [r[2] for r in res] == [300, 300]       # summed iterations
    assert res[0][3] != res[1][3]                  # seed + rank: different instances


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "_workload", lambda *a: called.append(a))
    bench.run_reference(argparse.Namespace())
    assert called == [] and capsys.readouterr().out == ""
