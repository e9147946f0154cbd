"""Multi-process paths of bench.py on CPU: two gloo ranks (127.0.0.1).

The GPU path runs independent replicas per rank (no collective on the data
path); what crosses ranks is the barrier around the timed region, the max of
the per-rank times and the whole-job throughput. Those helpers are run here
with world size 2 over gloo, plus the rank-0-only rule of the reference arm.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import bench
    r, w, local = bench.dist_env()
    dist = bench.init_dist(w, "gloo")
    bench.barrier(dist)
    t_local = 1.0 + 0.5 * r  # rank 1 is the slowest
    t_max = bench.max_over_ranks(dist, t_local)
    value = bench.aggregate(4, w, t_max)
    out.put((r, w, local, t_max, value))
    bench.barrier(dist)
    dist.destroy_process_group()


def test_helpers_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[0] for x in res] == [0, 1]
    for r, w, local, t_max, value in res:
        assert w == 2 and local == r
        assert t_max == pytest.approx(1.5)          # the max over ranks, seen by every rank
        assert value == pytest.approx(4 * 2 / 1.5)  # whole-job units over the slowest rank's time


def test_single_process_defaults(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    import bench
    assert bench.dist_env() == (0, 1, 0)
    assert bench.init_dist(1, "gloo") is None
    assert bench.max_over_ranks(None, 3.0) == 3.0
    assert bench.aggregate(5, 1, 2.0) == 2.5


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        workload = "dqd_128x128x96_4K"
        steps = 1
        warmup = 0
        gpus = 2

    called = []
    monkeypatch.setattr(bench, "oracle_sample", lambda *a, **k: called.append(1) or (1.0, 100))
    bench.reference_arm(Args())
    assert called == [] and capsys.readouterr().out == ""
