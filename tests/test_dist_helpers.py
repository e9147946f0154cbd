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
    monkeypatch.setattr(bench, "oracle_sample", lambda *a, **k: called.append(1) or (1.0, 100, 1.0))
    bench.reference_arm(Args())
    assert called == [] and capsys.readouterr().out == ""


def test_reference_arm_line_on_rank_zero(monkeypatch, capsys):
    # the reference arm's one JSON line: the contract's keys, the oracle's own cores and zero copies
    import json

    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)

    class Args:
        workload = "dqd_128x128x96_4K"
        steps = 2
        warmup = 1
        gpus = 1

    samples = iter([(3.0, 1000, 2.5), (2.0, 1000, 3.0), (4.0, 1000, 2.0)])
    monkeypatch.setattr(bench, "oracle_sample", lambda *a, **k: next(samples))
    bench.reference_arm(Args())
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    full = d["config"]["nodes"]
    assert abs(d["ms_per_step"] - 3000.0) < 1e-9                 # mean of the two timed samples
    assert abs(d["value"] - (1.0 / 3.0) * 1000 / full) < 1e-15      # solves/s scaled by the node ratio
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] == 3.0
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
