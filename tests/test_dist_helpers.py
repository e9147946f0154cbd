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
        workload = "dqd_256x256x128_0p5K"
        steps = 1
        warmup = 0
        gpus = 2

    called = []
    monkeypatch.setattr(bench, "oracle_pass", lambda *a, **k: called.append(1) or (1.0, 100, 1.0))
    bench.reference_arm(Args())
    assert called == [] and capsys.readouterr().out == ""


def test_reference_arm_line_on_rank_zero(monkeypatch, capsys):
    # the reference arm's one JSON line: the contract's keys, the oracle's own cores, zero copies,
    # and the full-mesh time from the power law through the two sample sizes
    import json
    import math

    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)

    class Args:
        workload = "dqd_256x256x128_0p5K"
        steps = 4
        warmup = 1
        gpus = 1

    # warm-up (small), then small, large, small, large: t = 1e-4 N^1.5 s exactly
    sizes = {bench.SAMPLES[0]: 1000, bench.SAMPLES[1]: 8000}
    cores = iter([2.0, 2.5, 3.0, 2.0, 1.5])
    seen = []

    def fake(workload, n):
        seen.append(n)
        N = sizes[n]
        return 1e-4 * N ** 1.5, N, next(cores)

    monkeypatch.setattr(bench, "oracle_pass", fake)
    bench.reference_arm(Args())
    assert seen == [bench.SAMPLES[0], bench.SAMPLES[0], bench.SAMPLES[1], bench.SAMPLES[0], bench.SAMPLES[1]]
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 4 and d["warmup"] == 1
    full = d["config"]["nodes"]
    assert abs(d["config"]["size_exponent"] - 1.5) < 1e-12
    assert math.isclose(d["value"], 1.0 / (1e-4 * full ** 1.5), rel_tol=1e-12)
    # mean time of the four timed passes
    assert math.isclose(d["ms_per_step"], 1000.0 * 1e-4 * (2 * 1000 ** 1.5 + 2 * 8000 ** 1.5) / 4, rel_tol=1e-12)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] == 3.0
    assert "N^1.50" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_power_law_extrapolation():
    import bench
    t, p = bench.extrapolate([2.0, 16.0], [100, 400], 1600)
    assert abs(p - 1.5) < 1e-12 and abs(t - 128.0) < 1e-9


def test_kernel_source_hash_tracks_the_sources():
    # the ncu counters are keyed by the hash of their kernel class's sources: it is stable, covers
    # the translation units and the local headers they include, and differs between classes whose
    # sources differ
    import bench
    h = bench.kernel_source_hash("apply32")
    assert h == bench.kernel_source_hash("apply32") and len(h) == 16
    assert bench.kernel_source_hash("residual") != h
    assert "linmarch.cuh" in bench._with_includes(bench.CLASS_UNITS["apply32"])
    assert "physics.cuh" in bench._with_includes(bench.CLASS_UNITS["residual"])
    assert "lobpcg.cu" not in bench._with_includes(bench.CLASS_UNITS["residual"])
    counters = {"entries": [{"kernel": "apply32", "workload": "w", "launch": [3, 8, 16], "dram_bytes": 5.0,
                             "source_hash": "0" * 16}]}
    v, note = bench.counter(counters, None, "apply32", "w", (3, 8, 16), "dram_bytes")
    assert v is None and note.startswith("stale")
    counters["entries"][0]["source_hash"] = h
    assert bench.counter(counters, None, "apply32", "w", (3, 8, 16), "dram_bytes")[0] == 5.0
    assert bench.counter(counters, None, "apply32", "w", (3, 8, 19), "dram_bytes")[0] is None


def test_ingest_ncu_averages_units(tmp_path, monkeypatch):
    # two captured evaluations of the two-pass residual (four launches) become one entry per unit
    import argparse
    import json as _json
    import bench
    monkeypatch.setattr(bench, "COUNTERS", str(tmp_path / "c.json"))
    rows = ['"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"']
    for i in range(4):
        rows.append('"%d","k%d","dram__bytes_read.sum","byte","%d"' % (i, i % 2, 100 * (i % 2 + 1)))
        rows.append('"%d","k%d","dram__bytes_write.sum","Kbyte","1"' % (i, i % 2))
        rows.append('"%d","k%d","sm__sass_thread_inst_executed_op_dfma_pred_on.sum","inst","10"' % (i, i % 2))
        rows.append('"%d","k%d","sm__sass_thread_inst_executed_op_dadd_pred_on.sum","inst","3"' % (i, i % 2))
    csv_path = tmp_path / "cap.csv"
    csv_path.write_text("==PROF== header line\n" + "\n".join(rows) + "\n")
    args = argparse.Namespace(ncu_counters=str(csv_path), kernel_class="residual", workload="w", launch="3,8,19",
                              per=2, profile_md="profiles/x.md")
    bench.ingest_ncu(args)
    e = _json.loads((tmp_path / "c.json").read_text())["entries"][0]
    assert e["dram_bytes"] == 100 + 200 + 2 * 1000
    assert e["fp64_flops"] == 2 * (2 * 10 + 3)
    assert e["launch"] == [3, 8, 19] and e["source_hash"] == bench.kernel_source_hash("residual")
