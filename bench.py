"""Benchmark of the QCAD finite-element hot path on GB300.

One step is one full pass of the path on the five-gate double-quantum-dot
device of the precision form, 256 x 256 x 128 Q1 elements (8,520,321 nodes)
over 200 x 200 x 100 nm at 0.5 K:
  Newton solve of the nonlinear Poisson equation from a cold start (Laplace
  guess), mixed precision (FP32 Krylov operator, vectors and multigrid
  preconditioner; FP64 residual, reductions and Newton update) to the FP64
  residual ||R||_inf < 1e-10 V*nm and ||dphi||_inf < 1e-10 V;
  the two dot electron counts; the adjoint 2 x 5 dot-to-gate capacitance and
  the 10 lowest Schrodinger eigenpairs on the 128 x 128 x 43-element quantum
  subdomain (these two concurrently, on two streams, through qcad_adjoint_eigs).
The metric is device solves per second (whole job over all ranks). The same
line reports:
  poisson_only: the Poisson solve rate in mixed precision and in plain FP64,
    both with the same multigrid-preconditioned PCG, at the same final FP64
    residual, with their Krylov counts and the potential difference;
  configs: the other configurations (the plain FP64 128 x 128 x 96 device with
    its potential and eigenvalue errors against the oracle's stored solution,
    the 96-instance batch in instances/s, the adjoint with the per-element
    fixed-charge gradient, the MOS capacitor);
  the roofline of the dominant kernel (timed with CUDA events inside the
  library during the timed steps), the op-apply roofline, and the CPU oracle
  timed on bounded samples of the same device.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Profiling workloads (ncu launch lists and single-kernel captures):
  python bench.py --profile step|solve|apply|eigs|batch [--workload NAME] [--launch v,r,z]
Recording an ncu metrics capture (CSV) of a kernel class as the line's traffic and flop counters:
  python bench.py --ncu-counters CSV --kernel-class residual|apply32 --workload NAME --launch v,r,z --per N
Multi-GPU: launched by torch.distributed.run; ranks solve independent
replicas of the device (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import glob
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Poisson solves/s & op-apply HBM GB/s; mixed vs FP64 at same residual"
WORKLOAD = "dqd_256x256x128_0p5K"   # the precision form: the largest single-GPU configuration
FP64_WORKLOAD = "dqd_128x128x96_4K"  # the plain FP64 configuration
ADJ_WORKLOAD = "dqd_128x128x96_4K_adjoint"
MOS_WORKLOAD = "mos_cap_16x16x32"
NEV = 10
# bounded CPU samples of the benchmark device (same stack and temperature, fewer elements) for the
# oracle timing; the size exponent fitted between them extrapolates to the full mesh
SAMPLES = ((16, 16, 12), (32, 32, 24))
SP_PLUNGER_V = 0.70  # both plunger gates in the Schrodinger-Poisson measurement (about 2.6 electrons)
COUNTERS = os.path.join(ROOT, "profiles", "ncu_counters.json")
ORACLE_C2 = os.path.join(ROOT, "tests", "golden", "dqd_128x128x96_4K_oracle.npz")


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-extras", action="store_true",
                    help="time the step only (no poisson_only, other configurations, S-P, calibration)")
    ap.add_argument("--sequential", action="store_true",
                    help="run the adjoint and the eigensolve one after the other (per-kernel profiles)")
    ap.add_argument("--cheb-degree", type=int, default=0,
                    help="preconditioner of the Krylov solves (0: the mesh's autotuner chooses)")
    ap.add_argument("--launch", default=None,
                    help="variant,tile_rows,z_chunk of the FP32 operators instead of the autotuner's choice "
                         "(profiling runs, whose timings the profiler distorts)")
    ap.add_argument("--profile", default=None, choices=["step", "solve", "apply", "eigs", "batch"],
                    help="run a profiling workload instead of the benchmark")
    ap.add_argument("--precision", type=int, default=1, help="precision of --profile apply")
    ap.add_argument("--reps", type=int, default=3, help="repetitions of --profile apply")
    ap.add_argument("--ncu-counters", default=None,
                    help="ncu --csv metrics capture of one kernel class to record in profiles/ncu_counters.json "
                         "(with --kernel-class, --workload, --launch, --per, --profile-md)")
    ap.add_argument("--kernel-class", default="residual")
    ap.add_argument("--per", type=int, default=1, help="launches per unit of --ncu-counters (residual: 2 passes)")
    ap.add_argument("--profile-md", default=None, help="the profiles/ summary that records the capture command")
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------
# distributed helpers (also exercised by the CPU gloo test)
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def init_dist(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist if world > 1 else None


def barrier(dist, device=None):
    if dist is not None:
        if device is not None:
            dist.barrier(device_ids=[device])
        else:
            dist.barrier()


def max_over_ranks(dist, value, device="cpu"):
    import torch
    if dist is None:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(units_per_rank, world, t_max):
    """Whole-job throughput: units of all ranks over the slowest rank's time."""
    return units_per_rank * world / t_max


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = [l.strip().split(",") for l in open(self.path) if l.strip()]
        os.unlink(self.path)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        peak = max(sm)
        loaded = [s for s in sm if s >= 0.5 * peak] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# ncu counters (DRAM bytes per launch, FP64 flops) of the kernel classes, written by
# `bench.py --ncu-counters` from the capture commands recorded beside them in profiles/. Each entry
# carries the hash of the sources of its kernel class (the translation units that hold the
# kernels and the local headers they include); an entry whose hash differs from the current
# sources is stale and not used.
CSRC = os.path.join(ROOT, "paper_1403_7561_gb300", "csrc")
CLASS_UNITS = {
    "residual": ["kernels_poisson.cu"],
    "apply32": ["kernels_poisson.cu", "kernels_lin.cu"],
    "apply64": ["kernels_poisson.cu", "kernels_lin.cu"],
    "update32": ["kernels_poisson.cu"],
    "update64": ["kernels_poisson.cu"],
}


def _with_includes(units):
    seen, todo = [], list(units)
    while todo:
        f = todo.pop()
        if f in seen or not os.path.exists(os.path.join(CSRC, f)):
            continue
        seen.append(f)
        with open(os.path.join(CSRC, f)) as fh:
            for line in fh:
                line = line.strip()
                if line.startswith('#include "'):
                    inc = line.split('"')[1]
                    if "/" not in inc:
                        todo.append(inc)
    return sorted(seen)


def kernel_source_hash(cls=None):
    """Hash of the sources of one kernel class (all of csrc/ when cls is None)."""
    if cls in CLASS_UNITS:
        files = _with_includes(CLASS_UNITS[cls])
    else:
        files = sorted(os.path.basename(p) for p in glob.glob(os.path.join(CSRC, "*"))
                       if p.endswith((".cu", ".cuh", ".h", ".cpp")))
    h = hashlib.sha256()
    for f in files:
        h.update(f.encode())
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def load_counters():
    if not os.path.exists(COUNTERS):
        return {}, None
    d = json.load(open(COUNTERS))
    return d, kernel_source_hash()


def counter(counters, cur_hash, kernel, workload, launch, key):
    """(value, note): the counter of this kernel class, workload and launch shape if current."""
    for e in counters.get("entries", []):
        if e["kernel"] == kernel and e["workload"] == workload and tuple(e.get("launch") or ()) == tuple(launch):
            if e.get("source_hash") != kernel_source_hash(kernel):
                return None, "stale: kernel sources changed since the capture (%s)" % e.get("source_hash")
            return e.get(key), "ncu capture %s" % e.get("profile", "")
    return None, "no capture for this kernel, workload and launch shape"


def ingest_ncu(args):
    """Average an ncu CSV capture (--metrics ... --csv) of one kernel class over its units (a unit is
    `--per` consecutive launches: 2 for the two-pass residual) and record DRAM bytes and FP64 flops
    per unit in the counters file, with the class's current source hash."""
    import csv
    rows = list(csv.reader(open(args.ncu_counters)))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r and "Metric Name" in r)
    h = rows[hi]
    ii, mi, vi, ui = h.index("ID"), h.index("Metric Name"), h.index("Metric Value"), h.index("Metric Unit")
    per_launch = {}
    for r in rows[hi + 1:]:
        if len(r) <= vi:
            continue
        v = float(r[vi].replace(",", ""))
        unit = r[ui]
        scale = {"Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6, "GB": 1e9}.get(unit, 1.0)
        per_launch.setdefault(r[ii], {})[r[mi]] = v * scale
    launches = list(per_launch.values())
    units = len(launches) / float(args.per)

    def total(name):
        return sum(l.get(name, 0.0) for l in launches) / units

    dram = total("dram__bytes_read.sum") + total("dram__bytes_write.sum")
    flops = (2 * total("sm__sass_thread_inst_executed_op_dfma_pred_on.sum") +
             total("sm__sass_thread_inst_executed_op_dadd_pred_on.sum") +
             total("sm__sass_thread_inst_executed_op_dmul_pred_on.sum"))
    d = json.load(open(COUNTERS)) if os.path.exists(COUNTERS) else {"entries": []}
    launch = [int(x) for x in args.launch.split(",")] if args.launch else []
    d["entries"] = [e for e in d.get("entries", []) if not (e["kernel"] == args.kernel_class and
                                                             e["workload"] == args.workload and
                                                             e.get("launch") == launch)]
    d["entries"].append({"kernel": args.kernel_class, "workload": args.workload, "launch": launch,
                         "source_hash": kernel_source_hash(args.kernel_class), "dram_bytes": dram,
                         "fp64_flops": flops or None, "launches_per_unit": args.per,
                         "units_captured": units, "profile": args.profile_md or ""})
    os.makedirs(os.path.dirname(COUNTERS), exist_ok=True)
    with open(COUNTERS, "w") as f:
        json.dump(d, f, indent=1)
    print(json.dumps(d["entries"][-1]))


# FP64 peak of this part: 2 DFMA lanes per SM per clock (ncu
# sm__sass_thread_inst_executed_op_dfma_pred_on.avg.peak_sustained) x 2 flops x 152 SMs.
FP64_FLOPS_PER_CLOCK = 2 * 2 * 152


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def algorithmic_bytes(cls, n_nodes, n_elems):
    """Bytes each launch must move at minimum given its stored linearization (per class)."""
    return {
        # p = z + beta p_prev (read z, p_prev; write p), Ap written, 8 FP32 qp coefficients per element
        "apply32": 16 * n_nodes + 32 * n_elems,
        "apply64": 32 * n_nodes + 64 * n_elems,
        # x, r, p, Ap, D^-1 read; x, r, z written
        "update32": 32 * n_nodes,
        "update64": 64 * n_nodes,
        # phi read; R, D^-1 (FP32), -R (FP32) written; FP32 qp coefficients written (mixed linearization)
        "residual": 24 * n_nodes + 32 * n_elems,
    }.get(cls)


# ---------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, on bounded samples of the benchmark device
def sample_device(workload, n):
    import workloads as W
    full = W.get(workload)
    if full["name"].startswith("mos"):
        return W.mos_capacitor(nx=n[0], ny=n[1], nz=n[2])
    return W.five_gate_device(n=n, T=full["bias"]["T"])


def oracle_pass(workload, n):
    """One pass of the whole path by the oracle on the sample of size n: (wall s, nodes, cores)."""
    from oracle import capacitance as OC
    from oracle import schrodinger as OS
    from oracle.poisson import PoissonProblem
    dev = sample_device(workload, n)
    t0 = time.perf_counter()
    c0 = time.process_time()
    P = PoissonProblem(dev)
    phi, rep = P.solve()
    OC.electron_counts(P, phi)
    if dev["dots"]:
        OC.adjoint(P, phi)
    if dev.get("subdomain"):
        OS.solve_device(P, phi, nev=NEV)
    dt = time.perf_counter() - t0
    cores = (time.process_time() - c0) / dt
    return dt, P.mesh.n_nodes, round(max(cores, 1.0), 2)


def extrapolate(times, nodes, full_nodes):
    """Power law t = a N^p through the mean time of each sample size; (t at full_nodes, p)."""
    (t0, n0), (t1, n1) = zip(times, nodes)
    p = math.log(t1 / t0) / math.log(n1 / n0)
    return t1 * (full_nodes / n1) ** p, p


def cpu_baseline_desc(workload, nodes, p, cores):
    return ("oracle (numpy/scipy FP64) whole path on the %s device at %s elements (%s nodes), one pass each; "
            "time extrapolated to the full mesh by the fitted power law t ~ N^%.2f; cores = process CPU time / "
            "wall time" % (workload, " and ".join("x".join(str(v) for v in s) for s in SAMPLES),
                           " and ".join(str(v) for v in nodes), p))


def reference_arm(args):
    """The oracle (plain FP64 CPU implementation) as the reference arm: each step one pass over one of
    the bounded samples (alternating sizes), the size exponent fitted between them."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import workloads as W
    full = W.n_nodes(W.get(args.workload))
    times = {0: [], 1: []}
    nodes = [None, None]
    used = []
    for s in range(args.warmup + args.steps):
        k = 0 if s < args.warmup else (s - args.warmup) % 2
        dt, nn, cores = oracle_pass(args.workload, SAMPLES[k])
        nodes[k] = nn
        if s >= args.warmup:
            times[k].append(dt)
            used.append(cores)
    if not times[1]:  # a single timed step: time the larger sample once more
        dt, nodes[1], cores = oracle_pass(args.workload, SAMPLES[1])
        times[1].append(dt)
    means = [sum(times[k]) / len(times[k]) for k in (0, 1)]
    t_full, p = extrapolate(means, nodes, full)
    value = 1.0 / t_full
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * (sum(times[0]) + sum(times[1])) / max(1, len(times[0]) + len(times[1])),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "nodes": full, "samples": [list(s) for s in SAMPLES],
                       "size_exponent": p},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": max(used) if used else None,
                             "kind": "oracle", "sample": cpu_baseline_desc(args.workload, nodes, p, used)},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def timed_events(torch, fn, reps, flush=None):
    """Best and mean of reps CUDA-event timings of fn() (seconds), with the last result."""
    ts, out = [], None
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        out = fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b) / 1000.0)
    return min(ts), sum(ts) / len(ts), out


def oracle_reference_c2():
    """The oracle's stored solution of the 128 x 128 x 96 device (written by tests/golden), or None."""
    if not os.path.exists(ORACLE_C2):
        return None
    import numpy as np
    d = np.load(ORACLE_C2)
    return {k: d[k] for k in d.files}


def other_configs(q, W, torch, flush):
    """The plain FP64 device, the adjoint with the fixed-charge gradient, the batch and the MOS capacitor."""
    import numpy as np
    out = {}
    # plain FP64 128 x 128 x 96 device at 4 K (and the mixed arm on it), errors against the oracle
    dev = W.get(FP64_WORKLOAD)
    bias = dev["bias"]
    m = q.qcad_mesh_create(dev)
    q.qcad_autotune(m, bias, precision=1)
    q.qcad_autotune(m, bias, precision=0)
    ref = oracle_reference_c2()
    arms = {}
    for name, prec in (("fp64", 0), ("mixed", 1)):
        phi = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
        opts = q.make_opts(precision=prec, cheb_degree=0)
        q.qcad_poisson_solve(m, bias, opts, phi)  # autotunes the preconditioner once per precision
        t, tm, rep = timed_events(torch, lambda: q.qcad_poisson_solve(m, bias, opts, phi), 2, flush)
        te, _, (E, erep) = timed_events(torch, lambda: q.qcad_schrodinger_eigs(m, bias, phi, nev=NEV, tol=1e-8), 2,
                                        flush)
        N = q.qcad_electron_counts(m, bias, phi)
        a = {"solves_per_s": 1.0 / t, "newton_iters": rep["newton_iters"], "krylov_iters": rep["krylov_iters_total"],
             "preconditioner": q.qcad_launch_info(m, 1 if prec == 0 else 2)[3], "final_res_inf": rep["final_res_inf"],
             "eigs_seconds": te, "E_meV": [1e3 * e for e in E]}
        if ref is not None:
            a["max_abs_phi_err_vs_oracle_V"] = float(np.max(np.abs(phi.cpu().numpy() - ref["phi"])))
            a["max_rel_eig_err_vs_oracle"] = float(np.max(np.abs(np.array(E) - ref["evals"]) / np.abs(ref["evals"])))
            a["max_rel_count_err_vs_oracle"] = float(np.max(np.abs(np.array(N) - ref["counts"]) /
                                                            np.abs(ref["counts"])))
        arms[name] = a
    out["plain_fp64"] = {"workload": FP64_WORKLOAD, "nodes": m.n_nodes,
                         "oracle_reference": os.path.relpath(ORACLE_C2, ROOT) if ref is not None else None,
                         "preconditioner_code": "-1 multigrid V-cycle, k >= 1 Chebyshev degree (autotuned)",
                         **arms}
    del m
    # a plunger sweep of the same device (8 bias points, a mesh each): the batched Newton and one
    # batched adjoint call for every point's 2 x 5 dN/dV, against the points solved one by one
    pts = []
    for k in range(8):
        b = dict(bias, V_gate=list(bias["V_gate"]))
        b["V_gate"][1] += 0.01 * (k - 3.5)
        pts.append(b)
    sm = [q.qcad_mesh_create(dev) for _ in pts]
    sphi = [torch.zeros(mm.n_nodes, dtype=torch.float64, device="cuda") for mm in sm]
    sopts = q.make_opts(precision=1, cheb_degree=-1)

    def sweep_batched():
        for p_ in sphi:
            p_.zero_()
        reps_, st_ = q.qcad_poisson_solve_batch(sm, pts, sopts, sphi)
        return st_, q.qcad_adjoint_batch(sm, pts, sopts, sphi)

    def sweep_one_by_one():
        out_ = []
        for mm, b, p_ in zip(sm, pts, sphi):
            q.qcad_poisson_solve(mm, b, sopts, p_)
            out_.append(q.qcad_adjoint(mm, b, p_, sopts))
        return out_

    sweep_batched()
    tb, _, (sst, sdn) = timed_events(torch, sweep_batched, 2, flush)
    sweep_one_by_one()
    ts1, _, sdn1 = timed_events(torch, sweep_one_by_one, 2, flush)
    out["bias_sweep"] = {"workload": "%s, plunger P1 swept over 8 points (-35..+35 mV), mixed, multigrid PCG"
                         % FP64_WORKLOAD, "points": len(pts), "status": sst,
                         "batched_points_per_s": len(pts) / tb, "one_by_one_points_per_s": len(pts) / ts1,
                         "max_abs_dNdV_batched_vs_one_by_one": float(np.max(np.abs(np.array(sdn) - np.array(sdn1)))),
                         "step": "Newton solve + 2 x 5 adjoint dN/dV per point (batched: qcad_poisson_solve_batch "
                                 "then qcad_adjoint_batch)"}
    del sm, sphi
    # the differentiation form: Newton with the interface fixed charge, then the adjoint with the
    # 2 x 5 capacitance and the gradient with respect to every element's fixed charge
    dev = W.get(ADJ_WORKLOAD)
    bias = dev["bias"]
    m = q.qcad_mesh_create(dev)
    q.qcad_autotune(m, bias, precision=1)
    th = torch.tensor(W.interface_fixed_charge(dev, seed=5), dtype=torch.float64, device="cuda")
    phi = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    dq = torch.empty(m.n_dots * m.n_elems, dtype=torch.float64, device="cuda")
    opts = q.make_opts(precision=1, cheb_degree=0)

    def adj_step():
        q.qcad_poisson_solve(m, bias, opts, phi, fixed_charge=th)
        return q.qcad_adjoint(m, bias, phi, opts, fixed_charge=th, dN_dq=dq)

    adj_step()
    t, _, dNdV = timed_events(torch, adj_step, 3, flush)
    out["adjoint"] = {"workload": ADJ_WORKLOAD, "step": "mixed Newton with the fixed-charge field + adjoint "
                      "(2 x 5 dN/dV and the 2 x %d fixed-charge gradient)" % m.n_elems,
                      "steps_per_s": 1.0 / t, "gradient_entries": 2 * m.n_elems,
                      "capacitance_aF": [[1.602176634e-1 * x for x in row] for row in dNdV],
                      "max_abs_dN_dtheta": float(torch.max(torch.abs(dq)).item())}
    del m, dq
    # the batched form: 96 instances of 48^3 .. 112^3 elements in lockstep Newton
    devs = W.batch_instances()
    meshes = [q.qcad_mesh_create(d) for d in devs]
    phis = [torch.zeros(mm.n_nodes, dtype=torch.float64, device="cuda") for mm in meshes]
    biases = [d["bias"] for d in devs]
    bopts = q.make_opts(precision=1, cheb_degree=-1)

    def batch():
        for p in phis:
            p.zero_()
        return q.qcad_poisson_solve_batch(meshes, biases, bopts, phis)

    batch()
    t, _, (reps, st) = timed_events(torch, batch, 2, flush)
    out["batch"] = {"workload": "96 five-gate instances, N^3 elements, N in 48..112 (seed 4), 4 K, mixed, "
                    "multigrid PCG per instance", "instances": len(devs),
                    "nodes": int(sum(mm.n_nodes for mm in meshes)), "status": st, "seconds": t,
                    "instances_per_s": len(devs) / t,
                    "newton_iters_max": max(r["newton_iters"] for r in reps),
                    "final_res_inf_max": max(r["final_res_inf"] for r in reps)}
    del meshes, phis
    # the plain FP64 MOS capacitor (16 x 16 x 32 elements, 300 K)
    dev = W.get(MOS_WORKLOAD)
    m = q.qcad_mesh_create(dev)
    phi = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    opts = q.make_opts(precision=0, cheb_degree=0)
    q.qcad_poisson_solve(m, dev["bias"], opts, phi)
    t, _, rep = timed_events(torch, lambda: q.qcad_poisson_solve(m, dev["bias"], opts, phi), 5)
    out["mos_capacitor"] = {"workload": MOS_WORKLOAD, "nodes": m.n_nodes, "precision": "fp64",
                            "solves_per_s": 1.0 / t, "newton_iters": rep["newton_iters"],
                            "final_res_inf": rep["final_res_inf"]}
    return out


def native_arm(args):
    import numpy as np
    import torch

    import paper_1403_7561_gb300 as q
    import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = init_dist(world, "nccl")
    dev = W.get(args.workload)
    bias = dev["bias"]
    m = q.qcad_mesh_create(dev)
    n_nodes, n_elems = m.n_nodes, m.n_elems
    mixed = q.make_opts(precision=1, cheb_degree=args.cheb_degree)  # 0: preconditioner autotuned per mesh
    phi = torch.zeros(n_nodes, dtype=torch.float64, device="cuda")
    evecs = torch.empty(NEV, m.n_sub_dof, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)

    solve_prof = {c: [0, 0.0] for c in q.PROF_CLASSES}  # kernel time inside the Newton solves

    def step():
        before = {c: q.qcad_profile_read(m, c) for c in q.PROF_CLASSES}
        rep = q.qcad_poisson_solve(m, bias, mixed, phi)
        for c in q.PROF_CLASSES:
            n1, t1 = q.qcad_profile_read(m, c)
            solve_prof[c][0] += n1 - before[c][0]
            solve_prof[c][1] += t1 - before[c][1]
        N = q.qcad_electron_counts(m, bias, phi)
        if args.sequential:
            dNdV = q.qcad_adjoint(m, bias, phi, mixed)
            E, erep = q.qcad_schrodinger_eigs(m, bias, phi, nev=NEV, tol=1e-8, evecs=evecs)
        else:
            # adjoint capacitance and eigenpairs at the converged potential, run concurrently
            dNdV, E, erep = q.qcad_adjoint_eigs(m, bias, phi, mixed, nev=NEV, tol=1e-8, evecs=evecs)
        return rep, N, dNdV, E, erep

    # launch tuning for this mesh (the autotuner picks tile rows and z chunk per precision)
    if args.launch:
        tune32 = tuple(int(x) for x in args.launch.split(",")) + (None,)
        q.qcad_set_launch(m, 2, tune32[0], tune32[1], tune32[2])
    else:
        tune32 = q.qcad_autotune(m, bias, precision=1)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    q.qcad_profile_reset(m)
    q.qcad_profile_enable(m, True)
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = q.qcad_launch_count()
    barrier(dist, local)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    info = None
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed steps' launches
    for s in range(args.steps):
        flush.zero_()  # L2 flush between timed steps (outside the timed interval)
        ev[s][0].record()
        info = step()
        ev[s][1].record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    barrier(dist, local)
    launches = q.qcad_launch_count() - launches0
    clk = clocks.stop()
    q.qcad_profile_enable(m, False)
    t_local = sum(a.elapsed_time(b) for a, b in ev) / 1000.0
    t_max = max_over_ranks(dist, t_local, device="cuda")
    value = aggregate(args.steps, world, t_max)
    rep, N, dNdV, E, erep = info

    # dominant kernel and its roofline
    peak, peak_kind = load_peaks()
    counters, cur_hash = load_counters()
    prof = {}
    for cls in q.PROF_CLASSES:
        nl, ms = q.qcad_profile_read(m, cls)
        prof[cls] = (nl, ms)
    total_ms = sum(v[1] for v in prof.values())
    # single-kernel classes with a roofline model (the multigrid tail is many small kernels; the
    # H/M class mixes FP32 and FP64 launches over blocks of different widths)
    dom = max((c for c in prof if algorithmic_bytes(c, n_nodes, n_elems) is not None), key=lambda c: prof[c][1])
    share = prof[dom][1] / total_ms if total_ms else None
    tune_key = tuple(tune32[:3])

    # measured arithmetic peaks of this GPU (microbenchmarks, outside the timed region): the
    # measured side of the FP64 residual's ALU roofline
    alu = q.qcad_alu_peaks()

    # rooflines use launches inside the Newton solves of the timed steps: the adjoint and the
    # eigensolve run concurrently on two streams, so their launches overlap
    def hbm_roofline(cls):
        nl, ms = solve_prof[cls]
        ach = algorithmic_bytes(cls, n_nodes, n_elems) / (ms / nl / 1000.0) / 1e9 if nl else None
        traffic, note = counter(counters, cur_hash, cls, args.workload, tune_key, "dram_bytes")
        return {"bound": "hbm", "kernel": cls, "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": (ach / peak) if ach else None, "traffic": traffic,
                "traffic_unit": "bytes per launch (ncu dram read + write, cold cache)", "traffic_source": note,
                "algorithmic_bytes": algorithmic_bytes(cls, n_nodes, n_elems),
                "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)", "launches": nl,
                "avg_ms": ms / nl if nl else None,
                "timed_launches": "inside the Newton solves of the timed steps (no concurrent work)"}

    def fp64_roofline(cls):
        nl, ms = solve_prof[cls]
        flops, fnote = counter(counters, cur_hash, cls, args.workload, tune_key, "fp64_flops")
        traffic, note = counter(counters, cur_hash, cls, args.workload, tune_key, "dram_bytes")
        mhz = clk.get("sm_mhz") or 2070.0
        pk = FP64_FLOPS_PER_CLOCK * mhz * 1e6 / 1e12
        ach = flops / (ms / nl / 1000.0) / 1e12 if (nl and flops) else None
        return {"bound": "alu", "kernel": cls, "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                "frac": (ach / pk) if ach else None, "traffic": traffic,
                "traffic_unit": "bytes per evaluation (ncu dram read + write, cold cache, both passes)",
                "traffic_source": note, "flops_source": fnote,
                "peak_kind": "derived: 2 DFMA lanes/SM/clock x 2 flops x 152 SMs x median SM clock under load",
                "flops_kind": "FP64 flops per evaluation counted by ncu (2 DFMA + DADD + DMUL)",
                "peak_measured": alu["fp64_tflops"],
                "frac_of_measured": (ach / alu["fp64_tflops"]) if ach else None,
                "peak_measured_kind": "FP64 FMA microbenchmark on this GPU (qcad_alu_peaks)",
                "launches": nl, "avg_ms": ms / nl if nl else None,
                "timed_launches": "residual evaluations inside the Newton solves of the timed steps"}

    roof = fp64_roofline(dom) if dom == "residual" else hbm_roofline(dom)
    roof["share_of_profiled_time"] = share
    op_apply = hbm_roofline("apply32")

    # end to end through the public API with host buffers: the gate voltages go in from the host
    # (inside the library, pinned staging), phi comes back to pinned host memory every step
    phi_host = torch.empty(n_nodes, dtype=torch.float64, pin_memory=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(args.steps):
        b = dict(bias, V_gate=list(bias["V_gate"]))
        q.qcad_poisson_solve(m, b, mixed, phi)
        q.qcad_electron_counts(m, b, phi)
        q.qcad_adjoint_eigs(m, b, phi, mixed, nev=NEV, tol=1e-8)
        phi_host.copy_(phi, non_blocking=True)
        torch.cuda.synchronize()
    t_e2e = max_over_ranks(dist, time.perf_counter() - t0, device="cuda")
    e2e = aggregate(args.steps, world, t_e2e)
    h2d = 8 * len(bias["V_gate"]) + 8 * 4  # gate voltages and bias scalars
    d2h = 8 * n_nodes + 8 * (len(N) + len(N) * len(bias["V_gate"]) + NEV)

    extras = {}
    if not args.no_extras:
        # Poisson only: mixed vs plain FP64 at the same final FP64 residual, both with the multigrid
        # V-cycle (the same preconditioner in each arm's precision), then the eigenpairs at each
        # arm's potential
        arms = {}
        phis = {}
        for name, prec in (("mixed", 1), ("fp64", 0)):
            opts = q.make_opts(precision=prec, cheb_degree=-1)
            p = torch.zeros(n_nodes, dtype=torch.float64, device="cuda")
            q.qcad_poisson_solve(m, bias, opts, p)  # builds this precision's graphs and V-cycle levels
            t, tm, r = timed_events(torch, lambda: q.qcad_poisson_solve(m, bias, opts, p), 2, flush)
            arms[name] = {"solves_per_s": 1.0 / t, "seconds": t, "newton_iters": r["newton_iters"],
                          "krylov_iters": r["krylov_iters_total"], "final_res_inf": r["final_res_inf"],
                          "final_dphi_inf": r["final_dphi_inf"], "preconditioner": "multigrid V-cycle"}
            phis[name] = p
        Em, _ = q.qcad_schrodinger_eigs(m, bias, phis["mixed"], nev=NEV, tol=1e-8)
        Ef, _ = q.qcad_schrodinger_eigs(m, bias, phis["fp64"], nev=NEV, tol=1e-8)
        extras["poisson_only"] = {
            "workload": args.workload, **arms,
            "mixed_over_fp64": arms["mixed"]["solves_per_s"] / arms["fp64"]["solves_per_s"],
            "max_abs_dphi_mixed_vs_fp64_V": float(torch.max(torch.abs(phis["mixed"] - phis["fp64"])).item()),
            "max_rel_eig_diff_mixed_vs_fp64": float(np.max(np.abs(np.array(Em) - np.array(Ef)) / np.abs(Ef))),
            "errors_vs_oracle": "the oracle's own solve of this 8.5M-node mesh is not stored (hours on the CPU); "
                                "see configs.plain_fp64 for both arms against the oracle's 1.6M-node solution",
        }
        del phis
        extras["configs"] = other_configs(q, W, torch, flush)

        # Self-consistent Schrodinger-Poisson solve (Sec. II.C predictor-corrector, V_xc on) of the
        # 128 x 128 x 96 device with both plungers at SP_PLUNGER_V, to the paper's potential tolerance
        # 1e-5 V; and the interface-charge calibration of dot 0 to one electron (Sec. III)
        cdev = W.get(FP64_WORKLOAD)
        cm = q.qcad_mesh_create(cdev)
        q.qcad_autotune(cm, cdev["bias"], precision=1)
        sp_bias = dict(cdev["bias"], V_gate=list(cdev["bias"]["V_gate"]))
        sp_bias["V_gate"][1] = sp_bias["V_gate"][3] = SP_PLUNGER_V
        phi_sp = torch.zeros(cm.n_nodes, dtype=torch.float64, device="cuda")
        copts = q.make_opts(precision=1, cheb_degree=0)
        t, _, (E_sp, rep_sp) = timed_events(
            torch, lambda: q.qcad_sp_solve(cm, sp_bias, phi_sp, copts, nev=NEV, eig_tol=1e-8, tol_dphi=1e-5,
                                           max_iter=100, use_vxc=True, allow_not_converged=True), 2, flush)
        extras["schrodinger_poisson"] = {
            "workload": "%s, plungers %.2f V, %d states, V_xc on" % (FP64_WORKLOAD, SP_PLUNGER_V, NEV),
            "seconds": t, "sp_solves_per_s": 1.0 / t, "status": rep_sp["status"], "sp_iters": rep_sp["sp_iters"],
            "final_dphi_V": rep_sp["dphi_inf"], "electrons_in_quantum_region": rep_sp["n_quantum"],
            "E_meV": [1e3 * e for e in E_sp]}
        pat = torch.tensor(W.interface_sheet_pattern(cdev), dtype=torch.float64, device="cuda")
        t, _, (sig, crep, _, _) = timed_events(
            torch, lambda: q.qcad_calibrate_sheet_charge(cm, cdev["bias"], pat, copts, dot=0, target=1.0, tol_N=1e-6,
                                                         max_iter=30, allow_not_converged=True), 2, flush)
        extras["interface_charge_calibration"] = {
            "workload": "%s, dot 0 to 1 electron, uniform interface sheet" % FP64_WORKLOAD, "seconds": t,
            "status": crep["status"], "solves": crep["iters"], "sigma_per_cm2": sig * 1e14, "N": crep["N"]}
        del cm

    cpu = None
    if rank == 0 and world == 1:
        ts, nodes, used = [], [], []
        for n in SAMPLES:
            dt, nn, cores = oracle_pass(args.workload, n)
            ts.append(dt)
            nodes.append(nn)
            used.append(cores)
        t_full, p = extrapolate(ts, nodes, n_nodes)
        cpu = {"value": 1.0 / t_full, "unit": "solves/s", "cores": max(used), "kind": "oracle",
               "sample": cpu_baseline_desc(args.workload, nodes, p, used), "size_exponent": p,
               "sample_seconds": ts}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": args.workload, "nodes": n_nodes, "elements": n_elems,
                       "step": "mixed Newton Poisson (FP64 residual 1e-10) + dot counts + 2x5 adjoint capacitance + "
                               "%d LOBPCG eigenpairs" % NEV,
                       "l2": "flushed between timed steps (256 MB write); the working set exceeds L2",
                       "parallelism": "replicas x%d" % world,
                       "apply_launch": {"variant": tune32[0], "tile_rows": tune32[1], "z_chunk": tune32[2],
                                        "chosen_by": "--launch" if args.launch else "autotuner"},
                       "preconditioner": args.cheb_degree or q.qcad_launch_info(m, 2)[3],
                       "adjoint_eigensolve": "sequential" if args.sequential else "concurrent (two streams)"},
            "roofline": roof,
            "alu_peaks": dict(alu, kind="microbenchmarks on this GPU: FMA chains (2 flops per FMA), FP64 exp()"),
            "op_apply_roofline": op_apply,
            "kernel_profile_ms": {c: round(v[1], 3) for c, v in prof.items()},
            "kernel_source_hash": {c: kernel_source_hash(c) for c in ("residual", "apply32")},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clk,
            **extras,
            "results": {"newton_iters": rep["newton_iters"], "krylov_iters": rep["krylov_iters_total"],
                        "final_res_inf": rep["final_res_inf"], "dot_electrons": N,
                        "capacitance_aF": [[1.602176634e-1 * x for x in row] for row in dNdV],
                        "E_meV": [1e3 * e for e in E], "lobpcg_iters": erep["krylov_iters_total"]},
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# Profiling workloads: what ncu captures (launch lists and single-kernel captures).
#   step:  autotune, one warm-up pass of the path (mixed Newton, counts, adjoint, eigenpairs, one
#          after the other), then one pass inside the NVTX range "step"
#   solve: autotune, one mixed Poisson solve (captures of the PCG and residual kernels)
#   apply: the Jacobian apply of one precision at the Laplace guess, --reps times
#   eigs:  one mixed solve, one warm-up eigensolve, then one inside the NVTX range "eigs"
#   batch: the 96-instance batch, one batched Newton solve
def profile_arm(args):
    import torch

    import paper_1403_7561_gb300 as q
    import workloads as W

    if args.profile == "batch":
        devs = W.batch_instances()
        meshes = [q.qcad_mesh_create(d) for d in devs]
        phis = [torch.zeros(mm.n_nodes, dtype=torch.float64, device="cuda") for mm in meshes]
        reps, st = q.qcad_poisson_solve_batch(meshes, [d["bias"] for d in devs],
                                              q.make_opts(precision=1, cheb_degree=-1), phis)
        torch.cuda.synchronize()
        print("batch done: %d instances, %s" % (len(devs), st))
        return
    dev = W.get(args.workload)
    bias = dev["bias"]
    m = q.qcad_mesh_create(dev)
    phi = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    if args.launch:
        v, r, c = (int(x) for x in args.launch.split(","))
        q.qcad_set_launch(m, 2, v, r, c)
    elif args.profile != "apply":
        q.qcad_autotune(m, bias, precision=1)
    opts = q.make_opts(precision=1, cheb_degree=args.cheb_degree)
    if args.profile == "solve":
        rep = q.qcad_poisson_solve(m, bias, opts, phi)
        torch.cuda.synchronize()
        print("solve done: %d nodes, %d Newton, %d Krylov iterations" % (m.n_nodes, rep["newton_iters"],
                                                                          rep["krylov_iters_total"]))
    elif args.profile == "eigs":
        q.qcad_poisson_solve(m, bias, opts, phi)
        evecs = torch.empty(NEV, m.n_sub_dof, dtype=torch.float64, device="cuda")
        q.qcad_schrodinger_eigs(m, bias, phi, nev=NEV, tol=1e-8, evecs=evecs)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("eigs")
        E, rep = q.qcad_schrodinger_eigs(m, bias, phi, nev=NEV, tol=1e-8, evecs=evecs)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print("eigs done: %d subdomain dof" % m.n_sub_dof)
    elif args.profile == "step":

        def step():
            q.qcad_poisson_solve(m, bias, opts, phi)
            q.qcad_electron_counts(m, bias, phi)
            q.qcad_adjoint(m, bias, phi, opts)
            q.qcad_schrodinger_eigs(m, bias, phi, nev=NEV, tol=1e-8)

        c0 = q.qcad_launch_count()
        step()
        c1 = q.qcad_launch_count()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("step")  # ncu --nvtx --nvtx-include "step/" keeps this pass only
        step()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        c2 = q.qcad_launch_count()
        print("launches warmup=%d step=%d" % (c1 - c0, c2 - c1))
    else:
        q.qcad_contact_values(m, bias, phi)
        v = torch.randn(m.n_nodes, dtype=torch.float64, device="cuda")
        y = torch.empty_like(v)
        for _ in range(args.reps):
            q.qcad_poisson_jv(m, bias, phi, v, y, args.precision)
        torch.cuda.synchronize()
        print("apply done: %d nodes, precision %d, %d reps" % (m.n_nodes, args.precision, args.reps))


def main():
    args = parse()
    if args.ncu_counters:
        ingest_ncu(args)
    elif args.impl == "reference":
        reference_arm(args)
    elif args.profile:
        profile_arm(args)
    else:
        native_arm(args)


if __name__ == "__main__":
    main()
