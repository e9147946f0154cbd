"""Benchmark of the QCAD finite-element hot path on GB300.

One step is one full pass of the path on the five-gate double-quantum-dot
device, 128 x 128 x 96 Q1 elements (1,614,177 nodes) over 200 x 200 x 100 nm
at 4 K:
  Newton solve of the nonlinear Poisson equation from a cold start (Laplace
  guess), mixed precision (FP32 Krylov, FP64 residual) to the FP64 residual
  ||R||_inf < 1e-10 V*nm and ||dphi||_inf < 1e-10 V;
  the two dot electron counts; the adjoint 2 x 5 dot-to-gate capacitance and
  the 10 lowest Schrodinger eigenpairs on the 64 x 64 x 32 quantum subdomain
  (these two concurrently, on two streams, through qcad_adjoint_eigs).
The metric is device solves per second (whole job over all ranks). The same
line reports the Poisson-only solve rate in mixed and in FP64 precision at
the same final FP64 residual, the roofline of the dominant kernel (timed with
CUDA events inside the library during the timed steps) and the CPU oracle
timed on a bounded sample of the same device.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Multi-GPU: launched by torch.distributed.run; ranks solve independent
replicas of the device (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Poisson solves/s & op-apply HBM GB/s; mixed vs FP64 at same residual"
WORKLOAD = "dqd_128x128x96_4K"
NEV = 10
SAMPLE_N = (32, 32, 24)  # bounded CPU sample of the same device for the oracle timing
SP_PLUNGER_V = 0.70  # both plunger gates in the Schrodinger-Poisson measurement (about 2.6 electrons)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison solve")
    ap.add_argument("--no-sp", action="store_true", help="skip the self-consistent Schrodinger-Poisson solve")
    ap.add_argument("--no-calib", action="store_true", help="skip the interface-charge calibration")
    ap.add_argument("--sequential", action="store_true",
                    help="run the adjoint and the eigensolve one after the other (per-kernel profiles)")
    ap.add_argument("--cheb-degree", type=int, default=0,
                    help="Chebyshev degree of the Krylov solves (0: the mesh's autotuner chooses)")
    ap.add_argument("--launch", default=None,
                    help="variant,tile_rows,z_chunk of the FP32 operators instead of the autotuner's choice "
                         "(profiling runs, whose timings the profiler distorts)")
    return ap.parse_args()


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
# DRAM bytes (read + write) per launch of a kernel class from one ncu capture, keyed by the
# workload and the launch shape (variant, tile rows, z chunk) it was taken with; see
# profiles/apply32_dqd_128x128x96_4K.md for the command. Valid for the kernel source it was
# measured on: retake it when the kernel changes.
NCU_TRAFFIC = {("apply32", "dqd_128x128x96_4K", 3, 8, 16): 65.3e6,
               # both passes of one residual evaluation; profiles/residual_fp64_dqd_128x128x96_4K.md
               ("residual", "dqd_128x128x96_4K", 3, 8, 16): 440.7e6}

# FP64 floating-point operations per residual evaluation (2 per DFMA, 1 per DADD and DMUL,
# counted by ncu over both passes at the fourth residual of a solve; the count follows the
# carrier regime, i.e. how many quadrature points take the exponential branches), with the
# command in profiles/residual_fp64_dqd_128x128x96_4K.md.
NCU_FP64_FLOPS = {("residual", "dqd_128x128x96_4K"): 1006.2e6}

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


def oracle_sample(seconds_budget=30.0):
    """Times the oracle on the bounded sample device.

    Returns (wall seconds of one sample pass, nodes of the sample, effective cores). The oracle is
    plain numpy/scipy; its BLAS may run some products on several threads, so the cores it used are
    measured as process CPU time over wall time for the pass.
    """
    import workloads as W
    from oracle import capacitance as OC
    from oracle import schrodinger as OS
    from oracle.poisson import PoissonProblem
    dev = W.five_gate_device(n=SAMPLE_N, T=4.0)
    t0 = time.perf_counter()
    c0 = time.process_time()
    P = PoissonProblem(dev)
    phi, rep = P.solve()
    OC.electron_counts(P, phi)
    OC.adjoint(P, phi)
    OS.solve_device(P, phi, nev=NEV)
    dt = time.perf_counter() - t0
    cores = (time.process_time() - c0) / dt
    return dt, P.mesh.n_nodes, round(max(cores, 1.0), 2)


def reference_arm(args):
    """The oracle (plain FP64 CPU implementation) as the reference arm, on a bounded sample per step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import workloads as W
    full = W.n_nodes(W.get(args.workload))
    times, used = [], []
    nodes = None
    for s in range(args.warmup + args.steps):
        dt, nodes, cores = oracle_sample()
        if s >= args.warmup:
            times.append(dt)
            used.append(cores)
    t = sum(times) / len(times)
    value = (1.0 / t) * (nodes / full)
    sample = ("five-gate device %dx%dx%d elements (%d nodes), full pipeline per step; solves/s scaled by node ratio "
              "%d/%d; cores = process CPU time / wall time" % (SAMPLE_N + (nodes, nodes, full)))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "nodes": full, "sample": list(SAMPLE_N)},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": max(used), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def native_arm(args):
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
    mixed = q.make_opts(precision=1, cheb_degree=args.cheb_degree)  # 0: degree autotuned per mesh
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
    prof = {}
    for cls in q.PROF_CLASSES:
        nl, ms = q.qcad_profile_read(m, cls)
        prof[cls] = (nl, ms)
    # single-kernel classes with a roofline model (the multigrid tail is many small kernels)
    dom = max((c for c in prof if algorithmic_bytes(c, n_nodes, n_elems) is not None), key=lambda c: prof[c][1])
    total_ms = sum(v[1] for v in prof.values())
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
        return {"bound": "hbm", "kernel": cls, "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": (ach / peak) if ach else None,
                "traffic": NCU_TRAFFIC.get((cls, args.workload) + tune_key),
                "traffic_unit": "bytes per launch (ncu dram read + write, cold cache)",
                "peak_kind": peak_kind, "launches": nl, "avg_ms": ms / nl if nl else None,
                "timed_launches": "inside the Newton solves of the timed steps (no concurrent work)"}

    def fp64_roofline(cls):
        nl, ms = solve_prof[cls]
        flops = NCU_FP64_FLOPS.get((cls, args.workload))
        mhz = clk.get("sm_mhz") or 2070.0
        pk = FP64_FLOPS_PER_CLOCK * mhz * 1e6 / 1e12
        ach = flops / (ms / nl / 1000.0) / 1e12 if (nl and flops) else None
        return {"bound": "alu", "kernel": cls, "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                "frac": (ach / pk) if ach else None,
                "traffic": NCU_TRAFFIC.get((cls, args.workload) + tune_key),
                "traffic_unit": "bytes per evaluation (ncu dram read + write, cold cache, both passes)",
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
        rep_e = q.qcad_poisson_solve(m, b, mixed, phi)
        Ne = q.qcad_electron_counts(m, b, phi)
        dNe, Ee, _ = q.qcad_adjoint_eigs(m, b, phi, mixed, nev=NEV, tol=1e-8)
        phi_host.copy_(phi, non_blocking=True)
        torch.cuda.synchronize()
    t_e2e = max_over_ranks(dist, time.perf_counter() - t0, device="cuda")
    e2e = aggregate(args.steps, world, t_e2e)
    h2d = 8 * len(bias["V_gate"]) + 8 * 4  # gate voltages and bias scalars
    d2h = 8 * n_nodes + 8 * (len(N) + len(N) * len(bias["V_gate"]) + NEV)

    # Poisson-only: mixed vs FP64 at the same final FP64 residual
    def poisson_rate(opts, reps):
        ts = []
        r = None
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize()
            a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            r = q.qcad_poisson_solve(m, bias, opts, phi)
            b_.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b_) / 1000.0)
        return 1.0 / (sum(ts) / len(ts)), r

    mixed_rate, mixed_rep = poisson_rate(mixed, 3)
    phi_mixed = phi.clone()
    fp64 = None
    if not args.no_fp64:
        fp64_rate, fp64_rep = poisson_rate(q.make_opts(precision=0), 1)
        fp64 = {"solves_per_s": fp64_rate, "newton_iters": fp64_rep["newton_iters"],
                "krylov_iters": fp64_rep["krylov_iters_total"], "final_res_inf": fp64_rep["final_res_inf"],
                "max_abs_dphi_vs_mixed_V": float(torch.max(torch.abs(phi - phi_mixed)).item())}

    # Self-consistent Schrodinger-Poisson solve (Sec. II.C predictor-corrector, V_xc on) of the same
    # device with both plungers at SP_PLUNGER_V (a few electrons in the dot levels), to the paper's
    # potential tolerance 1e-5 V; timed with CUDA events around the whole call
    sp = None
    if not args.no_sp:
        sp_bias = dict(bias, V_gate=list(bias["V_gate"]))
        sp_bias["V_gate"][1] = sp_bias["V_gate"][3] = SP_PLUNGER_V
        phi_sp = torch.zeros(n_nodes, dtype=torch.float64, device="cuda")
        ts, rep_sp, E_sp = [], None, None
        for _ in range(2):
            flush.zero_()
            torch.cuda.synchronize()
            a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            E_sp, rep_sp = q.qcad_sp_solve(m, sp_bias, phi_sp, mixed, nev=NEV, eig_tol=1e-8, tol_dphi=1e-5,
                                           max_iter=100, use_vxc=True, allow_not_converged=True)
            b_.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b_) / 1000.0)
        sp = {"workload": "%s, plungers %.2f V, %d states, V_xc on" % (args.workload, SP_PLUNGER_V, NEV),
              "seconds": min(ts), "sp_solves_per_s": 1.0 / min(ts), "status": rep_sp["status"],
              "sp_iters": rep_sp["sp_iters"], "final_dphi_V": rep_sp["dphi_inf"],
              "electrons_in_quantum_region": rep_sp["n_quantum"], "E_meV": [1e3 * e for e in E_sp]}

    # Interface-charge calibration (Sec. III): the uniform interface sheet that leaves one electron in
    # dot 0 at the step's gate voltages, Newton on the adjoint slope; timed around the whole call
    calib = None
    if not args.no_calib:
        pat = torch.tensor(W.interface_sheet_pattern(dev), dtype=torch.float64, device="cuda")
        ts, sig, crep = [], None, None
        for _ in range(2):
            flush.zero_()
            torch.cuda.synchronize()
            a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            sig, crep, _, _ = q.qcad_calibrate_sheet_charge(m, bias, pat, mixed, dot=0, target=1.0, tol_N=1e-6,
                                                            max_iter=30, allow_not_converged=True)
            b_.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b_) / 1000.0)
        calib = {"workload": "%s, dot 0 to 1 electron, uniform interface sheet" % args.workload,
                 "seconds": min(ts), "status": crep["status"], "solves": crep["iters"],
                 "sigma_per_cm2": sig * 1e14, "N": crep["N"]}

    cpu = None
    if rank == 0 and world == 1:
        dt, nodes, cores = oracle_sample()
        cpu_value = (1.0 / dt) * (nodes / n_nodes)
        cpu = {"value": cpu_value, "unit": "solves/s", "cores": cores, "kind": "oracle",
               "sample": "five-gate device %dx%dx%d elements (%d nodes), full pipeline; scaled by node ratio; "
                         "cores = process CPU time / wall time" % (SAMPLE_N + (nodes,))}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": args.workload, "nodes": n_nodes, "elements": n_elems,
                       "step": "mixed Newton Poisson (FP64 residual 1e-10) + dot counts + 2x5 adjoint capacitance + %d LOBPCG eigenpairs" % NEV,
                       "l2": "flushed between timed steps (256 MB write)", "parallelism": "replicas x%d" % world,
                       "apply_launch": {"variant": tune32[0], "tile_rows": tune32[1], "z_chunk": tune32[2],
                                        "chosen_by": "--launch" if args.launch else "autotuner"},
                       "cheb_degree": args.cheb_degree or q.qcad_launch_info(m, 2)[3],
                       "adjoint_eigensolve": "sequential" if args.sequential else "concurrent (two streams)"},
            "roofline": roof,
            "alu_peaks": dict(alu, kind="microbenchmarks on this GPU: FMA chains (2 flops per FMA), FP64 exp()"),
            "op_apply_roofline": op_apply,
            "kernel_profile_ms": {c: round(v[1], 3) for c, v in prof.items()},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clk,
            "schrodinger_poisson": sp,
            "interface_charge_calibration": calib,
            "poisson_only": {"mixed": {"solves_per_s": mixed_rate, "newton_iters": mixed_rep["newton_iters"],
                                       "krylov_iters": mixed_rep["krylov_iters_total"],
                                       "final_res_inf": mixed_rep["final_res_inf"]},
                             "fp64": fp64},
            "results": {"newton_iters": rep["newton_iters"], "krylov_iters": rep["krylov_iters_total"],
                        "final_res_inf": rep["final_res_inf"], "dot_electrons": N,
                        "capacitance_aF": [[1.602176634e-1 * x for x in row] for row in dNdV],
                        "E_meV": [1e3 * e for e in E], "lobpcg_iters": erep["krylov_iters_total"]},
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    else:
        native_arm(args)


if __name__ == "__main__":
    main()
