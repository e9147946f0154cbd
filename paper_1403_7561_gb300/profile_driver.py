"""Workloads for kernel profiling (ncu) of the library.

``step``: launch autotuning, then one warm-up pass of the full hot path on a
device (mixed Newton with the autotuned preconditioner, dot counts, adjoint,
eigenpairs, one after the other), then one more pass inside the NVTX range
"step"; prints the library's kernel-launch counts.

``solve``: launch autotuning, then one mixed-precision Poisson solve with the
autotuned Chebyshev degree; used for captures of the PCG kernels
(``ncu -k regex:PcgApply -s <n> -c <k>``).

``apply``: the Jacobian apply of one precision on a device's linearization
at the Laplace initial guess, repeated; used for single-kernel captures.

``eigs``: one mixed Poisson solve, one warm-up eigensolve (10 eigenpairs to
1e-8), then one more inside the NVTX range "eigs"; used for launch lists of the
eigensolver (``ncu --nvtx --nvtx-include "eigs/"``).

``batch``: the 96-instance batch of uneven meshes (48^3 .. 112^3 elements, 61.7M
nodes): the batched Newton with each instance's multigrid PCG and with the
one-launch batched Jacobi PCG, and the same instances solved one after the
other; prints instances/s (wall clock around each call, best of three).

Usage:
  python -m paper_1403_7561_gb300.profile_driver step  [--workload NAME]
  python -m paper_1403_7561_gb300.profile_driver solve [--workload NAME]
  python -m paper_1403_7561_gb300.profile_driver apply [--workload NAME] [--precision 0|1] [--reps N]
  python -m paper_1403_7561_gb300.profile_driver eigs  [--workload NAME]
  python -m paper_1403_7561_gb300.profile_driver batch
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("mode", choices=["step", "solve", "apply", "eigs", "batch"])
    ap.add_argument("--workload", default="dqd_128x128x96_4K")
    ap.add_argument("--precision", type=int, default=1)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--launch", default=None, help="variant,tile_rows,z_chunk instead of the autotuner")
    a = ap.parse_args()
    import torch

    import paper_1403_7561_gb300 as q
    import workloads as W

    if a.mode == "batch":
        run_batch(q, W, torch)
        return
    dev = W.get(a.workload)
    bias = dev["bias"]
    m = q.qcad_mesh_create(dev)
    phi = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    if a.mode in ("step", "solve", "eigs"):
        if a.launch:
            v, r, c = (int(x) for x in a.launch.split(","))
            q.qcad_set_launch(m, 2, v, r, c)
        else:
            q.qcad_autotune(m, bias, precision=1)
        opts = q.make_opts(precision=1, cheb_degree=0)
    if a.mode == "eigs":
        q.qcad_poisson_solve(m, bias, opts, phi)
        evecs = torch.empty(10, m.n_sub_dof, dtype=torch.float64, device="cuda")
        q.qcad_schrodinger_eigs(m, bias, phi, nev=10, tol=1e-8, evecs=evecs)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("eigs")
        E, rep = q.qcad_schrodinger_eigs(m, bias, phi, nev=10, tol=1e-8, evecs=evecs)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print("eigs done: %d subdomain dof, %d FP32 + %d FP64 iterations" % (m.n_sub_dof, rep["newton_iters"],
                                                                           rep["status_detail"]))
    elif a.mode == "solve":
        rep = q.qcad_poisson_solve(m, bias, opts, phi)
        torch.cuda.synchronize()
        print("solve done: %d nodes, %d Newton, %d Krylov iterations" % (m.n_nodes, rep["newton_iters"],
                                                                          rep["krylov_iters_total"]))
    elif a.mode == "step":

        def step():
            q.qcad_poisson_solve(m, bias, opts, phi)
            q.qcad_electron_counts(m, bias, phi)
            q.qcad_adjoint(m, bias, phi, opts)
            q.qcad_schrodinger_eigs(m, bias, phi, nev=10, tol=1e-8)

        c0 = q.qcad_launch_count()
        step()
        c1 = q.qcad_launch_count()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("step")  # ncu --nvtx --nvtx-include "step/" keeps this pass only
        step()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        c2 = q.qcad_launch_count()
        torch.cuda.synchronize()
        print("launches warmup=%d step=%d" % (c1 - c0, c2 - c1))
    else:
        q.qcad_contact_values(m, bias, phi)
        v = torch.randn(m.n_nodes, dtype=torch.float64, device="cuda")
        y = torch.empty_like(v)
        for _ in range(a.reps):
            q.qcad_poisson_jv(m, bias, phi, v, y, a.precision)
        torch.cuda.synchronize()
        print("apply done: %d nodes, precision %d, %d reps" % (m.n_nodes, a.precision, a.reps))


def run_batch(q, W, torch):
    import time
    devs = W.batch_instances()
    nodes = sum(W.n_nodes(d) for d in devs)
    meshes = [q.qcad_mesh_create(d) for d in devs]
    phis = [torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda") for m in meshes]
    biases = [d["bias"] for d in devs]

    def timed(fn):
        best = None
        for _ in range(3):
            for p in phis:
                p.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out = fn()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        return best, out

    print("instances %d, nodes %d" % (len(devs), nodes))
    for name, deg in (("batched Newton, multigrid PCG per instance", -1), ("batched Newton, batched Jacobi PCG", 1)):
        dt, (reps, st) = timed(lambda: q.qcad_poisson_solve_batch(meshes, biases,
                                                                  q.make_opts(precision=1, cheb_degree=deg), phis))
        print("%s: %s, %.3f s, %.1f instances/s, Newton max %d, Krylov max %d" % (
            name, st, dt, len(devs) / dt, max(r["newton_iters"] for r in reps),
            max(r["krylov_iters_total"] for r in reps)))

    def sequential():
        for m, b, p in zip(meshes, biases, phis):
            q.qcad_poisson_solve(m, b, q.make_opts(precision=1, cheb_degree=-1), p)
        return None

    dt, _ = timed(sequential)
    print("one instance after the other, multigrid PCG: %.3f s, %.1f instances/s" % (dt, len(devs) / dt))


if __name__ == "__main__":
    main()
