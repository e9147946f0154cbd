"""GPU parity of the Poisson path against the FP64 oracle (run on a GB300).

Every test calls the CUDA library through its C ABI (via the ctypes binding)
and compares with the oracle on the same seeded inputs, element by element.
Tolerances: potentials 1e-9 V (FP64 and mixed at the final FP64 residual
1e-10); residual and FP64 Jacobian applies to 1e-12 relative to the largest
entry; FP32 applies to 2e-6 relative (single precision).
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import capacitance as OC
from oracle.poisson import PoissonProblem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1403_7561_gb300 as qcad
    return qcad


def dev_tensor(a):
    return torch.tensor(np.asarray(a, dtype=np.float64), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


CASES = {
    "mos_cap_16x16x32": lambda: W.get("mos_cap_16x16x32"),
    "dqd_24x24x16_4K": lambda: W.five_gate_device(n=(24, 24, 16), T=4.0),
    "dqd_37x33x21_0p5K": lambda: W.five_gate_device(n=(37, 33, 21), T=0.5),     # ragged tiles
    "dqd_3x1x7_4K": lambda: W.five_gate_device(n=(3, 1, 7), T=4.0, with_subdomain=False),
    "tiny_1x1x2": lambda: W.mos_capacitor(nx=1, ny=1, nz=2, n_ox=1),
    "dqd_61x62x40_4K": lambda: W.five_gate_device(n=(61, 62, 40), T=4.0),        # several tiles, ragged
}


def perturbed_phi(P, seed, amp=0.01):
    phi = P.initial_guess()
    rng = np.random.default_rng(seed)
    phi[P.free] += amp * rng.standard_normal(P.free.sum())
    return phi


@pytest.mark.parametrize("name", list(CASES))
def test_contact_values(q, name):
    dev = CASES[name]()
    P = PoissonProblem(dev)
    m = q.qcad_mesh_create(dev)
    phi = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    gv, ov = q.qcad_contact_values(m, dev["bias"], phi)
    assert abs(ov - P.phi_ohm) < 1e-13
    g = host(phi)
    assert np.max(np.abs(g[P.dir] - P.g[P.dir])) < 1e-13
    assert np.all(g[P.free] == 0.0)


@pytest.mark.parametrize("name", list(CASES))
def test_residual_and_diagonal(q, name):
    dev = CASES[name]()
    P = PoissonProblem(dev)
    m = q.qcad_mesh_create(dev)
    phi_np = perturbed_phi(P, 1)
    phi = dev_tensor(phi_np)
    R = torch.empty_like(phi)
    D = torch.empty_like(phi)
    rmax, r2 = q.qcad_poisson_residual(m, dev["bias"], phi, R, D)
    Ro = P.residual(phi_np)
    scale = max(np.max(np.abs(Ro)), np.max(np.abs(P.K @ phi_np)))
    assert np.max(np.abs(host(R) - Ro)) <= 1e-12 * scale
    assert abs(rmax - np.max(np.abs(Ro))) <= 1e-12 * scale
    assert abs(r2 - np.sum(Ro * Ro)) <= 1e-10 * max(np.sum(Ro * Ro), 1e-300)
    Jd = P.jacobian(phi_np).diagonal()
    Jd[P.dir] = 1.0
    assert np.max(np.abs(host(D) - Jd) / np.abs(Jd)) < 1e-12


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", [0, 1])
def test_jacobian_apply(q, name, precision):
    dev = CASES[name]()
    P = PoissonProblem(dev)
    m = q.qcad_mesh_create(dev)
    phi_np = perturbed_phi(P, 2)
    rng = np.random.default_rng(3)
    v_np = rng.standard_normal(P.mesh.n_nodes)
    v_np[P.dir] = 0.0
    y = torch.empty(P.mesh.n_nodes, dtype=torch.float64, device="cuda")
    q.qcad_poisson_jv(m, dev["bias"], dev_tensor(phi_np), dev_tensor(v_np), y, precision)
    yo = P.jacobian(phi_np) @ v_np
    yo[P.dir] = 0.0
    tol = 1e-12 if precision == 0 else 2e-6
    assert np.max(np.abs(host(y) - yo)) <= tol * np.max(np.abs(yo))


@pytest.mark.parametrize("name", ["mos_cap_16x16x32", "dqd_24x24x16_4K", "dqd_37x33x21_0p5K", "dqd_3x1x7_4K",
                                  "tiny_1x1x2"])
@pytest.mark.parametrize("precision", [0, 1])
def test_newton_solve_matches_oracle(q, name, precision):
    dev = CASES[name]()
    P = PoissonProblem(dev)
    phi_o, rep_o = P.solve()
    assert rep_o["converged"]
    m = q.qcad_mesh_create(dev)
    phi = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    rep = q.qcad_poisson_solve(m, dev["bias"], q.make_opts(precision=precision), phi)
    assert rep["status"] == "OK", rep
    assert rep["final_res_inf"] < 1e-10 and rep["final_dphi_inf"] < 1e-10
    assert np.max(np.abs(host(phi) - phi_o)) <= 1e-9
    # the oracle's residual of the GPU solution
    assert np.max(np.abs(P.residual(host(phi)))) < 1e-9


@pytest.mark.parametrize("name", ["dqd_37x33x21_0p5K", "dqd_61x62x40_4K", "dqd_3x1x7_4K"])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_jacobian_apply_every_launch_shape(q, name, precision, variant):
    # every kernel variant and tile shape, z chunks from 1 plane to more than the mesh
    dev = CASES[name]()
    P = PoissonProblem(dev)
    m = q.qcad_mesh_create(dev)
    phi_np = perturbed_phi(P, 4)
    rng = np.random.default_rng(5)
    v_np = rng.standard_normal(P.mesh.n_nodes)
    v_np[P.dir] = 0.0
    yo = P.jacobian(phi_np) @ v_np
    yo[P.dir] = 0.0
    tol = 1e-12 if precision == 0 else 2e-6
    y = torch.empty(P.mesh.n_nodes, dtype=torch.float64, device="cuda")
    for rows, ch in ((4, 3), (8, 16), (16, 1), (32, 64), (8, 2)):
        q.qcad_set_launch(m, 2 if precision else 1, variant, rows, ch)
        y.fill_(float("nan"))
        q.qcad_poisson_jv(m, dev["bias"], dev_tensor(phi_np), dev_tensor(v_np), y, precision)
        assert np.max(np.abs(host(y) - yo)) <= tol * np.max(np.abs(yo)), (rows, ch)


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_is_independent_of_launch_configuration(q, precision):
    dev = CASES["dqd_37x33x21_0p5K"]()
    m = q.qcad_mesh_create(dev)
    ref = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    q.qcad_poisson_solve(m, dev["bias"], q.make_opts(precision=precision), ref)
    for variant in (0, 1, 2, 3):
        for degree in (1, 3):
            for rows, ch in ((4, 3), (16, 64), (8, 1)):
                for fam in (0, 1, 2):
                    q.qcad_set_launch(m, fam, variant, rows, ch)
                phi = torch.zeros_like(ref)
                q.qcad_poisson_solve(m, dev["bias"], q.make_opts(precision=precision, cheb_degree=degree), phi)
                assert torch.max(torch.abs(phi - ref)).item() <= 1e-9, (variant, degree, rows, ch)


def test_electron_counts_and_fixed_charge(q):
    dev = CASES["dqd_24x24x16_4K"]()
    theta = np.array(W.interface_fixed_charge(dev, seed=5))
    P = PoissonProblem(dev, fixed_charge=theta)
    phi_o, _ = P.solve()
    m = q.qcad_mesh_create(dev)
    th = dev_tensor(theta)
    phi = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    rep = q.qcad_poisson_solve(m, dev["bias"], q.make_opts(), phi, fixed_charge=th)
    assert rep["status"] == "OK"
    assert np.max(np.abs(host(phi) - phi_o)) <= 1e-9
    N = q.qcad_electron_counts(m, dev["bias"], phi, fixed_charge=th)
    No = OC.electron_counts(P, phi_o)
    assert np.all(No > 0.1)
    assert np.max(np.abs(np.array(N) - No) / No) < 1e-8


def test_invalid_arguments_are_rejected(q):
    dev = CASES["tiny_1x1x2"]()
    m = q.qcad_mesh_create(dev)
    phi = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    bad = dict(dev["bias"], V_gate=[0.1, 0.2])
    with pytest.raises(q.QcadError) as e:
        q.qcad_poisson_solve(m, bad, q.make_opts(), phi)
    assert e.value.code == 1
    with pytest.raises(q.QcadError):
        q.qcad_poisson_solve(m, dict(dev["bias"], T=-1.0), q.make_opts(), phi)
    with pytest.raises(q.QcadError):
        q.qcad_set_launch(m, 0, 0, 5, 16)
    with pytest.raises(q.QcadError):
        q.qcad_set_launch(m, 2, 4, 8, 16)
    bad_dev = dict(dev, nx=0)
    with pytest.raises(q.QcadError):
        q.qcad_mesh_create(bad_dev)


def test_not_converged_is_reported(q):
    dev = CASES["dqd_24x24x16_4K"]()
    m = q.qcad_mesh_create(dev)
    phi = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    rep = q.qcad_poisson_solve(m, dev["bias"], q.make_opts(max_newton=1), phi, allow_not_converged=True)
    assert rep["status"] == "NOT_CONVERGED"
    assert rep["newton_iters"] == 1
    assert torch.isfinite(phi).all()


@pytest.mark.parametrize("name", ["dqd_24x24x16_4K", "dqd_37x33x21_0p5K", "mos_cap_16x16x32"])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("degree", [2, 3, 5, 0])
def test_chebyshev_preconditioned_solve(q, name, precision, degree):
    # Chebyshev-Jacobi PCG (degree 0 = autotuned) converges to the same unique solution
    dev = CASES[name]()
    P = PoissonProblem(dev)
    phi_o, rep_o = P.solve()
    m = q.qcad_mesh_create(dev)
    phi = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    rep = q.qcad_poisson_solve(m, dev["bias"], q.make_opts(precision=precision, cheb_degree=degree), phi)
    assert rep["status"] == "OK", rep
    assert np.max(np.abs(host(phi) - phi_o)) <= 1e-9


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", [0, 1])
def test_multigrid_preconditioned_solve(q, name, precision):
    # geometric multigrid V-cycle PCG (FP32 V-cycle in mixed precision, FP64 V-cycle in plain
    # FP64) converges to the same unique solution; meshes too small for a coarse level fall back
    # to Jacobi
    dev = CASES[name]()
    P = PoissonProblem(dev)
    phi_o, rep_o = P.solve()
    m = q.qcad_mesh_create(dev)
    phi = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    rep = q.qcad_poisson_solve(m, dev["bias"], q.make_opts(precision=precision, cheb_degree=-1), phi)
    assert rep["status"] == "OK", rep
    assert np.max(np.abs(host(phi) - phi_o)) <= 1e-9
    if name == "dqd_61x62x40_4K":
        # the V-cycle needs several times fewer Krylov iterations than Jacobi on this mesh
        m2 = q.qcad_mesh_create(dev)
        phi2 = torch.zeros(m2.n_nodes, dtype=torch.float64, device="cuda")
        rep2 = q.qcad_poisson_solve(m2, dev["bias"], q.make_opts(precision=precision, cheb_degree=1), phi2)
        assert rep2["status"] == "OK", rep2
        assert 4 * rep["krylov_iters_total"] < rep2["krylov_iters_total"], (rep, rep2)


def test_multigrid_in_both_precisions_takes_the_same_path(q):
    # the FP64 and FP32 V-cycles are the same preconditioner in two precisions: the two Newton
    # solves of one device reach the same solution with Krylov counts within a few iterations
    dev = CASES["dqd_61x62x40_4K"]()
    reps, phis = [], []
    for prec in (0, 1):
        m = q.qcad_mesh_create(dev)
        phi = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
        reps.append(q.qcad_poisson_solve(m, dev["bias"], q.make_opts(precision=prec, cheb_degree=-1), phi))
        phis.append(host(phi))
    assert reps[0]["status"] == "OK" and reps[1]["status"] == "OK"
    assert np.max(np.abs(phis[0] - phis[1])) <= 1e-9
    k64, k32 = reps[0]["krylov_iters_total"], reps[1]["krylov_iters_total"]
    assert abs(k64 - k32) <= max(4, 0.25 * k64), (reps[0], reps[1])


def test_multigrid_option_is_validated(q):
    dev = CASES["dqd_24x24x16_4K"]()
    m = q.qcad_mesh_create(dev)
    phi = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    for prec, deg in ((0, -2), (1, -2), (1, 17), (0, 17)):
        with pytest.raises(q.QcadError) as e:
            q.qcad_poisson_solve(m, dev["bias"], q.make_opts(precision=prec, cheb_degree=deg), phi)
        assert e.value.code == 1


def batch_devices():
    # uneven sizes (ragged tiles, a mesh one tile wide) with their own seeds, so each
    # instance has its own gate voltages
    shapes = [(12, 12, 12), (20, 16, 12), (37, 33, 21), (8, 8, 16), (16, 16, 16)]
    return [W.five_gate_device(n=s, seed=7, stream=i, T=4.0, with_subdomain=False) for i, s in enumerate(shapes)]


@pytest.mark.parametrize("degree", [1, -1])
def test_batched_solve_matches_oracle(q, degree):
    # degree 1: one-launch batched Jacobi PCG; -1: each instance's multigrid PCG in lockstep
    devs = batch_devices()
    meshes = [q.qcad_mesh_create(d) for d in devs]
    phis = [torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda") for m in meshes]
    reps, status = q.qcad_poisson_solve_batch(meshes, [d["bias"] for d in devs],
                                              q.make_opts(precision=1, cheb_degree=degree), phis)
    assert status == "OK", reps
    for d, phi, rep in zip(devs, phis, reps):
        P = PoissonProblem(d)
        phi_o, rep_o = P.solve()
        assert rep_o["converged"]
        assert rep["final_res_inf"] < 1e-10 and rep["final_dphi_inf"] < 1e-10
        assert np.max(np.abs(host(phi) - phi_o)) <= 1e-9, (d["nx"], d["ny"])


@pytest.mark.parametrize("degree", [1, -1])
def test_batched_solve_agrees_with_single_solves_and_warm_starts(q, degree):
    devs = batch_devices()[:3]
    meshes = [q.qcad_mesh_create(d) for d in devs]
    phis = [torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda") for m in meshes]
    _, status = q.qcad_poisson_solve_batch(meshes, [d["bias"] for d in devs],
                                           q.make_opts(precision=1, cheb_degree=degree), phis)
    assert status == "OK"
    for d, m, phi in zip(devs, meshes, phis):
        one = torch.zeros_like(phi)
        q.qcad_poisson_solve(m, d["bias"], q.make_opts(precision=1), one)
        assert torch.max(torch.abs(one - phi)).item() <= 1e-9
    # warm start from the converged potentials: every instance stops after at most one step
    reps, status = q.qcad_poisson_solve_batch(meshes, [d["bias"] for d in devs],
                                              q.make_opts(precision=1, warm_start=1, cheb_degree=degree), phis)
    assert status == "OK"
    assert all(r["newton_iters"] <= 1 for r in reps)


def test_batched_solve_rejects_bad_batches(q):
    devs = batch_devices()[:2]
    meshes = [q.qcad_mesh_create(d) for d in devs]
    phis = [torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda") for m in meshes]
    biases = [d["bias"] for d in devs]
    with pytest.raises(q.QcadError) as e:
        q.qcad_poisson_solve_batch(meshes, biases, q.make_opts(precision=0), phis)
    assert e.value.code == 1
    with pytest.raises(q.QcadError):
        q.qcad_poisson_solve_batch([meshes[0], meshes[0]], [biases[0], biases[0]], q.make_opts(precision=1),
                                   [phis[0], phis[0]])
    # one instance capped at one Newton step is reported, the other converges
    reps, status = q.qcad_poisson_solve_batch(meshes, biases, q.make_opts(precision=1, max_newton=1), phis,
                                              allow_not_converged=True)
    assert status == "NOT_CONVERGED"
    assert all(r["newton_iters"] == 1 for r in reps)


def test_alu_peaks_are_plausible(q):
    # the FP64 pipe of this part runs at a small fraction of the FP32 rate; an exp() costs tens of
    # FP64 operations; a measured peak outside these bands means the microbenchmark lost its work
    p = q.qcad_alu_peaks()
    assert 0.3 < p["fp64_tflops"] < 5.0, p
    assert p["fp32_tflops"] > 10.0 * p["fp64_tflops"], p
    assert 1e9 < p["fp64_exp_per_s"] < p["fp64_tflops"] * 1e12, p
