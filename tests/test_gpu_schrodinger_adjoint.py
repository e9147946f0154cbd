"""GPU parity of the Schrodinger operators, LOBPCG, capacitance and adjoint against the oracle.

Tolerances: H and M applies 1e-12 relative (FP64), 2e-6 (FP32 apply);
eigenvalues 1e-9 relative; eigenvectors compared through principal angles of
each (near-)degenerate cluster; adjoint gate sensitivities and fixed-charge
gradients 1e-8 relative to the largest entry; finite-difference capacitance
1e-6 relative (two Newton solves to the FP64 residual 1e-10 on each side).
"""
import copy

import numpy as np
import pytest
import scipy.linalg
import torch

import workloads as W
from oracle import capacitance as OC
from oracle import schrodinger as OS
from oracle.poisson import PoissonProblem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1403_7561_gb300 as qcad
    return qcad


def dt(a):
    return torch.tensor(np.asarray(a, dtype=np.float64), device="cuda")


@pytest.fixture(scope="module")
def dqd(q):
    dev = W.five_gate_device(n=(32, 32, 24), T=4.0)
    P = PoissonProblem(dev)
    phi, rep = P.solve()
    assert rep["converged"]
    return dev, P, phi


@pytest.mark.parametrize("precision", [0, 1])
def test_hm_apply(q, dqd, precision):
    dev, P, phi = dqd
    me = (0.19, 0.21, 0.9)
    sel = P.mesh.subdomain_elements()
    inter = P.mesh.subdomain_interior_nodes()
    Vq = OS.device_potential(P, phi, sel)
    H, M, idx = OS.operators(P.mesh, sel, inter, me, Vq)
    m = q.qcad_mesh_create(dev)
    assert m.n_sub_dof == len(idx)
    rng = np.random.default_rng(7)
    X = rng.standard_normal((3, len(idx)))
    HX = torch.empty(3, len(idx), dtype=torch.float64, device="cuda")
    MX = torch.empty_like(HX)
    q.qcad_schrodinger_apply(m, dev["bias"], dt(phi), me, dt(X), HX, MX, precision)
    tol = 1e-12 if precision == 0 else 2e-6
    for j in range(3):
        ho, mo = H @ X[j], M @ X[j]
        assert np.max(np.abs(HX[j].cpu().numpy() - ho)) <= tol * np.max(np.abs(ho))
        assert np.max(np.abs(MX[j].cpu().numpy() - mo)) <= tol * np.max(np.abs(mo))


def test_lobpcg_matches_oracle_eigenpairs(q, dqd):
    dev, P, phi = dqd
    nev = 6
    Eo, Xo, idx, H, M = OS.solve_device(P, phi, nev=nev)
    m = q.qcad_mesh_create(dev)
    V = torch.empty(nev, m.n_sub_dof, dtype=torch.float64, device="cuda")
    E, rep = q.qcad_schrodinger_eigs(m, dev["bias"], dt(phi), nev=nev, tol=1e-8, evecs=V)
    assert rep["status"] == "OK", rep
    assert np.max(np.abs(np.array(E) - Eo) / np.abs(Eo)) < 1e-9
    Xg = V.cpu().numpy().T
    # M-orthonormal
    G = Xg.T @ (M @ Xg)
    assert np.max(np.abs(G - np.eye(nev))) < 1e-8
    # subspaces of each cluster of (near-)equal eigenvalues agree; a cluster reaching the
    # last computed pair may continue beyond nev and is not unique, so it is skipped
    start = 0
    while start < nev:
        end = start + 1
        while end < nev and abs(Eo[end] - Eo[start]) < 1e-8 * abs(Eo[start]):
            end += 1
        if end == nev:
            break
        # cosines of the principal angles between M-orthonormal bases
        sv = scipy.linalg.svdvals(Xo[:, start:end].T @ (M @ Xg[:, start:end]))
        assert np.min(sv) > 1 - 1e-7
        start = end


def test_lobpcg_soft_locking_leaves_the_eigenpairs(q, dqd, monkeypatch):
    # soft locking (columns of the FP64 phase already at the tolerance get no new search
    # directions) changes the work per iteration, not the answer: with and without it the
    # eigenvalues match the oracle's and each other
    dev, P, phi = dqd
    nev = 6
    Eo = OS.solve_device(P, phi, nev=nev)[0]
    m = q.qcad_mesh_create(dev)
    got = {}
    for lock in ("1", "0"):
        monkeypatch.setenv("QCAD_LOBPCG_LOCK", lock)
        E, rep = q.qcad_schrodinger_eigs(m, dev["bias"], dt(phi), nev=nev, tol=1e-8)
        assert rep["status"] == "OK", (lock, rep)
        got[lock] = np.array(E)
        assert np.max(np.abs(got[lock] - Eo) / np.abs(Eo)) < 1e-9, lock
    assert np.max(np.abs(got["1"] - got["0"]) / np.abs(Eo)) < 1e-9


def test_particle_in_box_closed_form(q):
    # vacuum-flat potential: a linear solve with equal gate voltages and no charge gives V ~ const near the top;
    # use an all-Si slab with grounded contacts so phi = phi_ohm everywhere and V is constant
    dev = dict(Lx=20.0, Ly=16.0, nx=10, ny=8, layers=[dict(material=0, thickness=12.0, n=6)],
               materials=[dict(W.SI, N_A=0.0, N_D=0.0)], gates=[], gate_work_function=None, bottom_ohmic=0,
               dots=[], subdomain=dict(i0=0, i1=10, j0=0, j1=8, k0=0, k1=6),
               bias=dict(T=4.0, V_gate=[], V_sub=0.0, statistics=1, incomplete_ionization=1))
    m = q.qcad_mesh_create(dev)
    phi = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    me = (0.19, 0.3, 0.98)
    E, rep = q.qcad_schrodinger_eigs(m, dev["bias"], phi, nev=5, m_eff=me, tol=1e-9)
    from oracle import physics
    import itertools, math
    P = PoissonProblem(dev)
    V0 = P.phi_r - P.si["chi"]
    h2m = physics.hbar2_over_2m0()
    ev = []
    for ks in itertools.product(range(1, 10), range(1, 8), range(1, 6)):
        lam = V0
        for k, Ld, nd, md in zip(ks, (20.0, 16.0, 12.0), (10, 8, 6), me):
            h = Ld / nd
            t = k * math.pi * h / Ld
            lam += h2m / md * 6.0 / h ** 2 * (1 - math.cos(t)) / (2 + math.cos(t))
        ev.append(lam)
    ev = np.sort(ev)[:5]
    assert np.max(np.abs(np.array(E) - ev) / np.abs(ev)) < 1e-10


@pytest.mark.parametrize("precision,degree", [(0, 1), (0, -1), (1, 1), (1, -1)])
def test_adjoint_matches_oracle(q, dqd, precision, degree):
    dev, P, phi = dqd
    theta = np.array(W.interface_fixed_charge(dev, seed=5))
    Pt = PoissonProblem(dev, fixed_charge=theta)
    phi_t, rep = Pt.solve(phi0=phi)
    dNdV_o, dNdq_o = OC.adjoint(Pt, phi_t)
    m = q.qcad_mesh_create(dev)
    th = dt(theta)
    phig = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    # degree 1: Jacobi (the dots' mixed-precision systems solved together); -1: multigrid (FP32 or FP64)
    opts = q.make_opts(precision=precision, cheb_degree=degree)
    r = q.qcad_poisson_solve(m, dev["bias"], opts, phig, fixed_charge=th)
    assert r["status"] == "OK"
    dq = torch.empty(m.n_dots * m.n_elems, dtype=torch.float64, device="cuda")
    dNdV = np.array(q.qcad_adjoint(m, dev["bias"], phig, opts, fixed_charge=th, dN_dq=dq))
    assert np.max(np.abs(dNdV - dNdV_o)) <= 1e-8 * np.max(np.abs(dNdV_o))
    g = dq.cpu().numpy().reshape(m.n_dots, m.n_elems)
    assert np.max(np.abs(g - dNdq_o)) <= 1e-8 * np.max(np.abs(dNdq_o))


@pytest.mark.parametrize("degree", [1, -1])
def test_bias_sweep_in_one_batched_launch(q, dqd, degree):
    # a plunger sweep of one device: each bias point an instance of the batched Newton (a mesh per
    # point), then each point's dot counts and 2x5 dN/dV from the adjoint, against the oracle
    dev, P, phi = dqd
    biases = []
    for dv in (-0.05, 0.0, 0.05):
        b = copy.deepcopy(dev["bias"])
        b["V_gate"][1] += dv
        biases.append(b)
    meshes = [q.qcad_mesh_create(dev) for _ in biases]
    phis = [torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda") for m in meshes]
    opts = q.make_opts(precision=1, cheb_degree=degree)
    reps, status = q.qcad_poisson_solve_batch(meshes, biases, opts, phis)
    assert status == "OK", reps
    # every point's 2 x 5 dN/dV from one batched adjoint call (the 3 x 2 systems in one batched PCG)
    batched = q.qcad_adjoint_batch(meshes, biases, q.make_opts(precision=1), phis)
    assert len(batched) == 3
    N0 = []
    for m, b, ph, dNdV_b in zip(meshes, biases, phis, batched):
        Pb = PoissonProblem(dev, bias=b)
        phi_o, rep = Pb.solve(phi0=phi)
        assert rep["converged"]
        assert np.max(np.abs(ph.cpu().numpy() - phi_o)) <= 1e-9
        N = np.array(q.qcad_electron_counts(m, b, ph))
        N_o = OC.electron_counts(Pb, phi_o)
        assert np.max(np.abs(N - N_o)) <= 1e-8 * np.max(np.abs(N_o))
        dNdV_o, _ = OC.adjoint(Pb, phi_o)
        assert np.max(np.abs(np.array(dNdV_b) - dNdV_o)) <= 1e-8 * np.max(np.abs(dNdV_o))
        dNdV = np.array(q.qcad_adjoint(m, b, ph, opts))
        assert np.max(np.abs(dNdV - dNdV_o)) <= 1e-8 * np.max(np.abs(dNdV_o))
        N0.append(N[0])
    assert N0[0] < N0[1] < N0[2]                                 # dot 0 fills as its plunger rises


def test_adjoint_batch_rejects_bad_batches(q, dqd):
    dev, P, phi = dqd
    m = q.qcad_mesh_create(dev)
    ph = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    q.qcad_poisson_solve(m, dev["bias"], q.make_opts(precision=1), ph)
    for opts, meshes in ((q.make_opts(precision=0), [m]), (q.make_opts(precision=1), [m, m])):
        with pytest.raises(q.QcadError) as e:
            q.qcad_adjoint_batch(meshes, [dev["bias"]] * len(meshes), opts, [ph] * len(meshes))
        assert e.value.code == 1
    # one mesh: the batched call equals the single-mesh adjoint
    one = np.array(q.qcad_adjoint_batch([m], [dev["bias"]], q.make_opts(precision=1), [ph])[0])
    ref = np.array(q.qcad_adjoint(m, dev["bias"], ph, q.make_opts(precision=1)))
    assert np.max(np.abs(one - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_fd_capacitance_matches_oracle(q, dqd):
    dev, P, phi = dqd
    Co, N1, N2 = OC.fd_capacitance(dev, gate=1, dV=0.01)
    m = q.qcad_mesh_create(dev)
    Cg = q.qcad_capacitance(m, dev["bias"], gate=1, dV=0.01)
    assert np.all(np.array(Co) > 0)
    assert np.max(np.abs(np.array(Cg) - Co) / np.abs(Co)) < 1e-6


def test_dot_charge_autograd(q, dqd):
    # QcadDotCharge: forward = solve + counts; backward = adjoint, checked against central
    # differences of the forward map (h = 1e-4 V, and a random direction in theta)
    dev, P, phi = dqd
    m = q.qcad_mesh_create(dev)
    opts = q.make_opts(precision=0)
    V = torch.tensor(dev["bias"]["V_gate"], dtype=torch.float64, requires_grad=True)
    theta = torch.tensor(np.array(W.interface_fixed_charge(dev, seed=5)), device="cuda", requires_grad=True)
    N = q.QcadDotCharge.apply(V, theta, m, dev["bias"], opts)
    assert N.shape == (m.n_dots,)
    w = torch.tensor([1.0, -0.5], dtype=torch.float64)
    (N * w).sum().backward()

    def f(v, th):
        with torch.no_grad():
            return (q.QcadDotCharge.apply(v, th, m, dev["bias"], opts) * w).sum().item()

    h = 1e-4
    for gi in range(len(V)):
        e = torch.zeros_like(V)
        e[gi] = h
        fd = (f(V.detach() + e, theta.detach()) - f(V.detach() - e, theta.detach())) / (2 * h)
        assert abs(V.grad[gi].item() - fd) <= 1e-5 * max(1.0, abs(fd)), gi
    rng = np.random.default_rng(8)
    d = torch.tensor(rng.standard_normal(m.n_elems), device="cuda") * theta.detach().abs().max()
    ht = 1e-2
    fd = (f(V.detach(), theta.detach() + ht * d) - f(V.detach(), theta.detach() - ht * d)) / (2 * ht)
    ad = torch.dot(theta.grad, d).item()
    assert abs(ad - fd) <= 1e-5 * max(abs(fd), abs(ad))


def test_adjoint_and_eigs_concurrently(q, dqd):
    # qcad_adjoint_eigs (eigensolve on a second stream and host thread) gives the results of the
    # two calls made one after the other
    dev, P, phi = dqd
    theta = np.array(W.interface_fixed_charge(dev, seed=5))
    m = q.qcad_mesh_create(dev)
    th = dt(theta)
    phig = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    q.qcad_poisson_solve(m, dev["bias"], q.make_opts(precision=1), phig, fixed_charge=th)
    opts = q.make_opts(precision=1)
    dq1 = torch.empty(m.n_dots * m.n_elems, dtype=torch.float64, device="cuda")
    V1 = np.array(q.qcad_adjoint(m, dev["bias"], phig, opts, fixed_charge=th, dN_dq=dq1))
    E1, _ = q.qcad_schrodinger_eigs(m, dev["bias"], phig, nev=6, tol=1e-9)
    for _ in range(2):
        dq2 = torch.empty_like(dq1)
        V2, E2, rep = q.qcad_adjoint_eigs(m, dev["bias"], phig, opts, fixed_charge=th, dN_dq=dq2, nev=6, tol=1e-9)
        assert rep["status"] == "OK"
        assert np.max(np.abs(np.array(V2) - V1)) <= 1e-12 * np.max(np.abs(V1))
        assert torch.max(torch.abs(dq2 - dq1)).item() <= 1e-12 * torch.max(torch.abs(dq1)).item()
        assert np.max(np.abs(np.array(E2) - E1) / np.abs(E1)) <= 1e-10
    # errors of either half surface as the call's status
    with pytest.raises(q.QcadError):
        q.qcad_adjoint_eigs(m, dev["bias"], phig, opts, nev=17)


# ---------------------------------------------------------------------------
# Self-consistent Schrodinger-Poisson loop (Sec. II.C), against the oracle's loop.

def sp_device():
    # plungers that put about ten electrons in the dot levels, the sixth level still empty
    dev = W.five_gate_device(n=(16, 16, 12), T=4.0)
    V = list(dev["bias"]["V_gate"])
    V[1] = V[3] = 0.9
    dev["bias"]["V_gate"] = V
    return dev


@pytest.fixture(scope="module")
def sp_oracle_k3():
    from oracle import sp as OSP
    dev = sp_device()
    return dev, OSP.sp_solve(dev, nev=6, fixed_iters=3)


@pytest.mark.parametrize("precision", [0, 1])
def test_sp_iterations_match_oracle(q, sp_oracle_k3, precision):
    # three predictor-corrector iterations: the same potential, levels, density and history
    dev, (phi_o, E_o, rep_o) = sp_oracle_k3
    m = q.qcad_mesh_create(dev)
    phi = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    E, rep = q.qcad_sp_solve(m, dev["bias"], phi, q.make_opts(precision=precision), nev=6, eig_tol=1e-10,
                             tol_dphi=0.0, max_iter=3)
    assert rep["status"] == "OK" and rep["sp_iters"] == 3
    assert np.max(np.abs(phi.cpu().numpy() - phi_o)) <= 1e-9
    assert np.max(np.abs(np.array(E) - E_o)) <= 1e-10          # eV; levels sit near E_F = 0
    assert abs(rep["n_quantum"] - rep_o["n_quantum"]) <= 1e-8 * rep_o["n_quantum"]
    assert np.max(np.abs(np.array(rep["dphi_hist"]) - np.array(rep_o["dphi"]))) <= 1e-9
    assert np.max(np.abs(np.array(rep["e1_hist"]) - np.array(rep_o["E1"]))) <= 1e-10


def test_sp_converges_to_the_oracle_fixed_point(q):
    from oracle import sp as OSP
    dev = sp_device()
    phi_o, E_o, rep_o = OSP.sp_solve(dev, nev=6, tol=1e-8, max_iter=80)
    m = q.qcad_mesh_create(dev)
    phi = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    E, rep = q.qcad_sp_solve(m, dev["bias"], phi, q.make_opts(precision=1), nev=6, eig_tol=1e-10, tol_dphi=1e-8,
                             max_iter=80)
    assert rep["status"] == "OK" and rep["converged"]
    d = np.array(rep["dphi_hist"])
    assert np.all(d[2:] <= d[1:-1] * (1 + 1e-6))                # monotonic after the first correction
    assert np.max(np.abs(phi.cpu().numpy() - phi_o)) <= 1e-7     # both within 1e-8 of one fixed point
    assert np.max(np.abs(np.array(E) - E_o)) <= 1e-8


def test_sp_depleted_dot_and_bad_arguments(q):
    # default gates: every level sits tens of meV above E_F, the quantum region holds no electrons
    dev = W.five_gate_device(n=(16, 16, 12), T=4.0)
    m = q.qcad_mesh_create(dev)
    phi = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    E, rep = q.qcad_sp_solve(m, dev["bias"], phi, q.make_opts(precision=1), nev=4, tol_dphi=1e-6, max_iter=10)
    assert rep["status"] == "OK" and rep["sp_iters"] <= 3
    assert rep["n_quantum"] < 1e-20 and min(E) > 0.02
    for kw in (dict(nev=0), dict(nev=17), dict(max_iter=0), dict(eig_tol=0.0)):
        args = dict(nev=4, tol_dphi=1e-6, max_iter=3)
        args.update(kw)
        with pytest.raises(q.QcadError) as e:
            q.qcad_sp_solve(m, dev["bias"], phi, q.make_opts(precision=1), **args)
        assert e.value.code == 1
    # the mesh's own Poisson solve is semiclassical again after the loop
    rep2 = q.qcad_poisson_solve(m, dev["bias"], q.make_opts(precision=1), phi)
    from oracle.poisson import PoissonProblem
    phi_o, _ = PoissonProblem(dev).solve()
    assert np.max(np.abs(phi.cpu().numpy() - phi_o)) <= 1e-9


@pytest.mark.parametrize("precision", [0, 1])
def test_sheet_charge_calibration_matches_oracle(q, precision):
    # Sec. III: the interface charge that leaves one electron in the dot, by Newton on the adjoint
    # slope here and by a bracketed root find on the oracle
    dev = W.five_gate_device(n=(12, 12, 8), T=4.0, with_subdomain=False)
    pat = np.array(W.interface_sheet_pattern(dev))
    sig_o, N_o, phi_o = OC.calibrate_sheet_charge(dev, 0, 1.0, pat)
    m = q.qcad_mesh_create(dev)
    sig, rep, phi, theta = q.qcad_calibrate_sheet_charge(m, dev["bias"], dt(pat),
                                                         q.make_opts(precision=precision, cheb_degree=0),
                                                         dot=0, target=1.0, tol_N=1e-10, max_iter=30)
    assert rep["status"] == "OK" and rep["converged"] and rep["iters"] <= 12, rep
    assert abs(rep["N"] - 1.0) <= 1e-10
    assert abs(sig - sig_o) <= 1e-9 * abs(sig_o)
    assert np.max(np.abs(phi.cpu().numpy() - phi_o)) <= 1e-8
    assert np.max(np.abs(theta.cpu().numpy() - sig * pat)) <= 1e-15 * np.max(np.abs(sig * pat))
