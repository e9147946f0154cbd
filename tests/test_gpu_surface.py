"""GPU parity of the surface terms (Sec. II.A.4): charged gates under the Robin condition and
surface charges (Eq. NeuBC4fc), against the oracle.

Tolerances as for the Dirichlet devices: residual and J v 1e-12 relative to the largest entry
(FP64), Newton solutions 1e-9 V in both precisions, adjoint dN/dV 1e-8 relative, finite-difference
capacitance 1e-6 relative.
"""
import copy

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


def dt(a):
    return torch.tensor(np.asarray(a, dtype=np.float64), device="cuda")


def charged_device(n=(24, 24, 16), all_gates=False):
    """Five-gate stack at 4 K, plunger P2 charged (or every gate, each with its own sheet), and a
    surface-charge patch on the Si/SiO2 interface plane z = 90 nm."""
    dev = W.five_gate_device(n=n, T=4.0)
    dev["bias"]["V_gate"] = [0.35, 0.95, 0.45, 1.1, 0.3]
    if all_gates:
        for g, G in enumerate(dev["gates"]):
            G["robin"] = dict(sigma=(-1) ** g * 4e-4, d=5.0 + 2.0 * g)
    else:
        dev["gates"][3]["robin"] = dict(sigma=5e-4, d=10.0)
    dev["surface_charges"] = [dict(z=90.0, x0=100.0, x1=150.0, y0=50.0, y1=150.0, sigma=2e-3)]
    return dev


@pytest.fixture(scope="module")
def solved():
    out = {}
    for key, all_gates in (("one", False), ("all", True)):
        dev = charged_device(all_gates=all_gates)
        P = PoissonProblem(dev)
        phi, rep = P.solve()
        assert rep["converged"]
        out[key] = (dev, P, phi)
    return out


@pytest.mark.parametrize("key", ["one", "all"])
def test_residual_and_jv_match_oracle(q, solved, key):
    dev, P, phi = solved[key]
    m = q.qcad_mesh_create(dev)
    rng = np.random.default_rng(11)
    ph = phi.copy()
    ph[P.free] += 2e-3 * rng.standard_normal(P.free.sum())
    R = torch.empty(m.n_nodes, dtype=torch.float64, device="cuda")
    q.qcad_poisson_residual(m, dev["bias"], dt(ph), R)
    Ro = P.residual(ph)
    assert np.max(np.abs(R.cpu().numpy() - Ro)) <= 1e-12 * np.max(np.abs(Ro))
    v = np.zeros(m.n_nodes)
    v[P.free] = rng.standard_normal(P.free.sum())
    y = torch.empty(m.n_nodes, dtype=torch.float64, device="cuda")
    q.qcad_poisson_jv(m, dev["bias"], dt(ph), dt(v), y, precision=0)
    yo = P.jacobian(ph) @ v
    yo[P.dir] = 0.0
    yg = y.cpu().numpy()
    yg[P.dir] = 0.0
    assert np.max(np.abs(yg - yo)) <= 1e-12 * np.max(np.abs(yo))


@pytest.mark.parametrize("precision,degree", [(0, 1), (1, 1), (1, 3), (1, -1)])
def test_solve_matches_oracle(q, solved, precision, degree):
    # degree -1 asks for the multigrid preconditioner, which a mesh with charged gates replaces by
    # Jacobi; the mixed solves refine to the same FP64 residual
    for key in ("one", "all"):
        dev, P, phi = solved[key]
        m = q.qcad_mesh_create(dev)
        assert q.qcad_launch_info(m, 2)[0] == 0                  # the element-gather variant
        g = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
        rep = q.qcad_poisson_solve(m, dev["bias"], q.make_opts(precision=precision, cheb_degree=degree), g)
        assert rep["status"] == "OK"
        assert rep["final_res_inf"] < 1e-10
        assert np.max(np.abs(g.cpu().numpy() - phi)) <= 1e-9, key


def test_surface_charges_alone_keep_the_multigrid(q):
    # without charged gates the Jacobian is unchanged: the V-cycle and the fast kernels stay, only the
    # residual carries the sheet's load
    dev = W.five_gate_device(n=(32, 32, 24), T=4.0)
    dev["surface_charges"] = [dict(z=90.0, x0=50.0, x1=150.0, y0=30.0, y1=170.0, sigma=-1.5e-3)]
    P = PoissonProblem(dev)
    phi, rep = P.solve()
    assert rep["converged"]
    m = q.qcad_mesh_create(dev)
    g = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    r = q.qcad_poisson_solve(m, dev["bias"], q.make_opts(precision=1, cheb_degree=-1), g)
    assert r["status"] == "OK"
    assert np.max(np.abs(g.cpu().numpy() - phi)) <= 1e-9
    # the sheet moves the solution well beyond the tolerance
    P0 = PoissonProblem(W.five_gate_device(n=(32, 32, 24), T=4.0))
    phi0, _ = P0.solve(phi0=phi)
    assert np.max(np.abs(phi0 - phi)) > 1e-3


@pytest.mark.parametrize("precision", [0, 1])
def test_adjoint_matches_oracle(q, solved, precision):
    dev, P, phi = solved["one"]
    dNdV_o, dNdq_o = OC.adjoint(P, phi)
    m = q.qcad_mesh_create(dev)
    g = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    opts = q.make_opts(precision=precision)
    q.qcad_poisson_solve(m, dev["bias"], opts, g)
    dq = torch.empty(m.n_dots * m.n_elems, dtype=torch.float64, device="cuda")
    dNdV = np.array(q.qcad_adjoint(m, dev["bias"], g, opts, dN_dq=dq))
    assert np.max(np.abs(dNdV - dNdV_o)) <= 1e-8 * np.max(np.abs(dNdV_o))
    assert abs(dNdV[1, 3]) > 1e-3 * np.max(np.abs(dNdV_o))      # the charged plunger's own entry
    gq = dq.cpu().numpy().reshape(m.n_dots, m.n_elems)
    assert np.max(np.abs(gq - dNdq_o)) <= 1e-8 * np.max(np.abs(dNdq_o))


def test_fd_capacitance_of_the_charged_gate(q, solved):
    dev, P, phi = solved["one"]
    Co, _, _ = OC.fd_capacitance(dev, gate=3, dV=0.01)
    m = q.qcad_mesh_create(dev)
    Cg = np.array(q.qcad_capacitance(m, dev["bias"], gate=3, dV=0.01))
    assert np.max(np.abs(Cg - Co)) <= 1e-6 * np.max(np.abs(Co))


def test_surface_terms_are_validated(q):
    dev = charged_device(n=(12, 12, 8))
    bad = copy.deepcopy(dev)
    bad["gates"][3]["robin"]["d"] = 0.0
    with pytest.raises(q.QcadError) as e:
        q.qcad_mesh_create(bad)
    assert e.value.code == 1
    bad = copy.deepcopy(dev)
    bad["surface_charges"][0]["z"] = 91.0                       # not a node plane
    with pytest.raises(q.QcadError) as e:
        q.qcad_mesh_create(bad)
    assert e.value.code == 1
    m = q.qcad_mesh_create(dev)
    with pytest.raises(q.QcadError):
        q.qcad_set_launch(m, 2, 3, 8, 16)                        # the plane-factorized variant
    phi = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    with pytest.raises(q.QcadError) as e:
        q.qcad_poisson_solve_batch([m], [dev["bias"]], q.make_opts(precision=1), [phi])
    assert e.value.code == 1
