"""Pins of the oracle's finite-element discretization and Newton solve (no GPU).

Closed forms: the series-capacitor potential of a linear dielectric stack and
its gate charge C = eps0 A / (t_ox/eps_ox + t_si/eps_si); O(h^2) L2 and O(h)
H1 convergence on a manufactured solution; bulk charge neutrality far from
the contacts. Identities: zero row sums and symmetry of K, discrete charge
conservation, the Jacobian against finite differences of the residual.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fem, physics
from oracle.mesh import Mesh
from oracle.poisson import PoissonProblem, solve_spd


def test_linear_dielectric_stack_is_nodally_exact():
    dev = W.mos_capacitor(nx=4, ny=3, nz=12, L=30.0, t_si=40.0, t_ox=8.0, n_ox=3, V_gate=0.7)
    P = PoissonProblem(dev, linear=True)
    phi = P.initial_guess()
    phi_b = P.phi_ohm
    eo, es = 3.9, 11.7
    t_ox, t_si, V = 8.0, 40.0, 0.7
    phi_i = (eo * V / t_ox + es * phi_b / t_si) / (eo / t_ox + es / t_si)
    z = P.mesh.coords[:, 2]
    exact = np.where(z <= t_si, phi_b + (phi_i - phi_b) * z / t_si, phi_i + (V - phi_i) * (z - t_si) / t_ox)
    assert np.max(np.abs(phi - exact)) < 1e-12
    # reaction on the gate nodes = enclosed flux: (K phi) summed over gate = A (V - phi_b) / (t_ox/eo + t_si/es)
    Kphi = P.K @ phi
    q_gate = Kphi[P.gate == 0].sum()
    A = 30.0 * 30.0
    expect = A * (V - phi_b) / (t_ox / eo + t_si / es)
    assert abs(q_gate / expect - 1.0) < 1e-12
    # and in farads: C = eps0 A / (t_ox/eo + t_si/es) for the series stack
    C = physics.EPS0 * q_gate * 1e-9 / (V - phi_b)
    assert abs(C / (physics.EPS0 * A * 1e-18 / ((t_ox / eo + t_si / es) * 1e-9)) - 1.0) < 1e-12


def test_stiffness_row_sums_and_symmetry():
    dev = W.five_gate_device(n=(6, 5, 7), T=4.0)
    P = PoissonProblem(dev)
    K = P.K
    kmax = abs(K).max()
    assert np.max(np.abs(K @ np.ones(K.shape[0]))) < 1e-14 * kmax * 27
    assert abs(K - K.T).max() < 1e-15 * kmax
    # single-slab parallel plate: C = eps0 eps_r A / d
    dev = dict(Lx=10.0, Ly=10.0, nx=2, ny=2, layers=[dict(material=1, thickness=5.0, n=4)],
               materials=[dict(W.SI), dict(W.SIO2)], gates=[dict(name="G", x0=0, x1=10, y0=0, y1=10)],
               gate_work_function=None, bottom_ohmic=1, dots=[], subdomain=None,
               bias=dict(T=300.0, V_gate=[1.0], V_sub=0.0, statistics=1, incomplete_ionization=1))
    P = PoissonProblem(dev, linear=True)
    phi = P.initial_guess()
    q = (P.K @ phi)[P.gate == 0].sum() / (1.0 - P.phi_ohm)
    assert abs(q / (3.9 * 100.0 / 5.0) - 1.0) < 1e-13


def _mms(n):
    L = 1.0
    dev = dict(Lx=L, Ly=L, nx=n, ny=n, layers=[dict(material=0, thickness=L, n=n)],
               materials=[dict(W.SI, eps_r=1.0)], gates=[], bottom_ohmic=0, dots=[], subdomain=None,
               bias=dict(T=300.0, V_gate=[]))
    m = Mesh(dev)
    wdet, grad = fem.geometry(m.elem_coords)
    K = fem.assemble_matrix(m.conn, fem.element_stiffness(wdet, grad, np.ones((m.n_elems, 3))), m.n_nodes)
    xq = np.einsum("qa,eai->eqi", fem.NQ, m.elem_coords)
    u = lambda p: np.sin(np.pi * p[..., 0]) * np.sin(np.pi * p[..., 1]) * np.sin(np.pi * p[..., 2])
    f = 3.0 * np.pi ** 2 * u(xq)
    F = fem.assemble_vector(m.conn, fem.element_load(wdet, f), m.n_nodes)
    bd = (m.ni == 0) | (m.ni == n) | (m.nj == 0) | (m.nj == n) | (m.nk == 0) | (m.nk == n)
    fr = ~bd
    uh = np.zeros(m.n_nodes)
    uh[fr] = solve_spd(K[fr][:, fr], F[fr])
    # errors by a 3x3x3 Gauss rule (one order higher than the discretization's)
    g3, w3 = np.polynomial.legendre.leggauss(3)
    err2, herr2 = 0.0, 0.0
    h = L / n
    for a, wa in zip(g3, w3):
        for b, wb in zip(g3, w3):
            for c, wc in zip(g3, w3):
                xi = np.array([a, b, c])
                N = fem.shape(xi)
                dN = fem.shape_grad_ref(xi) * (2.0 / h)
                p = np.einsum("a,eai->ei", N, m.elem_coords)
                val = uh[m.conn] @ N
                gr = np.einsum("ea,ai->ei", uh[m.conn], dN)
                ex = u(p)
                gx = np.stack([
                    np.pi * np.cos(np.pi * p[:, 0]) * np.sin(np.pi * p[:, 1]) * np.sin(np.pi * p[:, 2]),
                    np.pi * np.sin(np.pi * p[:, 0]) * np.cos(np.pi * p[:, 1]) * np.sin(np.pi * p[:, 2]),
                    np.pi * np.sin(np.pi * p[:, 0]) * np.sin(np.pi * p[:, 1]) * np.cos(np.pi * p[:, 2])], axis=1)
                wt = wa * wb * wc * (h / 2) ** 3
                err2 += wt * np.sum((val - ex) ** 2)
                herr2 += wt * np.sum((gr - gx) ** 2)
    return np.sqrt(err2), np.sqrt(herr2)


def test_manufactured_solution_convergence():
    ns = [4, 8, 16]
    e = [_mms(n) for n in ns]
    l2 = [x[0] for x in e]
    h1 = [x[1] for x in e]
    r_l2 = [np.log2(l2[i] / l2[i + 1]) for i in range(len(ns) - 1)]
    r_h1 = [np.log2(h1[i] / h1[i + 1]) for i in range(len(ns) - 1)]
    assert abs(r_l2[-1] - 2.0) < 0.1, r_l2
    assert abs(r_h1[-1] - 1.0) < 0.1, r_h1


@pytest.fixture(scope="module")
def small_dqd():
    dev = W.five_gate_device(n=(16, 16, 12), T=4.0)
    dev["bias"]["V_gate"] = [0.35, 0.95, 0.45, 0.9, 0.3]
    P = PoissonProblem(dev)
    phi, rep = P.solve()
    assert rep["converged"]
    return P, phi


def test_discrete_charge_conservation(small_dqd):
    P, phi = small_dqd
    # sum over all rows of R_full = -(q/eps0) int rho (K has zero row sums, N_a sum to one)
    Rf = P.residual(phi, full=True)
    rho, _, _, _ = P.qp_charge(phi)
    total = -P.qe * np.sum(P.wdet * rho)
    assert abs(Rf.sum() - total) < 1e-9 * max(1.0, abs(total))
    # at convergence the free rows vanish, so the Dirichlet reactions carry all the charge
    assert abs(Rf[P.dir].sum() - total) < 1e-8 * max(1.0, abs(total)) + P.free.sum() * 1e-12


def test_jacobian_matches_residual_differences(small_dqd):
    P, phi = small_dqd
    rng = np.random.default_rng(0)
    ph = phi.copy()
    ph[P.free] += 0.002 * rng.standard_normal(P.free.sum())
    J = P.jacobian(ph)
    v = np.zeros_like(ph)
    v[P.free] = rng.standard_normal(P.free.sum())
    u = np.zeros_like(ph)
    u[P.free] = rng.standard_normal(P.free.sum())
    eps = 1e-6
    fd = (P.residual(ph + eps * v) - P.residual(ph - eps * v)) / (2 * eps)
    Jv = J @ v
    Jv[P.dir] = 0.0
    assert np.linalg.norm(Jv - fd) / np.linalg.norm(Jv) < 1e-7
    assert abs(u @ (J @ v) - v @ (J @ u)) < 1e-13 * abs(u @ (J @ v))


def test_newton_solution_is_unique(small_dqd):
    P, phi = small_dqd
    start = P.g.copy()  # contact values with zero elsewhere instead of the Laplace guess
    phi2, rep = P.solve(phi0=start)
    assert rep["converged"]
    assert np.max(np.abs(phi2 - phi)) < 1e-10
    assert np.max(np.abs(P.residual(phi))) < 1e-10


def test_bulk_neutrality_far_from_contacts():
    T = 300.0
    dev = W.mos_capacitor(nx=2, ny=2, nz=64, L=20.0, t_si=300.0, t_ox=5.0, n_ox=2, V_gate=0.0, T=T, N_A=1e-3)
    P = PoissonProblem(dev)
    phi, rep = P.solve()
    assert rep["converged"]
    root = physics.neutral_root(P.si, T, P.phi_r, 0.0, 1, 1)
    z = P.mesh.coords[:, 2]
    mid = np.abs(z - 150.0) < 12.0
    assert np.max(np.abs(phi[mid] - root)) < 1e-6


def test_jacobian_matches_residual_differences_in_every_regime():
    # random temperature (4-300 K), statistics (FD; MB from 77 K up, where it is meaningful), ionization
    # model, gate voltages and potential perturbations: the hand-derived Jacobian against central
    # differences of the residual (step 1e-3 kT), through every branch of the carrier statistics
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=20, deadline=None)
    @hyp.given(st.sampled_from([4.0, 20.0, 77.0, 300.0]), st.booleans(), st.booleans(),
               st.lists(st.floats(-0.5, 1.2), min_size=5, max_size=5), st.integers(0, 2 ** 31 - 1))
    def check(T, mb, incomplete, V, seed):
        stat = 0 if (mb and T >= 77.0) else 1
        dev = W.five_gate_device(n=(6, 6, 5), T=T, statistics=stat, incomplete_ionization=int(incomplete))
        dev["bias"]["V_gate"] = list(V)
        P = PoissonProblem(dev)
        rng = np.random.default_rng(seed)
        ph = P.initial_guess(solver="direct")
        ph[P.free] += 0.05 * rng.standard_normal(P.free.sum())
        v = np.zeros_like(ph)
        v[P.free] = rng.standard_normal(P.free.sum())
        h = 1e-3 * physics.kT_eV(T)
        fd = (P.residual(ph + h * v) - P.residual(ph - h * v)) / (2 * h)
        Jv = P.jacobian(ph) @ v
        Jv[P.dir] = 0.0
        assert np.linalg.norm(Jv - fd) <= 1e-6 * np.linalg.norm(Jv)

    check()


def test_general_hexahedra_match_the_affine_closed_forms():
    # the oracle's element geometry is general (isoparametric); the devices only use boxes, whose
    # Jacobian is diagonal and would hide a transposed inverse. On random sheared affine elements
    # x = A xi + b: mass = |det A| (x)_d [[2/3, 1/3], [1/3, 2/3]], and the stiffness equals
    # |det A| int grad_xi N_a^T (A^-1 A^-T) grad_xi N_b, integrated here by 3x3x3 Gauss-Legendre
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies
    m1 = np.array([[2.0, 1.0], [1.0, 2.0]]) / 3.0
    mass_ref = np.kron(m1, np.kron(m1, m1))               # corner a = ax + 2 ay + 4 az: z (x) y (x) x
    g3, w3 = np.polynomial.legendre.leggauss(3)
    sgn = np.array([[2 * (a & 1) - 1, 2 * ((a >> 1) & 1) - 1, 2 * ((a >> 2) & 1) - 1] for a in range(8)], float)

    def grad_ref(xi):                                      # dN_a/dxi_d of (1 + s xi)(1 + s eta)(1 + s zeta)/8
        g = np.empty((8, 3))
        for a in range(8):
            f = 1.0 + sgn[a] * xi
            g[a] = sgn[a] * np.array([f[1] * f[2], f[0] * f[2], f[0] * f[1]]) / 8.0
        return g

    @hyp.settings(max_examples=20, deadline=None)
    @hyp.given(st.lists(st.floats(0.5, 3.0), min_size=3, max_size=3),
               st.lists(st.floats(-0.4, 0.4), min_size=6, max_size=6), st.lists(st.floats(-5, 5), min_size=3, max_size=3))
    def check(diag, shear, shift):
        A = np.diag(diag)
        A[0, 1], A[0, 2], A[1, 2], A[1, 0], A[2, 0], A[2, 1] = [s * max(diag) for s in shear]
        det = np.linalg.det(A)
        hyp.assume(det > 0.05 * np.prod(diag))
        X = (sgn @ A.T + np.array(shift))[None]              # (1, 8, 3) corners at xi = +-1
        wdet, grad = fem.geometry(X)
        Me = fem.element_mass(wdet, np.ones((1, 8)))[0]
        assert np.max(np.abs(Me - det * mass_ref)) < 1e-12 * det
        Ke = fem.element_stiffness(wdet, grad, np.ones((1, 3)))[0]
        G = np.linalg.inv(A) @ np.linalg.inv(A).T
        ref = np.zeros((8, 8))
        for a, wa in zip(g3, w3):
            for b, wb in zip(g3, w3):
                for c, wc in zip(g3, w3):
                    gr = grad_ref(np.array([a, b, c]))
                    ref += wa * wb * wc * det * gr @ G @ gr.T
        assert np.max(np.abs(Ke - ref)) < 1e-11 * np.max(np.abs(ref))

    check()
