"""Pins of the oracle's self-consistent Schrodinger-Poisson loop (Sec. II.C), CPU only.

Each test checks the oracle against something other than its own formulas: textbook limits of
the local-density exchange-correlation potential, the exact normalization of the quantum
density, the Fermi factor's identities, the fixed point the loop converges to, and the
convergence behaviour the paper reports for 3D-confined devices.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import fem, physics
from oracle import schrodinger as S
from oracle import sp
from oracle.poisson import PoissonProblem


def slater_exchange(n, eps_r):
    """Textbook local exchange potential -(q^2/(4 pi eps)) (3 n / pi)^(1/3), eV for n in nm^-3."""
    e2 = physics.Q_E ** 2 / (4.0 * math.pi * physics.EPS0 * eps_r) / physics.Q_E * 1e9  # eV nm
    return -e2 * (3.0 * np.asarray(n) / math.pi) ** (1.0 / 3.0)


def test_bohr_radius_and_isotropic_exchange_mass():
    # CODATA 2018 a0 (the constants used here reproduce it to their own uncertainty)
    assert abs(sp.bohr_nm() / 0.0529177210903 - 1.0) < 1e-8
    assert abs(sp.m_xc(0.3, 0.3) - 0.3) < 1e-15                 # one mass in every direction


def test_vxc_limits():
    eps_r, mxc = 11.7, sp.m_xc(0.98, 0.19)
    assert sp.vxc(np.array([0.0]), eps_r, mxc)[0] == 0.0
    n = np.logspace(-12, 4, 50)
    v = sp.vxc(n, eps_r, mxc)
    assert np.all(v < 0) and np.all(np.diff(v) < 0)          # attractive, deeper with density
    # high density: the correlation factor -> 1 and V_xc -> the Slater exchange potential
    r_hi = sp.vxc(np.array([1e4]), eps_r, mxc)[0] / slater_exchange(1e4, eps_r)
    assert 1.0 < r_hi < 1.005
    # low density: x ln(1 + 1/x) -> 1, so V_xc -> (1 + 0.7734) x the exchange potential
    r_lo = sp.vxc(np.array([1e-20]), eps_r, mxc)[0] / slater_exchange(1e-20, eps_r)
    assert abs(r_lo - 1.7734) < 1e-4


def test_fermi_factor_identities():
    a = np.linspace(-99.0, 99.0, 397)
    f, g = sp.fermi3d(a)
    fm, _ = sp.fermi3d(-a)
    assert np.max(np.abs(f + fm - 1.0)) < 1e-15                 # particle-hole symmetry
    h = 1e-5
    fp, _ = sp.fermi3d(a + h)
    fn, _ = sp.fermi3d(a - h)
    assert np.max(np.abs(-(fp - fn) / (2 * h) - g)) < 1e-9      # g = -df/da
    # the low-temperature replacement joins the Fermi factor at the cutoff
    f1, _ = sp.fermi3d(np.array([100.0]))
    f2, _ = sp.fermi3d(np.array([100.0 + 1e-12]))
    assert abs(f2[0] / f1[0] - 1.0) < 1e-11


@pytest.fixture(scope="module")
def small_dot():
    dev = W.five_gate_device(n=(16, 16, 12), T=4.0)
    V = list(dev["bias"]["V_gate"])
    # plungers that pull the lowest levels below E_F while the sixth stays empty (the loop
    # needs every occupied level among the states it computes)
    V[1] = V[3] = 0.9
    dev["bias"]["V_gate"] = V
    return dev


def test_quantum_density_normalization(small_dot):
    # M-orthonormal eigenvectors integrate to 1 under the same 2x2x2 quadrature, so the Gauss-point
    # weights 4|psi_i|^2 integrate to 4 per state, and the electron count is sum_i 4 f_i
    P = PoissonProblem(small_dot)
    phi, _ = P.solve()
    E, X, idx, H, M = S.solve_device(P, phi, nev=4)
    psi = np.zeros((P.mesh.n_nodes, 4))
    psi[idx] = X
    sel = P.mesh.subdomain_elements()
    Wq = sp.qp_weights(P, psi, sel)
    integ = np.einsum("e,eqi->i", P.wdet[sel][:, 0], Wq)
    assert np.max(np.abs(integ - 4.0)) < 1e-12
    kT = physics.kT_eV(P.T)
    f, _ = sp.fermi3d((E - P.E_F) / kT)
    assert abs(sp.quantum_electrons(P, Wq, E, phi, phi) - 4.0 * np.sum(f)) < 1e-10 * max(1.0, 4 * np.sum(f))


def test_predictor_density_derivative(small_dot):
    P = PoissonProblem(small_dot)
    phi, _ = P.solve()
    E, X, idx, _, _ = S.solve_device(P, phi, nev=4)
    psi = np.zeros((P.mesh.n_nodes, 4))
    psi[idx] = X
    sel = P.mesh.subdomain_elements()
    Wq = sp.qp_weights(P, psi, sel)
    kT = physics.kT_eV(P.T)
    conn = P.mesh.conn[sel]
    phq = fem.interpolate(phi, conn)
    rng = np.random.default_rng(3)
    base = phq + 1e-3 * rng.standard_normal(phq.shape)
    n0, dn = sp.predictor_density(Wq, E, base, phq, P.E_F, kT)
    h = 1e-8
    n1, _ = sp.predictor_density(Wq, E, base + h, phq, P.E_F, kT)
    n2, _ = sp.predictor_density(Wq, E, base - h, phq, P.E_F, kT)
    fd = (n1 - n2) / (2 * h)
    assert np.max(np.abs(fd - dn)) <= 1e-5 * np.max(np.abs(dn)) + 1e-14
    # a higher potential lowers every level (the minus sign): the density rises
    assert np.all(dn >= 0)


def test_sp_loop_converges_monotonically_to_a_fixed_point(small_dot):
    phi, E, rep = sp.sp_solve(small_dot, nev=6, tol=1e-7, max_iter=80)
    assert rep["converged"], rep["dphi"]
    d = np.array(rep["dphi"])
    # Sec. III: monotonic convergence of the potential for the 3D dot at 4 K
    assert np.all(d[2:] <= d[1:-1] * (1 + 1e-6))
    assert rep["n_quantum"] > 0.5                               # the dot holds electrons
    # fixed point: the eigenpairs in V(phi*) + V_xc(n*), n* the density the last step left, are
    # those the last step used, and the Poisson residual with the exact quantum density of those
    # eigenpairs at phi* vanishes to the loop tolerance
    P = sp.SPPoissonProblem(small_dot)
    sel = P.mesh.subdomain_elements()
    interior = P.mesh.subdomain_interior_nodes()
    si = P.si
    Vq = S.device_potential(P, phi, sel) + sp.vxc(rep["n_q"], si["eps_r"], sp.m_xc(si["m_l"], si["m_t"]))
    H, M, idx = S.operators(P.mesh, sel, interior, (0.19, 0.19, 0.19), Vq)
    E1, X1 = S.lowest_eigenpairs(H, M, 6, sigma=float(np.min(Vq)) - 1e-2)
    assert np.max(np.abs(E1 - E)) < 1e-5
    P.set_quantum(E, rep["W"], phi)
    R = P.residual(phi)
    assert np.max(np.abs(R[P.free])) < 1e-5 * np.max(np.abs(P.K @ phi))


def test_predictor_density_derivative_on_both_sides_of_the_cutoff():
    # one level at a = (E_i - E_F - dphi)/kT drawn from [-150, 250], so the Fermi factor and its
    # exp(-a) replacement above a = 100 both occur: d n~/d phi against central differences
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=40, deadline=None)
    @hyp.given(st.floats(0.5, 300.0), st.floats(-150.0, 250.0), st.integers(0, 2 ** 31 - 1))
    def check(T, a_level, seed):
        rng = np.random.default_rng(seed)
        kT = physics.kT_eV(T)
        E = np.array([a_level * kT])                      # E_F = 0
        Wq = rng.uniform(0.1, 1.0, (3, 8, 1))
        prev = rng.normal(0.0, 1.0, (3, 8))
        ph = prev + 0.3 * kT * rng.standard_normal((3, 8))
        n0, dn = sp.predictor_density(Wq, E, ph, prev, 0.0, kT)
        h = 3e-4 * kT
        n1, _ = sp.predictor_density(Wq, E, ph + h, prev, 0.0, kT)
        n2, _ = sp.predictor_density(Wq, E, ph - h, prev, 0.0, kT)
        fd = (n1 - n2) / (2 * h)
        # (the difference quotient of n~ carries ~1e-16 n / h of rounding, which dominates for deeply
        # occupied levels where d n~/d phi is tiny next to n~)
        assert np.all(np.abs(fd - dn) <= 1e-6 * np.abs(dn) + 1e-14 * np.abs(n0) / h)
        assert np.all(dn >= 0) and np.all(n0 >= 0)

    check()
    # and n~ joins continuously at the cutoff
    kT = physics.kT_eV(4.0)
    W1 = np.ones((1, 8, 1))
    z = np.zeros((1, 8))
    lo, _ = sp.predictor_density(W1, np.array([100.0 * kT * (1 - 1e-12)]), z, z, 0.0, kT)
    hi, _ = sp.predictor_density(W1, np.array([100.0 * kT * (1 + 1e-12)]), z, z, 0.0, kT)
    assert abs(hi[0, 0] / lo[0, 0] - 1.0) < 1e-9
