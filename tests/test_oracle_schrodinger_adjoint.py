"""Pins of the oracle's Schrodinger eigenpairs, capacitance and adjoint (no GPU).

- Particle in a box: for Q1 elements with consistent mass on a uniform box
  with psi = 0 walls the discrete spectrum is known in closed form,
  lambda = sum_d (hbar^2/2m_d) (6/h_d^2) (1 - cos t_d)/(2 + cos t_d),
  t_d = k_d pi h_d / L_d (the paper's 2D/3D infinite-well check, Sec. II.B).
- Harmonic oscillator: E_0 = (3/2) hbar omega with O(h^2) convergence (the
  paper's parabolic-well check, Sec. II.B).
- Triangular well: levels (hbar^2 F^2 / 2m)^(1/3) |a_i| with a_i the zeros of the Airy
  function, O(h^2); finite square well: the roots of the even and odd matching
  conditions k tan(ka) = kappa, -k cot(ka) = kappa, O(h^2) (the paper's 1D wells,
  Sec. II.B), both as z-strips whose one transverse mode has a closed-form energy.
- Appendix B: the paper's triangular-well formula gives E_1 = 7.11 meV at
  F = 8.256e6 V/m after the 25.003 meV shift (Sec. III).
- Adjoint sensitivities against central finite differences of full solves.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
import scipy.optimize
import scipy.special

import workloads as W
from oracle import capacitance as C
from oracle import fem, physics
from oracle import schrodinger as S
from oracle.mesh import Mesh
from oracle.poisson import PoissonProblem

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _box(L, n):
    dev = dict(Lx=L[0], Ly=L[1], nx=n[0], ny=n[1], layers=[dict(material=0, thickness=L[2], n=n[2])],
               materials=[dict(W.SI)], gates=[], bottom_ohmic=0, dots=[],
               subdomain=dict(i0=0, i1=n[0], j0=0, j1=n[1], k0=0, k1=n[2]), bias=dict(T=4.0, V_gate=[]))
    return Mesh(dev)


def test_box_spectrum_closed_form():
    L, n, me = (20.0, 16.0, 12.0), (10, 8, 6), (0.19, 0.3, 0.98)
    m = _box(L, n)
    sel, inter = m.subdomain_elements(), m.subdomain_interior_nodes()
    H, M, _ = S.operators(m, sel, inter, me, np.zeros((sel.sum(), 8)))
    E, X = S.lowest_eigenpairs(H, M, 8, sigma=-1.0)
    h2m = physics.hbar2_over_2m0()
    ev = []
    for ks in itertools.product(range(1, n[0]), range(1, n[1]), range(1, n[2])):
        lam = 0.0
        for k, Ld, nd, md in zip(ks, L, n, me):
            h = Ld / nd
            t = k * math.pi * h / Ld
            lam += h2m / md * 6.0 / h ** 2 * (1 - math.cos(t)) / (2 + math.cos(t))
        ev.append(lam)
    ev = np.sort(ev)[:8]
    assert np.max(np.abs(E - ev) / ev) < 1e-10
    # M-orthonormal eigenvectors
    G = X.T @ (M @ X)
    assert np.max(np.abs(G - np.eye(8))) < 1e-10
    # a constant potential shifts the whole spectrum
    H2, M2, _ = S.operators(m, sel, inter, me, np.full((sel.sum(), 8), -0.2))
    E2, _ = S.lowest_eigenpairs(H2, M2, 8, sigma=-1.0)
    assert np.max(np.abs(E2 - (E - 0.2))) < 1e-12


def _oscillator(n, hw=0.01, m_rel=0.19):
    h2m = physics.hbar2_over_2m0() / m_rel
    ell2 = 2.0 * h2m / hw  # hbar/(m omega) in nm^2
    L = 10.0 * math.sqrt(ell2)
    mesh = _box((L, L, L), (n, n, n))
    sel, inter = mesh.subdomain_elements(), mesh.subdomain_interior_nodes()
    xq = np.einsum("qa,eai->eqi", fem.NQ, mesh.elem_coords)
    r2 = np.sum((xq - L / 2) ** 2, axis=2)
    Vq = hw ** 2 * r2 / (4.0 * h2m)  # (1/2) m omega^2 r^2
    H, M, _ = S.operators(mesh, sel, inter, (m_rel,) * 3, Vq)
    E, _ = S.lowest_eigenpairs(H, M, 4, sigma=-0.01)
    return E


def test_harmonic_oscillator_convergence():
    hw = 0.01
    Es = [_oscillator(n, hw) for n in (12, 24)]
    err = [abs(E[0] - 1.5 * hw) for E in Es]
    rate = math.log2(err[0] / err[1])
    assert abs(rate - 2.0) < 0.15, rate
    assert err[1] < 0.02 * hw
    # first excited level is threefold degenerate at 2.5 hbar omega
    assert np.max(np.abs(Es[1][1:4] - 2.5 * hw)) < 0.05 * hw
    assert np.max(Es[1][1:4]) - np.min(Es[1][1:4]) < 1e-9 * hw


def _strip_levels(Lz, nz, V_of_z, m, nev):
    """z-levels of a 2 nm x 2 nm strip with two elements across x and y (one transverse mode, whose
    discrete energy 2 x (hbar^2/2m) (6/h^2)(1 - cos(pi/2))/(2 + cos(pi/2)) is subtracted)."""
    dev = dict(Lx=2.0, Ly=2.0, nx=2, ny=2, layers=[dict(material=0, thickness=Lz, n=nz)],
               materials=[dict(W.SI)], gates=[], bottom_ohmic=0, dots=[],
               subdomain=dict(i0=0, i1=2, j0=0, j1=2, k0=0, k1=nz), bias=dict(T=4.0, V_gate=[]))
    mesh = Mesh(dev)
    sel, inter = mesh.subdomain_elements(), mesh.subdomain_interior_nodes()
    zq = np.einsum("qa,ea->eq", fem.NQ, mesh.elem_coords[:, :, 2])
    H, M, _ = S.operators(mesh, sel, inter, (m, m, m), V_of_z(zq))
    E, _ = S.lowest_eigenpairs(H, M, nev, sigma=-0.01)
    return E - 2.0 * (physics.hbar2_over_2m0() / m) * 6.0 * 0.5


def test_triangular_well_airy_levels():
    # V = F z above a hard wall at z = 0: E_i = (hbar^2 F^2 / 2m)^(1/3) |a_i| (a_i Airy zeros); the
    # far wall at 25 nm is 16 decay lengths past the third level's turning point
    m, F = 0.98, 0.01                                       # m_l, 10 mV/nm
    exact = -scipy.special.ai_zeros(3)[0] * (physics.hbar2_over_2m0() / m * F ** 2) ** (1.0 / 3.0)
    errs = [np.abs(_strip_levels(25.0, nz, lambda z: F * z, m, 3) - exact) / exact for nz in (50, 100)]
    assert np.all(np.abs(np.log2(errs[0] / errs[1]) - 2.0) < 0.05), errs
    assert np.max(errs[1]) < 3e-3


def test_finite_square_well_levels():
    # well of half-width a = 5 nm and depth 0.3 eV (edges on node planes), one mass: the levels solve
    # k tan(ka) = kappa (even) and -k cot(ka) = kappa (odd), k = sqrt(E/h2m), kappa = sqrt((V0-E)/h2m)
    m, V0, a = 0.19, 0.3, 5.0
    h2m = physics.hbar2_over_2m0() / m

    def match(E, odd):
        k, kap = math.sqrt(E / h2m), math.sqrt((V0 - E) / h2m)
        return (-k / math.tan(k * a) if odd else k * math.tan(k * a)) - kap

    exact = []
    for odd, (lo, hi) in ((0, (0.0, 0.5)), (1, (0.5, 1.0)), (0, (1.0, 1.5))):  # ka / pi brackets
        e_lo = h2m * ((lo * math.pi + 1e-9) / a) ** 2
        e_hi = min(h2m * ((hi * math.pi - 1e-9) / a) ** 2, V0 - 1e-12)
        exact.append(scipy.optimize.brentq(lambda E: match(E, odd), e_lo, e_hi, xtol=1e-16, rtol=1e-15))
    exact = np.array(exact)
    well = lambda z: np.where(np.abs(z - 20.0) < a, 0.0, V0)
    errs = [np.abs(_strip_levels(40.0, nz, well, m, 3) - exact) / exact for nz in (80, 160)]
    assert np.all(np.abs(np.log2(errs[0] / errs[1]) - 2.0) < 0.05), errs
    assert np.max(errs[1]) < 4e-3


def test_appendix_b_triangular_well_e1():
    # E_i = (hbar^2 q^2 F^2 / (2 m_l))^(1/3) [3 pi/2 (i - 1/4)]^(2/3), shifted down by 25.003 meV
    F = GOLD["triangular_well_field_V_per_m"]["value"] * 1e-9  # V/nm
    shift = GOLD["triangular_well_shift_eV"]["value"]
    h2m_l = physics.hbar2_over_2m0() / W.SI["m_l"]
    E1 = (h2m_l * F ** 2) ** (1.0 / 3.0) * (1.5 * math.pi * 0.75) ** (2.0 / 3.0) - shift
    assert abs(E1 * 1e3 - GOLD["triangular_well_E1_meV"]["value"]) < 0.015
    # the transverse mass would miss it by more than 2 meV: the constants are pinned
    h2m_t = physics.hbar2_over_2m0() / W.SI["m_t"]
    E1t = (h2m_t * F ** 2) ** (1.0 / 3.0) * (1.5 * math.pi * 0.75) ** (2.0 / 3.0) - shift
    assert abs(E1t * 1e3 - 7.11) > 2.0


@pytest.fixture(scope="module")
def dqd():
    dev = W.five_gate_device(n=(24, 24, 16), T=4.0)
    P = PoissonProblem(dev)
    phi, rep = P.solve()
    assert rep["converged"]
    return dev, P, phi


def test_dots_hold_electrons(dqd):
    dev, P, phi = dqd
    N = C.electron_counts(P, phi)
    assert np.all(N > 0.1) and np.all(N < 100.0)


def test_adjoint_gate_sensitivity_vs_central_fd(dqd):
    dev, P, phi = dqd
    dN_dV, _ = C.adjoint(P, phi)
    h = 1e-4
    for g in range(len(dev["bias"]["V_gate"])):
        Ns = []
        for s in (+1, -1):
            b = dict(dev["bias"])
            b["V_gate"] = list(b["V_gate"])
            b["V_gate"][g] += s * h
            Pg = PoissonProblem(dev, bias=b)
            pg, rep = Pg.solve(phi0=phi)
            assert rep["converged"]
            Ns.append(C.electron_counts(Pg, pg))
        fd = (Ns[0] - Ns[1]) / (2 * h)
        scale = np.max(np.abs(dN_dV))
        assert np.max(np.abs(fd - dN_dV[:, g])) < 1e-5 * scale, (g, fd, dN_dV[:, g])
    # plungers load their own dot most strongly
    assert dN_dV[0, 1] > dN_dV[0, 3] and dN_dV[1, 3] > dN_dV[1, 1]


def test_adjoint_fixed_charge_gradient_vs_fd(dqd):
    dev, P, phi = dqd
    theta = np.array(W.interface_fixed_charge(dev, seed=5))
    P0 = PoissonProblem(dev, fixed_charge=theta)
    ph0, rep = P0.solve(phi0=phi)
    assert rep["converged"]
    _, dN_dth = C.adjoint(P0, ph0)
    rng = np.random.default_rng(1)
    eps = 1e-4 * np.max(np.abs(theta))
    for _ in range(2):
        d = rng.standard_normal(theta.size) * (theta != 0)
        Ns = []
        for s in (+1, -1):
            Ps = PoissonProblem(dev, fixed_charge=theta + s * eps * d)
            ps, rep = Ps.solve(phi0=ph0)
            assert rep["converged"]
            Ns.append(C.electron_counts(Ps, ps))
        fd = (Ns[0] - Ns[1]) / (2 * eps)
        ad = dN_dth @ d
        assert np.max(np.abs(fd - ad)) < 1e-5 * np.max(np.abs(ad)), (fd, ad)


def test_fd_capacitance_agrees_with_adjoint(dqd):
    dev, P, phi = dqd
    dN_dV, _ = C.adjoint(P, phi)
    Cf, N1, N2 = C.fd_capacitance(dev, gate=1, dV=GOLD["capacitance_dV_V"]["value"], phi0=phi)
    # forward difference with dV = 0.01 V: first-order agreement with q dN/dV
    Ca = C.Q_AF * dN_dV[:, 1]
    assert np.all(Cf > 0)
    assert np.max(np.abs(Cf - Ca) / np.abs(Ca)) < 0.1


def test_sheet_charge_calibration_reaches_the_target():
    # Sec. III: the effective interface charge is tuned so that the dot holds one electron; the
    # count rises monotonically with a positive sheet, and the adjoint slope dN/dsigma equals the
    # finite-difference slope of the calibrated count
    from oracle.poisson import PoissonProblem
    dev = W.five_gate_device(n=(12, 12, 8), T=4.0, with_subdomain=False)
    pat = np.array(W.interface_sheet_pattern(dev))
    sig, N, phi = C.calibrate_sheet_charge(dev, 0, 1.0, pat)
    assert abs(N - 1.0) < 1e-9
    Ns = []
    for s in (sig - 1e-4, sig, sig + 1e-4):
        P = PoissonProblem(dev, fixed_charge=s * pat)
        ph, _ = P.solve()
        Ns.append(C.electron_counts(P, ph)[0])
    assert Ns[0] < Ns[1] < Ns[2]
    P = PoissonProblem(dev, fixed_charge=sig * pat)
    _, dNdq = C.adjoint(P, phi)
    slope = float(dNdq[0] @ pat)
    h = 1e-6
    Pp = PoissonProblem(dev, fixed_charge=(sig + h) * pat)
    Pm = PoissonProblem(dev, fixed_charge=(sig - h) * pat)
    php, _ = Pp.solve(phi0=phi)
    phm, _ = Pm.solve(phi0=phi)
    fd = (C.electron_counts(Pp, php)[0] - C.electron_counts(Pm, phm)[0]) / (2 * h)
    assert abs(slope - fd) <= 1e-5 * abs(fd)


# ---------------------------------------------------------------------------
# Pins of electron_counts (Sec. III: N is the integrated electron density of the dot region) and
# of device_potential (Eq. SchrodPotEnergy: V = q phi_ref - chi - q phi).

def _count_device(statistics):
    # 100 x 100 nm, 10 x 10 elements of 10 nm; Si 50 nm in 10 layers of 5 nm under SiO2 10 nm in two;
    # element centroids at x, y = 5, 15, ..., 95 and z = 2.5, 7.5, ..., 57.5
    dev = W.mos_capacitor(nx=10, ny=10, nz=12, L=100.0, t_si=50.0, t_ox=10.0, n_ox=2, T=300.0,
                          statistics=statistics)
    dev["dots"] = [
        # faces through element centroids: x centroids 15, 25, 35, y 45, 55, 65 (closed box), z centroids
        # 42.5, 47.5 in Si and 52.5, 57.5 in the oxide (not semiconductor): 3 x 3 x 2 Si elements
        dict(x0=15.0, x1=35.0, y0=45.0, y1=65.0, z0=42.5, z1=57.5),
        # oxide only: no electrons
        dict(x0=0.0, x1=100.0, y0=0.0, y1=100.0, z0=51.0, z1=60.0),
        # faces just inside the centroids 15 and 35: the single column x = 25, one layer z = 2.5
        dict(x0=15.000001, x1=34.999999, y0=55.0, y1=55.0, z0=0.0, z1=5.0),
    ]
    return dev


@pytest.mark.parametrize("statistics", [0, 1])
def test_electron_counts_uniform_potential_closed_form(statistics):
    # at a uniform potential the density is one number n(phi) in every Si element, so
    # N_d = n(phi) x (volume of the dot's Si elements) exactly: 18 elements of 500 nm^3, none, and 1
    dev = _count_device(statistics)
    P = PoissonProblem(dev)
    phi0 = 0.31
    n_pt = physics.carrier_terms(np.array([phi0]), P.si, P.T, P.phi_r, P.E_F, statistics, 1)["n"][0]
    N = C.electron_counts(P, np.full(P.mesh.n_nodes, phi0))
    vol = np.array([18 * 500.0, 0.0, 1 * 500.0])
    assert N.shape == (3,)
    assert np.max(np.abs(N - n_pt * vol)) <= 1e-12 * n_pt * vol[0]
    if statistics == 0:
        # Maxwell-Boltzmann: N scales as exp(q dphi / k_B T) (CODATA constants, no oracle physics)
        dphi = 0.02
        N2 = C.electron_counts(P, np.full(P.mesh.n_nodes, phi0 + dphi))
        kT = 1.380649e-23 * 300.0 / 1.602176634e-19
        assert abs(N2[0] / N[0] - math.exp(dphi / kT)) <= 1e-12 * math.exp(dphi / kT)


def test_electron_counts_integrates_a_varying_density():
    # potential linear in x across the dot: n varies exponentially (MB), and the 2x2x2 Gauss sum of
    # each element approximates its integral (closed form of exp over an interval) to O(h^4) per element
    dev = _count_device(0)
    P = PoissonProblem(dev)
    a = 0.004  # V/nm
    phi = 0.25 + a * (P.mesh.coords[:, 0] - 50.0)
    N = C.electron_counts(P, phi)
    kT = 1.380649e-23 * 300.0 / 1.602176634e-19
    n0 = physics.carrier_terms(np.array([0.25]), P.si, P.T, P.phi_r, P.E_F, 0, 1)["n"][0]
    beta = a / kT  # n(x) = n0 exp(beta (x - 50))
    ix = math.exp(beta * (35.0 + 5.0 - 50.0)) - math.exp(beta * (15.0 - 5.0 - 50.0))
    exact = n0 * ix / beta * 30.0 * 10.0  # dot 0: x in [10, 40], y extent 30, z extent 10 (Si)
    assert abs(N[0] - exact) <= 2e-3 * exact


def _ramp_device():
    # 2 x 2 nm strip (one transverse mode), Si 40 nm in 160 layers of 0.25 nm, gate -1 V on top,
    # Ohmic bottom, 300 K; Schrodinger subdomain z in [10, 40] nm
    dev = W.mos_capacitor(nx=2, ny=2, nz=160, L=2.0, t_si=40.0, t_ox=1.0, n_ox=1, V_gate=-1.0, T=300.0)
    dev["layers"] = [dict(material=0, thickness=40.0, n=160)]
    dev["subdomain"] = dict(i0=0, i1=2, j0=0, j1=2, k0=40, k1=160)
    return dev


def test_device_potential_on_a_linear_potential_and_its_airy_levels():
    dev = _ramp_device()
    P = PoissonProblem(dev, linear=True)
    phi = P.initial_guess()  # the charge-free solution: linear in z, nodally exact for Q1
    m = P.mesh
    phib, phit = phi[m.nk == 0][0], phi[m.nk == m.nz][0]
    assert abs(phit - (-1.0)) < 1e-14 and phib > phit
    sel = m.subdomain_elements()
    Vq = S.device_potential(P, phi, sel)
    # Gauss points of each element in z: centre +- h / (2 sqrt 3)
    h = 0.25
    zc = m.elem_coords[sel][:, :, 2].mean(axis=1)
    sz = np.array([2 * ((q >> 2) & 1) - 1 for q in range(8)], dtype=float)
    zq = zc[:, None] + sz[None, :] * h / (2.0 * math.sqrt(3.0))
    phiq = phib + (phit - phib) * zq / 40.0
    assert np.max(np.abs(Vq - (P.phi_r - P.si["chi"] - phiq))) < 1e-13
    # the energy rises with z (V = q phi_ref - chi - q phi, phi falls towards the gate): a triangular
    # well on the subdomain's lower wall, E_1 = V(10 nm) + (hbar^2 F^2 / 2m)^(1/3) |a_1|
    m_rel = 0.19
    F = (phib - phit) / 40.0
    kap = physics.hbar2_over_2m0() / m_rel
    a1 = -scipy.special.ai_zeros(1)[0][0]
    V0 = P.phi_r - P.si["chi"] - (phib + (phit - phib) * 10.0 / 40.0)
    E_exact = V0 + (kap * F ** 2) ** (1.0 / 3.0) * a1
    trans = 2.0 * kap * 6.0 * 0.5  # the strip's transverse mode (2 elements of 1 nm per axis)
    E, _, _, _, _ = S.solve_device(P, phi, nev=1, m_eff=(m_rel,) * 3)
    assert abs(E[0] - trans - E_exact) <= 3e-3 * (E_exact - V0), (E[0] - trans, E_exact)
    # a sign slip (V = q phi_ref - chi + q phi) puts the well against the upper wall, tenths of an eV away
    H, M, _ = S.operators(m, sel, m.subdomain_interior_nodes(), (m_rel,) * 3, P.phi_r - P.si["chi"] + phiq)
    Ef, _ = S.lowest_eigenpairs(H, M, 1, sigma=float(np.min(P.phi_r - P.si["chi"] + phiq)) - 0.01)
    assert abs(Ef[0] - trans - E_exact) > 0.1
