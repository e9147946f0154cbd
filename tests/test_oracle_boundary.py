"""Pins of the oracle's surface terms: charged gates (Robin) and surface charges (Sec. II.A.4), CPU only.

Each test checks the oracle against something other than its own formulas: the closed-form
bilinear face mass and the area of tilted faces; the series-capacitor network of a laterally
uniform stack, where a sheet charge and a gate behind a gap of thickness d are lumped capacitors
and charges (Gauss's law, nodally exact for linear elements); the thin-dielectric-layer model the
Robin condition stands in for (the paper's own alternative: a layer of thin elements over the
gate, a Dirichlet gate on top of it and a Neumann sheet under it); the Dirichlet gate it tends to
as d -> 0; and the adjoint against central differences.
"""
import copy

import numpy as np
import pytest

import workloads as W
from oracle import boundary
from oracle import capacitance as C
from oracle.mesh import Mesh
from oracle.poisson import PoissonProblem

BILINEAR_MASS = np.array([[4, 2, 2, 1], [2, 4, 1, 2], [2, 1, 4, 2], [1, 2, 2, 4]]) / 36.0


def test_face_mass_closed_form_and_tilted_faces():
    dev = W.mos_capacitor(nx=3, ny=4, nz=6, L=30.0, t_si=40.0, t_ox=8.0, n_ox=3)
    m = Mesh(dev)
    faces = boundary.plane_faces(m, m.nz, dev["gates"][0])
    assert faces.shape == (12, 4)
    wdA = boundary.face_geometry(m.coords[faces])
    # rectangle hx x hy: M = hx hy / 36 [[4 2 2 1] ...] (corner a = ax + 2 ay)
    assert np.max(np.abs(boundary.face_mass(wdA) - 10.0 * 7.5 * BILINEAR_MASS)) < 1e-13
    # a parallelogram tilted out of every coordinate plane: the map is affine, so the same matrix
    # times its area |u x v|
    o, u, v = np.array([1.0, -2.0, 0.5]), np.array([3.0, 1.0, 2.0]), np.array([-1.0, 2.5, 0.7])
    X = np.array([[o, o + u, o + v, o + u + v]])
    area = np.linalg.norm(np.cross(u, v))
    Mf = boundary.face_mass(boundary.face_geometry(X))[0]
    assert np.max(np.abs(Mf - area * BILINEAR_MASS)) < 1e-13 * area
    # a planar trapezoid: int 1 dGamma equals its shoelace area
    X = np.array([[[0.0, 0.0, 2.0], [4.0, 0.0, 2.0], [1.0, 3.0, 2.0], [3.0, 3.0, 2.0]]])
    shoelace = 0.5 * 3.0 * (4.0 + 2.0)
    assert abs(boundary.face_load(boundary.face_geometry(X)).sum() - shoelace) < 1e-13
    # and its mass matrix, whose surface Jacobian varies over the face: int N_a N_b dGamma by a
    # 3x3 Gauss-Legendre rule on the map written as (1-s)(1-t) X0 + s(1-t) X1 + (1-s)t X2 + st X3,
    # its tangents by central differences (exact: the map is linear in each variable)
    Xc = X[0]

    def basis(s, t):
        return np.array([(1 - s) * (1 - t), s * (1 - t), (1 - s) * t, s * t])

    def point(s, t):
        return basis(s, t) @ Xc

    g3, w3 = np.polynomial.legendre.leggauss(3)
    ref = np.zeros((4, 4))
    for a, wa in zip(g3, w3):
        for b, wb in zip(g3, w3):
            s, t = (1 + a) / 2, (1 + b) / 2
            ts = (point(s + 0.25, t) - point(s - 0.25, t)) / 0.5
            tt = (point(s, t + 0.25) - point(s, t - 0.25)) / 0.5
            Nv = basis(s, t)
            ref += 0.25 * wa * wb * np.linalg.norm(np.cross(ts, tt)) * np.outer(Nv, Nv)
    assert np.max(np.abs(boundary.face_mass(boundary.face_geometry(X))[0] - ref)) < 1e-13
    with pytest.raises(ValueError):
        boundary.node_plane(m, 41.0)
    assert boundary.node_plane(m, 48.0) == m.nz


def _stack(V_gate=0.7):
    return W.mos_capacitor(nx=3, ny=4, nz=12, L=30.0, t_si=40.0, t_ox=8.0, n_ox=3, V_gate=V_gate)


@pytest.mark.parametrize("sigma", [0.0, 2e-3, -3e-3])
def test_charged_gate_is_the_series_capacitor_network(sigma):
    # gap d (oxide) between the gate at phi0 and the top surface, sheet q sigma on the surface, then
    # the oxide and silicon layers down to the Ohmic contact: capacitors per unit area eps_r / t
    d = 10.0
    dev = _stack()
    dev["gates"][0]["robin"] = dict(sigma=sigma, d=d)
    P = PoissonProblem(dev, linear=True)
    assert not np.any(P.dir[P.gate == 0])                   # the charged gate's nodes are unknowns
    phi = P.initial_guess(solver="direct")
    c_gap, c_ox, c_si = 3.9 / d, 3.9 / 8.0, 11.7 / 40.0
    c_s = 1.0 / (1.0 / c_ox + 1.0 / c_si)
    pb = P.phi_ohm
    p_top = (c_gap * 0.7 + c_s * pb + P.qe * sigma) / (c_gap + c_s)
    p_if = pb + (p_top - pb) * c_s / c_si
    z = P.mesh.coords[:, 2]
    exact = np.where(z <= 40.0, pb + (p_if - pb) * z / 40.0, p_if + (p_top - p_if) * (z - 40.0) / 8.0)
    assert np.max(np.abs(phi - exact)) < 1e-13
    # positive sheet charge raises the potential under it
    if sigma:
        dev0 = _stack()
        dev0["gates"][0]["robin"] = dict(sigma=0.0, d=d)
        top = P.mesh.nk == P.mesh.nz
        top0 = PoissonProblem(dev0, linear=True).initial_guess(solver="direct")[top]
        assert np.all(np.sign(phi[top] - top0) == np.sign(sigma))


@pytest.mark.parametrize("sigma", [1.5e-3, -2e-3])
def test_surface_charge_kinks_the_stack_by_gauss_law(sigma):
    # sheet on the Si/SiO2 interface: D jumps by q sigma there (Eq. NeuBC4fc)
    dev = _stack()
    dev["surface_charges"] = [dict(z=40.0, x0=0.0, x1=30.0, y0=0.0, y1=30.0, sigma=sigma)]
    P = PoissonProblem(dev, linear=True)
    phi = P.initial_guess(solver="direct")
    c_ox, c_si = 3.9 / 8.0, 11.7 / 40.0
    pb = P.phi_ohm
    p_if = (c_ox * 0.7 + c_si * pb + P.qe * sigma) / (c_ox + c_si)
    z = P.mesh.coords[:, 2]
    exact = np.where(z <= 40.0, pb + (p_if - pb) * z / 40.0, p_if + (0.7 - p_if) * (z - 40.0) / 8.0)
    assert np.max(np.abs(phi - exact)) < 1e-13


def test_surface_charge_patch_total_flux():
    # a patch smaller than the device: the contacts' reactions carry exactly the sheet's charge
    dev = W.mos_capacitor(nx=6, ny=6, nz=8, L=60.0, t_si=40.0, t_ox=8.0, n_ox=2, V_gate=0.3)
    sig = 2.5e-3
    dev["surface_charges"] = [dict(z=40.0, x0=10.0, x1=40.0, y0=20.0, y1=50.0, sigma=sig)]
    P = PoissonProblem(dev, linear=True)
    phi = P.initial_guess(solver="direct")
    Rf = P.residual(phi, full=True)
    assert np.max(np.abs(Rf[P.free])) < 1e-12
    assert abs(Rf[P.dir].sum() / (-P.qe * sig * 30.0 * 30.0) - 1.0) < 1e-12
    assert abs(P.dsig_sheet[0].sum() / (P.qe * 900.0) - 1.0) < 1e-13


def _mos_with_interface_charge():
    dev = W.mos_capacitor(nx=8, ny=8, nz=12, L=80.0, t_si=50.0, t_ox=10.0, n_ox=4, V_gate=0.4, T=300.0)
    theta = np.array(W.interface_fixed_charge(dev, seed=7, sigma_std=2e-3))
    return dev, theta


def test_charged_gate_equals_a_thin_dielectric_gap():
    # the alternative the Robin condition replaces: one extra oxide element layer of thickness d, the
    # gate as a Dirichlet plane on top of it and the sheet as a surface charge under it. The two agree
    # as d -> 0 (the random interface charge makes the solution laterally non-uniform, so the gap
    # layer's lateral stiffness matters), while flipping the sheet's sign in either model would leave
    # a difference of q sigma d / eps_ox = 7e-3 V at d = 1 nm.
    dev, theta = _mos_with_interface_charge()
    sig = -1.5e-3
    diffs = []
    for d in (1.0, 0.5, 0.25):
        rob = copy.deepcopy(dev)
        rob["gates"][0]["robin"] = dict(sigma=sig, d=d)
        P = PoissonProblem(rob, fixed_charge=theta)
        phi_r, rep = P.solve()
        assert rep["converged"]
        gap = copy.deepcopy(dev)
        gap["layers"] = gap["layers"] + [dict(material=1, thickness=d, n=1)]
        gap["surface_charges"] = [dict(z=60.0, x0=0.0, x1=80.0, y0=0.0, y1=80.0, sigma=sig)]
        P2 = PoissonProblem(gap, fixed_charge=np.concatenate([theta, np.zeros(64)]))
        phi_g, rep2 = P2.solve()
        assert rep2["converged"]
        diffs.append(np.max(np.abs(phi_r - phi_g[:P.mesh.n_nodes])))
    assert diffs[0] < 2e-5, diffs
    assert diffs[1] < diffs[0] / 4 and diffs[2] < diffs[1] / 4, diffs


def test_charged_gates_tend_to_dirichlet_gates():
    # five gates on grid lines (5 nm cells), 4 K: with sigma = 0 and d -> 0 the Robin condition pins
    # the top surface under each gate to phi0, the Dirichlet gate; the difference is O(d)
    dev = W.five_gate_device(n=(40, 40, 8), T=4.0, with_subdomain=False)
    dev["bias"]["V_gate"] = [0.35, 0.95, 0.45, 0.9, 0.3]
    phi_d, rep = PoissonProblem(dev).solve()
    assert rep["converged"]
    errs = []
    for d in (1e-2, 5e-3):
        rob = copy.deepcopy(dev)
        for G in rob["gates"]:
            G["robin"] = dict(sigma=0.0, d=d)
        phi, rep = PoissonProblem(rob).solve(phi0=phi_d)
        assert rep["converged"]
        errs.append(np.max(np.abs(phi - phi_d)))
    assert errs[0] < 0.03 and 1.8 < errs[0] / errs[1] < 2.2, errs


def test_charged_gate_and_surface_charge_sensitivities():
    dev = W.five_gate_device(n=(16, 16, 12), T=4.0)
    dev["bias"]["V_gate"] = [0.35, 0.95, 0.45, 1.1, 0.3]
    dev["gates"][3]["robin"] = dict(sigma=5e-4, d=10.0)       # plunger P2 charged
    dev["surface_charges"] = [dict(z=90.0, x0=100.0, x1=150.0, y0=50.0, y1=150.0, sigma=2e-3)]
    P = PoissonProblem(dev)
    phi, rep = P.solve()
    assert rep["converged"]
    dN_dV, _ = C.adjoint(P, phi)
    sheet, gate = C.surface_charge_sensitivity(P, phi)

    def counts(edit):
        d2 = copy.deepcopy(dev)
        edit(d2)
        P2 = PoissonProblem(d2)
        ph, r = P2.solve(phi0=phi)
        assert r["converged"]
        return C.electron_counts(P2, ph)

    def central(edit, h):
        return (counts(lambda d2: edit(d2, h)) - counts(lambda d2: edit(d2, -h))) / (2 * h)

    for g in (2, 3):                                            # a Dirichlet and the charged gate
        fd = central(lambda d2, s: d2["bias"]["V_gate"].__setitem__(g, d2["bias"]["V_gate"][g] + s), 1e-4)
        assert np.max(np.abs(fd - dN_dV[:, g])) < 1e-5 * np.max(np.abs(dN_dV[:, g]))
    fd = central(lambda d2, s: d2["surface_charges"][0].__setitem__("sigma", 2e-3 + s), 1e-5)
    assert np.max(np.abs(fd - sheet[:, 0])) < 1e-4 * np.max(np.abs(sheet[:, 0]))
    fd = central(lambda d2, s: d2["gates"][3]["robin"].__setitem__("sigma", 5e-4 + s), 1e-5)
    assert np.max(np.abs(fd - gate[3])) < 1e-4 * np.max(np.abs(gate[3]))
    assert dN_dV[1, 3] > 1.0 and gate[3][1] > 0.0              # the plunger and its charge fill dot 1


def test_random_stacks_match_the_capacitor_network():
    # random linear stacks (layer permittivities, thicknesses and element counts), a charged top gate
    # (random sigma and d) and sheets on random interfaces: at every layer boundary the potential is
    # that of the lumped network of per-area capacitors eps_r/t with the sheets as node charges and the
    # gate behind c = eps_top/d (Gauss's law; linear elements are nodally exact on such stacks)
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies

    @hyp.settings(max_examples=25, deadline=None)
    @hyp.given(st.lists(st.tuples(st.floats(1.5, 15.0), st.integers(1, 6), st.integers(1, 3)), min_size=1, max_size=4),
               st.floats(-1.0, 1.0), st.floats(-3e-3, 3e-3), st.floats(0.5, 20.0),
               st.lists(st.floats(-3e-3, 3e-3), min_size=3, max_size=3))
    def check(layers, V, sig_g, d, sig_if):
        mats = [dict(W.SI, eps_r=11.7)] + [dict(W.SIO2, eps_r=e) for e, _, _ in layers]
        dev = dict(Lx=20.0, Ly=10.0, nx=2, ny=1,
                   layers=[dict(material=q + 1, thickness=2.0 * t, n=n) for q, (_, t, n) in enumerate(layers)],
                   materials=mats, gates=[dict(name="G", x0=0.0, x1=20.0, y0=0.0, y1=10.0, robin=dict(sigma=sig_g, d=d))],
                   gate_work_function=None, bottom_ohmic=1, dots=[], subdomain=None,
                   bias=dict(T=300.0, V_gate=[V], V_sub=0.0, statistics=1, incomplete_ionization=1))
        zb = np.cumsum([0.0] + [2.0 * t for _, t, _ in layers])      # layer boundaries
        sheets = [dict(z=float(zb[j]), x0=0.0, x1=20.0, y0=0.0, y1=10.0, sigma=sig_if[j - 1])
                  for j in range(1, len(layers))]
        dev["surface_charges"] = sheets
        P = PoissonProblem(dev, linear=True)
        phi = P.initial_guess(solver="direct")
        m = len(layers)
        c = [e / (2.0 * t) for e, t, _ in layers]
        A = np.zeros((m, m))
        b = np.zeros(m)
        for j in range(1, m + 1):                # unknown u_j at boundary j (u_0 = phi_ohm)
            A[j - 1, j - 1] += c[j - 1]
            if j > 1:
                A[j - 1, j - 2] -= c[j - 1]
            else:
                b[0] += c[0] * P.phi_ohm
            if j < m:
                A[j - 1, j - 1] += c[j]
                A[j - 1, j] -= c[j]
                b[j - 1] += P.qe * sig_if[j - 1]
        cg = layers[-1][0] / d
        A[m - 1, m - 1] += cg
        b[m - 1] += cg * V + P.qe * sig_g
        u = np.linalg.solve(A, b)
        z = P.mesh.coords[:, 2]
        for j in range(1, m + 1):
            at = np.abs(z - zb[j]) < 1e-9
            assert np.max(np.abs(phi[at] - u[j - 1])) < 1e-11 * max(1.0, np.max(np.abs(u)))

    check()


def test_plane_faces_are_the_quads_inside_the_closed_rectangle():
    # random rectangles, including edges on grid lines: the selected quads are exactly those whose
    # four corners lie in the closed rectangle (brute force over every quad of the plane)
    hyp = pytest.importorskip("hypothesis")
    st = hyp.strategies
    dev = W.mos_capacitor(nx=7, ny=5, nz=2, L=35.0, t_si=4.0, t_ox=2.0, n_ox=1)
    m = Mesh(dev)
    coord = st.one_of(st.floats(-2.0, 37.0), st.sampled_from([0.0, 5.0, 10.0, 17.5, 25.0, 35.0]))

    @hyp.settings(max_examples=60, deadline=None)
    @hyp.given(coord, coord, coord, coord, st.integers(0, 2))
    def check(xa, xb, ya, yb, k):
        R = dict(x0=min(xa, xb), x1=max(xa, xb), y0=min(ya, yb), y1=max(ya, yb))
        got = {tuple(sorted(f)) for f in boundary.plane_faces(m, k, R).tolist()}
        want = set()
        for j in range(m.ny):
            for i in range(m.nx):
                ids = [m.node_id(i + (a & 1), j + (a >> 1), k) for a in range(4)]
                xy = m.coords[ids][:, :2]
                if np.all((xy[:, 0] >= R["x0"]) & (xy[:, 0] <= R["x1"]) & (xy[:, 1] >= R["y0"]) & (xy[:, 1] <= R["y1"])):
                    want.add(tuple(sorted(ids)))
        assert got == want

    check()
