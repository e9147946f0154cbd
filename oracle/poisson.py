"""Nonlinear Poisson problem and its Newton solve (oracle, FP64).

Test infrastructure only. Follows Sec. II.A of Gao et al.:
-div(eps grad phi) = q (p - n + ND+ - NA-)   (Eq. Poisson)
in the weak form of Eq. PoissonWeakForm with natural Neumann boundaries,
gate Dirichlet values from Eq. ContOnIns and Ohmic values from the contact
formulas of Sec. II.A.4. The residual is scaled by 1/eps0:

    R_i(phi) = sum_e int eps_r grad phi . grad N_i  -  (q/eps0) int rho(phi) N_i

on free nodes, R_i = 0 on Dirichlet nodes (where phi is held at its value).
Devices may add the surface terms of ``oracle.boundary`` (charged gates under
the Robin condition, surface charges under Eq. NeuBC4fc): R gains K_R phi - b,
K_R = sum over charged gates of (eps_r/d) int_Gamma N_a N_b and b the constant
surface loads, both zero on every device without those keys.
The Jacobian J = K + K_R - (q/eps0) M[rho'] is differentiated by hand (the paper
uses automatic differentiation, Sec. II.C.2). Every linear
system is solved on the free-free block by a sparse direct solve (SuperLU) or
by Jacobi-preconditioned CG to a relative residual of 1e-14.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import boundary, fem, physics
from .mesh import Mesh


def semiconductor_material(dev):
    for m in dev["materials"]:
        if m["semiconductor"]:
            return m
    return dev["materials"][0]


class PoissonProblem:
    def __init__(self, dev: dict, bias: dict | None = None, fixed_charge=None, linear=False, mesh=None):
        self.dev = dev
        self.bias = dict(dev["bias"] if bias is None else bias)
        self.mesh = Mesh(dev) if mesh is None else mesh
        m = self.mesh
        self.T = self.bias["T"]
        self.si = semiconductor_material(dev)
        # One reference potential for the whole device: that of its semiconductor (Eq. qPhiRef).
        self.phi_r = physics.phi_ref(self.si, self.T)
        self.E_F = -self.bias.get("V_sub", 0.0)  # E_F = -q V_sub (Sec. II.A.2)
        self.linear = linear
        self.wdet, self.grad = fem.geometry(m.elem_coords)
        eps = np.array([dev["materials"][k]["eps_r"] for k in m.elem_mat])
        self.K = fem.assemble_matrix(m.conn, fem.element_stiffness(self.wdet, self.grad, np.repeat(eps[:, None], 3, axis=1)), m.n_nodes)
        self.qe = physics.q_over_eps0()
        self.theta = np.zeros(m.n_elems) if fixed_charge is None else np.asarray(fixed_charge, dtype=np.float64)
        # Dirichlet sets and values; the nodes of charged (Robin) gates stay unknowns
        gate = m.gate_of_node()
        ohm = m.ohmic_nodes()
        self.gate = gate
        charged = np.zeros(m.n_nodes, dtype=bool)
        for gi, G in enumerate(dev["gates"]):
            if G.get("robin"):
                charged |= gate == gi
        self.dir = ((gate >= 0) & ~charged) | ohm
        self.free = ~self.dir
        self.g = np.zeros(m.n_nodes)
        for gi, Vg in enumerate(self.bias["V_gate"]):
            if not dev["gates"][gi].get("robin"):
                self.g[gate == gi] = physics.gate_potential(Vg, self.phi_r, dev.get("gate_work_function"))
        self.phi_ohm = physics.ohmic_potential(self.si, self.T, self.phi_r, V_a=self.bias.get("V_sub", 0.0),
                                               statistics=self.bias.get("statistics", 1),
                                               incomplete=self.bias.get("incomplete_ionization", 1))
        self.g[ohm & (gate < 0)] = self.phi_ohm
        self.mat_of_elem = m.elem_mat
        self._surface_terms()

    def _surface_terms(self):
        """K_R, the surface load b and their derivatives with respect to V_g and sigma (oracle.boundary).

        dV[g]: d b / d V_g of charged gate g, (eps_r/d) int N_a (the Robin phi_0 = phi_ins of
        Eq. ContOnIns moves one-for-one with V_g); dsig_gate[g], dsig_sheet[s]: d b / d sigma,
        (q/eps0) int N_a over the faces.
        """
        m, dev = self.mesh, self.dev
        n = m.n_nodes
        self.KR = sp.csr_matrix((n, n))
        self.b_surf = np.zeros(n)
        self.dV = {}
        self.dsig_gate = {}
        self.dsig_sheet = []
        eps_top = dev["materials"][m.layer_mat[m.nz - 1]]["eps_r"]
        for gi, G in enumerate(dev["gates"]):
            rb = G.get("robin")
            if not rb:
                continue
            faces = boundary.plane_faces(m, m.nz, G)
            wdA = boundary.face_geometry(m.coords[faces])
            alpha = eps_top / rb.get("d", boundary.DEFAULT_GAP_NM)
            self.KR = self.KR + _assemble4(faces, alpha * boundary.face_mass(wdA), n)
            intN = fem.assemble_vector(faces, boundary.face_load(wdA), n)
            phi0 = physics.gate_potential(self.bias["V_gate"][gi], self.phi_r, dev.get("gate_work_function"))
            self.dV[gi] = alpha * intN
            self.dsig_gate[gi] = self.qe * intN
            self.b_surf += alpha * phi0 * intN + self.qe * rb.get("sigma", 0.0) * intN
        for S in dev.get("surface_charges", []):
            faces = boundary.plane_faces(m, boundary.node_plane(m, S["z"]), S)
            intN = fem.assemble_vector(faces, boundary.face_load(boundary.face_geometry(m.coords[faces])), n)
            self.dsig_sheet.append(self.qe * intN)
            self.b_surf += self.qe * S["sigma"] * intN
        self.KR = self.KR.tocsr()

    # ---------------------------------------------------------------
    def qp_charge(self, phi):
        """rho and d rho/d phi at every element qp (nm^-3, nm^-3/V), plus n and dn/dphi."""
        m = self.mesh
        phq = fem.interpolate(phi, m.conn)
        rho = np.zeros_like(phq)
        drho = np.zeros_like(phq)
        n = np.zeros_like(phq)
        dn = np.zeros_like(phq)
        if not self.linear:
            for mi, mat in enumerate(self.dev["materials"]):
                sel = self.mat_of_elem == mi
                if not np.any(sel) or not mat["semiconductor"]:
                    continue
                t = physics.carrier_terms(phq[sel], mat, self.T, self.phi_r, self.E_F,
                                          self.bias.get("statistics", 1), self.bias.get("incomplete_ionization", 1))
                rho[sel] = t["rho"]
                drho[sel] = t["drho"]
                n[sel] = t["n"]
                dn[sel] = t["dn"]
        rho = rho + self.theta[:, None]  # fixed charge adds to rho
        return rho, drho, n, dn

    def residual(self, phi, full=False):
        """R(phi) = (K + K_R) phi - (q/eps0) int rho N - b (free rows); zero on Dirichlet rows unless full."""
        rho, _, _, _ = self.qp_charge(phi)
        F = fem.assemble_vector(self.mesh.conn, fem.element_load(self.wdet, rho), self.mesh.n_nodes)
        R = self.K @ phi + self.KR @ phi - self.qe * F - self.b_surf
        if not full:
            R[self.dir] = 0.0
        return R

    def jacobian(self, phi):
        """J = K + K_R - (q/eps0) int rho'(phi) N_a N_b (all rows; callers restrict to free)."""
        _, drho, _, _ = self.qp_charge(phi)
        Mc = fem.assemble_matrix(self.mesh.conn, fem.element_mass(self.wdet, -self.qe * drho), self.mesh.n_nodes)
        return (self.K + self.KR + Mc).tocsr()

    def initial_guess(self, solver="cg"):
        """Laplace solve with the contact values and surface terms (rho = 0), the initial guess (the paper states none)."""
        phi = self.g.copy()
        f, d = self.free, self.dir
        A = (self.K + self.KR).tocsr()
        rhs = self.b_surf[f] - (A[f][:, d] @ self.g[d])
        phi[f] = solve_spd(A[f][:, f], rhs, solver)
        return phi

    def solve(self, phi0=None, tol_R=1e-10, tol_dphi=1e-10, max_newton=200, solver="cg", verbose=False):
        """Newton with backtracking on ||R||_2 (Armijo 1e-4, halving up to 30 times); the paper
        states no globalization.

        Stops when ||R||_inf < tol_R on free nodes and ||alpha delta||_inf < tol_dphi.
        Returns (phi, report).
        """
        phi = self.initial_guess(solver) if phi0 is None else np.array(phi0, dtype=np.float64)
        phi[self.dir] = self.g[self.dir]
        f = self.free
        R = self.residual(phi)
        nR = np.linalg.norm(R)
        hist = []
        for it in range(1, max_newton + 1):
            J = self.jacobian(phi)
            delta = np.zeros_like(phi)
            delta[f] = solve_spd(J[f][:, f], -R[f], solver)
            alpha = 1.0
            for _ in range(31):
                trial = phi + alpha * delta
                Rt = self.residual(trial)
                nRt = np.linalg.norm(Rt)
                if np.isfinite(nRt) and nRt <= (1.0 - 1e-4 * alpha) * nR:
                    break
                alpha *= 0.5
            phi, R, nR = trial, Rt, nRt
            step = alpha * np.max(np.abs(delta))
            rinf = np.max(np.abs(R))
            hist.append((it, alpha, rinf, step))
            if verbose:
                print("newton %3d alpha %.3g |R|inf %.3e |dphi|inf %.3e" % (it, alpha, rinf, step))
            if rinf < tol_R and step < tol_dphi:
                return phi, dict(newton_iters=it, res_inf=rinf, dphi_inf=step, history=hist, converged=True)
        return phi, dict(newton_iters=max_newton, res_inf=rinf, dphi_inf=step, history=hist, converged=False)


def _assemble4(faces, Mf, n):
    rows = np.repeat(faces, 4, axis=1).ravel()
    cols = np.tile(faces, (1, 4)).ravel()
    return sp.coo_matrix((Mf.ravel(), (rows, cols)), shape=(n, n)).tocsr()


def solve_spd(A, b, solver="cg", rtol=1e-14):
    """Solve A x = b for SPD A: Jacobi-PCG to relative residual rtol, or SuperLU ("direct").

    If CG stalls above rtol (it never has on the devices used here) the
    direct solve is used instead.
    """
    A = sp.csc_matrix(A) if solver == "direct" else sp.csr_matrix(A)
    if solver == "direct":
        return spla.spsolve(A, b)
    d = A.diagonal()
    Minv = spla.LinearOperator(A.shape, matvec=lambda r: r / d)
    x, info = spla.cg(A, b, rtol=rtol, atol=0.0, M=Minv, maxiter=200000)
    if info != 0:
        return spla.spsolve(sp.csc_matrix(A), b)
    return x
