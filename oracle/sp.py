"""Self-consistent Schrodinger-Poisson loop by the predictor-corrector scheme (oracle, FP64).

Test infrastructure only (see ``oracle/__init__``). Follows Sec. II.C of Gao et
al. for electrons confined in all three directions (quantum dots):

- quantum region: the Schrodinger subdomain (Sec. II.B; its elements are all
  silicon); outside it the electron density stays semiclassical (Sec. II.A);
- exact quantum density (Eq. VolEDens3DConfined):
      n = sum_i 4 |psi_i|^2 / (1 + exp((E_i - E_F)/kT)),
  4 = two Delta_2 valleys x two spins, psi_i normalized to 1 over the region
  (M-orthonormal), with exp(-(E_i - E_F)/kT) in place of the Fermi factor
  when its argument exceeds 100 (the paper's low-temperature safeguard);
- predictor density (Eq. ApproxEDens3DConfined, the "minus sign" form):
  the same with E_i replaced by E_i - q(phi - phi^(k)), phi^(k) the potential
  the eigenpairs were computed at, so n~ depends on phi explicitly and the
  Poisson Jacobian has the analytic term d n~/d phi;
- potential energy V = q phi_ref - chi - q phi + V_xc(n) (Eq. SchrodPotEnergy)
  with the Hedin-Lundqvist local-density V_xc (Eq. Vxc) and the scalar mass of
  Eq. mxc;
- the procedure of Sec. II.C.2: (1) semiclassical Newton solve, V without
  V_xc; (2) eigenpairs in V^(k-1); (3) Newton solve of the Poisson equation
  with n~^(k), then n~^(k) and V^(k) with V_xc(n~^(k)) at the new potential;
  (4) stop when max |phi^(k) - phi^(k-1)| < delta for k >= 2.

Readings where the paper leaves a choice: the quantum density and V_xc live on the
2x2x2 Gauss points of the quantum region's elements (where the Poisson load
and the Schrodinger potential are integrated); q(phi - phi^(k)) in eV is
numerically phi - phi^(k) in V.
"""
from __future__ import annotations

import math

import numpy as np

from . import fem, physics
from . import schrodinger as S
from .poisson import PoissonProblem

DEGENERACY_3D = 4.0          # valleys x spins, Eq. VolEDens3DConfined
FERMI_CUTOFF = 100.0         # argument above which exp(-a) replaces 1/(1 + e^a)
HL_A, HL_B = 0.7734, 21.0    # Hedin-Lundqvist constants of Eq. Vxc


def m_xc(m_l, m_t):
    """Scalar exchange-correlation mass (units m0), Eq. mxc: 1/m = (1/m_l + 2/m_t)/3."""
    return 1.0 / ((1.0 / m_l + 2.0 / m_t) / 3.0)


def coulomb_ev_nm():
    """q^2 / (4 pi eps0) in eV*nm."""
    return physics.Q_E / (4.0 * math.pi * physics.EPS0) * 1e9


def bohr_nm():
    """Bohr radius a0 = 4 pi eps0 hbar^2 / (m0 q^2) in nm."""
    return 4.0 * math.pi * physics.EPS0 * physics.HBAR ** 2 / (physics.M0 * physics.Q_E ** 2) * 1e9


def vxc(n, eps_r, mxc):
    """Hedin-Lundqvist exchange-correlation potential energy (eV) at density n (nm^-3), Eq. Vxc.

    V_xc = -(q^2 / (4 pi^2 eps_s)) (3 pi^2 n)^(1/3) [1 + 0.7734 x ln(1 + 1/x)],
    x = (1/21) (4 pi n b^3 / 3)^(-1/3), b = 4 pi eps_s hbar^2 / (m_xc q^2)
    (b is the effective Bohr radius eps_r a0 / m_xc). V_xc(0) = 0.
    """
    n = np.asarray(n, dtype=np.float64)
    out = np.zeros_like(n)
    pos = n > 0
    npos = n[pos]
    b = eps_r * bohr_nm() / mxc
    x = (4.0 * math.pi * npos * b ** 3 / 3.0) ** (-1.0 / 3.0) / HL_B
    pref = coulomb_ev_nm() / (math.pi * eps_r)     # q^2/(4 pi^2 eps_s) = (q^2/(4 pi eps0)) / (pi eps_r)
    out[pos] = -pref * (3.0 * math.pi ** 2 * npos) ** (1.0 / 3.0) * (1.0 + HL_A * x * np.log1p(1.0 / x))
    return out


def fermi3d(a):
    """Occupation 1/(1 + e^a) and its derivative with respect to -a, with exp(-a) for a > 100.

    Returns (f, g) with g = -df/da: f (1 - f) below the cutoff, exp(-a) above it.
    """
    a = np.asarray(a, dtype=np.float64)
    f = np.empty_like(a)
    g = np.empty_like(a)
    hi = a > FERMI_CUTOFF
    f[hi] = np.exp(-a[hi])
    g[hi] = f[hi]
    lo = ~hi
    e = np.exp(np.minimum(a[lo], FERMI_CUTOFF))
    f[lo] = 1.0 / (1.0 + e)
    g[lo] = f[lo] * (1.0 - f[lo])
    return f, g


def qp_weights(problem, psi_full, sel):
    """4 |psi_i|^2 at the Gauss points of the quantum elements, shape (n_sel, 8, nev).

    psi_full: (n_nodes, nev), zero outside the region's interior (Dirichlet).
    """
    conn = problem.mesh.conn[sel]
    nev = psi_full.shape[1]
    W = np.empty((conn.shape[0], 8, nev))
    for i in range(nev):
        W[:, :, i] = DEGENERACY_3D * fem.interpolate(psi_full[:, i], conn) ** 2
    return W


def predictor_density(W, E, phi_q, phi_prev_q, E_F, kT):
    """n~ and d n~/d phi at the Gauss points, Eq. ApproxEDens3DConfined (the minus-sign form)."""
    a = (E[None, None, :] - E_F - (phi_q - phi_prev_q)[:, :, None]) / kT
    f, g = fermi3d(a)
    return np.sum(W * f, axis=2), np.sum(W * g, axis=2) / kT


class SPPoissonProblem(PoissonProblem):
    """The nonlinear Poisson problem of step (3): n~ replaces the semiclassical n in the quantum region."""

    def set_quantum(self, E, W, phi_prev):
        self.q_sel = self.mesh.subdomain_elements()
        self.q_E = np.asarray(E, dtype=np.float64)
        self.q_W = W
        self.q_phi_prev = fem.interpolate(phi_prev, self.mesh.conn[self.q_sel])

    def qp_charge(self, phi):
        rho, drho, n, dn = super().qp_charge(phi)
        if getattr(self, "q_sel", None) is None or self.linear:
            return rho, drho, n, dn
        sel = self.q_sel
        phq = fem.interpolate(phi, self.mesh.conn[sel])
        nt, dnt = predictor_density(self.q_W, self.q_E, phq, self.q_phi_prev, self.E_F, physics.kT_eV(self.T))
        rho = rho.copy()
        drho = drho.copy()
        n = n.copy()
        dn = dn.copy()
        # rho = p - n + ND+ - NA- (+ theta): swap the semiclassical n for n~
        rho[sel] += n[sel] - nt
        drho[sel] += dn[sel] - dnt
        n[sel] = nt
        dn[sel] = dnt
        return rho, drho, n, dn


def quantum_electrons(problem, W, E, phi, phi_prev):
    """Integral of n~ over the quantum region at phi (electrons)."""
    sel = problem.mesh.subdomain_elements()
    conn = problem.mesh.conn[sel]
    nt, _ = predictor_density(W, np.asarray(E), fem.interpolate(phi, conn), fem.interpolate(phi_prev, conn),
                              problem.E_F, physics.kT_eV(problem.T))
    return float(np.sum(problem.wdet[sel] * nt))


def sp_solve(dev, nev=10, m_eff=None, tol=1e-5, max_iter=60, use_vxc=True, fixed_iters=None, solver="cg",
             tol_R=1e-10, tol_dphi=1e-10):
    """Predictor-corrector S-P loop of Sec. II.C.2.

    Returns (phi, E, report) with report = dict(iters, dphi (per iteration), E1 (per iteration),
    n_quantum, converged, W (the last eigenpairs' Gauss-point weights), n_q (n~ at the last
    potential, Gauss points of the quantum region)). fixed_iters = K runs exactly K outer
    iterations.
    """
    if m_eff is None:
        m_eff = (0.19, 0.19, 0.19)
    P0 = PoissonProblem(dev)
    phi, rep0 = P0.solve(tol_R=tol_R, tol_dphi=tol_dphi, solver=solver)          # step (1)
    mesh = P0.mesh
    sel = mesh.subdomain_elements()
    interior = mesh.subdomain_interior_nodes()
    si = P0.si
    mxc = m_xc(si["m_l"], si["m_t"])
    vx_q = np.zeros((int(sel.sum()), 8))
    hist_d, hist_e = [], []
    E = None
    nq = 0.0
    converged = False
    k = 0
    while True:
        k += 1
        # step (2): eigenpairs in V^(k-1) = q phi_ref - chi - q phi^(k-1) + V_xc
        Vq = S.device_potential(P0, phi, sel) + vx_q
        H, M, idx = S.operators(mesh, sel, interior, m_eff, Vq)
        E, X = S.lowest_eigenpairs(H, M, nev, sigma=float(np.min(Vq)) - 1e-2)
        psi = np.zeros((mesh.n_nodes, nev))
        psi[idx, :] = X
        W = qp_weights(P0, psi, sel)
        # step (3): Poisson with n~^(k), warm-started at phi^(k-1)
        Pk = SPPoissonProblem(dev)
        Pk.set_quantum(E, W, phi)
        phi_new, rk = Pk.solve(phi0=phi, tol_R=tol_R, tol_dphi=tol_dphi, solver=solver)
        conn = mesh.conn[sel]
        nt, _ = predictor_density(W, E, fem.interpolate(phi_new, conn), fem.interpolate(phi, conn), P0.E_F,
                                  physics.kT_eV(P0.T))
        vx_q = vxc(nt, si["eps_r"], mxc) if use_vxc else np.zeros_like(nt)
        nq = float(np.sum(P0.wdet[sel] * nt))
        # step (4)
        d = float(np.max(np.abs(phi_new - phi)))
        hist_d.append(d)
        hist_e.append(float(E[0]))
        phi = phi_new
        if fixed_iters is not None:
            if k >= fixed_iters:
                break
            continue
        if k >= 2 and d < tol:
            converged = True
            break
        if k >= max_iter:
            break
    return phi, E, dict(iters=k, dphi=hist_d, E1=hist_e, n_quantum=nq, converged=converged, W=W, n_q=nt)
