"""Dot electron counts, finite-difference capacitance and adjoint sensitivities (oracle).

Test infrastructure only.

- N_d = int_{dot d} n dOmega by 2x2x2 Gauss quadrature (Sec. III, capacitance
  equation: N_{1,2} is the integrated electron density of the quantum region).
- C = q (N_2 - N_1) / dV with dV on one gate (Sec. III), reported in aF.
- Adjoint (reading of the differentiation form): with R(phi, V, theta) = 0 on
  the free nodes and phi held at the gate values on Dirichlet nodes,
      J_ff lambda = dN/dphi_f,
      dN/dV_g   = dN/dphi_D . e_g - lambda . (J_fD e_g - db_f/dV_g),
      dN/dtheta_e = (q/eps0) sum_{a in e, free} lambda_a int_e N_a,
      dN/dsigma  = lambda . db_f/dsigma   (surface charges, charged gates),
  b the surface load of ``oracle.boundary`` (db/dV_g nonzero only for a
  charged gate, whose potential enters through the Robin condition).
  J is symmetric, so the adjoint system uses J itself.
"""
from __future__ import annotations

import numpy as np

from . import fem, physics
from .poisson import PoissonProblem, solve_spd

Q_AF = physics.Q_E * 1e18  # q in C scaled to aF*V


def electron_counts(problem: PoissonProblem, phi):
    """N_d for every dot (electrons)."""
    _, _, n, _ = problem.qp_charge(phi)
    out = []
    for d in range(len(problem.dev["dots"])):
        sel = problem.mesh.dot_elements(d)
        out.append(float(np.sum(problem.wdet[sel] * n[sel])))
    return np.array(out)


def count_gradient(problem: PoissonProblem, phi, d):
    """dN_d/dphi as a nodal vector: sum_{e in dot} sum_q w|J| n'(phi_q) N_a(q)."""
    _, _, _, dn = problem.qp_charge(phi)
    sel = problem.mesh.dot_elements(d)
    coef = np.where(sel[:, None], dn, 0.0)
    return fem.assemble_vector(problem.mesh.conn, fem.element_load(problem.wdet, coef), problem.mesh.n_nodes)


def fd_capacitance(dev, gate, dV=0.01, fixed_charge=None, phi0=None, **solve_kw):
    """Forward-difference dot-to-gate capacitances C_d = q (N_d(V+dV) - N_d(V)) / dV in aF (Sec. III)."""
    P1 = PoissonProblem(dev, fixed_charge=fixed_charge)
    phi1, _ = P1.solve(phi0=phi0, **solve_kw)
    N1 = electron_counts(P1, phi1)
    bias = dict(dev["bias"])
    bias["V_gate"] = list(bias["V_gate"])
    bias["V_gate"][gate] += dV
    P2 = PoissonProblem(dev, bias=bias, fixed_charge=fixed_charge)
    phi2, _ = P2.solve(phi0=phi1, **solve_kw)
    N2 = electron_counts(P2, phi2)
    return Q_AF * (N2 - N1) / dV, N1, N2


def adjoint(problem: PoissonProblem, phi, solver="cg"):
    """(dN/dV  [n_dots x n_gates],  dN/dtheta [n_dots x n_elems]) at a converged phi."""
    m = problem.mesh
    f, D = problem.free, problem.dir
    J = problem.jacobian(phi)
    Jff = J[f][:, f]
    JfD = J[f][:, D]
    n_g = len(problem.bias["V_gate"])
    n_d = len(problem.dev["dots"])
    dN_dV = np.zeros((n_d, n_g))
    dN_dth = np.zeros((n_d, m.n_elems))
    # int_e N_a for every element corner
    intN = np.einsum("eq,qa->ea", problem.wdet, fem.NQ)
    for d in range(n_d):
        g = count_gradient(problem, phi, d)
        lam = np.zeros(m.n_nodes)
        lam[f] = solve_spd(Jff, g[f], solver)
        for gi in range(n_g):
            e_g = (problem.gate[D] == gi).astype(np.float64)  # d phi_D / d V_g (Eq. ContOnIns)
            db = problem.dV.get(gi, np.zeros(m.n_nodes))[f]
            dN_dV[d, gi] = g[D] @ e_g - lam[f] @ (JfD @ e_g - db)
        lam_free = np.where(f, lam, 0.0)
        dN_dth[d] = problem.qe * np.sum(intN * lam_free[m.conn], axis=1)
    return dN_dV, dN_dth


def surface_charge_sensitivity(problem: PoissonProblem, phi, solver="cg"):
    """dN_d/dsigma (electrons per nm^-2) at a converged phi.

    Returns (by_sheet [n_dots x n_surface_charges], by_gate {g: [n_dots]} for charged gates):
    dN/dsigma = lambda . db_f/dsigma with J_ff lambda = dN/dphi_f.
    """
    f = problem.free
    Jff = problem.jacobian(phi)[f][:, f]
    n_d = len(problem.dev["dots"])
    sheet = np.zeros((n_d, len(problem.dsig_sheet)))
    gate = {g: np.zeros(n_d) for g in problem.dsig_gate}
    for d in range(n_d):
        lam = solve_spd(Jff, count_gradient(problem, phi, d)[f], solver)
        for s, db in enumerate(problem.dsig_sheet):
            sheet[d, s] = lam @ db[f]
        for g, db in problem.dsig_gate.items():
            gate[g][d] = lam @ db[f]
    return sheet, gate


def calibrate_sheet_charge(dev, dot, target, pattern, bracket=(-5e-3, 5e-3), xtol=1e-14, **solve_kw):
    """Interface sheet charge sigma (nm^-2) with N_dot(sigma) = target (Sec. III: the effective
    interface charge Q_it is tuned until the dot holds the target number of electrons).

    The fixed charge is theta = sigma * pattern (pattern: theta of a unit sheet). A plain bracketed
    root find (Brent) on N_dot(sigma) - target with the oracle's Newton solve at each sigma.
    Returns (sigma, N_dot, phi).
    """
    from scipy.optimize import brentq
    pattern = np.asarray(pattern, dtype=np.float64)
    cache = {}

    def f(sig):
        P = PoissonProblem(dev, fixed_charge=sig * pattern)
        phi, _ = P.solve(**solve_kw)
        N = electron_counts(P, phi)[dot]
        cache[sig] = (N, phi)
        return N - target

    sig = brentq(f, bracket[0], bracket[1], xtol=xtol, rtol=4 * np.finfo(float).eps, maxiter=200)
    if sig not in cache:
        f(sig)
    N, phi = cache[sig]
    return sig, N, phi
