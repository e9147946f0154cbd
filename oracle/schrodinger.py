"""Effective-mass Schrodinger eigenpairs on the quantum subdomain (oracle, FP64).

Test infrastructure only. Follows Sec. II.B of Gao et al.: the weak form of
Eq. SchrodEqnWeakForm with a diagonal mass tensor (Eq. Schrodinger3D: m_t in
x, y and m_l in z; the devices here use one isotropic mass),
psi = 0 on the subdomain boundary (Dirichlet, Sec. II.B) and the potential
energy of Eq. SchrodPotEnergy without V_xc:

    V = q phi_ref - chi - q phi      (eV).

H = sum_d (hbar^2 / 2 m_d) int d_d N_a d_d N_b + int V N_a N_b,
M = int N_a N_b, both by 2x2x2 Gauss quadrature, restricted to the interior
nodes. The lowest eigenpairs of H psi = E M psi come from SciPy's ARPACK in
shift-invert mode (the paper uses Trilinos/Anasazi, Sec. II.B).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import fem, physics


def operators(mesh, elem_sel, interior, m_eff, Vq):
    """Assembled (H, M) restricted to `interior` nodes.

    elem_sel: boolean element mask of the quantum region; interior: boolean node
    mask of unknowns; m_eff: (m_x, m_y, m_z) in m0; Vq: potential energy (eV)
    at the qp of the selected elements, shape (n_sel, 8).
    """
    conn = mesh.conn[elem_sel]
    wdet, grad = fem.geometry(mesh.elem_coords[elem_sel])
    h2m = physics.hbar2_over_2m0()
    kappa = np.tile(np.array([h2m / m_eff[0], h2m / m_eff[1], h2m / m_eff[2]]), (conn.shape[0], 1))
    Ke = fem.element_stiffness(wdet, grad, kappa)
    MVe = fem.element_mass(wdet, Vq)
    Me = fem.element_mass(wdet, np.ones_like(Vq))
    H = fem.assemble_matrix(conn, Ke + MVe, mesh.n_nodes)
    M = fem.assemble_matrix(conn, Me, mesh.n_nodes)
    idx = np.nonzero(interior)[0]
    return H[idx][:, idx].tocsc(), M[idx][:, idx].tocsc(), idx


def device_potential(problem, phi, elem_sel):
    """V(phi) = q phi_ref - chi_Si - q phi at the qp of the selected elements (Eq. SchrodPotEnergy, no V_xc)."""
    phq = fem.interpolate(phi, problem.mesh.conn[elem_sel])
    return problem.phi_r - problem.si["chi"] - phq


def lowest_eigenpairs(H, M, nev, sigma):
    """nev smallest eigenpairs of H x = E M x (ascending), M-orthonormal eigenvectors.

    sigma must lie below the spectrum (min V is a lower bound: H - V_min M is
    positive semidefinite), so shift-invert returns the smallest eigenvalues.
    """
    vals, vecs = spla.eigsh(H, k=nev, M=M, sigma=sigma, which="LM", tol=0.0)
    order = np.argsort(vals)
    vals, vecs = vals[order], vecs[:, order]
    # normalize in the M inner product (eigsh already does; re-do for clarity)
    for k in range(nev):
        vecs[:, k] /= np.sqrt(vecs[:, k] @ (M @ vecs[:, k]))
    return vals, vecs


def solve_device(problem, phi, nev=10, m_eff=None):
    """Eigenpairs of the device subdomain at potential phi. Returns (E, psi_full_interior, idx)."""
    mesh = problem.mesh
    sel = mesh.subdomain_elements()
    interior = mesh.subdomain_interior_nodes()
    if m_eff is None:
        m_eff = (0.19, 0.19, 0.19)
    Vq = device_potential(problem, phi, sel)
    H, M, idx = operators(mesh, sel, interior, m_eff, Vq)
    # shift: the lowest eigenvalue is above min V
    sigma = float(np.min(Vq)) - 1e-2
    E, X = lowest_eigenpairs(H, M, nev, sigma=sigma)
    return E, X, idx, H, M
