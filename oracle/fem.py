"""Q1 hexahedral finite elements by 2x2x2 Gauss quadrature (oracle).

Test infrastructure only. Implements the weak forms the paper discretizes:
the Poisson weak form, Sec. II.A.3, Eq. PoissonWeakForm (boundary term
dropped = natural Neumann, Sec. II.A.4), and the Schrodinger weak form,
Sec. II.B, Eq. SchrodEqnWeakForm. Every volume integral uses 2x2x2 Gauss
quadrature on the trilinear map of each element (the paper names no rule; this one
is exact for stiffness and consistent mass on boxes, no lumping). The element geometry is
handled in the general isoparametric form (Jacobian of the trilinear map), so
nothing here assumes axis-aligned boxes.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

_G = 1.0 / np.sqrt(3.0)
# Reference corners a = ax + 2 ay + 4 az at xi = -1/+1; Gauss points q likewise at -/+ 1/sqrt(3).
CORNER_SIGN = np.array([[2 * (a & 1) - 1, 2 * ((a >> 1) & 1) - 1, 2 * ((a >> 2) & 1) - 1] for a in range(8)], dtype=np.float64)
QP = CORNER_SIGN * _G
QW = np.ones(8)


def shape(xi):
    """N_a(xi) = prod_d (1 + s_ad xi_d)/2 for the 8 corners."""
    return np.prod(0.5 * (1.0 + CORNER_SIGN * xi[None, :]), axis=1)


def shape_grad_ref(xi):
    """dN_a/dxi_d, shape (8, 3)."""
    f = 0.5 * (1.0 + CORNER_SIGN * xi[None, :])
    g = np.empty((8, 3))
    for d in range(3):
        others = [e for e in range(3) if e != d]
        g[:, d] = 0.5 * CORNER_SIGN[:, d] * f[:, others[0]] * f[:, others[1]]
    return g


NQ = np.stack([shape(QP[q]) for q in range(8)])            # (q, a)
DNQ = np.stack([shape_grad_ref(QP[q]) for q in range(8)])  # (q, a, d)


def geometry(elem_coords):
    """Per element and qp: weight*|J| (Ne, 8) and physical shape gradients (Ne, 8q, 8a, 3)."""
    # J[e,q,i,d] = sum_a x[e,a,i] dN_a/dxi_d(q)
    J = np.einsum("eai,qad->eqid", elem_coords, DNQ)
    detJ = np.linalg.det(J)
    if np.any(detJ <= 0):
        raise ValueError("inverted element")
    Jinv = np.linalg.inv(J)  # [e,q,d,i]
    # grad_x N_a = J^{-T} grad_xi N_a : g[e,q,a,i] = sum_d Jinv[e,q,d,i] dN[q,a,d]
    grad = np.einsum("eqdi,qad->eqai", Jinv, DNQ)
    wdet = detJ * QW[None, :]
    return wdet, grad


def interpolate(vals_at_nodes, conn):
    """Value at each element qp: u[e,q] = sum_a N_a(q) v[conn[e,a]]."""
    return np.einsum("qa,ea->eq", NQ, vals_at_nodes[conn])


def element_stiffness(wdet, grad, kappa):
    """K_e[a,b] = sum_q w|J| sum_d kappa_d grad_d N_a grad_d N_b; kappa shape (Ne, 3)."""
    return np.einsum("eq,ed,eqad,eqbd->eab", wdet, kappa, grad, grad)


def element_mass(wdet, coef):
    """M_e[a,b] = sum_q w|J| coef[e,q] N_a(q) N_b(q)."""
    return np.einsum("eq,eq,qa,qb->eab", wdet, coef, NQ, NQ)


def element_load(wdet, f):
    """F_e[a] = sum_q w|J| f[e,q] N_a(q)."""
    return np.einsum("eq,eq,qa->ea", wdet, f, NQ)


def assemble_matrix(conn, Ke, n):
    rows = np.repeat(conn, 8, axis=1).ravel()
    cols = np.tile(conn, (1, 8)).ravel()
    return sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(n, n)).tocsr()


def assemble_vector(conn, Fe, n):
    out = np.zeros(n)
    np.add.at(out, conn.ravel(), Fe.ravel())
    return out
