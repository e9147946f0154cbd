"""Surface terms of the Poisson weak form: charged gates (Robin) and surface charges (oracle, FP64).

Test infrastructure only (see ``oracle/__init__``). Sec. II.A.4 of Gao et al.:

- non-flux-conserving Neumann condition on an explicit surface, Eq. NeuBC4fc:
  the jump of the normal displacement across the surface equals a given sheet
  charge q sigma_s, enforced in integral form, so the weak form gains the load
  int_Gamma q sigma_s w dGamma (divided by eps0 like every other term here);
- Robin condition for a charged gate (Fig. RobinBCDiagram): the gate's potential
  phi_0 is pinned a distance d outside the surface and a sheet charge q sigma_s
  sits on the surface, so the outward flux is
      eps_s d phi/dn = eps_s (phi_0 - phi)/d + q sigma_s,
  which adds (eps_r/d) int_Gamma phi w to the bilinear form and
  int_Gamma ((eps_r/d) phi_0 + (q/eps0) sigma_s) w to the load.

Readings where the paper is silent or at odds with itself: the sign of the phi term is the one Gauss's
law across the gap gives (the well-posed sign; the paper states the Robin
coefficient and its figure with opposite signs); sigma_s > 0 is positive charge, as
in the Neumann jump condition; eps_s is the permittivity of the element under the
face; a gate's faces are the top-plane quads whose four corners lie in its closed
rectangle, and a charged gate's nodes are unknowns (not Dirichlet nodes); a surface
charge sits on the node plane at its z coordinate. Face integrals use 2x2 Gauss
quadrature on the bilinear map of each quad (exact for products of bilinear
functions on parallelograms).
"""
from __future__ import annotations

import numpy as np

_G = 1.0 / np.sqrt(3.0)
FACE_SIGN = np.array([[2 * (a & 1) - 1, 2 * ((a >> 1) & 1) - 1] for a in range(4)], dtype=np.float64)
FACE_QP = FACE_SIGN * _G
# N_a at the 4 Gauss points (q, a) and dN_a/dxi, dN_a/deta there (q, a, 2)
FACE_NQ = np.prod(0.5 * (1.0 + FACE_SIGN[None, :, :] * FACE_QP[:, None, :]), axis=2)
FACE_DNQ = np.stack([0.5 * FACE_SIGN[None, :, 0] * 0.5 * (1.0 + FACE_SIGN[None, :, 1] * FACE_QP[:, None, 1]),
                     0.5 * FACE_SIGN[None, :, 1] * 0.5 * (1.0 + FACE_SIGN[None, :, 0] * FACE_QP[:, None, 0])],
                    axis=2)
DEFAULT_GAP_NM = 10.0        # d of the charged-gate condition (the paper's choice)


def plane_faces(mesh, k, rect):
    """Node ids (nf, 4) of the quads of node plane k whose corners all lie in the closed rectangle.

    rect: dict with x0, x1, y0, y1 (nm). Corner a = ax + 2 ay of the quad at (i, j) is node
    (i + ax, j + ay, k).
    """
    if not 0 <= k <= mesh.nz:
        raise ValueError("node plane out of range")
    ix = np.nonzero((mesh.x[:-1] >= rect["x0"]) & (mesh.x[1:] <= rect["x1"]))[0]
    jy = np.nonzero((mesh.y[:-1] >= rect["y0"]) & (mesh.y[1:] <= rect["y1"]))[0]
    I, J = np.meshgrid(ix, jy, indexing="xy")
    I, J = I.ravel(), J.ravel()
    return np.stack([mesh.node_id(I + (a & 1), J + ((a >> 1) & 1), np.full_like(I, k)) for a in range(4)], axis=1)


def face_geometry(X):
    """Weight * surface Jacobian at the 4 Gauss points of each quad, shape (nf, 4).

    X: corner coordinates (nf, 4, 3). dGamma = |dx/dxi x dx/deta| dxi deta.
    """
    t = np.einsum("fai,qad->fqid", X, FACE_DNQ)
    n = np.cross(t[..., 0], t[..., 1])
    dA = np.linalg.norm(n, axis=2)
    if np.any(dA <= 0):
        raise ValueError("degenerate face")
    return dA


def face_mass(wdA, coef=None):
    """M_f[a, b] = sum_q w dA coef N_a(q) N_b(q), shape (nf, 4, 4)."""
    c = wdA if coef is None else wdA * coef
    return np.einsum("fq,qa,qb->fab", c, FACE_NQ, FACE_NQ)


def face_load(wdA, f=None):
    """F_f[a] = sum_q w dA f N_a(q), shape (nf, 4)."""
    c = wdA if f is None else wdA * f
    return np.einsum("fq,qa->fa", c, FACE_NQ)


def node_plane(mesh, z):
    """Index of the node plane at height z (nm); ValueError if the mesh has none there."""
    k = int(np.argmin(np.abs(mesh.z - z)))
    if abs(mesh.z[k] - z) > 1e-9 * max(1.0, abs(z)):
        raise ValueError("no node plane at z = %g nm" % z)
    return k
