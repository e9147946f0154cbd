"""Oracle residual at sampled nodes of meshes too large for the assembled oracle.

Test infrastructure only. The residual of Eq. PoissonWeakForm at a node is a
sum over the (at most 8) elements that contain it, so it can be evaluated
element by element from the oracle's own building blocks (oracle.fem for the
Gauss quadrature, oracle.physics for the charge and the contact values)
without assembling the whole mesh. The node and element numbering, the
coordinates and the Dirichlet sets follow oracle.mesh.Mesh; test_sampled_oracle
checks on small meshes that this evaluation reproduces PoissonProblem.residual
exactly.
"""
from __future__ import annotations

import numpy as np

from oracle import fem, physics
from oracle.poisson import semiconductor_material


class SampledPoisson:
    def __init__(self, dev: dict, fixed_charge=None):
        self.dev = dev
        self.bias = dict(dev["bias"])
        self.nx, self.ny = dev["nx"], dev["ny"]
        self.nz = sum(L["n"] for L in dev["layers"])
        self.nxn, self.nyn, self.nzn = self.nx + 1, self.ny + 1, self.nz + 1
        self.x = np.linspace(0.0, dev["Lx"], self.nx + 1)
        self.y = np.linspace(0.0, dev["Ly"], self.ny + 1)
        zs, mats = [0.0], []
        for L in dev["layers"]:
            h = L["thickness"] / L["n"]
            z0 = zs[-1]
            for m in range(L["n"]):
                zs.append(z0 + (m + 1) * h)
                mats.append(L["material"])
        self.z = np.array(zs)
        self.layer_mat = np.array(mats, dtype=np.int64)
        self.T = self.bias["T"]
        self.si = semiconductor_material(dev)
        self.phi_r = physics.phi_ref(self.si, self.T)
        self.E_F = -self.bias.get("V_sub", 0.0)
        self.qe = physics.q_over_eps0()
        self.theta = None if fixed_charge is None else np.asarray(fixed_charge, dtype=np.float64)

    def node(self, i, j, k):
        return i + self.nxn * (j + self.nyn * k)

    def is_dirichlet(self, i, j, k):
        i, j, k = np.asarray(i), np.asarray(j), np.asarray(k)
        d = np.zeros(i.shape, dtype=bool)
        if self.dev.get("bottom_ohmic", 1):
            d |= k == 0
        top = k == self.nz
        xs, ys = self.x[i], self.y[j]
        for G in self.dev.get("gates", []):
            d |= top & (xs >= G["x0"]) & (xs <= G["x1"]) & (ys >= G["y0"]) & (ys <= G["y1"])
        return d

    def residual_at(self, phi, ijk):
        """R at the nodes ijk (n x 3 integer array), free or not (full rows, as residual(full=True))."""
        ijk = np.asarray(ijk, dtype=np.int64)
        nodes = self.node(ijk[:, 0], ijk[:, 1], ijk[:, 2])
        elems = set()
        for i, j, k in ijk:
            for di in (-1, 0):
                for dj in (-1, 0):
                    for dk in (-1, 0):
                        ei, ej, ek = i + di, j + dj, k + dk
                        if 0 <= ei < self.nx and 0 <= ej < self.ny and 0 <= ek < self.nz:
                            elems.add((ei, ej, ek))
        E = np.array(sorted(elems), dtype=np.int64)
        conn = np.empty((len(E), 8), dtype=np.int64)
        coords = np.empty((len(E), 8, 3))
        for a in range(8):
            ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
            conn[:, a] = self.node(E[:, 0] + ax, E[:, 1] + ay, E[:, 2] + az)
            coords[:, a, 0] = self.x[E[:, 0] + ax]
            coords[:, a, 1] = self.y[E[:, 1] + ay]
            coords[:, a, 2] = self.z[E[:, 2] + az]
        emat = self.layer_mat[E[:, 2]]
        wdet, grad = fem.geometry(coords)
        eps = np.array([self.dev["materials"][m]["eps_r"] for m in emat])
        Ke = fem.element_stiffness(wdet, grad, np.repeat(eps[:, None], 3, axis=1))
        phq = fem.interpolate(phi, conn)
        rho = np.zeros_like(phq)
        for mi, mat in enumerate(self.dev["materials"]):
            sel = emat == mi
            if not np.any(sel) or not mat["semiconductor"]:
                continue
            t = physics.carrier_terms(phq[sel], mat, self.T, self.phi_r, self.E_F, self.bias.get("statistics", 1),
                                      self.bias.get("incomplete_ionization", 1))
            rho[sel] = t["rho"]
        if self.theta is not None:
            rho = rho + self.theta[E[:, 0] + self.nx * (E[:, 1] + self.ny * E[:, 2])][:, None]
        Re = np.einsum("eab,eb->ea", Ke, phi[conn]) - self.qe * fem.element_load(wdet, rho)
        order = np.argsort(nodes)
        sn = nodes[order]
        R = np.zeros(len(nodes))
        pos = np.searchsorted(sn, conn.ravel())
        pos = np.minimum(pos, len(sn) - 1)
        hit = sn[pos] == conn.ravel()
        np.add.at(R, order[pos[hit]], Re.ravel()[hit])
        return R

    def sample_nodes(self, count, seed, free_only=True):
        """Random nodes plus the nodes of the dot regions' corners and the gate edges."""
        rng = np.random.default_rng(seed)
        pts = [np.stack([rng.integers(0, self.nxn, count), rng.integers(0, self.nyn, count),
                         rng.integers(0, self.nzn, count)], axis=1)]
        # a vertical line through the device centre (oxide, interface, dots, bottom)
        kk = np.arange(self.nzn)
        pts.append(np.stack([np.full_like(kk, self.nxn // 2), np.full_like(kk, self.nyn // 2), kk], axis=1))
        ijk = np.unique(np.concatenate(pts), axis=0)
        if free_only:
            ijk = ijk[~self.is_dirichlet(ijk[:, 0], ijk[:, 1], ijk[:, 2])]
        return ijk
