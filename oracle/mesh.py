"""Tensor-product hexahedral mesh built from a device description (oracle).

Test infrastructure only. The paper meshes CAD geometry with Cubit into
material blocks (Sec. I, Sec. III); the synthetic devices used here are
layered boxes, so the mesh is a structured Q1 hex grid with per-axis node
planes: uniform spacing in x and y, uniform spacing within each z layer
group. Node index n = i + (nx+1)*(j + (ny+1)*k); element index
e = i + nx*(j + ny*k); element corner a = ax + 2*ay + 4*az.
"""
from __future__ import annotations

import numpy as np


class Mesh:
    def __init__(self, dev: dict):
        self.dev = dev
        self.nx, self.ny = dev["nx"], dev["ny"]
        self.nz = sum(L["n"] for L in dev["layers"])
        self.x = np.linspace(0.0, dev["Lx"], self.nx + 1)
        self.y = np.linspace(0.0, dev["Ly"], self.ny + 1)
        zs = [0.0]
        layer_mat = []
        for L in dev["layers"]:
            h = L["thickness"] / L["n"]
            z0 = zs[-1]
            for m in range(L["n"]):
                zs.append(z0 + (m + 1) * h)
                layer_mat.append(L["material"])
        self.z = np.array(zs)
        self.layer_mat = np.array(layer_mat, dtype=np.int64)  # per element layer
        self.materials = dev["materials"]
        self.nxn, self.nyn, self.nzn = self.nx + 1, self.ny + 1, self.nz + 1
        self.n_nodes = self.nxn * self.nyn * self.nzn
        self.n_elems = self.nx * self.ny * self.nz

        # element -> 8 corner nodes
        ei, ej, ek = np.meshgrid(np.arange(self.nx), np.arange(self.ny), np.arange(self.nz), indexing="ij")
        ei, ej, ek = ei.transpose(2, 1, 0).ravel(), ej.transpose(2, 1, 0).ravel(), ek.transpose(2, 1, 0).ravel()
        self.ei, self.ej, self.ek = ei, ej, ek
        conn = np.empty((self.n_elems, 8), dtype=np.int64)
        for a in range(8):
            ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
            conn[:, a] = self.node_id(ei + ax, ej + ay, ek + az)
        self.conn = conn
        # node coordinates
        ni, nj, nk = np.meshgrid(np.arange(self.nxn), np.arange(self.nyn), np.arange(self.nzn), indexing="ij")
        ni, nj, nk = ni.transpose(2, 1, 0).ravel(), nj.transpose(2, 1, 0).ravel(), nk.transpose(2, 1, 0).ravel()
        self.ni, self.nj, self.nk = ni, nj, nk
        self.coords = np.stack([self.x[ni], self.y[nj], self.z[nk]], axis=1)
        self.elem_mat = self.layer_mat[ek]
        self.elem_coords = self.coords[conn]  # (Ne, 8, 3)

    def node_id(self, i, j, k):
        return i + self.nxn * (j + self.nyn * k)

    def elem_id(self, i, j, k):
        return i + self.nx * (j + self.ny * k)

    # ---------------- contacts (Sec. II.A.4) ----------------
    def gate_of_node(self):
        """Gate index of each node (-1 if none): top-face nodes inside a gate's closed rectangle."""
        g = np.full(self.n_nodes, -1, dtype=np.int64)
        top = self.nk == self.nz
        for gi, G in enumerate(self.dev["gates"]):
            inside = top & (self.coords[:, 0] >= G["x0"]) & (self.coords[:, 0] <= G["x1"]) \
                & (self.coords[:, 1] >= G["y0"]) & (self.coords[:, 1] <= G["y1"])
            g[inside & (g < 0)] = gi
        return g

    def ohmic_nodes(self):
        """Bottom face z = 0 is the Ohmic back contact when bottom_ohmic is set."""
        if self.dev.get("bottom_ohmic", 1):
            return self.nk == 0
        return np.zeros(self.n_nodes, dtype=bool)

    def dirichlet_mask(self):
        return (self.gate_of_node() >= 0) | self.ohmic_nodes()

    # ---------------- regions ----------------
    def dot_elements(self, d):
        """Semiconductor elements whose centroid lies in dot box d (the dot's quantum region)."""
        D = self.dev["dots"][d]
        cen = self.elem_coords.mean(axis=1)
        semi = np.array([self.materials[m]["semiconductor"] for m in self.elem_mat], dtype=bool)
        return semi & (cen[:, 0] >= D["x0"]) & (cen[:, 0] <= D["x1"]) & (cen[:, 1] >= D["y0"]) \
            & (cen[:, 1] <= D["y1"]) & (cen[:, 2] >= D["z0"]) & (cen[:, 2] <= D["z1"])

    def subdomain_elements(self):
        S = self.dev["subdomain"]
        return (self.ei >= S["i0"]) & (self.ei < S["i1"]) & (self.ej >= S["j0"]) & (self.ej < S["j1"]) \
            & (self.ek >= S["k0"]) & (self.ek < S["k1"])

    def subdomain_interior_nodes(self):
        """Nodes strictly inside the Schrodinger subdomain box (psi = 0 on its boundary, Sec. II.B)."""
        S = self.dev["subdomain"]
        return (self.ni > S["i0"]) & (self.ni < S["i1"]) & (self.nj > S["j0"]) & (self.nj < S["j1"]) \
            & (self.nk > S["k0"]) & (self.nk < S["k1"])
