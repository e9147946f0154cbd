"""Seeded synthetic device descriptions shared by the oracle and the CUDA path.

This module holds geometry parameters, material constants and random draws
only. It performs none of the method's arithmetic (no mesh coordinates, no
carrier statistics, no contact potentials): both the oracle and the CUDA
library derive everything else from the plain dictionaries returned here.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), written from its published
definition: uniforms are (x >> 11) * 2**-53, normals use the Box-Muller
transform.

Device shapes follow the five-gate Si/SiO2 stacks of the paper's application
sections (Sec. III, Fig. 7 dot region; Sec. IV, Fig. 12 gate fingers): the
paper's SEM-derived CAD geometries are not available, so rectangular
top-face gate patches over a SiO2 layer on a p-type Si body stand in for them.
"""
from __future__ import annotations

import copy
import math

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator (64-bit state, golden-gamma increment)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) with 53 random bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_range(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.uniform()

    def normal(self) -> float:
        """Standard normal by Box-Muller (one value per two uniforms)."""
        u1 = 1.0 - self.uniform()  # (0, 1]
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


def stream_seed(seed: int, stream: int) -> int:
    """Seed of independent stream `stream` derived from base `seed`."""
    return ((seed & 0xFFFFFFFF) << 32) | (stream & 0xFFFFFFFF)


# ---------------------------------------------------------------------------
# Materials (the paper gives the formulas but not these values).
# Units: eps relative; chi, Eg, E_a, E_d in eV; masses in m0; doping in nm^-3.
# ---------------------------------------------------------------------------
SI = dict(name="Si", eps_r=11.7, chi=4.05, Eg=1.12, semiconductor=1,
          m_l=0.98, m_t=0.19, m_hh=0.49, m_lh=0.16,
          N_A=1e-6, N_D=0.0, E_a=0.044, E_d=0.046, g_A=4.0, g_D=2.0)
SIO2 = dict(name="SiO2", eps_r=3.9, chi=0.95, Eg=9.0, semiconductor=0,
            m_l=0.5, m_t=0.5, m_hh=0.5, m_lh=0.5,
            N_A=0.0, N_D=0.0, E_a=0.0, E_d=0.0, g_A=4.0, g_D=2.0)

# Five gate fingers on the top face (x extents on a 200 nm device), all spanning
# y in [30, 170] nm, separated by 5 nm gaps: barrier B1, plunger P1, barrier B2,
# plunger P2, barrier B3 (layout reading; the paper's layouts are SEM-derived).
FIVE_GATES_X = [(25.0, 45.0), (50.0, 90.0), (95.0, 105.0), (110.0, 150.0), (155.0, 175.0)]
GATES_Y = (30.0, 170.0)
GATE_NAMES = ["B1", "P1", "B2", "P2", "B3"]
# Dot d: Si elements whose centroid lies under plunger P_d, y in [70, 130],
# within 15 nm of the Si/SiO2 interface.
DOT_X = [(50.0, 90.0), (110.0, 150.0)]
DOT_Y = (70.0, 130.0)


def _stack_layers(nz: int, t_si: float, t_ox: float, n_ox: int | None = None):
    """Layer groups bottom->top: Si body then SiO2; oxide element count rounds nz*t_ox/L_z."""
    if n_ox is None:
        n_ox = int(round(nz * t_ox / (t_si + t_ox)))
        n_ox = max(1, n_ox)
    return [dict(material=0, thickness=t_si, n=nz - n_ox),
            dict(material=1, thickness=t_ox, n=n_ox)]


def mos_capacitor(nx=16, ny=16, nz=32, L=100.0, t_si=50.0, t_ox=10.0, n_ox=5,
                  V_gate=0.5, T=300.0, statistics=1, incomplete_ionization=1,
                  N_A=1e-6, N_D=0.0):
    """3D MOS capacitor: whole top face is one gate, grounded Ohmic back contact."""
    si = dict(SI, N_A=N_A, N_D=N_D)
    return dict(
        name="mos_capacitor",
        Lx=L, Ly=L, nx=nx, ny=ny,
        layers=_stack_layers(nz, t_si, t_ox, n_ox),
        materials=[si, dict(SIO2)],
        gates=[dict(name="G", x0=0.0, x1=L, y0=0.0, y1=L)],
        # metal gate with Phi_m = q phi_ref, so the gate Dirichlet value is V_gate itself
        gate_work_function=None,
        bottom_ohmic=1,
        dots=[],
        subdomain=None,
        bias=dict(T=T, V_gate=[V_gate], V_sub=0.0, statistics=statistics,
                  incomplete_ionization=incomplete_ionization),
    )


def five_gate_device(n=(128, 128, 96), seed=2, T=4.0, L=200.0, t_si=90.0, t_ox=10.0,
                     v_range=(-0.5, 1.0), with_subdomain=True,
                     statistics=1, incomplete_ionization=1, stream=None):
    """Five-gate double-dot Si/SiO2 stack over L x L x (t_si + t_ox) nm.

    Gate voltages are drawn uniform in v_range from SplitMix64(seed) (or from
    stream `stream` of `seed`). The Schrodinger subdomain is the central half
    of the x-y extent times the Si element layers within t_si*32/86 nm of the
    interface (64 x 64 x 32 elements on the 128 x 128 x 96 mesh).
    """
    nx, ny, nz = n
    layers = _stack_layers(nz, t_si, t_ox)
    n_si = layers[0]["n"]
    rng = SplitMix64(seed if stream is None else stream_seed(seed, stream))
    V = [rng.uniform_range(v_range[0], v_range[1]) for _ in range(5)]
    gates = [dict(name=GATE_NAMES[g], x0=FIVE_GATES_X[g][0] * L / 200.0,
                  x1=FIVE_GATES_X[g][1] * L / 200.0,
                  y0=GATES_Y[0] * L / 200.0, y1=GATES_Y[1] * L / 200.0) for g in range(5)]
    zi = t_si
    dots = [dict(x0=DOT_X[d][0] * L / 200.0, x1=DOT_X[d][1] * L / 200.0,
                 y0=DOT_Y[0] * L / 200.0, y1=DOT_Y[1] * L / 200.0, z0=zi - 15.0, z1=zi)
            for d in range(2)]
    sub = None
    if with_subdomain:
        i0, i1 = nx // 4, 3 * nx // 4
        j0, j1 = ny // 4, 3 * ny // 4
        kz = int(round(n_si * 32.0 / 86.0))
        sub = dict(i0=i0, i1=i1, j0=j0, j1=j1, k0=n_si - kz, k1=n_si)
    return dict(
        name="five_gate_%dx%dx%d" % (nx, ny, nz),
        Lx=L, Ly=L, nx=nx, ny=ny,
        layers=layers,
        materials=[dict(SI), dict(SIO2)],
        gates=gates,
        bottom_ohmic=1,
        dots=dots,
        subdomain=sub,
        # Depletion gates of degenerately As-doped polysilicon (Sec. III): work
        # function at the Si conduction band edge, Phi_m = chi_Si (eV).
        gate_work_function=SI["chi"],
        bias=dict(T=T, V_gate=V, V_sub=0.0, statistics=statistics,
                  incomplete_ionization=incomplete_ionization),
    )


def interface_fixed_charge(dev: dict, seed: int, sigma_std=1e-4):
    """Per-element fixed charge theta (nm^-3), length n_elems, x fastest.

    sigma_e ~ N(0, sigma_std nm^-2) on the single layer of Si elements that
    touches the Si/SiO2 interface, theta_e = sigma_e / h_z of that layer;
    zero elsewhere. Element order: i + nx*(j + ny*k).
    """
    nx, ny = dev["nx"], dev["ny"]
    nz = sum(L["n"] for L in dev["layers"])
    k_if = dev["layers"][0]["n"] - 1
    hz = dev["layers"][0]["thickness"] / dev["layers"][0]["n"]
    rng = SplitMix64(seed)
    theta = [0.0] * (nx * ny * nz)
    base = nx * ny * k_if
    for e in range(nx * ny):
        theta[base + e] = rng.normal() * sigma_std / hz
    return theta


def interface_sheet_pattern(dev: dict):
    """Per-element fixed charge (nm^-3) of a uniform interface sheet of 1 nm^-2: 1/h_z on the Si
    element layer touching the Si/SiO2 interface, 0 elsewhere (the layer of
    interface_fixed_charge). Element order: i + nx*(j + ny*k)."""
    nx, ny = dev["nx"], dev["ny"]
    nz = sum(L["n"] for L in dev["layers"])
    k_if = dev["layers"][0]["n"] - 1
    hz = dev["layers"][0]["thickness"] / dev["layers"][0]["n"]
    pat = [0.0] * (nx * ny * nz)
    for e in range(nx * ny):
        pat[nx * ny * k_if + e] = 1.0 / hz
    return pat


def batch_instances(count=96, seed=4, sizes=tuple(range(48, 113, 8)), T=4.0):
    """Batched form: `count` five-gate instances with N^3 elements, N drawn from `sizes`."""
    rng = SplitMix64(seed)
    out = []
    for i in range(count):
        N = sizes[int(rng.uniform() * len(sizes)) % len(sizes)]
        dev = five_gate_device(n=(N, N, N), seed=seed, stream=i, T=T, with_subdomain=False)
        dev["name"] = "batch_%02d_N%d" % (i, N)
        out.append(dev)
    return out


CONFIGS = {
    # Plain FP64 nonlinear Poisson, 3D MOS capacitor (16x16x32 over 100x100x60 nm, 300 K).
    "mos_cap_16x16x32": lambda: mos_capacitor(),
    # Plain FP64 double quantum dot at 4 K on 128x128x96 (~1.6M nodes) + Schrodinger block.
    "dqd_128x128x96_4K": lambda: five_gate_device(n=(128, 128, 96), seed=2, T=4.0),
    # Precision form: the same device (same gate voltages) on 256x256x128 (~8.5M nodes) at 0.5 K.
    "dqd_256x256x128_0p5K": lambda: five_gate_device(n=(256, 256, 128), seed=2, T=0.5),
    # Differentiation form: the same 128x128x96 device at 4 K; the fixed-charge
    # field is drawn by interface_fixed_charge(dev, seed=5).
    "dqd_128x128x96_4K_adjoint": lambda: five_gate_device(n=(128, 128, 96), seed=2, T=4.0),
}


def get(name: str) -> dict:
    return copy.deepcopy(CONFIGS[name]())


def n_elems(dev: dict) -> int:
    return dev["nx"] * dev["ny"] * sum(L["n"] for L in dev["layers"])


def n_nodes(dev: dict) -> int:
    return (dev["nx"] + 1) * (dev["ny"] + 1) * (sum(L["n"] for L in dev["layers"]) + 1)
