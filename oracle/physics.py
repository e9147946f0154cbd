"""Semiclassical carrier statistics and contact potentials (oracle, FP64).

Test infrastructure only (see ``oracle/__init__``). Units: potential V,
energy eV, length nm, density nm^-3. With energies in eV, q*phi in eV is
numerically phi in V.

Every function cites the passage of Gao et al. (arXiv:1403.7561) it follows.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, optimize

# CODATA 2018 values (SI). q and k_B are exact by definition.
Q_E = 1.602176634e-19        # C
K_B = 1.380649e-23           # J/K
HBAR = 1.054571817e-34       # J s
M0 = 9.1093837015e-31        # kg
EPS0 = 8.8541878128e-12      # F/m


def kT_eV(T):
    """Thermal energy k_B T in eV."""
    return K_B * T / Q_E


def q_over_eps0():
    """q/eps0 in V*nm (the residual is scaled by 1/eps0)."""
    return Q_E / EPS0 * 1e9


def hbar2_over_2m0():
    """hbar^2 / (2 m0) in eV*nm^2."""
    return HBAR * HBAR / (2.0 * M0) / Q_E * 1e18


# ---------------------------------------------------------------------------
# Sec. II.A.1, Eqs. EffectiveMass and EffectiveDOS
# ---------------------------------------------------------------------------
def dos_masses(mat):
    """Electron and hole DOS effective masses (units m0), Eq. EffectiveMass.

    m_n* = 6^(2/3) (m_l m_t^2)^(1/3) (six equivalent conduction minima);
    m_p* = (m_hh^(3/2) + m_lh^(3/2))^(2/3).
    """
    mn = 6.0 ** (2.0 / 3.0) * (mat["m_l"] * mat["m_t"] ** 2) ** (1.0 / 3.0)
    mp = (mat["m_hh"] ** 1.5 + mat["m_lh"] ** 1.5) ** (2.0 / 3.0)
    return mn, mp


def effective_dos(m_rel, T):
    """N = 2 (m* k_B T / (2 pi hbar^2))^(3/2) in nm^-3, Eq. EffectiveDOS."""
    a = m_rel * M0 * K_B * T / (2.0 * math.pi * HBAR * HBAR) * 1e-18  # nm^-2
    return 2.0 * a ** 1.5


def band_params(mat, T):
    """(N_C, N_V) of a semiconductor material at temperature T."""
    mn, mp = dos_masses(mat)
    return effective_dos(mn, T), effective_dos(mp, T)


# ---------------------------------------------------------------------------
# Sec. II.A.1, Eqs. FDIntegral and FDIntApprox
# ---------------------------------------------------------------------------
def fd_half_integral(x):
    """F_1/2(x) = (2/sqrt(pi)) int_0^inf sqrt(e) / (1 + exp(e - x)) de, Eq. FDIntegral.

    Adaptive quadrature; used only to pin the approximation below.
    """
    def f(e):
        # 1/(1+exp(e-x)) written without overflow
        t = e - x
        if t > 0:
            w = math.exp(-t) / (1.0 + math.exp(-t))
        else:
            w = 1.0 / (1.0 + math.exp(t))
        return math.sqrt(e) * w
    pts = [max(x, 0.0)] if x > 0 else None
    upper = max(x, 0.0) + 60.0
    val, _ = integrate.quad(f, 0.0, upper, points=pts, limit=400, epsabs=0.0, epsrel=1e-13)
    return 2.0 / math.sqrt(math.pi) * val


def fd_mhalf_integral(x):
    """F_-1/2(x) = (1/sqrt(pi)) int_0^inf e^-1/2 / (1 + exp(e - x)) de = dF_1/2/dx.

    Substitution e = s^2 removes the endpoint singularity.
    """
    def f(s):
        t = s * s - x
        if t > 0:
            w = math.exp(-t) / (1.0 + math.exp(-t))
        else:
            w = 1.0 / (1.0 + math.exp(t))
        return 2.0 * w
    upper = math.sqrt(max(x, 0.0) + 60.0)
    pts = [math.sqrt(x)] if x > 0 else None
    val, _ = integrate.quad(f, 0.0, upper, points=pts, limit=400, epsabs=0.0, epsrel=1e-13)
    return val / math.sqrt(math.pi)


FD_CLAMP_X = -50.0
_C_BED = 3.0 * math.sqrt(math.pi) / 4.0


def fd_half(x):
    """Bednarczyk approximation of F_1/2, Eq. FDIntApprox, with the x < -50 clamp.

    F(x) ~ ( e^-x + (3 sqrt(pi)/4) v^(-3/8) )^-1,
    v = x^4 + 50 + 33.6 x [1 - 0.68 exp(-0.17 (x+1)^2)]   (the printed formula
    leaves a bracket open; this closing reproduces its stated 0.4 % accuracy), and F(x) = e^x for x < -50 (Sec. II.A.1, last paragraph).
    Accepts scalars or numpy arrays.
    """
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    lo = x < FD_CLAMP_X
    out[lo] = np.exp(x[lo])
    xh = x[~lo]
    g = np.exp(-0.17 * (xh + 1.0) ** 2)
    v = xh ** 4 + 50.0 + 33.6 * xh * (1.0 - 0.68 * g)
    out[~lo] = 1.0 / (np.exp(-xh) + _C_BED * v ** (-0.375))
    return out if out.ndim else float(out)


def fd_half_deriv(x):
    """dF/dx of the implemented approximation (the Jacobian differentiates what the residual uses).

    With D = e^-x + C v^(-3/8):  F = 1/D,  F' = (e^-x + (3/8) C v^(-11/8) v') / D^2,
    v' = 4x^3 + 33.6 (1 - 0.68 g) + 33.6 x * 0.68 * 0.34 (x+1) g,  g = exp(-0.17 (x+1)^2).
    For x < -50 the clamp gives F' = e^x.
    """
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    lo = x < FD_CLAMP_X
    out[lo] = np.exp(x[lo])
    xh = x[~lo]
    g = np.exp(-0.17 * (xh + 1.0) ** 2)
    v = xh ** 4 + 50.0 + 33.6 * xh * (1.0 - 0.68 * g)
    dv = 4.0 * xh ** 3 + 33.6 * (1.0 - 0.68 * g) + 33.6 * xh * 0.68 * 0.34 * (xh + 1.0) * g
    D = np.exp(-xh) + _C_BED * v ** (-0.375)
    dD = -np.exp(-xh) - 0.375 * _C_BED * v ** (-1.375) * dv
    out[~lo] = -dD / (D * D)
    return out if out.ndim else float(out)


# ---------------------------------------------------------------------------
# Sec. II.A.4, Eq. FDintInverse (Nilsson)
# ---------------------------------------------------------------------------
def fd_half_inverse(u):
    """eta with F_1/2(eta) = u, Nilsson's approximation, Eq. FDintInverse.

    eta = -ln(u)/(u^2 - 1) + nu / (1 + (0.24 + 1.08 nu)^-2),
    nu = (3 sqrt(pi) u / 4)^(2/3).  At u = 1 the first term takes its limit -1/2.
    """
    u = float(u)
    if abs(u - 1.0) < 1e-12:
        first = -0.5
    else:
        first = -math.log(u) / (u * u - 1.0)
    nu = (3.0 * math.sqrt(math.pi) * u / 4.0) ** (2.0 / 3.0)
    return first + nu / (1.0 + (0.24 + 1.08 * nu) ** -2)


# ---------------------------------------------------------------------------
# Sec. II.A.2, Eqs. qPhiRef and EcEv_phi
# ---------------------------------------------------------------------------
def phi_ref(mat, T):
    """Reference potential q phi_ref = E_0 - E_i(Si), Eq. qPhiRef.

    E_i = (E_C + E_V)/2 + (kT/2) ln(N_V/N_C), so
    q phi_ref = chi + E_g/2 + (kT/2) ln(N_C/N_V).
    """
    NC, NV = band_params(mat, T)
    return mat["chi"] + 0.5 * mat["Eg"] + 0.5 * kT_eV(T) * math.log(NC / NV)


def band_edges(phi, mat, phi_r):
    """E_C = -q(phi - phi_ref) - chi, E_V = E_C - E_g, Eq. EcEv_phi (eV)."""
    Ec = -(np.asarray(phi) - phi_r) - mat["chi"]
    return Ec, Ec - mat["Eg"]


# ---------------------------------------------------------------------------
# Densities: Eqs. MBstatistics, FDstatistics, FinalIonization
# ---------------------------------------------------------------------------
def _sigmoid_pair(zeta, g):
    """s = 1/(1 + g e^zeta) and 1 - s, overflow-safe."""
    zeta = np.asarray(zeta, dtype=np.float64)
    s = np.empty_like(zeta)
    one_m_s = np.empty_like(zeta)
    pos = zeta > 0
    ez = np.exp(-zeta[pos])
    s[pos] = ez / (ez + g)
    one_m_s[pos] = g / (ez + g)
    ez = np.exp(zeta[~pos])
    s[~pos] = 1.0 / (1.0 + g * ez)
    one_m_s[~pos] = g * ez / (1.0 + g * ez)
    return s, one_m_s


def carrier_terms(phi, mat, T, phi_r, E_F=0.0, statistics=1, incomplete=1):
    """Charge density terms and their phi-derivatives at potential phi.

    Returns dict with n, p, ND+, NA- (nm^-3), rho = p - n + ND+ - NA-, and
    drho = d rho / d phi (nm^-3 / V).

    n = N_C F(eta_n), eta_n = (E_F - E_C)/kT; p = N_V F(eta_p), eta_p = (E_V - E_F)/kT
    with F = exp (MB, Eq. MBstatistics) or the Bednarczyk F_1/2 (FD, Eq. FDstatistics).
    Ionized dopants by Eq. FinalIonization (g_D, g_A of Sec. II.A.3); complete
    ionization sets ND+ = N_D and NA- = N_A. Insulators carry no charge.
    """
    phi = np.asarray(phi, dtype=np.float64)
    zero = np.zeros_like(phi)
    if not mat["semiconductor"]:
        return dict(n=zero, p=zero, ND=zero, NA=zero, rho=zero, drho=zero,
                    dn=zero, dp=zero, dND=zero, dNA=zero)
    kT = kT_eV(T)
    NC, NV = band_params(mat, T)
    Ec, Ev = band_edges(phi, mat, phi_r)
    eta_n = (E_F - Ec) / kT
    eta_p = (Ev - E_F) / kT
    if statistics == 1:
        n = NC * fd_half(eta_n)
        p = NV * fd_half(eta_p)
        dn = NC * fd_half_deriv(eta_n) / kT          # d eta_n / d phi = +1/kT
        dp = -NV * fd_half_deriv(eta_p) / kT         # d eta_p / d phi = -1/kT
    else:
        n = NC * np.exp(eta_n)
        p = NV * np.exp(eta_p)
        dn = n / kT
        dp = -p / kT
    ND, NA = mat["N_D"], mat["N_A"]
    if incomplete:
        # N_D+ = N_D / (1 + g_D exp((E_F + E_d - q phi_ref + chi + q phi)/kT))
        zD = (E_F + mat["E_d"] - phi_r + mat["chi"] + phi) / kT
        sD, omsD = _sigmoid_pair(zD, mat["g_D"])
        NDp = ND * sD
        dNDp = -ND * sD * omsD / kT
        # N_A- = N_A / (1 + g_A exp((-E_F + E_a + q phi_ref - chi - E_g - q phi)/kT))
        zA = (-E_F + mat["E_a"] + phi_r - mat["chi"] - mat["Eg"] - phi) / kT
        sA, omsA = _sigmoid_pair(zA, mat["g_A"])
        NAm = NA * sA
        dNAm = NA * sA * omsA / kT
    else:
        NDp = np.full_like(phi, ND)
        NAm = np.full_like(phi, NA)
        dNDp = zero
        dNAm = zero
    rho = p - n + NDp - NAm
    drho = dp - dn + dNDp - dNAm
    return dict(n=n, p=p, ND=NDp, NA=NAm, rho=rho, drho=drho, dn=dn, dp=dp, dND=dNDp, dNA=dNAm)


# ---------------------------------------------------------------------------
# Contacts, Sec. II.A.4
# ---------------------------------------------------------------------------
def gate_potential(V_g, phi_r, work_function=None):
    """phi_ins = V_g - (Phi_m - q phi_ref)/q, Eq. ContOnIns. Phi_m defaults to q phi_ref (the paper gives none)."""
    Phi_m = phi_r if work_function is None else work_function
    return V_g - (Phi_m - phi_r)


LOW_T_LOG_APPROX_K = 50.0


def ohmic_potential(mat, T, phi_r, V_a=0.0, statistics=1, incomplete=1):
    """Ohmic-contact Dirichlet value from thermal equilibrium and charge neutrality.

    - MB, complete ionization: Eq. PotBC4MBCompIon.
    - MB, incomplete: Eq. PotBC4MBIncompIon with y_n, y_p of Eq. Yval4MBIncompIon,
      or their logarithms by Eq. ApproxLogTerms when T < 50 K (the paper's
      "very low temperatures", taken as below 50 K).
      For p-type the sign of E_a follows the derivation from y_p's definition,
      +E_a (the printed -E_a contradicts Eq. Yval4MBIncompIon; pinned by the
      neutral-root test).
    - FD, complete: Eq. PotBC4FDCompIon with Nilsson's inverse, Eq. FDintInverse.
    - FD, incomplete: the MB-incomplete value (the paper's stated approximation).
    The contact is n-type when N_D > N_A, p-type otherwise.
    """
    kT = kT_eV(T)
    NC, NV = band_params(mat, T)
    chi, Eg = mat["chi"], mat["Eg"]
    ntype = mat["N_D"] > mat["N_A"]
    if mat["N_D"] == 0.0 and mat["N_A"] == 0.0:
        return 0.0 + V_a  # undoped: intrinsic level (phi = 0 puts E_i at E_F)
    if incomplete:
        if ntype:
            if T < LOW_T_LOG_APPROX_K:
                ln_y = 0.5 * math.log(mat["N_D"] / (2.0 * NC)) + mat["E_d"] / (2.0 * kT)
            else:
                y = -0.25 + 0.25 * math.sqrt(1.0 + 8.0 * mat["N_D"] / NC * math.exp(mat["E_d"] / kT))
                ln_y = math.log(y)
            return (-mat["E_d"] + phi_r - chi) + kT * ln_y + V_a
        if T < LOW_T_LOG_APPROX_K:
            ln_y = 0.5 * math.log(mat["N_A"] / (4.0 * NV)) + mat["E_a"] / (2.0 * kT)
        else:
            y = -0.125 + 0.125 * math.sqrt(1.0 + 16.0 * mat["N_A"] / NV * math.exp(mat["E_a"] / kT))
            ln_y = math.log(y)
        return (mat["E_a"] + phi_r - chi - Eg) - kT * ln_y + V_a
    if statistics == 0:
        if ntype:
            return (phi_r - chi) + kT * math.log(mat["N_D"] / NC) + V_a
        return (phi_r - chi - Eg) - kT * math.log(mat["N_A"] / NV) + V_a
    if ntype:
        eta = fd_half_inverse(mat["N_D"] / NC)
        return (phi_r - chi) + kT * eta + V_a
    eta = fd_half_inverse(mat["N_A"] / NV)
    return (phi_r - chi - Eg) - kT * eta + V_a


def neutral_root(mat, T, phi_r, E_F=0.0, statistics=1, incomplete=1, lo=-3.0, hi=3.0):
    """phi where rho(phi) = p - n + ND+ - NA- = 0, by bracketing (used to pin contacts)."""
    def f(phi):
        t = carrier_terms(np.array([phi]), mat, T, phi_r, E_F, statistics, incomplete)
        return float(t["rho"][0])
    return optimize.brentq(f, lo, hi, xtol=1e-15, rtol=4 * np.finfo(float).eps, maxiter=500)
