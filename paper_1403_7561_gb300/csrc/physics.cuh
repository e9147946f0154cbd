// Semiclassical charge density at a quadrature point (FP64), Sec. II.A.
//
// n = N_C F(eta_n), p = N_V F(eta_p) with eta_n = (E_F - E_C)/kT,
// eta_p = (E_V - E_F)/kT, E_C = -q(phi - phi_ref) - chi, E_V = E_C - E_g
// (Eqs. EcEv_phi, MBstatistics, FDstatistics); F is exp (MB) or the
// Bednarczyk approximation of F_1/2 (Eq. FDIntApprox) with the paper's
// replacement F(x) = e^x for x < -50. Ionized dopants follow Eq.
// FinalIonization. Derivatives are those of the implemented expressions, so
// the Jacobian is exact for the residual the solver uses.
//
// FP64 division is a long instruction sequence on this GPU (FP64 runs at
// 1/57 of the FP32 rate), so 1/kT is applied as a multiplication and each
// logistic factor takes one reciprocal.
#pragma once
#include "qcad_internal.cuh"

namespace qcad {

// F_1/2 and its derivative. Below x = xmin, F = e^x is taken as zero (xmin: -150, where
// N_C F < 1e-60 nm^-3, for the dot counts; the residual's cutoff otherwise, see RHO_RESID_FLOOR
// in qcad_internal.cuh).
__device__ __forceinline__ void fd_half_d(double x, double& F, double& dF, double xmin = -150.0) {
  if (x < xmin) {
    F = 0.0;
    dF = 0.0;
    return;
  }
  if (x < -50.0) {
    F = exp(x);
    dF = F;
    return;
  }
  const double xp1 = x + 1.0;
  const double g = exp(-0.17 * xp1 * xp1);
  const double x2 = x * x;
  const double v = x2 * x2 + 50.0 + 33.6 * x * (1.0 - 0.68 * g);
  const double dv = 4.0 * x2 * x + 33.6 * (1.0 - 0.68 * g) + 33.6 * 0.68 * 0.34 * x * xp1 * g;
  const double emx = exp(-x);
  const double C = 1.32934038817913702047;  // 3 sqrt(pi) / 4
  const double vp = pow(v, -0.375);
  const double D = emx + C * vp;
  F = 1.0 / D;
  const double dD = -emx - 0.375 * C * vp / v * dv;
  dF = -dD * F * F;
}

// s = 1/(1 + g e^z) and 1 - s without overflow. Beyond z = zmax, e^{-z} is taken as zero (746:
// below half the smallest subnormal; the residual's cutoff otherwise, see RHO_RESID_FLOOR); below
// z = -45 the call and the reciprocal are skipped (s = 1).
__device__ __forceinline__ void sigmoid_pair(double z, double g, double& s, double& oms, double zmax = 746.0) {
  if (z > 0.0) {
    if (z > zmax) {
      s = 0.0;
      oms = 1.0;
      return;
    }
    const double e = exp(-z);
    const double r = 1.0 / (e + g);
    s = e * r;
    oms = g * r;
  } else {
    if (z < -45.0) {
      // g e^z < 3e-20 g: for degeneracies g below 3000, 1 / (1 + g e^z) rounds to exactly 1, and
      // 1 - s (which only scales the derivative) is taken as zero
      s = 1.0;
      oms = 0.0;
      return;
    }
    const double ge = g * exp(z);
    const double r = 1.0 / (1.0 + ge);
    s = r;
    oms = ge * r;
  }
}

struct Charge {
  double rho, drho, n, dn;
};

// resid: the residual's below-resolution cutoffs (elements outside the dots); else the 1e-60
// nm^-3 cutoffs of the electron counts.
__device__ __forceinline__ Charge charge_at(const Phys& P, double phi, bool resid = false) {
  Charge c;
  const double ik = P.inv_kT;
  const double eta_n = (P.EF + phi - P.phi_ref + P.chi) * ik;
  const double eta_p = (-phi + P.phi_ref - P.chi - P.Eg - P.EF) * ik;
  const double xn = resid ? P.eta_min_n : -150.0, xp = resid ? P.eta_min_p : -150.0;
  double n, dn, p, dp;
  if (P.statistics == 1) {
    double F, dF;
    fd_half_d(eta_n, F, dF, xn);
    n = P.NC * F;
    dn = P.NC * dF * ik;
    fd_half_d(eta_p, F, dF, xp);
    p = P.NV * F;
    dp = -P.NV * dF * ik;
  } else {
    n = eta_n < xn ? 0.0 : P.NC * exp(eta_n);
    dn = n * ik;
    p = eta_p < xp ? 0.0 : P.NV * exp(eta_p);
    dp = -p * ik;
  }
  double NDp = P.ND, dND = 0.0, NAm = P.NA, dNA = 0.0;
  if (P.incomplete) {
    if (P.nd_on) {
      double s, oms;
      sigmoid_pair((P.EF + P.Ed - P.phi_ref + P.chi + phi) * ik, P.gD, s, oms, resid ? P.z_max_d : 746.0);
      NDp = P.ND * s;
      dND = -P.ND * s * oms * ik;
    }
    if (P.na_on) {
      double s, oms;
      sigmoid_pair((-P.EF + P.Ea + P.phi_ref - P.chi - P.Eg - phi) * ik, P.gA, s, oms, resid ? P.z_max_a : 746.0);
      NAm = P.NA * s;
      dNA = P.NA * s * oms * ik;
    }
  }
  c.rho = p - n + NDp - NAm;
  c.drho = dp - dn + dND - dNA;
  c.n = n;
  c.dn = dn;
  return c;
}

// The constant-charge zone of a potential for charge_resid: -1 where some term needs evaluating,
// else A + 2 D with A (D) = 1 when the acceptors (donors) count as fully ionized.
__device__ __forceinline__ int charge_zone(const Phys& P, double phi) {
  if (!(phi < P.phi_n_on && phi > P.phi_p_on)) return -1;
  int z = 0;
  if (P.incomplete) {
    if (P.na_on) {
      if (phi > P.phi_a_hi)
        z += 1;
      else if (!(phi < P.phi_a_lo))
        return -1;
    }
    if (P.nd_on) {
      if (phi < P.phi_d_lo)
        z += 2;
      else if (!(phi > P.phi_d_hi))
        return -1;
    }
  }
  return z;
}

// charge_zone of a potential given as its double_key (integer comparisons only).
__device__ __forceinline__ int charge_zone_key(const Phys& P, unsigned long long key) {
  if (!(key < P.key_n_on && key > P.key_p_on)) return -1;
  int z = 0;
  if (P.incomplete) {
    if (P.na_on) {
      if (key > P.key_a_hi)
        z += 1;
      else if (!(key < P.key_a_lo))
        return -1;
    }
    if (P.nd_on) {
      if (key < P.key_d_lo)
        z += 2;
      else if (!(key > P.key_d_hi))
        return -1;
    }
  }
  return z;
}

// The charge of a constant-charge zone (the value charge_resid returns there); host and device
// evaluate it in the same order.
__host__ __device__ __forceinline__ double zone_charge(const Phys& P, int zone) {
  if (!P.incomplete) return P.ND - P.NA;
  double rho = 0.0;
  if (P.na_on) rho -= (zone & 1) ? P.NA : 0.0;
  if (P.nd_on) rho += (zone & 2) ? P.ND : 0.0;
  return rho;
}

// Slots of the residual's per-layer load table ([nz][8], ResidualArgs::wq): w_k = -(q/eps0) w|J|
// of one Gauss point of a layer-k element, and w_k times each constant charge, so that an element
// in a constant-charge zone takes its load from the table without FP64 arithmetic.
constexpr int WQ_ZONE_COMPLETE = 4;  // w_k (N_D - N_A): complete ionization
constexpr int WQ_WEIGHT = 5;         // w_k
constexpr int WQ_ZERO = 6;           // 0: no charge (oxide, padding)
// zones 0..3 (incomplete ionization): w_k zone_charge(zone)

// The residual's charge outside the dots: where phi lies outside every cutoff band (n and p below
// resolution, each dopant fully ionized or below resolution) the charge is a constant and its
// derivative zero, found by a few comparisons; elsewhere the full evaluation with the residual's
// cutoffs. Both give the same values as charge_at(P, phi, true).
__device__ __forceinline__ Charge charge_resid(const Phys& P, double phi) {
  const bool no_n = phi < P.phi_n_on, no_p = phi > P.phi_p_on;
  bool flat = no_n && no_p;
  double rho = 0.0;
  if (P.incomplete) {
    if (P.na_on) {
      flat = flat && (phi < P.phi_a_lo || phi > P.phi_a_hi);
      rho -= phi > P.phi_a_hi ? P.NA : 0.0;  // z_a < -45: fully ionized; above the cutoff: none
    }
    if (P.nd_on) {
      flat = flat && (phi < P.phi_d_lo || phi > P.phi_d_hi);
      rho += phi < P.phi_d_lo ? P.ND : 0.0;
    }
  } else {
    rho = P.ND - P.NA;
  }
  if (flat) return Charge{rho, 0.0, 0.0, 0.0};
  return charge_at(P, phi, true);
}

}  // namespace qcad
