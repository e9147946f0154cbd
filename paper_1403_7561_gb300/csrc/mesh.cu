// Mesh and geometry setup, bias-point physics and contact values (host side),
// plus the shared runtime helpers (errors, profiling events).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>

#include "dfloat.cuh"
#include "mesh.h"
#include "physics.cuh"

namespace qcad {

void check_cuda(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(e == cudaErrorMemoryAllocation ? QCAD_ERR_OOM : QCAD_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
  }
}

// ---------------------------------------------------------------------------
// Profiler: pairs of CUDA events around kernel launches on the mesh stream.
cudaEvent_t Profiler::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  CK(cudaEventCreate(&e));
  return e;
}
void Profiler::begin(int cls, cudaStream_t s, Pair& out) {
  std::lock_guard<std::mutex> lk(mu);
  out.a = get();
  out.b = get();
  out.cls = cls;
  CK(cudaEventRecord(out.a, s));
}
void Profiler::end(Pair& p, cudaStream_t s) {
  std::lock_guard<std::mutex> lk(mu);
  CK(cudaEventRecord(p.b, s));
  open.push_back(p);
}
void Profiler::harvest() {
  std::lock_guard<std::mutex> lk(mu);
  std::vector<Pair> keep;  // pairs of another stream that has not reached them yet
  for (auto& p : open) {
    const cudaError_t q = cudaEventQuery(p.b);
    if (q == cudaErrorNotReady) {
      keep.push_back(p);
      continue;
    }
    float t = 0.f;
    if (q == cudaSuccess && cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
      ms[p.cls] += t;
      launches[p.cls] += 1;
    } else {
      cudaGetLastError();
    }
    pool.push_back(p.a);
    pool.push_back(p.b);
  }
  open.swap(keep);
}
void Profiler::add(int cls, double ms_) {
  std::lock_guard<std::mutex> lk(mu);
  ms[cls] += ms_;
  launches[cls] += 1;
}
Profiler::~Profiler() {
  for (auto& p : open) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : pool) cudaEventDestroy(e);
}

// ---------------------------------------------------------------------------
// Constants (CODATA 2018) and bias-point physics, Sec. II.A.
static const double kQ = 1.602176634e-19, kKB = 1.380649e-23, kHBAR = 1.054571817e-34, kM0 = 9.1093837015e-31,
                    kEPS0 = 8.8541878128e-12;

double host_kT(double T) { return kKB * T / kQ; }
double host_qe() { return kQ / kEPS0 * 1e9; }
double host_h2m0() { return kHBAR * kHBAR / (2.0 * kM0) / kQ * 1e18; }

// Effective density of states 2 (m* k_B T / (2 pi hbar^2))^(3/2) in nm^-3 (Eq. EffectiveDOS).
static double eff_dos(double m_rel, double T) {
  const double a = m_rel * kM0 * kKB * T / (2.0 * M_PI * kHBAR * kHBAR) * 1e-18;
  return 2.0 * a * std::sqrt(a);
}

// DOS masses of Eq. EffectiveMass.
static void dos_masses(const qcad_material& m, double& mn, double& mp) {
  mn = std::pow(6.0, 2.0 / 3.0) * std::cbrt(m.m_l * m.m_t * m.m_t);
  mp = std::pow(std::pow(m.m_hh, 1.5) + std::pow(m.m_lh, 1.5), 2.0 / 3.0);
}

// Nilsson's inverse of F_1/2 (Eq. FDintInverse).
static double fd_inverse(double u) {
  const double first = std::fabs(u - 1.0) < 1e-12 ? -0.5 : -std::log(u) / (u * u - 1.0);
  const double nu = std::pow(3.0 * std::sqrt(M_PI) * u / 4.0, 2.0 / 3.0);
  const double w = 0.24 + 1.08 * nu;
  return first + nu / (1.0 + 1.0 / (w * w));
}

Phys make_phys(const qcad_mesh_s* m, const qcad_bias* b) {
  return make_phys_material(m->mats[m->semi >= 0 ? m->semi : 0], b);
}

Phys make_phys_material(const qcad_material& s, const qcad_bias* b) {
  Phys P{};
  P.kT = host_kT(b->T);
  P.inv_kT = 1.0 / P.kT;
  double mn, mp;
  dos_masses(s, mn, mp);
  P.NC = eff_dos(mn, b->T);
  P.NV = eff_dos(mp, b->T);
  // q phi_ref = E_0 - E_i(Si) = chi + E_g/2 + (kT/2) ln(N_C/N_V)  (Eq. qPhiRef)
  P.phi_ref = s.chi + 0.5 * s.Eg + 0.5 * P.kT * std::log(P.NC / P.NV);
  P.chi = s.chi;
  P.Eg = s.Eg;
  P.EF = -b->V_sub;  // E_F = -q V_sub (Sec. II.A.2)
  P.NA = s.N_A;
  P.ND = s.N_D;
  P.Ea = s.E_a;
  P.Ed = s.E_d;
  P.gA = s.g_A;
  P.gD = s.g_D;
  P.qe = host_qe();
  P.statistics = b->statistics;
  P.incomplete = b->incomplete_ionization;
  P.na_on = s.N_A != 0.0;
  P.nd_on = s.N_D != 0.0;
  // below-resolution cutoffs (physics.cuh): N F(eta) < floor for eta < ln(floor / N) (F <= e^eta),
  // N s < floor for s ~ e^-z / g below floor / N; never tighter than the count cutoffs (eta -150,
  // z 746)
  const double fl = RHO_RESID_FLOOR;
  P.eta_min_n = std::max(-150.0, std::log(fl / P.NC));
  P.eta_min_p = std::max(-150.0, std::log(fl / P.NV));
  P.z_max_a = s.N_A > 0 ? std::min(746.0, std::log(s.N_A / (s.g_A * fl))) : 746.0;
  P.z_max_d = s.N_D > 0 ? std::min(746.0, std::log(s.N_D / (s.g_D * fl))) : 746.0;
  // as potentials, widened by 1e-9 V so that rounding of the argument never skips a term the
  // FP64 test would evaluate: eta_n = (phi - cn) / kT, eta_p = (cp - phi) / kT, z_a = (ca - phi) / kT,
  // z_d = (phi - cd) / kT
  const double kT = P.kT, w = 1e-9;
  const double cn = P.phi_ref - s.chi - P.EF, cp = P.phi_ref - s.chi - s.Eg - P.EF;
  const double ca = -P.EF + s.E_a + P.phi_ref - s.chi - s.Eg, cd = -(P.EF + s.E_d - P.phi_ref + s.chi);
  P.phi_n_on = cn + P.eta_min_n * kT - w;
  P.phi_p_on = cp - P.eta_min_p * kT + w;
  P.phi_a_lo = ca - P.z_max_a * kT - w;
  P.phi_a_hi = ca + 45.0 * kT + w;
  P.phi_d_lo = cd - 45.0 * kT - w;
  P.phi_d_hi = cd + P.z_max_d * kT + w;
  auto key = [](double v) {
    unsigned long long b;
    std::memcpy(&b, &v, sizeof(b));
    return double_key(b);
  };
  P.key_n_on = key(P.phi_n_on);
  P.key_p_on = key(P.phi_p_on);
  P.key_a_lo = key(P.phi_a_lo);
  P.key_a_hi = key(P.phi_a_hi);
  P.key_d_lo = key(P.phi_d_lo);
  P.key_d_hi = key(P.phi_d_hi);
  return P;
}

// Ohmic contact potential, Sec. II.A.4 (Eqs. PotBC4MBCompIon, Yval4MBIncompIon,
// PotBC4MBIncompIon, ApproxLogTerms, PotBC4FDCompIon). For p-type with
// incomplete ionization the acceptor energy enters with +E_a, as follows from
// the definition of y_p.
double ohmic_value(const qcad_mesh_s* m, const qcad_bias* b, const Phys& P) {
  const qcad_material& s = m->mats[m->semi >= 0 ? m->semi : 0];
  const double kT = P.kT, Va = b->V_sub;
  if (s.N_A == 0.0 && s.N_D == 0.0) return Va;
  const bool ntype = s.N_D > s.N_A;
  const bool lowT = b->T < 50.0;
  if (b->incomplete_ionization) {
    if (ntype) {
      const double ln_y = lowT ? 0.5 * std::log(s.N_D / (2.0 * P.NC)) + s.E_d / (2.0 * kT)
                               : std::log(-0.25 + 0.25 * std::sqrt(1.0 + 8.0 * s.N_D / P.NC * std::exp(s.E_d / kT)));
      return (-s.E_d + P.phi_ref - s.chi) + kT * ln_y + Va;
    }
    const double ln_y = lowT ? 0.5 * std::log(s.N_A / (4.0 * P.NV)) + s.E_a / (2.0 * kT)
                             : std::log(-0.125 + 0.125 * std::sqrt(1.0 + 16.0 * s.N_A / P.NV * std::exp(s.E_a / kT)));
    return (s.E_a + P.phi_ref - s.chi - s.Eg) - kT * ln_y + Va;
  }
  if (b->statistics == 0) {
    if (ntype) return (P.phi_ref - s.chi) + kT * std::log(s.N_D / P.NC) + Va;
    return (P.phi_ref - s.chi - s.Eg) - kT * std::log(s.N_A / P.NV) + Va;
  }
  if (ntype) return (P.phi_ref - s.chi) + kT * fd_inverse(s.N_D / P.NC) + Va;
  return (P.phi_ref - s.chi - s.Eg) - kT * fd_inverse(s.N_A / P.NV) + Va;
}

// Gate Dirichlet value phi_ins = V_g - (Phi_m - q phi_ref)/q (Eq. ContOnIns).
double gate_value(const qcad_mesh_s* m, double Vg, const Phys& P) {
  const double Phi_m = m->wf_set ? m->wf : P.phi_ref;
  return Vg - (Phi_m - P.phi_ref);
}

// ---------------------------------------------------------------------------
// 1D assembled linear-element operators on node coordinates x[0..n]: rows (coefficients of
// nodes i-1, i, i+1) of the mass and stiffness with per-element weights kappa (null: 1).
void row_ops_raw(const double* x, int n, const double* kappa, double* M, double* K) {
  for (int i = 0; i < 3 * (n + 1); ++i) M[i] = K[i] = 0.0;
  for (int i = 0; i <= n; ++i) {
    if (i > 0) {
      const double h = x[i] - x[i - 1], kp = kappa ? kappa[i - 1] : 1.0;
      M[3 * i + 0] += kp * h / 6.0;
      M[3 * i + 1] += kp * h / 3.0;
      K[3 * i + 0] += -kp / h;
      K[3 * i + 1] += kp / h;
    }
    if (i < n) {
      const double h = x[i + 1] - x[i], kp = kappa ? kappa[i] : 1.0;
      M[3 * i + 1] += kp * h / 3.0;
      M[3 * i + 2] += kp * h / 6.0;
      K[3 * i + 1] += kp / h;
      K[3 * i + 2] += -kp / h;
    }
  }
}

static void row_ops(const std::vector<double>& x, const std::vector<double>& kappa, std::vector<double>& M,
                    std::vector<double>& K) {
  const int n = (int)x.size() - 1;
  M.assign(3 * (n + 1), 0.0);
  K.assign(3 * (n + 1), 0.0);
  row_ops_raw(x.data(), n, kappa.data(), M.data(), K.data());
}

GridTables make_tables(const std::vector<double>& x, const std::vector<double>& y, const std::vector<double>& z,
                       const std::vector<double>& kx_layer, const std::vector<double>& ky_layer,
                       const std::vector<double>& kz_layer) {
  GridTables t;
  std::vector<double> ones_x(x.size() - 1, 1.0), ones_y(y.size() - 1, 1.0);
  row_ops(x, ones_x, t.mx, t.kx);
  row_ops(y, ones_y, t.my, t.ky);
  std::vector<double> dummy;
  row_ops(z, kx_layer, t.mzx, dummy);
  row_ops(z, ky_layer, t.mzy, dummy);
  std::vector<double> dm;
  row_ops(z, kz_layer, dm, t.kzz);
  return t;
}

template <class T>
static void upload(DevBuf& b, const std::vector<double>& v, cudaStream_t s) {
  std::vector<T> h(v.begin(), v.end());
  b.ensure(h.size() * sizeof(T) + 16);
  CK(cudaMemcpyAsync(b.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
}

template <class T>
void build_grid(GridDev<T>& gd, const GridTables& t, const std::vector<double>& hx, const std::vector<double>& hy,
                const std::vector<double>& hz, cudaStream_t s) {
  upload<T>(gd.mx, t.mx, s);
  upload<T>(gd.kx, t.kx, s);
  upload<T>(gd.my, t.my, s);
  upload<T>(gd.ky, t.ky, s);
  upload<T>(gd.mzx, t.mzx, s);
  upload<T>(gd.mzy, t.mzy, s);
  upload<T>(gd.kzz, t.kzz, s);
  std::vector<double> zt(12 * (t.kzz.size() / 3), 0.0);
  for (size_t k = 0; k < t.kzz.size() / 3; ++k)
    for (int q = 0; q < 3; ++q) {
      zt[12 * k + q] = t.mzx[3 * k + q];
      zt[12 * k + 3 + q] = t.mzy[3 * k + q];
      zt[12 * k + 6 + q] = t.kzz[3 * k + q];
    }
  upload<T>(gd.zt, zt, s);
  upload<T>(gd.hx, hx, s);
  upload<T>(gd.hy, hy, s);
  upload<T>(gd.hz, hz, s);
  Grid<T>& g = gd.g;
  g.nx = (int)hx.size();
  g.ny = (int)hy.size();
  g.nz = (int)hz.size();
  g.nxn = g.nx + 1;
  g.nyn = g.ny + 1;
  g.nzn = g.nz + 1;
  g.plane = (long long)g.nxn * g.nyn;
  g.mx = gd.mx.template as<T>();
  g.kx = gd.kx.template as<T>();
  g.my = gd.my.template as<T>();
  g.ky = gd.ky.template as<T>();
  g.mzx = gd.mzx.template as<T>();
  g.mzy = gd.mzy.template as<T>();
  g.kzz = gd.kzz.template as<T>();
  g.zt = gd.zt.template as<T>();
  g.hx = gd.hx.template as<T>();
  g.hy = gd.hy.template as<T>();
  g.hz = gd.hz.template as<T>();
}
template void build_grid<float>(GridDev<float>&, const GridTables&, const std::vector<double>&,
                                const std::vector<double>&, const std::vector<double>&, cudaStream_t);
template void build_grid<double>(GridDev<double>&, const GridTables&, const std::vector<double>&,
                                 const std::vector<double>&, const std::vector<double>&, cudaStream_t);
template void build_grid<dfl>(GridDev<dfl>&, const GridTables&, const std::vector<double>&,
                              const std::vector<double>&, const std::vector<double>&, cudaStream_t);

// Faces (fi, fj) of a node plane whose four corners lie in the closed rectangle: fi in [i0, i1),
// fj in [j0, j1) (empty ranges when none).
static void rect_faces(const qcad_mesh_s* m, double x0, double x1, double y0, double y1, int r[4]) {
  r[0] = m->nx, r[1] = 0, r[2] = m->ny, r[3] = 0;
  for (int i = 0; i < m->nx; ++i)
    if (m->xc[i] >= x0 && m->xc[i + 1] <= x1) r[0] = std::min(r[0], i), r[1] = std::max(r[1], i + 1);
  for (int j = 0; j < m->ny; ++j)
    if (m->yc[j] >= y0 && m->yc[j + 1] <= y1) r[2] = std::min(r[2], j), r[3] = std::max(r[3], j + 1);
}

// Surface terms of the weak form (Sec. II.A.4): the charged gates' face coefficients eps_r/d and
// their vectors (eps_r/d) int_f N_a, and the bias-independent load (q/eps0) sigma int_f N_a of the
// charged gates' sheets and of the surface charges (int_f N_a = h_x h_y / 4 on a rectangle face).
static void build_surface_terms(qcad_mesh_s* m, const qcad_device* dev) {
  m->has_robin = dev->n_charged_gates > 0;
  m->has_surface = m->has_robin || dev->n_surface_charges > 0;
  if (!m->has_surface) return;
  const long long plane = (long long)m->nxn * m->nyn;
  const double qe = host_qe();
  std::vector<double> b0((size_t)m->nxn * m->nyn * m->nzn, 0.0);
  std::vector<double> alpha((size_t)m->nx * m->ny, 0.0);
  auto add_faces = [&](const int r[4], long long base, double w, double* dst) {
    for (int fj = r[2]; fj < r[3]; ++fj)
      for (int fi = r[0]; fi < r[1]; ++fi) {
        const double q = w * m->hxv[fi] * m->hyv[fj] * 0.25;
        for (int a = 0; a < 4; ++a) dst[base + (fi + (a & 1)) + (long long)m->nxn * (fj + (a >> 1))] += q;
      }
  };
  const double eps_top = m->mats[m->layer_mat[m->nz - 1]].eps_r;
  const long long top = (long long)m->nz * plane;
  for (int c = 0; c < dev->n_charged_gates; ++c) {
    const qcad_charged_gate& C = dev->charged_gates[c];
    const qcad_rect& G = dev->gates[C.gate];
    int r[4];
    rect_faces(m, G.x0, G.x1, G.y0, G.y1, r);
    const double a = eps_top / C.d;
    for (int fj = r[2]; fj < r[3]; ++fj)
      for (int fi = r[0]; fi < r[1]; ++fi) alpha[fi + (size_t)m->nx * fj] += a;
    std::vector<double> rv((size_t)plane, 0.0);
    add_faces(r, 0, a, rv.data());
    m->charged_gate.push_back(C.gate);
    m->charged_r.push_back(std::move(rv));
    add_faces(r, top, qe * C.sigma, b0.data());
  }
  for (int q = 0; q < dev->n_surface_charges; ++q) {
    const qcad_surface_charge& S = dev->surface_charges[q];
    if (!std::isfinite(S.z) || !std::isfinite(S.sigma)) throw Error(QCAD_ERR_INVALID_ARG, "non-finite surface charge");
    int k = -1;
    for (int kk = 0; kk <= m->nz; ++kk)
      if (std::fabs(m->zc[kk] - S.z) <= 1e-9 * std::max(1.0, std::fabs(S.z))) k = kk;
    if (k < 0) throw Error(QCAD_ERR_INVALID_ARG, "a surface charge's z is not a node plane of the mesh");
    int r[4];
    rect_faces(m, S.x0, S.x1, S.y0, S.y1, r);
    add_faces(r, (long long)k * plane, qe * S.sigma, b0.data());
  }
  m->bsig_top.assign(b0.begin() + top, b0.begin() + top + plane);
  m->btop = m->bsig_top;
  cudaStream_t s = m->stream;
  m->d_bsurf.ensure(b0.size() * sizeof(double) + 64);
  CK(cudaMemcpyAsync(m->d_bsurf.p, b0.data(), b0.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  if (m->has_robin) {
    std::vector<double> rall;
    for (const auto& rv : m->charged_r) rall.insert(rall.end(), rv.begin(), rv.end());
    m->d_charged_r.ensure(rall.size() * sizeof(double) + 64);
    CK(cudaMemcpyAsync(m->d_charged_r.p, rall.data(), rall.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    std::vector<float> a32(alpha.begin(), alpha.end());
    m->d_face64.ensure(alpha.size() * sizeof(double) + 64);
    m->d_face32.ensure(alpha.size() * sizeof(float) + 64);
    CK(cudaMemcpyAsync(m->d_face64.p, alpha.data(), alpha.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(m->d_face32.p, a32.data(), a32.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    // the element-gather kernels carry the face term
    m->cfg64.variant = 0;
    m->cfg32.variant = 0;
  }
  CK(cudaStreamSynchronize(s));
}

// Checks of a device description shared by every entry point that takes one (mesh_create and
// the allocation-free residual): sizes, gate and dot lists, layers, materials (at most one
// semiconductor material, permittivities > 0), and the limits of the kernels' 32-bit node and
// coefficient indices and of the z-grid dimension. Returns the element-layer count.
int validate_device(const qcad_device* dev) {
  if (!dev) throw Error(QCAD_ERR_INVALID_ARG, "null device description");
  if (dev->nx < 1 || dev->ny < 1 || dev->n_layers < 1 || !dev->layer_n || !dev->layer_thickness ||
      !dev->layer_material || dev->n_materials < 1 || !dev->materials || !(dev->Lx > 0) || !(dev->Ly > 0))
    throw Error(QCAD_ERR_INVALID_ARG, "invalid mesh sizes or layer description");
  if (dev->n_gates < 0 || dev->n_gates > QCAD_MAX_GATES || (dev->n_gates > 0 && !dev->gates))
    throw Error(QCAD_ERR_INVALID_ARG, "invalid gate list");
  if (dev->n_dots < 0 || dev->n_dots > QCAD_MAX_DOTS || (dev->n_dots > 0 && !dev->dots))
    throw Error(QCAD_ERR_INVALID_ARG, "invalid dot list");
  if (dev->nx > 8192 || dev->ny > 8192) throw Error(QCAD_ERR_INVALID_ARG, "mesh too large along x or y");
  int semi = -1;
  for (int i = 0; i < dev->n_materials; ++i)
    if (dev->materials[i].semiconductor) {
      if (semi >= 0 && std::memcmp(&dev->materials[i], &dev->materials[semi], sizeof(qcad_material)) != 0)
        throw Error(QCAD_ERR_INVALID_ARG, "at most one semiconductor material is supported");
      semi = i;
    }
  for (int i = 0; i < dev->n_materials; ++i)
    if (!(dev->materials[i].eps_r > 0)) throw Error(QCAD_ERR_INVALID_ARG, "material permittivity must be > 0");
  long long nz = 0;
  for (int L = 0; L < dev->n_layers; ++L) {
    const int mat = dev->layer_material[L];
    if (dev->layer_n[L] < 1 || !(dev->layer_thickness[L] > 0) || mat < 0 || mat >= dev->n_materials)
      throw Error(QCAD_ERR_INVALID_ARG, "invalid layer group");
    nz += dev->layer_n[L];
  }
  if (nz > 65535) throw Error(QCAD_ERR_INVALID_ARG, "too many element layers");
  // kernels index nodes and element coefficient arrays with 32-bit integers
  if ((long long)(dev->nx + 1) * (dev->ny + 1) * (nz + 1) >= (1LL << 31) ||
      8LL * dev->nx * dev->ny * nz >= (1LL << 31))
    throw Error(QCAD_ERR_INVALID_ARG, "mesh too large for 32-bit node and coefficient indices");
  return (int)nz;
}

void mesh_create(const qcad_device* dev, void* stream, qcad_mesh_t* out) {
  if (!dev || !out) throw Error(QCAD_ERR_INVALID_ARG, "null device description or output");
  validate_device(dev);
  if (dev->nx < 1 || dev->ny < 1 || dev->n_layers < 1 || !dev->layer_n || !dev->layer_thickness ||
      !dev->layer_material || dev->n_materials < 1 || !dev->materials || !(dev->Lx > 0) || !(dev->Ly > 0))
    throw Error(QCAD_ERR_INVALID_ARG, "invalid mesh sizes or layer description");
  if (dev->n_gates < 0 || dev->n_gates > QCAD_MAX_GATES || (dev->n_gates > 0 && !dev->gates))
    throw Error(QCAD_ERR_INVALID_ARG, "invalid gate list");
  if (dev->n_dots < 0 || dev->n_dots > QCAD_MAX_DOTS || (dev->n_dots > 0 && !dev->dots))
    throw Error(QCAD_ERR_INVALID_ARG, "invalid dot list");
  if (dev->nx > 8192 || dev->ny > 8192) throw Error(QCAD_ERR_INVALID_ARG, "mesh too large along x or y");
  auto m = new qcad_mesh_s();
  try {
    CK(cudaGetDevice(&m->device));
    m->stream = (cudaStream_t)stream;
    if (m->stream == nullptr) {
      // a blocking stream: it still orders with the legacy default stream, but unlike it can be
      // captured into CUDA graphs
      CK(cudaStreamCreateWithFlags(&m->stream, cudaStreamDefault));
      m->owns_stream = true;
    }
    m->nx = dev->nx;
    m->ny = dev->ny;
    m->mats.assign(dev->materials, dev->materials + dev->n_materials);
    m->semi = -1;
    for (int i = 0; i < dev->n_materials; ++i)
      if (dev->materials[i].semiconductor) {
        if (m->semi >= 0 && std::memcmp(&dev->materials[i], &dev->materials[m->semi], sizeof(qcad_material)) != 0)
          throw Error(QCAD_ERR_INVALID_ARG, "at most one semiconductor material is supported");
        m->semi = i;
      }
    for (int i = 0; i < dev->n_materials; ++i)
      if (!(dev->materials[i].eps_r > 0)) throw Error(QCAD_ERR_INVALID_ARG, "material permittivity must be > 0");
    // node planes
    m->xc.resize(m->nx + 1);
    m->yc.resize(m->ny + 1);
    for (int i = 0; i <= m->nx; ++i) m->xc[i] = dev->Lx * i / m->nx;
    for (int j = 0; j <= m->ny; ++j) m->yc[j] = dev->Ly * j / m->ny;
    m->zc.assign(1, 0.0);
    for (int L = 0; L < dev->n_layers; ++L) {
      const int n = dev->layer_n[L];
      const double t = dev->layer_thickness[L];
      const int mat = dev->layer_material[L];
      if (n < 1 || !(t > 0) || mat < 0 || mat >= dev->n_materials)
        throw Error(QCAD_ERR_INVALID_ARG, "invalid layer group");
      const double z0 = m->zc.back();
      for (int s = 0; s < n; ++s) {
        m->zc.push_back(z0 + t * (s + 1) / n);
        m->layer_mat.push_back(mat);
      }
    }
    m->nz = (int)m->layer_mat.size();
    if (m->nz > 65535) throw Error(QCAD_ERR_INVALID_ARG, "too many element layers");
    // kernels index nodes and element coefficient arrays with 32-bit integers
    if ((long long)(m->nx + 1) * (m->ny + 1) * (m->nz + 1) >= (1LL << 31) ||
        8LL * m->nx * m->ny * m->nz >= (1LL << 31))
      throw Error(QCAD_ERR_INVALID_ARG, "mesh too large for 32-bit node and coefficient indices");
    m->nxn = m->nx + 1;
    m->nyn = m->ny + 1;
    m->nzn = m->nz + 1;
    m->n_nodes = m->nxn * m->nyn * m->nzn;
    m->n_elems = (long long)m->nx * m->ny * m->nz;
    for (int i = 0; i < m->nx; ++i) m->hxv.push_back(m->xc[i + 1] - m->xc[i]);
    for (int j = 0; j < m->ny; ++j) m->hyv.push_back(m->yc[j + 1] - m->yc[j]);
    for (int k = 0; k < m->nz; ++k) m->hzv.push_back(m->zc[k + 1] - m->zc[k]);
    std::vector<double> eps(m->nz);
    m->layer_semi.resize(m->nz);
    for (int k = 0; k < m->nz; ++k) {
      eps[k] = m->mats[m->layer_mat[k]].eps_r;
      m->layer_semi[k] = (unsigned char)(m->mats[m->layer_mat[k]].semiconductor ? 1 : 0);
    }
    // contacts: gate of every top-plane node (first gate containing it)
    m->n_gates = dev->n_gates;
    m->wf_set = dev->gate_work_function_set;
    m->wf = dev->gate_work_function;
    m->bottom_ohmic = dev->bottom_ohmic;
    // charged gates (Robin condition): their nodes stay unknowns
    if (dev->n_charged_gates < 0 || dev->n_charged_gates > dev->n_gates ||
        (dev->n_charged_gates > 0 && !dev->charged_gates) || dev->n_surface_charges < 0 ||
        (dev->n_surface_charges > 0 && !dev->surface_charges))
      throw Error(QCAD_ERR_INVALID_ARG, "invalid charged-gate or surface-charge list");
    std::vector<char> charged(std::max(1, dev->n_gates), 0);
    for (int c = 0; c < dev->n_charged_gates; ++c) {
      const qcad_charged_gate& C = dev->charged_gates[c];
      if (C.gate < 0 || C.gate >= dev->n_gates || charged[C.gate])
        throw Error(QCAD_ERR_INVALID_ARG, "charged gate index out of range or repeated");
      if (!(C.d > 0) || !std::isfinite(C.d) || !std::isfinite(C.sigma))
        throw Error(QCAD_ERR_INVALID_ARG, "a charged gate needs d > 0 and a finite sigma");
      charged[C.gate] = 1;
    }
    m->gate_top.assign(m->nxn * m->nyn, -1);
    std::vector<unsigned char> dir_top(m->nxn * m->nyn, 0);
    for (long long j = 0; j < m->nyn; ++j)
      for (long long i = 0; i < m->nxn; ++i) {
        for (int gi = 0; gi < dev->n_gates; ++gi) {
          const qcad_rect& G = dev->gates[gi];
          if (m->xc[i] >= G.x0 && m->xc[i] <= G.x1 && m->yc[j] >= G.y0 && m->yc[j] <= G.y1) {
            if (!charged[gi]) {
              m->gate_top[i + m->nxn * j] = (signed char)gi;
              dir_top[i + m->nxn * j] = 1;
            }
            break;
          }
        }
      }
    build_surface_terms(m, dev);
    m->dots.n = dev->n_dots;
    for (int d = 0; d < dev->n_dots; ++d) {
      const qcad_box& B = dev->dots[d];
      double b6[6] = {B.x0, B.x1, B.y0, B.y1, B.z0, B.z1};
      for (int s = 0; s < 6; ++s) m->dots.b[d][s] = b6[s];
    }
    m->has_sub = dev->has_subdomain;
    if (m->has_sub) {
      for (int s = 0; s < 6; ++s) m->sub[s] = dev->sub[s];
      if (!(m->sub[0] >= 0 && m->sub[1] <= m->nx && m->sub[1] - m->sub[0] >= 2 && m->sub[2] >= 0 &&
            m->sub[3] <= m->ny && m->sub[3] - m->sub[2] >= 2 && m->sub[4] >= 0 && m->sub[5] <= m->nz &&
            m->sub[5] - m->sub[4] >= 2))
        throw Error(QCAD_ERR_INVALID_ARG, "invalid Schrodinger subdomain");
    }
    // device geometry
    cudaStream_t s = m->stream;
    GridTables t = make_tables(m->xc, m->yc, m->zc, eps, eps, eps);
    build_grid<double>(m->g64, t, m->hxv, m->hyv, m->hzv, s);
    build_grid<float>(m->g32, t, m->hxv, m->hyv, m->hzv, s);
    upload<double>(m->d_xn, m->xc, s);
    upload<double>(m->d_yn, m->yc, s);
    upload<double>(m->d_zn, m->zc, s);
    m->d_layer_semi.ensure(m->nz + 16);
    CK(cudaMemcpyAsync(m->d_layer_semi.p, m->layer_semi.data(), m->nz, cudaMemcpyHostToDevice, s));
    // the residual's per-layer load table: -(q/eps0) w|J| of one Gauss point of a layer-k element
    // (uniform x and y spacing, the tensor-product grid of every device) and its products with
    // the semiconductor's constant charges (slots in physics.cuh)
    {
      Phys Pz{};
      if (m->semi >= 0) {
        Pz.NA = m->mats[m->semi].N_A;
        Pz.ND = m->mats[m->semi].N_D;
        Pz.na_on = Pz.NA != 0.0;
        Pz.nd_on = Pz.ND != 0.0;
      }
      std::vector<double> wq(8 * (size_t)m->nz, 0.0);
      const double hxy = (dev->Lx / m->nx) * (dev->Ly / m->ny);
      for (int k = 0; k < m->nz; ++k) {
        const double w = -host_qe() * hxy * m->hzv[k] * 0.125;
        Pz.incomplete = 1;
        for (int z = 0; z < 4; ++z) wq[8 * k + z] = w * zone_charge(Pz, z);
        Pz.incomplete = 0;
        wq[8 * k + WQ_ZONE_COMPLETE] = w * zone_charge(Pz, 0);
        wq[8 * k + WQ_WEIGHT] = w;
      }
      m->d_wq.ensure(wq.size() * sizeof(double) + 16);
      CK(cudaMemcpyAsync(m->d_wq.p, wq.data(), wq.size() * sizeof(double), cudaMemcpyHostToDevice, s));
      m->d_ecode.ensure((size_t)m->nx * m->ny * m->nz + 16);
      CK(cudaStreamSynchronize(s));
    }
    m->d_gate_top.ensure(m->gate_top.size() + 16);
    CK(cudaMemcpyAsync(m->d_gate_top.p, m->gate_top.data(), m->gate_top.size(), cudaMemcpyHostToDevice, s));
    m->d_dir_top.ensure(dir_top.size() + 16);
    CK(cudaMemcpyAsync(m->d_dir_top.p, dir_top.data(), dir_top.size(), cudaMemcpyHostToDevice, s));
    m->d_vgate.ensure(sizeof(double) * (QCAD_MAX_GATES + 1));
    CK(cudaStreamSynchronize(s));
    for (auto* g : {&m->g64.g}) {
      g->dir_top = m->d_dir_top.as<unsigned char>();
      g->dir_bottom = m->bottom_ohmic;
      g->dir_boundary = 0;
    }
    m->g32.g.dir_top = m->d_dir_top.as<unsigned char>();
    m->g32.g.dir_bottom = m->bottom_ohmic;
    m->g32.g.dir_boundary = 0;
    CK(cudaMallocHost(&m->h_scal, sizeof(PcgScalars)));
    CK(cudaMallocHost(&m->h_small, 64 * sizeof(double)));
    m->scal.ensure(sizeof(PcgScalars));
    m->stats.ensure(64 * sizeof(double));
    m->counts.ensure(QCAD_MAX_DOTS_K * sizeof(double));
  } catch (...) {
    delete m;
    throw;
  }
  *out = m;
}

}  // namespace qcad

qcad_mesh_s::~qcad_mesh_s() {
  if (owns_stream && stream) cudaStreamDestroy(stream);
  if (h_scal) cudaFreeHost(h_scal);
  if (h_small) cudaFreeHost(h_small);
  if (h_small2) cudaFreeHost(h_small2);
  if (stream2) cudaStreamDestroy(stream2);
}
