// Self-consistent Schrodinger-Poisson loop by the predictor-corrector scheme (Sec. II.C), for
// electrons confined in three dimensions: the quantum region is the Schrodinger subdomain, where
// the electron density of the Poisson equation is the predictor density of
// Eq. ApproxEDens3DConfined built from the last eigenpairs; V = q phi_ref - chi - q phi + V_xc(n)
// with the Hedin-Lundqvist V_xc of Eq. Vxc (scalar mass of Eq. mxc).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "mesh.h"
#include "qcad_dense.h"

namespace qcad {

qcad_status poisson_solve(qcad_mesh_s* m, const qcad_bias* b, const qcad_solver_opts* o, const double* theta,
                          double* phi, qcad_solve_report* rep);
qcad_status schrodinger_eigs_sp(qcad_mesh_s* m, const qcad_bias* b, const double* phi, int nev, const double* m_eff,
                                double tol, const double* vxq, const double* x0, double* evals, double* evecs,
                                qcad_solve_report* rep);
Phys make_phys(const qcad_mesh_s* m, const qcad_bias* b);
void set_message(const std::string& msg);

namespace {

constexpr int SP_THREADS = 256;

// One thread per (quantum element, Gauss point); the 8 lanes of an element hold its corners and
// its Gauss points under the same index (ix + 2 iy + 4 iz), so B (x) B (x) B is three butterflies.
struct SpGeom {
  int i0, j0, k0;       // first element of the region in the mesh
  int nx, ny, nz;       // region elements per axis
  long long nxn, nyn;   // mesh nodes per axis (x, y)
};

__device__ __forceinline__ double sp_interp(double v) {
  const double A = GaussConst<double>::a(), B = GaussConst<double>::b();
  v = A * v + B * __shfl_xor_sync(FULL_MASK, v, 1);
  v = A * v + B * __shfl_xor_sync(FULL_MASK, v, 2);
  v = A * v + B * __shfl_xor_sync(FULL_MASK, v, 4);
  return v;
}

// w[(8 qe + q) nev + i] = 4 psi_i(x_q)^2 from the interior-node eigenvectors (column-major,
// ndof rows; psi = 0 on the region's boundary nodes), and phiq[8 qe + q] = phi(x_q).
__global__ void __launch_bounds__(SP_THREADS) sp_tables_kernel(const SpGeom G, int nev, const double* __restrict__ evecs,
                                                               long long ndof, const double* __restrict__ phi,
                                                               double* w, double* phiq) {
  const long long ne = (long long)G.nx * G.ny * G.nz;
  const long long t = blockIdx.x * (long long)SP_THREADS + threadIdx.x;
  const bool valid = t < 8 * ne;
  const long long qe = valid ? (t >> 3) : 0;
  const int l = threadIdx.x & 7;
  const int is = (int)(qe % G.nx), js = (int)((qe / G.nx) % G.ny), ks = (int)(qe / ((long long)G.nx * G.ny));
  // this lane's corner, in region-local node coordinates
  const int a = is + (l & 1), b = js + ((l >> 1) & 1), c = ks + (l >> 2);
  const bool interior = a > 0 && b > 0 && c > 0 && a < G.nx && b < G.ny && c < G.nz;
  const long long d = interior ? (a - 1) + (long long)(G.nx - 1) * ((b - 1) + (long long)(G.ny - 1) * (c - 1)) : 0;
  const long long node = (G.i0 + a) + G.nxn * ((G.j0 + b) + G.nyn * (long long)(G.k0 + c));
  const double pq = sp_interp(valid ? phi[node] : 0.0);
  if (valid) phiq[t] = pq;
  for (int i = 0; i < nev; ++i) {
    const double psi = sp_interp(valid && interior ? evecs[(long long)i * ndof + d] : 0.0);
    if (valid) w[t * nev + i] = 4.0 * psi * psi;
  }
}

// Hedin-Lundqvist V_xc (eV) at density n (nm^-3): -pref (3 pi^2 n)^(1/3) [1 + 0.7734 x ln(1 + 1/x)],
// x = (1/21) (3 / (4 pi n b^3))^(1/3); 0 for n <= 0.
__device__ __forceinline__ double sp_vxc(double n, double pref, double b3) {
  if (!(n > 0.0)) return 0.0;
  const double x = cbrt(3.0 / (4.0 * 3.14159265358979323846 * n * b3)) / 21.0;
  return -pref * cbrt(3.0 * 3.14159265358979323846 * 3.14159265358979323846 * n) * (1.0 + 0.7734 * x * log1p(1.0 / x));
}

// n~ at phi (the predictor density with the tables of the last eigenpairs), V_xc(n~) into vxq
// (0 without V_xc), and the electron count of the region (sum of wdet n~) into acc[0].
__global__ void __launch_bounds__(SP_THREADS) sp_density_kernel(const SpGeom G, const QuantumDensity qd,
                                                                const double* __restrict__ phi, const double* hx,
                                                                const double* hy, const double* hz, double EF,
                                                                double ik, int use_vxc, double pref, double b3,
                                                                double* vxq, double* acc) {
  const long long ne = (long long)G.nx * G.ny * G.nz;
  const long long t = blockIdx.x * (long long)SP_THREADS + threadIdx.x;
  const bool valid = t < 8 * ne;
  const long long qe = valid ? (t >> 3) : 0;
  const int l = threadIdx.x & 7;
  const int is = (int)(qe % G.nx), js = (int)((qe / G.nx) % G.ny), ks = (int)(qe / ((long long)G.nx * G.ny));
  const long long node = (G.i0 + is + (l & 1)) + G.nxn * ((G.j0 + js + ((l >> 1) & 1)) +
                                                          G.nyn * (long long)(G.k0 + ks + (l >> 2)));
  const double pq = sp_interp(valid ? phi[node] : 0.0);
  double cnt = 0.0;
  if (valid) {
    double n, dn;
    qd_density(qd, qe, l, pq, EF, ik, n, dn);
    vxq[t] = use_vxc ? sp_vxc(n, pref, b3) : 0.0;
    cnt = hx[G.i0 + is] * hy[G.j0 + js] * hz[G.k0 + ks] * 0.125 * n;
  }
  double s[1] = {cnt};
  block_sum_atomic<1>(s, acc);
}

// max |a - b| over n entries into *out (non-negative doubles order like their bit patterns).
__global__ void sp_maxdiff_kernel(long long n, const double* a, const double* b, double* out) {
  double m = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(a[i] - b[i]));
  block_max_atomic(m, out);
}

int blocks_of(long long n) { return (int)std::max<long long>(1, (n + SP_THREADS - 1) / SP_THREADS); }

}  // namespace

// The predictor-corrector loop. phi: device, n_nodes, output (the semiclassical solve starts it);
// evals: host, nev. tol_dphi <= 0 runs exactly max_iter outer iterations.
qcad_status sp_solve(qcad_mesh_s* m, const qcad_bias* b, const qcad_solver_opts* o, int nev, const double* m_eff,
                     double eig_tol, double tol_dphi, int max_iter, int use_vxc, double* phi, double* evals,
                     qcad_sp_report* rep) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!m->has_sub) throw Error(QCAD_ERR_INVALID_ARG, "mesh has no Schrodinger subdomain (the quantum region)");
  if (m->has_surface)
    throw Error(QCAD_ERR_INVALID_ARG, "the Schrodinger-Poisson loop does not take charged gates or surface charges");
  if (!b || !o || !phi || !evals || !m_eff) throw Error(QCAD_ERR_INVALID_ARG, "null pointer");
  if (nev < 1 || nev > QD_MAX_STATES) throw Error(QCAD_ERR_INVALID_ARG, "nev must be in [1, 16]");
  if (max_iter < 1 || max_iter > 1000) throw Error(QCAD_ERR_INVALID_ARG, "max_iter must be in [1, 1000]");
  if (!(eig_tol > 0)) throw Error(QCAD_ERR_INVALID_ARG, "eig_tol must be > 0");
  cudaStream_t s = m->stream;
  const long long n = m->n_nodes;
  SpGeom G;
  G.i0 = m->sub[0];
  G.j0 = m->sub[2];
  G.k0 = m->sub[4];
  G.nx = m->sub[1] - m->sub[0];
  G.ny = m->sub[3] - m->sub[2];
  G.nz = m->sub[5] - m->sub[4];
  G.nxn = m->nxn;
  G.nyn = m->nyn;
  const long long nqe = (long long)G.nx * G.ny * G.nz;
  const long long ndof = (long long)(G.nx - 1) * (G.ny - 1) * (G.nz - 1);
  if (ndof < 3 * (nev + 4)) throw Error(QCAD_ERR_INVALID_ARG, "quantum region too small for nev");
  m->sp_w.ensure((size_t)8 * nqe * nev * sizeof(double) + 64);
  m->sp_phiq.ensure((size_t)8 * nqe * sizeof(double) + 64);
  m->sp_vxq.ensure((size_t)8 * nqe * sizeof(double) + 64);
  m->sp_evecs.ensure((size_t)ndof * nev * sizeof(double) + 64);
  m->sp_prev.ensure((size_t)n * sizeof(double) + 64);
  m->stats.ensure(64 * sizeof(double));
  double* prev = m->sp_prev.as<double>();
  double* acc = m->stats.as<double>() + 56;  // [0] count, [1] max |dphi|
  // V_xc constants: q^2/(4 pi^2 eps_s) = (q^2/(4 pi eps0)) / (pi eps_r) and b = eps_r a0 / m_xc
  const double kQ = 1.602176634e-19, kEPS0 = 8.8541878128e-12, kHBAR = 1.054571817e-34, kM0 = 9.1093837015e-31;
  const double pi = 3.14159265358979323846;
  const double coul = kQ / (4.0 * pi * kEPS0) * 1e9;                       // eV nm
  const double a0 = 4.0 * pi * kEPS0 * kHBAR * kHBAR / (kM0 * kQ * kQ) * 1e9;  // nm
  if (m->semi < 0) throw Error(QCAD_ERR_INVALID_ARG, "device has no semiconductor");
  const qcad_material& si = m->mats[m->semi];
  const double mxc = 1.0 / ((1.0 / si.m_l + 2.0 / si.m_t) / 3.0);
  const double pref = coul / (pi * si.eps_r);
  const double bb = si.eps_r * a0 / mxc;
  const double b3 = bb * bb * bb;
  const Phys P = make_phys(m, b);

  qcad_sp_report r{};
  // step (1): semiclassical solve, V without V_xc
  m->qd_active = false;
  qcad_status st = poisson_solve(m, b, o, nullptr, phi, nullptr);
  if (st != QCAD_OK) return st;
  CK(cudaMemsetAsync(m->sp_vxq.p, 0, (size_t)8 * nqe * sizeof(double), s));
  qcad_solver_opts ow = *o;
  ow.warm_start = 1;
  bool converged = false;
  int k = 0;
  std::vector<double> E(nev);
  try {
    for (k = 1; k <= max_iter; ++k) {
      // step (2): eigenpairs in V(phi^(k-1)) + V_xc
      qcad_solve_report er{};
      // the previous eigenvectors start the block from the second iteration on
      st = schrodinger_eigs_sp(m, b, phi, nev, m_eff, eig_tol, use_vxc ? m->sp_vxq.as<double>() : nullptr,
                               k > 1 ? m->sp_evecs.as<double>() : nullptr, E.data(), m->sp_evecs.as<double>(), &er);
      if (st != QCAD_OK) break;
      note_launch(), sp_tables_kernel<<<blocks_of(8 * nqe), SP_THREADS, 0, s>>>(
          G, nev, m->sp_evecs.as<double>(), ndof, phi, m->sp_w.as<double>(), m->sp_phiq.as<double>());
      QuantumDensity& qd = m->qd;
      qd = QuantumDensity{};
      qd.w = m->sp_w.as<double>();
      qd.phiq = m->sp_phiq.as<double>();
      for (int i = 0; i < nev; ++i) qd.E[i] = E[i];
      qd.nev = nev;
      qd.i0 = G.i0;
      qd.j0 = G.j0;
      qd.k0 = G.k0;
      qd.nx = G.nx;
      qd.ny = G.ny;
      qd.nz = G.nz;
      // step (3): Poisson with n~^(k) from phi^(k-1)
      CK(cudaMemcpyAsync(prev, phi, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      m->qd_active = true;
      st = poisson_solve(m, b, &ow, nullptr, phi, nullptr);
      if (st != QCAD_OK) break;
      CK(cudaMemsetAsync(acc, 0, 2 * sizeof(double), s));
      note_launch(), sp_density_kernel<<<blocks_of(8 * nqe), SP_THREADS, 0, s>>>(
          G, qd, phi, m->g64.g.hx, m->g64.g.hy, m->g64.g.hz, P.EF, P.inv_kT, use_vxc, pref, b3,
          m->sp_vxq.as<double>(), acc);
      // step (4)
      note_launch(), sp_maxdiff_kernel<<<std::min(blocks_of(n), 4 * 152), SP_THREADS, 0, s>>>(n, phi, prev, acc + 1);
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(m->h_small + 50, acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      const double dphi = m->h_small[51];
      r.n_quantum = m->h_small[50];
      r.dphi_inf = dphi;
      if (k <= QCAD_SP_HIST) {
        r.dphi_hist[k - 1] = dphi;
        r.e1_hist[k - 1] = E[0];
      }
      if (!std::isfinite(dphi)) {
        st = QCAD_ERR_NONFINITE;
        break;
      }
      if (tol_dphi > 0 && k >= 2 && dphi < tol_dphi) {
        converged = true;
        break;
      }
    }
  } catch (...) {
    m->qd_active = false;
    throw;
  }
  m->qd_active = false;
  for (int i = 0; i < nev; ++i) evals[i] = E[i];
  r.sp_iters = std::min(k, max_iter);
  r.converged = converged ? 1 : 0;
  r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (rep) *rep = r;
  if (st != QCAD_OK) return st;
  if (tol_dphi > 0 && !converged) {
    set_message("the Schrodinger-Poisson loop did not reach the potential tolerance");
    return QCAD_ERR_NOT_CONVERGED;
  }
  return QCAD_OK;
}

}  // namespace qcad
