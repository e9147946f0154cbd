// Schrodinger operators on the quantum subdomain and the LOBPCG eigensolver
// (Sec. II.B: H psi = E M psi from the weak form Eq. SchrodEqnWeakForm; the
// paper solves it with a Trilinos/Anasazi eigensolver).
//
// LOBPCG (Knyazev's locally optimal block preconditioned CG): the search
// space [X, W, P] with W the Jacobi-preconditioned residual block and P the
// previous step direction; W and P are M-orthonormalized by Cholesky QR before
// the Rayleigh-Ritz step, whose small generalized problem is solved in FP64
// on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "mesh.h"

namespace qcad {

Phys make_phys(const qcad_mesh_s* m, const qcad_bias* b);
GridTables make_tables(const std::vector<double>& x, const std::vector<double>& y, const std::vector<double>& z,
                       const std::vector<double>& kx_layer, const std::vector<double>& ky_layer,
                       const std::vector<double>& kz_layer);
template <class T>
void build_grid(GridDev<T>& gd, const GridTables& t, const std::vector<double>& hx, const std::vector<double>& hy,
                const std::vector<double>& hz, cudaStream_t s);
double host_h2m0();
void set_message(const std::string& msg);

struct SubSetup {
  SubdomainMap sm;
  long long ns;     // subdomain nodes
  long long ndof;   // interior nodes
  GridDev<double> g64;
  GridDev<float> g32;
  DevBuf cV64, cV32, dinv, interior;
  double vmin;
};

static void setup_sub(qcad_mesh_s* m, const qcad_bias* b, const double* phi, const double* m_eff, int need32,
                      SubSetup& S) {
  if (!m->has_sub) throw Error(QCAD_ERR_INVALID_ARG, "mesh has no Schrodinger subdomain");
  for (int d = 0; d < 3; ++d)
    if (!(m_eff[d] > 0)) throw Error(QCAD_ERR_INVALID_ARG, "effective masses must be > 0");
  cudaStream_t s = m->stream;
  SubdomainMap& sm = S.sm;
  sm.i0 = m->sub[0];
  sm.j0 = m->sub[2];
  sm.k0 = m->sub[4];
  sm.nxs = m->sub[1] - m->sub[0];
  sm.nys = m->sub[3] - m->sub[2];
  sm.nzs = m->sub[5] - m->sub[4];
  sm.nxn = m->nxn;
  sm.nyn = m->nyn;
  S.ns = (long long)(sm.nxs + 1) * (sm.nys + 1) * (sm.nzs + 1);
  S.ndof = (long long)(sm.nxs - 1) * (sm.nys - 1) * (sm.nzs - 1);
  std::vector<double> xs(m->xc.begin() + sm.i0, m->xc.begin() + sm.i0 + sm.nxs + 1);
  std::vector<double> ys(m->yc.begin() + sm.j0, m->yc.begin() + sm.j0 + sm.nys + 1);
  std::vector<double> zs(m->zc.begin() + sm.k0, m->zc.begin() + sm.k0 + sm.nzs + 1);
  std::vector<double> hx(m->hxv.begin() + sm.i0, m->hxv.begin() + sm.i0 + sm.nxs);
  std::vector<double> hy(m->hyv.begin() + sm.j0, m->hyv.begin() + sm.j0 + sm.nys);
  std::vector<double> hz(m->hzv.begin() + sm.k0, m->hzv.begin() + sm.k0 + sm.nzs);
  const double h2m = host_h2m0();
  // kinetic coefficients hbar^2 / (2 m_d) for each direction (Eq. Schrodinger3D)
  std::vector<double> kx(sm.nzs, h2m / m_eff[0]), ky(sm.nzs, h2m / m_eff[1]), kz(sm.nzs, h2m / m_eff[2]);
  GridTables t = make_tables(xs, ys, zs, kx, ky, kz);
  build_grid<double>(S.g64, t, hx, hy, hz, s);
  S.g64.g.dir_boundary = 1;
  S.g64.g.dir_bottom = 0;
  S.g64.g.dir_top = nullptr;
  if (need32) {
    build_grid<float>(S.g32, t, hx, hy, hz, s);
    S.g32.g.dir_boundary = 1;
    S.g32.g.dir_bottom = 0;
    S.g32.g.dir_top = nullptr;
  }
  // potential energy at the qp: V = q phi_ref - chi - q phi (Eq. SchrodPotEnergy, no V_xc)
  const Phys P = make_phys(m, b);
  const long long nes = (long long)sm.nxs * sm.nys * sm.nzs;
  S.cV64.ensure(nes * 8 * sizeof(double) + 64);
  double* vmin_d = m->stats.as<double>() + 40;
  const double big = 1e300;
  CK(cudaMemcpyAsync(vmin_d, &big, sizeof(double), cudaMemcpyHostToDevice, s));
  launch_potential<double>(sm, phi, P.phi_ref - P.chi, m->g64.g.hx, m->g64.g.hy, m->g64.g.hz,
                           S.cV64.as<double>(), vmin_d, s);
  if (need32) {
    S.cV32.ensure(nes * 8 * sizeof(float) + 64);
    launch_potential<float>(sm, phi, P.phi_ref - P.chi, m->g64.g.hx, m->g64.g.hy, m->g64.g.hz, S.cV32.as<float>(),
                            vmin_d, s);
  }
  CK(cudaGetLastError());
  double vmin_shift = 0;
  CK(cudaMemcpyAsync(&vmin_shift, vmin_d, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  S.vmin = vmin_shift - 100.0;
  // Jacobi preconditioner from the kinetic diagonal, interior mask
  std::vector<double> dinv(S.ns, 0.0);
  std::vector<unsigned char> inter(S.ns, 0);
  const int nxn = sm.nxs + 1, nyn = sm.nys + 1;
  for (int k = 1; k < sm.nzs; ++k)
    for (int j = 1; j < sm.nys; ++j)
      for (int i = 1; i < sm.nxs; ++i) {
        const long long n = i + (long long)nxn * (j + (long long)nyn * k);
        const double d = t.kx[3 * i + 1] * t.my[3 * j + 1] * t.mzx[3 * k + 1] +
                         t.mx[3 * i + 1] * t.ky[3 * j + 1] * t.mzy[3 * k + 1] +
                         t.mx[3 * i + 1] * t.my[3 * j + 1] * t.kzz[3 * k + 1];
        dinv[n] = 1.0 / d;
        inter[n] = 1;
      }
  S.dinv.ensure(S.ns * sizeof(double) + 64);
  S.interior.ensure(S.ns + 64);
  CK(cudaMemcpyAsync(S.dinv.p, dinv.data(), S.ns * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(S.interior.p, inter.data(), S.ns, cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
}

static void hm_apply(qcad_mesh_s* m, SubSetup& S, int prec, int nvec, const double* X, double* HX, double* MX,
                     DevBuf* tmp32) {
  cudaStream_t s = m->stream;
  Profiler::Pair pp;
  if (prec == 0) {
    HmArgs<double> a{};
    a.x = X;
    a.hx = HX;
    a.mx = MX;
    a.cV = S.cV64.as<double>();
    a.ld = S.ns;
    a.nvec = nvec;
    if (m->prof.on) m->prof.begin(PROF_HM, s, pp);
    launch_hm_apply<double>(S.g64.g, a, LaunchCfg{8, 16}, s);
    if (m->prof.on) m->prof.end(pp, s);
  } else {
    const long long tot = S.ns * nvec;
    tmp32->ensure(3 * tot * sizeof(float) + 64);
    float* x32 = tmp32->as<float>();
    float* h32 = x32 + tot;
    float* m32 = h32 + tot;
    launch_d2f(tot, X, x32, s);
    HmArgs<float> a{};
    a.x = x32;
    a.hx = HX ? h32 : nullptr;
    a.mx = MX ? m32 : nullptr;
    a.cV = S.cV32.as<float>();
    a.ld = S.ns;
    a.nvec = nvec;
    if (m->prof.on) m->prof.begin(PROF_HM, s, pp);
    launch_hm_apply<float>(S.g32.g, a, LaunchCfg{8, 16}, s);
    if (m->prof.on) m->prof.end(pp, s);
    if (HX) launch_f2d(tot, h32, HX, s);
    if (MX) launch_f2d(tot, m32, MX, s);
  }
  CK(cudaGetLastError());
}

qcad_status schrodinger_apply(qcad_mesh_s* m, const qcad_bias* b, const double* phi, const double* m_eff, int nvec,
                              const double* X, double* HX, double* MX, int precision) {
  if (!b || !phi || !m_eff || !X || nvec < 1) throw Error(QCAD_ERR_INVALID_ARG, "null pointer or nvec < 1");
  if (precision != 0 && precision != 1) throw Error(QCAD_ERR_INVALID_ARG, "precision must be 0 or 1");
  SubSetup S;
  setup_sub(m, b, phi, m_eff, precision, S);
  cudaStream_t s = m->stream;
  DevBuf full, tmp;
  full.ensure(3 * S.ns * nvec * sizeof(double) + 64);
  double* xf = full.as<double>();
  double* hf = xf + S.ns * nvec;
  double* mf = hf + S.ns * nvec;
  CK(cudaMemsetAsync(xf, 0, S.ns * nvec * sizeof(double), s));
  launch_pack(S.sm, nvec, xf, S.ns, const_cast<double*>(X), S.ndof, 1, s);
  hm_apply(m, S, precision, nvec, xf, HX ? hf : nullptr, MX ? mf : nullptr, &tmp);
  if (HX) launch_pack(S.sm, nvec, hf, S.ns, HX, S.ndof, 0, s);
  if (MX) launch_pack(S.sm, nvec, mf, S.ns, MX, S.ndof, 0, s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  if (m->prof.on) m->prof.harvest();
  return QCAD_OK;
}

// ---------------------------------------------------------------------------
// One LOBPCG run in storage/apply precision T (FP32 for the iteration phase,
// FP64 to polish). The blocks S = [X | W | P], HS = H S, MS = M S are kept
// together (column-major, ns x 3nb each) so that the Rayleigh-Ritz Gram
// matrices are two kernel launches; all block updates are row-wise in place.
template <class T>
struct LobpcgRun {
  qcad_mesh_s* m;
  SubSetup* S;
  cudaStream_t s;
  int nb, nev;
  long long ns;
  T* Sx;
  T* HS;
  T* MS;
  const T* dinv;
  double* G;
  T* Cd;  // device combination coefficients
  std::vector<double> lam;
  std::vector<double> rel;
  int applies = 0;
  int iters = 0;
  DevBuf tmp32;

  T* blk(T* base, int b) { return base + (long long)b * ns * nb; }

  void apply(int b) {
    HmArgs<T> a{};
    a.x = blk(Sx, b);
    a.hx = blk(HS, b);
    a.mx = blk(MS, b);
    a.cV = cv();
    a.ld = ns;
    a.nvec = nb;
    Profiler::Pair pp;
    if (m->prof.on) m->prof.begin(PROF_HM, s, pp);
    launch_hm_apply<T>(grid(), a, LaunchCfg{8, 16}, s);
    if (m->prof.on) m->prof.end(pp, s);
    applies += nb;
  }
  const T* cv();
  const Grid<T>& grid();

  void gram(int p, int q, const T* A, const T* B, std::vector<double>& out) {
    CK(cudaMemsetAsync(G, 0, (size_t)p * q * sizeof(double), s));
    launch_gram<T>(ns, p, q, A, ns, B, ns, G, s);
    out.resize((size_t)p * q);
    CK(cudaMemcpyAsync(out.data(), G, (size_t)p * q * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int j = 0; j < q && p == q; ++j)
      for (int i = 0; i < j; ++i) {
        const double v = 0.5 * (out[(size_t)j * p + i] + out[(size_t)i * p + j]);
        out[(size_t)j * p + i] = out[(size_t)i * p + j] = v;
      }
  }

  // For S, HS and MS: columns [src, src+p) times C (p x q); output columns < q1 to block dst1,
  // the rest to block dst2 (in place).
  void combine(int src_blk, int p, const std::vector<double>& C, int q, int q1, int dst1, int dst2) {
    std::vector<T> ct(C.begin(), C.end());
    CK(cudaMemcpyAsync(Cd, ct.data(), ct.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    T* bases[3] = {Sx, HS, MS};
    for (T* base : bases)
      launch_combine<T>(ns, p, q, q1, blk(base, src_blk), ns, Cd, blk(base, dst1), blk(base, dst2), ns, s);
    CK(cudaStreamSynchronize(s));  // ct must outlive the pageable copy
  }

  bool orthonormalize(int b) {
    std::vector<double> g;
    gram(nb, nb, blk(Sx, b), blk(MS, b), g);
    if (!dense_cholesky(nb, g.data())) return false;
    std::vector<double> R((size_t)nb * nb);
    dense_inv_lt(nb, g.data(), R.data());
    for (double v : R)
      if (!std::isfinite(v)) return false;
    combine(b, nb, R, nb, nb, b, b);
    return true;
  }

  // Rayleigh-Ritz on block 0 alone.
  void rr_x() {
    std::vector<double> GH, GM, w(nb), C((size_t)nb * nb);
    gram(nb, nb, blk(Sx, 0), blk(HS, 0), GH);
    gram(nb, nb, blk(Sx, 0), blk(MS, 0), GM);
    if (!dense_gen_eig(nb, GH.data(), GM.data(), w.data(), C.data()))
      throw Error(QCAD_ERR_NONFINITE, "LOBPCG: Rayleigh-Ritz on X failed");
    combine(0, nb, C, nb, nb, 0, 0);
    lam.assign(w.begin(), w.end());
  }

  // Iterates until the first nev relative residuals are <= tol; returns true when converged.
  bool run(double tol, int maxit, DevBuf& lam_d, DevBuf& norms_d) {
    bool haveP = false;
    std::vector<double> norms(2 * nb), GH, GM, w, C;
    rel.assign(nb, 1.0);
    for (int it = 1; it <= maxit; ++it) {
      CK(cudaMemcpyAsync(lam_d.p, lam.data(), nb * sizeof(double), cudaMemcpyHostToDevice, s));
      CK(cudaMemsetAsync(norms_d.p, 0, 2 * nb * sizeof(double), s));
      launch_residual_block<T>(ns, nb, blk(HS, 0), blk(MS, 0), ns, lam_d.as<double>(), dinv, blk(Sx, 1),
                               norms_d.as<double>(), s);
      CK(cudaMemcpyAsync(norms.data(), norms_d.p, 2 * nb * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      bool all = true;
      for (int j = 0; j < nb; ++j) {
        const double scale = std::max(std::fabs(lam[j]), 1e-12) * std::sqrt(std::max(norms[2 * j + 1], 1e-300));
        rel[j] = std::sqrt(norms[2 * j]) / scale;
        if (j < nev && !(rel[j] <= tol)) all = false;
      }
      if (all) return true;
      ++iters;
      apply(1);
      if (!orthonormalize(1)) {
        launch_random_block<T>(ns, nb, ns, S->interior.as<unsigned char>(), 0xABCDEF00ull + iters, blk(Sx, 1), s);
        apply(1);
        if (!orthonormalize(1)) throw Error(QCAD_ERR_NONFINITE, "LOBPCG: W block lost rank");
      }
      if (haveP && !orthonormalize(2)) haveP = false;
      int nuse = haveP ? 3 * nb : 2 * nb;
      gram(nuse, nuse, Sx, HS, GH);
      gram(nuse, nuse, Sx, MS, GM);
      w.resize(nuse);
      C.resize((size_t)nuse * nuse);
      bool ok = dense_gen_eig(nuse, GH.data(), GM.data(), w.data(), C.data());
      if (!ok && haveP) {
        haveP = false;
        const int n2 = 2 * nb;
        std::vector<double> gh2((size_t)n2 * n2), gm2((size_t)n2 * n2);
        for (int j = 0; j < n2; ++j)
          for (int i = 0; i < n2; ++i) {
            gh2[(size_t)j * n2 + i] = GH[(size_t)j * nuse + i];
            gm2[(size_t)j * n2 + i] = GM[(size_t)j * nuse + i];
          }
        nuse = n2;
        w.resize(nuse);
        C.resize((size_t)nuse * nuse);
        ok = dense_gen_eig(nuse, gh2.data(), gm2.data(), w.data(), C.data());
      }
      if (!ok) throw Error(QCAD_ERR_NONFINITE, "LOBPCG Rayleigh-Ritz failed");
      // new X = [X W P] C[:, :nb];  new P = [W P] C[nb:, :nb] = [X W P] (C[:, :nb] with the X rows zeroed)
      std::vector<double> Cxp((size_t)nuse * 2 * nb, 0.0);
      for (int j = 0; j < nb; ++j)
        for (int i = 0; i < nuse; ++i) {
          Cxp[(size_t)j * nuse + i] = C[(size_t)j * nuse + i];
          Cxp[(size_t)(nb + j) * nuse + i] = i < nb ? 0.0 : C[(size_t)j * nuse + i];
        }
      combine(0, nuse, Cxp, 2 * nb, nb, 0, 2);
      haveP = true;
      lam.assign(w.begin(), w.begin() + nb);
      if (iters % 25 == 0) apply(0);  // refresh H X, M X against recurrence drift
    }
    return false;
  }
};

template <> const double* LobpcgRun<double>::cv() { return S->cV64.as<double>(); }
template <> const float* LobpcgRun<float>::cv() { return S->cV32.as<float>(); }
template <> const Grid<double>& LobpcgRun<double>::grid() { return S->g64.g; }
template <> const Grid<float>& LobpcgRun<float>::grid() { return S->g32.g; }

template <class T>
static void init_run(LobpcgRun<T>& L, qcad_mesh_s* m, SubSetup* S, int nb, int nev, DevBuf& work, const T* dinv) {
  L.m = m;
  L.S = S;
  L.s = m->stream;
  L.nb = nb;
  L.nev = nev;
  L.ns = S->ns;
  const long long ns = S->ns;
  work.ensure((size_t)9 * nb * ns * sizeof(T) + (size_t)9 * nb * nb * (sizeof(double) + 2 * sizeof(T)) + 1024);
  L.Sx = work.as<T>();
  L.HS = L.Sx + 3 * nb * ns;
  L.MS = L.HS + 3 * nb * ns;
  unsigned char* tail = reinterpret_cast<unsigned char*>(L.MS + 3 * nb * ns);
  tail = reinterpret_cast<unsigned char*>(((uintptr_t)tail + 255) & ~(uintptr_t)255);
  L.G = reinterpret_cast<double*>(tail);
  L.Cd = reinterpret_cast<T*>(tail + (size_t)9 * nb * nb * sizeof(double) + 256);
  L.dinv = dinv;
}

qcad_status schrodinger_eigs(qcad_mesh_s* m, const qcad_bias* b, const double* phi, int nev, const double* m_eff,
                             double tol, double* evals, double* evecs, qcad_solve_report* rep) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!b || !phi || !m_eff || !evals) throw Error(QCAD_ERR_INVALID_ARG, "null pointer");
  if (nev < 1 || nev > 16) throw Error(QCAD_ERR_INVALID_ARG, "nev must be in [1, 16]");
  if (!(tol > 0)) throw Error(QCAD_ERR_INVALID_ARG, "tol must be > 0");
  SubSetup S;
  setup_sub(m, b, phi, m_eff, 1, S);
  if (S.ndof < 3 * (nev + 4)) throw Error(QCAD_ERR_INVALID_ARG, "subdomain too small for nev");
  cudaStream_t s = m->stream;
  const int nb = (int)std::min<long long>(nev + std::max(2, nev / 4), S.ndof / 3);
  const long long ns = S.ns;
  DevBuf lam_d, norms_d, dinv32;
  lam_d.ensure(nb * sizeof(double) + 64);
  norms_d.ensure(2 * nb * sizeof(double) + 64);
  dinv32.ensure(ns * sizeof(float) + 64);
  launch_d2f(ns, S.dinv.as<double>(), dinv32.as<float>(), s);

  // Phase 1: FP32 storage, applies and block arithmetic (FP64 Gram accumulation and host
  // Rayleigh-Ritz) until the residuals reach the single-precision level.
  DevBuf w32, w64;
  LobpcgRun<float> A;
  init_run<float>(A, m, &S, nb, nev, w32, dinv32.as<float>());
  launch_random_block<float>(ns, nb, ns, S.interior.as<unsigned char>(), 0x51ED5EEDull, A.Sx, s);
  A.apply(0);
  A.rr_x();
  const double tol32 = std::max(tol, 1e-5);
  A.run(tol32, 3000, lam_d, norms_d);

  // Phase 2: FP64 from the FP32 Ritz vectors to the requested tolerance.
  LobpcgRun<double> B;
  init_run<double>(B, m, &S, nb, nev, w64, S.dinv.as<double>());
  launch_f2d(ns * nb, A.Sx, B.Sx, s);
  B.apply(0);
  B.rr_x();
  bool converged = B.run(tol, 500, lam_d, norms_d);
  // final Rayleigh-Ritz with fresh FP64 applies
  B.apply(0);
  B.rr_x();
  for (int j = 0; j < nev; ++j) evals[j] = B.lam[j];
  if (evecs) launch_pack(S.sm, nev, B.Sx, ns, evecs, S.ndof, 0, s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  if (m->prof.on) m->prof.harvest();
  if (rep) {
    rep->newton_iters = A.iters;  // FP32-phase iterations
    rep->krylov_iters_total = A.iters + B.iters;
    rep->applies_total = A.applies + B.applies;
    double worst = 0;
    for (int j = 0; j < nev; ++j) worst = std::max(worst, B.rel[j]);
    rep->final_res_inf = worst;
    rep->final_dphi_inf = 0;
    rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    rep->status_detail = B.iters;  // FP64-phase iterations
  }
  if (!converged) set_message("LOBPCG did not reach the requested tolerance");
  return converged ? QCAD_OK : QCAD_ERR_NOT_CONVERGED;
}

}  // namespace qcad
