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
struct Lobpcg {
  qcad_mesh_s* m;
  SubSetup* S;
  int nb;           // block size
  long long ns;
  double *Sx, *HS, *MS;  // [X | W | P] blocks, each ns x 3nb
  double* T;             // temporary ns x nb
  double* G;             // device gram buffer
  std::vector<double> hG;
  DevBuf tmp32;
  cudaStream_t s;

  double* X() { return Sx; }
  double* W() { return Sx + ns * nb; }
  double* P() { return Sx + 2 * ns * nb; }
  double* blk(double* base, int b) { return base + (long long)b * ns * nb; }

  // G = A^T B (p x q) to host.
  void gram(int p, int q, const double* A, const double* B, std::vector<double>& out) {
    CK(cudaMemsetAsync(G, 0, (size_t)p * q * sizeof(double), s));
    launch_gram(ns, p, q, A, ns, B, ns, G, s);
    out.resize((size_t)p * q);
    CK(cudaMemcpyAsync(out.data(), G, (size_t)p * q * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }

  // In-place A[:, 0:q] = A[:, 0:p] C for the three aligned blocks (S, HS, MS) at offset off.
  void combine3(int off_blk, int p, int q, const std::vector<double>& C, int dst_blk) {
    double* bases[3] = {Sx, HS, MS};
    DevBuf cbuf;
    cbuf.ensure((size_t)p * q * sizeof(double) + 64);
    CK(cudaMemcpyAsync(cbuf.p, C.data(), (size_t)p * q * sizeof(double), cudaMemcpyHostToDevice, s));
    for (int t = 0; t < 3; ++t) {
      launch_combine(ns, p, q, blk(bases[t], off_blk), ns, cbuf.as<double>(), T, ns, 0.0, s);
      CK(cudaMemcpyAsync(blk(bases[t], dst_blk), T, (size_t)ns * q * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    CK(cudaStreamSynchronize(s));
  }

  // M-orthonormalize block b (nb columns) by Cholesky QR; false if rank deficient.
  bool orthonormalize(int b) {
    std::vector<double> g;
    gram(nb, nb, blk(Sx, b), blk(MS, b), g);
    for (int j = 0; j < nb; ++j)
      for (int i = 0; i < j; ++i) {
        const double v = 0.5 * (g[(size_t)j * nb + i] + g[(size_t)i * nb + j]);
        g[(size_t)j * nb + i] = g[(size_t)i * nb + j] = v;
      }
    if (!dense_cholesky(nb, g.data())) return false;
    std::vector<double> R((size_t)nb * nb);
    dense_inv_lt(nb, g.data(), R.data());
    for (double v : R)
      if (!std::isfinite(v)) return false;
    combine3(b, nb, nb, R, b);
    return true;
  }
};

qcad_status schrodinger_eigs(qcad_mesh_s* m, const qcad_bias* b, const double* phi, int nev, const double* m_eff,
                             double tol, double* evals, double* evecs, qcad_solve_report* rep) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!b || !phi || !m_eff || !evals) throw Error(QCAD_ERR_INVALID_ARG, "null pointer");
  if (nev < 1 || nev > 16) throw Error(QCAD_ERR_INVALID_ARG, "nev must be in [1, 16]");
  if (!(tol > 0)) throw Error(QCAD_ERR_INVALID_ARG, "tol must be > 0");
  SubSetup S;
  setup_sub(m, b, phi, m_eff, 0, S);
  if (S.ndof < 3 * (nev + 4)) throw Error(QCAD_ERR_INVALID_ARG, "subdomain too small for nev");
  cudaStream_t s = m->stream;
  Lobpcg L;
  L.m = m;
  L.S = &S;
  L.nb = std::min<long long>(nev + std::max(2, nev / 4), S.ndof / 3);
  const int nb = L.nb;
  L.ns = S.ns;
  L.s = s;
  const long long ns = S.ns;
  DevBuf work;
  work.ensure((size_t)(3 * 3 * nb + nb) * ns * sizeof(double) + (size_t)9 * nb * nb * sizeof(double) + 256);
  L.Sx = work.as<double>();
  L.HS = L.Sx + 3 * nb * ns;
  L.MS = L.HS + 3 * nb * ns;
  L.T = L.MS + 3 * nb * ns;
  L.G = L.T + nb * ns;
  // random start on interior nodes, H and M of it, Rayleigh-Ritz
  launch_random_block(ns, nb, ns, S.interior.as<unsigned char>(), 0x51ED5EEDull, L.X(), s);
  hm_apply(m, S, 0, nb, L.X(), L.blk(L.HS, 0), L.blk(L.MS, 0), &L.tmp32);
  std::vector<double> GH, GM, w(3 * nb), C((size_t)9 * nb * nb);
  L.gram(nb, nb, L.X(), L.blk(L.HS, 0), GH);
  L.gram(nb, nb, L.X(), L.blk(L.MS, 0), GM);
  if (!dense_gen_eig(nb, GH.data(), GM.data(), w.data(), C.data()))
    throw Error(QCAD_ERR_NONFINITE, "initial Rayleigh-Ritz failed");
  L.combine3(0, nb, nb, std::vector<double>(C.begin(), C.begin() + (size_t)nb * nb), 0);
  std::vector<double> lam(w.begin(), w.begin() + nb);
  DevBuf lam_d, norms_d;
  lam_d.ensure(nb * sizeof(double) + 64);
  norms_d.ensure(2 * nb * sizeof(double) + 64);
  std::vector<double> norms(2 * nb);
  bool haveP = false;
  int it = 0, applies = nb;
  bool converged = false;
  const int maxit = 2000;
  std::vector<double> rel(nb, 1.0);
  for (it = 1; it <= maxit; ++it) {
    // residual block W = D^-1 (H X - M X Lambda) and its norms
    CK(cudaMemcpyAsync(lam_d.p, lam.data(), nb * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(norms_d.p, 0, 2 * nb * sizeof(double), s));
    launch_residual_block(ns, nb, L.blk(L.HS, 0), L.blk(L.MS, 0), ns, lam_d.as<double>(), S.dinv.as<double>(), L.W(),
                          norms_d.as<double>(), s);
    CK(cudaMemcpyAsync(norms.data(), norms_d.p, 2 * nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    bool all = true;
    for (int j = 0; j < nb; ++j) {
      const double scale = std::max(std::fabs(lam[j]), 1e-12) * std::sqrt(std::max(norms[2 * j + 1], 1e-300));
      rel[j] = std::sqrt(norms[2 * j]) / scale;
      if (j < nev && !(rel[j] <= tol)) all = false;
    }
    if (all) {
      converged = true;
      break;
    }
    // H W, M W; orthonormalize W against itself in the M inner product
    hm_apply(m, S, 0, nb, L.W(), L.blk(L.HS, 1), L.blk(L.MS, 1), &L.tmp32);
    applies += nb;
    if (!L.orthonormalize(1)) {
      // W numerically rank deficient: perturb with fresh random directions
      launch_random_block(ns, nb, ns, S.interior.as<unsigned char>(), 0xABCDEF00ull + it, L.W(), s);
      hm_apply(m, S, 0, nb, L.W(), L.blk(L.HS, 1), L.blk(L.MS, 1), &L.tmp32);
      applies += nb;
      if (!L.orthonormalize(1)) throw Error(QCAD_ERR_NONFINITE, "LOBPCG: W block lost rank");
    }
    if (haveP && !L.orthonormalize(2)) haveP = false;
    const int nbas = haveP ? 3 * nb : 2 * nb;
    L.gram(nbas, nbas, L.Sx, L.HS, GH);
    L.gram(nbas, nbas, L.Sx, L.MS, GM);
    w.resize(nbas);
    C.resize((size_t)nbas * nbas);
    bool ok = dense_gen_eig(nbas, GH.data(), GM.data(), w.data(), C.data());
    if (!ok && haveP) {
      haveP = false;
      const int n2 = 2 * nb;
      std::vector<double> gh2((size_t)n2 * n2), gm2((size_t)n2 * n2);
      for (int j = 0; j < n2; ++j)
        for (int i = 0; i < n2; ++i) {
          gh2[(size_t)j * n2 + i] = GH[(size_t)j * nbas + i];
          gm2[(size_t)j * n2 + i] = GM[(size_t)j * nbas + i];
        }
      w.resize(n2);
      C.resize((size_t)n2 * n2);
      ok = dense_gen_eig(n2, gh2.data(), gm2.data(), w.data(), C.data());
      if (!ok) throw Error(QCAD_ERR_NONFINITE, "LOBPCG Rayleigh-Ritz failed");
    }
    const int nuse = haveP ? 3 * nb : 2 * nb;
    // new P = [W P] C[nb:, :nb]; new X = [X W P] C[:, :nb]
    std::vector<double> Cx((size_t)nuse * nb), Cp((size_t)(nuse - nb) * nb);
    for (int j = 0; j < nb; ++j) {
      for (int i = 0; i < nuse; ++i) Cx[(size_t)j * nuse + i] = C[(size_t)j * nuse + i];
      for (int i = nb; i < nuse; ++i) Cp[(size_t)j * (nuse - nb) + (i - nb)] = C[(size_t)j * nuse + i];
    }
    L.combine3(1, nuse - nb, nb, Cp, 2);  // reads W (and old P) blocks, writes P
    // X update must read the old P: recombine it from the stored (unchanged) blocks before P was overwritten.
    // combine3 wrote P after reading [W, P_old]; rebuild X from X, W and (P_new - W Cw) is avoided by
    // computing X as X C_X + P_new, since P_new = [W P_old] C[nb:, :nb].
    {
      std::vector<double> Cxx((size_t)nb * nb);
      for (int j = 0; j < nb; ++j)
        for (int i = 0; i < nb; ++i) Cxx[(size_t)j * nb + i] = C[(size_t)j * nuse + i];
      DevBuf cbuf;
      cbuf.ensure((size_t)nb * nb * sizeof(double) + 64);
      CK(cudaMemcpyAsync(cbuf.p, Cxx.data(), (size_t)nb * nb * sizeof(double), cudaMemcpyHostToDevice, s));
      double* bases[3] = {L.Sx, L.HS, L.MS};
      for (int t = 0; t < 3; ++t) {
        // T = X C_X ; X = T + P_new
        launch_combine(ns, nb, nb, L.blk(bases[t], 0), ns, cbuf.as<double>(), L.T, ns, 0.0, s);
        CK(cudaMemcpyAsync(L.blk(bases[t], 0), L.T, (size_t)ns * nb * sizeof(double), cudaMemcpyDeviceToDevice, s));
        std::vector<double> I((size_t)nb * nb, 0.0);
        for (int q = 0; q < nb; ++q) I[(size_t)q * nb + q] = 1.0;
        DevBuf ibuf;
        ibuf.ensure((size_t)nb * nb * sizeof(double) + 64);
        CK(cudaMemcpyAsync(ibuf.p, I.data(), (size_t)nb * nb * sizeof(double), cudaMemcpyHostToDevice, s));
        launch_combine(ns, nb, nb, L.blk(bases[t], 2), ns, ibuf.as<double>(), L.blk(bases[t], 0), ns, 1.0, s);
        CK(cudaStreamSynchronize(s));
      }
    }
    haveP = true;
    lam.assign(w.begin(), w.begin() + nb);
    // periodically refresh H X and M X to stop drift of the recurrences
    if (it % 25 == 0) {
      hm_apply(m, S, 0, nb, L.X(), L.blk(L.HS, 0), L.blk(L.MS, 0), &L.tmp32);
      applies += nb;
    }
  }
  // final Rayleigh-Ritz on X with fresh applies (FP64)
  hm_apply(m, S, 0, nb, L.X(), L.blk(L.HS, 0), L.blk(L.MS, 0), &L.tmp32);
  applies += nb;
  L.gram(nb, nb, L.X(), L.blk(L.HS, 0), GH);
  L.gram(nb, nb, L.X(), L.blk(L.MS, 0), GM);
  w.resize(nb);
  C.resize((size_t)nb * nb);
  if (!dense_gen_eig(nb, GH.data(), GM.data(), w.data(), C.data()))
    throw Error(QCAD_ERR_NONFINITE, "final Rayleigh-Ritz failed");
  L.combine3(0, nb, nb, C, 0);
  for (int j = 0; j < nev; ++j) evals[j] = w[j];
  if (evecs) launch_pack(S.sm, nev, L.X(), ns, evecs, S.ndof, 0, s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  if (m->prof.on) m->prof.harvest();
  if (rep) {
    rep->newton_iters = 0;
    rep->krylov_iters_total = it;
    rep->applies_total = applies;
    double worst = 0;
    for (int j = 0; j < nev; ++j) worst = std::max(worst, rel[j]);
    rep->final_res_inf = worst;
    rep->final_dphi_inf = 0;
    rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    rep->status_detail = 0;
  }
  return converged ? QCAD_OK : QCAD_ERR_NOT_CONVERGED;
}

}  // namespace qcad
