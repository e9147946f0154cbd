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
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "dfloat.cuh"
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

// Stream and scratch of one eigensolve: the mesh's own, or a second set so that an
// eigensolve can run concurrently with another call on the mesh stream.
struct EigIo {
  cudaStream_t s;
  double* stats;    // device scratch, >= 64 doubles
  double* h_small;  // pinned host scratch, >= 64 doubles
};
static EigIo mesh_io(qcad_mesh_s* m) { return EigIo{m->stream, m->stats.as<double>(), m->h_small}; }

static int debug_level() {
  static const int lvl = std::getenv("QCAD_DEBUG") ? std::max(1, std::atoi(std::getenv("QCAD_DEBUG"))) : 0;
  return lvl;
}

struct SubSetup {
  SubdomainMap sm;
  long long ns;     // subdomain nodes
  long long ndof;   // interior nodes
  GridDev<double> g64;
  GridDev<float> g32;
  GridDev<dfl> gdf;  // double-float tables: the FP64 phase's H and M applies
  DevBuf cV64, cV32, dinv, interior;
  double vmin;
  double inv_kx;    // 1 / kappa_x = 2 m_x / hbar^2 (scale of the separable mass stencil)
  double shift = 0.0;  // constant added to the potential (eV)
};

// vxq: an extra potential energy at the subdomain's Gauss points (eV, [element][point]) or null;
// shift_floor > 0: the whole potential is raised by the constant that brings its minimum to
// shift_floor (returned in S.shift, subtracted from the eigenvalues), so that every eigenvalue
// stays well away from zero for the relative residual test.
static void setup_sub(qcad_mesh_s* m, const qcad_bias* b, const double* phi, const double* m_eff, int need32,
                      SubSetup& S, const EigIo& io, const double* vxq = nullptr, double shift_floor = 0.0) {
  if (!m->has_sub) throw Error(QCAD_ERR_INVALID_ARG, "mesh has no Schrodinger subdomain");
  for (int d = 0; d < 3; ++d)
    if (!(m_eff[d] > 0)) throw Error(QCAD_ERR_INVALID_ARG, "effective masses must be > 0");
  cudaStream_t s = io.s;
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
  S.inv_kx = m_eff[0] / h2m;
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
    build_grid<dfl>(S.gdf, t, hx, hy, hz, s);
    S.gdf.g.dir_boundary = 1;
    S.gdf.g.dir_bottom = 0;
    S.gdf.g.dir_top = nullptr;
  }
  // potential energy at the qp: V = q phi_ref - chi - q phi (Eq. SchrodPotEnergy, no V_xc)
  const Phys P = make_phys(m, b);
  const long long nes = (long long)sm.nxs * sm.nys * sm.nzs;
  S.cV64.ensure(nes * 8 * sizeof(double) + 64);
  double* vmin_d = io.stats + 40;
  const double big = 1e300;
  CK(cudaMemcpyAsync(vmin_d, &big, sizeof(double), cudaMemcpyHostToDevice, s));
  auto potentials = [&](double V0) {
    CK(cudaMemcpyAsync(vmin_d, &big, sizeof(double), cudaMemcpyHostToDevice, s));
    launch_potential<double>(sm, phi, V0, m->g64.g.hx, m->g64.g.hy, m->g64.g.hz, vxq, S.cV64.as<double>(), vmin_d,
                             s);
    if (need32) {
      S.cV32.ensure(nes * 8 * sizeof(float) + 64);
      launch_potential<float>(sm, phi, V0, m->g64.g.hx, m->g64.g.hy, m->g64.g.hz, vxq, S.cV32.as<float>(), vmin_d,
                              s);
    }
    CK(cudaGetLastError());
    double vmin_shift = 0;
    CK(cudaMemcpyAsync(&vmin_shift, vmin_d, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    S.vmin = vmin_shift - 100.0;
  };
  potentials(P.phi_ref - P.chi);
  S.shift = 0.0;
  if (shift_floor > 0.0 && S.vmin < shift_floor) {
    S.shift = shift_floor - S.vmin;
    potentials(P.phi_ref - P.chi + S.shift);
  }
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
    a.mscale = S.inv_kx;
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
    a.mscale = S.inv_kx;
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
  setup_sub(m, b, phi, m_eff, precision, S, mesh_io(m));
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
// Chebyshev-Jacobi preconditioner of the LOBPCG residual block, applied in FP32 in both
// phases (a preconditioner needs no more precision than that): W = p_k(D^-1 H) D^-1 R with
// the Chebyshev polynomial of the interval [b / (4k^2), b] of D^-1 H, b = 1.1 lambda_max
// (power iteration). The degree is odd, so the preconditioner stays positive definite above
// an underestimated lambda_max. k <= 1 means plain Jacobi.
struct ChebPre {
  int k = 0;
  double theta = 0.0, delta = 0.0, lam_max = 0.0;
  qcad_mesh_s* m = nullptr;
  SubSetup* S = nullptr;
  int nb = 0;
  long long ns = 0;
  DevBuf buf;
  float *R32 = nullptr, *W = nullptr, *D = nullptr, *HD = nullptr;
  const float* dinv = nullptr;
  EigIo io{};

  void hmul(const float* X, float* HX, int nvec) {
    HmArgs<float> a{};
    a.x = X;
    a.hx = HX;
    a.mx = nullptr;
    a.cV = S->cV32.as<float>();
    a.ld = ns;
    a.nvec = nvec;
    a.mscale = S->inv_kx;
    launch_hm_apply<float>(S->g32.g, a, LaunchCfg{8, 16}, io.s);
  }
  void init(qcad_mesh_s* m_, const EigIo& io_, SubSetup* S_, int nb_, int k_, const float* dinv32) {
    m = m_;
    io = io_;
    S = S_;
    nb = nb_;
    ns = S->ns;
    k = k_;
    dinv = dinv32;
    if (k < 2) return;
    buf.ensure((size_t)4 * nb * ns * sizeof(float) + 256);
    R32 = buf.as<float>();
    W = R32 + nb * ns;
    D = W + nb * ns;
    HD = D + nb * ns;
    cudaStream_t s = io.s;
    // largest eigenvalue of D^-1 H by power iteration on one vector (uses W and D as scratch)
    launch_random_block<float>(ns, 1, ns, S->interior.as<unsigned char>(), 0xC4EB5EEDull, W, s);
    double* acc = io.stats + 48;
    double lam = 0.0;
    for (int it = 0; it < 12; ++it) {
      hmul(W, HD, 1);
      CK(cudaMemsetAsync(acc, 0, 3 * sizeof(double), s));
      launch_power_sub<float>(ns, W, HD, dinv, D, acc, s);
      CK(cudaMemcpyAsync(io.h_small + 40, acc, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      const double a0 = io.h_small[40], a1 = io.h_small[41], a2 = io.h_small[42];
      if (!(a1 > 0.0) || !(a2 > 0.0)) break;
      lam = a0 / a1;
      launch_scale<float>(ns, D, 1.0 / std::sqrt(a2), s);
      std::swap(W, D);
    }
    if (!(lam > 0.0)) {
      k = 0;
      return;
    }
    lam_max = lam;
    set_degree(k);
  }
  // Polynomial degree k >= 2 on the interval [b / 4k^2, b], b = 1.1 lambda_max.
  void set_degree(int k_) {
    if (!(lam_max > 0.0) || k_ < 2) return;
    k = k_;
    const double b = 1.1 * lam_max, a = b / (4.0 * k * k);
    theta = 0.5 * (a + b);
    delta = 0.5 * (b - a);
  }
  // Z = p_k(D^-1 H) D^-1 R for nvec <= nb columns (Z may alias R). Each step's H apply carries
  // the recurrence in its epilogue, the direction block alternating between D and HD.
  void apply(const float* R, float* Z, int nvec) {
    cudaStream_t s = io.s;
    launch_cheb_block_init<float>(ns, nvec, ns, R, dinv, 1.0 / theta, W, D, Z, s);
    const double sigma = theta / delta;
    double rho_prev = 1.0 / sigma, rho = rho_prev;
    float *dcur = D, *dnext = HD;
    for (int j = 1; j < k; ++j) {
      rho_prev = rho;
      rho = 1.0 / (2.0 * sigma - rho_prev);
      ChebHmArgs a{};
      a.din = dcur;
      a.dout = dnext;
      a.w = W;
      a.z = Z;
      a.dinv = dinv;
      a.cV = S->cV32.as<float>();
      a.ld = ns;
      a.nvec = nvec;
      a.c1 = (float)(rho * rho_prev);
      a.c2 = (float)(2.0 * rho / delta);
      launch_cheb_hm_step(S->g32.g, a, s);
      std::swap(dcur, dnext);
    }
  }
};

// FP32 preconditioning of nvec residual columns (ns rows each) stored in precision T.
static void precondition_block(ChebPre& P, float* Rb, int nvec) { P.apply(Rb, Rb, nvec); }
static void precondition_block(ChebPre& P, double* Rb, int nvec) {
  const long long tot = P.ns * nvec;
  launch_d2f(tot, Rb, P.R32, P.io.s);
  P.apply(P.R32, P.R32, nvec);
  launch_f2d(tot, P.R32, Rb, P.io.s);
}

// One LOBPCG run in storage/apply precision T (FP32 for the iteration phase,
// FP64 to polish). The blocks S = [X | W | P], HS = H S, MS = M S are kept
// together (column-major, ns x 3nb each) so that the Rayleigh-Ritz Gram
// matrices of H and M are one kernel launch; all block updates are row-wise
// in place. An iteration synchronizes with the host twice: after the residual
// norms of the Ritz pairs (which decide convergence and the active columns)
// and after the Rayleigh-Ritz Gram matrices. Small matrices travel through
// pinned host buffers, so the block combinations need no wait.
template <class T>
struct LobpcgRun {
  qcad_mesh_s* m = nullptr;
  SubSetup* S = nullptr;
  cudaStream_t s = nullptr;
  int nb = 0, nev = 0;
  long long ns = 0;
  T* Sx = nullptr;
  T* HS = nullptr;
  T* MS = nullptr;
  const T* dinv = nullptr;
  double* G = nullptr;     // device Gram outputs (two 3nb x 3nb)
  double* part = nullptr;  // device Gram partial sums
  T* Cd = nullptr;         // device combination coefficients
  double* hG = nullptr;    // pinned: two 3nb x 3nb Gram matrices, then 2nb residual norms, nb eigenvalues
  T* hC = nullptr;         // pinned: combination coefficients
  std::vector<double> lam;
  std::vector<double> rel;
  int applies = 0;
  int iters = 0;
  double t_sync = 0.0, t_host = 0.0;  // seconds waiting for the device, in host dense algebra
  ChebPre* pre = nullptr;             // Chebyshev-Jacobi preconditioner (else Jacobi)

  ~LobpcgRun() {
    if (hG) cudaFreeHost(hG);
    if (hC) cudaFreeHost(hC);
  }
  double* h_norms() { return hG + 2 * 9 * nb * nb; }
  double* h_lam() { return h_norms() + 2 * nb; }

  T* blk(T* base, int b) { return base + (long long)b * ns * nb; }

  // H and M of the first nvec columns of block b (all nb by default).
  void apply(int b, int nvec = 0) {
    if (nvec <= 0) nvec = nb;
    HmArgs<T> a{};
    a.x = blk(Sx, b);
    a.hx = blk(HS, b);
    a.mx = blk(MS, b);
    a.cV = cv();
    a.ld = ns;
    a.nvec = nvec;
    a.mscale = S->inv_kx;
    Profiler::Pair pp;
    if (m->prof.on) m->prof.begin(PROF_HM, s, pp);
    if constexpr (sizeof(T) == 8) {
      // FP64 vectors: H and M in double-float arithmetic on the FP32 pipes while the residuals are
      // above DF_FLOOR, FP64 applies below it; QCAD_LOBPCG_NATIVE64 selects FP64 ones throughout
      if (df_ok && use_df_apply())
        launch_hm_apply_df(S->gdf.g, a, s);
      else
        launch_hm_apply<T>(grid(), a, LaunchCfg{8, 16}, s);
    } else {
      launch_hm_apply<T>(grid(), a, LaunchCfg{8, 16}, s);
    }
    if (m->prof.on) m->prof.end(pp, s);
    applies += nvec;
  }
  static bool use_df_apply() {
    static const bool df = std::getenv("QCAD_LOBPCG_NATIVE64") == nullptr;
    return df;
  }
  // The double-float apply carries a 2^-46 relative error per term; the stiffness part of H w
  // cancels to about (h/L)^2 of its terms for smooth w, so its result is good to about 1e-10
  // relative. Below DF_FLOOR the phase refreshes H X, M X with FP64 applies and continues with
  // them, and the final Rayleigh-Ritz step always uses FP64 applies.
  T* xbest = nullptr;     // copy of X at the best iteration (stall mode), or null
  bool restored = false;  // run() returned that copy: H X, M X and lam no longer match X
  int rr_restarts = 0;
  static constexpr double DF_FLOOR = 1e-9;
  bool df_ok = true;
  bool fresh64 = false;  // the run ended right after an FP64 refresh and Rayleigh-Ritz step
  // Soft locking (the FP64 phase): columns whose residual is at or below the tolerance get no W
  // and P directions. In the FP32 phase the tolerance sits near the single-precision floor, where
  // locked columns are pulled back up by the rotations of the others and the iteration loses
  // stability, so that phase keeps every column active.
  bool soft_lock = false;
  const T* cv();
  const Grid<T>& grid();

  // Enqueues G1 = A^T B1 (and G2 = A^T B2) for p columns of A and q of B, with the copy of
  // both to hG (G1 at hG, G2 at hG + p*q); the caller synchronizes.
  void gram_async(int p, int q, const T* A, const T* B1, const T* B2, bool upper = false) {
    launch_gram<T>(ns, p, q, A, ns, B1, B2, ns, G, B2 ? G + (size_t)p * q : nullptr, part, s, upper);
    CK(cudaMemcpyAsync(hG, G, (size_t)p * q * (B2 ? 2 : 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  // Symmetrized copy of the p x p Gram matrix at hG + off.
  // upper: only the entries a p + b with a <= b were formed; they are mirrored.
  std::vector<double> gram_sym(int p, size_t off, bool upper = false) const {
    std::vector<double> out(hG + off, hG + off + (size_t)p * p);
    for (int j = 0; j < p; ++j)
      for (int i = 0; i < j; ++i) {
        const double v = upper ? out[(size_t)i * p + j] : 0.5 * (out[(size_t)j * p + i] + out[(size_t)i * p + j]);
        out[(size_t)j * p + i] = out[(size_t)i * p + j] = v;
      }
    return out;
  }
  // The FP64 phase's Rayleigh-Ritz Gram matrices from their upper triangles (H S and M S come from
  // the double-float applies, accurate to about 1e-10, so the two triangles agree far below the
  // tolerance; QCAD_LOBPCG_GRAM=full forms and averages both)
  static bool gram_upper() {
    static const bool up = [] {
      const char* e = std::getenv("QCAD_LOBPCG_GRAM");
      return sizeof(T) == 8 && !(e && std::string(e) == "full");
    }();
    return up;
  }
  void sync() {
    const auto t0 = std::chrono::steady_clock::now();
    CK(cudaStreamSynchronize(s));
    t_sync += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }

  // For S, HS and MS: columns [src, src+p) times C (p x q); output columns < q1 to block dst1,
  // the rest to block dst2 (in place). hC is reused only after a later synchronization.
  void combine(int src_blk, int p, const std::vector<double>& C, int q, int q1, int dst1, int dst2) {
    for (size_t t = 0; t < (size_t)p * q; ++t) hC[t] = (T)C[t];
    CK(cudaMemcpyAsync(Cd, hC, (size_t)p * q * sizeof(T), cudaMemcpyHostToDevice, s));
    // S, H S and M S (laid out 3 nb ns apart) in one launch
    launch_combine<T>(ns, p, q, q1, blk(Sx, src_blk), ns, Cd, blk(Sx, dst1), blk(Sx, dst2), ns, s, 3,
                      (long long)3 * nb * ns);
  }

  // Rayleigh-Ritz on block 0 alone.
  void rr_x() {
    gram_async(nb, nb, blk(Sx, 0), blk(HS, 0), blk(MS, 0));
    sync();
    std::vector<double> GH = gram_sym(nb, 0), GM = gram_sym(nb, (size_t)nb * nb), w(nb), C((size_t)nb * nb);
    if (!dense_gen_eig(nb, GH.data(), GM.data(), w.data(), C.data()))
      throw Error(QCAD_ERR_NONFINITE, "LOBPCG: Rayleigh-Ritz on X failed");
    combine(0, nb, C, nb, nb, 0, 0);
    lam.assign(w.begin(), w.end());
  }

  // The residuals H X - M X diag(lam) of all nb Ritz pairs into block 1 (times D^-1 when the
  // preconditioner is plain Jacobi) and their norms, copied to the pinned buffer (read after the
  // next synchronization).
  bool cheb() const { return pre && pre->k >= 2; }
  void residual(DevBuf& lam_d, DevBuf& norms_d) {
    std::copy(lam.begin(), lam.end(), h_lam());
    CK(cudaMemcpyAsync(lam_d.p, h_lam(), nb * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(norms_d.p, 0, 2 * nb * sizeof(double), s));
    launch_residual_block<T>(ns, nb, blk(HS, 0), blk(MS, 0), ns, lam_d.as<double>(), cheb() ? nullptr : dinv,
                             blk(Sx, 1), norms_d.as<double>(), s);
    CK(cudaMemcpyAsync(h_norms(), norms_d.p, 2 * nb * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  // Soft locking: the W and P directions of the active columns `act` (residual above the phase's
  // tolerance) only, packed after X: W to columns [nb, nb + na), P (if present, from block 2) to
  // [nb + na, nb + 2 na), in S and (P) in H S and M S. The Ritz vectors of locked columns stay in X
  // and in every Rayleigh-Ritz step.
  void pack_active(const std::vector<int>& act, bool haveP) {
    const int na = (int)act.size();
    ColMoves ms{}, mp{};
    for (int t = 0; t < na; ++t)
      if (act[t] != t) {
        ms.src[ms.n] = (short)(nb + act[t]);
        ms.dst[ms.n++] = (short)(nb + t);
      }
    if (haveP)
      for (int t = 0; t < na; ++t) {
        const int src = 2 * nb + act[t], dst = nb + na + t;
        if (src == dst) continue;
        ms.src[ms.n] = mp.src[mp.n] = (short)src;
        ms.dst[ms.n++] = mp.dst[mp.n++] = (short)dst;
      }
    if (ms.n > 40) throw Error(QCAD_ERR_INVALID_ARG, "LOBPCG: more than 40 column moves");
    launch_move_cols<T>(ns, Sx, ns, ms, s, 1, 0);
    launch_move_cols<T>(ns, HS, ns, mp, s, 2, (long long)3 * nb * ns);
    if (cheb()) precondition_block(*pre, blk(Sx, 1), na);
  }
  // Relative residuals ||H x - lam M x|| / (|lam| ||M x||) from the copied norms; true when the
  // first nev are <= tol.
  bool converged(double tol) {
    const double* nr = h_norms();
    bool all = true;
    for (int j = 0; j < nb; ++j) {
      const double scale = std::max(std::fabs(lam[j]), 1e-12) * std::sqrt(std::max(nr[2 * j + 1], 1e-300));
      rel[j] = std::sqrt(nr[2 * j]) / scale;
      if (j < nev && !(rel[j] <= tol)) all = false;
    }
    return all;
  }
  // R = L^-T for the Cholesky factor of the k x k diagonal block at `off` of the n x n matrix
  // G; false if the block is not numerically SPD.
  static bool chol_inv(const std::vector<double>& Gm, int n, int off, int k, std::vector<double>& R) {
    std::vector<double> sub((size_t)k * k);
    for (int j = 0; j < k; ++j)
      for (int i = 0; i < k; ++i) sub[(size_t)j * k + i] = Gm[(size_t)(off + j) * n + off + i];
    if (!dense_cholesky(k, sub.data())) return false;
    R.assign((size_t)k * k, 0.0);
    dense_inv_lt(k, sub.data(), R.data());
    for (double v : R)
      if (!std::isfinite(v)) return false;
    return true;
  }

  // Iterates until the first nev relative residuals are <= tol; returns true when converged.
  // With stall > 0 it also stops (returning false) once the largest of those residuals has
  // not dropped below 0.9 of its best value for `stall` iterations (the storage precision's
  // floor is reached).
  bool run(double tol, int maxit, DevBuf& lam_d, DevBuf& norms_d, int stall = 0) {
    bool haveP = false;
    rel.assign(nb, 1.0);
    double best = 1e300;
    int since = 0;
    for (int it = 1; it <= maxit + 1; ++it) {
      residual(lam_d, norms_d);
      sync();
      bool conv = converged(tol);
      if (debug_level() >= 2)
        std::fprintf(stderr, "[qcad] lobpcg %s it %d worst %.3e\n", sizeof(T) == 4 ? "fp32" : "fp64", it,
                     *std::max_element(rel.begin(), rel.begin() + nev));
      if (debug_level() >= 3) {
        std::fprintf(stderr, "[qcad]   rel");
        for (int i = 0; i < nb; ++i) std::fprintf(stderr, " %.1e", rel[i]);
        std::fprintf(stderr, "\n");
      }
      if constexpr (sizeof(T) == 8) {
        if (df_ok && use_df_apply() &&
            (conv || *std::max_element(rel.begin(), rel.begin() + nev) < DF_FLOOR)) {
          // switch to FP64 applies: fresh H X, M X, Rayleigh-Ritz on X, and the residuals again
          df_ok = false;
          apply(0);
          rr_x();
          haveP = false;
          residual(lam_d, norms_d);
          sync();
          if (converged(tol)) {
            fresh64 = true;  // X, H X, M X and the eigenvalues are FP64 Rayleigh-Ritz results
            return true;
          }
          conv = false;
        }
      }
      if (conv) return true;
      if (it > maxit) break;
      if (stall > 0) {
        // the storage precision's floor: stop once the largest residual has not dropped below 0.9
        // of its best for `stall` iterations, or has grown tenfold past a best below 1e-4 (LOBPCG
        // started at or near that floor, e.g. from the previous eigenvectors, can drift away from
        // it); the X of the best iteration is kept and restored
        const double worst = *std::max_element(rel.begin(), rel.begin() + nev);
        if (worst < 0.9 * best) {
          best = worst;
          since = 0;
          if (xbest != nullptr)
            CK(cudaMemcpyAsync(xbest, blk(Sx, 0), (size_t)ns * nb * sizeof(T), cudaMemcpyDeviceToDevice, s));
        } else if (++since >= stall || (worst > 10.0 * best && best < 1e-4)) {
          if (xbest != nullptr && worst > best) {
            CK(cudaMemcpyAsync(blk(Sx, 0), xbest, (size_t)ns * nb * sizeof(T), cudaMemcpyDeviceToDevice, s));
            restored = true;
          }
          return false;
        }
      }
      // the active columns (with soft locking those with a residual above tol, at least one; else
      // all): the basis is [X, W, P] with na columns each of W and P
      std::vector<int> act;
      for (int j = 0; j < nb; ++j)
        if (!soft_lock || !(rel[j] <= tol)) act.push_back(j);
      if (act.empty()) act.push_back(nb - 1);
      const int na = (int)act.size();
      pack_active(act, haveP);
      apply(1, na);
      // Rayleigh-Ritz Gram matrices of [X W P] with W and P as they are: the Cholesky QR of W and
      // of P is applied to the small matrices on the host (G -> T^T G T), which gives the
      // Rayleigh-Ritz problem of the orthonormalized blocks without forming them
      int nuse = haveP ? nb + 2 * na : nb + na;
      const bool up = gram_upper() && nuse % 4 == 0;
      gram_async(nuse, nuse, Sx, HS, MS, up);
      sync();
      ++iters;
      const auto th = std::chrono::steady_clock::now();
      std::vector<double> GH = gram_sym(nuse, 0, up), GM = gram_sym(nuse, (size_t)nuse * nuse, up), RW, RP;
      if (!chol_inv(GM, nuse, nb, na, RW)) {
        // W lost rank: restart it from a random block (and drop P)
        haveP = false;
        nuse = nb + na;
        launch_random_block<T>(ns, na, ns, S->interior.as<unsigned char>(), 0xABCDEF00ull + iters, blk(Sx, 1), s);
        apply(1, na);
        gram_async(nuse, nuse, Sx, HS, MS);
        sync();
        GH = gram_sym(nuse, 0);
        GM = gram_sym(nuse, (size_t)nuse * nuse);
        if (!chol_inv(GM, nuse, nb, na, RW)) throw Error(QCAD_ERR_NONFINITE, "LOBPCG: W block lost rank");
      }
      if (haveP && !chol_inv(GM, nuse, nb + na, na, RP)) haveP = false;
      // T = diag(I, RW, RP): the basis [X, W RW, P RP] has unit M-Gram blocks on its diagonal
      auto reduce_to = [&](int n2) {
        if (n2 == nuse) return;
        std::vector<double> gh2((size_t)n2 * n2), gm2((size_t)n2 * n2);
        for (int j = 0; j < n2; ++j)
          for (int i = 0; i < n2; ++i) {
            gh2[(size_t)j * n2 + i] = GH[(size_t)j * nuse + i];
            gm2[(size_t)j * n2 + i] = GM[(size_t)j * nuse + i];
          }
        GH.swap(gh2);
        GM.swap(gm2);
        nuse = n2;
      };
      if (!haveP) reduce_to(nb + na);
      auto make_T = [&]() {
        std::vector<double> Tq((size_t)nuse * nuse, 0.0);
        for (int i = 0; i < nb; ++i) Tq[(size_t)i * nuse + i] = 1.0;
        for (int j = 0; j < na; ++j)
          for (int i = 0; i < na; ++i) {
            Tq[(size_t)(nb + j) * nuse + nb + i] = RW[(size_t)j * na + i];
            if (nuse == nb + 2 * na) Tq[(size_t)(nb + na + j) * nuse + nb + na + i] = RP[(size_t)j * na + i];
          }
        return Tq;
      };
      // the diagonal block of T holding row/column i: [0, nb), [nb, nb + na) or [nb + na, nuse)
      auto blk_lo = [&](int i) { return i < nb ? 0 : (i < nb + na ? nb : nb + na); };
      auto blk_hi = [&](int i) { return i < nb ? nb : (i < nb + na ? nb + na : nuse); };
      // G' = T^T G T (column-major n x n)
      auto congruence = [&](const std::vector<double>& Tm, const std::vector<double>& Gm) {
        const int n = nuse;
        std::vector<double> GT((size_t)n * n, 0.0), out((size_t)n * n, 0.0);
        for (int j = 0; j < n; ++j)
          for (int k = 0; k < n; ++k) {
            const double t = Tm[(size_t)j * n + k];
            if (t == 0.0) continue;
            for (int i = 0; i < n; ++i) GT[(size_t)j * n + i] += Gm[(size_t)k * n + i] * t;
          }
        // T is block diagonal: column i of T is nonzero only in i's block
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) {
            const int kb = blk_lo(i), ke = blk_hi(i);
            double acc = 0.0;
            for (int k = kb; k < ke; ++k) acc += Tm[(size_t)i * n + k] * GT[(size_t)j * n + k];
            out[(size_t)j * n + i] = acc;
          }
        return out;
      };
      std::vector<double> Tm = make_T();
      std::vector<double> GHt = congruence(Tm, GH), GMt = congruence(Tm, GM), w(nuse), Ct((size_t)nuse * nuse);
      bool ok = dense_gen_eig(nuse, GHt.data(), GMt.data(), w.data(), Ct.data());
      if (!ok && haveP) {
        haveP = false;
        reduce_to(nb + na);
        Tm = make_T();
        GHt = congruence(Tm, GH);
        GMt = congruence(Tm, GM);
        w.assign(nuse, 0.0);
        Ct.assign((size_t)nuse * nuse, 0.0);
        ok = dense_gen_eig(nuse, GHt.data(), GMt.data(), w.data(), Ct.data());
      }
      if (!ok && debug_level() >= 2) {
        std::fprintf(stderr, "[qcad] lobpcg %s Rayleigh-Ritz failed at it %d (basis %d); M-Gram diagonal:",
                     sizeof(T) == 4 ? "fp32" : "fp64", it, nuse);
        for (int i = 0; i < nuse; ++i) std::fprintf(stderr, " %.3e", GMt[(size_t)i * nuse + i]);
        std::fprintf(stderr, "\n");
      }
      if (!ok) {
        // the projected M-Gram matrix lost definiteness (the basis became nearly dependent in the
        // storage precision): restart the search space from the current X
        if (++rr_restarts > 10) throw Error(QCAD_ERR_NONFINITE, "LOBPCG Rayleigh-Ritz failed");
        apply(0);
        rr_x();
        haveP = false;
        continue;
      }
      // the Ritz vectors in the stored basis: C = T C'
      std::vector<double> C((size_t)nuse * nuse, 0.0);
      for (int j = 0; j < nb; ++j)
        for (int k = 0; k < nuse; ++k) {
          const double c = Ct[(size_t)j * nuse + k];
          if (c == 0.0) continue;
          for (int i = 0; i < nuse; ++i) C[(size_t)j * nuse + i] += Tm[(size_t)k * nuse + i] * c;
        }
      // new P = [W P] C[nb:, :nb] (all nb columns, into block 2) and new X = X C[:nb, :nb] + new P,
      // in one pass over the rows
      t_host += std::chrono::duration<double>(std::chrono::steady_clock::now() - th).count();
      for (size_t t = 0; t < (size_t)nuse * nb; ++t) hC[t] = (T)C[t];
      CK(cudaMemcpyAsync(Cd, hC, (size_t)nuse * nb * sizeof(T), cudaMemcpyHostToDevice, s));
      launch_lobpcg_update<T>(ns, nb, nuse - nb, Sx, ns, Cd, s, 3, (long long)3 * nb * ns);
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
static void init_run(LobpcgRun<T>& L, qcad_mesh_s* m, const EigIo& io, SubSetup* S, int nb, int nev, DevBuf& work,
                     const T* dinv) {
  L.m = m;
  L.S = S;
  L.s = io.s;
  L.nb = nb;
  L.nev = nev;
  L.ns = S->ns;
  const long long ns = S->ns;
  const size_t gram_d = (size_t)2 * 9 * nb * nb, part_d = gram_part_doubles(3 * nb, 3 * nb);
  work.ensure((size_t)9 * nb * ns * sizeof(T) + (gram_d + part_d) * sizeof(double) +
              (size_t)9 * nb * nb * 2 * sizeof(T) + 2048);
  L.Sx = work.as<T>();
  L.HS = L.Sx + 3 * nb * ns;
  L.MS = L.HS + 3 * nb * ns;
  unsigned char* tail = reinterpret_cast<unsigned char*>(L.MS + 3 * nb * ns);
  tail = reinterpret_cast<unsigned char*>(((uintptr_t)tail + 255) & ~(uintptr_t)255);
  L.G = reinterpret_cast<double*>(tail);
  L.part = L.G + gram_d;
  L.Cd = reinterpret_cast<T*>(L.part + part_d);
  L.dinv = dinv;
  CK(cudaMallocHost(&L.hG, (gram_d + 3 * nb + 16) * sizeof(double)));
  CK(cudaMallocHost(&L.hC, (size_t)9 * nb * nb * 2 * sizeof(T) + 64));
}

qcad_status schrodinger_eigs_io(qcad_mesh_s* m, const EigIo& io, const qcad_bias* b, const double* phi, int nev,
                                const double* m_eff, double tol, double* evals, double* evecs,
                                qcad_solve_report* rep, const double* vxq = nullptr, double shift_floor = 0.0,
                                const double* x0 = nullptr) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!b || !phi || !m_eff || !evals) throw Error(QCAD_ERR_INVALID_ARG, "null pointer");
  if (nev < 1 || nev > 16) throw Error(QCAD_ERR_INVALID_ARG, "nev must be in [1, 16]");
  if (!(tol > 0)) throw Error(QCAD_ERR_INVALID_ARG, "tol must be > 0");
  SubSetup S;
  setup_sub(m, b, phi, m_eff, 1, S, io, vxq, shift_floor);
  const double t_setup = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (S.ndof < 3 * (nev + 4)) throw Error(QCAD_ERR_INVALID_ARG, "subdomain too small for nev");
  cudaStream_t s = io.s;
  // block size: nev plus guard vectors (QCAD_LOBPCG_GUARD overrides the count). The lowest levels
  // of a double dot cluster within a few meV, so convergence is set by the gap to the first level
  // outside the block: with a multigrid V-cycle of K + M_{V - min V} as the preconditioner the
  // worst residual fell by the same factor per iteration (about 0.7) as with this polynomial, and
  // more guard vectors cost more per iteration than they save
  const char* ge = std::getenv("QCAD_LOBPCG_GUARD");
  const int guard = ge ? std::max(1, std::atoi(ge)) : std::max(2, nev / 4);
  // (at most 20 columns: the [X W P] kernels take up to 64 columns and the host eigensolver 60)
  const int nb = (int)std::min<long long>(std::min(nev + guard, 20), S.ndof / 3);
  const long long ns = S.ns;
  DevBuf lam_d, norms_d, dinv32;
  lam_d.ensure(nb * sizeof(double) + 64);
  norms_d.ensure(2 * nb * sizeof(double) + 64);
  dinv32.ensure(ns * sizeof(float) + 64);
  launch_d2f(ns, S.dinv.as<double>(), dinv32.as<float>(), s);

  // Phase 1: FP32 storage, applies and block arithmetic (FP64 Gram accumulation and host
  // Rayleigh-Ritz) until the residuals reach the single-precision level.
  DevBuf w32, w64;
  ChebPre pre;
  // Chebyshev degrees of the two phases (environment QCAD_LOBPCG_DEG32 / QCAD_LOBPCG_DEG64 override)
  auto env_int = [](const char* name, int def) {
    const char* e = std::getenv(name);
    return e ? std::max(1, std::atoi(e)) : def;
  };
  const int deg32 = env_int("QCAD_LOBPCG_DEG32", 5), deg64 = env_int("QCAD_LOBPCG_DEG64", 5);
  pre.init(m, io, &S, nb, deg32, dinv32.as<float>());
  LobpcgRun<float> A;
  init_run<float>(A, m, io, &S, nb, nev, w32, dinv32.as<float>());
  A.pre = &pre;
  {
    // a cold start: the nb lowest modes of the subdomain box (by the kinetic energy of the separable
    // sines on its physical extents) with a 1 % random part, which spares the first iterations the
    // damping of a random block's high frequencies (c3: 35 + 16 iterations instead of 47 + 23); a
    // warm start (the first nev columns given) keeps random guard columns, as does
    // QCAD_LOBPCG_START=random
    const char* st = std::getenv("QCAD_LOBPCG_START");
    if (x0 != nullptr || (st && std::string(st) == "random")) {
      launch_random_block<float>(ns, nb, ns, S.interior.as<unsigned char>(), 0x51ED5EEDull, A.Sx, s);
    } else {
      const double Lx = m->xc[S.sm.i0 + S.sm.nxs] - m->xc[S.sm.i0], Ly = m->yc[S.sm.j0 + S.sm.nys] - m->yc[S.sm.j0];
      const double Lz = m->zc[S.sm.k0 + S.sm.nzs] - m->zc[S.sm.k0];
      struct Mode {
        double e;
        int a, b, c;
      };
      std::vector<Mode> modes;
      for (int a = 1; a <= nb; ++a)
        for (int b = 1; b <= nb; ++b)
          for (int c = 1; c <= nb; ++c)
            if (a < S.sm.nxs && b < S.sm.nys && c < S.sm.nzs)
              modes.push_back({(a * a) / (Lx * Lx * m_eff[0]) + (b * b) / (Ly * Ly * m_eff[1]) +
                                   (c * c) / (Lz * Lz * m_eff[2]), a, b, c});
      std::sort(modes.begin(), modes.end(), [](const Mode& p, const Mode& q) { return p.e < q.e; });
      if ((int)modes.size() >= nb && nb <= 32) {
        BoxModes bm{};
        for (int j = 0; j < nb; ++j) {
          bm.a[j] = modes[j].a;
          bm.b[j] = modes[j].b;
          bm.c[j] = modes[j].c;
        }
        launch_box_mode_block<float>(ns, nb, ns, S.sm.nxs, S.sm.nys, S.sm.nzs, bm, 1e-2, S.interior.as<unsigned char>(),
                                     0x51ED5EEDull, A.Sx, s);
      } else {
        launch_random_block<float>(ns, nb, ns, S.interior.as<unsigned char>(), 0x51ED5EEDull, A.Sx, s);
      }
    }
  }
  if (x0) {
    // warm start: the first nev columns from the given vectors (interior nodes), the guard
    // columns stay random
    DevBuf full;
    full.ensure((size_t)ns * nev * sizeof(double) + 64);
    CK(cudaMemsetAsync(full.p, 0, (size_t)ns * nev * sizeof(double), s));
    launch_pack(S.sm, nev, full.as<double>(), ns, const_cast<double*>(x0), S.ndof, 1, s);
    launch_d2f(ns * nev, full.as<double>(), A.Sx, s);
    CK(cudaStreamSynchronize(s));
  }
  A.apply(0);
  A.rr_x();
  // the FP32 phase stops at 3e-6 relative residual, above where single-precision LOBPCG loses
  // the P block's conditioning (near 2e-6 on these devices), or when it stops improving
  const double tol32 = std::max(tol, 3e-6);
  DevBuf xbest32;
  xbest32.ensure((size_t)nb * ns * sizeof(float) + 64);
  A.xbest = xbest32.as<float>();
  A.run(tol32, 3000, lam_d, norms_d, 15);
  const double t_a = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();

  // Phase 2: FP64 from the FP32 Ritz vectors to the requested tolerance.
  LobpcgRun<double> B;
  init_run<double>(B, m, io, &S, nb, nev, w64, S.dinv.as<double>());
  B.pre = &pre;
  B.soft_lock = !(std::getenv("QCAD_LOBPCG_LOCK") && std::string(std::getenv("QCAD_LOBPCG_LOCK")) == "0");
  pre.set_degree(deg64);
  launch_f2d(ns * nb, A.Sx, B.Sx, s);
  B.apply(0);
  B.rr_x();
  bool converged = B.run(tol, 500, lam_d, norms_d);
  // final Rayleigh-Ritz with fresh FP64 applies (unless the run just did one)
  B.df_ok = false;
  if (!B.fresh64) {
    B.apply(0);
    B.rr_x();
  }
  for (int j = 0; j < nev; ++j) evals[j] = B.lam[j] - S.shift;
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
  if (std::getenv("QCAD_DEBUG")) {
    const double t_all = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    std::fprintf(stderr,
                 "[qcad] lobpcg setup %.1f ms, fp32 %.1f ms (%d it, sync %.1f, host %.1f), fp64 %.1f ms "
                 "(%d it, sync %.1f, host %.1f)\n",
                 1e3 * t_setup, 1e3 * (t_a - t_setup), A.iters, 1e3 * A.t_sync, 1e3 * A.t_host,
                 1e3 * (t_all - t_a), B.iters, 1e3 * B.t_sync, 1e3 * B.t_host);
  }
  if (!converged) set_message("LOBPCG did not reach the requested tolerance");
  return converged ? QCAD_OK : QCAD_ERR_NOT_CONVERGED;
}

qcad_status schrodinger_eigs(qcad_mesh_s* m, const qcad_bias* b, const double* phi, int nev, const double* m_eff,
                             double tol, double* evals, double* evecs, qcad_solve_report* rep) {
  return schrodinger_eigs_io(m, mesh_io(m), b, phi, nev, m_eff, tol, evals, evecs, rep);
}

// The eigensolve of the self-consistent loop: potential V(phi) + vxq, shifted so that its minimum
// sits at 0.1 eV while LOBPCG runs (levels near the Fermi level would otherwise make the
// relative residual test |lambda|-relative around lambda = 0).
// x0 (interior nodes x nev, or null) starts the block: the previous iteration's eigenvectors.
qcad_status schrodinger_eigs_sp(qcad_mesh_s* m, const qcad_bias* b, const double* phi, int nev, const double* m_eff,
                                double tol, const double* vxq, const double* x0, double* evals, double* evecs,
                                qcad_solve_report* rep) {
  return schrodinger_eigs_io(m, mesh_io(m), b, phi, nev, m_eff, tol, evals, evecs, rep, vxq, 0.1, x0);
}

// The eigensolve on the mesh's second stream and scratch (created on first use), for running
// concurrently with work on the mesh stream (the two share only read-only mesh data).
qcad_status schrodinger_eigs_stream2(qcad_mesh_s* m, const qcad_bias* b, const double* phi, int nev,
                                     const double* m_eff, double tol, double* evals, double* evecs,
                                     qcad_solve_report* rep) {
  if (!m->stream2) {
    // the eigensolve issues short, latency-bound kernels between host synchronizations: the
    // highest priority lets its blocks start ahead of the concurrent work's queued blocks
    int lo = 0, hi = 0;
    CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    CK(cudaStreamCreateWithPriority(&m->stream2, cudaStreamNonBlocking, hi));
  }
  m->stats2.ensure(64 * sizeof(double));
  if (!m->h_small2) CK(cudaMallocHost(&m->h_small2, 64 * sizeof(double)));
  return schrodinger_eigs_io(m, EigIo{m->stream2, m->stats2.as<double>(), m->h_small2}, b, phi, nev, m_eff, tol,
                             evals, evecs, rep);
}

}  // namespace qcad
