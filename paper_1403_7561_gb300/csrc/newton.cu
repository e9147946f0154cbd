// Solver drivers (host): preconditioned CG with device-resident scalars and
// CUDA-graph-captured iteration chunks, the Newton iteration of the nonlinear
// Poisson problem (Sec. II.A.3: "solved by a nonlinear Newton solver"),
// electron counts, finite-difference capacitance (Sec. III) and the adjoint.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "mesh.h"

namespace qcad {

Phys make_phys(const qcad_mesh_s* m, const qcad_bias* b);
double ohmic_value(const qcad_mesh_s* m, const qcad_bias* b, const Phys& P);
double gate_value(const qcad_mesh_s* m, double Vg, const Phys& P);
double host_qe();
void set_message(const std::string& msg);

static bool debug_on() {
  static const bool on = std::getenv("QCAD_DEBUG") != nullptr;
  return on;
}

static const int PCG_CHUNK = 8;

template <class T> struct Prec;
template <> struct Prec<double> {
  static PcgBufs<double>& bufs(qcad_mesh_s* m) { return m->k64; }
  static PcgGraph& graph(qcad_mesh_s* m) { return m->graph64; }
  static const Grid<double>& grid(qcad_mesh_s* m) { return m->g64.g; }
  static LaunchCfg cfg(qcad_mesh_s* m) { return m->cfg64; }
  static const int prof_apply = PROF_APPLY64, prof_update = PROF_UPDATE64;
};
template <> struct Prec<float> {
  static PcgBufs<float>& bufs(qcad_mesh_s* m) { return m->k32; }
  static PcgGraph& graph(qcad_mesh_s* m) { return m->graph32; }
  static const Grid<float>& grid(qcad_mesh_s* m) { return m->g32.g; }
  static LaunchCfg cfg(qcad_mesh_s* m) { return m->cfg32; }
  static const int prof_apply = PROF_APPLY32, prof_update = PROF_UPDATE32;
};

template <class T>
static PcgVecs<T> ensure_pcg(qcad_mesh_s* m) {
  PcgBufs<T>& b = Prec<T>::bufs(m);
  const size_t nb = (size_t)m->n_nodes * sizeof(T) + 64;
  b.x.ensure(nb);
  b.r.ensure(nb);
  b.z.ensure(nb);
  b.p.ensure(2 * nb);
  b.Ap.ensure(nb);
  b.b.ensure(nb);
  b.dinv.ensure(nb);
  b.c.ensure((size_t)m->n_elems * 8 * sizeof(T) + 64);
  PcgVecs<T> v;
  v.x = b.x.template as<T>();
  v.r = b.r.template as<T>();
  v.z = b.z.template as<T>();
  v.p[0] = b.p.template as<T>();
  v.p[1] = v.p[0] + (nb / sizeof(T));
  v.Ap = b.Ap.template as<T>();
  v.b = b.b.template as<T>();
  v.dinv = b.dinv.template as<T>();
  v.c = b.c.template as<T>();
  return v;
}

static void ensure_newton(qcad_mesh_s* m) {
  const size_t nb = (size_t)m->n_nodes * sizeof(double) + 64;
  m->phi_a.ensure(nb);
  m->phi_b.ensure(nb);
  m->R.ensure(nb);
}

// Captures PCG_CHUNK iterations (apply + update kernels) into a graph; with
// profiling on, every kernel is bracketed by event-record nodes.
template <class T>
static void build_graph(qcad_mesh_s* m, const PcgVecs<T>& v) {
  PcgGraph& G = Prec<T>::graph(m);
  if (G.exec) {
    cudaGraphExecDestroy(G.exec);
    G.exec = nullptr;
  }
  for (auto& p : G.events) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  G.events.clear();
  cudaStream_t s = m->stream;
  const bool prof = m->prof.on;
  if (prof) {
    for (int i = 0; i < 2 * PCG_CHUNK; ++i) {
      Profiler::Pair p;
      CK(cudaEventCreate(&p.a));
      CK(cudaEventCreate(&p.b));
      p.cls = (i & 1) ? Prec<T>::prof_update : Prec<T>::prof_apply;
      G.events.push_back(p);
    }
  }
  PcgScalars* sc = m->scal.as<PcgScalars>();
  const long long n = m->n_nodes;
  const long long launches_before = launch_count();
  CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  for (int it = 0; it < PCG_CHUNK; ++it) {
    if (prof) CK(cudaEventRecordWithFlags(G.events[2 * it].a, s, cudaEventRecordExternal));
    launch_pcg_apply<T>(Prec<T>::grid(m), v, sc, Prec<T>::cfg(m), s);
    if (prof) CK(cudaEventRecordWithFlags(G.events[2 * it].b, s, cudaEventRecordExternal));
    if (prof) CK(cudaEventRecordWithFlags(G.events[2 * it + 1].a, s, cudaEventRecordExternal));
    launch_pcg_update<T>(n, v, sc, s);
    if (prof) CK(cudaEventRecordWithFlags(G.events[2 * it + 1].b, s, cudaEventRecordExternal));
  }
  cudaGraph_t graph;
  CK(cudaStreamEndCapture(s, &graph));
  note_launch((int)(launches_before - launch_count()));  // captured kernels run only when replayed
  cudaError_t e = cudaGraphInstantiate(&G.exec, graph, 0);
  cudaGraphDestroy(graph);
  CK(e);
  G.chunk = PCG_CHUNK;
}

struct PcgResult {
  int iters = 0;
  bool nonfinite = false;
  bool converged = false;
};

// Solves J x = b (b, dinv, c already in the precision's buffers) to ||r|| <= rtol ||b||.
template <class T>
static PcgResult pcg_run(qcad_mesh_s* m, double rtol, int maxit) {
  PcgVecs<T> v = ensure_pcg<T>(m);
  PcgGraph& G = Prec<T>::graph(m);
  const bool prof_match = m->prof.on == !G.events.empty();
  if (!G.exec || G.key != (const void*)v.x || !prof_match) {
    build_graph<T>(m, v);
    G.key = (const void*)v.x;
  }
  cudaStream_t s = m->stream;
  PcgScalars* h = m->h_scal;
  std::memset(h, 0, sizeof(PcgScalars));
  h->tol2 = rtol * rtol;
  h->maxit = maxit;
  PcgScalars* sc = m->scal.as<PcgScalars>();
  CK(cudaMemcpyAsync(sc, h, sizeof(PcgScalars), cudaMemcpyHostToDevice, s));
  launch_pcg_init<T>(m->n_nodes, v, sc, s);
  CK(cudaGetLastError());
  int t_prev = 0;
  int guard = 0;
  for (;;) {
    CK(cudaGraphLaunch(G.exec, s));
    note_launch(2 * PCG_CHUNK);
    CK(cudaMemcpyAsync(h, sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (m->prof.on) {
      const int ran = std::min(PCG_CHUNK, h->t - t_prev);
      for (int it = 0; it < PCG_CHUNK; ++it) {
        for (int q = 0; q < 2; ++q) {
          Profiler::Pair& p = G.events[2 * it + q];
          // the apply of iteration t_prev+it ran iff it < ran; the update likewise
          if (it < ran) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
              m->prof.ms[p.cls] += ms;
              m->prof.launches[p.cls] += 1;
            } else {
              cudaGetLastError();
            }
          }
        }
      }
    }
    t_prev = h->t;
    if (h->done) break;
    if (++guard > maxit / PCG_CHUNK + 4) break;
  }
  PcgResult r;
  r.iters = h->t;
  r.nonfinite = h->nonfinite != 0;
  r.converged = h->done && !h->nonfinite && (h->rr0 == 0.0 || h->rr[h->t & 3] <= h->tol2 * h->rr0);
  return r;
}

// Residual at phi with the linearization written in precision `prec`.
struct ResStats {
  double rmax, r2;
};

static ResStats eval_residual(qcad_mesh_s* m, const Phys& P, const double* phi, const double* theta, int linear,
                              int prec, double* counts_out, double* diag_out = nullptr) {
  cudaStream_t s = m->stream;
  ResidualArgs a{};
  a.phi = phi;
  a.theta = theta;
  a.R = m->R.as<double>();
  if (prec == 0) {
    PcgVecs<double> v = ensure_pcg<double>(m);
    a.c64 = const_cast<double*>(v.c);
    a.dinv64 = const_cast<double*>(v.dinv);
    a.b64 = const_cast<double*>(v.b);
  } else {
    PcgVecs<float> v = ensure_pcg<float>(m);
    a.c32 = const_cast<float*>(v.c);
    a.dinv32 = const_cast<float*>(v.dinv);
    a.b32 = const_cast<float*>(v.b);
  }
  a.layer_semi = m->d_layer_semi.as<unsigned char>();
  a.xn = m->d_xn.as<double>();
  a.yn = m->d_yn.as<double>();
  a.zn = m->d_zn.as<double>();
  a.P = P;
  a.dots = m->dots;
  a.linear = linear;
  a.diag = diag_out;
  a.stats = m->stats.as<double>();
  CK(cudaMemsetAsync(a.stats, 0, 2 * sizeof(double), s));
  if (counts_out) {
    a.counts = m->counts.as<double>();
    CK(cudaMemsetAsync(a.counts, 0, QCAD_MAX_DOTS_K * sizeof(double), s));
  }
  Profiler::Pair pp;
  if (m->prof.on) m->prof.begin(PROF_RESIDUAL, s, pp);
  launch_residual(m->g64.g, a, m->cfg_res, s);
  if (m->prof.on) m->prof.end(pp, s);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(m->h_small, a.stats, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (counts_out)
    CK(cudaMemcpyAsync(m->h_small + 8, a.counts, QCAD_MAX_DOTS_K * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (m->prof.on) m->prof.harvest();
  ResStats r;
  r.rmax = m->h_small[0];
  r.r2 = m->h_small[1];
  if (counts_out)
    for (int d = 0; d < m->dots.n; ++d) counts_out[d] = m->h_small[8 + d];
  return r;
}

void set_contacts(qcad_mesh_s* m, const qcad_bias* b, const Phys& P, double* phi, double* gate_vals,
                  double* ohm_val) {
  if (b->n_gates != m->n_gates || (m->n_gates > 0 && !b->V_gate))
    throw Error(QCAD_ERR_INVALID_ARG, "bias gate count does not match the mesh");
  double vg[QCAD_MAX_GATES];
  for (int g = 0; g < m->n_gates; ++g) vg[g] = gate_value(m, b->V_gate[g], P);
  const double vo = ohmic_value(m, b, P);
  if (gate_vals)
    for (int g = 0; g < m->n_gates; ++g) gate_vals[g] = vg[g];
  if (ohm_val) *ohm_val = vo;
  if (!phi) return;
  std::memcpy(m->h_small + 16, vg, sizeof(double) * std::max(1, m->n_gates));
  CK(cudaMemcpyAsync(m->d_vgate.p, m->h_small + 16, sizeof(double) * std::max(1, m->n_gates),
                     cudaMemcpyHostToDevice, m->stream));
  launch_set_dirichlet(m->nxn, m->nyn, m->nzn, m->bottom_ohmic, vo, m->d_gate_top.as<signed char>(),
                       m->d_vgate.as<double>(), phi, m->stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(m->stream));
}

static void validate_bias(const qcad_mesh_s* m, const qcad_bias* b) {
  if (!b) throw Error(QCAD_ERR_INVALID_ARG, "null bias");
  if (!(b->T > 0.0) || !std::isfinite(b->T)) throw Error(QCAD_ERR_INVALID_ARG, "temperature must be > 0");
  if (b->n_gates != m->n_gates) throw Error(QCAD_ERR_INVALID_ARG, "bias gate count does not match the mesh");
  if (b->statistics != 0 && b->statistics != 1) throw Error(QCAD_ERR_INVALID_ARG, "statistics must be 0 or 1");
  for (int g = 0; g < b->n_gates; ++g)
    if (!std::isfinite(b->V_gate[g])) throw Error(QCAD_ERR_INVALID_ARG, "non-finite gate voltage");
}

// Newton iteration; phi (device, n_nodes) is input guess (warm) and output.
template <class T>
static qcad_status newton_impl(qcad_mesh_s* m, const qcad_bias* b, const qcad_solver_opts* o, const double* theta,
                               double* phi, qcad_solve_report* rep) {
  const auto t0 = std::chrono::steady_clock::now();
  const int prec = sizeof(T) == 8 ? 0 : 1;
  cudaStream_t s = m->stream;
  const long long n = m->n_nodes;
  ensure_newton(m);
  PcgVecs<T> v = ensure_pcg<T>(m);
  const Phys P = make_phys(m, b);
  double* pa = m->phi_a.as<double>();
  double* pb = m->phi_b.as<double>();
  if (o->warm_start)
    CK(cudaMemcpyAsync(pa, phi, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  else
    CK(cudaMemsetAsync(pa, 0, n * sizeof(double), s));
  set_contacts(m, b, P, pa, nullptr, nullptr);
  const double floor_eta = prec == 0 ? 1e-12 : 1e-5;
  const int maxk = o->max_krylov > 0 ? o->max_krylov : 20000;
  int kry = 0;
  qcad_status st = QCAD_OK;
  if (!o->warm_start) {
    // Laplace initial guess with the contact values (rho = 0)
    eval_residual(m, P, pa, theta, 1, prec, nullptr);
    PcgResult pr = pcg_run<T>(m, prec == 0 ? 1e-10 : 1e-6, maxk);
    kry += pr.iters;
    if (debug_on()) std::fprintf(stderr, "[qcad] laplace pcg iters %d conv %d\n", pr.iters, (int)pr.converged);
    if (pr.nonfinite) {
      set_message("PCG breakdown in the Laplace initial-guess solve after " + std::to_string(pr.iters) +
                  " iterations");
      return QCAD_ERR_NONFINITE;
    }
    CK(cudaMemsetAsync(m->stats.p, 0, sizeof(double), s));
    launch_newton_trial<T>(n, pa, v.x, 1.0, pb, m->stats.as<double>(), s);
    std::swap(pa, pb);
  }
  ResStats R = eval_residual(m, P, pa, theta, o->linear, prec, nullptr);
  if (!std::isfinite(R.r2)) {
    set_message("non-finite residual at the initial guess");
    return QCAD_ERR_NONFINITE;
  }
  const double R0 = std::sqrt(R.r2);
  int it = 0;
  double step = 0.0;
  bool converged = false;
  int ls_fail = 0;
  const int maxn = o->max_newton > 0 ? o->max_newton : 100;
  if (R.rmax < o->newton_tol_R && o->warm_start && R.rmax == 0.0) converged = true;
  while (!converged && it < maxn) {
    ++it;
    const double nR = std::sqrt(R.r2);
    double eta = R0 > 0 ? std::min(1e-2, nR / R0) : 1e-2;
    eta = std::max(eta, floor_eta);
    PcgResult pr = pcg_run<T>(m, eta, maxk);
    kry += pr.iters;
    if (pr.nonfinite) {
      set_message("PCG breakdown at Newton iteration " + std::to_string(it) + " after " +
                  std::to_string(pr.iters) + " iterations");
      st = QCAD_ERR_NONFINITE;
      break;
    }
    double alpha = 1.0;
    ResStats Rt{};
    for (int ls = 0; ls <= 30; ++ls) {
      CK(cudaMemsetAsync(m->stats.p, 0, sizeof(double), s));
      launch_newton_trial<T>(n, pa, v.x, alpha, pb, m->stats.as<double>(), s);
      CK(cudaMemcpyAsync(m->h_small + 4, m->stats.p, sizeof(double), cudaMemcpyDeviceToHost, s));
      // the trial residual also refreshes the linearization (c, dinv, b) at pb
      Rt = eval_residual(m, P, pb, theta, o->linear, prec, nullptr);
      step = m->h_small[4];
      if (std::isfinite(Rt.r2) && std::sqrt(Rt.r2) <= (1.0 - 1e-4 * alpha) * nR) break;
      if (ls == 30) ls_fail = 1;
      alpha *= 0.5;
    }
    // eval_residual overwrote h_small[0..1]; step was read before it
    std::swap(pa, pb);
    R = Rt;
    if (debug_on())
      std::fprintf(stderr, "[qcad] newton %d eta %.2e pcg %d alpha %.3g |R|inf %.3e |dphi|inf %.3e\n", it, eta,
                   pr.iters, alpha, R.rmax, step);
    if (!std::isfinite(R.r2)) {
      set_message("non-finite residual at Newton iteration " + std::to_string(it));
      st = QCAD_ERR_NONFINITE;
      break;
    }
    if (R.rmax < o->newton_tol_R && step < o->newton_tol_dphi) converged = true;
  }
  CK(cudaMemcpyAsync(phi, pa, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  if (rep) {
    rep->newton_iters = it;
    rep->krylov_iters_total = kry;
    rep->applies_total = kry;
    rep->final_res_inf = R.rmax;
    rep->final_dphi_inf = step;
    rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    rep->status_detail = ls_fail;
  }
  if (st != QCAD_OK) return st;
  if (!converged) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "Newton stopped after %d iterations: |R|inf %.3e, |dphi|inf %.3e", it, R.rmax,
                  step);
    set_message(buf);
  }
  return converged ? QCAD_OK : QCAD_ERR_NOT_CONVERGED;
}

static void validate_opts(const qcad_solver_opts* o) {
  if (!o) throw Error(QCAD_ERR_INVALID_ARG, "null solver options");
  if (o->precision != 0 && o->precision != 1) throw Error(QCAD_ERR_INVALID_ARG, "precision must be 0 or 1");
  if (!(o->newton_tol_R > 0) || !(o->newton_tol_dphi > 0)) throw Error(QCAD_ERR_INVALID_ARG, "tolerances must be > 0");
}

qcad_status poisson_solve(qcad_mesh_s* m, const qcad_bias* b, const qcad_solver_opts* o, const double* theta,
                          double* phi, qcad_solve_report* rep) {
  validate_bias(m, b);
  validate_opts(o);
  if (!phi) throw Error(QCAD_ERR_INVALID_ARG, "null phi");
  if (o->precision == 0) return newton_impl<double>(m, b, o, theta, phi, rep);
  return newton_impl<float>(m, b, o, theta, phi, rep);
}

qcad_status poisson_residual(qcad_mesh_s* m, const qcad_bias* b, const double* theta, const double* phi, double* R,
                             double* diag, double* stats) {
  validate_bias(m, b);
  if (!phi || !R) throw Error(QCAD_ERR_INVALID_ARG, "null phi or R");
  ensure_newton(m);
  const Phys P = make_phys(m, b);
  ResStats st = eval_residual(m, P, phi, theta, 0, 0, nullptr, diag);
  cudaStream_t s = m->stream;
  CK(cudaMemcpyAsync(R, m->R.p, m->n_nodes * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  if (stats) {
    stats[0] = st.rmax;
    stats[1] = st.r2;
  }
  return QCAD_OK;
}

qcad_status poisson_jv(qcad_mesh_s* m, const qcad_bias* b, const double* phi, const double* vin, double* y,
                       int precision) {
  validate_bias(m, b);
  if (!phi || !vin || !y) throw Error(QCAD_ERR_INVALID_ARG, "null pointer");
  if (precision != 0 && precision != 1) throw Error(QCAD_ERR_INVALID_ARG, "precision must be 0 or 1");
  ensure_newton(m);
  const Phys P = make_phys(m, b);
  eval_residual(m, P, phi, nullptr, 0, precision, nullptr);
  cudaStream_t s = m->stream;
  if (precision == 0) {
    PcgVecs<double> v = ensure_pcg<double>(m);
    ApplyArgs<double> a{};
    a.v = vin;
    a.y = y;
    a.c = v.c;
    launch_apply<double>(m->g64.g, a, m->cfg64, s);
  } else {
    PcgVecs<float> v = ensure_pcg<float>(m);
    launch_d2f(m->n_nodes, vin, v.r, s);
    ApplyArgs<float> a{};
    a.v = v.r;
    a.y = v.Ap;
    a.c = v.c;
    launch_apply<float>(m->g32.g, a, m->cfg32, s);
    launch_f2d(m->n_nodes, v.Ap, y, s);
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return QCAD_OK;
}

qcad_status electron_counts(qcad_mesh_s* m, const qcad_bias* b, const double* theta, const double* phi, double* N) {
  validate_bias(m, b);
  if (!phi || !N) throw Error(QCAD_ERR_INVALID_ARG, "null pointer");
  ensure_newton(m);
  const Phys P = make_phys(m, b);
  eval_residual(m, P, phi, theta, 0, 0, N);
  return QCAD_OK;
}

qcad_status capacitance(qcad_mesh_s* m, const qcad_bias* b, const qcad_solver_opts* o, int gate, double dV,
                        const double* theta, double* phi, double* C_aF) {
  validate_bias(m, b);
  validate_opts(o);
  if (gate < 0 || gate >= m->n_gates) throw Error(QCAD_ERR_INVALID_ARG, "gate index out of range");
  if (!(dV != 0.0) || !std::isfinite(dV)) throw Error(QCAD_ERR_INVALID_ARG, "dV must be finite and nonzero");
  if (!C_aF) throw Error(QCAD_ERR_INVALID_ARG, "null output");
  double* work = phi;
  if (!work) {
    m->scratch.ensure(m->n_nodes * sizeof(double) + 64);
    work = m->scratch.as<double>();
  }
  qcad_status st = poisson_solve(m, b, o, theta, work, nullptr);
  if (st != QCAD_OK) return st;
  double N1[QCAD_MAX_DOTS_K], N2[QCAD_MAX_DOTS_K];
  electron_counts(m, b, theta, work, N1);
  std::vector<double> V(b->V_gate, b->V_gate + b->n_gates);
  V[gate] += dV;
  qcad_bias b2 = *b;
  b2.V_gate = V.data();
  qcad_solver_opts o2 = *o;
  o2.warm_start = 1;
  st = poisson_solve(m, &b2, &o2, theta, work, nullptr);
  if (st != QCAD_OK) return st;
  electron_counts(m, &b2, theta, work, N2);
  const double q_aF = 1.602176634e-19 * 1e18;
  for (int d = 0; d < m->dots.n; ++d) C_aF[d] = q_aF * (N2[d] - N1[d]) / dV;
  return QCAD_OK;
}

// Solve J lam = g on free rows (g zero on Dirichlet rows) in FP64, or by
// iterative refinement around FP32 PCG in mixed precision.
static void adjoint_solve(qcad_mesh_s* m, int prec, const double* g, double* lam, int maxk) {
  cudaStream_t s = m->stream;
  const long long n = m->n_nodes;
  PcgVecs<double> v = ensure_pcg<double>(m);
  if (prec == 0) {
    CK(cudaMemcpyAsync(const_cast<double*>(v.b), g, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    PcgResult pr = pcg_run<double>(m, 1e-13, maxk);
    if (pr.nonfinite) throw Error(QCAD_ERR_NONFINITE, "adjoint linear solve produced a non-finite value");
    CK(cudaMemcpyAsync(lam, v.x, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    return;
  }
  PcgVecs<float> w = ensure_pcg<float>(m);
  m->scratch.ensure(3 * n * sizeof(double) + 64);
  double* y = m->scratch.as<double>();
  double* r = y + n;
  CK(cudaMemsetAsync(lam, 0, n * sizeof(double), s));
  CK(cudaMemcpyAsync(r, g, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  launch_d2f(n, g, const_cast<float*>(w.b), s);
  double* d2 = m->stats.as<double>() + 8;
  CK(cudaMemsetAsync(d2, 0, sizeof(double), s));
  launch_dot<double>(n, g, g, d2, s);
  CK(cudaMemcpyAsync(m->h_small + 20, d2, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const double g2 = m->h_small[20];
  for (int rf = 0; rf < 12; ++rf) {
    PcgResult pr = pcg_run<float>(m, 1e-5, maxk);
    if (pr.nonfinite) throw Error(QCAD_ERR_NONFINITE, "adjoint refinement produced a non-finite value");
    launch_axpy<float>(n, 1.0, w.x, lam, s);
    ApplyArgs<double> a{};
    a.v = lam;
    a.y = y;
    a.c = v.c;
    launch_apply<double>(m->g64.g, a, m->cfg64, s);
    launch_sub(n, g, y, r, const_cast<float*>(w.b), s);
    CK(cudaMemsetAsync(d2, 0, sizeof(double), s));
    launch_dot<double>(n, r, r, d2, s);
    CK(cudaMemcpyAsync(m->h_small + 20, d2, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (m->h_small[20] <= 1e-26 * g2) break;
  }
}

qcad_status adjoint(qcad_mesh_s* m, const qcad_bias* b, const qcad_solver_opts* o, const double* phi,
                    const double* theta, double* dN_dV, double* dN_dq) {
  validate_bias(m, b);
  validate_opts(o);
  if (!phi || !dN_dV) throw Error(QCAD_ERR_INVALID_ARG, "null pointer");
  cudaStream_t s = m->stream;
  const long long n = m->n_nodes;
  ensure_newton(m);
  const Phys P = make_phys(m, b);
  // linearization at phi in FP64 (and FP32 for the mixed refinement)
  eval_residual(m, P, phi, theta, 0, 0, nullptr);
  if (o->precision == 1) eval_residual(m, P, phi, theta, 0, 1, nullptr);
  DevBuf work;
  work.ensure(4 * n * sizeof(double) + 64);
  double* g = work.as<double>();
  double* lam = g + n;
  double* eg = g + 2 * n;
  double* Jeg = g + 3 * n;
  double* zero_v = m->stats.as<double>() + 32;  // 16 zeros for masking Dirichlet rows
  CK(cudaMemsetAsync(zero_v, 0, 16 * sizeof(double), s));
  const int maxk = o->max_krylov > 0 ? o->max_krylov : 20000;
  std::vector<double> gD(m->n_gates * QCAD_MAX_DOTS_K, 0.0);
  for (int d = 0; d < m->dots.n; ++d) {
    launch_count_gradient(m->g64.g, phi, m->d_layer_semi.as<unsigned char>(), m->d_xn.as<double>(),
                          m->d_yn.as<double>(), m->d_zn.as<double>(), P, m->dots, d, g, m->cfg_res, s);
    // dN/dphi_D . e_g before masking
    for (int gi = 0; gi < m->n_gates; ++gi) {
      CK(cudaMemsetAsync(eg, 0, n * sizeof(double), s));
      std::vector<double> one(m->n_gates, 0.0);
      one[gi] = 1.0;
      std::memcpy(m->h_small + 16, one.data(), sizeof(double) * m->n_gates);
      CK(cudaMemcpyAsync(m->d_vgate.p, m->h_small + 16, sizeof(double) * m->n_gates, cudaMemcpyHostToDevice, s));
      launch_set_dirichlet(m->nxn, m->nyn, m->nzn, 0, 0.0, m->d_gate_top.as<signed char>(), m->d_vgate.as<double>(),
                           eg, s);
      double* acc = m->stats.as<double>() + 10;
      CK(cudaMemsetAsync(acc, 0, sizeof(double), s));
      launch_dot<double>(n, g, eg, acc, s);
      CK(cudaMemcpyAsync(m->h_small + 30, acc, sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      gD[d * m->n_gates + gi] = m->h_small[30];
    }
    // zero the Dirichlet rows of the right-hand side
    launch_set_dirichlet(m->nxn, m->nyn, m->nzn, m->bottom_ohmic, 0.0, m->d_gate_top.as<signed char>(), zero_v, g, s);
    adjoint_solve(m, o->precision, g, lam, maxk);
    for (int gi = 0; gi < m->n_gates; ++gi) {
      CK(cudaMemsetAsync(eg, 0, n * sizeof(double), s));
      std::vector<double> one(m->n_gates, 0.0);
      one[gi] = 1.0;
      std::memcpy(m->h_small + 16, one.data(), sizeof(double) * m->n_gates);
      CK(cudaMemcpyAsync(m->d_vgate.p, m->h_small + 16, sizeof(double) * m->n_gates, cudaMemcpyHostToDevice, s));
      launch_set_dirichlet(m->nxn, m->nyn, m->nzn, 0, 0.0, m->d_gate_top.as<signed char>(), m->d_vgate.as<double>(),
                           eg, s);
      ApplyArgs<double> a{};
      a.v = eg;
      a.y = Jeg;
      a.c = ensure_pcg<double>(m).c;
      a.raw = 1;
      launch_apply<double>(m->g64.g, a, m->cfg64, s);
      double* acc = m->stats.as<double>() + 11;
      CK(cudaMemsetAsync(acc, 0, sizeof(double), s));
      launch_dot<double>(n, lam, Jeg, acc, s);
      CK(cudaMemcpyAsync(m->h_small + 31, acc, sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      dN_dV[d * m->n_gates + gi] = gD[d * m->n_gates + gi] - m->h_small[31];
    }
    if (dN_dq) {
      launch_theta_gradient(m->nx, m->ny, m->nz, m->g64.g.hx, m->g64.g.hy, m->g64.g.hz, lam, P.qe,
                            dN_dq + (long long)d * m->n_elems, s);
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
  }
  return QCAD_OK;
}

}  // namespace qcad
