// Solver drivers (host): preconditioned CG with device-resident scalars and
// CUDA-graph-captured iteration chunks, the Newton iteration of the nonlinear
// Poisson problem (Sec. II.A.3, which solves it by Newton's method),
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
#include "mg.h"

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
// Iterations per captured graph with the multigrid preconditioner: its solves take a handful of
// iterations, and the iterations captured after convergence still launch (and return at once)
static const int MG_CHUNK = 4;
// Preconditioner code of the geometric multigrid V-cycle (other codes: Chebyshev degree >= 1).
static const int DEG_MG = -1;

template <class T> struct Prec;
template <> struct Prec<double> {
  static PcgBufs<double>& bufs(qcad_mesh_s* m) { return m->k64; }
  static PcgGraph& graph(qcad_mesh_s* m) { return m->graph64; }
  static const Grid<double>& grid(qcad_mesh_s* m) { return m->g64.g; }
  static LaunchCfg cfg(qcad_mesh_s* m) { return m->cfg64; }
  // the charged gates' face coefficients (Robin condition) or null
  static const double* face(qcad_mesh_s* m) { return m->has_robin ? m->d_face64.as<double>() : nullptr; }
  static const int prof_apply = PROF_APPLY64, prof_update = PROF_UPDATE64;
};
template <> struct Prec<float> {
  static PcgBufs<float>& bufs(qcad_mesh_s* m) { return m->k32; }
  static PcgGraph& graph(qcad_mesh_s* m) { return m->graph32; }
  static const Grid<float>& grid(qcad_mesh_s* m) { return m->g32.g; }
  static LaunchCfg cfg(qcad_mesh_s* m) { return m->cfg32; }
  static const float* face(qcad_mesh_s* m) { return m->has_robin ? m->d_face32.as<float>() : nullptr; }
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
  b.w.ensure(nb);
  b.d.ensure(2 * nb);
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
  v.w = b.w.template as<T>();
  v.d[0] = b.d.template as<T>();
  v.d[1] = v.d[0] + (nb / sizeof(T));
  return v;
}

static void ensure_newton(qcad_mesh_s* m) {
  const size_t nb = (size_t)m->n_nodes * sizeof(double) + 64;
  m->phi_a.ensure(nb);
  m->phi_b.ensure(nb);
  m->R.ensure(nb);
}

// One PCG iteration's kernels: apply, update, and for degree >= 2 the Chebyshev steps.
template <class T>
static void enqueue_iteration(qcad_mesh_s* m, const PcgVecs<T>& v, PcgScalars* sc, int degree, cudaStream_t s,
                              std::vector<Profiler::Pair>* ev) {
  auto rec = [&](int idx, bool start) {
    if (ev) {
      Profiler::Pair& p = (*ev)[idx];
      CK(cudaEventRecordWithFlags(start ? p.a : p.b, s, cudaEventRecordExternal));
    }
  };
  int e = 0;
  rec(e, true);
  launch_pcg_apply<T>(Prec<T>::grid(m), v, sc, Prec<T>::cfg(m), s, Prec<T>::face(m));
  rec(e++, false);
  rec(e, true);
  if (degree == DEG_MG) {
    mg_enqueue_update<T>(m, v, sc, s);
    rec(e++, false);
    return;
  }
  if (degree <= 1)
    launch_pcg_update<T>(m->n_nodes, v, sc, s);
  else
    launch_pcg_update_cheb<T>(m->n_nodes, v, sc, s);
  rec(e++, false);
  for (int j = 1; j < degree; ++j) {
    rec(e, true);
    launch_cheb_step<T>(Prec<T>::grid(m), v, sc, j, j == degree - 1, Prec<T>::cfg(m), s, Prec<T>::face(m));
    rec(e++, false);
  }
}

// Captures PCG_CHUNK (MG_CHUNK) iterations into a graph; with profiling on, every kernel is
// bracketed by external event-record nodes (recorded whenever the graph runs).
template <class T>
static void build_graph(qcad_mesh_s* m, const PcgVecs<T>& v, int degree) {
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
  const int per_it = 1 + std::max(1, degree);  // event pairs per iteration (MG: apply, tail)
  const int chunk = degree == DEG_MG ? MG_CHUNK : PCG_CHUNK;
  std::vector<Profiler::Pair> evs;
  if (prof) {
    for (int i = 0; i < per_it * chunk; ++i) {
      Profiler::Pair p;
      CK(cudaEventCreate(&p.a));
      CK(cudaEventCreate(&p.b));
      const int q = i % per_it;
      p.cls = (q == 1) ? (degree == DEG_MG ? PROF_MG : Prec<T>::prof_update) : Prec<T>::prof_apply;
      evs.push_back(p);
    }
  }
  PcgScalars* sc = m->scal.as<PcgScalars>();
  const long long launches_before = launch_count();
  CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  for (int it = 0; it < chunk; ++it) {
    std::vector<Profiler::Pair> sub;
    if (prof) sub.assign(evs.begin() + it * per_it, evs.begin() + (it + 1) * per_it);
    enqueue_iteration<T>(m, v, sc, degree, s, prof ? &sub : nullptr);
  }
  cudaGraph_t graph;
  CK(cudaStreamEndCapture(s, &graph));
  note_launch((int)(launches_before - launch_count()));  // captured kernels run only when replayed
  cudaError_t e = cudaGraphInstantiate(&G.exec, graph, 0);
  cudaGraphDestroy(graph);
  CK(e);
  G.events = evs;
  G.chunk = chunk;
  G.degree = degree;
}

struct PcgResult {
  int iters = 0;
  bool nonfinite = false;
  bool converged = false;
};

// Largest eigenvalue of D^-1 J by power iteration (Rayleigh quotient in the D inner product).
template <class T>
static double lambda_max(qcad_mesh_s* m, int steps) {
  PcgVecs<T> v = ensure_pcg<T>(m);
  cudaStream_t s = m->stream;
  const long long n = m->n_nodes;
  T* x = v.d[0];
  T* y = v.d[1];
  T* xn = v.w;
  launch_random_free<T>(Prec<T>::grid(m), 0x5EEDull, x, s);
  double* acc = m->stats.as<double>() + 48;
  double lam = 0.0;
  for (int it = 0; it < steps; ++it) {
    ApplyArgs<T> a{};
    a.v = x;
    a.y = y;
    a.c = v.c;
    launch_apply<T>(Prec<T>::grid(m), a, Prec<T>::cfg(m), s, Prec<T>::face(m));
    CK(cudaMemsetAsync(acc, 0, 3 * sizeof(double), s));
    launch_power_step<T>(n, x, y, v.dinv, xn, acc, s);
    CK(cudaMemcpyAsync(m->h_small + 40, acc, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double a0 = m->h_small[40], a1 = m->h_small[41], a2 = m->h_small[42];
    if (!(a1 > 0.0) || !(a2 > 0.0)) break;
    lam = a0 / a1;
    launch_scale<T>(n, xn, 1.0 / std::sqrt(a2), s);
    std::swap(x, xn);
  }
  return lam;
}

static double cheb_alpha(int degree) {
  static const char* env = std::getenv("QCAD_CHEB_ALPHA");
  if (env) return std::atof(env);
  return 4.0 * degree * degree;
}

// Solves J x = b (b, dinv, c already in the precision's buffers) to ||r|| <= rtol ||b||
// with Jacobi (degree 1) or Chebyshev-Jacobi (degree >= 2) preconditioning.
template <class T>
static PcgResult pcg_run_once(qcad_mesh_s* m, double rtol, int maxit, int degree, double lam_factor,
                              int fresh_steps) {
  PcgVecs<T> v = ensure_pcg<T>(m);
  PcgGraph& G = Prec<T>::graph(m);
  bool mg = false;
  mg = degree == DEG_MG && mg_prepare(m);
  if (mg) mg_reserve<T>(m);  // level buffers exist before the graph captures their pointers
  degree = mg ? DEG_MG : std::max(1, std::min(degree, 16));
  const bool prof_match = m->prof.on == !G.events.empty();
  if (!G.exec || G.key != (const void*)v.x || !prof_match || G.degree != degree) {
    build_graph<T>(m, v, degree);
    G.key = (const void*)v.x;
  }
  cudaStream_t s = m->stream;
  double lam = 0.0;
  const int pi = sizeof(T) == 8 ? 0 : 1;
  if (degree >= 2) {
    if (fresh_steps == 0 && m->lam_ver[pi] == m->lin_ver[pi]) {
      lam = m->lam_cache[pi];
    } else {
      // the cache keeps the estimate scaled so that the default margin reproduces this bound
      lam = lambda_max<T>(m, fresh_steps > 0 ? fresh_steps : 12) * (lam_factor / 1.1);
      m->lam_cache[pi] = lam;
      m->lam_ver[pi] = m->lin_ver[pi];
    }
  }
  PcgScalars* h = m->h_scal;
  std::memset(h, 0, sizeof(PcgScalars));
  h->tol2 = rtol * rtol;
  h->maxit = maxit;
  h->degree = degree;
  if (degree >= 2) {
    // Chebyshev interval [b/alpha, b] of D^-1 J with b = 1.1 lambda_max
    const double bmax = 1.1 * (lam > 0 ? lam : 2.0), amin = bmax / cheb_alpha(degree);  // lam carries the margin
    h->theta = 0.5 * (bmax + amin);
    h->delta = 0.5 * (bmax - amin);
  } else {
    h->theta = 1.0;
    h->delta = 0.5;
  }
  PcgScalars* sc = m->scal.as<PcgScalars>();
  CK(cudaMemcpyAsync(sc, h, sizeof(PcgScalars), cudaMemcpyHostToDevice, s));
  if (mg) {
    mg_setup<T>(m, s);
    mg_enqueue_init<T>(m, v, sc, s);
  } else if (degree <= 1) {
    launch_pcg_init<T>(m->n_nodes, v, sc, s);
  } else {
    launch_pcg_init_cheb<T>(m->n_nodes, v, sc, s);
    for (int j = 1; j < degree; ++j) launch_cheb_step<T>(Prec<T>::grid(m), v, sc, j, j == degree - 1, Prec<T>::cfg(m), s, Prec<T>::face(m));
  }
  CK(cudaGetLastError());
  int t_prev = 0;
  int guard = 0;
  const int per_it = mg ? 2 : 1 + degree;  // event pairs per iteration
  const int launches_it = mg ? mg_launches_per_iteration(m) : 1 + degree;
  for (;;) {
    CK(cudaGraphLaunch(G.exec, s));
    note_launch(launches_it * G.chunk);
    CK(cudaMemcpyAsync(h, sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (m->prof.on) {
      const int ran = std::min(G.chunk, h->t - t_prev);
      for (int it = 0; it < ran; ++it) {
        for (int q = 0; q < per_it; ++q) {
          Profiler::Pair& p = G.events[it * per_it + q];
          float ms = 0.f;
          if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            m->prof.add(p.cls, ms);
          } else {
            cudaGetLastError();
          }
        }
      }
    }
    t_prev = h->t;
    if (h->done) break;
    if (++guard > maxit / G.chunk + 4) break;
  }
  PcgResult r;
  r.iters = h->t;
  r.nonfinite = h->nonfinite != 0;
  r.converged = h->done && !h->nonfinite && (h->rr0 == 0.0 || h->rr[h->t & 3] <= h->tol2 * h->rr0);
  return r;
}

// Chebyshev degree autotuner: times complete solves of the current system for each
// candidate degree and keeps the fastest for the mesh and precision (once per mesh).
// PCG with the given preconditioner degree. A Chebyshev breakdown (the polynomial is not
// positive on the whole spectrum when the power iteration underestimates its top) is retried
// once with a 60-step estimate and a 30 % margin, then with Jacobi.
template <class T>
static PcgResult pcg_run(qcad_mesh_s* m, double rtol, int maxit, int degree = 1) {
  PcgResult r = pcg_run_once<T>(m, rtol, maxit, degree, 1.1, 0);
  if (r.nonfinite && degree == DEG_MG) {
    if (debug_on()) std::fprintf(stderr, "[qcad] multigrid PCG breakdown: retrying with Jacobi\n");
    return pcg_run_once<T>(m, rtol, maxit, 1, 1.1, 0);
  }
  if (!r.nonfinite || degree < 2) return r;
  if (debug_on()) std::fprintf(stderr, "[qcad] chebyshev breakdown at degree %d: re-estimating\n", degree);
  r = pcg_run_once<T>(m, rtol, maxit, degree, 1.3, 60);
  if (!r.nonfinite) return r;
  return pcg_run_once<T>(m, rtol, maxit, 1, 1.1, 0);
}

template <class T>
static int choose_degree(qcad_mesh_s* m, double rtol, int maxit) {
  const int prec = sizeof(T) == 8 ? 0 : 1;
  if (m->cheb_auto[prec] != 0) return m->cheb_auto[prec];
  // odd degrees only: their polynomial stays positive above the estimated top of the spectrum,
  // so an underestimated lambda_max slows the solve but cannot make it break down; the multigrid
  // V-cycle (in the solve's own precision) competes too
  std::vector<int> cand = {1, 3, 5, 7};
  if (mg_prepare(m)) cand.push_back(DEG_MG);
  int best = 1;
  double best_t = 1e300;
  for (int d : cand) {
    // a first untimed run builds the candidate's graph; the timed run then pays what every
    // new linearization pays (the power iteration, or the multigrid setup)
    pcg_run<T>(m, rtol, maxit, d);
    if (d == DEG_MG) mg_invalidate(m);
    const int pi = sizeof(T) == 8 ? 0 : 1;
    m->lam_ver[pi] = -1;
    CK(cudaStreamSynchronize(m->stream));
    const auto t0 = std::chrono::steady_clock::now();
    PcgResult r = pcg_run<T>(m, rtol, maxit, d);
    const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (debug_on()) std::fprintf(stderr, "[qcad] cheb degree %d: %d iterations, %.3f ms\n", d, r.iters, 1e3 * dt);
    if (r.converged && dt < best_t) {
      best_t = dt;
      best = d;
    }
  }
  m->cheb_auto[prec] = best;
  return best;
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
  // prec 0: the FP64 linearization, 1: the FP32 one, 2: both from the one evaluation
  if (prec == 0 || prec == 2) {
    PcgVecs<double> v = ensure_pcg<double>(m);
    a.c64 = const_cast<double*>(v.c);
    a.dinv64 = const_cast<double*>(v.dinv);
    a.b64 = const_cast<double*>(v.b);
  }
  if (prec == 1 || prec == 2) {
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
  if (m->qd_active) a.qd = m->qd;  // predictor density in the quantum region (Sec. II.C)
  a.wq = m->d_wq.as<double>();
  a.ecode = m->d_ecode.as<unsigned char>();
  if (m->has_surface) a.bsurf = m->d_bsurf.as<double>();  // charged gates, surface charges
  CK(cudaMemsetAsync(a.stats, 0, 2 * sizeof(double), s));
  if (counts_out) {
    a.counts = m->counts.as<double>();
    CK(cudaMemsetAsync(a.counts, 0, QCAD_MAX_DOTS_K * sizeof(double), s));
  }
  Profiler::Pair pp;
  if (m->prof.on) m->prof.begin(PROF_RESIDUAL, s, pp);
  m->el_res.ensure((size_t)16 * m->n_elems * sizeof(double) + 64);
  launch_residual_2pass(m->g64.g, a, m->el_res.as<double>(), m->cfg_res, s, Prec<double>::face(m));
  if (prec != 1) m->lin_ver[0] += 1;  // the stored linearizations changed
  if (prec != 0) m->lin_ver[1] += 1;
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

// Top plane of the surface load b at the bias: the charged gates' (eps_r/d) phi_0 int_f N_a (the
// Robin condition, Sec. II.A.4; phi_0 of Eq. ContOnIns) on top of the bias-independent sheets.
static void update_surface_load(qcad_mesh_s* m, const qcad_bias* b, const Phys& P) {
  if (!m->has_robin) return;
  const long long plane = (long long)m->nxn * m->nyn;
  m->btop = m->bsig_top;
  for (size_t c = 0; c < m->charged_gate.size(); ++c) {
    const double v = gate_value(m, b->V_gate[m->charged_gate[c]], P);
    const std::vector<double>& r = m->charged_r[c];
    for (long long q = 0; q < plane; ++q) m->btop[q] += v * r[q];
  }
  CK(cudaMemcpyAsync(m->d_bsurf.as<double>() + (size_t)m->nz * plane, m->btop.data(), plane * sizeof(double),
                     cudaMemcpyHostToDevice, m->stream));
  CK(cudaStreamSynchronize(m->stream));
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
  update_surface_load(m, b, P);
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
  int degree = o->cheb_degree != 0 ? o->cheb_degree : m->cheb_auto[prec];
  if (!o->warm_start) {
    // Laplace initial guess with the contact values (rho = 0), solved to 1e-3: it only starts
    // the Newton iteration, whose first step replaces it by the nonlinear correction
    eval_residual(m, P, pa, theta, 1, prec, nullptr);
    if (degree == 0) degree = choose_degree<T>(m, 1e-3, maxk);
    PcgResult pr = pcg_run<T>(m, 1e-3, maxk, degree);
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
    // no tighter than the tolerance needs: the linear part of the next residual, eta ||R||_2,
    // at a tenth of tol_R bounds its max norm below tol_R
    if (nR > 0) eta = std::max(eta, std::min(1e-2, 0.1 * o->newton_tol_R / nR));
    if (degree == 0) degree = choose_degree<T>(m, eta, maxk);
    PcgResult pr = pcg_run<T>(m, eta, maxk, degree);
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
  if (o->cheb_degree < -1 || o->cheb_degree > 16) throw Error(QCAD_ERR_INVALID_ARG, "cheb_degree must be in [-1, 16]");
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
  update_surface_load(m, b, P);
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
    launch_apply<double>(m->g64.g, a, m->cfg64, s, Prec<double>::face(m));
  } else {
    PcgVecs<float> v = ensure_pcg<float>(m);
    launch_d2f(m->n_nodes, vin, v.r, s);
    ApplyArgs<float> a{};
    a.v = v.r;
    a.y = v.Ap;
    a.c = v.c;
    launch_apply<float>(m->g32.g, a, m->cfg32, s, Prec<float>::face(m));
    launch_f2d(m->n_nodes, v.Ap, y, s);
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return QCAD_OK;
}

// Element box of dot d: the elements whose centroid lies in its coordinate box (a box again, the
// node planes being sorted); false when it is empty.
static bool dot_element_box(const qcad_mesh_s* m, int d, int box[6]) {
  const double* B = m->dots.b[d];
  const std::vector<double>* c[3] = {&m->xc, &m->yc, &m->zc};
  for (int a = 0; a < 3; ++a) {
    const std::vector<double>& x = *c[a];
    int lo = -1, hi = -1;
    for (int i = 0; i + 1 < (int)x.size(); ++i) {
      const double xc = 0.5 * (x[i] + x[i + 1]);
      if (xc >= B[2 * a] && xc <= B[2 * a + 1]) {
        if (lo < 0) lo = i;
        hi = i + 1;
      }
    }
    if (lo < 0) return false;
    box[2 * a] = lo;
    box[2 * a + 1] = hi;
  }
  return true;
}

qcad_status electron_counts(qcad_mesh_s* m, const qcad_bias* b, const double* theta, const double* phi, double* N) {
  validate_bias(m, b);
  if (!phi || !N) throw Error(QCAD_ERR_INVALID_ARG, "null pointer");
  ensure_newton(m);
  const Phys P = make_phys(m, b);
  // the dots' element boxes; overlapping boxes (an element counts for the first dot that holds it)
  // take the residual's fused count instead
  int boxes[QCAD_MAX_DOTS_K][6];
  bool have[QCAD_MAX_DOTS_K];
  bool overlap = false;
  for (int d = 0; d < m->dots.n; ++d) {
    have[d] = dot_element_box(m, d, boxes[d]);
    for (int e = 0; e < d && have[d]; ++e)
      if (have[e] && boxes[d][0] < boxes[e][1] && boxes[e][0] < boxes[d][1] && boxes[d][2] < boxes[e][3] &&
          boxes[e][2] < boxes[d][3] && boxes[d][4] < boxes[e][5] && boxes[e][4] < boxes[d][5])
        overlap = true;
  }
  if (overlap) {
    eval_residual(m, P, phi, theta, 0, 0, N);
    return QCAD_OK;
  }
  cudaStream_t s = m->stream;
  double* acc = m->counts.as<double>();
  CK(cudaMemsetAsync(acc, 0, QCAD_MAX_DOTS_K * sizeof(double), s));
  for (int d = 0; d < m->dots.n; ++d)
    if (have[d]) launch_dot_count(m->g64.g, phi, m->d_layer_semi.as<unsigned char>(), P, boxes[d], acc + d, s);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(m->h_small + 8, acc, QCAD_MAX_DOTS_K * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int d = 0; d < m->dots.n; ++d) N[d] = m->h_small[8 + d];
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

// ---------------------------------------------------------------------------
// Batched form: n independent meshes (uneven sizes, own biases) solved by a
// lockstep Newton iteration. Every device pass covers all instances at once:
// the FP64 residual (with the FP32 linearization) is one launch over a work
// table of (instance, tile), each PCG iteration is one apply launch and one
// update launch over work tables (chunks of 8 iterations captured once as a
// CUDA graph, instances dropping out on their own device-resident scalars),
// and the line search evaluates the trial points of all instances still
// searching in one residual launch. FP32 Krylov with Jacobi preconditioning,
// FP64 residual and Newton update per instance.
struct BatchCtx {
  int n = 0;
  cudaStream_t s = nullptr;
  std::vector<qcad_mesh_s*> ms;       // mesh of each entry (entries may share a mesh)
  std::vector<PcgVecs<float>> vecs;   // FP32 PCG vectors of each entry
  std::vector<PcgScalars*> scd;       // device PCG scalars of each entry
  std::vector<int> kch;               // z chunk of each entry's apply
  std::vector<Phys> P;
  DevBuf tab_a, tab_v, tab_r, status, rstats;
  int total_a = 0, total_v = 0;
  int* h_status = nullptr;
  double* h_rstats = nullptr;
  PcgScalars* h_sc = nullptr;         // pinned host staging of the entries' scalars
  cudaGraphExec_t exec = nullptr;
  // streams the entries' multigrid PCG graphs are spread over (instances run concurrently), with
  // the events that fork them from s and join them back
  static constexpr int NPOOL = 8;
  cudaStream_t pool[NPOOL] = {};
  cudaEvent_t fork = nullptr, join[NPOOL] = {};
  void ensure_pool() {
    if (fork) return;
    CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    for (int k = 0; k < NPOOL; ++k) {
      CK(cudaStreamCreateWithFlags(&pool[k], cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&join[k], cudaEventDisableTiming));
    }
  }
  ~BatchCtx() {
    for (int k = 0; k < NPOOL; ++k) {
      if (pool[k]) cudaStreamDestroy(pool[k]);
      if (join[k]) cudaEventDestroy(join[k]);
    }
    if (fork) cudaEventDestroy(fork);
    if (exec) cudaGraphExecDestroy(exec);
    if (h_status) cudaFreeHost(h_status);
    if (h_rstats) cudaFreeHost(h_rstats);
    if (h_sc) cudaFreeHost(h_sc);
  }
};

static void batch_setup(BatchCtx& B) {
  std::vector<BatchApplyEntry> ta(B.n);
  std::vector<BatchVecEntry> tv(B.n);
  int ba = 0, bv = 0;
  for (int i = 0; i < B.n; ++i) {
    qcad_mesh_s* m = B.ms[i];
    const PcgVecs<float>& v = B.vecs[i];
    BatchApplyEntry& a = ta[i];
    a.g = m->g32.g;
    a.v = v;
    a.sc = B.scd[i];
    a.kchunk = std::min(128, std::max(2, B.kch[i] > 0 ? B.kch[i] : 16));
    a.tiles_x = (m->g32.g.nxn + 29) / 30;  // plane-factorized tiles: 30 x 14 interior nodes
    a.tiles_y = (m->g32.g.nyn + 13) / 14;
    a.begin = ba;
    ba += a.tiles_x * a.tiles_y * ((m->g32.g.nzn + a.kchunk - 1) / a.kchunk);
    BatchVecEntry& e = tv[i];
    e.v = v;
    e.sc = a.sc;
    e.n = (int)m->n_nodes;
    e.blocks = std::max(1, (int)((m->n_nodes + 2047) / 2048));
    e.begin = bv;
    bv += e.blocks;
  }
  B.total_a = ba;
  B.total_v = bv;
  B.tab_a.ensure(ta.size() * sizeof(BatchApplyEntry) + 64);
  B.tab_v.ensure(tv.size() * sizeof(BatchVecEntry) + 64);
  B.tab_r.ensure((size_t)B.n * sizeof(BatchResEntry) + 64);
  B.status.ensure((size_t)4 * B.n * sizeof(int) + 64);
  B.rstats.ensure((size_t)3 * B.n * sizeof(double) + 64);
  CK(cudaMemcpyAsync(B.tab_a.p, ta.data(), ta.size() * sizeof(BatchApplyEntry), cudaMemcpyHostToDevice, B.s));
  CK(cudaMemcpyAsync(B.tab_v.p, tv.data(), tv.size() * sizeof(BatchVecEntry), cudaMemcpyHostToDevice, B.s));
  CK(cudaMallocHost(&B.h_status, (size_t)4 * B.n * sizeof(int)));
  CK(cudaMallocHost(&B.h_rstats, (size_t)3 * B.n * sizeof(double)));
  CK(cudaMallocHost(&B.h_sc, (size_t)B.n * sizeof(PcgScalars)));
  CK(cudaStreamSynchronize(B.s));
  const long long before = launch_count();
  CK(cudaStreamBeginCapture(B.s, cudaStreamCaptureModeThreadLocal));
  for (int it = 0; it < PCG_CHUNK; ++it) {
    launch_batch_lin_apply(B.tab_a.as<BatchApplyEntry>(), B.n, B.total_a, B.s);
    launch_batch_pcg_update(B.tab_v.as<BatchVecEntry>(), B.n, B.total_v, B.s);
  }
  launch_batch_status(B.tab_v.as<BatchVecEntry>(), B.n, B.status.as<int>(), B.s);
  cudaGraph_t graph;
  CK(cudaStreamEndCapture(B.s, &graph));
  note_launch((int)(before - launch_count()));
  cudaError_t e = cudaGraphInstantiate(&B.exec, graph, 0);
  cudaGraphDestroy(graph);
  CK(e);
}

// FP64 residuals of the instances `idx` at phi[i] in one launch (mixed linearization written
// for each); R[i] = {max |R|, sum R^2} and, when `trial`, step[i] = the trial slot (max |alpha
// delta| written by the trial kernels before).
static void batch_residual(BatchCtx& B, const std::vector<int>& idx, const std::vector<double*>& phi, int linear,
                           std::vector<ResStats>& R, std::vector<double>* step) {
  if (idx.empty()) return;
  std::vector<BatchResEntry> tr(idx.size());
  int total = 0, total_q = 0;
  for (size_t q = 0; q < idx.size(); ++q) {
    const int i = idx[q];
    qcad_mesh_s* m = B.ms[i];
    PcgVecs<float> v = ensure_pcg<float>(m);
    BatchResEntry& e = tr[q];
    e = BatchResEntry{};
    e.g = m->g64.g;
    ResidualArgs& a = e.a;
    a.phi = phi[i];
    a.R = m->R.as<double>();
    a.c32 = const_cast<float*>(v.c);
    a.dinv32 = const_cast<float*>(v.dinv);
    a.b32 = const_cast<float*>(v.b);
    a.layer_semi = m->d_layer_semi.as<unsigned char>();
    a.xn = m->d_xn.as<double>();
    a.yn = m->d_yn.as<double>();
    a.zn = m->d_zn.as<double>();
    a.P = B.P[i];
    a.dots = m->dots;
    a.linear = linear;
    a.stats = m->stats.as<double>();
    a.wq = m->d_wq.as<double>();
    a.ecode = m->d_ecode.as<unsigned char>();
    e.kchunk = std::max(2, m->cfg_res.kchunk);
    e.tiles_x = (e.g.nxn + QCAD_BX - 3) / (QCAD_BX - 2);
    e.tiles_y = (e.g.nyn + 8 - 3) / (8 - 2);
    e.begin = total;
    total += e.tiles_x * e.tiles_y * ((e.g.nzn + e.kchunk - 1) / e.kchunk);
    m->el_res.ensure((size_t)16 * m->n_elems * sizeof(double) + 64);
    e.el = m->el_res.as<double>();
    e.qbegin = total_q;
    total_q += (int)((8 * m->n_elems + 255) / 256);
    m->lin_ver[1] += 1;  // the FP32 linearization of this mesh is rewritten
  }
  const int nq = (int)idx.size();
  CK(cudaMemcpyAsync(B.tab_r.p, tr.data(), tr.size() * sizeof(BatchResEntry), cudaMemcpyHostToDevice, B.s));
  const BatchResEntry* tab = B.tab_r.as<BatchResEntry>();
  launch_batch_stats(tab, nq, 0, nullptr, B.s);
  launch_batch_residual_2pass(tab, nq, total_q, total, B.s);
  launch_batch_stats(tab, nq, 2, B.rstats.as<double>(), B.s);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(B.h_rstats, B.rstats.p, (size_t)3 * nq * sizeof(double), cudaMemcpyDeviceToHost, B.s));
  CK(cudaStreamSynchronize(B.s));
  for (int q = 0; q < nq; ++q) {
    R[idx[q]].rmax = B.h_rstats[3 * q];
    R[idx[q]].r2 = B.h_rstats[3 * q + 1];
    if (step) (*step)[idx[q]] = B.h_rstats[3 * q + 2];
  }
}

// One batched linear solve: instance i solves its J x = b to rtol[i] (rtol[i] <= 0: skipped).
static void batch_pcg(BatchCtx& B, const std::vector<double>& rtol, int maxit, std::vector<int>& iters,
                      std::vector<int>& nonfinite) {
  for (int i = 0; i < B.n; ++i) {
    PcgScalars* h = B.h_sc + i;
    std::memset(h, 0, sizeof(PcgScalars));
    h->tol2 = rtol[i] * rtol[i];
    h->maxit = maxit;
    h->degree = 1;
    h->phase = 1;
    h->theta = 1.0;
    h->delta = 0.5;
    if (!(rtol[i] > 0)) h->done = 1;
  }
  CK(cudaMemcpyAsync(B.scd[0], B.h_sc, sizeof(PcgScalars), cudaMemcpyHostToDevice, B.s));
  for (int i = 1; i < B.n; ++i)
    CK(cudaMemcpyAsync(B.scd[i], B.h_sc + i, sizeof(PcgScalars), cudaMemcpyHostToDevice, B.s));
  for (int i = 0; i < B.n; ++i)
    if (rtol[i] > 0) launch_pcg_init<float>(B.ms[i]->n_nodes, B.vecs[i], B.scd[i], B.s);
  CK(cudaGetLastError());
  int guard = 0;
  for (;;) {
    CK(cudaGraphLaunch(B.exec, B.s));
    note_launch(2 * PCG_CHUNK + 1);
    CK(cudaMemcpyAsync(B.h_status, B.status.p, (size_t)4 * B.n * sizeof(int), cudaMemcpyDeviceToHost, B.s));
    CK(cudaStreamSynchronize(B.s));
    bool all = true;
    for (int i = 0; i < B.n; ++i) all = all && B.h_status[4 * i] != 0;
    if (all || ++guard > maxit / PCG_CHUNK + 4) break;
  }
  iters.assign(B.n, 0);
  nonfinite.assign(B.n, 0);
  for (int i = 0; i < B.n; ++i) {
    iters[i] = rtol[i] > 0 ? B.h_status[4 * i + 1] : 0;
    nonfinite[i] = B.h_status[4 * i + 2];
  }
}

// The batched linear solve with each instance's multigrid-preconditioned PCG: every round
// replays the captured 4-iteration graph of each unfinished instance back to back on the batch
// stream, then one status gather and one host read serve all instances.
static void batch_pcg_mg(BatchCtx& B, const std::vector<double>& rtol, int maxit, std::vector<int>& iters,
                         std::vector<int>& nonfinite) {
  for (int i = 0; i < B.n; ++i) {
    qcad_mesh_s* m = B.ms[i];
    PcgGraph& G = m->graph32;
    const bool prof_match = m->prof.on == !G.events.empty();
    mg_reserve<float>(m);  // level buffers exist before the graph captures their pointers
    if (!G.exec || G.key != (const void*)B.vecs[i].x || !prof_match || G.degree != DEG_MG) {
      build_graph<float>(m, B.vecs[i], DEG_MG);
      G.key = (const void*)B.vecs[i].x;
    }
  }
  // each entry's scalars, multigrid setup and PCG start on the stream pool (entries are distinct
  // meshes), joined back into s
  B.ensure_pool();
  CK(cudaEventRecord(B.fork, B.s));
  for (int k = 0; k < BatchCtx::NPOOL; ++k) CK(cudaStreamWaitEvent(B.pool[k], B.fork, 0));
  for (int i = 0; i < B.n; ++i) {
    qcad_mesh_s* m = B.ms[i];
    cudaStream_t ps = B.pool[i % BatchCtx::NPOOL];
    PcgScalars* h = B.h_sc + i;
    std::memset(h, 0, sizeof(PcgScalars));
    h->tol2 = rtol[i] * rtol[i];
    h->maxit = maxit;
    h->degree = DEG_MG;
    h->theta = 1.0;
    h->delta = 0.5;
    if (!(rtol[i] > 0)) h->done = 1;
    CK(cudaMemcpyAsync(B.scd[i], h, sizeof(PcgScalars), cudaMemcpyHostToDevice, ps));
    if (rtol[i] > 0) {
      mg_setup<float>(m, ps);
      mg_enqueue_init<float>(m, B.vecs[i], B.scd[i], ps);
    }
  }
  for (int k = 0; k < BatchCtx::NPOOL; ++k) {
    CK(cudaEventRecord(B.join[k], B.pool[k]));
    CK(cudaStreamWaitEvent(B.s, B.join[k], 0));
  }
  CK(cudaGetLastError());
  std::vector<char> active(B.n);
  for (int i = 0; i < B.n; ++i) active[i] = rtol[i] > 0;
  int guard = 0;
  for (;;) {
    // each active entry's chunk of PCG iterations (its captured graph), the entries spread over
    // the stream pool so that the small instances' kernels overlap
    CK(cudaEventRecord(B.fork, B.s));
    for (int k = 0; k < BatchCtx::NPOOL; ++k) CK(cudaStreamWaitEvent(B.pool[k], B.fork, 0));
    int slot = 0;
    for (int i = 0; i < B.n; ++i) {
      if (!active[i]) continue;
      CK(cudaGraphLaunch(B.ms[i]->graph32.exec, B.pool[slot++ % BatchCtx::NPOOL]));
      note_launch(mg_launches_per_iteration(B.ms[i]) * B.ms[i]->graph32.chunk);
    }
    for (int k = 0; k < BatchCtx::NPOOL; ++k) {
      CK(cudaEventRecord(B.join[k], B.pool[k]));
      CK(cudaStreamWaitEvent(B.s, B.join[k], 0));
    }
    launch_batch_status(B.tab_v.as<BatchVecEntry>(), B.n, B.status.as<int>(), B.s);
    CK(cudaMemcpyAsync(B.h_status, B.status.p, (size_t)4 * B.n * sizeof(int), cudaMemcpyDeviceToHost, B.s));
    CK(cudaStreamSynchronize(B.s));
    bool any = false;
    for (int i = 0; i < B.n; ++i) {
      if (active[i] && B.h_status[4 * i] != 0) active[i] = 0;
      any = any || active[i];
    }
    if (!any || ++guard > maxit / MG_CHUNK + 4) break;
  }
  iters.assign(B.n, 0);
  nonfinite.assign(B.n, 0);
  for (int i = 0; i < B.n; ++i) {
    iters[i] = rtol[i] > 0 ? B.h_status[4 * i + 1] : 0;
    nonfinite[i] = B.h_status[4 * i + 2];
  }
}

// ---------------------------------------------------------------------------
// Adjoint sensitivities of the dot counts (Sec. III's capacitance by the adjoint): one linear
// solve J lam_d = dN_d/dphi per dot (free rows), then dN_d/dV_g = dN_d/dphi_D . e_g -
// lam_d . (J e_g) with e_g the unit lift of gate g, and dN_d/dtheta_e = (q/eps0)(|e|/8) sum of
// lam_d over the corners of e.

// FP64 solve of one right-hand side (precision 0).
static void adjoint_solve64(qcad_mesh_s* m, const double* g, double* lam, int maxk, int degree) {
  cudaStream_t s = m->stream;
  PcgVecs<double> v = ensure_pcg<double>(m);
  CK(cudaMemcpyAsync(const_cast<double*>(v.b), g, m->n_nodes * sizeof(double), cudaMemcpyDeviceToDevice, s));
  PcgResult pr = pcg_run<double>(m, 1e-13, maxk, degree);
  if (pr.nonfinite) throw Error(QCAD_ERR_NONFINITE, "adjoint linear solve produced a non-finite value");
  CK(cudaMemcpyAsync(lam, v.x, m->n_nodes * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
}

// Mixed precision, one right-hand side with the multigrid-preconditioned FP32 PCG: corrections
// to a tenth of the 1e-13 target of ||g - J lam|| / ||g||, each followed by the FP64 residual.
static void adjoint_solve_mixed_mg(qcad_mesh_s* m, const double* g, double* lam, int maxk) {
  cudaStream_t s = m->stream;
  const long long n = m->n_nodes;
  PcgVecs<double> v = ensure_pcg<double>(m);
  PcgVecs<float> w = ensure_pcg<float>(m);
  m->scratch.ensure(2 * n * sizeof(double) + 64);
  double* y = m->scratch.as<double>();
  double* r = y + n;
  CK(cudaMemsetAsync(lam, 0, n * sizeof(double), s));
  launch_d2f(n, g, const_cast<float*>(w.b), s);
  double* d2 = m->stats.as<double>() + 12;
  CK(cudaMemsetAsync(d2, 0, sizeof(double), s));
  launch_dot<double>(n, g, g, d2, s);
  CK(cudaMemcpyAsync(m->h_small + 20, d2, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const double g2 = m->h_small[20];
  double r2 = g2;
  for (int rf = 0; rf < 12 && r2 > 1e-26 * g2; ++rf) {
    const double rt = std::max(1e-5, std::min(1e-2, 1e-14 * std::sqrt(g2 / std::max(r2, 1e-300))));
    PcgResult pr = pcg_run<float>(m, rt, maxk, DEG_MG);
    if (pr.nonfinite) throw Error(QCAD_ERR_NONFINITE, "adjoint refinement produced a non-finite value");
    launch_axpy<float>(n, 1.0, w.x, lam, s);
    ApplyArgs<double> a{};
    a.v = lam;
    a.y = y;
    a.c = v.c;
    launch_apply<double>(m->g64.g, a, m->cfg64, s, Prec<double>::face(m));
    launch_sub(n, g, y, r, const_cast<float*>(w.b), s);
    CK(cudaMemsetAsync(d2, 0, sizeof(double), s));
    launch_dot<double>(n, r, r, d2, s);
    CK(cudaMemcpyAsync(m->h_small + 20, d2, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    r2 = m->h_small[20];
  }
}

struct AdjCtx {
  int nd = 0, kc = 0;
  const float* x0 = nullptr;
  BatchCtx B;
};

// Mixed precision, all dots at once: FP32 Jacobi-PCG corrections of the nd systems advance
// together (one apply launch and one update launch per iteration for every right-hand side,
// the batched form's kernels over a table of nd entries on this mesh), each round followed by
// the FP64 residuals g_d - J lam_d, until every residual is below 1e-13 ||g_d||.
static void adjoint_solve_mixed(qcad_mesh_s* m, int nd, const double* G, double* LAM, int maxk) {
  cudaStream_t s = m->stream;
  const long long n = m->n_nodes;
  PcgVecs<double> v64 = ensure_pcg<double>(m);
  PcgVecs<float> w0 = ensure_pcg<float>(m);
  const int kc = (m->cfg32.variant == 3 && m->cfg32.by == 8) ? m->cfg32.kchunk : 16;
  // the context (work tables and the captured PCG graph) is kept on the mesh while the
  // right-hand side count, the chunk and the vectors stay the same
  std::shared_ptr<AdjCtx> ctx = std::static_pointer_cast<AdjCtx>(m->adj_ctx);
  if (!ctx || ctx->nd != nd || ctx->kc != kc || ctx->x0 != w0.x) {
    m->adj_ctx.reset();
    ctx = std::make_shared<AdjCtx>();
    ctx->nd = nd;
    ctx->kc = kc;
    ctx->x0 = w0.x;
    m->scal_x.ensure((size_t)nd * sizeof(PcgScalars) + 64);
    BatchCtx& B = ctx->B;
    B.n = nd;
    B.s = s;
    const size_t nb = (size_t)n * sizeof(float) + 64;
    for (int d = 0; d < nd; ++d) {
      PcgVecs<float> v = w0;
      if (d > 0) {
        PcgBufs<float>& k = m->k32x[d - 1];
        k.x.ensure(nb);
        k.r.ensure(nb);
        k.z.ensure(nb);
        k.p.ensure(2 * nb);
        k.Ap.ensure(nb);
        k.b.ensure(nb);
        v.x = k.x.as<float>();
        v.r = k.r.as<float>();
        v.z = k.z.as<float>();
        v.p[0] = k.p.as<float>();
        v.p[1] = v.p[0] + nb / sizeof(float);
        v.Ap = k.Ap.as<float>();
        v.b = k.b.as<float>();  // dinv and c are the shared linearization
      }
      B.ms.push_back(m);
      B.vecs.push_back(v);
      B.scd.push_back(d == 0 ? m->scal.as<PcgScalars>() : m->scal_x.as<PcgScalars>() + d);
      B.kch.push_back(kc);
    }
    batch_setup(B);
    m->adj_ctx = ctx;
  }
  BatchCtx& B = ctx->B;
  m->scratch.ensure((size_t)(nd + 1) * n * sizeof(double) + 64);
  double* y = m->scratch.as<double>();
  double* Rr = y + n;
  double* d2 = m->stats.as<double>() + 12;  // nd <= 8 squared norms
  CK(cudaMemsetAsync(LAM, 0, (size_t)nd * n * sizeof(double), s));
  CK(cudaMemsetAsync(d2, 0, nd * sizeof(double), s));
  for (int d = 0; d < nd; ++d) {
    const double* g = G + (size_t)d * n;
    CK(cudaMemcpyAsync(Rr + (size_t)d * n, g, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    launch_d2f(n, g, const_cast<float*>(B.vecs[d].b), s);
    launch_dot<double>(n, g, g, d2 + d, s);
  }
  CK(cudaMemcpyAsync(m->h_small + 20, d2, nd * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<double> g2(m->h_small + 20, m->h_small + 20 + nd), r2 = g2, rtol(nd);
  std::vector<int> iters, nonf;
  for (int rf = 0; rf < 12; ++rf) {
    bool any = false;
    for (int d = 0; d < nd; ++d) {
      rtol[d] = 0.0;
      if (r2[d] <= 1e-26 * g2[d]) continue;
      any = true;
      // each correction needs only to bring the residual to a tenth of the 1e-13 target
      rtol[d] = std::max(1e-5, std::min(1e-2, 1e-14 * std::sqrt(g2[d] / std::max(r2[d], 1e-300))));
    }
    if (!any) break;
    batch_pcg(B, rtol, maxk, iters, nonf);
    CK(cudaMemsetAsync(d2, 0, nd * sizeof(double), s));
    for (int d = 0; d < nd; ++d) {
      if (!(rtol[d] > 0)) continue;
      if (nonf[d]) throw Error(QCAD_ERR_NONFINITE, "adjoint refinement produced a non-finite value");
      double* lam = LAM + (size_t)d * n;
      double* r = Rr + (size_t)d * n;
      launch_axpy<float>(n, 1.0, B.vecs[d].x, lam, s);
      ApplyArgs<double> a{};
      a.v = lam;
      a.y = y;
      a.c = v64.c;
      launch_apply<double>(m->g64.g, a, m->cfg64, s, Prec<double>::face(m));
      launch_sub(n, G + (size_t)d * n, y, r, const_cast<float*>(B.vecs[d].b), s);
      launch_dot<double>(n, r, r, d2 + d, s);
    }
    CK(cudaMemcpyAsync(m->h_small + 20, d2, nd * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int d = 0; d < nd; ++d)
      if (rtol[d] > 0) r2[d] = m->h_small[20 + d];
  }
}

// The adjoint of one mesh in three phases: prepare (linearizations at phi, the right-hand sides
// G_d = dN_d/dphi with their Dirichlet rows zeroed, the gate lifts' raw J e_g and dN_d/dphi . e_g),
// the linear solves J lam_d = G_d (filled into LAM by the caller), and finish (dN_d/dV_g and dN/dtheta).
struct AdjWork {
  qcad_mesh_s* m = nullptr;
  const qcad_bias* b = nullptr;
  Phys P{};
  int nd = 0, ng = 0;
  DevBuf work, accs;
  double *G = nullptr, *LAM = nullptr, *JE = nullptr, *eg = nullptr, *acc = nullptr, *zero_v = nullptr;
};

static void adjoint_prepare(AdjWork& A, qcad_mesh_s* m, const qcad_bias* b, const qcad_solver_opts* o,
                            const double* phi, const double* theta) {
  cudaStream_t s = m->stream;
  const long long n = m->n_nodes;
  A.m = m;
  A.b = b;
  A.nd = m->dots.n;
  A.ng = m->n_gates;
  const int nd = A.nd, ng = A.ng;
  ensure_newton(m);
  A.P = make_phys(m, b);
  const Phys& P = A.P;
  // linearization at phi in FP64 (and FP32 for the mixed refinement)
  eval_residual(m, P, phi, theta, 0, o->precision == 1 ? 2 : 0, nullptr);
  const long long plane2 = 2LL * m->nxn * m->nyn;  // the top two node planes
  A.work.ensure(((size_t)(2 * nd + 1) * n + (size_t)std::max(ng, 1) * plane2) * sizeof(double) + 64);
  double* G = A.G = A.work.as<double>();    // nd right-hand sides dN_d/dphi
  A.LAM = G + (size_t)nd * n;               // nd adjoint solutions
  double* eg = A.eg = A.LAM + (size_t)nd * n;
  double* JE = A.JE = eg + n;  // ng raw J e_g on planes nz-1, nz (zero below)
  const size_t nacc = (size_t)2 * nd * ng + QCAD_MAX_GATES + 1;
  A.accs.ensure(nacc * sizeof(double) + 64);
  double* acc = A.acc = A.accs.as<double>();  // [0, nd*ng): dN/dphi_D . e_g; then lam_d . J e_g
  A.zero_v = acc + 2 * nd * ng;               // one zero per gate, for masking Dirichlet rows
  CK(cudaMemsetAsync(acc, 0, nacc * sizeof(double), s));
  m->el_res.ensure((size_t)16 * m->n_elems * sizeof(double) + 64);
  for (int d = 0; d < nd; ++d) {
    int box[6];
    const bool have = dot_element_box(m, d, box);
    CK(cudaMemsetAsync(G + (size_t)d * n, 0, n * sizeof(double), s));
    launch_count_gradient(m->g64.g, phi, m->d_layer_semi.as<unsigned char>(), m->d_xn.as<double>(),
                          m->d_yn.as<double>(), m->d_zn.as<double>(), P, m->dots, d, have ? box : nullptr,
                          G + (size_t)d * n, m->el_res.as<double>(), s);
  }
  // gate lifts e_g: their raw J e_g (shared by every dot) and dN_d/dphi . e_g before masking. e_g
  // lives on the top node plane, so J e_g vanishes below plane nz-1: it is applied on the view of
  // the top element layer (the same products as the whole mesh's apply there), and the dots run
  // over the top plane
  const Grid<double>& g64 = m->g64.g;
  const int kl = m->nz - 1;
  Grid<double> gtop = g64;
  gtop.nz = 1;
  gtop.nzn = 2;
  gtop.mzx = g64.mzx + 3 * kl;
  gtop.mzy = g64.mzy + 3 * kl;
  gtop.kzz = g64.kzz + 3 * kl;
  gtop.zt = g64.zt ? g64.zt + 12 * kl : nullptr;
  gtop.hz = g64.hz + kl;
  gtop.dir_bottom = 0;
  const long long plane = g64.plane, off = (long long)kl * plane, top = (long long)m->nz * plane;
  const size_t coff = (size_t)8 * kl * m->nx * m->ny;
  CK(cudaMemsetAsync(eg, 0, n * sizeof(double), s));
  for (int gi = 0; gi < ng; ++gi) {
    CK(cudaMemsetAsync(eg + top, 0, plane * sizeof(double), s));
    for (int q = 0; q < ng; ++q) m->h_small[16 + q] = q == gi ? 1.0 : 0.0;
    CK(cudaMemcpyAsync(m->d_vgate.p, m->h_small + 16, sizeof(double) * ng, cudaMemcpyHostToDevice, s));
    launch_set_dirichlet(m->nxn, m->nyn, m->nzn, 0, 0.0, m->d_gate_top.as<signed char>(), m->d_vgate.as<double>(),
                         eg, s);
    double* je = JE + (size_t)gi * plane2;
    CK(cudaMemsetAsync(je, 0, plane2 * sizeof(double), s));
    ApplyArgs<double> a{};
    a.v = eg + off;
    a.y = je;
    a.c = ensure_pcg<double>(m).c + coff;
    a.raw = 1;
    launch_apply<double>(gtop, a, m->cfg64, s, Prec<double>::face(m));
    for (int d = 0; d < nd; ++d) launch_dot<double>(plane, G + (size_t)d * n + top, eg + top, acc + d * ng + gi, s);
    CK(cudaStreamSynchronize(s));  // h_small is reused by the next gate's upload
  }
  // zero the Dirichlet rows of the right-hand sides
  for (int d = 0; d < nd; ++d)
    launch_set_dirichlet(m->nxn, m->nyn, m->nzn, m->bottom_ohmic, 0.0, m->d_gate_top.as<signed char>(), A.zero_v,
                         G + (size_t)d * n, s);
  CK(cudaStreamSynchronize(s));
}

static void adjoint_finish(AdjWork& A, double* dN_dV, double* dN_dq) {
  qcad_mesh_s* m = A.m;
  cudaStream_t s = m->stream;
  const long long n = m->n_nodes;
  const int nd = A.nd, ng = A.ng;
  double* acc = A.acc;
  // J e_g vanishes below plane nz-1
  const long long plane = (long long)m->nxn * m->nyn, off = (long long)(m->nz - 1) * plane;
  for (int d = 0; d < nd; ++d)
    for (int gi = 0; gi < ng; ++gi)
      launch_dot<double>(2 * plane, A.LAM + (size_t)d * n + off, A.JE + (size_t)gi * 2 * plane,
                         acc + nd * ng + d * ng + gi, s);
  // charged gates (Robin condition): V_g enters through the load, d b / d V_g = (eps_r/d) int_f N_a
  // on the gate's faces (top plane), so dN_d/dV_g gains lam_d . d b / d V_g (lam is 0 on Dirichlet rows)
  const int nc = (int)m->charged_gate.size();
  DevBuf racc;
  std::vector<double> hr((size_t)std::max(1, nd * nc), 0.0);
  if (nc > 0) {
    racc.ensure((size_t)nd * nc * sizeof(double) + 64);
    CK(cudaMemsetAsync(racc.p, 0, (size_t)nd * nc * sizeof(double), s));
    for (int d = 0; d < nd; ++d)
      for (int c = 0; c < nc; ++c)
        launch_dot<double>(plane, A.LAM + (size_t)d * n + (size_t)m->nz * plane,
                           m->d_charged_r.as<double>() + (size_t)c * plane, racc.as<double>() + d * nc + c, s);
    CK(cudaMemcpyAsync(hr.data(), racc.p, (size_t)nd * nc * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  std::vector<double> h(2 * nd * ng);
  CK(cudaMemcpyAsync(h.data(), acc, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (dN_dq)
    for (int d = 0; d < nd; ++d)
      launch_theta_gradient(m->nx, m->ny, m->nz, m->g64.g.hx, m->g64.g.hy, m->g64.g.hz, A.LAM + (size_t)d * n,
                            A.P.qe, dN_dq + (long long)d * m->n_elems, s);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  for (int d = 0; d < nd; ++d)
    for (int gi = 0; gi < ng; ++gi) dN_dV[d * ng + gi] = h[d * ng + gi] - h[nd * ng + d * ng + gi];
  for (int d = 0; d < nd; ++d)
    for (int c = 0; c < nc; ++c) dN_dV[d * ng + m->charged_gate[c]] += hr[d * nc + c];
}

qcad_status adjoint(qcad_mesh_s* m, const qcad_bias* b, const qcad_solver_opts* o, const double* phi,
                    const double* theta, double* dN_dV, double* dN_dq) {
  validate_bias(m, b);
  validate_opts(o);
  if (!phi || !dN_dV) throw Error(QCAD_ERR_INVALID_ARG, "null pointer");
  const long long n = m->n_nodes;
  const int nd = m->dots.n;
  if (nd == 0) return QCAD_OK;
  AdjWork A;
  adjoint_prepare(A, m, b, o, phi, theta);
  const int maxk = o->max_krylov > 0 ? o->max_krylov : 20000;
  double* G = A.G;
  double* LAM = A.LAM;
  const int degree = o->cheb_degree != 0 ? o->cheb_degree : m->cheb_auto[1];
  if (o->precision == 1 && degree == DEG_MG && mg_prepare(m)) {
    for (int d = 0; d < nd; ++d) adjoint_solve_mixed_mg(m, G + (size_t)d * n, LAM + (size_t)d * n, maxk);
  } else if (o->precision == 1 && !m->has_robin) {
    adjoint_solve_mixed(m, nd, G, LAM, maxk);
  } else {
    // (charged gates: the batched kernels of the mixed multi-dot solve carry no face term)
    // the preconditioner of the FP64 solves: the request, else the mesh's tuned FP64 choice
    // (the multigrid V-cycle in FP64 where the mesh has a hierarchy), else Jacobi
    int deg64 = o->cheb_degree != 0 ? o->cheb_degree : m->cheb_auto[0];
    if (deg64 == 0 || (deg64 == DEG_MG && !mg_prepare(m))) deg64 = 1;
    for (int d = 0; d < nd; ++d) adjoint_solve64(m, G + (size_t)d * n, LAM + (size_t)d * n, maxk, deg64);
  }
  adjoint_finish(A, dN_dV, dN_dq);
  return QCAD_OK;
}

// Batched adjoint over several meshes (bias points of a sweep, or different devices). With a
// multigrid hierarchy on every mesh (the default preconditioner), the systems advance one dot
// index at a time: in each round every mesh's system J_i lam = dN_d/dphi runs its own
// multigrid-preconditioned FP32 PCG (the captured 4-iteration graphs of all meshes replayed back
// to back, one status read per round, as the batched Newton does). Otherwise (cheb_degree 1, or
// a mesh without a coarse level) all (mesh, dot) systems advance together in one batched FP32
// Jacobi-PCG: one apply launch and one update launch per iteration over a work table of every
// system. Either way each round of corrections is followed by every system's FP64 residual,
// until each is below 1e-13 of its right-hand side (as adjoint_solve_mixed does for the dots of
// one mesh).
qcad_status adjoint_batch(int n, const qcad_mesh_t* ms, const qcad_bias* bs, const qcad_solver_opts* o,
                          const double* const* phis, double* dN_dV) {
  if (n < 1 || !ms || !bs || !o || !phis || !dN_dV) throw Error(QCAD_ERR_INVALID_ARG, "invalid batch arguments");
  validate_opts(o);
  if (o->precision != 1) throw Error(QCAD_ERR_INVALID_ARG, "the batched adjoint runs in mixed precision (precision 1)");
  int max_nd = 0;
  for (int i = 0; i < n; ++i) {
    if (!ms[i] || !phis[i]) throw Error(QCAD_ERR_INVALID_ARG, "null mesh or phi in batch");
    if (ms[i]->has_surface)
      throw Error(QCAD_ERR_INVALID_ARG, "the batched adjoint does not take charged gates or surface charges");
    if (ms[i]->device != ms[0]->device) throw Error(QCAD_ERR_INVALID_ARG, "batch meshes must share one device");
    if (ms[i]->dots.n > QCAD_MAX_DOTS_K) throw Error(QCAD_ERR_INVALID_ARG, "too many dots");
    for (int j = 0; j < i; ++j)
      if (ms[j] == ms[i]) throw Error(QCAD_ERR_INVALID_ARG, "a mesh appears twice in the batch");
    validate_bias(ms[i], &bs[i]);
    max_nd = std::max(max_nd, ms[i]->dots.n);
  }
  std::vector<AdjWork> A(n);
  for (int i = 0; i < n; ++i) adjoint_prepare(A[i], ms[i], &bs[i], o, phis[i], nullptr);
  bool use_mg = o->cheb_degree == 0 || o->cheb_degree == -1;
  for (int i = 0; i < n && use_mg; ++i) use_mg = mg_prepare(ms[i]);
  const int maxk = o->max_krylov > 0 ? o->max_krylov : 20000;
  struct Sys {
    int i, d;
  };
  // FP32 PCG vectors of system (mesh m, dot d): the mesh's own for dot 0 (or for every dot in the
  // multigrid rounds, which solve one dot of each mesh at a time), an extra set otherwise
  auto vecs_for = [&](qcad_mesh_s* m, int d) {
    PcgVecs<float> v = ensure_pcg<float>(m);
    if (d == 0) return v;
    const size_t nb = (size_t)m->n_nodes * sizeof(float) + 64;
    PcgBufs<float>& k = m->k32x[d - 1];
    k.x.ensure(nb);
    k.r.ensure(nb);
    k.z.ensure(nb);
    k.p.ensure(2 * nb);
    k.Ap.ensure(nb);
    k.b.ensure(nb);
    v.x = k.x.as<float>();
    v.r = k.r.as<float>();
    v.z = k.z.as<float>();
    v.p[0] = k.p.as<float>();
    v.p[1] = v.p[0] + nb / sizeof(float);
    v.Ap = k.Ap.as<float>();
    v.b = k.b.as<float>();  // dinv and c are the mesh's shared linearization
    return v;
  };
  // one round: the systems `sys` (entry q of B is system q) to 1e-13 by FP32 corrections and FP64
  // residuals
  auto refine = [&](BatchCtx& B, const std::vector<Sys>& sys) {
    const int ns = (int)sys.size();
    cudaStream_t s = B.s;
    DevBuf d2buf;
    d2buf.ensure((size_t)ns * sizeof(double) + 64);
    double* d2 = d2buf.as<double>();
    std::vector<double> g2(ns), r2(ns), rtol(ns), hd(ns);
    std::vector<int> iters, nonf;
    auto rhs = [&](int q) { return A[sys[q].i].G + (size_t)sys[q].d * ms[sys[q].i]->n_nodes; };
    auto lam = [&](int q) { return A[sys[q].i].LAM + (size_t)sys[q].d * ms[sys[q].i]->n_nodes; };
    // per mesh scratch: y (n) then one residual per dot (nd x n)
    auto ybuf = [&](int q) { return ms[sys[q].i]->scratch.as<double>(); };
    auto rbuf = [&](int q) {
      return ms[sys[q].i]->scratch.as<double>() + (size_t)(1 + sys[q].d) * ms[sys[q].i]->n_nodes;
    };
    CK(cudaMemsetAsync(d2, 0, ns * sizeof(double), s));
    for (int q = 0; q < ns; ++q) {
      const long long nn = ms[sys[q].i]->n_nodes;
      CK(cudaMemsetAsync(lam(q), 0, nn * sizeof(double), s));
      CK(cudaMemcpyAsync(rbuf(q), rhs(q), nn * sizeof(double), cudaMemcpyDeviceToDevice, s));
      launch_d2f(nn, rhs(q), const_cast<float*>(B.vecs[q].b), s);
      launch_dot<double>(nn, rhs(q), rhs(q), d2 + q, s);
    }
    CK(cudaMemcpyAsync(hd.data(), d2, ns * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    g2 = hd;
    r2 = hd;
    for (int rf = 0; rf < 12; ++rf) {
      bool any = false;
      for (int q = 0; q < ns; ++q) {
        rtol[q] = 0.0;
        if (r2[q] <= 1e-26 * g2[q]) continue;
        any = true;
        // each correction needs only to bring the residual to a tenth of the 1e-13 target
        rtol[q] = std::max(1e-5, std::min(1e-2, 1e-14 * std::sqrt(g2[q] / std::max(r2[q], 1e-300))));
      }
      if (!any) break;
      if (use_mg)
        batch_pcg_mg(B, rtol, maxk, iters, nonf);
      else
        batch_pcg(B, rtol, maxk, iters, nonf);
      CK(cudaMemsetAsync(d2, 0, ns * sizeof(double), s));
      for (int q = 0; q < ns; ++q) {
        if (!(rtol[q] > 0)) continue;
        if (nonf[q]) throw Error(QCAD_ERR_NONFINITE, "batched adjoint refinement produced a non-finite value");
        qcad_mesh_s* m = ms[sys[q].i];
        const long long nn = m->n_nodes;
        launch_axpy<float>(nn, 1.0, B.vecs[q].x, lam(q), s);
        ApplyArgs<double> a{};
        a.v = lam(q);
        a.y = ybuf(q);
        a.c = ensure_pcg<double>(m).c;
        launch_apply<double>(m->g64.g, a, m->cfg64, s, nullptr);
        launch_sub(nn, rhs(q), ybuf(q), rbuf(q), const_cast<float*>(B.vecs[q].b), s);
        launch_dot<double>(nn, rbuf(q), rbuf(q), d2 + q, s);
      }
      CK(cudaMemcpyAsync(hd.data(), d2, ns * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (int q = 0; q < ns; ++q)
        if (rtol[q] > 0) r2[q] = hd[q];
    }
  };
  for (int i = 0; i < n; ++i) {
    qcad_mesh_s* m = ms[i];
    m->scratch.ensure((size_t)(A[i].nd + 1) * m->n_nodes * sizeof(double) + 64);
    m->scal_x.ensure((size_t)std::max(1, A[i].nd) * sizeof(PcgScalars) + 64);
    m->adj_ctx.reset();  // the single-mesh adjoint context shares these vectors: rebuild it next time
  }
  if (use_mg) {
    for (int d = 0; d < max_nd; ++d) {
      BatchCtx B;
      B.s = ms[0]->stream;
      std::vector<Sys> sys;
      for (int i = 0; i < n; ++i) {
        if (A[i].nd <= d) continue;
        B.ms.push_back(ms[i]);
        B.vecs.push_back(vecs_for(ms[i], 0));
        B.scd.push_back(ms[i]->scal.as<PcgScalars>());
        B.kch.push_back(ms[i]->batch_kchunk);
        sys.push_back(Sys{i, d});
      }
      B.n = (int)sys.size();
      batch_setup(B);
      refine(B, sys);
    }
  } else {
    BatchCtx B;
    B.s = ms[0]->stream;
    std::vector<Sys> sys;
    for (int i = 0; i < n; ++i) {
      qcad_mesh_s* m = ms[i];
      const int kc = (m->cfg32.variant == 3 && m->cfg32.by == 8) ? m->cfg32.kchunk : 16;
      for (int d = 0; d < A[i].nd; ++d) {
        B.ms.push_back(m);
        B.vecs.push_back(vecs_for(m, d));
        B.scd.push_back(d == 0 ? m->scal.as<PcgScalars>() : m->scal_x.as<PcgScalars>() + d);
        B.kch.push_back(kc);
        sys.push_back(Sys{i, d});
      }
    }
    if (!sys.empty()) {
      B.n = (int)sys.size();
      batch_setup(B);
      refine(B, sys);
    }
  }
  size_t off = 0;
  for (int i = 0; i < n; ++i) {
    if (A[i].nd > 0) adjoint_finish(A[i], dN_dV + off, nullptr);
    off += (size_t)A[i].nd * A[i].ng;
  }
  return QCAD_OK;
}

// ---------------------------------------------------------------------------
// Interface-charge calibration (Sec. III): the sheet density sigma of a fixed-charge pattern
// (theta = sigma * pattern) such that dot `dot` holds target_N electrons, by Newton on sigma with
// the adjoint slope dN/dsigma = (dN/dtheta) . pattern, kept inside the bracket the iterates
// establish (N rises with sigma) and bisected when a step would leave it.
qcad_status calibrate_sheet(qcad_mesh_s* m, const qcad_bias* b, const qcad_solver_opts* o, int dot, double target,
                            const double* pattern, double sigma0, double tol_N, int max_iter, double* phi,
                            double* theta, double* sigma_out, qcad_calib_report* rep) {
  const auto t0 = std::chrono::steady_clock::now();
  validate_bias(m, b);
  validate_opts(o);
  if (dot < 0 || dot >= m->dots.n) throw Error(QCAD_ERR_INVALID_ARG, "dot index out of range");
  if (!pattern || !phi || !theta || !sigma_out) throw Error(QCAD_ERR_INVALID_ARG, "null pointer");
  if (!(tol_N > 0) || !std::isfinite(target) || !std::isfinite(sigma0))
    throw Error(QCAD_ERR_INVALID_ARG, "tol_N must be > 0 and target_N, sigma0 finite");
  if (max_iter < 1 || max_iter > QCAD_CALIB_HIST) throw Error(QCAD_ERR_INVALID_ARG, "max_iter must be in [1, 32]");
  cudaStream_t s = m->stream;
  const long long ne = m->n_elems;
  DevBuf dq;
  dq.ensure((size_t)m->dots.n * ne * sizeof(double) + 64);
  std::vector<double> dNdV(std::max(1, m->dots.n * m->n_gates)), N(QCAD_MAX_DOTS_K);
  qcad_calib_report r{};
  double sigma = sigma0, lo = 0, hi = 0, slope = 0;
  bool have_lo = false, have_hi = false, converged = false;
  qcad_solver_opts ow = *o;
  qcad_status st = QCAD_OK;
  int it = 0;
  for (it = 1; it <= max_iter; ++it) {
    CK(cudaMemcpyAsync(theta, pattern, ne * sizeof(double), cudaMemcpyDeviceToDevice, s));
    launch_scale<double>(ne, theta, sigma, s);
    st = poisson_solve(m, b, &ow, theta, phi, nullptr);
    if (st != QCAD_OK) break;
    ow.warm_start = 1;
    electron_counts(m, b, theta, phi, N.data());
    const double f = N[dot] - target;
    r.sigma_hist[it - 1] = sigma;
    r.N_hist[it - 1] = N[dot];
    r.N = N[dot];
    if (std::fabs(f) <= tol_N) {
      converged = true;
      break;
    }
    if (f > 0) {
      hi = sigma;
      have_hi = true;
    } else {
      lo = sigma;
      have_lo = true;
    }
    st = adjoint(m, b, o, phi, theta, dNdV.data(), dq.as<double>());
    if (st != QCAD_OK) break;
    double* acc = m->stats.as<double>() + 60;
    CK(cudaMemsetAsync(acc, 0, sizeof(double), s));
    launch_dot<double>(ne, dq.as<double>() + (size_t)dot * ne, pattern, acc, s);
    CK(cudaMemcpyAsync(m->h_small + 60, acc, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    slope = m->h_small[60];
    r.dN_dsigma = slope;
    double next = slope > 0 ? sigma - f / slope : NAN;
    const bool inside = std::isfinite(next) && (!have_lo || next > lo) && (!have_hi || next < hi);
    if (!inside) {
      if (have_lo && have_hi)
        next = 0.5 * (lo + hi);
      else  // no bracket on that side yet: step away from the known side
        next = sigma + (f > 0 ? -1.0 : 1.0) * std::max(1e-4, 2.0 * std::fabs(sigma - (have_lo ? lo : hi)));
    }
    sigma = next;
  }
  *sigma_out = sigma;
  r.iters = std::min(it, max_iter);
  r.converged = converged ? 1 : 0;
  r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (rep) *rep = r;
  if (st != QCAD_OK) return st;
  if (!converged) {
    set_message("the sheet-charge calibration did not reach tol_N");
    return QCAD_ERR_NOT_CONVERGED;
  }
  return QCAD_OK;
}

qcad_status poisson_solve_batch_impl(int n, const qcad_mesh_t* ms, const qcad_bias* bs, const qcad_solver_opts* o,
                                     double* const* phis, qcad_solve_report* reps) {
  const auto t0 = std::chrono::steady_clock::now();
  if (n < 1 || !ms || !bs || !o || !phis) throw Error(QCAD_ERR_INVALID_ARG, "invalid batch arguments");
  validate_opts(o);
  if (o->precision != 1) throw Error(QCAD_ERR_INVALID_ARG, "the batched form runs in mixed precision (precision 1)");
  BatchCtx B;
  B.n = n;
  B.ms.assign(ms, ms + n);
  for (int i = 0; i < n; ++i) {
    if (!ms[i] || !phis[i]) throw Error(QCAD_ERR_INVALID_ARG, "null mesh or phi in batch");
    if (ms[i]->has_surface)
      throw Error(QCAD_ERR_INVALID_ARG, "the batched solve does not take charged gates or surface charges");
    if (ms[i]->device != ms[0]->device) throw Error(QCAD_ERR_INVALID_ARG, "batch meshes must share one device");
    for (int j = 0; j < i; ++j)
      if (ms[j] == ms[i]) throw Error(QCAD_ERR_INVALID_ARG, "a mesh appears twice in the batch");
    validate_bias(ms[i], &bs[i]);
    ensure_newton(ms[i]);
  }
  B.s = ms[0]->stream;
  for (int i = 0; i < n; ++i) {
    B.vecs.push_back(ensure_pcg<float>(ms[i]));
    B.scd.push_back(ms[i]->scal.as<PcgScalars>());
    B.kch.push_back(ms[i]->batch_kchunk);
  }
  batch_setup(B);
  // the instances' multigrid-preconditioned PCG (cheb_degree 0 or -1) when every mesh has a
  // hierarchy, else the one-launch-per-iteration batched Jacobi PCG (cheb_degree 1)
  bool use_mg = o->cheb_degree == 0 || o->cheb_degree == -1;
  for (int i = 0; i < n && use_mg; ++i) use_mg = mg_prepare(ms[i]);
  const int maxk = o->max_krylov > 0 ? o->max_krylov : 20000;
  const int maxn = o->max_newton > 0 ? o->max_newton : 100;
  B.P.resize(n);
  std::vector<double*> pa(n), pb(n);
  std::vector<ResStats> R(n), Rt(n);
  std::vector<double> R0(n), step(n, 0.0), rtol(n), alpha(n);
  std::vector<int> kry(n, 0), its(n, 0), conv(n, 0), bad(n, 0), iters, nonf, all(n);
  for (int i = 0; i < n; ++i) {
    qcad_mesh_s* m = ms[i];
    all[i] = i;
    B.P[i] = make_phys(m, &bs[i]);
    pa[i] = m->phi_a.as<double>();
    pb[i] = m->phi_b.as<double>();
    if (o->warm_start)
      CK(cudaMemcpyAsync(pa[i], phis[i], m->n_nodes * sizeof(double), cudaMemcpyDeviceToDevice, m->stream));
    else
      CK(cudaMemsetAsync(pa[i], 0, m->n_nodes * sizeof(double), m->stream));
    set_contacts(m, &bs[i], B.P[i], pa[i], nullptr, nullptr);  // synchronizes the mesh stream
  }
  // trial points pb = pa + alpha x for the instances `idx` (max |alpha x| into each stats slot)
  auto trials = [&](const std::vector<int>& idx) {
    if (idx.empty()) return;
    for (int i : idx) {
      qcad_mesh_s* m = ms[i];
      CK(cudaMemsetAsync(m->stats.as<double>() + 8, 0, sizeof(double), B.s));
      launch_newton_trial<float>(m->n_nodes, pa[i], ensure_pcg<float>(m).x, alpha[i], pb[i],
                                 m->stats.as<double>() + 8, B.s);
    }
  };
  if (!o->warm_start) {
    // Laplace initial guesses to 1e-3 (rho = 0), all instances at once
    batch_residual(B, all, pa, 1, R, nullptr);
    for (int i = 0; i < n; ++i) rtol[i] = 1e-3;
    if (use_mg)
      batch_pcg_mg(B, rtol, maxk, iters, nonf);
    else
      batch_pcg(B, rtol, maxk, iters, nonf);
    for (int i = 0; i < n; ++i) {
      kry[i] += iters[i];
      if (nonf[i]) bad[i] = 1;
      alpha[i] = 1.0;
    }
    trials(all);
    for (int i = 0; i < n; ++i) std::swap(pa[i], pb[i]);
  }
  batch_residual(B, all, pa, o->linear, R, nullptr);
  for (int i = 0; i < n; ++i) {
    R0[i] = std::sqrt(R[i].r2);
    if (!std::isfinite(R[i].r2)) bad[i] = 1;
  }
  for (int it = 1; it <= maxn; ++it) {
    bool any = false;
    for (int i = 0; i < n; ++i) {
      rtol[i] = 0.0;
      if (conv[i] || bad[i]) continue;
      any = true;
      const double nR = std::sqrt(R[i].r2);
      rtol[i] = std::max(1e-5, R0[i] > 0 ? std::min(1e-2, nR / R0[i]) : 1e-2);
      if (nR > 0) rtol[i] = std::max(rtol[i], std::min(1e-2, 0.1 * o->newton_tol_R / nR));
    }
    if (!any) break;
    if (use_mg)
      batch_pcg_mg(B, rtol, maxk, iters, nonf);
    else
      batch_pcg(B, rtol, maxk, iters, nonf);
    std::vector<int> search;
    for (int i = 0; i < n; ++i) {
      if (!(rtol[i] > 0)) continue;
      kry[i] += iters[i];
      its[i] = it;
      if (nonf[i]) {
        bad[i] = 1;
        continue;
      }
      alpha[i] = 1.0;
      search.push_back(i);
    }
    // backtracking on ||R||_2 for every searching instance at once (halving up to 30 times)
    for (int ls = 0; ls <= 30 && !search.empty(); ++ls) {
      trials(search);
      batch_residual(B, search, pb, o->linear, Rt, &step);
      std::vector<int> next;
      for (int i : search) {
        const double nR = std::sqrt(R[i].r2);
        const bool ok = std::isfinite(Rt[i].r2) && std::sqrt(Rt[i].r2) <= (1.0 - 1e-4 * alpha[i]) * nR;
        if (ok || ls == 30) {
          std::swap(pa[i], pb[i]);
          R[i] = Rt[i];
          if (!std::isfinite(R[i].r2)) bad[i] = 1;
          if (R[i].rmax < o->newton_tol_R && step[i] < o->newton_tol_dphi) conv[i] = 1;
        } else {
          alpha[i] *= 0.5;
          next.push_back(i);
        }
      }
      search.swap(next);
    }
  }
  qcad_status worst = QCAD_OK;
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int i = 0; i < n; ++i) {
    qcad_mesh_s* m = ms[i];
    CK(cudaMemcpyAsync(phis[i], pa[i], m->n_nodes * sizeof(double), cudaMemcpyDeviceToDevice, B.s));
    // the mesh's own buffers now hold this iterate in phi_a (keep single-mesh solves consistent)
    if (pa[i] != m->phi_a.as<double>())
      CK(cudaMemcpyAsync(m->phi_a.p, pa[i], m->n_nodes * sizeof(double), cudaMemcpyDeviceToDevice, B.s));
    if (reps) {
      reps[i].newton_iters = its[i];
      reps[i].krylov_iters_total = kry[i];
      reps[i].applies_total = kry[i];
      reps[i].final_res_inf = R[i].rmax;
      reps[i].final_dphi_inf = step[i];
      reps[i].seconds = secs;
      reps[i].status_detail = 0;
    }
    const qcad_status st = bad[i] ? QCAD_ERR_NONFINITE : (conv[i] ? QCAD_OK : QCAD_ERR_NOT_CONVERGED);
    if (worst == QCAD_OK && st != QCAD_OK) worst = st;
  }
  CK(cudaStreamSynchronize(B.s));
  if (worst != QCAD_OK) set_message("at least one batch instance did not converge or produced a non-finite value");
  return worst;
}

}  // namespace qcad
