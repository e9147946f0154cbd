// C ABI of libqcad (include/qcad.h): argument checks, error translation and
// the launch-configuration autotuner. No C++ exception crosses this boundary.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <exception>
#include <string>
#include <thread>
#include <vector>

#include "mesh.h"

namespace qcad {
void mesh_create(const qcad_device* dev, void* stream, qcad_mesh_t* out);
Phys make_phys(const qcad_mesh_s* m, const qcad_bias* b);
qcad_status calibrate_sheet(qcad_mesh_s* m, const qcad_bias* b, const qcad_solver_opts* o, int dot, double target,
                            const double* pattern, double sigma0, double tol_N, int max_iter, double* phi,
                            double* theta, double* sigma_out, qcad_calib_report* rep);
qcad_status sp_solve(qcad_mesh_s* m, const qcad_bias* b, const qcad_solver_opts* o, int nev, const double* m_eff,
                     double eig_tol, double tol_dphi, int max_iter, int use_vxc, double* phi, double* evals,
                     qcad_sp_report* rep);
void set_contacts(qcad_mesh_s* m, const qcad_bias* b, const Phys& P, double* phi, double* gate_vals, double* ohm_val);
qcad_status poisson_solve(qcad_mesh_s* m, const qcad_bias* b, const qcad_solver_opts* o, const double* theta,
                          double* phi, qcad_solve_report* rep);
qcad_status poisson_residual(qcad_mesh_s* m, const qcad_bias* b, const double* theta, const double* phi, double* R,
                             double* diag, double* stats);
qcad_status poisson_jv(qcad_mesh_s* m, const qcad_bias* b, const double* phi, const double* v, double* y,
                       int precision);
qcad_status electron_counts(qcad_mesh_s* m, const qcad_bias* b, const double* theta, const double* phi, double* N);
qcad_status capacitance(qcad_mesh_s* m, const qcad_bias* b, const qcad_solver_opts* o, int gate, double dV,
                        const double* theta, double* phi, double* C_aF);
qcad_status adjoint(qcad_mesh_s* m, const qcad_bias* b, const qcad_solver_opts* o, const double* phi,
                    const double* theta, double* dN_dV, double* dN_dq);
qcad_status schrodinger_apply(qcad_mesh_s* m, const qcad_bias* b, const double* phi, const double* m_eff, int nvec,
                              const double* X, double* HX, double* MX, int precision);
qcad_status schrodinger_eigs(qcad_mesh_s* m, const qcad_bias* b, const double* phi, int nev, const double* m_eff,
                             double tol, double* evals, double* evecs, qcad_solve_report* rep);
qcad_status schrodinger_eigs_stream2(qcad_mesh_s* m, const qcad_bias* b, const double* phi, int nev,
                                     const double* m_eff, double tol, double* evals, double* evecs,
                                     qcad_solve_report* rep);
qcad_status poisson_solve_batch(int n, const qcad_mesh_t* ms, const qcad_bias* bs, const qcad_solver_opts* o,
                                double* const* phis, qcad_solve_report* reps);
qcad_status adjoint_batch(int n, const qcad_mesh_t* ms, const qcad_bias* bs, const qcad_solver_opts* o,
                          const double* const* phis, double* dN_dV);
qcad_status autotune(qcad_mesh_s* m, const qcad_bias* b, int precision, int* variant, int* tile_rows, int* z_chunk,
                     float* best);
qcad_status noalloc_residual(const qcad_device* dev, const qcad_bias* b, void* stream, const double* theta,
                             const double* phi, double* R, double* stats);
qcad_status alu_peaks(double* fp64_tflops, double* fp32_tflops, double* fp64_exp_per_s);
}  // namespace qcad

static thread_local std::string g_last_error;

template <class F>
static qcad_status guarded(F&& f) {
  g_last_error.clear();
  try {
    return f();
  } catch (const qcad::Error& e) {
    g_last_error = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return QCAD_ERR_OOM;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return QCAD_ERR_CUDA;
  } catch (...) {
    g_last_error = "unknown error";
    return QCAD_ERR_CUDA;
  }
}

static void need_mesh(qcad_mesh_t m) {
  if (!m) throw qcad::Error(QCAD_ERR_INVALID_ARG, "null mesh");
  int dev = -1;
  qcad::check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev != m->device) throw qcad::Error(QCAD_ERR_INVALID_ARG, "current CUDA device differs from the mesh's device");
}

extern "C" {

qcad_status qcad_mesh_create(const qcad_device* dev, void* cuda_stream, qcad_mesh_t* out) {
  return guarded([&] {
    qcad::mesh_create(dev, cuda_stream, out);
    return QCAD_OK;
  });
}

void qcad_mesh_destroy(qcad_mesh_t m) {
  if (!m) return;
  cudaStreamSynchronize(m->stream);
  delete m;
}

qcad_status qcad_mesh_info(qcad_mesh_t m, int64_t* n_nodes, int64_t* n_elems, int* n_gates, int* n_dots,
                           int64_t* n_sub_dof) {
  return guarded([&] {
    if (!m) throw qcad::Error(QCAD_ERR_INVALID_ARG, "null mesh");
    if (n_nodes) *n_nodes = m->n_nodes;
    if (n_elems) *n_elems = m->n_elems;
    if (n_gates) *n_gates = m->n_gates;
    if (n_dots) *n_dots = m->dots.n;
    if (n_sub_dof)
      *n_sub_dof = m->has_sub ? (int64_t)(m->sub[1] - m->sub[0] - 1) * (m->sub[3] - m->sub[2] - 1) *
                                    (m->sub[5] - m->sub[4] - 1)
                              : 0;
    return QCAD_OK;
  });
}

qcad_status qcad_contact_values(qcad_mesh_t m, const qcad_bias* b, double* phi, double* phi_gate,
                                double* phi_ohmic) {
  return guarded([&] {
    need_mesh(m);
    if (!b || b->n_gates != m->n_gates) throw qcad::Error(QCAD_ERR_INVALID_ARG, "bias does not match the mesh");
    const qcad::Phys P = qcad::make_phys(m, b);
    qcad::set_contacts(m, b, P, phi, phi_gate, phi_ohmic);
    return QCAD_OK;
  });
}

qcad_status qcad_poisson_residual(qcad_mesh_t m, const qcad_bias* b, const double* fixed_charge_elem,
                                  const double* phi, double* R, double* diag, double* stats) {
  return guarded([&] {
    need_mesh(m);
    return qcad::poisson_residual(m, b, fixed_charge_elem, phi, R, diag, stats);
  });
}

qcad_status qcad_poisson_jv(qcad_mesh_t m, const qcad_bias* b, const double* phi, const double* v, double* y,
                            int precision) {
  return guarded([&] {
    need_mesh(m);
    return qcad::poisson_jv(m, b, phi, v, y, precision);
  });
}

qcad_status qcad_poisson_solve(qcad_mesh_t m, const qcad_bias* b, const qcad_solver_opts* o,
                               const double* fixed_charge_elem, double* phi, qcad_solve_report* rep) {
  return guarded([&] {
    need_mesh(m);
    return qcad::poisson_solve(m, b, o, fixed_charge_elem, phi, rep);
  });
}

qcad_status qcad_electron_counts(qcad_mesh_t m, const qcad_bias* b, const double* fixed_charge_elem,
                                 const double* phi, double* N) {
  return guarded([&] {
    need_mesh(m);
    return qcad::electron_counts(m, b, fixed_charge_elem, phi, N);
  });
}

qcad_status qcad_capacitance(qcad_mesh_t m, const qcad_bias* b, const qcad_solver_opts* o, int gate, double dV,
                             const double* fixed_charge_elem, double* phi, double* C_aF) {
  return guarded([&] {
    need_mesh(m);
    return qcad::capacitance(m, b, o, gate, dV, fixed_charge_elem, phi, C_aF);
  });
}

qcad_status qcad_adjoint(qcad_mesh_t m, const qcad_bias* b, const qcad_solver_opts* o, const double* phi,
                         const double* fixed_charge_elem, double* dN_dV, double* dN_dq) {
  return guarded([&] {
    need_mesh(m);
    return qcad::adjoint(m, b, o, phi, fixed_charge_elem, dN_dV, dN_dq);
  });
}

qcad_status qcad_schrodinger_apply(qcad_mesh_t m, const qcad_bias* b, const double* phi, const double* m_eff,
                                   int nvec, const double* X, double* HX, double* MX, int precision) {
  return guarded([&] {
    need_mesh(m);
    return qcad::schrodinger_apply(m, b, phi, m_eff, nvec, X, HX, MX, precision);
  });
}

qcad_status qcad_schrodinger_eigs(qcad_mesh_t m, const qcad_bias* b, const double* phi, int nev,
                                  const double* m_eff, double tol, double* evals, double* evecs,
                                  qcad_solve_report* rep) {
  return guarded([&] {
    need_mesh(m);
    return qcad::schrodinger_eigs(m, b, phi, nev, m_eff, tol, evals, evecs, rep);
  });
}

qcad_status qcad_calibrate_sheet_charge(qcad_mesh_t m, const qcad_bias* b, const qcad_solver_opts* o, int dot,
                                        double target_N, const double* pattern, double sigma0, double tol_N,
                                        int max_iter, double* phi, double* theta, double* sigma,
                                        qcad_calib_report* rep) {
  return guarded([&] {
    need_mesh(m);
    return qcad::calibrate_sheet(m, b, o, dot, target_N, pattern, sigma0, tol_N, max_iter, phi, theta, sigma, rep);
  });
}

qcad_status qcad_sp_solve(qcad_mesh_t m, const qcad_bias* b, const qcad_solver_opts* o, int nev, const double* m_eff,
                          double eig_tol, double tol_dphi, int max_iter, int use_vxc, double* phi, double* evals,
                          qcad_sp_report* rep) {
  return guarded([&] {
    need_mesh(m);
    if (!o) throw qcad::Error(QCAD_ERR_INVALID_ARG, "null solver options");
    return qcad::sp_solve(m, b, o, nev, m_eff, eig_tol, tol_dphi, max_iter, use_vxc, phi, evals, rep);
  });
}

qcad_status qcad_adjoint_eigs(qcad_mesh_t m, const qcad_bias* b, const qcad_solver_opts* o, const double* phi,
                              const double* fixed_charge_elem, double* dN_dV, double* dN_dq, int nev,
                              const double* m_eff, double tol, double* evals, double* evecs,
                              qcad_solve_report* eig_rep) {
  return guarded([&] {
    need_mesh(m);
    // the eigensolve on the mesh's second stream from a second host thread, the adjoint here
    qcad_status st_eig = QCAD_OK;
    std::string eig_msg;
    std::exception_ptr eig_exc;
    std::thread th([&] {
      try {
        CK(cudaSetDevice(m->device));
        st_eig = qcad::schrodinger_eigs_stream2(m, b, phi, nev, m_eff, tol, evals, evecs, eig_rep);
        if (st_eig != QCAD_OK) eig_msg = g_last_error;
      } catch (...) {
        eig_exc = std::current_exception();
      }
    });
    qcad_status st_adj = QCAD_OK;
    try {
      st_adj = qcad::adjoint(m, b, o, phi, fixed_charge_elem, dN_dV, dN_dq);
    } catch (...) {
      th.join();
      throw;
    }
    th.join();
    if (eig_exc) std::rethrow_exception(eig_exc);
    if (st_adj != QCAD_OK) return st_adj;
    if (st_eig != QCAD_OK) g_last_error = eig_msg;
    return st_eig;
  });
}

qcad_status qcad_poisson_solve_batch(int n, const qcad_mesh_t* ms, const qcad_bias* bs, const qcad_solver_opts* o,
                                     double* const* phis, qcad_solve_report* reps) {
  return guarded([&] { return qcad::poisson_solve_batch(n, ms, bs, o, phis, reps); });
}

qcad_status qcad_adjoint_batch(int n, const qcad_mesh_t* ms, const qcad_bias* bs, const qcad_solver_opts* o,
                               const double* const* phis, double* dN_dV) {
  return guarded([&] { return qcad::adjoint_batch(n, ms, bs, o, phis, dN_dV); });
}

qcad_status qcad_alu_peaks(double* fp64_tflops, double* fp32_tflops, double* fp64_exp_per_s) {
  return guarded([&] { return qcad::alu_peaks(fp64_tflops, fp32_tflops, fp64_exp_per_s); });
}

qcad_status qcad_profile_enable(qcad_mesh_t m, int enable) {
  return guarded([&] {
    if (!m) throw qcad::Error(QCAD_ERR_INVALID_ARG, "null mesh");
    m->prof.on = enable != 0;
    return QCAD_OK;
  });
}

qcad_status qcad_profile_reset(qcad_mesh_t m) {
  return guarded([&] {
    if (!m) throw qcad::Error(QCAD_ERR_INVALID_ARG, "null mesh");
    for (int c = 0; c < qcad::PROF_NCLASS; ++c) {
      m->prof.launches[c] = 0;
      m->prof.ms[c] = 0.0;
    }
    return QCAD_OK;
  });
}

qcad_status qcad_profile_read(qcad_mesh_t m, int kernel_class, int64_t* launches, double* total_ms) {
  return guarded([&] {
    if (!m) throw qcad::Error(QCAD_ERR_INVALID_ARG, "null mesh");
    if (kernel_class < 0 || kernel_class >= qcad::PROF_NCLASS)
      throw qcad::Error(QCAD_ERR_INVALID_ARG, "kernel class out of range");
    if (launches) *launches = m->prof.launches[kernel_class];
    if (total_ms) *total_ms = m->prof.ms[kernel_class];
    return QCAD_OK;
  });
}

qcad_status qcad_set_launch(qcad_mesh_t m, int family, int variant, int tile_rows, int z_chunk) {
  return guarded([&] {
    if (!m) throw qcad::Error(QCAD_ERR_INVALID_ARG, "null mesh");
    if (tile_rows != 4 && tile_rows != 8 && tile_rows != 16 && tile_rows != 32)
      throw qcad::Error(QCAD_ERR_INVALID_ARG, "tile_rows must be 4, 8, 16 or 32");
    if (z_chunk < 1 || z_chunk > 4096) throw qcad::Error(QCAD_ERR_INVALID_ARG, "z_chunk out of range");
    if (variant < 0 || variant > 3) throw qcad::Error(QCAD_ERR_INVALID_ARG, "variant must be 0..3");
    if (m->has_robin && family != 0 && variant != 0)
      throw qcad::Error(QCAD_ERR_INVALID_ARG, "a mesh with charged gates runs the element-gather variant 0 only");
    qcad::LaunchCfg c;
    c.by = tile_rows;
    c.kchunk = z_chunk;
    c.variant = (family == 1 && variant == 1) ? 0 : variant;
    if (family == 0)
      m->cfg_res = c;
    else if (family == 1)
      m->cfg64 = c;
    else if (family == 2)
      m->cfg32 = c;
    else
      throw qcad::Error(QCAD_ERR_INVALID_ARG, "family must be 0, 1 or 2");
    // graphs captured with the old configuration are rebuilt on next use
    m->graph64.key = nullptr;
    m->graph32.key = nullptr;
    return QCAD_OK;
  });
}

qcad_status qcad_launch_info(qcad_mesh_t m, int family, int* variant, int* tile_rows, int* z_chunk,
                             int* cheb_degree) {
  return guarded([&] {
    if (!m) throw qcad::Error(QCAD_ERR_INVALID_ARG, "null mesh");
    if (family < 0 || family > 2) throw qcad::Error(QCAD_ERR_INVALID_ARG, "family must be 0, 1 or 2");
    const qcad::LaunchCfg& c = family == 0 ? m->cfg_res : family == 1 ? m->cfg64 : m->cfg32;
    if (variant) *variant = c.variant;
    if (tile_rows) *tile_rows = c.by;
    if (z_chunk) *z_chunk = c.kchunk;
    if (cheb_degree) *cheb_degree = family == 0 ? 0 : m->cheb_auto[family == 1 ? 0 : 1];
    return QCAD_OK;
  });
}

qcad_status qcad_autotune(qcad_mesh_t m, const qcad_bias* b, int precision, int* variant, int* tile_rows,
                          int* z_chunk, float* best_ms) {
  return guarded([&] {
    need_mesh(m);
    return qcad::autotune(m, b, precision, variant, tile_rows, z_chunk, best_ms);
  });
}

qcad_status qcad_poisson_residual_noalloc(const qcad_device* dev, const qcad_bias* b, void* cuda_stream,
                                          const double* fixed_charge_elem, const double* phi, double* R,
                                          double* stats) {
  return guarded([&] { return qcad::noalloc_residual(dev, b, cuda_stream, fixed_charge_elem, phi, R, stats); });
}

qcad_status qcad_launch_count(int64_t* count) {
  return guarded([&] {
    if (!count) throw qcad::Error(QCAD_ERR_INVALID_ARG, "null output");
    *count = qcad::launch_count();
    return QCAD_OK;
  });
}

const char* qcad_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

namespace qcad {
// Message for a non-OK status returned without an exception (kept until the next call).
void set_message(const std::string& msg) { g_last_error = msg; }
}  // namespace qcad
