// Batched Poisson solves and the launch-configuration autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "mesh.h"

namespace qcad {

qcad_status poisson_solve(qcad_mesh_s* m, const qcad_bias* b, const qcad_solver_opts* o, const double* theta,
                          double* phi, qcad_solve_report* rep);

// Times the Jacobian apply of the mesh's current linearization for every
// (tile rows, z chunk) candidate and keeps the fastest for that precision.
qcad_status autotune(qcad_mesh_s* m, const qcad_bias* b, int precision, int* tile_rows, int* z_chunk, float* best) {
  (void)b;
  if (precision != 0 && precision != 1) throw Error(QCAD_ERR_INVALID_ARG, "precision must be 0 or 1");
  cudaStream_t s = m->stream;
  const long long n = m->n_nodes;
  const size_t es = precision == 0 ? sizeof(double) : sizeof(float);
  DevBuf v, y, c;
  v.ensure(n * es + 64);
  y.ensure(n * es + 64);
  c.ensure((size_t)m->n_elems * 8 * es + 64);
  CK(cudaMemsetAsync(v.p, 0, n * es, s));
  CK(cudaMemsetAsync(c.p, 0, (size_t)m->n_elems * 8 * es, s));
  const int rows[4] = {4, 8, 16, 32};
  const int chunks[5] = {8, 16, 32, 64, 128};
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best_ms = 1e30f;
  LaunchCfg best_cfg;
  for (int r : rows) {
    for (int ch : chunks) {
      if (ch > 2 * (int)m->nzn && ch != 8) continue;
      LaunchCfg cfg;
      cfg.by = r;
      cfg.kchunk = ch;
      auto run = [&]() {
        if (precision == 0) {
          ApplyArgs<double> a{};
          a.v = v.as<double>();
          a.y = y.as<double>();
          a.c = c.as<double>();
          launch_apply<double>(m->g64.g, a, cfg, s);
        } else {
          ApplyArgs<float> a{};
          a.v = v.as<float>();
          a.y = y.as<float>();
          a.c = c.as<float>();
          launch_apply<float>(m->g32.g, a, cfg, s);
        }
      };
      run();
      CK(cudaGetLastError());
      const int reps = 5;
      CK(cudaEventRecord(e0, s));
      for (int q = 0; q < reps; ++q) run();
      CK(cudaEventRecord(e1, s));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      ms /= reps;
      if (ms < best_ms) {
        best_ms = ms;
        best_cfg = cfg;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (precision == 0)
    m->cfg64 = best_cfg;
  else
    m->cfg32 = best_cfg;
  m->graph64.key = nullptr;
  m->graph32.key = nullptr;
  if (tile_rows) *tile_rows = best_cfg.by;
  if (z_chunk) *z_chunk = best_cfg.kchunk;
  if (best) *best = best_ms;
  return QCAD_OK;
}

qcad_status poisson_solve_batch(int n, const qcad_mesh_t* ms, const qcad_bias* bs, const qcad_solver_opts* o,
                                double* const* phis, qcad_solve_report* reps) {
  if (n < 1 || !ms || !bs || !o || !phis) throw Error(QCAD_ERR_INVALID_ARG, "invalid batch arguments");
  qcad_status worst = QCAD_OK;
  for (int i = 0; i < n; ++i) {
    if (!ms[i]) throw Error(QCAD_ERR_INVALID_ARG, "null mesh in batch");
    qcad_status st = poisson_solve(ms[i], &bs[i], o, nullptr, phis[i], reps ? &reps[i] : nullptr);
    if (st != QCAD_OK && worst == QCAD_OK) worst = st;
  }
  return worst;
}

}  // namespace qcad
