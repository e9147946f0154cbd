// Batched Poisson solves and the launch-configuration autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstring>
#include <vector>

#include "mesh.h"

namespace qcad {

qcad_status poisson_solve(qcad_mesh_s* m, const qcad_bias* b, const qcad_solver_opts* o, const double* theta,
                          double* phi, qcad_solve_report* rep);

// Times the Jacobian apply (zero input and coefficients: the time does not depend on the
// values) for every (variant, tile rows, z chunk) candidate and keeps the fastest for that
// precision.
qcad_status autotune(qcad_mesh_s* m, const qcad_bias* b, int precision, int* variant_out, int* tile_rows,
                     int* z_chunk, float* best) {
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
  const int chunks[5] = {8, 16, 32, 64, 128};
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best_ms = 1e30f;
  LaunchCfg best_cfg;
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device));
  // (variant, warps) shapes: element-gather 0, element-gather with two nodes per thread 1
  // (FP32), plane-factorized with one 2 or two 3 node rows per thread
  // (charged gates: the element-gather kernels alone carry the Robin face term)
  std::vector<std::pair<int, int>> shapes;
  for (int r : {4, 8, 16, 32}) shapes.push_back({0, r});
  if (precision == 1 && !m->has_robin)
    for (int r : {4, 8, 16}) shapes.push_back({1, r});
  for (int r : {4, 8, 16, 32})
    if ((precision == 1 || r <= 8) && !m->has_robin) shapes.push_back({2, r});
  for (int r : {4, 8, 16})
    if ((precision == 1 || r <= 8) && !m->has_robin) shapes.push_back({3, r});
  for (const auto& sh : shapes) {
    const int variant = sh.first, r = sh.second;
    // z-chunk lengths that put whole waves of resident blocks on the SMs, plus fixed ones
    const int bps = apply_blocks_per_sm(precision, r, variant);
    const int cols = variant == 1 ? 60 : 30;
    const int trows = (variant == 3 ? 2 * r : r) - 2;
    const long long tiles_xy = (long long)((m->nxn + cols - 1) / cols) * ((m->nyn + trows - 1) / trows);
    std::vector<int> cands(chunks, chunks + 5);
    for (int w = 1; w <= 6 && bps > 0; ++w) {
      const long long nch = std::max<long long>(1, (long long)w * sms * bps / std::max<long long>(1, tiles_xy));
      cands.push_back((int)std::max<long long>(2, (m->nzn + nch - 1) / nch));
    }
    std::sort(cands.begin(), cands.end());
    cands.erase(std::unique(cands.begin(), cands.end()), cands.end());
    for (int ch : cands) {
      if (ch > 2 * (int)m->nzn && ch != 8) continue;
      LaunchCfg cfg;
      cfg.by = r;
      cfg.kchunk = ch;
      cfg.variant = variant;
      auto run = [&]() {
        if (precision == 0) {
          ApplyArgs<double> a{};
          a.v = v.as<double>();
          a.y = y.as<double>();
          a.c = c.as<double>();
          launch_apply<double>(m->g64.g, a, cfg, s, m->has_robin ? m->d_face64.as<double>() : nullptr);
        } else {
          ApplyArgs<float> a{};
          a.v = v.as<float>();
          a.y = y.as<float>();
          a.c = c.as<float>();
          launch_apply<float>(m->g32.g, a, cfg, s, m->has_robin ? m->d_face32.as<float>() : nullptr);
        }
      };
      run();
      CK(cudaGetLastError());
      const int reps = 20;
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
  if (variant_out) *variant_out = best_cfg.variant;
  if (tile_rows) *tile_rows = best_cfg.by;
  if (z_chunk) *z_chunk = best_cfg.kchunk;
  if (best) *best = best_ms;
  return QCAD_OK;
}

qcad_status poisson_solve_batch_impl(int n, const qcad_mesh_t* ms, const qcad_bias* bs, const qcad_solver_opts* o,
                                     double* const* phis, qcad_solve_report* reps);

// z-chunk of the batched FP32 apply (plane-factorized, 8 warps, two rows per thread) for one
// mesh: the fastest of a few lengths, timed on the mesh's own grid.
static int tune_batch_kchunk(qcad_mesh_s* m) {
  cudaStream_t s = m->stream;
  const long long n = m->n_nodes;
  DevBuf v, y, c;
  v.ensure(n * sizeof(float) + 64);
  y.ensure(n * sizeof(float) + 64);
  c.ensure((size_t)m->n_elems * 8 * sizeof(float) + 64);
  CK(cudaMemsetAsync(v.p, 0, n * sizeof(float), s));
  CK(cudaMemsetAsync(c.p, 0, (size_t)m->n_elems * 8 * sizeof(float), s));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int best = 32;
  float best_ms = 1e30f;
  for (int ch : {8, 16, 32, 64}) {
    LaunchCfg cfg;
    cfg.by = 8;
    cfg.kchunk = ch;
    cfg.variant = 3;
    ApplyArgs<float> a{};
    a.v = v.as<float>();
    a.y = y.as<float>();
    a.c = c.as<float>();
    launch_apply<float>(m->g32.g, a, cfg, s);
    CK(cudaEventRecord(e0, s));
    for (int q = 0; q < 10; ++q) launch_apply<float>(m->g32.g, a, cfg, s);
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best_ms) {
      best_ms = ms;
      best = ch;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

// Batched solve: one timing run per size bucket sets the z chunk of every instance of that
// bucket in the shared work table (a mesh keeps its chunk across calls).
qcad_status poisson_solve_batch(int n, const qcad_mesh_t* ms, const qcad_bias* bs, const qcad_solver_opts* o,
                                double* const* phis, qcad_solve_report* reps) {
  if (n < 1 || !ms || !bs || !o || !phis) throw Error(QCAD_ERR_INVALID_ARG, "invalid batch arguments");
  // one tuning run per size bucket (meshes with equal element counts per axis)
  std::vector<std::pair<std::array<int, 3>, int>> buckets;
  for (int i = 0; i < n; ++i) {
    if (!ms[i]) throw Error(QCAD_ERR_INVALID_ARG, "null mesh in batch");
    if (ms[i]->has_surface)
      throw Error(QCAD_ERR_INVALID_ARG, "the batched solve does not take charged gates or surface charges");
    const std::array<int, 3> key = {ms[i]->nx, ms[i]->ny, ms[i]->nz};
    int ch = -1;
    for (auto& b : buckets)
      if (b.first == key) ch = b.second;
    if (ch < 0) {
      ch = ms[i]->batch_kchunk > 0 ? ms[i]->batch_kchunk : tune_batch_kchunk(ms[i]);
      buckets.push_back({key, ch});
    }
    ms[i]->batch_kchunk = ch;
  }
  return poisson_solve_batch_impl(n, ms, bs, o, phis, reps);
}

}  // namespace qcad
