// Batched kernels: one launch covers the PCG apply (or update) of every
// instance of a batch of meshes of different sizes. A work table maps each
// block to (instance, tile); each instance keeps its own device-resident PCG
// scalars, so instances converge and drop out independently (their blocks
// return at once). Included at the end of kernels_poisson.cu, whose operator
// ops and PCG bookkeeping it reuses.
#pragma once

namespace qcad {

// Index of the last table entry whose begin <= b (entries sorted by begin).
template <class E>
__device__ __forceinline__ int batch_find(const E* tab, int n, int b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tab[mid].begin <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

template <int BY>
__global__ void __launch_bounds__(QCAD_BX * BY) batch_pcg_apply_kernel(const BatchApplyEntry* tab, int n_inst) {
  const int b = blockIdx.x;
  const BatchApplyEntry& e = tab[batch_find(tab, n_inst, b)];
  const int local = b - e.begin;
  const int bx = local % e.tiles_x;
  const int by = (local / e.tiles_x) % e.tiles_y;
  const int bz = local / (e.tiles_x * e.tiles_y);
  PcgApplyOp<float> op = {};
  op.v = e.v;
  op.sc = e.sc;
  march_body<float, BY, PcgApplyOp<float>>(e.g, op, e.kchunk, bx, by, bz);
}

__global__ void __launch_bounds__(VEC_THREADS) batch_pcg_update_kernel(const BatchVecEntry* tab, int n_inst) {
  const int b = blockIdx.x;
  const BatchVecEntry& e = tab[batch_find(tab, n_inst, b)];
  pcg_update_body<float>(e.n, e.v, e.sc, b - e.begin, e.blocks);
}

// status[i] = {done, t, nonfinite, iters} of instance i (one read for the whole batch).
__global__ void batch_status_kernel(const BatchVecEntry* tab, int n_inst, int* status) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_inst; i += gridDim.x * blockDim.x) {
    const PcgScalars* sc = tab[i].sc;
    status[4 * i + 0] = sc->done;
    status[4 * i + 1] = sc->t;
    status[4 * i + 2] = sc->nonfinite;
    status[4 * i + 3] = sc->iters;
  }
}

template <int BY>
__global__ void __launch_bounds__(QCAD_BX * BY) batch_residual_kernel(const BatchResEntry* tab, int n_inst) {
  const int b = blockIdx.x;
  const BatchResEntry& e = tab[batch_find(tab, n_inst, b)];
  const int local = b - e.begin;
  const int bx = local % e.tiles_x;
  const int by = (local / e.tiles_x) % e.tiles_y;
  const int bz = local / (e.tiles_x * e.tiles_y);
  ResidualOp op = {};
  op.a = e.a;
  march_body<double, BY, ResidualOp>(e.g, op, e.kchunk, bx, by, bz);
}

// Entry of block b for the Gauss-point pass (entries sorted by qbegin).
__device__ __forceinline__ int batch_find_q(const BatchResEntry* tab, int n, int b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tab[mid].qbegin <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Two-pass residual over the instances: Gauss-point pass, then the node gather.
__global__ void __launch_bounds__(256) batch_residual_qp_kernel(const BatchResEntry* tab, int n_inst) {
  const int b = blockIdx.x;
  const BatchResEntry& e = tab[batch_find_q(tab, n_inst, b)];
  const long long ne = (long long)e.g.nx * e.g.ny * e.g.nz;
  residual_qp_body(e.g, e.a, e.el, e.el + 8 * ne, (long long)(b - e.qbegin) * 256 + threadIdx.x);
}

template <int BY>
__global__ void __launch_bounds__(QCAD_BX * BY) batch_residual_gather_kernel(const BatchResEntry* tab, int n_inst) {
  const int b = blockIdx.x;
  const BatchResEntry& e = tab[batch_find(tab, n_inst, b)];
  const int local = b - e.begin;
  const int bx = local % e.tiles_x;
  const int by = (local / e.tiles_x) % e.tiles_y;
  const int bz = local / (e.tiles_x * e.tiles_y);
  const long long ne = (long long)e.g.nx * e.g.ny * e.g.nz;
  const ResidualGatherOp op = make_gather_op(e.a, e.el, e.el + 8 * ne);
  march_body<double, BY, ResidualGatherOp>(e.g, op, e.kchunk, bx, by, bz);
}

__global__ void batch_stats_kernel(const BatchResEntry* tab, int n_inst, int mode, double* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_inst; i += gridDim.x * blockDim.x) {
    double* st = tab[i].a.stats;
    if (mode == 0) {
      st[0] = 0.0;
      st[1] = 0.0;
    } else if (mode == 1) {
      st[8] = 0.0;
    } else {
      out[3 * i + 0] = st[0];
      out[3 * i + 1] = st[1];
      out[3 * i + 2] = st[8];
    }
  }
}

void launch_batch_residual(const BatchResEntry* tab, int n_inst, int total_blocks, cudaStream_t s) {
  note_launch(), batch_residual_kernel<8><<<total_blocks, dim3(QCAD_BX, 8), 0, s>>>(tab, n_inst);
}

void launch_batch_residual_2pass(const BatchResEntry* tab, int n_inst, int qp_blocks, int node_blocks,
                                 cudaStream_t s) {
  note_launch(), batch_residual_qp_kernel<<<qp_blocks, 256, 0, s>>>(tab, n_inst);
  note_launch(), batch_residual_gather_kernel<8><<<node_blocks, dim3(QCAD_BX, 8), 0, s>>>(tab, n_inst);
}

void launch_batch_stats(const BatchResEntry* tab, int n_inst, int mode, double* out, cudaStream_t s) {
  note_launch(), batch_stats_kernel<<<(n_inst + 127) / 128, 128, 0, s>>>(tab, n_inst, mode, out);
}

void launch_batch_pcg_apply(const BatchApplyEntry* tab, int n_inst, int total_blocks, int by, cudaStream_t s) {
  if (by == 16)
    note_launch(), batch_pcg_apply_kernel<16><<<total_blocks, dim3(QCAD_BX, 16), 0, s>>>(tab, n_inst);
  else
    note_launch(), batch_pcg_apply_kernel<8><<<total_blocks, dim3(QCAD_BX, 8), 0, s>>>(tab, n_inst);
}

void launch_batch_pcg_update(const BatchVecEntry* tab, int n_inst, int total_blocks, cudaStream_t s) {
  note_launch(), batch_pcg_update_kernel<<<total_blocks, VEC_THREADS, 0, s>>>(tab, n_inst);
}

void launch_batch_status(const BatchVecEntry* tab, int n_inst, int* status, cudaStream_t s) {
  note_launch(), batch_status_kernel<<<(n_inst + 127) / 128, 128, 0, s>>>(tab, n_inst, status);
}

}  // namespace qcad
