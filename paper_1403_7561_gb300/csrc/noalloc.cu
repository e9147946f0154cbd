// Allocation-free residual evaluation.
//
// Some callers cannot allocate device memory: code running inside another
// framework's memory pool or allocator hooks, in a real-time loop that forbids
// cudaMalloc/cudaFree, or in a process whose device allocator is owned by
// someone else. qcad_poisson_residual_noalloc serves them: it evaluates the
// same FP64 residual as qcad_poisson_residual without a mesh object and
// without allocating device memory. The caller passes the device description,
// phi and R; the per-call scratch (geometry tables, contact masks and the
// reduction accumulators) lives in one file-scope device array of
// QCAD_NOALLOC_SCRATCH_BYTES that every GPU loading this library keeps until
// process exit. Host-side tables are staged in a static host buffer of the
// same size, so a successful call performs no heap allocation either.
//
// The description is checked exactly as qcad_mesh_create checks it (the same
// host function), plus the scratch limit. Every call shares the array and
// leaves the last call's contents in it; accumulators are cleared at the start
// of each call. Calls whose GPU work overlaps (different streams, or different
// host threads on one device) race on the array; the host side is serialized
// by a mutex, the device side is not. The first call on a device looks up the
// array's device address (cudaGetSymbolAddress) with that device current.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/qcad.h"
#include "mesh.h"

#define QCAD_NOALLOC_SCRATCH_BYTES (2u << 20)
#define QCAD_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_noalloc_scratch[QCAD_NOALLOC_SCRATCH_BYTES];

namespace qcad {
void set_message(const std::string& msg);

namespace {

std::mutex g_noalloc_mu;
void* g_noalloc_addr[QCAD_NOALLOC_MAX_DEVICES] = {};
alignas(256) unsigned char g_stage[QCAD_NOALLOC_SCRATCH_BYTES];

// Bump allocator over a fixed region (host staging and device scratch share offsets).
struct Arena {
  size_t off = 0;
  bool ok = true;
  size_t take(size_t bytes) {
    const size_t o = (off + 255) & ~(size_t)255;
    if (o + bytes > QCAD_NOALLOC_SCRATCH_BYTES) {
      ok = false;
      return 0;
    }
    off = o + bytes;
    return o;
  }
};

}  // namespace

qcad_status noalloc_residual(const qcad_device* dev, const qcad_bias* b, void* stream, const double* theta,
                             const double* phi, double* R, double* stats) {
  if (!dev || !b || !phi || !R) {
    set_message("null device description, bias, phi or R");
    return QCAD_ERR_INVALID_ARG;
  }
  if (!(b->T > 0) || !std::isfinite(b->T)) {
    set_message("temperature must be > 0");
    return QCAD_ERR_INVALID_ARG;
  }
  // the checks of qcad_mesh_create, including the 32-bit index limits of the kernels
  const int nz = validate_device(dev);
  if (dev->n_charged_gates != 0 || dev->n_surface_charges != 0) {
    set_message("the allocation-free residual does not take charged gates or surface charges");
    return QCAD_ERR_INVALID_ARG;
  }
  const int nx = dev->nx, ny = dev->ny;
  const long long nxn = nx + 1, nyn = ny + 1, nzn = nz + 1;
  int semi = -1;  // the semiconductor material (validate_device allows one)
  for (int i = 0; i < dev->n_materials; ++i)
    if (dev->materials[i].semiconductor) semi = i;
  const qcad_material& s = dev->materials[semi >= 0 ? semi : 0];

  // Scratch layout (same offsets in the host staging buffer and the device array).
  Arena A;
  const size_t o_stats = A.take(2 * sizeof(double));
  const size_t o_x = A.take(nxn * sizeof(double)), o_y = A.take(nyn * sizeof(double)),
               o_z = A.take(nzn * sizeof(double));
  const size_t o_hx = A.take(nx * sizeof(double)), o_hy = A.take(ny * sizeof(double)),
               o_hz = A.take(nz * sizeof(double)), o_eps = A.take(nz * sizeof(double));
  const size_t o_mx = A.take(3 * nxn * sizeof(double)), o_kx = A.take(3 * nxn * sizeof(double));
  const size_t o_my = A.take(3 * nyn * sizeof(double)), o_ky = A.take(3 * nyn * sizeof(double));
  const size_t o_mz = A.take(3 * nzn * sizeof(double)), o_kz = A.take(3 * nzn * sizeof(double));
  const size_t o_semi = A.take(nz), o_dir = A.take(nxn * nyn);
  if (!A.ok) {
    set_message("mesh too large for the allocation-free scratch (" +
                std::to_string(QCAD_NOALLOC_SCRATCH_BYTES) + " bytes)");
    return QCAD_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  int device = -1;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess || device < 0 || device >= QCAD_NOALLOC_MAX_DEVICES) {
    set_message("no usable current CUDA device");
    return QCAD_ERR_CUDA;
  }
  if (g_noalloc_addr[device] == nullptr) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || ptr == nullptr) {
      cudaGetLastError();
      set_message(std::string("cudaGetSymbolAddress of the static scratch failed: ") + cudaGetErrorString(e));
      return QCAD_ERR_CUDA;
    }
    g_noalloc_addr[device] = ptr;
  }
  unsigned char* dbase = static_cast<unsigned char*>(g_noalloc_addr[device]);

  unsigned char* H = g_stage;
  double* x = reinterpret_cast<double*>(H + o_x);
  double* y = reinterpret_cast<double*>(H + o_y);
  double* z = reinterpret_cast<double*>(H + o_z);
  double* hx = reinterpret_cast<double*>(H + o_hx);
  double* hy = reinterpret_cast<double*>(H + o_hy);
  double* hz = reinterpret_cast<double*>(H + o_hz);
  double* eps = reinterpret_cast<double*>(H + o_eps);
  unsigned char* lsemi = H + o_semi;
  unsigned char* dtop = H + o_dir;
  for (int i = 0; i <= nx; ++i) x[i] = dev->Lx * i / nx;
  for (int j = 0; j <= ny; ++j) y[j] = dev->Ly * j / ny;
  z[0] = 0.0;
  int k = 0;
  for (int L = 0; L < dev->n_layers; ++L) {
    const double z0 = z[k];
    const qcad_material& mat = dev->materials[dev->layer_material[L]];
    for (int q = 0; q < dev->layer_n[L]; ++q) {
      z[k + 1] = z0 + dev->layer_thickness[L] * (q + 1) / dev->layer_n[L];
      eps[k] = mat.eps_r;
      lsemi[k] = (unsigned char)(mat.semiconductor ? 1 : 0);
      ++k;
    }
  }
  for (int i = 0; i < nx; ++i) hx[i] = x[i + 1] - x[i];
  for (int j = 0; j < ny; ++j) hy[j] = y[j + 1] - y[j];
  for (int q = 0; q < nz; ++q) hz[q] = z[q + 1] - z[q];
  row_ops_raw(x, nx, nullptr, reinterpret_cast<double*>(H + o_mx), reinterpret_cast<double*>(H + o_kx));
  row_ops_raw(y, ny, nullptr, reinterpret_cast<double*>(H + o_my), reinterpret_cast<double*>(H + o_ky));
  row_ops_raw(z, nz, eps, reinterpret_cast<double*>(H + o_mz), reinterpret_cast<double*>(H + o_kz));
  for (long long j = 0; j < nyn; ++j)
    for (long long i = 0; i < nxn; ++i) {
      unsigned char in = 0;
      for (int g = 0; g < dev->n_gates && !in; ++g) {
        const qcad_rect& G = dev->gates[g];
        in = (x[i] >= G.x0 && x[i] <= G.x1 && y[j] >= G.y0 && y[j] <= G.y1) ? 1 : 0;
      }
      dtop[i + nxn * j] = in;
    }

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // one copy of everything after the accumulators, then clear the accumulators
  const size_t first = o_x, bytes = A.off - o_x;
  e = cudaMemcpyAsync(dbase + first, H + first, bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dbase + o_stats, 0, 2 * sizeof(double), st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_message(std::string("staging the scratch failed: ") + cudaGetErrorString(e));
    return QCAD_ERR_CUDA;
  }

  Grid<double> g{};
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.nxn = (int)nxn;
  g.nyn = (int)nyn;
  g.nzn = (int)nzn;
  g.plane = nxn * nyn;
  g.mx = reinterpret_cast<const double*>(dbase + o_mx);
  g.kx = reinterpret_cast<const double*>(dbase + o_kx);
  g.my = reinterpret_cast<const double*>(dbase + o_my);
  g.ky = reinterpret_cast<const double*>(dbase + o_ky);
  g.mzx = reinterpret_cast<const double*>(dbase + o_mz);
  g.mzy = reinterpret_cast<const double*>(dbase + o_mz);
  g.kzz = reinterpret_cast<const double*>(dbase + o_kz);
  g.hx = reinterpret_cast<const double*>(dbase + o_hx);
  g.hy = reinterpret_cast<const double*>(dbase + o_hy);
  g.hz = reinterpret_cast<const double*>(dbase + o_hz);
  g.dir_top = dbase + o_dir;
  g.dir_bottom = dev->bottom_ohmic;
  g.dir_boundary = 0;

  const Phys P = make_phys_material(s, b);

  ResidualArgs a{};
  a.phi = phi;
  a.theta = theta;
  a.R = R;
  a.layer_semi = dbase + o_semi;
  a.xn = reinterpret_cast<const double*>(dbase + o_x);
  a.yn = reinterpret_cast<const double*>(dbase + o_y);
  a.zn = reinterpret_cast<const double*>(dbase + o_z);
  a.P = P;
  a.dots.n = 0;
  a.stats = reinterpret_cast<double*>(dbase + o_stats);
  a.linear = 0;
  LaunchCfg cfg;
  launch_residual(g, a, cfg, st);
  e = cudaGetLastError();
  double hs[2] = {0.0, 0.0};
  if (e == cudaSuccess && stats) e = cudaMemcpyAsync(hs, dbase + o_stats, sizeof(hs), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_message(std::string("residual launch failed: ") + cudaGetErrorString(e));
    return QCAD_ERR_CUDA;
  }
  if (stats) {
    stats[0] = hs[0];
    stats[1] = hs[1];
  }
  return QCAD_OK;
}

}  // namespace qcad
