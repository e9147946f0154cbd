// Host-side mesh object of libqcad and its helpers.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <mutex>
#include <vector>

#include "../../include/qcad.h"
#include "qcad_dense.h"
#include "qcad_host.h"
#include "qcad_internal.cuh"

namespace qcad {

struct Error : std::runtime_error {
  qcad_status code;
  Error(qcad_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

void check_cuda(cudaError_t e, const char* what);
#define CK(x) ::qcad::check_cuda((x), #x)

// Owning device allocation.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  void ensure(size_t b) {
    if (bytes >= b && p) return;
    release();
    cudaError_t e = cudaMalloc(&p, b ? b : 16);
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      throw Error(e == cudaErrorMemoryAllocation ? QCAD_ERR_OOM : QCAD_ERR_CUDA,
                  std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    bytes = b;
  }
  template <class T>
  T* as() const { return reinterpret_cast<T*>(p); }
};

// Host helpers shared by mesh_create and the allocation-free residual (mesh.cu).
int validate_device(const qcad_device* dev);  // throws Error(INVALID_ARG); returns the layer count
Phys make_phys_material(const qcad_material& semiconductor, const qcad_bias* b);
void row_ops_raw(const double* x, int n, const double* kappa, double* M, double* K);

// Host description of one structured grid's 1D operator tables.
struct GridTables {
  std::vector<double> mx, kx, my, ky, mzx, mzy, kzz;
};

// Per-precision device copy of a grid's tables.
template <class T>
struct GridDev {
  DevBuf mx, kx, my, ky, mzx, mzy, kzz, zt, hx, hy, hz;
  Grid<T> g{};
};

// Kernel classes timed with CUDA events when profiling is enabled.
enum ProfClass { PROF_APPLY32 = 0, PROF_APPLY64, PROF_UPDATE32, PROF_UPDATE64, PROF_RESIDUAL, PROF_HM, PROF_MG, PROF_NCLASS };

struct Profiler {
  std::mutex mu;  // begin/end/harvest/add may come from two host threads
  bool on = false;
  long long launches[PROF_NCLASS] = {};
  double ms[PROF_NCLASS] = {};
  std::vector<std::pair<cudaEvent_t, int>> pending_start;  // (start event, class) awaiting stop
  std::vector<cudaEvent_t> pool;
  struct Pair {
    cudaEvent_t a, b;
    int cls;
  };
  std::vector<Pair> open;
  cudaEvent_t get();
  void begin(int cls, cudaStream_t s, Pair& out);
  void end(Pair& p, cudaStream_t s);
  void harvest();  // after a stream sync: accumulate elapsed times of completed pairs
  void add(int cls, double ms_);
  ~Profiler();
};

template <class T>
struct PcgBufs {
  DevBuf x, r, z, p, Ap, b, dinv, c, w, d;
};

struct PcgGraph {
  cudaGraphExec_t exec = nullptr;
  const void* key = nullptr;  // vector buffer the graph was captured with
  int degree = 0;             // Chebyshev degree the graph was captured with
  int chunk = 0;
  std::vector<Profiler::Pair> events;  // fixed event pairs inside the graph (profiling only)
  ~PcgGraph() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

}  // namespace qcad

struct qcad_mesh_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool owns_stream = false;
  // geometry
  int nx = 0, ny = 0, nz = 0;
  long long nxn = 0, nyn = 0, nzn = 0, n_nodes = 0, n_elems = 0;
  std::vector<double> xc, yc, zc;          // node coordinates
  std::vector<double> hxv, hyv, hzv;       // element sizes
  std::vector<int> layer_mat;              // per element layer
  std::vector<qcad_material> mats;
  int semi = -1;                           // index of the semiconductor material
  std::vector<unsigned char> layer_semi;
  std::vector<signed char> gate_top;       // gate id of top-plane nodes, -1 none
  int n_gates = 0;
  int wf_set = 0;
  double wf = 0.0;
  int bottom_ohmic = 1;
  qcad::DotBoxes dots{};
  int has_sub = 0;
  int sub[6] = {0, 0, 0, 0, 0, 0};
  // device geometry
  qcad::GridDev<double> g64;
  qcad::GridDev<float> g32;
  qcad::DevBuf d_xn, d_yn, d_zn, d_layer_semi, d_gate_top, d_dir_top, d_vgate;
  qcad::DevBuf d_wq;  // [nz][8] the residual's per-layer load table (slots in physics.cuh)
  qcad::DevBuf d_ecode;  // [n_elems] the residual's per-element load codes (kernels_poisson.cu)
  // surface terms (charged gates under the Robin condition, surface charges): the face
  // coefficients eps_r/d of the top plane (FP64 and FP32, in the grids' face_alpha), the
  // constant load b = sum_sheets (q/eps0) sigma int N + sum_charged ((eps_r/d) phi_0 + (q/eps0)
  // sigma) int N (nodal FP64; its top plane is rebuilt for every bias), and per charged gate
  // its top-plane vector (eps_r/d) int N (host, nxn*nyn), the d b / d V_g of the adjoint
  bool has_surface = false;                      // any surface term (the residual carries b)
  bool has_robin = false;                        // charged gates (the linear operators carry K_R)
  std::vector<int> charged_gate;                 // gate index of each charged gate
  std::vector<std::vector<double>> charged_r;    // its (eps_r/d) int_f N_a on the top plane
  std::vector<double> bsig_top;                  // bias-independent load on the top plane
  std::vector<double> btop;                      // host staging of the top plane of b
  qcad::DevBuf d_face64, d_face32, d_bsurf, d_charged_r;  // d_charged_r: charged_r concatenated
  // solver state
  qcad::PcgBufs<double> k64;
  qcad::PcgBufs<float> k32;
  qcad::PcgBufs<float> k32x[QCAD_MAX_DOTS - 1];  // further FP32 right-hand sides (adjoint of dots 1, 2, ...)
  qcad::DevBuf scal_x;                           // their PCG scalars
  std::shared_ptr<void> adj_ctx;                 // cached batched-PCG context of the adjoint
  std::shared_ptr<void> mg;                      // multigrid hierarchy (built on first use)
  // self-consistent Schrodinger-Poisson loop: quantum density of the residual while active
  qcad::QuantumDensity qd{};
  bool qd_active = false;
  qcad::DevBuf sp_w, sp_phiq, sp_vxq, sp_evecs, sp_prev;
  qcad::DevBuf phi_a, phi_b, R, diag, stats, counts, scal, scratch;
  qcad::DevBuf el_res;                     // residual corner contributions, 16 doubles per element
  qcad::PcgScalars* h_scal = nullptr;      // pinned host mirror
  double* h_small = nullptr;               // pinned host scratch (64 doubles)
  // second stream and scratch for an eigensolve that runs concurrently with the mesh stream
  cudaStream_t stream2 = nullptr;
  qcad::DevBuf stats2;
  double* h_small2 = nullptr;
  qcad::PcgGraph graph64, graph32;
  // residual passes (16-row tiles: the FP64 node pass is pipe-bound, so its halo rows cost the most),
  // FP64 and FP32 operators
  qcad::LaunchCfg cfg_res{16, 16, 3}, cfg64, cfg32;
  int cheb_auto[2] = {0, 0};               // autotuned Chebyshev degree per precision (0 = not yet)
  int batch_kchunk = 0;                    // z chunk of this mesh in batched launches (0 = not tuned)
  // largest eigenvalue of D^-1 J of the stored linearization per precision, valid while
  // lam_ver matches lin_ver (lin_ver counts the residual evaluations that rewrote it)
  long long lin_ver[2] = {0, 0};
  long long lam_ver[2] = {-1, -1};
  double lam_cache[2] = {0.0, 0.0};
  qcad::Profiler prof;                     // thread-safe: concurrent calls may record
  // Schrodinger workspace
  qcad::DevBuf s_mx, s_kx, s_my, s_ky, s_mzx, s_mzy, s_kzz, s_cV, s_dinv, s_interior, s_blocks, s_gram;
  ~qcad_mesh_s();
};
