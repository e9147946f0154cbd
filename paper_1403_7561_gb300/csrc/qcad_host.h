// Host-side interfaces between the kernel translation units and the solver
// driver of libqcad (not part of the public C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "qcad_internal.cuh"

namespace qcad {

// Device-resident scalars of one preconditioned CG solve. Slots are indexed
// by iteration modulo 4 so that a kernel can accumulate the next dot product
// while the current one is still being read; t is advanced by the last block
// of the update kernel, so a captured sequence of kernels needs no host input.
struct PcgScalars {
  double rz[4];
  double pAp[4];
  double rr[4];
  double rr0;
  double tol2;
  int t;
  int done;
  int iters;
  int maxit;
  unsigned int counter;
  int nonfinite;
  // Chebyshev-Jacobi preconditioner: degree (1 = Jacobi), spectral interval [theta - delta,
  // theta + delta] of D^-1 J, and the phase of the solve (0 during the initial residual, 1 after)
  int degree;
  int phase;
  double theta;
  double delta;
};

template <class T>
struct PcgVecs {
  T* x;
  T* r;
  T* z;
  T* p[2];     // search direction, ping-ponged by iteration parity
  T* Ap;
  const T* b;
  const T* dinv;
  const T* c;   // element quadrature coefficients of the operator (8 per element)
  T* w;         // Chebyshev inner residual
  T* d[2];      // Chebyshev correction, ping-ponged by step parity
};

struct ResidualArgs {
  const double* phi;
  const double* theta;       // fixed charge per element or null
  double* R;
  double* diag;              // or null
  double* c64;               // or null
  float* c32;                // or null
  double* dinv64;            // or null
  float* dinv32;             // or null
  double* b64;               // -R or null
  float* b32;                // -R or null
  const unsigned char* layer_semi;
  const double* xn;          // node coordinates (for dot membership)
  const double* yn;
  const double* zn;
  Phys P;
  DotBoxes dots;
  double* counts;            // [n_dots] accumulated electron counts or null
  double* stats;             // [2] {max|R| (as ordered bits), sum R^2} or null
  int linear;
  QuantumDensity qd;         // quantum density in the quantum region (inactive: qd.w null)
  const double* bsurf;       // [n_nodes] constant surface load b (R -= b; two-pass residual) or null
  const double* wq;          // [nz][8] per-layer load table of constant-charge elements (physics.cuh) or null
  unsigned char* ecode;      // [n_elems] per-element load code between the two residual passes, or null
};

template <class T>
struct ApplyArgs {
  const T* v;
  T* y;
  const T* c;
  double* dot;   // accumulate v.y (writer nodes) or null
  int raw;       // 1: no identity override on Dirichlet rows (adjoint column sums)
};

// Launch shape of the z-marching kernels: by warps (tile rows) per block, kchunk node planes
// per block, and for the linear operators the kernel variant: 0 element-gather, 1 element-gather
// with two nodes per thread and packed f32x2 arithmetic (FP32 only), 2 plane-factorized with one
// node row per thread, 3 plane-factorized with two node rows per thread.
struct LaunchCfg {
  int by = 8;
  int kchunk = 16;
  int variant = 3;
};

void launch_residual(const Grid<double>& g, const ResidualArgs& a, LaunchCfg cfg, cudaStream_t s);
// Adds the electron count of the elements [box0, box1) x [box2, box3) x [box4, box5) to *out.
void launch_dot_count(const Grid<double>& g, const double* phi, const unsigned char* layer_semi, const Phys& P,
                      const int box[6], double* out, cudaStream_t s);
// Same outputs in two passes (carrier density once per quadrature point); el: 16 doubles per element.
// face: the charged gates' [nx*ny] face coefficients (Robin condition) or null; with a.bsurf set,
// the surface load is subtracted and the face mass enters the stiffness and the diagonal.
void launch_residual_2pass(const Grid<double>& g, const ResidualArgs& a, double* el, LaunchCfg cfg, cudaStream_t s,
                           const double* face = nullptr);

template <class T>
void launch_apply(const Grid<T>& g, const ApplyArgs<T>& a, LaunchCfg cfg, cudaStream_t s, const T* face = nullptr);

template <class T>
void launch_pcg_init(long long n, PcgVecs<T> v, PcgScalars* sc, cudaStream_t s);
template <class T>
void launch_pcg_apply(const Grid<T>& g, PcgVecs<T> v, PcgScalars* sc, LaunchCfg cfg, cudaStream_t s,
                      const T* face = nullptr);
template <class T>
void launch_pcg_update(long long n, PcgVecs<T> v, PcgScalars* sc, cudaStream_t s);
// Chebyshev-Jacobi form: the update kernel starts the recurrence (w = r, d = D^-1 r / theta,
// z = d) and step j = 1..degree-1 applies J to d_{j-1}; the last step forms r.z and finishes
// the iteration (or the initial residual when phase = 0).
template <class T>
void launch_pcg_update_cheb(long long n, PcgVecs<T> v, PcgScalars* sc, cudaStream_t s);
template <class T>
void launch_pcg_init_cheb(long long n, PcgVecs<T> v, PcgScalars* sc, cudaStream_t s);
template <class T>
void launch_cheb_step(const Grid<T>& g, PcgVecs<T> v, PcgScalars* sc, int step, int last, LaunchCfg cfg,
                      cudaStream_t s, const T* face = nullptr);
// One power step for the largest eigenvalue of D^-1 J: v_next = D^-1 (J v) / |.|; acc[0] += v.Jv,
// acc[1] += v.D v, acc[2] += |D^-1 J v|^2 (the caller normalizes with acc[2]).
template <class T>
void launch_power_step(long long n, const T* v, const T* Jv, const T* dinv, T* vnext, double* acc, cudaStream_t s);
template <class T>
void launch_scale(long long n, T* v, double a, cudaStream_t s);
template <class T>
void launch_random_free(const Grid<T>& g, unsigned long long seed, T* v, cudaStream_t s);

// phi_out = phi + alpha * delta on every node; stats[0] accumulates max |alpha delta| (ordered bits).
template <class T>
void launch_newton_trial(long long n, const double* phi, const T* delta, double alpha, double* phi_out,
                         double* stats, cudaStream_t s);

// Dirichlet values: bottom plane (if set) gets v_bottom, top-plane nodes with gate id >= 0 get v_gate[id].
void launch_set_dirichlet(long long nxn, long long nyn, long long nzn, int bottom, double v_bottom,
                          const signed char* gate_top, const double* v_gate, double* phi, cudaStream_t s);

// Elementwise conversions.
void launch_d2f(long long n, const double* a, float* b, cudaStream_t s);
void launch_f2d(long long n, const float* a, double* b, cudaStream_t s);

// dN_d/dphi as a nodal vector for dot d: sum over dot elements of w|J| n'(phi_q) N_a(q), written
// at the nodes of the dot's element box (the caller zeroes out beforehand). box: the
// dot's element box {i0, i1, j0, j1, k0, k1} (elements i0 <= i < i1, ...) or null when it is empty;
// el: scratch of 8 doubles per box element.
void launch_count_gradient(const Grid<double>& g, const double* phi, const unsigned char* layer_semi,
                           const double* xn, const double* yn, const double* zn, const Phys& P,
                           const DotBoxes& dots, int d, const int* box, double* out, double* el, cudaStream_t s);

// theta-gradient of N_d: out[e] = qe * (|e|/8) * sum of lam over the 8 corners of e (lam is
// zero on Dirichlet nodes); |e|/8 = int_e N_a exactly on a box.
void launch_theta_gradient(int nx, int ny, int nz, const double* hx, const double* hy, const double* hz,
                           const double* lam, double qe, double* out, cudaStream_t s);

// Schrodinger operators on the subdomain grid (field 0: H, field 1: M).
template <class T>
struct HmArgs {
  const T* x;      // nvec full-subdomain vectors, stride ldx
  T* hx;           // or null
  T* mx;           // or null
  const T* cV;     // V * w|J| at the qp of every subdomain element
  long long ld;    // vector stride (n_sub_nodes)
  int nvec;
  double mscale;   // 1 / kappa_x: the consistent mass is the kappa_x-weighted z mass stencil times this
};
// variant >= 2: plane-factorized kernel (M applied as the separable mass stencil), else
// element-gather.
template <class T>
void launch_hm_apply(const Grid<T>& g, const HmArgs<T>& a, LaunchCfg cfg, cudaStream_t s);
template <class T>
void launch_hm_apply_lin(const Grid<T>& g, const HmArgs<T>& a, LaunchCfg cfg, cudaStream_t s);
// One fused step of the LOBPCG Chebyshev-Jacobi block preconditioner (kernels_lin.cu): the H apply
// of D_in (nvec columns at stride ld, coefficients cV) with the recurrence W -= H D_in,
// D_out = c1 D_in + c2 D^-1 W, Z += D_out in its epilogue.
struct ChebHmArgs {
  const float* din;
  float* dout;
  float* w;
  float* z;
  const float* dinv;
  const float* cV;
  long long ld;
  int nvec;
  float c1, c2;
};
void launch_cheb_hm_step(const Grid<float>& g, const ChebHmArgs& args, cudaStream_t s);
struct dfl;
// The H and M applies of FP64 vectors in double-float arithmetic on the FP32 pipes (g: the
// subdomain grid's tables as double-float pairs; a.cV the FP64 coefficients).
void launch_hm_apply_df(const Grid<dfl>& g, const HmArgs<double>& a, cudaStream_t s);

}  // namespace qcad

namespace qcad {
template <class T>
void launch_dot(long long n, const T* a, const T* b, double* out, cudaStream_t s);
template <class T>
void launch_axpy(long long n, double a, const T* x, double* y, cudaStream_t s);
void launch_sub(long long n, const double* g, const double* y, double* r, float* r32, cudaStream_t s);
}  // namespace qcad

namespace qcad {
// Kernel launches issued by the library (graph replays count their kernels).
void note_launch(int n = 1);
long long launch_count();
}  // namespace qcad

namespace qcad {
// Plane-factorized launches of the linear ops (variants 2 and 3).
template <class T>
void launch_apply_lin(const Grid<T>& g, const ApplyArgs<T>& args, LaunchCfg cfg, cudaStream_t s);
template <class T>
void launch_pcg_apply_lin(const Grid<T>& g, PcgVecs<T> vecs, PcgScalars* sc, LaunchCfg cfg, cudaStream_t s);
template <class T>
void launch_cheb_step_lin(const Grid<T>& g, PcgVecs<T> vecs, PcgScalars* sc, int step, int last, LaunchCfg cfg,
                          cudaStream_t s);
int lin_blocks_per_sm(int precision, int by, int rows);

// Resident blocks per SM of the Jacobian apply of a precision (0 FP64, 1 FP32) and variant.
int apply_blocks_per_sm(int precision, int by, int variant);

// Work-table entries of the batched kernels (sorted by begin = first block of the entry).
struct BatchApplyEntry {
  Grid<float> g;
  PcgVecs<float> v;
  PcgScalars* sc;
  int kchunk;
  int tiles_x, tiles_y;
  int begin;
};
struct BatchVecEntry {
  PcgVecs<float> v;
  PcgScalars* sc;
  int n;
  int blocks;
  int begin;
};
// Work-table entry of the batched FP64 residual (element-gather march, 8 warps).
struct BatchResEntry {
  Grid<double> g;
  ResidualArgs a;
  int kchunk;
  int tiles_x, tiles_y;
  int begin;       // first block of the node pass (z-march tiles)
  int qbegin;      // first block of the Gauss-point pass (256 threads each)
  double* el;      // the instance's corner-contribution scratch, 16 doubles per element
};
void launch_batch_pcg_apply(const BatchApplyEntry* tab, int n_inst, int total_blocks, int by, cudaStream_t s);
// Plane-factorized batched PCG apply (8 warps, two rows per thread: tiles of 30 x 14 interior nodes).
void launch_batch_lin_apply(const BatchApplyEntry* tab, int n_inst, int total_blocks, cudaStream_t s);
void launch_batch_residual(const BatchResEntry* tab, int n_inst, int total_blocks, cudaStream_t s);
// Two-pass batched residual: Gauss-point pass over qp_blocks blocks, then the node pass.
void launch_batch_residual_2pass(const BatchResEntry* tab, int n_inst, int qp_blocks, int node_blocks,
                                 cudaStream_t s);
// Per-instance stats slots: mode 0 zeroes the residual slots (stats[0] max |R| as ordered bits,
// stats[1] sum R^2), mode 1 zeroes the trial-step slot stats[8], mode 2 gathers the three into
// out[3i .. 3i+2].
void launch_batch_stats(const BatchResEntry* tab, int n_inst, int mode, double* out, cudaStream_t s);
void launch_batch_pcg_update(const BatchVecEntry* tab, int n_inst, int total_blocks, cudaStream_t s);
void launch_batch_status(const BatchVecEntry* tab, int n_inst, int* status, cudaStream_t s);
}  // namespace qcad
