// Launches of the plane-factorized z-march (linmarch.cuh) for the linear ops:
// Jacobian apply, PCG apply with the fused search-direction update, and the
// Chebyshev preconditioner step, in FP32 and FP64.
#include <cuda_runtime.h>

#include <type_traits>

#include "dfloat.cuh"
#include "linmarch.cuh"
#include "mg.h"
#include "pcg_ops.cuh"

namespace qcad {

// The kernels take more than the default 48 KB of dynamic shared memory; the opt-in is
// set once per kernel and device.
template <class T, int BY, int R, class Op>
static void lin_launch(const Grid<T>& g, const Op& op, int kchunk, cudaStream_t s) {
  using S = LinShape<T, BY, R>;
  static bool attr_set[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 && !attr_set[dev]) {
    // the whole shared-memory carveout: blocks per SM are limited by shared memory otherwise
    if (cudaFuncSetAttribute(lin_march_kernel<T, BY, R, Op>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)S::dyn_bytes) == cudaSuccess &&
        cudaFuncSetAttribute(lin_march_kernel<T, BY, R, Op>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             100) == cudaSuccess)
      attr_set[dev] = true;
  }
  const dim3 grid = lin_grid(g.nxn, g.nyn, g.nzn, BY, R, kchunk);
  note_launch(), lin_march_kernel<T, BY, R, Op><<<grid, dim3(32, BY), S::dyn_bytes, s>>>(g, op, kchunk);
}

// Supported (warps, rows per thread): FP32 4/8/16/32 x 1 and 4/8/16 x 2; FP64 4/8 x 1 and
// 4/8 x 2 (shared memory). Other requests are clamped to the nearest supported shape.
template <class T, class Op>
static void run_lin(const Grid<T>& g, const Op& op, LaunchCfg cfg, cudaStream_t s) {
  const int kc = cfg.kchunk > 0 ? (cfg.kchunk < 128 ? cfg.kchunk : 128) : 16;  // LinShape::ZMAX
  const bool two = cfg.variant == 3;
  if constexpr (std::is_same<T, float>::value) {
    if (two) {
      if (cfg.by == 4) lin_launch<T, 4, 2>(g, op, kc, s);
      else if (cfg.by >= 16) lin_launch<T, 16, 2>(g, op, kc, s);
      else lin_launch<T, 8, 2>(g, op, kc, s);
    } else {
      if (cfg.by == 4) lin_launch<T, 4, 1>(g, op, kc, s);
      else if (cfg.by == 16) lin_launch<T, 16, 1>(g, op, kc, s);
      else if (cfg.by >= 32) lin_launch<T, 32, 1>(g, op, kc, s);
      else lin_launch<T, 8, 1>(g, op, kc, s);
    }
  } else {
    if (two) {
      if (cfg.by == 4) lin_launch<T, 4, 2>(g, op, kc, s);
      else lin_launch<T, 8, 2>(g, op, kc, s);
    } else {
      if (cfg.by == 4) lin_launch<T, 4, 1>(g, op, kc, s);
      else lin_launch<T, 8, 1>(g, op, kc, s);
    }
  }
}

template <class T>
void launch_apply_lin(const Grid<T>& g, const ApplyArgs<T>& args, LaunchCfg cfg, cudaStream_t s) {
  ApplyOp<T> op = {};
  op.a = args;
  run_lin<T>(g, op, cfg, s);
}
template void launch_apply_lin<float>(const Grid<float>&, const ApplyArgs<float>&, LaunchCfg, cudaStream_t);
template void launch_apply_lin<double>(const Grid<double>&, const ApplyArgs<double>&, LaunchCfg, cudaStream_t);

template <class T>
void launch_pcg_apply_lin(const Grid<T>& g, PcgVecs<T> vecs, PcgScalars* sc, LaunchCfg cfg, cudaStream_t s) {
  PcgApplyOp<T> op = {};
  op.v = vecs;
  op.sc = sc;
  run_lin<T>(g, op, cfg, s);
}
template void launch_pcg_apply_lin<float>(const Grid<float>&, PcgVecs<float>, PcgScalars*, LaunchCfg, cudaStream_t);
template void launch_pcg_apply_lin<double>(const Grid<double>&, PcgVecs<double>, PcgScalars*, LaunchCfg,
                                           cudaStream_t);

template <class T>
void launch_cheb_step_lin(const Grid<T>& g, PcgVecs<T> vecs, PcgScalars* sc, int step, int last, LaunchCfg cfg,
                          cudaStream_t s) {
  ChebStepOp<T> op = {};
  op.v = vecs;
  op.sc = sc;
  op.step = step;
  op.last = last;
  run_lin<T>(g, op, cfg, s);
}
template void launch_cheb_step_lin<float>(const Grid<float>&, PcgVecs<float>, PcgScalars*, int, int, LaunchCfg,
                                          cudaStream_t);
template void launch_cheb_step_lin<double>(const Grid<double>&, PcgVecs<double>, PcgScalars*, int, int, LaunchCfg,
                                           cudaStream_t);

// ---------------------------------------------------------------------------
// Multigrid V-cycle on level 0 (the mesh itself): the residual after pre-smoothing,
// w = r - J zp with zp = d[0] = omega D^-1 r, and the post-smoothing step that also closes the
// PCG iteration, z = zq + omega D^-1 (r - J zq) with zq = d[1] = zp + P e (coarse correction),
// accumulating r.z and running the last block's bookkeeping as the Chebyshev step does.
template <class T>
struct MgResid0Op {
  static constexpr int NIN = 1;
  static constexpr bool SEPM = false;
  struct Pre {
    T r;
  };
  PcgVecs<T> v;
  PcgScalars* sc;
  __device__ bool skip() const { return sc->done != 0; }
  __device__ void set_vec(int) {}
  __device__ const T* coeffs() const { return v.c; }
  __device__ const T* lin_src(int) const { return v.d[0]; }
  __device__ T lin_mix(T x0, T) const { return x0; }
  __device__ T lin_in(int n) const { return v.d[0][n]; }
  __device__ Pre lin_pre(int n) const { return Pre{v.r[n]}; }
  __device__ bool lin_dir() const { return true; }
  __device__ void lin_out(int n, const Pre& p, T, T y) { v.w[n] = p.r - y; }
  __device__ void finish() {}
};

template <class T>
struct MgPost0Op {
  static constexpr int NIN = 1;
  static constexpr bool SEPM = false;
  struct Pre {
    T r, dinv;
  };
  PcgVecs<T> v;
  PcgScalars* sc;
  const T* par;
  T om;
  int t, slot;
  T acc;
  __device__ bool skip() const { return sc->done != 0; }
  __device__ void set_vec(int) {
    t = sc->t;
    slot = sc->phase == 0 ? 0 : ((t + 1) & 3);
    om = mg_omega<T>(par, 0);
  }
  __device__ const T* coeffs() const { return v.c; }
  __device__ const T* lin_src(int) const { return v.d[1]; }
  __device__ T lin_mix(T x0, T) const { return x0; }
  __device__ T lin_in(int n) const { return v.d[1][n]; }
  __device__ Pre lin_pre(int n) const { return Pre{v.r[n], v.dinv[n]}; }
  __device__ bool lin_dir() const { return true; }
  __device__ void lin_out(int n, const Pre& p, T zq, T y) {
    const T z = zq + om * p.dinv * (p.r - y);
    v.z[n] = z;
    acc += p.r * z;
  }
  __device__ void finish() {
    double s1[1] = {(double)acc};
    block_sum_atomic<1>(s1, &sc->rz[slot]);
    if (last_block(&sc->counter) && threadIdx.x == 0 && threadIdx.y == 0) pcg_finish(sc, t, 1.0);
  }
};

template <class T>
void launch_mg_resid0(const Grid<T>& g, PcgVecs<T> v, PcgScalars* sc, LaunchCfg cfg, cudaStream_t s) {
  MgResid0Op<T> op = {};
  op.v = v;
  op.sc = sc;
  run_lin<T>(g, op, cfg, s);
}
template void launch_mg_resid0<float>(const Grid<float>&, PcgVecs<float>, PcgScalars*, LaunchCfg, cudaStream_t);
template void launch_mg_resid0<double>(const Grid<double>&, PcgVecs<double>, PcgScalars*, LaunchCfg, cudaStream_t);

template <class T>
void launch_mg_post0(const Grid<T>& g, PcgVecs<T> v, PcgScalars* sc, const T* par, LaunchCfg cfg, cudaStream_t s) {
  MgPost0Op<T> op = {};
  op.v = v;
  op.sc = sc;
  op.par = par;
  run_lin<T>(g, op, cfg, s);
}
template void launch_mg_post0<float>(const Grid<float>&, PcgVecs<float>, PcgScalars*, const float*, LaunchCfg,
                                     cudaStream_t);
template void launch_mg_post0<double>(const Grid<double>&, PcgVecs<double>, PcgScalars*, const double*, LaunchCfg,
                                      cudaStream_t);

// Schrodinger operators for nvec vectors (blockIdx.z runs over (vector, z chunk)): H = kinetic
// stencil (kappa_d = hbar^2/(2 m_d)) plus the V quadrature-point mass term, M = consistent mass,
// both zero on the subdomain boundary (psi = 0 there).
template <class T>
struct HmLinOp {
  static constexpr int NIN = 1;
  static constexpr bool SEPM = true;
  struct Pre {};
  HmArgs<T> a;
  T mscale;
  const T* xv;
  T* hv;
  T* mv;
  __device__ bool skip() const { return false; }
  __device__ void set_vec(int vec) {
    const long long o = (long long)vec * a.ld;
    xv = a.x + o;
    hv = a.hx ? a.hx + o : nullptr;
    mv = a.mx ? a.mx + o : nullptr;
  }
  __device__ const T* coeffs() const { return a.cV; }
  __device__ const T* lin_src(int) const { return xv; }
  __device__ T lin_mix(T x0, T) const { return x0; }
  __device__ T lin_in(int n) const { return xv[n]; }
  __device__ Pre lin_pre(int) const { return Pre{}; }
  __device__ bool lin_dir() const { return true; }
  __device__ T m_scale() const { return mscale; }
  __device__ void lin_out(int, const Pre&, T, T) {}
  __device__ void lin_out2(int n, T yh, T ym) {
    if (hv) hv[n] = yh;
    if (mv) mv[n] = ym;
  }
  __device__ void finish() {}
};

// Double-float coefficients from the FP64 chunks staged in shared memory.
template <>
__device__ __forceinline__ void lin_lds_c8<dfl>(const uint4* p, dfl* c) {
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const double2 a = *reinterpret_cast<const double2*>(p + 32 * h);
    c[2 * h] = dfl_from_bits(a.x);
    c[2 * h + 1] = dfl_from_bits(a.y);
  }
}

// H and M of FP64 vectors in double-float arithmetic: the z-march stages the FP64 inputs and
// coefficients as raw 8-byte values, which are split into double-float pairs where they are read;
// outputs are rounded to FP64.
struct HmDfOp {
  static constexpr int NIN = 1;
  static constexpr bool SEPM = true;
  struct Pre {};
  const double* x;
  double* hx;
  double* mx;
  const double* cV;
  long long ld;
  dfl mscale;
  const double* xv;
  double* hv;
  double* mv;
  __device__ bool skip() const { return false; }
  __device__ void set_vec(int vec) {
    const long long o = (long long)vec * ld;
    xv = x + o;
    hv = hx ? hx + o : nullptr;
    mv = mx ? mx + o : nullptr;
  }
  __device__ const dfl* coeffs() const { return reinterpret_cast<const dfl*>(cV); }
  __device__ const dfl* lin_src(int) const { return reinterpret_cast<const dfl*>(xv); }
  // a staged value holds the bytes of an FP64 input
  __device__ dfl lin_mix(dfl raw, dfl) const {
    return dfl_from_bits(__longlong_as_double((long long)(((unsigned long long)__float_as_uint(raw.l) << 32) |
                                                          __float_as_uint(raw.h))));
  }
  __device__ dfl lin_in(int n) const { return dfl_from_bits(xv[n]); }
  __device__ Pre lin_pre(int) const { return Pre{}; }
  __device__ bool lin_dir() const { return true; }
  __device__ dfl m_scale() const { return mscale; }
  __device__ void lin_out(int, const Pre&, dfl, dfl) {}
  __device__ void lin_out2(int n, dfl yh, dfl ym) {
    if (hv) hv[n] = dfl_to_double(yh);
    if (mv) mv[n] = dfl_to_double(ym);
  }
  __device__ void finish() {}
};

template <class T, int BY, int R, class Op>
static void lin_launch_vec(const Grid<T>& g, const Op& op, int kchunk, int nvec, cudaStream_t s) {
  using S = LinShape<T, BY, R>;
  static bool attr_set[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 && !attr_set[dev]) {
    if (cudaFuncSetAttribute(lin_march_kernel<T, BY, R, Op>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)S::dyn_bytes) == cudaSuccess &&
        cudaFuncSetAttribute(lin_march_kernel<T, BY, R, Op>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             100) == cudaSuccess)
      attr_set[dev] = true;
  }
  const dim3 grid = lin_grid(g.nxn, g.nyn, g.nzn, BY, R, kchunk, nvec);
  note_launch(), lin_march_kernel<T, BY, R, Op><<<grid, dim3(32, BY), S::dyn_bytes, s>>>(g, op, kchunk);
}

template <class T>
void launch_hm_apply_lin(const Grid<T>& g, const HmArgs<T>& args, LaunchCfg cfg, cudaStream_t s) {
  HmLinOp<T> op = {};
  op.a = args;
  op.mscale = (T)args.mscale;
  const int kc = cfg.kchunk > 0 ? (cfg.kchunk < 128 ? cfg.kchunk : 128) : 16;
  if (cfg.variant == 3)
    lin_launch_vec<T, 8, 2>(g, op, kc, args.nvec, s);
  else
    lin_launch_vec<T, 8, 1>(g, op, kc, args.nvec, s);
}
template void launch_hm_apply_lin<float>(const Grid<float>&, const HmArgs<float>&, LaunchCfg, cudaStream_t);
template void launch_hm_apply_lin<double>(const Grid<double>&, const HmArgs<double>&, LaunchCfg, cudaStream_t);

// One step of the eigensolver's Chebyshev-Jacobi block preconditioner fused into the H apply of its
// direction block: with h = (H D_in)_n at every node (Dirichlet rows: h = D_in = 0 there),
//   W <- W - h,  D_out <- c1 D_in + c2 D^-1 W,  Z <- Z + D_out
// (the recurrence of cheb_block_step_kernel). D is double-buffered: other tiles still read D_in.
struct ChebHmOp {
  static constexpr int NIN = 1;
  static constexpr bool SEPM = false;
  struct Pre {
    float w, z;
  };
  ChebHmArgs a;
  const float *din, *dinv;
  float *dout, *w, *z;
  __device__ bool skip() const { return false; }
  __device__ void set_vec(int vec) {
    const long long o = (long long)vec * a.ld;
    din = a.din + o;
    dout = a.dout + o;
    w = a.w + o;
    z = a.z + o;
    dinv = a.dinv;
  }
  __device__ const float* coeffs() const { return a.cV; }
  __device__ const float* lin_src(int) const { return din; }
  __device__ float lin_mix(float x0, float) const { return x0; }
  __device__ float lin_in(int n) const { return din[n]; }
  __device__ Pre lin_pre(int n) const { return Pre{w[n], z[n]}; }
  __device__ bool lin_dir() const { return true; }
  __device__ float m_scale() const { return 0.0f; }
  __device__ void lin_out(int n, const Pre& pre, float vin, float h) {
    const float wn = pre.w - h;
    const float d = a.c1 * vin + a.c2 * dinv[n] * wn;
    w[n] = wn;
    dout[n] = d;
    z[n] = pre.z + d;
  }
  __device__ void lin_out2(int, float, float) {}
  __device__ void finish() {}
};

void launch_cheb_hm_step(const Grid<float>& g, const ChebHmArgs& args, cudaStream_t s) {
  ChebHmOp op = {};
  op.a = args;
  lin_launch_vec<float, 8, 2>(g, op, 16, args.nvec, s);
}

void launch_hm_apply_df(const Grid<dfl>& g, const HmArgs<double>& args, cudaStream_t s) {
  HmDfOp op = {};
  op.x = args.x;
  op.hx = args.hx;
  op.mx = args.mx;
  op.cV = args.cV;
  op.ld = args.ld;
  op.mscale = dfl(args.mscale);
  lin_launch_vec<dfl, 8, 2>(g, op, 16, args.nvec, s);
}

// Batched PCG apply: a work table maps each block to (instance, tile) of instances of different
// sizes; plane-factorized march with 8 warps and two rows per thread.
__device__ __forceinline__ int lin_batch_find(const BatchApplyEntry* tab, int n, int b) {
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

__global__ void __launch_bounds__(256, (lin_min_blocks<float, 8, 2>()))
    batch_lin_apply_kernel(const BatchApplyEntry* tab, int n_inst) {
  extern __shared__ __align__(16) unsigned char lin_dyn[];
  const int b = blockIdx.x;
  const BatchApplyEntry& e = tab[lin_batch_find(tab, n_inst, b)];
  const int local = b - e.begin;
  const int bx = local % e.tiles_x;
  const int by = (local / e.tiles_x) % e.tiles_y;
  const int bz = local / (e.tiles_x * e.tiles_y);
  PcgApplyOp<float> op = {};
  op.v = e.v;
  op.sc = e.sc;
  lin_body<float, 8, 2, PcgApplyOp<float>>(e.g, op, e.kchunk, bx, by, bz, lin_dyn);
}

void launch_batch_lin_apply(const BatchApplyEntry* tab, int n_inst, int total_blocks, cudaStream_t s) {
  using S = LinShape<float, 8, 2>;
  static bool attr_set[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 && !attr_set[dev]) {
    if (cudaFuncSetAttribute(batch_lin_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)S::dyn_bytes) == cudaSuccess &&
        cudaFuncSetAttribute(batch_lin_apply_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100) ==
            cudaSuccess)
      attr_set[dev] = true;
  }
  note_launch(), batch_lin_apply_kernel<<<total_blocks, dim3(32, 8), S::dyn_bytes, s>>>(tab, n_inst);
}

// Resident blocks per SM of the plane-factorized apply (0 if the query fails).
template <class T, int BY, int R>
static int lin_occupancy() {
  using S = LinShape<T, BY, R>;
  int n = 0;
  cudaFuncSetAttribute(lin_march_kernel<T, BY, R, ApplyOp<T>>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)S::dyn_bytes);
  cudaFuncSetAttribute(lin_march_kernel<T, BY, R, ApplyOp<T>>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, lin_march_kernel<T, BY, R, ApplyOp<T>>, 32 * BY,
                                                    S::dyn_bytes) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

int lin_blocks_per_sm(int precision, int by, int rows) {
  if (precision == 1) {
    if (rows == 2) return by == 4 ? lin_occupancy<float, 4, 2>() : by >= 16 ? lin_occupancy<float, 16, 2>()
                                                                             : lin_occupancy<float, 8, 2>();
    return by == 4 ? lin_occupancy<float, 4, 1>() : by == 16 ? lin_occupancy<float, 16, 1>()
                                                  : by >= 32 ? lin_occupancy<float, 32, 1>()
                                                             : lin_occupancy<float, 8, 1>();
  }
  if (rows == 2) return by == 4 ? lin_occupancy<double, 4, 2>() : lin_occupancy<double, 8, 2>();
  return by == 4 ? lin_occupancy<double, 4, 1>() : lin_occupancy<double, 8, 1>();
}

}  // namespace qcad
