// Linear operator ops of the z-marching skeletons (Jacobian apply, PCG apply
// with the fused search-direction update, Chebyshev step) and the device-side
// PCG bookkeeping they share. Included by the kernel translation units.
#pragma once

#include "qcad_host.h"
#include "qcad_internal.cuh"

namespace qcad {

template <class T>
__device__ __forceinline__ int elem_index(const Grid<T>& g, int i, int j, int k) {
  return i + g.nx * (j + g.ny * k);
}

template <class T>
__device__ __forceinline__ C8<T> load_coeffs(const T* c, int e) {
  C8<T> r;
  load_c8<T>(c, e, r.c);
  return r;
}

// ---------------------------------------------------------------------------
// y = J v: separable stiffness stencil plus the element quadrature-point mass
// term with stored coefficients c; identity on Dirichlet rows unless raw.
// The optional v.y partial sums run in the storage precision per thread and
// in FP64 across threads.
template <class T>
struct ApplyOp {
  static constexpr int NF = 1;
  static constexpr bool STIFF = true;
  using ED = C8<T>;
  ApplyArgs<T> a;
  T acc;
  __device__ bool skip() const { return false; }
  __device__ void set_vec(int) {}
  __device__ T load(const Grid<T>&, int n, bool in, int, int, int) const { return in ? a.v[n] : T(0); }
  __device__ ED edata(const Grid<T>& g, int i, int j, int k) const { return load_coeffs<T>(a.c, elem_index(g, i, j, k)); }
  __device__ const T* coeffs() const { return a.c; }
  // plane-factorized kernels: unpredicated input (n always in range), Dirichlet override
  // flag (the kernel substitutes the input on Dirichlet rows) and the store
  struct Pre {};
  static constexpr int NIN = 1;
  static constexpr bool SEPM = false;  // no separable-mass second output
  __device__ const T* lin_src(int) const { return a.v; }
  __device__ T lin_mix(T x0, T) const { return x0; }
  __device__ T lin_in(int n) const { return a.v[n]; }
  __device__ Pre lin_pre(int) const { return Pre{}; }
  __device__ bool lin_dir() const { return !a.raw; }
  __device__ void lin_out(int n, const Pre&, T vin, T y) {
    a.y[n] = y;
    acc += vin * y;
  }
  __device__ void elem(const Grid<T>&, int, int, int, const T* v, const ED& ed, T (*out)[8], bool) const {
    qp_mass<T>(v, ed.c, out[0]);
  }
  __device__ void node(const Grid<T>& g, int n, int i, int j, int k, T vin, T stiff, const T* mass) {
    T y = stiff + mass[0];
    if (!a.raw && grid_is_dir(g, i, j, k)) y = vin;
    a.y[n] = y;
    acc += vin * y;
  }
  __device__ void finish() {
    if (a.dot) {
      double s[1] = {(double)acc};
      block_sum_atomic<1>(s, a.dot);
    }
  }
};

// ---------------------------------------------------------------------------
// Preconditioned CG with device-resident scalars.
//
// Iteration t: apply kernel forms p_t = z_t + beta_t p_{t-1} while loading
// (beta_t = rz_t / rz_{t-1}), writes p_t and Ap_t and accumulates p.Ap into
// pAp[t%4]; update kernel forms alpha_t = rz_t / pAp_t, updates x, r, the
// Jacobi-preconditioned z = D^-1 r, accumulates r.z and r.r into slot
// (t+1)%4, and its last block advances t, tests convergence and clears the
// slots the next iteration accumulates into.
template <class T>
struct PcgApplyOp {
  static constexpr int NF = 1;
  static constexpr bool STIFF = true;
  using ED = C8<T>;
  PcgVecs<T> v;
  PcgScalars* sc;
  int t;
  T beta;
  T acc;
  __device__ bool skip() const { return sc->done != 0; }
  const T* pprev;  // p_{t-1} (in p[(t+1)&1]); p_t goes to p[t&1], so halo reads never see new values
  T* pcur;
  const T* pin_src;
  __device__ void set_vec(int) {
    t = sc->t;
    beta = t > 0 ? (T)(sc->rz[t & 3] / sc->rz[(t - 1) & 3]) : T(0);
    // selected, not indexed: a runtime index into v.p would put the op in local memory
    pprev = (t & 1) ? v.p[0] : v.p[1];
    pcur = (t & 1) ? v.p[1] : v.p[0];
    pin_src = t > 0 ? pprev : v.z;  // at t = 0 beta = 0 and p_{-1} is never read
  }
  struct Pre {};
  static constexpr int NIN = 2;
  static constexpr bool SEPM = false;
  __device__ const T* lin_src(int q) const { return q == 0 ? v.z : pin_src; }
  __device__ T lin_mix(T z, T p) const { return z + beta * p; }
  __device__ T lin_in(int n) const { return v.z[n] + beta * pin_src[n]; }
  __device__ Pre lin_pre(int) const { return Pre{}; }
  __device__ bool lin_dir() const { return true; }
  __device__ void lin_out(int n, const Pre&, T pin, T y) {
    pcur[n] = pin;
    v.Ap[n] = y;
    acc += pin * y;
  }
  __device__ T load(const Grid<T>&, int n, bool in, int, int, int) const {
    if (!in) return T(0);
    return t > 0 ? v.z[n] + beta * pprev[n] : v.z[n];
  }
  __device__ ED edata(const Grid<T>& g, int i, int j, int k) const { return load_coeffs<T>(v.c, elem_index(g, i, j, k)); }
  __device__ const T* coeffs() const { return v.c; }
  __device__ void elem(const Grid<T>&, int, int, int, const T* x, const ED& ed, T (*out)[8], bool) const {
    qp_mass<T>(x, ed.c, out[0]);
  }
  __device__ void node(const Grid<T>& g, int n, int i, int j, int k, T pin, T stiff, const T* mass) {
    T y = stiff + mass[0];
    if (grid_is_dir(g, i, j, k)) y = pin;
    pcur[n] = pin;
    v.Ap[n] = y;
    acc += pin * y;
  }
  __device__ void finish() {
    double s[1] = {(double)acc};
    block_sum_atomic<1>(s, &sc->pAp[t & 3]);
  }
};

// Last block of a grid: returns true in exactly one block after all blocks' prior writes are visible.
__device__ __forceinline__ bool last_block_of(unsigned int* counter, unsigned int total) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) am_last = atomicAdd(counter, 1u) == total - 1;
  __syncthreads();
  return am_last;
}
__device__ __forceinline__ bool last_block(unsigned int* counter) {
  return last_block_of(counter, gridDim.x * gridDim.y * gridDim.z);
}

__device__ __forceinline__ double ld_volatile(const double* p) { return *(volatile const double*)p; }

// Last block's bookkeeping after r.z is complete. Phase 1 (after iteration t): advance t,
// clear the slots the next iteration accumulates into, test convergence. Phase 0 (after
// the initial residual of a Chebyshev-preconditioned solve): record ||r0||^2, start at t = 0.
__device__ __forceinline__ void pcg_finish(PcgScalars* sc, int t, double alpha_d) {
  if (sc->phase == 0) {
    const double rr0 = ld_volatile(&sc->rr[0]);
    const double rz0 = ld_volatile(&sc->rz[0]);
    sc->rr0 = rr0;
    sc->t = 0;
    sc->iters = 0;
    sc->phase = 1;
    sc->pAp[0] = 0.0;
    sc->rz[1] = 0.0;
    sc->rr[1] = 0.0;
    if (!(rr0 == rr0) || !(rz0 == rz0) || rr0 > 1e300 || rz0 < 0.0) {
      sc->nonfinite = 1;
      sc->done = 1;
    } else if (rr0 == 0.0) {
      sc->done = 1;
    }
    sc->counter = 0;
    return;
  }
  const double rr_new = ld_volatile(&sc->rr[(t + 1) & 3]);
  const double rz_new = ld_volatile(&sc->rz[(t + 1) & 3]);
  const int tn = t + 1;
  sc->t = tn;
  sc->pAp[tn & 3] = 0.0;
  sc->rz[(tn + 1) & 3] = 0.0;
  sc->rr[(tn + 1) & 3] = 0.0;
  const bool bad = !(alpha_d == alpha_d) || !(rr_new == rr_new) || !(rz_new == rz_new) || fabs(alpha_d) > 1e300 ||
                   alpha_d <= 0.0 || rz_new < 0.0;
  if (bad) {
    sc->nonfinite = 1;
    sc->done = 1;
    sc->iters = tn;
  } else if (rr_new <= sc->tol2 * sc->rr0 || tn >= sc->maxit) {
    sc->done = 1;
    sc->iters = tn;
  }
  sc->counter = 0;
}

template <class T>
struct ChebStepOp {
  static constexpr int NF = 1;
  static constexpr bool STIFF = true;
  using ED = C8<T>;
  PcgVecs<T> v;
  PcgScalars* sc;
  int step, last;
  int t, slot;
  const T* dprev;  // d_{step-1} and d_step (ping-pong by step parity)
  T* dcur;
  T c1, c2;
  T acc;
  __device__ bool skip() const { return sc->done != 0; }
  __device__ void set_vec(int) {
    t = sc->t;
    slot = sc->phase == 0 ? 0 : ((t + 1) & 3);
    const double sigma = sc->theta / sc->delta;
    double rho_prev = 1.0 / sigma, rho = rho_prev;
    for (int q = 1; q <= step; ++q) {
      rho_prev = rho;
      rho = 1.0 / (2.0 * sigma - rho_prev);
    }
    c1 = (T)(rho * rho_prev);
    c2 = (T)(2.0 * rho / sc->delta);
    dprev = (step & 1) ? v.d[0] : v.d[1];
    dcur = (step & 1) ? v.d[1] : v.d[0];
  }
  // the node data of the epilogue, loaded at the start of the plane (latency off the critical path)
  struct Pre {
    T w, dinv, z, r;
  };
  static constexpr int NIN = 1;
  static constexpr bool SEPM = false;  // no separable-mass second output
  __device__ const T* lin_src(int) const { return dprev; }
  __device__ T lin_mix(T x0, T) const { return x0; }
  __device__ T lin_in(int n) const { return dprev[n]; }
  __device__ Pre lin_pre(int n) const {
    Pre p;
    p.w = v.w[n];
    p.dinv = v.dinv[n];
    p.z = v.z[n];
    p.r = last ? v.r[n] : T(0);
    return p;
  }
  __device__ bool lin_dir() const { return true; }
  __device__ void lin_out(int n, const Pre& p, T dold, T y) {
    const T wn = p.w - y;
    const T dn = c1 * dold + c2 * p.dinv * wn;
    const T zn = p.z + dn;
    v.w[n] = wn;
    v.z[n] = zn;
    dcur[n] = dn;
    if (last) acc += p.r * zn;
  }
  __device__ T load(const Grid<T>&, int n, bool in, int, int, int) const { return in ? dprev[n] : T(0); }
  __device__ ED edata(const Grid<T>& g, int i, int j, int k) const { return load_coeffs<T>(v.c, elem_index(g, i, j, k)); }
  __device__ const T* coeffs() const { return v.c; }
  __device__ void elem(const Grid<T>&, int, int, int, const T* x, const ED& ed, T (*out)[8], bool) const {
    qp_mass<T>(x, ed.c, out[0]);
  }
  __device__ void node(const Grid<T>& g, int n, int i, int j, int k, T dold, T stiff, const T* mass) {
    T y = stiff + mass[0];
    if (grid_is_dir(g, i, j, k)) y = dold;
    const T wn = v.w[n] - y;
    const T dn = c1 * dold + c2 * v.dinv[n] * wn;
    const T zn = v.z[n] + dn;
    v.w[n] = wn;
    v.z[n] = zn;
    dcur[n] = dn;
    if (last) acc += v.r[n] * zn;
  }
  __device__ void finish() {
    if (!last) return;
    double s1[1] = {(double)acc};
    block_sum_atomic<1>(s1, &sc->rz[slot]);
    if (last_block(&sc->counter) && threadIdx.x == 0 && threadIdx.y == 0) pcg_finish(sc, t, 1.0);
  }
};

}  // namespace qcad
