// Poisson kernels: FP64 nonlinear residual with fused Jacobian linearization,
// matrix-free Jacobian apply (FP32 / FP64), fused preconditioned-CG kernels
// and the Newton update. Sec. II.A (Eqs. Poisson, PoissonWeakForm,
// MBstatistics, FDstatistics, FDIntApprox, FinalIonization).
#include <cuda_runtime.h>

#include <type_traits>

#include "march2.cuh"
#include "pcg_ops.cuh"
#include "physics.cuh"
#include "qcad_host.h"
#include "qcad_internal.cuh"

namespace qcad {


// Diagonal of the assembled stiffness from the 1D operator rows.
template <class T>
__device__ __forceinline__ T stiff_diag(const Grid<T>& g, int i, int j, int k) {
  const T mxc = g.mx[3 * i + 1], kxc = g.kx[3 * i + 1];
  const T myc = g.my[3 * j + 1], kyc = g.ky[3 * j + 1];
  return kxc * myc * g.mzx[3 * k + 1] + mxc * kyc * g.mzy[3 * k + 1] + mxc * myc * g.kzz[3 * k + 1];
}

__device__ __forceinline__ int dot_of_element(const ResidualArgs& a, int i, int j, int k) {
  const double xc = 0.5 * (a.xn[i] + a.xn[i + 1]);
  const double yc = 0.5 * (a.yn[j] + a.yn[j + 1]);
  const double zc = 0.5 * (a.zn[k] + a.zn[k + 1]);
  for (int d = 0; d < a.dots.n; ++d) {
    const double* B = a.dots.b[d];
    if (xc >= B[0] && xc <= B[1] && yc >= B[2] && yc <= B[3] && zc >= B[4] && zc <= B[5]) return d;
  }
  return -1;
}


// ---------------------------------------------------------------------------
// Residual R(phi), Jacobian quadrature coefficients c_q = -(q/eps0) w|J| rho'(phi_q),
// the Jacobian diagonal, norms of R and dot electron counts in one z-march (FP64).
struct ResidualOp {
  static constexpr int NF = 2;
  static constexpr bool STIFF = true;
  using ED = double;  // fixed charge of the element
  ResidualArgs a;
  double acc_dot0, acc_dot1;  // the first two dots in registers; further dots add atomically
  double acc_r2;
  double acc_rmax;
  __device__ bool skip() const { return false; }
  __device__ void set_vec(int) {}
  __device__ double load(const Grid<double>&, int n, bool in, int, int, int) const { return in ? a.phi[n] : 0.0; }
  __device__ double edata(const Grid<double>& g, int i, int j, int k) const {
    return a.theta ? a.theta[elem_index(g, i, j, k)] : 0.0;
  }
  __device__ void elem(const Grid<double>& g, int i, int j, int k, const double* v, double th, double (*out)[8],
                       bool own) {
    const double wdet = g.hx[i] * g.hy[j] * g.hz[k] * 0.125;
    const int e = elem_index(g, i, j, k);
    double f[8], c[8];
    if (a.layer_semi[k] && !a.linear) {
      double pq[8];
      tp_apply(v, pq, GaussConst<double>::a(), GaussConst<double>::b());
      double nsum = 0.0;
      // the residual's below-resolution cutoffs, except in the dots when their counts are formed
      const int d = a.counts != nullptr ? dot_of_element(a, i, j, k) : -1;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const Charge ch = d < 0 ? charge_resid(a.P, pq[q]) : charge_at(a.P, pq[q]);
        f[q] = -a.P.qe * wdet * (ch.rho + th);
        c[q] = -a.P.qe * wdet * ch.drho;
        nsum += ch.n;
      }
      if (a.counts != nullptr && own) {  // each element counted once
        if (d == 0)
          acc_dot0 += wdet * nsum;
        else if (d == 1)
          acc_dot1 += wdet * nsum;
        else if (d > 1)
          atomicAdd(a.counts + d, wdet * nsum);
      }
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        f[q] = -a.P.qe * wdet * th;
        c[q] = 0.0;
      }
    }
    tp_apply(f, out[0], GaussConst<double>::a(), GaussConst<double>::b());
    const double a2 = GaussConst<double>::a() * GaussConst<double>::a();
    const double b2 = GaussConst<double>::b() * GaussConst<double>::b();
    tp_apply(c, out[1], a2, b2);
    if (a.c64) {
      double2* p = reinterpret_cast<double2*>(a.c64 + 8 * (size_t)e);
#pragma unroll
      for (int s = 0; s < 4; ++s) p[s] = make_double2(c[2 * s], c[2 * s + 1]);
    }
    if (a.c32) {
      float4* p = reinterpret_cast<float4*>(a.c32 + 8 * (size_t)e);
      p[0] = make_float4((float)c[0], (float)c[1], (float)c[2], (float)c[3]);
      p[1] = make_float4((float)c[4], (float)c[5], (float)c[6], (float)c[7]);
    }
  }
  __device__ void node(const Grid<double>& g, int n, int i, int j, int k, double, double stiff, const double* mass) {
    double R = stiff + mass[0];
    double dg = stiff_diag(g, i, j, k) + mass[1];
    if (grid_is_dir(g, i, j, k)) {
      R = 0.0;
      dg = 1.0;
    }
    a.R[n] = R;
    if (a.diag) a.diag[n] = dg;
    if (a.dinv64) a.dinv64[n] = 1.0 / dg;
    if (a.dinv32) a.dinv32[n] = (float)(1.0 / dg);
    if (a.b64) a.b64[n] = -R;
    if (a.b32) a.b32[n] = (float)(-R);
    acc_r2 += R * R;
    acc_rmax = fmax(acc_rmax, fabs(R));
  }
  __device__ void finish() {
    if (a.stats) {
      double s[1] = {acc_r2};
      block_sum_atomic<1>(s, a.stats + 1);
      block_max_atomic(acc_rmax, a.stats);
    }
    if (a.counts) {
      double s[2] = {acc_dot0, acc_dot1};
      block_sum_atomic<2>(s, a.counts);
    }
  }
};


template <class T, class Op>
static void run_march(const Grid<T>& g, const Op& op, LaunchCfg cfg, cudaStream_t s, int nvec = 1) {
  switch (cfg.by) {
    case 4: {
      dim3 grid = march_grid(g.nxn, g.nyn, g.nzn, 4, cfg.kchunk, nvec);
      note_launch(), march_kernel<T, 4, Op><<<grid, dim3(QCAD_BX, 4), 0, s>>>(g, op, cfg.kchunk);
      break;
    }
    case 16: {
      dim3 grid = march_grid(g.nxn, g.nyn, g.nzn, 16, cfg.kchunk, nvec);
      note_launch(), march_kernel<T, 16, Op><<<grid, dim3(QCAD_BX, 16), 0, s>>>(g, op, cfg.kchunk);
      break;
    }
    case 32: {
      dim3 grid = march_grid(g.nxn, g.nyn, g.nzn, 32, cfg.kchunk, nvec);
      note_launch(), march_kernel<T, 32, Op><<<grid, dim3(QCAD_BX, 32), 0, s>>>(g, op, cfg.kchunk);
      break;
    }
    default: {
      dim3 grid = march_grid(g.nxn, g.nyn, g.nzn, 8, cfg.kchunk, nvec);
      note_launch(), march_kernel<T, 8, Op><<<grid, dim3(QCAD_BX, 8), 0, s>>>(g, op, cfg.kchunk);
      break;
    }
  }
}

// The skeleton with the charged gates' face term (alpha: [nx*ny] face coefficients, Robin
// condition of Sec. II.A.4); 8 or 16 warps per block.
template <class T, class Op>
static void run_march_face(const Grid<T>& g, const Op& op, LaunchCfg cfg, cudaStream_t s, const T* alpha,
                           int nvec = 1) {
  if (cfg.by == 16 || cfg.by == 32) {
    dim3 grid = march_grid(g.nxn, g.nyn, g.nzn, 16, cfg.kchunk, nvec);
    note_launch(), march_face_kernel<T, 16, Op><<<grid, dim3(QCAD_BX, 16), 0, s>>>(g, op, cfg.kchunk, alpha);
  } else {
    dim3 grid = march_grid(g.nxn, g.nyn, g.nzn, 8, cfg.kchunk, nvec);
    note_launch(), march_face_kernel<T, 8, Op><<<grid, dim3(QCAD_BX, 8), 0, s>>>(g, op, cfg.kchunk, alpha);
  }
}

// FP32 pair-kernel launchers (two nodes per thread, packed f32x2), defined below.
void launch_apply_pair(const Grid<float>& g, const ApplyArgs<float>& a, LaunchCfg cfg, cudaStream_t s);
void launch_pcg_apply_pair(const Grid<float>& g, PcgVecs<float> v, PcgScalars* sc, LaunchCfg cfg, cudaStream_t s);
void launch_cheb_step_pair(const Grid<float>& g, PcgVecs<float> v, PcgScalars* sc, int step, int last,
                           LaunchCfg cfg, cudaStream_t s);

void launch_residual(const Grid<double>& g, const ResidualArgs& args, LaunchCfg cfg, cudaStream_t s) {
  ResidualOp op = {};
  op.a = args;
  LaunchCfg c = cfg;
  if (c.by == 32) c.by = 16;  // FP64 residual: 1024-thread tiles exceed its register budget
  run_march<double>(g, op, c, s);
}

// ---------------------------------------------------------------------------
// Two-pass residual: the same R, c, diagonal, norms and counts as ResidualOp, with the carrier
// density (the FP64 transcendental part) evaluated exactly once per quadrature point.
//
// Pass 1: one thread per (element, quadrature point); the 8 lanes of an element hold its
// corners and quadrature points under the same index (ix + 2 iy + 4 iz), so the Gauss
// interpolation B (x) B (x) B and its transpose are three butterfly stages over lane bits 0, 1, 2
// (B = [[a, b], [b, a]] along each axis). Writes c_q, the element's corner contributions to the
// load -(q/eps0) int (rho + theta) N_i (elR) and to the mass diagonal sum_q c_q N_i(q)^2 (elD),
// [8 e + corner] each, and the dot electron counts.
// Body of pass 1 for thread t of a mesh (the batched form calls it with its own block numbering;
// t & 7 == threadIdx.x & 7 there too).
__device__ __forceinline__ void residual_qp_body(const Grid<double>& g, const ResidualArgs& a, double* elR,
                                                 double* elD, long long t) {
  const long long ne = (long long)g.nx * g.ny * g.nz;
  const bool valid = t < 8 * ne;  // an element's 8 lanes share one warp and one validity
  const int e = valid ? (int)(t >> 3) : 0;
  const int l = threadIdx.x & 7;
  const int i = e % g.nx, r = e / g.nx;
  const int j = r % g.ny, k = r / g.ny;
  const bool semi = valid && a.layer_semi[k] && !a.linear;
  const double A = GaussConst<double>::a(), B = GaussConst<double>::b();
  double v = 0.0;
  if (semi)
    v = __ldg(a.phi + (i + (l & 1)) + (long long)g.nxn * ((j + ((l >> 1) & 1)) + (long long)g.nyn * (k + (l >> 2))));
  // Flat elements: the Gauss-point potentials are convex combinations of the corner values, so
  // when all eight corners lie in one of charge_resid's constant-charge zones, every Gauss point
  // does, rho is that zone's constant and rho' = 0. The element's load is then
  // -(q/eps0) w|J| (rho + theta) at each corner (the Gauss weights of each corner's shape function
  // sum to 1) and its Jacobian coefficients vanish. A warp whose elements are all flat (or not
  // semiconductor) skips the interpolation and the transposed interpolation.
  if (a.counts == nullptr && a.qd.w == nullptr) {
    // -2: no charge term at all (oxide, padding)
    const int zone = semi ? charge_zone_key(a.P, double_key((unsigned long long)__double_as_longlong(v))) : -2;
    int zmin = zone, zmax = zone;
#pragma unroll
    for (int sft = 1; sft < 8; sft <<= 1) {
      zmin = min(zmin, __shfl_xor_sync(FULL_MASK, zmin, sft));
      zmax = max(zmax, __shfl_xor_sync(FULL_MASK, zmax, sft));
    }
    const bool eflat = zmin == zmax && zmin != -1;
    if (__all_sync(FULL_MASK, eflat)) {
      if (valid) {
        if (a.wq != nullptr && a.theta == nullptr) {
          const int slot = zone >= 0 ? (a.P.incomplete ? zone : WQ_ZONE_COMPLETE) : WQ_ZERO;
          if (a.ecode != nullptr) {
            // the element's corner loads are one table entry and its diagonal contributions zero:
            // pass 2 reads the code (1 + the slot) instead of 128 bytes of corner values
            if (l == 0) a.ecode[e] = (unsigned char)(1 + slot);
          } else {
            elR[t] = a.wq[8 * k + slot];
            elD[t] = 0.0;
          }
        } else {
          const double th = a.theta ? a.theta[e] : 0.0;
          const double rho = zone >= 0 ? zone_charge(a.P, zone) : 0.0;
          const double w = a.wq != nullptr ? a.wq[8 * k + WQ_WEIGHT] : -a.P.qe * (g.hx[i] * g.hy[j] * g.hz[k] * 0.125);
          elR[t] = w * (rho + th);
          elD[t] = 0.0;
          if (a.ecode != nullptr && l == 0) a.ecode[e] = 0;
        }
        if (a.c64) a.c64[t] = 0.0;
        if (a.c32) a.c32[t] = 0.0f;
      }
      return;
    }
  }
  v = A * v + B * __shfl_xor_sync(FULL_MASK, v, 1);
  v = A * v + B * __shfl_xor_sync(FULL_MASK, v, 2);
  v = A * v + B * __shfl_xor_sync(FULL_MASK, v, 4);
  double f = 0.0, c = 0.0, nq = 0.0;
  // the residual's below-resolution cutoffs, except in the dots when their counts are formed
  const int dot = (semi && a.counts != nullptr) ? dot_of_element(a, i, j, k) : -1;
  if (valid) {
    const double wdet = g.hx[i] * g.hy[j] * g.hz[k] * 0.125;
    const double th = a.theta ? a.theta[e] : 0.0;
    if (semi) {
      Charge ch = dot < 0 ? charge_resid(a.P, v) : charge_at(a.P, v);
      if (a.qd.w != nullptr) {
        // in the quantum region the predictor density n~ replaces the semiclassical n (Sec. II.C)
        const int iq = i - a.qd.i0, jq = j - a.qd.j0, kq = k - a.qd.k0;
        if (iq >= 0 && jq >= 0 && kq >= 0 && iq < a.qd.nx && jq < a.qd.ny && kq < a.qd.nz) {
          double nt, dnt;
          qd_density(a.qd, iq + (long long)a.qd.nx * (jq + (long long)a.qd.ny * kq), l, v, a.P.EF, a.P.inv_kT, nt,
                     dnt);
          ch.rho += ch.n - nt;
          ch.drho += ch.dn - dnt;
          ch.n = nt;
          ch.dn = dnt;
        }
      }
      f = -a.P.qe * wdet * (ch.rho + th);
      c = -a.P.qe * wdet * ch.drho;
      nq = wdet * ch.n;
    } else {
      f = -a.P.qe * wdet * th;
    }
    if (a.c64) a.c64[t] = c;
    if (a.c32) a.c32[t] = (float)c;
  }
  const double A2 = A * A, B2 = B * B;
  // the transposed interpolation of each field, skipped where the whole warp holds zeros (the
  // neutral bulk, where every density is below resolution, and the fully ionized depletion
  // region, where the Jacobian coefficients vanish): the warp-uniform branch keeps the shuffles
  // converged
  if (__any_sync(FULL_MASK, f != 0.0)) {
    f = A * f + B * __shfl_xor_sync(FULL_MASK, f, 1);
    f = A * f + B * __shfl_xor_sync(FULL_MASK, f, 2);
    f = A * f + B * __shfl_xor_sync(FULL_MASK, f, 4);
  }
  if (__any_sync(FULL_MASK, c != 0.0)) {
    c = A2 * c + B2 * __shfl_xor_sync(FULL_MASK, c, 1);
    c = A2 * c + B2 * __shfl_xor_sync(FULL_MASK, c, 2);
    c = A2 * c + B2 * __shfl_xor_sync(FULL_MASK, c, 4);
  }
  if (valid) {
    elR[t] = f;
    elD[t] = c;
    if (a.ecode != nullptr && l == 0) a.ecode[e] = 0;
  }
  if (a.counts != nullptr) {
    double s[2] = {0.0, 0.0};
    if (semi) {
      const int d = dot;
      if (d == 0)
        s[0] = nq;
      else if (d == 1)
        s[1] = nq;
      else if (d > 1)
        atomicAdd(a.counts + d, nq);
    }
    block_sum_atomic<2>(s, a.counts);
  }
}

__global__ void __launch_bounds__(256) residual_qp_kernel(const __grid_constant__ Grid<double> g,
                                                          const __grid_constant__ ResidualArgs a, double* elR,
                                                          double* elD) {
  residual_qp_body(g, a, elR, elD, blockIdx.x * 256LL + threadIdx.x);
}

// Pass 2: the z-march node pass. Each node gathers the corner contributions of its elements
// and adds the stiffness K phi (separable 27-point stencil); Dirichlet rows as in ResidualOp.
struct ResidualGatherOp {
  static constexpr int NF = 2;
  static constexpr bool STIFF = true;
  using ED = unsigned char;  // the element's load code from pass 1 (0: corner values in elR, elD)
  const double* phi;
  const double* elR;
  const double* elD;
  const unsigned char* ecode;
  const double* wq;
  double *R, *diag, *dinv64, *b64, *stats;
  float *dinv32, *b32;
  double acc_r2, acc_rmax;
  __device__ bool skip() const { return false; }
  __device__ void set_vec(int) {}
  __device__ double load(const Grid<double>&, int n, bool in, int, int, int) const { return in ? phi[n] : 0.0; }
  __device__ unsigned char edata(const Grid<double>& g, int i, int j, int k) const {
    return ecode != nullptr ? ecode[elem_index(g, i, j, k)] : (unsigned char)0;
  }
  __device__ void elem(const Grid<double>& g, int i, int j, int k, const double*, unsigned char code,
                       double (*out)[8], bool) const {
    if (code != 0) {
      // a constant-charge element: every corner load is the layer's table entry, no diagonal term
      const double v = wq[8 * k + code - 1];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        out[0][q] = v;
        out[1][q] = 0.0;
      }
      return;
    }
    const long long e = elem_index(g, i, j, k);
    load_c8<double>(elR, e, out[0]);
    load_c8<double>(elD, e, out[1]);
  }
  __device__ void node(const Grid<double>& g, int n, int i, int j, int k, double, double stiff, const double* mass) {
    double Rn = stiff + mass[0];
    double dg = stiff_diag(g, i, j, k) + mass[1];
    if (grid_is_dir(g, i, j, k)) {
      Rn = 0.0;
      dg = 1.0;
    }
    R[n] = Rn;
    if (diag) diag[n] = dg;
    if (dinv64) dinv64[n] = 1.0 / dg;
    // the FP32 Jacobi scale as an FP32 reciprocal (an FP64 division is a long sequence on the
    // FP64 pipe; the rounded diagonal's reciprocal is within an FP32 ulp of the rounded inverse)
    if (dinv32) dinv32[n] = __frcp_rn(__double2float_rn(dg));
    if (b64) b64[n] = -Rn;
    if (b32) b32[n] = (float)(-Rn);
    acc_r2 += Rn * Rn;
    acc_rmax = fmax(acc_rmax, fabs(Rn));
  }
  __device__ void finish() {
    if (stats) {
      double s[1] = {acc_r2};
      block_sum_atomic<1>(s, stats + 1);
      block_max_atomic(acc_rmax, stats);
    }
  }
};

// Pass 2 of a device with surface terms (Sec. II.A.4): the constant surface load b of the charged
// gates and surface charges is subtracted, and the charged gates' face mass adds to the diagonal
// (the face term of K_R phi comes from the skeleton's FACE instantiation).
struct SurfaceGatherOp : ResidualGatherOp {
  const double* bsurf;
  const double* face;  // charged gates' face coefficients or null
  __device__ void node(const Grid<double>& g, int n, int i, int j, int k, double, double stiff, const double* mass) {
    double Rn = stiff + mass[0] - bsurf[n];
    double dg = stiff_diag(g, i, j, k) + mass[1];
    if (face != nullptr && k == g.nz) dg += face_diag(g, face, i, j);
    if (grid_is_dir(g, i, j, k)) {
      Rn = 0.0;
      dg = 1.0;
    }
    R[n] = Rn;
    if (diag) diag[n] = dg;
    if (dinv64) dinv64[n] = 1.0 / dg;
    // the FP32 Jacobi scale as an FP32 reciprocal (an FP64 division is a long sequence on the
    // FP64 pipe; the rounded diagonal's reciprocal is within an FP32 ulp of the rounded inverse)
    if (dinv32) dinv32[n] = __frcp_rn(__double2float_rn(dg));
    if (b64) b64[n] = -Rn;
    if (b32) b32[n] = (float)(-Rn);
    acc_r2 += Rn * Rn;
    acc_rmax = fmax(acc_rmax, fabs(Rn));
  }
};

__host__ __device__ inline ResidualGatherOp make_gather_op(const ResidualArgs& args, double* elR, double* elD) {
  ResidualGatherOp op = {};
  op.phi = args.phi;
  op.elR = elR;
  op.elD = elD;
  op.ecode = args.ecode;
  op.wq = args.wq;
  op.R = args.R;
  op.diag = args.diag;
  op.dinv64 = args.dinv64;
  op.b64 = args.b64;
  op.stats = args.stats;
  op.dinv32 = args.dinv32;
  op.b32 = args.b32;
  return op;
}

void launch_residual_2pass(const Grid<double>& g, const ResidualArgs& args, double* el, LaunchCfg cfg,
                           cudaStream_t s, const double* face) {
  const long long ne = (long long)g.nx * g.ny * g.nz;
  double* elR = el;
  double* elD = el + 8 * ne;
  const int blocks = (int)((8 * ne + 255) / 256);
  note_launch(), residual_qp_kernel<<<blocks, 256, 0, s>>>(g, args, elR, elD);
  const ResidualGatherOp op = make_gather_op(args, elR, elD);
  LaunchCfg c = cfg;
  if (c.by == 32) c.by = 16;
  if (args.bsurf != nullptr) {
    SurfaceGatherOp sop;
    static_cast<ResidualGatherOp&>(sop) = op;
    sop.bsurf = args.bsurf;
    sop.face = face;
    if (face != nullptr)
      run_march_face<double>(g, sop, c, s, face);
    else
      run_march<double>(g, sop, c, s);
    return;
  }
  run_march<double>(g, op, c, s);
}

template <class T>
void launch_apply(const Grid<T>& g, const ApplyArgs<T>& args, LaunchCfg cfg, cudaStream_t s, const T* face) {
  if (face != nullptr) {  // charged gates: the element-gather skeleton carries the face term
    ApplyOp<T> op = {};
    op.a = args;
    run_march_face<T>(g, op, cfg, s, face);
    return;
  }
  if (cfg.variant >= 2) {
    launch_apply_lin<T>(g, args, cfg, s);
    return;
  }
  if constexpr (std::is_same<T, float>::value) {
    if (cfg.variant == 1) {
      launch_apply_pair(g, args, cfg, s);
      return;
    }
  }
  ApplyOp<T> op = {};
  op.a = args;
  run_march<T>(g, op, cfg, s);
}
template void launch_apply<float>(const Grid<float>&, const ApplyArgs<float>&, LaunchCfg, cudaStream_t,
                                  const float*);
template void launch_apply<double>(const Grid<double>&, const ApplyArgs<double>&, LaunchCfg, cudaStream_t,
                                   const double*);

// ---------------------------------------------------------------------------
// Electron count of one dot: the semiclassical n at the Gauss points of the dot's elements (an
// element box), weighted by w|J| and summed into *out; corners to Gauss points by the lane
// butterflies of residual_qp_kernel.
__global__ void __launch_bounds__(256) dot_count_kernel(const __grid_constant__ Grid<double> g, const double* phi,
                                                        const unsigned char* layer_semi, const __grid_constant__ Phys P,
                                                        int i0, int j0, int k0, int bx, int by, int bz, double* out) {
  const long long ne = (long long)bx * by * bz;
  const long long t = blockIdx.x * 256LL + threadIdx.x;
  const bool valid = t < 8 * ne;
  const long long be = valid ? (t >> 3) : 0;
  const int l = threadIdx.x & 7;
  const int i = i0 + (int)(be % bx), j = j0 + (int)((be / bx) % by), k = k0 + (int)(be / ((long long)bx * by));
  const bool semi = valid && layer_semi[k];
  const double A = GaussConst<double>::a(), B = GaussConst<double>::b();
  double v = 0.0;
  if (semi)
    v = __ldg(phi + (i + (l & 1)) + (long long)g.nxn * ((j + ((l >> 1) & 1)) + (long long)g.nyn * (k + (l >> 2))));
  v = A * v + B * __shfl_xor_sync(FULL_MASK, v, 1);
  v = A * v + B * __shfl_xor_sync(FULL_MASK, v, 2);
  v = A * v + B * __shfl_xor_sync(FULL_MASK, v, 4);
  double s[1] = {0.0};
  if (semi) s[0] = g.hx[i] * g.hy[j] * g.hz[k] * 0.125 * charge_at(P, v).n;
  block_sum_atomic<1>(s, out);
}

void launch_dot_count(const Grid<double>& g, const double* phi, const unsigned char* layer_semi, const Phys& P,
                      const int box[6], double* out, cudaStream_t s) {
  const long long ne = (long long)(box[1] - box[0]) * (box[3] - box[2]) * (box[5] - box[4]);
  if (ne <= 0) return;
  note_launch(), dot_count_kernel<<<(int)((8 * ne + 255) / 256), 256, 0, s>>>(
      g, phi, layer_semi, P, box[0], box[2], box[4], box[1] - box[0], box[3] - box[2], box[5] - box[4], out);
}

// ---------------------------------------------------------------------------
// dN_d/dphi nodal vector of one dot, in two passes over the dot's element box only (every other
// element has no count, and its nodes get zero).

// Pass 1: wdet dn/dphi at the quadrature points of the box's elements that belong to dot d (the
// first dot holding the element's centroid), mapped to the element corners by the transposed
// interpolation (lane butterflies as in residual_qp_kernel); [8 be + corner], be the element's
// index inside the box (x fastest).
__global__ void __launch_bounds__(256) count_grad_qp_kernel(const __grid_constant__ Grid<double> g,
                                                            const __grid_constant__ ResidualArgs a, int d, int i0,
                                                            int j0, int k0, int bx, int by, int bz, double* el) {
  const long long ne = (long long)bx * by * bz;
  const long long t = blockIdx.x * 256LL + threadIdx.x;
  const bool valid = t < 8 * ne;
  const long long be = valid ? (t >> 3) : 0;
  const int l = threadIdx.x & 7;
  const int i = i0 + (int)(be % bx), j = j0 + (int)((be / bx) % by), k = k0 + (int)(be / ((long long)bx * by));
  const bool in = valid && a.layer_semi[k] && dot_of_element(a, i, j, k) == d;
  const double A = GaussConst<double>::a(), B = GaussConst<double>::b();
  double v = 0.0;
  if (in)
    v = __ldg(a.phi + (i + (l & 1)) + (long long)g.nxn * ((j + ((l >> 1) & 1)) + (long long)g.nyn * (k + (l >> 2))));
  v = A * v + B * __shfl_xor_sync(FULL_MASK, v, 1);
  v = A * v + B * __shfl_xor_sync(FULL_MASK, v, 2);
  v = A * v + B * __shfl_xor_sync(FULL_MASK, v, 4);
  double f = 0.0;
  if (in) f = g.hx[i] * g.hy[j] * g.hz[k] * 0.125 * charge_at(a.P, v).dn;
  f = A * f + B * __shfl_xor_sync(FULL_MASK, f, 1);
  f = A * f + B * __shfl_xor_sync(FULL_MASK, f, 2);
  f = A * f + B * __shfl_xor_sync(FULL_MASK, f, 4);
  if (valid) el[t] = f;
}

// Pass 2: each node of the box's node range sums the corner values of its (up to eight) box
// elements: element (li - cx, lj - cy, lk - cz) holds the node as its corner cx + 2 cy + 4 cz.
__global__ void __launch_bounds__(256) count_grad_gather_kernel(const __grid_constant__ Grid<double> g,
                                                                const double* el, int i0, int j0, int k0, int bx,
                                                                int by, int bz, double* out) {
  const long long nn = (long long)(bx + 1) * (by + 1) * (bz + 1);
  const long long t = blockIdx.x * 256LL + threadIdx.x;
  if (t >= nn) return;
  const int li = (int)(t % (bx + 1)), lj = (int)((t / (bx + 1)) % (by + 1));
  const int lk = (int)(t / ((long long)(bx + 1) * (by + 1)));
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int ei = li - (c & 1), ej = lj - ((c >> 1) & 1), ek = lk - (c >> 2);
    if (ei >= 0 && ei < bx && ej >= 0 && ej < by && ek >= 0 && ek < bz)
      s += el[8 * (ei + (long long)bx * (ej + (long long)by * ek)) + c];
  }
  out[(i0 + li) + (long long)g.nxn * ((j0 + lj) + (long long)g.nyn * (k0 + lk))] = s;
}

void launch_count_gradient(const Grid<double>& g, const double* phi, const unsigned char* layer_semi,
                           const double* xn, const double* yn, const double* zn, const Phys& P,
                           const DotBoxes& dots, int d, const int* box, double* out, double* el, cudaStream_t s) {
  if (box == nullptr) return;
  const int bx = box[1] - box[0], by = box[3] - box[2], bz = box[5] - box[4];
  const long long ne = (long long)bx * by * bz;
  if (ne <= 0) return;
  ResidualArgs a{};
  a.phi = phi;
  a.layer_semi = layer_semi;
  a.xn = xn;
  a.yn = yn;
  a.zn = zn;
  a.P = P;
  a.dots = dots;
  note_launch(), count_grad_qp_kernel<<<(int)((8 * ne + 255) / 256), 256, 0, s>>>(g, a, d, box[0], box[2], box[4],
                                                                                  bx, by, bz, el);
  const long long nn = (long long)(bx + 1) * (by + 1) * (bz + 1);
  note_launch(), count_grad_gather_kernel<<<(int)((nn + 255) / 256), 256, 0, s>>>(g, el, box[0], box[2], box[4], bx,
                                                                                  by, bz, out);
}


template <class T>
void launch_pcg_apply(const Grid<T>& g, PcgVecs<T> vecs, PcgScalars* sc, LaunchCfg cfg, cudaStream_t s,
                      const T* face) {
  if (face != nullptr) {  // charged gates: the element-gather skeleton carries the face term
    PcgApplyOp<T> op = {};
    op.v = vecs;
    op.sc = sc;
    run_march_face<T>(g, op, cfg, s, face);
    return;
  }
  if (cfg.variant >= 2) {
    launch_pcg_apply_lin<T>(g, vecs, sc, cfg, s);
    return;
  }
  if constexpr (std::is_same<T, float>::value) {
    if (cfg.variant == 1) {
      launch_pcg_apply_pair(g, vecs, sc, cfg, s);
      return;
    }
  }
  PcgApplyOp<T> op = {};
  op.v = vecs;
  op.sc = sc;
  run_march<T>(g, op, cfg, s);
}
template void launch_pcg_apply<float>(const Grid<float>&, PcgVecs<float>, PcgScalars*, LaunchCfg, cudaStream_t,
                                      const float*);
template void launch_pcg_apply<double>(const Grid<double>&, PcgVecs<double>, PcgScalars*, LaunchCfg, cudaStream_t,
                                       const double*);


constexpr int VEC_THREADS = 256;

// Grid of the vector kernels: at most four blocks per SM of the 152 (a multiple of the SM
// count, few same-address reduction atomics, enough loads in flight to saturate HBM).
static int vec_blocks(long long n) {
  long long b = (n + VEC_THREADS - 1) / VEC_THREADS;
  const long long cap = 152 * 4;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}


// Sums two per-thread partials over the block (FP64 across threads) and adds them to dst0, dst1.
__device__ __forceinline__ void block_sum2_atomic(double v0, double v1, double* dst0, double* dst1) {
  __shared__ double red[2][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v0 = warp_sum(v0);
  v1 = warp_sum(v1);
  if (lane == 0) {
    red[0][warp] = v0;
    red[1][warp] = v1;
  }
  __syncthreads();
  if (warp == 0) {
    double w0 = lane < (int)(blockDim.x >> 5) ? red[0][lane] : 0.0;
    double w1 = lane < (int)(blockDim.x >> 5) ? red[1][lane] : 0.0;
    w0 = warp_sum(w0);
    w1 = warp_sum(w1);
    if (lane == 0) {
      atomicAdd(dst0, w0);
      atomicAdd(dst1, w1);
    }
  }
}

template <class T>
__global__ void __launch_bounds__(VEC_THREADS) pcg_init_kernel(int n, PcgVecs<T> v, PcgScalars* sc) {
  T rz = T(0), rr = T(0);
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    const T r = v.b[idx];
    const T z = v.dinv[idx] * r;
    v.x[idx] = T(0);
    v.r[idx] = r;
    v.z[idx] = z;
    rz += r * z;
    rr += r * r;
  }
  block_sum2_atomic((double)rz, (double)rr, &sc->rz[0], &sc->rr[0]);
  if (last_block(&sc->counter) && threadIdx.x == 0) {
    const double rr0 = ld_volatile(&sc->rr[0]);
    const double rz0 = ld_volatile(&sc->rz[0]);
    sc->rr0 = rr0;
    sc->t = 0;
    sc->iters = 0;
    sc->phase = 1;
    sc->pAp[0] = 0.0;
    sc->rz[1] = 0.0;
    sc->rr[1] = 0.0;
    if (!(rr0 == rr0) || !(rz0 == rz0) || rr0 > 1e300) {
      sc->nonfinite = 1;
      sc->done = 1;
    } else if (rr0 == 0.0) {
      sc->done = 1;
    }
    sc->counter = 0;
  }
}

template <class T>
void launch_pcg_init(long long n, PcgVecs<T> v, PcgScalars* sc, cudaStream_t s) {
  note_launch(), pcg_init_kernel<T><<<vec_blocks(n), VEC_THREADS, 0, s>>>((int)n, v, sc);
}
template void launch_pcg_init<float>(long long, PcgVecs<float>, PcgScalars*, cudaStream_t);
template void launch_pcg_init<double>(long long, PcgVecs<double>, PcgScalars*, cudaStream_t);

// x += alpha p, r -= alpha Ap, z = D^-1 r, partial r.z and r.r per thread in the storage
// precision (a handful of terms each), FP64 across threads.
template <class T>
__device__ __forceinline__ void pcg_update_body(int n, const PcgVecs<T>& v, PcgScalars* sc, int blk, int nblk) {
  if (sc->done) return;
  const int t = sc->t;
  const double alpha_d = sc->rz[t & 3] / sc->pAp[t & 3];
  const T alpha = (T)alpha_d;
  const T* __restrict__ p = v.p[t & 1];
  T rz = T(0), rr = T(0);
  for (int idx = blk * blockDim.x + threadIdx.x; idx < n; idx += nblk * blockDim.x) {
    const T pp = p[idx];
    const T ap = v.Ap[idx];
    const T xo = v.x[idx];
    const T ro = v.r[idx];
    const T di = v.dinv[idx];
    v.x[idx] = xo + alpha * pp;
    const T r = ro - alpha * ap;
    const T z = di * r;
    v.r[idx] = r;
    v.z[idx] = z;
    rz += r * z;
    rr += r * r;
  }
  block_sum2_atomic((double)rz, (double)rr, &sc->rz[(t + 1) & 3], &sc->rr[(t + 1) & 3]);
  if (last_block_of(&sc->counter, nblk) && threadIdx.x == 0) pcg_finish(sc, t, alpha_d);
}

template <class T>
__global__ void __launch_bounds__(VEC_THREADS) pcg_update_kernel(int n, PcgVecs<T> v, PcgScalars* sc) {
  pcg_update_body<T>(n, v, sc, blockIdx.x, gridDim.x);
}

template <class T>
void launch_pcg_update(long long n, PcgVecs<T> v, PcgScalars* sc, cudaStream_t s) {
  note_launch(), pcg_update_kernel<T><<<vec_blocks(n), VEC_THREADS, 0, s>>>((int)n, v, sc);
}
template void launch_pcg_update<float>(long long, PcgVecs<float>, PcgScalars*, cudaStream_t);
template void launch_pcg_update<double>(long long, PcgVecs<double>, PcgScalars*, cudaStream_t);

// ---------------------------------------------------------------------------
// Chebyshev-Jacobi preconditioner z = p_k(D^-1 J) D^-1 r (Chebyshev iteration for J z = r
// with Jacobi scaling from z_0 = 0 on the interval [theta - delta, theta + delta] of D^-1 J):
//   d_0 = D^-1 r / theta, z_1 = d_0, w_1 = r,
//   w_{j+1} = w_j - J d_{j-1},  d_j = rho_j rho_{j-1} d_{j-1} + (2 rho_j / delta) D^-1 w_{j+1},
//   z_{j+1} = z_j + d_j,  rho_0 = delta/theta, rho_j = 1 / (2 theta/delta - rho_{j-1}).
template <class T>
__global__ void __launch_bounds__(VEC_THREADS) pcg_update_cheb_kernel(int n, PcgVecs<T> v, PcgScalars* sc) {
  if (sc->done) return;
  const int t = sc->t;
  const double alpha_d = sc->rz[t & 3] / sc->pAp[t & 3];
  if (!(alpha_d == alpha_d) || alpha_d <= 0.0 || fabs(alpha_d) > 1e300) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      sc->nonfinite = 1;
      sc->iters = t;
      sc->done = 1;
    }
    return;
  }
  const T alpha = (T)alpha_d;
  const T inv_theta = (T)(1.0 / sc->theta);
  const T* __restrict__ p = v.p[t & 1];
  T* __restrict__ d0 = v.d[0];
  T rr = T(0);
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    v.x[idx] += alpha * p[idx];
    const T r = v.r[idx] - alpha * v.Ap[idx];
    const T d = v.dinv[idx] * r * inv_theta;
    v.r[idx] = r;
    v.w[idx] = r;
    d0[idx] = d;
    v.z[idx] = d;
    rr += r * r;
  }
  double s1[1] = {(double)rr};
  block_sum_atomic<1>(s1, &sc->rr[(t + 1) & 3]);
}

template <class T>
void launch_pcg_update_cheb(long long n, PcgVecs<T> v, PcgScalars* sc, cudaStream_t s) {
  note_launch(), pcg_update_cheb_kernel<T><<<vec_blocks(n), VEC_THREADS, 0, s>>>((int)n, v, sc);
}
template void launch_pcg_update_cheb<float>(long long, PcgVecs<float>, PcgScalars*, cudaStream_t);
template void launch_pcg_update_cheb<double>(long long, PcgVecs<double>, PcgScalars*, cudaStream_t);

template <class T>
__global__ void __launch_bounds__(VEC_THREADS) pcg_init_cheb_kernel(int n, PcgVecs<T> v, PcgScalars* sc) {
  const T inv_theta = (T)(1.0 / sc->theta);
  T rr = T(0);
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    const T r = v.b[idx];
    const T d = v.dinv[idx] * r * inv_theta;
    v.x[idx] = T(0);
    v.r[idx] = r;
    v.w[idx] = r;
    v.d[0][idx] = d;
    v.z[idx] = d;
    rr += r * r;
  }
  double s1[1] = {(double)rr};
  block_sum_atomic<1>(s1, &sc->rr[0]);
}

template <class T>
void launch_pcg_init_cheb(long long n, PcgVecs<T> v, PcgScalars* sc, cudaStream_t s) {
  note_launch(), pcg_init_cheb_kernel<T><<<vec_blocks(n), VEC_THREADS, 0, s>>>((int)n, v, sc);
}
template void launch_pcg_init_cheb<float>(long long, PcgVecs<float>, PcgScalars*, cudaStream_t);
template void launch_pcg_init_cheb<double>(long long, PcgVecs<double>, PcgScalars*, cudaStream_t);


template <class T>
void launch_cheb_step(const Grid<T>& g, PcgVecs<T> vecs, PcgScalars* sc, int step, int last, LaunchCfg cfg,
                      cudaStream_t s, const T* face) {
  if (face != nullptr) {  // charged gates: the element-gather skeleton carries the face term
    ChebStepOp<T> op = {};
    op.v = vecs;
    op.sc = sc;
    op.step = step;
    op.last = last;
    run_march_face<T>(g, op, cfg, s, face);
    return;
  }
  if (cfg.variant >= 2) {
    launch_cheb_step_lin<T>(g, vecs, sc, step, last, cfg, s);
    return;
  }
  if constexpr (std::is_same<T, float>::value) {
    if (cfg.variant == 1) {
      launch_cheb_step_pair(g, vecs, sc, step, last, cfg, s);
      return;
    }
  }
  ChebStepOp<T> op = {};
  op.v = vecs;
  op.sc = sc;
  op.step = step;
  op.last = last;
  run_march<T>(g, op, cfg, s);
}
template void launch_cheb_step<float>(const Grid<float>&, PcgVecs<float>, PcgScalars*, int, int, LaunchCfg,
                                      cudaStream_t, const float*);
template void launch_cheb_step<double>(const Grid<double>&, PcgVecs<double>, PcgScalars*, int, int, LaunchCfg,
                                       cudaStream_t, const double*);

// ---------------------------------------------------------------------------
// FP32 pair-kernel ops (march2_kernel): one node per callback, element pairs inside the skeleton.
struct Apply2Op {
  ApplyArgs<float> a;
  float acc;
  __device__ bool skip() const { return false; }
  __device__ void set_vec(int) {}
  __device__ float load(int n, bool) const { return a.v[n]; }
  __device__ void edata(const Grid<float>& g, int i, int j, int k, float (&c)[8]) const {
    load_c8<float>(a.c, elem_index(g, i, j, k), c);
  }
  __device__ void node(const Grid<float>& g, int n, int i, int j, int k, float vin, float y) {
    if (!a.raw && grid_is_dir(g, i, j, k)) y = vin;
    a.y[n] = y;
    acc += vin * y;
  }
  __device__ void finish() {
    if (a.dot) {
      double s1[1] = {(double)acc};
      block_sum_atomic<1>(s1, a.dot);
    }
  }
};

struct PcgApply2Op {
  PcgVecs<float> v;
  PcgScalars* sc;
  int t;
  float beta;
  float acc;
  __device__ bool skip() const { return sc->done != 0; }
  const float* pprev;
  float* pcur;
  __device__ void set_vec(int) {
    t = sc->t;
    beta = t > 0 ? (float)(sc->rz[t & 3] / sc->rz[(t - 1) & 3]) : 0.f;
    pprev = (t & 1) ? v.p[0] : v.p[1];
    pcur = (t & 1) ? v.p[1] : v.p[0];
  }
  __device__ float load(int n, bool) const { return t > 0 ? v.z[n] + beta * pprev[n] : v.z[n]; }
  __device__ void edata(const Grid<float>& g, int i, int j, int k, float (&c)[8]) const {
    load_c8<float>(v.c, elem_index(g, i, j, k), c);
  }
  __device__ void node(const Grid<float>& g, int n, int i, int j, int k, float pin, float y) {
    if (grid_is_dir(g, i, j, k)) y = pin;
    pcur[n] = pin;
    v.Ap[n] = y;
    acc += pin * y;
  }
  __device__ void finish() {
    double s1[1] = {(double)acc};
    block_sum_atomic<1>(s1, &sc->pAp[t & 3]);
  }
};

struct ChebStep2Op {
  PcgVecs<float> v;
  PcgScalars* sc;
  int step, last;
  int t, slot;
  const float* dprev;
  float* dcur;
  float c1, c2;
  float acc;
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
    c1 = (float)(rho * rho_prev);
    c2 = (float)(2.0 * rho / sc->delta);
    dprev = (step & 1) ? v.d[0] : v.d[1];
    dcur = (step & 1) ? v.d[1] : v.d[0];
  }
  __device__ float load(int n, bool) const { return dprev[n]; }
  __device__ void edata(const Grid<float>& g, int i, int j, int k, float (&c)[8]) const {
    load_c8<float>(v.c, elem_index(g, i, j, k), c);
  }
  __device__ void node(const Grid<float>& g, int n, int i, int j, int k, float dold, float y) {
    if (grid_is_dir(g, i, j, k)) y = dold;
    const float wn = v.w[n] - y;
    const float dn = c1 * dold + c2 * v.dinv[n] * wn;
    const float zn = v.z[n] + dn;
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

template <class Op>
static void run_march2(const Grid<float>& g, const Op& op, LaunchCfg cfg, cudaStream_t s) {
  const int by = (cfg.by == 4 || cfg.by == 16) ? cfg.by : 8;
  dim3 grid = march2_grid(g.nxn, g.nyn, g.nzn, by, cfg.kchunk);
  if (by == 4)
    note_launch(), march2_kernel<4, Op><<<grid, dim3(32, 4), 0, s>>>(g, op, cfg.kchunk);
  else if (by == 16)
    note_launch(), march2_kernel<16, Op><<<grid, dim3(32, 16), 0, s>>>(g, op, cfg.kchunk);
  else
    note_launch(), march2_kernel<8, Op><<<grid, dim3(32, 8), 0, s>>>(g, op, cfg.kchunk);
}

void launch_apply_pair(const Grid<float>& g, const ApplyArgs<float>& a, LaunchCfg cfg, cudaStream_t s) {
  Apply2Op op = {};
  op.a = a;
  run_march2(g, op, cfg, s);
}
void launch_pcg_apply_pair(const Grid<float>& g, PcgVecs<float> v, PcgScalars* sc, LaunchCfg cfg, cudaStream_t s) {
  PcgApply2Op op = {};
  op.v = v;
  op.sc = sc;
  run_march2(g, op, cfg, s);
}
void launch_cheb_step_pair(const Grid<float>& g, PcgVecs<float> v, PcgScalars* sc, int step, int last,
                           LaunchCfg cfg, cudaStream_t s) {
  ChebStep2Op op = {};
  op.v = v;
  op.sc = sc;
  op.step = step;
  op.last = last;
  run_march2(g, op, cfg, s);
}

template <class T>
__global__ void __launch_bounds__(VEC_THREADS)
power_step_kernel(int n, const T* v, const T* Jv, const T* dinv, T* vn, double* acc) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    const double x = (double)v[idx], y = (double)Jv[idx], di = (double)dinv[idx];
    const double z = di * y;
    vn[idx] = (T)z;
    a0 += x * y;
    a1 += x * x / di;
    a2 += z * z;
  }
  double s3[3] = {a0, a1, a2};
  block_sum_atomic<3>(s3, acc);
}

template <class T>
void launch_power_step(long long n, const T* v, const T* Jv, const T* dinv, T* vnext, double* acc, cudaStream_t s) {
  note_launch(), power_step_kernel<T><<<vec_blocks(n), VEC_THREADS, 0, s>>>((int)n, v, Jv, dinv, vnext, acc);
}
template void launch_power_step<float>(long long, const float*, const float*, const float*, float*, double*,
                                       cudaStream_t);
template void launch_power_step<double>(long long, const double*, const double*, const double*, double*, double*,
                                        cudaStream_t);

// Counter-based random vector (SplitMix64 finalizer of the index), zero on Dirichlet nodes.
template <class T>
__global__ void random_free_kernel(Grid<T> g, unsigned long long seed, T* v) {
  const int n = (int)(g.plane * g.nzn);
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    const int i = idx % g.nxn, j = (idx / g.nxn) % g.nyn, k = idx / (int)g.plane;
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(idx + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    v[idx] = grid_is_dir(g, i, j, k) ? T(0) : (T)u;
  }
}
template <class T>
void launch_random_free(const Grid<T>& g, unsigned long long seed, T* v, cudaStream_t s) {
  note_launch(), random_free_kernel<T><<<vec_blocks(g.plane * g.nzn), VEC_THREADS, 0, s>>>(g, seed, v);
}
template void launch_random_free<float>(const Grid<float>&, unsigned long long, float*, cudaStream_t);
template void launch_random_free<double>(const Grid<double>&, unsigned long long, double*, cudaStream_t);

template <class T>
__global__ void scale_kernel(int n, T* v, double a) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) v[idx] = (T)(a * v[idx]);
}
template <class T>
void launch_scale(long long n, T* v, double a, cudaStream_t s) {
  note_launch(), scale_kernel<T><<<vec_blocks(n), VEC_THREADS, 0, s>>>((int)n, v, a);
}
template void launch_scale<float>(long long, float*, double, cudaStream_t);
template void launch_scale<double>(long long, double*, double, cudaStream_t);

// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(VEC_THREADS)
newton_trial_kernel(long long n, const double* phi, const T* delta, double alpha, double* out, double* stats) {
  double m = 0.0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const double d = alpha * (double)delta[idx];
    out[idx] = phi[idx] + d;
    m = fmax(m, fabs(d));
  }
  const double w = warp_max(m);
  if ((threadIdx.x & 31) == 0 && w > 0.0) atomic_max_nonneg(stats, w);
}

template <class T>
void launch_newton_trial(long long n, const double* phi, const T* delta, double alpha, double* phi_out,
                         double* stats, cudaStream_t s) {
  note_launch(), newton_trial_kernel<T><<<vec_blocks(n), VEC_THREADS, 0, s>>>(n, phi, delta, alpha, phi_out, stats);
}
template void launch_newton_trial<float>(long long, const double*, const float*, double, double*, double*, cudaStream_t);
template void launch_newton_trial<double>(long long, const double*, const double*, double, double*, double*, cudaStream_t);

__global__ void set_dirichlet_kernel(long long nxn, long long nyn, long long nzn, int bottom, double vb,
                                     const signed char* gate_top, const double* vg, double* phi) {
  const long long plane = nxn * nyn;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < plane;
       idx += (long long)gridDim.x * blockDim.x) {
    if (bottom) phi[idx] = vb;
    const int gid = gate_top ? gate_top[idx] : -1;
    if (gid >= 0) phi[(nzn - 1) * plane + idx] = vg[gid];
  }
}

void launch_set_dirichlet(long long nxn, long long nyn, long long nzn, int bottom, double v_bottom,
                          const signed char* gate_top, const double* v_gate, double* phi, cudaStream_t s) {
  note_launch(), set_dirichlet_kernel<<<vec_blocks(nxn * nyn), VEC_THREADS, 0, s>>>(nxn, nyn, nzn, bottom, v_bottom, gate_top,
                                                                    v_gate, phi);
}

__global__ void d2f_kernel(long long n, const double* a, float* b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void f2d_kernel(long long n, const float* a, double* b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}
void launch_d2f(long long n, const double* a, float* b, cudaStream_t s) {
  note_launch(), d2f_kernel<<<vec_blocks(n), VEC_THREADS, 0, s>>>(n, a, b);
}
void launch_f2d(long long n, const float* a, double* b, cudaStream_t s) {
  note_launch(), f2d_kernel<<<vec_blocks(n), VEC_THREADS, 0, s>>>(n, a, b);
}

// theta gradient: out[e] = qe * (|e|/8) * sum of lam over the corners of e.
__global__ void theta_gradient_kernel(int nx, int ny, int nz, const double* hx, const double* hy, const double* hz,
                                      const double* lam, double qe, double* out) {
  const long long ne = (long long)nx * ny * nz;
  const long long nxn = nx + 1, plane = (long long)(nx + 1) * (ny + 1);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % nx);
    const int j = (int)((e / nx) % ny);
    const int k = (int)(e / ((long long)nx * ny));
    const long long n0 = i + nxn * j + plane * k;
    const double s = lam[n0] + lam[n0 + 1] + lam[n0 + nxn] + lam[n0 + nxn + 1] + lam[n0 + plane] +
                     lam[n0 + plane + 1] + lam[n0 + plane + nxn] + lam[n0 + plane + nxn + 1];
    out[e] = qe * (hx[i] * hy[j] * hz[k] * 0.125) * s;
  }
}

void launch_theta_gradient(int nx, int ny, int nz, const double* hx, const double* hy, const double* hz,
                           const double* lam, double qe, double* out, cudaStream_t s) {
  const long long ne = (long long)nx * ny * nz;
  note_launch(), theta_gradient_kernel<<<vec_blocks(ne), VEC_THREADS, 0, s>>>(nx, ny, nz, hx, hy, hz, lam, qe, out);
}

}  // namespace qcad

namespace qcad {

// out[0] += sum_i a_i b_i (FP64 accumulation).
template <class T>
__global__ void __launch_bounds__(VEC_THREADS) dot_kernel(long long n, const T* a, const T* b, double* out) {
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += (double)a[i] * (double)b[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0 && s != 0.0) atomicAdd(out, s);
}
template <class T>
void launch_dot(long long n, const T* a, const T* b, double* out, cudaStream_t s) {
  note_launch(), dot_kernel<T><<<vec_blocks(n), VEC_THREADS, 0, s>>>(n, a, b, out);
}
template void launch_dot<float>(long long, const float*, const float*, double*, cudaStream_t);
template void launch_dot<double>(long long, const double*, const double*, double*, cudaStream_t);

// y = a x + y with mixed types (FP64 y, T x).
template <class T>
__global__ void axpy_kernel(long long n, double a, const T* x, double* y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] += a * (double)x[i];
}
template <class T>
void launch_axpy(long long n, double a, const T* x, double* y, cudaStream_t s) {
  note_launch(), axpy_kernel<T><<<vec_blocks(n), VEC_THREADS, 0, s>>>(n, a, x, y);
}
template void launch_axpy<float>(long long, double, const float*, double*, cudaStream_t);
template void launch_axpy<double>(long long, double, const double*, double*, cudaStream_t);

// r = g - y (FP64), also writes the FP32 copy; zero on Dirichlet rows is inherited from g and y.
__global__ void sub_kernel(long long n, const double* g, const double* y, double* r, float* r32) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = g[i] - y[i];
    r[i] = v;
    if (r32) r32[i] = (float)v;
  }
}
void launch_sub(long long n, const double* g, const double* y, double* r, float* r32, cudaStream_t s) {
  note_launch(), sub_kernel<<<vec_blocks(n), VEC_THREADS, 0, s>>>(n, g, y, r, r32);
}

}  // namespace qcad

#include <atomic>
namespace qcad {
static std::atomic<long long> g_launches{0};
void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace qcad

namespace qcad {
// Resident blocks per SM of the plain Jacobian apply kernel for a launch shape (autotuner).
int apply_blocks_per_sm(int precision, int by, int variant) {
  if (variant >= 2) return lin_blocks_per_sm(precision, by, variant == 3 ? 2 : 1);
  int n = 0;
  cudaError_t e = cudaSuccess;
  if (precision == 1 && variant == 1) {
    if (by == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, march2_kernel<4, Apply2Op>, 32 * 4, 0);
    else if (by == 16) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, march2_kernel<16, Apply2Op>, 32 * 16, 0);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, march2_kernel<8, Apply2Op>, 32 * 8, 0);
  } else if (precision == 1) {
    if (by == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, march_kernel<float, 4, ApplyOp<float>>, 128, 0);
    else if (by == 16) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, march_kernel<float, 16, ApplyOp<float>>, 512, 0);
    else if (by == 32) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, march_kernel<float, 32, ApplyOp<float>>, 1024, 0);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, march_kernel<float, 8, ApplyOp<float>>, 256, 0);
  } else {
    if (by == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, march_kernel<double, 4, ApplyOp<double>>, 128, 0);
    else if (by == 16) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, march_kernel<double, 16, ApplyOp<double>>, 512, 0);
    else if (by == 32) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, march_kernel<double, 32, ApplyOp<double>>, 1024, 0);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, march_kernel<double, 8, ApplyOp<double>>, 256, 0);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}
}  // namespace qcad

#include "batch_kernels.cuh"
