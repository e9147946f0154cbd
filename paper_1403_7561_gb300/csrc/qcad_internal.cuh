// Internal declarations of libqcad: device views of the mesh, physics
// parameters, and the z-marching tile skeleton shared by every operator
// kernel (Poisson residual, Jacobian apply, Schrodinger H/M apply).
//
// Discretization (Sec. II.A.3 Eq. PoissonWeakForm, Sec. II.B Eq.
// SchrodEqnWeakForm): Q1 hexahedra on a tensor-product mesh with 2x2x2 Gauss
// quadrature. On an axis-aligned box the stiffness term of every element is
// separable, kappa_x K(x) M(y) M(z) + kappa_y M K M + kappa_z M M K with 1D
// linear-element stiffness K and consistent mass M; because kappa depends on
// the z layer only, the assembled stiffness is the sum of three Kronecker
// products of assembled 1D tridiagonal operators. The kernels therefore apply
// stiffness node-centrically as a separable 27-point stencil and only the
// quadrature-point mass term (nonlinear charge term, potential energy) element
// by element.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define QCAD_BX 32
#define FULL_MASK 0xffffffffu
#define QCAD_MAX_DOTS_K 8

namespace qcad {

// Device view of a structured Q1 grid (the Poisson mesh or the Schrodinger
// subdomain). 1D assembled operator rows hold the coefficients of nodes
// (n-1, n, n+1); entries for missing elements are zero.
template <class T>
struct Grid {
  int nx, ny, nz;        // elements
  int nxn, nyn, nzn;     // nodes
  long long plane;       // nxn * nyn
  const T* mx;           // [nxn*3] assembled 1D mass along x
  const T* kx;           // [nxn*3] assembled 1D stiffness along x
  const T* my;
  const T* ky;
  const T* mzx;          // [nzn*3] kappa_x-weighted 1D mass along z
  const T* mzy;          // [nzn*3] kappa_y-weighted 1D mass along z
  const T* kzz;          // [nzn*3] kappa_z-weighted 1D stiffness along z
  const T* zt;           // [nzn*12] mzx, mzy, kzz rows of each plane packed (3 zeros pad), or null
  const T* hx;           // [nx] element sizes
  const T* hy;           // [ny]
  const T* hz;           // [nz]
  const unsigned char* dir_top;  // [nxn*nyn] Dirichlet mask of the top plane or null
  int dir_bottom;        // every node of plane k = 0 is Dirichlet
  int dir_boundary;      // every boundary node is Dirichlet (Schrodinger subdomain)
};

// Charged gates (the Robin condition): alpha[fi + nx fj] = eps_r/d of every top-plane face (0 off
// the charged gates); the linear operators add the face mass sum_f alpha_f int_f N_a N_b on the
// top plane. The coefficients travel as a kernel argument of their own instantiations, not in
// Grid, so the kernels of devices without charged gates are unchanged.
//
// Face term of node (i, j) of the top plane: sum over its (up to four) faces f of
// alpha_f (h_x h_y / 36) (4 v_self + 2 v_x-neighbour + 2 v_y-neighbour + v_diagonal), the row of
// the bilinear face mass; v(di, dj) returns the value at (i + di, j + dj).
template <class T, class V>
__device__ __forceinline__ T face_row(const Grid<T>& g, const T* alpha, int i, int j, V v) {
  T y = 0;
#pragma unroll
  for (int sy = -1; sy <= 0; ++sy)
#pragma unroll
    for (int sx = -1; sx <= 0; ++sx) {
      const int fi = i + sx, fj = j + sy;
      if (fi < 0 || fj < 0 || fi >= g.nx || fj >= g.ny) continue;
      const T a = alpha[fi + g.nx * fj];
      if (a == T(0)) continue;
      const int dx = sx == 0 ? 1 : -1, dy = sy == 0 ? 1 : -1;  // the face's other corner offsets
      const T w = a * g.hx[fi] * g.hy[fj] * T(1.0 / 36.0);
      y += w * (T(4) * v(0, 0) + T(2) * v(dx, 0) + T(2) * v(0, dy) + v(dx, dy));
    }
  return y;
}

// Diagonal of the face mass at node (i, j) of the top plane: sum_f alpha_f h_x h_y / 9.
template <class T>
__device__ __forceinline__ T face_diag(const Grid<T>& g, const T* alpha, int i, int j) {
  T d = 0;
  for (int sy = -1; sy <= 0; ++sy)
    for (int sx = -1; sx <= 0; ++sx) {
      const int fi = i + sx, fj = j + sy;
      if (fi < 0 || fj < 0 || fi >= g.nx || fj >= g.ny) continue;
      d += alpha[fi + g.nx * fj] * g.hx[fi] * g.hy[fj] * T(1.0 / 9.0);
    }
  return d;
}

template <class T>
__device__ __forceinline__ bool grid_is_dir(const Grid<T>& g, int i, int j, int k) {
  if (g.dir_boundary && (i == 0 || j == 0 || k == 0 || i == g.nx || j == g.ny || k == g.nz)) return true;
  if (g.dir_bottom && k == 0) return true;
  if (k == g.nz && g.dir_top != nullptr && g.dir_top[i + g.nxn * j]) return true;
  return false;
}

// Density below which a carrier or ionized-dopant term of the residual is not evaluated, outside
// the dot regions (nm^-3; 1e-25 nm^-3 is 1e-4 carriers per cm^3). Its contribution to a residual
// entry, (q/eps0) |e| rho N_a <= 18.1 V nm^-2 x |e| x 1e-25, stays below 1e-20 V nm on elements of
// up to 5000 nm^3, and to the Jacobian, (q/eps0) |e| rho / kT, below 1e-16 of a stiffness entry
// at 0.5 K: far under the FP64 rounding of the stiffness term K phi and the 1e-10 V nm
// tolerance. The dot electron counts keep the 1e-60 nm^-3 cutoffs (eta -150, z 746).
constexpr double RHO_RESID_FLOOR = 1e-25;

// Semiconductor parameters at the bias point (one semiconductor per device).
struct Phys {
  double kT, inv_kT;      // eV, 1/eV
  double NC, NV;          // nm^-3
  double phi_ref;         // V (q phi_ref in eV, Eq. qPhiRef)
  double chi, Eg;         // eV
  double EF;              // eV
  double NA, ND;          // nm^-3
  double Ea, Ed, gA, gD;
  double qe;              // q/eps0, V*nm
  int statistics;         // 0 MB, 1 FD
  int incomplete;         // 1: Eq. FinalIonization
  int na_on, nd_on;       // NA != 0, ND != 0 (tested on the integer pipes)
  // Below-resolution cutoffs of the residual outside the dots (densities under RHO_RESID_FLOOR,
  // physics.cuh): n and p are not evaluated for eta below eta_min_n / eta_min_p, and the ionized
  // acceptor (donor) density is taken as zero for an ionization argument above z_max_a (z_max_d).
  double eta_min_n, eta_min_p, z_max_a, z_max_d;
  // the same cutoffs as potentials (V): n needs evaluating only for phi >= phi_n_on, p only for
  // phi <= phi_p_on; the acceptor (donor) ionization is a constant (0 or 1) outside
  // [phi_a_lo, phi_a_hi] ([phi_d_lo, phi_d_hi]), where its argument is beyond the cutoff or below -45
  double phi_n_on, phi_p_on, phi_a_lo, phi_a_hi, phi_d_lo, phi_d_hi;
  // the same potentials as order-preserving integer keys (double_key), compared on the integer
  // pipes instead of the 2-lane FP64 pipe
  unsigned long long key_n_on, key_p_on, key_a_lo, key_a_hi, key_d_lo, key_d_hi;
};

// An unsigned integer key of a double that orders like the doubles (non-NaN): the sign bit set
// for non-negative values, all bits flipped for negative ones.
__host__ __device__ __forceinline__ unsigned long long double_key(unsigned long long bits) {
  return (bits >> 63) ? ~bits : (bits | 0x8000000000000000ull);
}

struct DotBoxes {
  int n;
  double b[8][6];         // x0, x1, y0, y1, z0, z1 of element centroids
};

// Quantum electron density of the self-consistent Schrodinger-Poisson loop (Sec. II.C) in the
// quantum region (an element box): the predictor density of Eq. ApproxEDens3DConfined,
// n~(phi) = sum_i w_i / (1 + exp((E_i - E_F - (phi - phi_prev)) / kT)) at the Gauss points, with
// w_i = 4 |psi_i|^2 there. Inactive when w is null.
constexpr int QD_MAX_STATES = 16;
struct QuantumDensity {
  const double* w;        // [quantum element][Gauss point][state]
  const double* phiq;     // [quantum element][Gauss point]: phi the eigenpairs were computed at
  double E[QD_MAX_STATES];  // eigenvalues, eV
  int nev;
  int i0, j0, k0, nx, ny, nz;  // first element and extent of the quantum region
};

// Occupation 1 / (1 + e^a) and g = -df/da, with exp(-a) for a > 100 (the paper's safeguard for
// states far above the Fermi level; exp(-a) is below half the smallest subnormal beyond 746).
__device__ __forceinline__ void qd_fermi(double a, double& f, double& g) {
  if (a > 100.0) {
    f = a > 746.0 ? 0.0 : exp(-a);
    g = f;
  } else {
    const double e = exp(a);
    f = 1.0 / (1.0 + e);
    g = f * (1.0 - f);
  }
}

// n~ and d n~/d phi at Gauss point q of quantum element qe, at potential phi (E_F in eV, ik = 1/kT).
__device__ __forceinline__ void qd_density(const QuantumDensity& qd, long long qe, int q, double phi, double EF,
                                           double ik, double& n, double& dn) {
  const double dphi = phi - qd.phiq[8 * qe + q];
  const double* w = qd.w + (8 * qe + q) * qd.nev;
  double s = 0.0, ds = 0.0;
  for (int i = 0; i < qd.nev; ++i) {
    double f, g;
    qd_fermi((qd.E[i] - EF - dphi) * ik, f, g);
    s += w[i] * f;
    ds += w[i] * g;
  }
  n = s;
  dn = ds * ik;
}

// ---------------------------------------------------------------------------
// Gauss-point interpolation on the reference element: the 1D matrix
// B[node][qp] = [[a, b], [b, a]], a = (1 + 1/sqrt3)/2, b = (1 - 1/sqrt3)/2,
// applied along x, y, z. B is symmetric, so the same routine maps corner
// values to quadrature points and quadrature-point values back to corners.
// Corner / qp index: ix + 2 iy + 4 iz.
template <class T>
__device__ __forceinline__ void tp_apply(const T* in, T* out, T a, T b) {
  T t[8], u[8];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    t[2 * p] = a * in[2 * p] + b * in[2 * p + 1];
    t[2 * p + 1] = b * in[2 * p] + a * in[2 * p + 1];
  }
#pragma unroll
  for (int z = 0; z < 2; ++z) {
#pragma unroll
    for (int x = 0; x < 2; ++x) {
      const int i0 = x + 4 * z, i1 = i0 + 2;
      u[i0] = a * t[i0] + b * t[i1];
      u[i1] = b * t[i0] + a * t[i1];
    }
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    out[p] = a * u[p] + b * u[p + 4];
    out[p + 4] = b * u[p] + a * u[p + 4];
  }
}

template <class T> struct GaussConst;
template <> struct GaussConst<double> {
  static __device__ __forceinline__ double a() { return 0.78867513459481288225; }
  static __device__ __forceinline__ double b() { return 0.21132486540518711775; }
};
template <> struct GaussConst<float> {
  static __device__ __forceinline__ float a() { return 0.78867513459481288225f; }
  static __device__ __forceinline__ float b() { return 0.21132486540518711775f; }
};

// Element mass-like operator: out = B (c o (B v)), c at the 8 quadrature points
// (weights and Jacobian already folded into c).
template <class T>
__device__ __forceinline__ void qp_mass(const T* v, const T* c, T* out) {
  T u[8];
  tp_apply(v, u, GaussConst<T>::a(), GaussConst<T>::b());
#pragma unroll
  for (int q = 0; q < 8; ++q) u[q] *= c[q];
  tp_apply(u, out, GaussConst<T>::a(), GaussConst<T>::b());
}

// The 8 quadrature coefficients of element e (vector loads; arrays are 16-byte aligned).
template <class T>
__device__ __forceinline__ void load_c8(const T* c, long long e, T* out);
template <>
__device__ __forceinline__ void load_c8<float>(const float* c, long long e, float* out) {
  const float4* p = reinterpret_cast<const float4*>(c + 8 * e);
  const float4 a = __ldg(p), b = __ldg(p + 1);
  out[0] = a.x; out[1] = a.y; out[2] = a.z; out[3] = a.w;
  out[4] = b.x; out[5] = b.y; out[6] = b.z; out[7] = b.w;
}
template <>
__device__ __forceinline__ void load_c8<double>(const double* c, long long e, double* out) {
  const double2* p = reinterpret_cast<const double2*>(c + 8 * e);
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const double2 a = __ldg(p + s);
    out[2 * s] = a.x;
    out[2 * s + 1] = a.y;
  }
}

// ---------------------------------------------------------------------------
// Block reductions (double accumulation).
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL_MASK, v, o));
  return v;
}

// Sums NS values over the block and adds them atomically to dst[0..NS).
template <int NS>
__device__ __forceinline__ void block_sum_atomic(double (&v)[NS], double* dst) {
  __shared__ double red[NS][32];
  const int lane = (threadIdx.x + blockDim.x * threadIdx.y) & 31;
  const int warp = (threadIdx.x + blockDim.x * threadIdx.y) >> 5;
  const int nwarps = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double w = warp_sum(v[s]);
    if (lane == 0) red[s][warp] = w;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double w = lane < nwarps ? red[s][lane] : 0.0;
      w = warp_sum(w);
      if (lane == 0 && w != 0.0) atomicAdd(dst + s, w);
    }
  }
  __syncthreads();
}

// Max of non-negative doubles via the ordering of their bit patterns.
__device__ __forceinline__ void atomic_max_nonneg(double* dst, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(dst), (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ void block_max_atomic(double v, double* dst) {
  __shared__ double red[32];
  const int lane = (threadIdx.x + blockDim.x * threadIdx.y) & 31;
  const int warp = (threadIdx.x + blockDim.x * threadIdx.y) >> 5;
  const int nwarps = (blockDim.x * blockDim.y + 31) >> 5;
  double w = warp_max(v);
  if (lane == 0) red[warp] = w;
  __syncthreads();
  if (warp == 0) {
    w = lane < nwarps ? red[lane] : 0.0;
    w = warp_max(w);
    if (lane == 0 && w > 0.0) atomic_max_nonneg(dst, w);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// z-marching tile skeleton.
//
// A block of 32 x BY threads owns the node tile (i, j) = (bx*30 - 1 + tx,
// by*(BY-2) - 1 + ty): the outer ring of threads is a one-node halo, so tiles
// overlap by two nodes and every interior thread of the tile writes its node.
// The block walks node planes k0 .. k1-1 (a z chunk). For node plane k it
// holds planes k-1, k, k+1 of the input in a shared ring, computes the
// element layer k (between planes k and k+1) once per element, and gathers
// element corner outputs to nodes: along x with warp shuffles (a warp is one
// tile row), along y through shared memory, along z by carrying the upper
// corner sums of layer k to plane k+1 in registers. The stiffness part is
// applied in three separable stages: z from the ring, y through shared
// memory, x by shuffles.
//
// The march is software-pipelined: the input of plane k+2 and the element
// data of layer k+1 are loaded into registers while layer k is computed, so
// global-load latency overlaps the arithmetic and the barriers.
//
// Op supplies:
//   NF                      number of gathered fields (field 0 gets the stencil)
//   STIFF                   whether field 0 includes the stiffness stencil
//   ED                      per-element data loaded from memory (coefficients)
//   T load(g, n, in, i, j, k)           input value at node n (0 when !in)
//   ED edata(g, i, j, k)                element data of element (i, j, k)
//   void elem(g, i, j, k, v[8], ed, out[NF][8], own)  element corner outputs; own is
//                           true in exactly one thread per element (per-element reductions)
//   void node(g, n, i, j, k, vin, stiff, mass[NF])  writer epilogue
//   void finish()                       block-level epilogue (all threads)
//   bool skip()                         uniform early exit (all threads)
//   void set_vec(int)                   vector index of this block (block applies)
// The Op is copied per thread, so its data members double as per-thread
// accumulators (constructed zeroed on the host). Node and element indices are
// 32-bit; mesh creation rejects meshes whose 8*n_elems or n_nodes exceed 2^31.
// Body of the skeleton for tile (bx, by) and (vector, z chunk) index bz; called by
// march_kernel with the block index and by the batched kernels with a tile from a work table.
// FACE: the charged gates' face term (face_alpha) is added to the stiffness of the top plane.
template <class T, int BY, class Op, bool FACE = false>
__device__ __forceinline__ void march_body(const Grid<T>& g, const Op& op_in, int kchunk, int bx, int by, int bz,
                                           const T* face_alpha = nullptr) {
  constexpr int BX = QCAD_BX;
  constexpr int NF = Op::NF;
  using ED = typename Op::ED;
  if (op_in.skip()) return;
  // bz enumerates (vector, z chunk) pairs
  const int nch = (g.nzn + kchunk - 1) / kchunk;
  Op op = op_in;
  op.set_vec(bz / nch);
  __shared__ T ring[4][BY][BX];
  __shared__ T s1[NF][BY][BX];
  __shared__ T s2[NF][BY][BX];
  __shared__ T sax[BY][BX];
  __shared__ T say[BY][BX];
  __shared__ T sb[BY][BX];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = bx * (BX - 2) - 1 + tx;
  const int j = by * (BY - 2) - 1 + ty;
  const int k0 = (bz % nch) * kchunk;
  const int k1 = min(k0 + kchunk, g.nzn);
  const int plane = (int)g.plane;
  const bool nin = (i >= 0 && i < g.nxn && j >= 0 && j < g.nyn);
  const bool writer = nin && tx >= 1 && tx < BX - 1 && ty >= 1 && ty < BY - 1;
  const bool eij = (i >= 0 && i < g.nx && j >= 0 && j < g.ny) && tx < BX - 1 && ty < BY - 1;
  const bool own_ij = tx >= 1 && ty >= 1;
  const int txp = min(tx + 1, BX - 1), typ = min(ty + 1, BY - 1), tym = max(ty - 1, 0);
  T cmx[3] = {0, 0, 0}, ckx[3] = {0, 0, 0}, cmy[3] = {0, 0, 0}, cky[3] = {0, 0, 0};
  if (nin) {
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      cmx[s] = g.mx[3 * i + s];
      ckx[s] = g.kx[3 * i + s];
      cmy[s] = g.my[3 * j + s];
      cky[s] = g.ky[3 * j + s];
    }
  }
  const int nij = nin ? i + g.nxn * j : 0;
  T carry[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) carry[f] = T(0);

  if (k0 > 0) ring[(k0 - 1) & 3][ty][tx] = op.load(g, nij + (k0 - 1) * plane, nin, i, j, k0 - 1);
  ring[k0 & 3][ty][tx] = op.load(g, nij + k0 * plane, nin, i, j, k0);
  // first prefetch: input plane k0+1 and element data of layer k0
  T vnext = (k0 + 1 < g.nzn) ? op.load(g, nij + (k0 + 1) * plane, nin, i, j, k0 + 1) : T(0);
  ED ednext{};
  if (eij && k0 < g.nz) ednext = op.edata(g, i, j, k0);
  __syncthreads();
  if (k0 > 0) {
    // upper corners of element layer k0-1 feed node plane k0
    T out[NF][8];
    const int k = k0 - 1;
    if (eij) {
      T v[8];
      v[0] = ring[k & 3][ty][tx];
      v[1] = ring[k & 3][ty][txp];
      v[2] = ring[k & 3][typ][tx];
      v[3] = ring[k & 3][typ][txp];
      v[4] = ring[k0 & 3][ty][tx];
      v[5] = ring[k0 & 3][ty][txp];
      v[6] = ring[k0 & 3][typ][tx];
      v[7] = ring[k0 & 3][typ][txp];
      const ED ed = op.edata(g, i, j, k);
      op.elem(g, i, j, k, v, ed, out, false);
    } else {
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int a = 0; a < 8; ++a) out[f][a] = T(0);
    }
    T hy0[NF], hy1[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      hy0[f] = out[f][4] + __shfl_up_sync(FULL_MASK, out[f][5], 1);
      hy1[f] = out[f][6] + __shfl_up_sync(FULL_MASK, out[f][7], 1);
      s2[f][ty][tx] = hy1[f];
    }
    __syncthreads();
#pragma unroll
    for (int f = 0; f < NF; ++f) carry[f] = hy0[f] + (ty > 0 ? s2[f][ty - 1][tx] : T(0));
  }

  for (int k = k0; k < k1; ++k) {
    const int kp = k + 1;
    ring[kp & 3][ty][tx] = vnext;
    const ED ed = ednext;
    if (k + 1 < k1) {
      // issue the next iteration's loads before this iteration's arithmetic
      vnext = (k + 2 < g.nzn) ? op.load(g, nij + (k + 2) * plane, nin, i, j, k + 2) : T(0);
      if (eij && k + 1 < g.nz) ednext = op.edata(g, i, j, k + 1);
    }
    __syncthreads();
    T out[NF][8];
    if (eij && k < g.nz) {
      T v[8];
      v[0] = ring[k & 3][ty][tx];
      v[1] = ring[k & 3][ty][txp];
      v[2] = ring[k & 3][typ][tx];
      v[3] = ring[k & 3][typ][txp];
      v[4] = ring[kp & 3][ty][tx];
      v[5] = ring[kp & 3][ty][txp];
      v[6] = ring[kp & 3][typ][tx];
      v[7] = ring[kp & 3][typ][txp];
      op.elem(g, i, j, k, v, ed, out, own_ij);
    } else {
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int a = 0; a < 8; ++a) out[f][a] = T(0);
    }
    T ly0[NF], hy0[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      ly0[f] = out[f][0] + __shfl_up_sync(FULL_MASK, out[f][1], 1);
      const T ly1 = out[f][2] + __shfl_up_sync(FULL_MASK, out[f][3], 1);
      hy0[f] = out[f][4] + __shfl_up_sync(FULL_MASK, out[f][5], 1);
      const T hy1 = out[f][6] + __shfl_up_sync(FULL_MASK, out[f][7], 1);
      s1[f][ty][tx] = ly1;
      s2[f][ty][tx] = hy1;
    }
    const T vc = ring[k & 3][ty][tx];
    T ax = 0, ay = 0, bz = 0;
    if (Op::STIFF) {
      const T vm = (k > 0) ? ring[(k - 1) & 3][ty][tx] : T(0);
      const T vp = ring[kp & 3][ty][tx];
      const T* zx = g.mzx + 3 * k;
      const T* zy = g.mzy + 3 * k;
      const T* zz = g.kzz + 3 * k;
      ax = zx[0] * vm + zx[1] * vc + zx[2] * vp;
      ay = zy[0] * vm + zy[1] * vc + zy[2] * vp;
      bz = zz[0] * vm + zz[1] * vc + zz[2] * vp;
      sax[ty][tx] = ax;
      say[ty][tx] = ay;
      sb[ty][tx] = bz;
    }
    __syncthreads();
    T mass[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      mass[f] = ly0[f] + (ty > 0 ? s1[f][ty - 1][tx] : T(0)) + carry[f];
      carry[f] = hy0[f] + (ty > 0 ? s2[f][ty - 1][tx] : T(0));
    }
    T stiff = 0;
    if (Op::STIFF) {
      const T c1 = cmy[0] * sax[tym][tx] + cmy[1] * ax + cmy[2] * sax[typ][tx];
      const T c2 = cky[0] * say[tym][tx] + cky[1] * ay + cky[2] * say[typ][tx];
      const T c3 = cmy[0] * sb[tym][tx] + cmy[1] * bz + cmy[2] * sb[typ][tx];
      const T d = c2 + c3;
      const T c1m = __shfl_up_sync(FULL_MASK, c1, 1);
      const T c1p = __shfl_down_sync(FULL_MASK, c1, 1);
      const T dm = __shfl_up_sync(FULL_MASK, d, 1);
      const T dp = __shfl_down_sync(FULL_MASK, d, 1);
      stiff = ckx[0] * c1m + ckx[1] * c1 + ckx[2] * c1p + cmx[0] * dm + cmx[1] * d + cmx[2] * dp;
      // charged gates: the Robin face mass on the top plane, from the ring's 3x3 neighbourhood
      // (a writer's neighbours are inside its tile)
      if constexpr (FACE) {
        if (k == g.nz && writer)
          stiff += face_row(g, face_alpha, i, j, [&](int dx, int dy) { return ring[k & 3][ty + dy][tx + dx]; });
      }
    }
    if (writer) op.node(g, nij + k * plane, i, j, k, vc, stiff, mass);
  }
  op.finish();
}

template <class T, int BY, class Op>
__global__ void __launch_bounds__(QCAD_BX * BY)
march_kernel(const Grid<T> g, const Op op_in, int kchunk) {
  march_body<T, BY, Op>(g, op_in, kchunk, blockIdx.x, blockIdx.y, blockIdx.z);
}

// The skeleton with the charged gates' face term (alpha: [nx*ny] face coefficients).
template <class T, int BY, class Op>
__global__ void __launch_bounds__(QCAD_BX * BY)
march_face_kernel(const Grid<T> g, const Op op_in, int kchunk, const T* alpha) {
  march_body<T, BY, Op, true>(g, op_in, kchunk, blockIdx.x, blockIdx.y, blockIdx.z, alpha);
}

// Launch geometry of the skeleton for a grid (nvec vectors along blockIdx.z).
inline dim3 march_grid(int nxn, int nyn, int nzn, int by, int kchunk, int nvec = 1) {
  return dim3((nxn + QCAD_BX - 3) / (QCAD_BX - 2), (nyn + by - 3) / (by - 2),
              ((nzn + kchunk - 1) / kchunk) * nvec);
}

// Eight quadrature coefficients of one element.
template <class T>
struct C8 {
  T c[8];
};

}  // namespace qcad
