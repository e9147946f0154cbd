// Geometric multigrid V-cycle preconditioner (see mg.h): hierarchy construction, Galerkin
// setup per linearization (FP32 or FP64), and the V-cycle kernels of the coarse levels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <deque>
#include <memory>
#include <vector>

#include "mesh.h"
#include "mg.h"
#include "pcg_ops.cuh"

namespace qcad {

namespace {

constexpr int MG_THREADS = 256;

// Host side of one level: geometry and transfers shared by both precisions, operator and
// vectors per precision (index 0 FP64, 1 FP32, the mesh's linearization-version index).
struct MgLevel {
  int nx = 0, ny = 0, nz = 0;
  long long n = 0, ne = 0;
  std::vector<double> xs[3];  // node coordinates along x, y, z
  DevBuf mask;
  DevBuf A[2], dinv[2], b[2], x[2], w[2];
  DevBuf em[3], pr[3], rs[3], ch[3];  // transfers to the next coarser level
  MgLevelDev<double> d64{};
  MgLevelDev<float> d32{};
};

template <class T> constexpr int prec_index() { return sizeof(T) == 8 ? 0 : 1; }
template <class T> MgLevelDev<T>& level_dev(MgLevel& l);
template <> MgLevelDev<double>& level_dev<double>(MgLevel& l) { return l.d64; }
template <> MgLevelDev<float>& level_dev<float>(MgLevel& l) { return l.d32; }

struct MgHier {
  std::deque<MgLevel> L;  // a deque: levels are created in place and never move
  DevBuf par[2];          // per level: Gershgorin bound hi of D^-1 J (in the precision's type)
  bool ok = false;
  bool alloc[2] = {false, false};  // the precision's operators and vectors exist
  long long lin_ver[2] = {-1, -1}; // linearization the operators were built for
  // The stiffness-only parts, built once per precision (the stiffness and the Dirichlet masks do
  // not change between linearizations): level-1 element matrices P^T K P (64 per coarse element)
  // and the level-0 Gershgorin row sums sum_j |K_ij| (per node). Where every coefficient c of the
  // elements involved is zero (no charge response) the operator is the stiffness alone, and the
  // setup copies these instead of rebuilding them.
  DevBuf S1[2], ra0[2];
  bool stiff_ok[2] = {false, false};
};

MgHier* hier(qcad_mesh_s* m) { return static_cast<MgHier*>(m->mg.get()); }

// Coarsening of one axis with node coordinates xf (n_e = xf.size() - 1 elements): the coarse
// nodes are the even fine nodes plus the last one; an axis with one element is kept.
struct AxisMap {
  std::vector<int> cidx;  // fine index of each coarse node
  std::vector<MgElemMap> em;
  std::vector<MgProl> pr;
  std::vector<MgRestr> rs;
  std::vector<MgChild> ch;
  std::vector<double> xc;
};

AxisMap coarsen_axis(const std::vector<double>& xf) {
  AxisMap a;
  const int ne = (int)xf.size() - 1;
  if (ne >= 2) {
    for (int f = 0; f <= ne; f += 2) a.cidx.push_back(f);
    if (a.cidx.back() != ne) a.cidx.push_back(ne);
  } else {
    for (int f = 0; f <= ne; ++f) a.cidx.push_back(f);
  }
  const int nc = (int)a.cidx.size();
  for (int C = 0; C < nc; ++C) a.xc.push_back(xf[a.cidx[C]]);
  // coarse interval of each fine element and of each fine node
  std::vector<int> interval(ne);
  for (int C = 0; C + 1 < nc; ++C)
    for (int i = a.cidx[C]; i < a.cidx[C + 1]; ++i) interval[i] = C;
  a.ch.resize(nc - 1);
  for (int C = 0; C + 1 < nc; ++C) a.ch[C] = MgChild{a.cidx[C], a.cidx[C + 1] - a.cidx[C]};
  a.em.resize(ne);
  for (int i = 0; i < ne; ++i) {
    const int E = interval[i];
    const double X0 = a.xc[E], X1 = a.xc[E + 1];
    const double t0 = (xf[i] - X0) / (X1 - X0), t1 = (xf[i + 1] - X0) / (X1 - X0);
    a.em[i] = MgElemMap{E, (float)(1.0 - t0), (float)t0, (float)(1.0 - t1), (float)t1};
  }
  a.pr.resize(ne + 1);
  std::vector<int> coarse_of(ne + 1, -1);
  for (int C = 0; C < nc; ++C) coarse_of[a.cidx[C]] = C;
  for (int f = 0; f <= ne; ++f) {
    if (coarse_of[f] >= 0) {
      a.pr[f] = MgProl{coarse_of[f], coarse_of[f], 1.0f, 0.0f};
    } else {
      const int C0 = interval[f];  // f lies strictly inside coarse interval C0
      const double t = (xf[f] - a.xc[C0]) / (a.xc[C0 + 1] - a.xc[C0]);
      a.pr[f] = MgProl{C0, C0 + 1, (float)(1.0 - t), (float)t};
    }
  }
  a.rs.resize(nc);
  for (int C = 0; C < nc; ++C) {
    const int f0 = a.cidx[C];
    MgRestr r{f0, f0, f0, 1.0f, 0.0f, 0.0f};
    if (f0 - 1 >= 0 && coarse_of[f0 - 1] < 0 && a.pr[f0 - 1].c1 == C) {
      r.f1 = f0 - 1;
      r.w1 = a.pr[f0 - 1].w1;
    }
    if (f0 + 1 <= ne && coarse_of[f0 + 1] < 0 && a.pr[f0 + 1].c0 == C) {
      r.f2 = f0 + 1;
      r.w2 = a.pr[f0 + 1].w0;
    }
    a.rs[C] = r;
  }
  return a;
}

template <class T>
void upload_vec(DevBuf& b, const std::vector<T>& v, cudaStream_t s) {
  b.ensure(v.size() * sizeof(T) + 64);
  CK(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
}

int blocks_for(long long n, int threads = MG_THREADS) {
  return (int)std::max<long long>(1, (n + threads - 1) / threads);
}

}  // namespace

// ---------------------------------------------------------------------------
// Kernels: masks and Galerkin setup.

template <class T>
__device__ __forceinline__ void node_ijk(const MgLevelDev<T>& L, long long n, int& i, int& j, int& k) {
  i = (int)(n % L.nxn);
  const long long r = n / L.nxn;
  j = (int)(r % L.nyn);
  k = (int)(r / L.nyn);
}

__global__ void mg_mask0_kernel(const Grid<float> g, unsigned char* mask) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nn = (long long)g.nxn * g.nyn * g.nzn;
  if (n >= nn) return;
  const int i = (int)(n % g.nxn);
  const long long r = n / g.nxn;
  const int j = (int)(r % g.nyn), k = (int)(r / g.nyn);
  mask[n] = grid_is_dir(g, i, j, k) ? 1 : 0;
}

// Coarse node Dirichlet iff its coincident fine node is.
__global__ void mg_mask_coarsen_kernel(const MgLevelDev<float> F, const MgLevelDev<float> C, unsigned char* cmask) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nn = (long long)C.nxn * C.nyn * C.nzn;
  if (n >= nn) return;
  int I, J, K;
  node_ijk(C, n, I, J, K);
  const long long f = F.rs[0][I].f0 + (long long)F.nxn * (F.rs[1][J].f0 + (long long)F.nyn * F.rs[2][K].f0);
  cmask[n] = F.mask[f];
}

// Row `a` of a fine element matrix P-transformed from the right, accumulated into the coarse
// element matrix: AE[R][C] += P[a][R] (row_a P)[C], with P = px (x) py (x) pz (2 x 2 factors,
// [fine corner][coarse corner]).
template <class T>
__device__ __forceinline__ void mg_accum_row(T (&AE)[64], const T (&row)[8], int a, const T (&px)[4],
                                             const T (&py)[4], const T (&pz)[4]) {
  T u[8], t[8];
  // right multiplication by P, one axis at a time: t[C] = sum_b row[b] P[b][C]
#pragma unroll
  for (int yz = 0; yz < 4; ++yz) {
    const T r0 = row[2 * yz], r1 = row[2 * yz + 1];
    u[2 * yz] = r0 * px[0] + r1 * px[2];
    u[2 * yz + 1] = r0 * px[1] + r1 * px[3];
  }
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int x = 0; x < 2; ++x) {
      const T r0 = u[x + 4 * z], r1 = u[x + 2 + 4 * z];
      t[x + 4 * z] = r0 * py[0] + r1 * py[2];
      t[x + 2 + 4 * z] = r0 * py[1] + r1 * py[3];
    }
#pragma unroll
  for (int xy = 0; xy < 4; ++xy) {
    const T r0 = t[xy], r1 = t[xy + 4];
    u[xy] = r0 * pz[0] + r1 * pz[2];
    u[xy + 4] = r0 * pz[1] + r1 * pz[3];
  }
  // P[a][R] factors by selection (a is a runtime index; indexing the arrays with it would
  // move them to local memory)
  const bool ax = a & 1, ay = (a >> 1) & 1, az = a >> 2;
  const T qx[2] = {ax ? px[2] : px[0], ax ? px[3] : px[1]};
  const T qy[2] = {ay ? py[2] : py[0], ay ? py[3] : py[1]};
  const T qz[2] = {az ? pz[2] : pz[0], az ? pz[3] : pz[1]};
#pragma unroll
  for (int R = 0; R < 8; ++R) {
    const T pa = qx[R & 1] * qy[(R >> 1) & 1] * qz[R >> 2];
#pragma unroll
    for (int C = 0; C < 8; ++C) AE[8 * R + C] += pa * u[C];
  }
}

__device__ __forceinline__ void store4(float* o, const float (&v)[4]) {
  *reinterpret_cast<float4*>(o) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store4(double* o, const double (&v)[4]) {
  reinterpret_cast<double2*>(o)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(o)[1] = make_double2(v[2], v[3]);
}

template <class T>
__device__ __forceinline__ void mg_store_masked(const MgLevelDev<T>& Cl, int I, int J, int K, T (&AE)[64], T* out) {
  bool dm[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const long long nd = (I + (c & 1)) + (long long)Cl.nxn * ((J + ((c >> 1) & 1)) + (long long)Cl.nyn * (K + (c >> 2)));
    dm[c] = Cl.mask[nd] != 0;
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    T v[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int R = (4 * q + s) >> 3, C = (4 * q + s) & 7;
      v[s] = (dm[R] || dm[C]) ? T(0) : AE[4 * q + s];
    }
    store4(out + 4 * q, v);
  }
}

// Row a of the fine-mesh element matrix of element (i, j, k) (stiffness from the 1D element
// matrices, mass term from the 8 quadrature coefficients c), with the columns of Dirichlet
// corners zeroed.
template <class T>
__device__ __forceinline__ void mg_fine_row(const Grid<T>& g, int i, int j, int k, const T (&c)[8],
                                            const bool (&dm)[8], int a, T (&row)[8]) {
  const T mxo = g.mx[3 * i + 2], kxo = g.kx[3 * i + 2];
  const T myo = g.my[3 * j + 2], kyo = g.ky[3 * j + 2];
  const T mzxo = g.mzx[3 * k + 2], mzyo = g.mzy[3 * k + 2], kzo = g.kzz[3 * k + 2];
  const int ax = a & 1, ay = (a >> 1) & 1, az = a >> 2;
  const T GA = GaussConst<T>::a(), GB = GaussConst<T>::b();
  T u[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const T bq = ((q & 1) == ax ? GA : GB) * (((q >> 1) & 1) == ay ? GA : GB) * ((q >> 2) == az ? GA : GB);
    u[q] = c[q] * bq;
  }
  T mrow[8];
  tp_apply<T>(u, mrow, GA, GB);
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const int bx = b & 1, by = (b >> 1) & 1, bz = b >> 2;
    const T Mx = (bx == ax ? T(2) : T(1)) * mxo, Kx = (bx == ax ? -kxo : kxo);
    const T My = (by == ay ? T(2) : T(1)) * myo, Ky = (by == ay ? -kyo : kyo);
    const T Mzx = (bz == az ? T(2) : T(1)) * mzxo, Mzy = (bz == az ? T(2) : T(1)) * mzyo;
    const T Kz = (bz == az ? -kzo : kzo);
    const T v = Kx * My * Mzx + Mx * Ky * Mzy + Mx * My * Kz + mrow[b];
    row[b] = dm[b] ? T(0) : v;
  }
}

// All eight coefficients of element e zero (no charge response).
template <class T>
__device__ __forceinline__ bool mg_coef_zero(const T* __restrict__ coef, long long e) {
  T c[8];
  load_c8<T>(coef, e, c);
  bool z = true;
#pragma unroll
  for (int q = 0; q < 8; ++q) z = z && c[q] == T(0);
  return z;
}

// Level-1 element matrices from the mesh operator (coefficients c, 8 per element). STIFF: the
// stiffness-only matrices (c taken as zero, coef unused), stored once as S1. Otherwise a coarse
// element whose children all have zero coefficients copies its S1 matrix (the same values the
// rebuild would give), and the others are rebuilt.
template <class T, bool STIFF>
__global__ void __launch_bounds__(128) mg_galerkin0_kernel(const Grid<T> g, const T* __restrict__ coef,
                                                           const T* __restrict__ S1, const MgLevelDev<T> F,
                                                           const MgLevelDev<T> Cl, T* Aout) {
  const long long E = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long ne = (long long)Cl.nx * Cl.ny * Cl.nz;
  if (E >= ne) return;
  const int I = (int)(E % Cl.nx);
  const long long r = E / Cl.nx;
  const int J = (int)(r % Cl.ny), K = (int)(r / Cl.ny);
  const MgChild cx = F.ch[0][I], cy = F.ch[1][J], cz = F.ch[2][K];
  if (!STIFF) {
    bool zero = true;
    for (int k = cz.first; k < cz.first + cz.count; ++k)
      for (int j = cy.first; j < cy.first + cy.count; ++j)
        for (int i = cx.first; i < cx.first + cx.count; ++i)
          zero = zero && mg_coef_zero<T>(coef, i + (long long)g.nx * (j + (long long)g.ny * k));
    if (zero) {
      const uint4* src = reinterpret_cast<const uint4*>(S1 + 64 * E);
      uint4* dst = reinterpret_cast<uint4*>(Aout + 64 * E);
#pragma unroll
      for (int q = 0; q < (int)(64 * sizeof(T) / 16); ++q) dst[q] = __ldg(src + q);
      return;
    }
  }
  T AE[64];
#pragma unroll
  for (int q = 0; q < 64; ++q) AE[q] = T(0);
  for (int k = cz.first; k < cz.first + cz.count; ++k)
    for (int j = cy.first; j < cy.first + cy.count; ++j)
      for (int i = cx.first; i < cx.first + cx.count; ++i) {
        const MgElemMap ex = F.em[0][i], ey = F.em[1][j], ez = F.em[2][k];
        const T px[4] = {(T)ex.p00, (T)ex.p01, (T)ex.p10, (T)ex.p11};
        const T py[4] = {(T)ey.p00, (T)ey.p01, (T)ey.p10, (T)ey.p11};
        const T pz[4] = {(T)ez.p00, (T)ez.p01, (T)ez.p10, (T)ez.p11};
        T c[8];
        if (STIFF) {
#pragma unroll
          for (int q = 0; q < 8; ++q) c[q] = T(0);
        } else {
          load_c8<T>(coef, i + (long long)g.nx * (j + (long long)g.ny * k), c);
        }
        bool dm[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
          dm[q] = F.mask[(i + (q & 1)) + (long long)F.nxn * ((j + ((q >> 1) & 1)) + (long long)F.nyn * (k + (q >> 2)))] != 0;
        for (int a = 0; a < 8; ++a) {
          if (dm[a]) continue;
          T row[8];
          mg_fine_row<T>(g, i, j, k, c, dm, a, row);
          mg_accum_row<T>(AE, row, a, px, py, pz);
        }
      }
  mg_store_masked<T>(Cl, I, J, K, AE, Aout + 64 * E);
}

// Level l+1 element matrices from the stored level-l ones.
template <class T>
__global__ void __launch_bounds__(128) mg_galerkin_kernel(const MgLevelDev<T> F, const MgLevelDev<T> Cl, T* Aout) {
  const long long E = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long ne = (long long)Cl.nx * Cl.ny * Cl.nz;
  if (E >= ne) return;
  const int I = (int)(E % Cl.nx);
  const long long r = E / Cl.nx;
  const int J = (int)(r % Cl.ny), K = (int)(r / Cl.ny);
  T AE[64];
#pragma unroll
  for (int q = 0; q < 64; ++q) AE[q] = T(0);
  const MgChild cx = F.ch[0][I], cy = F.ch[1][J], cz = F.ch[2][K];
  for (int k = cz.first; k < cz.first + cz.count; ++k)
    for (int j = cy.first; j < cy.first + cy.count; ++j)
      for (int i = cx.first; i < cx.first + cx.count; ++i) {
        const MgElemMap ex = F.em[0][i], ey = F.em[1][j], ez = F.em[2][k];
        const T px[4] = {(T)ex.p00, (T)ex.p01, (T)ex.p10, (T)ex.p11};
        const T py[4] = {(T)ey.p00, (T)ey.p01, (T)ey.p10, (T)ey.p11};
        const T pz[4] = {(T)ez.p00, (T)ez.p01, (T)ez.p10, (T)ez.p11};
        const T* Ae = F.A + 64 * (i + (long long)F.nx * (j + (long long)F.ny * k));
        for (int a = 0; a < 8; ++a) {
          T row[8];
#pragma unroll
          for (int b = 0; b < 8; ++b) row[b] = __ldg(Ae + 8 * a + b);
          mg_accum_row<T>(AE, row, a, px, py, pz);
        }
      }
  mg_store_masked<T>(Cl, I, J, K, AE, Aout + 64 * E);
}

// For every element E of level L that contains node (i, j, k): f(row of the node in E's matrix,
// E's first corner node, the node's corner in E).
template <class T, class F>
__device__ __forceinline__ void mg_for_adjacent(const MgLevelDev<T>& L, int i, int j, int k, F&& f) {
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int ex = e & 1, ey = (e >> 1) & 1, ez = e >> 2;
    const int I = i - 1 + ex, J = j - 1 + ey, K = k - 1 + ez;
    if (I < 0 || J < 0 || K < 0 || I >= L.nx || J >= L.ny || K >= L.nz) continue;
    const int c = (1 - ex) + 2 * (1 - ey) + 4 * (1 - ez);  // this node's corner in E
    const long long E = I + (long long)L.nx * (J + (long long)L.ny * K);
    const long long n0 = I + (long long)L.nxn * (J + (long long)L.nyn * K);
    f(L.A + 64 * E + 8 * c, n0, c);
  }
}

__device__ __forceinline__ void load_row8(const float* row, float (&r)[8]) {
  const float4 r0 = __ldg(reinterpret_cast<const float4*>(row)), r1 = __ldg(reinterpret_cast<const float4*>(row) + 1);
  r[0] = r0.x, r[1] = r0.y, r[2] = r0.z, r[3] = r0.w, r[4] = r1.x, r[5] = r1.y, r[6] = r1.z, r[7] = r1.w;
}
__device__ __forceinline__ void load_row8(const double* row, double (&r)[8]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(row) + q);
    r[2 * q] = v.x, r[2 * q + 1] = v.y;
  }
}

template <class T>
__device__ __forceinline__ T mg_row_dot(const MgLevelDev<T>& L, const T* row, long long n0, const T* x) {
  T r[8];
  load_row8(row, r);
  const long long sy = L.nxn, sz = (long long)L.nxn * L.nyn;
  return r[0] * x[n0] + r[1] * x[n0 + 1] + r[2] * x[n0 + sy] + r[3] * x[n0 + sy + 1] + r[4] * x[n0 + sz] +
         r[5] * x[n0 + sz + 1] + r[6] * x[n0 + sz + sy] + r[7] * x[n0 + sz + sy + 1];
}

// Maximum over the block of non-negative values, folded into *dst by an integer atomicMax on the
// bit pattern (non-negative IEEE values order like their bit patterns; the FP64 overload is in
// qcad_internal.cuh).
__device__ __forceinline__ void atomic_max_nonneg(float* dst, float v) {
  atomicMax(reinterpret_cast<int*>(dst), __float_as_int(v));
}

template <class T>
__device__ __forceinline__ void mg_block_max(T v, T* dst) {
  __shared__ T red[32];
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(FULL_MASK, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : T(0);
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(FULL_MASK, v, o));
    if (lane == 0 && v > T(0)) atomic_max_nonneg(dst, v);
  }
}

// Diagonal, D^-1 and the Gershgorin bound max_i sum_j |J_ij| / J_ii of a coarse level.
template <class T>
__global__ void mg_diag_kernel(const MgLevelDev<T> L, T* dinv, T* par_l) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nn = (long long)L.nxn * L.nyn * L.nzn;
  T ratio = T(0);
  if (n < nn) {
    int i, j, k;
    node_ijk(L, n, i, j, k);
    T dg = T(0), ra = T(0);
    mg_for_adjacent(L, i, j, k, [&](const T* row, long long, int c) {
      dg += row[c];
#pragma unroll
      for (int q = 0; q < 8; ++q) ra += fabs(row[q]);
    });
    const bool dir = L.mask[n] != 0 || !(dg > T(0));
    dinv[n] = dir ? T(0) : T(1) / dg;
    ratio = dir ? T(0) : ra / dg;
  }
  mg_block_max<T>(ratio, par_l);
}

// Gershgorin bound of D^-1 J on the mesh (rows of the element matrices rebuilt from the
// coefficients; Dirichlet rows are identity rows there, ratio 1). STIFF: the stiffness-only row
// sums sum_j |K_ij| into ra0 (c taken as zero). Otherwise a node whose adjacent elements all have
// zero coefficients takes its row sum from ra0 (the value the rebuild would give).
template <class T, bool STIFF>
__global__ void mg_gersh0_kernel(const Grid<T> g, const T* __restrict__ coef, const MgLevelDev<T> F,
                                 const T* dinv0, T* ra0, T* par0) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nn = (long long)F.nxn * F.nyn * F.nzn;
  T ratio = T(0);
  if (n < nn) {
    int i, j, k;
    node_ijk(F, n, i, j, k);
    if (F.mask[n]) {
      ratio = T(1);
      if (STIFF) ra0[n] = T(0);
    } else {
      bool zero = true;
      if (!STIFF) {
        for (int e = 0; e < 8; ++e) {
          const int I = i - 1 + (e & 1), J = j - 1 + ((e >> 1) & 1), K = k - 1 + (e >> 2);
          if (I < 0 || J < 0 || K < 0 || I >= F.nx || J >= F.ny || K >= F.nz) continue;
          zero = zero && mg_coef_zero<T>(coef, I + (long long)g.nx * (J + (long long)g.ny * K));
        }
      }
      T ra = T(0);
      if (!STIFF && zero) {
        ra = ra0[n];
      } else {
        for (int e = 0; e < 8; ++e) {
          const int ex = e & 1, ey = (e >> 1) & 1, ez = e >> 2;
          const int I = i - 1 + ex, J = j - 1 + ey, K = k - 1 + ez;
          if (I < 0 || J < 0 || K < 0 || I >= F.nx || J >= F.ny || K >= F.nz) continue;
          const int a = (1 - ex) + 2 * (1 - ey) + 4 * (1 - ez);
          T c[8];
          if (STIFF) {
#pragma unroll
            for (int q = 0; q < 8; ++q) c[q] = T(0);
          } else {
            load_c8<T>(coef, I + (long long)g.nx * (J + (long long)g.ny * K), c);
          }
          bool dm[8];
#pragma unroll
          for (int q = 0; q < 8; ++q)
            dm[q] = F.mask[(I + (q & 1)) + (long long)F.nxn * ((J + ((q >> 1) & 1)) + (long long)F.nyn * (K + (q >> 2)))] != 0;
          T row[8];
          mg_fine_row<T>(g, I, J, K, c, dm, a, row);
#pragma unroll
          for (int q = 0; q < 8; ++q) ra += fabs(row[q]);
        }
      }
      if (STIFF)
        ra0[n] = ra;
      else
        ratio = ra * dinv0[n];
    }
  }
  if (!STIFF) mg_block_max<T>(ratio, par0);
}

// ---------------------------------------------------------------------------
// V-cycle kernels. Every kernel returns at once when the PCG has finished (sc->done), so the
// iterations captured after convergence cost a launch each and nothing more.

// PCG start with the multigrid preconditioner: x = 0, r = b, ||r||^2, and the level-0
// pre-smoothing zp = omega D^-1 r (into d[0]).
template <class T>
__global__ void mg_pcg_init_kernel(int n, PcgVecs<T> v, PcgScalars* sc, const T* par) {
  const T om = mg_omega<T>(par, 0);
  T rr = T(0);
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    const T r = v.b[idx];
    v.x[idx] = T(0);
    v.r[idx] = r;
    v.d[0][idx] = om * v.dinv[idx] * r;
    rr += r * r;
  }
  double s1[1] = {(double)rr};
  block_sum_atomic<1>(s1, &sc->rr[0]);
}

// PCG update (alpha = rz / pAp): x += alpha p, r -= alpha Ap, ||r||^2, then zp = omega D^-1 r.
template <class T>
__global__ void mg_pcg_update_kernel(int n, PcgVecs<T> v, PcgScalars* sc, const T* par) {
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
  const T om = mg_omega<T>(par, 0);
  const T* __restrict__ p = (t & 1) ? v.p[1] : v.p[0];
  T rr = T(0);
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    v.x[idx] += alpha * p[idx];
    const T r = v.r[idx] - alpha * v.Ap[idx];
    v.r[idx] = r;
    v.d[0][idx] = om * v.dinv[idx] * r;
    rr += r * r;
  }
  double s1[1] = {(double)rr};
  block_sum_atomic<1>(s1, &sc->rr[(t + 1) & 3]);
}

// Restriction to level l+1 of the fine residual wf: b = P^T wf on the coarse free nodes, and
// the coarse pre-smoothing x = omega D^-1 b.
template <class T>
__global__ void mg_restrict_kernel(const MgLevelDev<T> F, const T* __restrict__ wf, const MgLevelDev<T> C,
                                   const T* par, int lc, const PcgScalars* sc) {
  if (sc->done) return;
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nn = (long long)C.nxn * C.nyn * C.nzn;
  if (n >= nn) return;
  int I, J, K;
  node_ijk(C, n, I, J, K);
  T b = T(0);
  if (!C.mask[n]) {
    const MgRestr rx = F.rs[0][I], ry = F.rs[1][J], rz = F.rs[2][K];
    const int fx[3] = {rx.f0, rx.f1, rx.f2}, fy[3] = {ry.f0, ry.f1, ry.f2}, fz[3] = {rz.f0, rz.f1, rz.f2};
    const T wx[3] = {(T)rx.w0, (T)rx.w1, (T)rx.w2}, wy[3] = {(T)ry.w0, (T)ry.w1, (T)ry.w2};
    const T wz[3] = {(T)rz.w0, (T)rz.w1, (T)rz.w2};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (wz[c] == T(0)) continue;
#pragma unroll
      for (int bb = 0; bb < 3; ++bb) {
        if (wy[bb] == T(0)) continue;
        const long long base = (long long)F.nxn * (fy[bb] + (long long)F.nyn * fz[c]);
        const T wyz = wy[bb] * wz[c];
        b += wyz * (wx[0] * wf[base + fx[0]] + wx[1] * wf[base + fx[1]] + wx[2] * wf[base + fx[2]]);
      }
    }
  }
  C.b[n] = b;
  C.x[n] = mg_omega<T>(par, lc) * C.dinv[n] * b;
}

// Residual after pre-smoothing on a coarse level: w = b - A x.
template <class T>
__global__ void mg_resid_kernel(const MgLevelDev<T> L, const PcgScalars* sc) {
  if (sc->done) return;
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nn = (long long)L.nxn * L.nyn * L.nzn;
  if (n >= nn) return;
  int i, j, k;
  node_ijk(L, n, i, j, k);
  T y = T(0);
  mg_for_adjacent(L, i, j, k, [&](const T* row, long long n0, int) { y += mg_row_dot<T>(L, row, n0, L.x); });
  L.w[n] = L.b[n] - y;
}

// Coarse correction of level l from the solution ec of level l+1: out = base + P ec on free
// nodes (base on Dirichlet nodes).
template <class T>
__global__ void mg_prolong_kernel(const MgLevelDev<T> F, const T* __restrict__ ec, const MgLevelDev<T> C,
                                  const T* base, T* out, const PcgScalars* sc) {
  if (sc->done) return;
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nn = (long long)F.nxn * F.nyn * F.nzn;
  if (n >= nn) return;
  T v = base[n];
  if (!F.mask[n]) {
    int i, j, k;
    node_ijk(F, n, i, j, k);
    const MgProl px = F.pr[0][i], py = F.pr[1][j], pz = F.pr[2][k];
    const long long sy = C.nxn, sz = (long long)C.nxn * C.nyn;
    const long long z0 = pz.c0 * sz, z1 = pz.c1 * sz, y0 = py.c0 * sy, y1 = py.c1 * sy;
    const T xw0 = px.w0, xw1 = px.w1, yw0 = py.w0, yw1 = py.w1, zw0 = pz.w0, zw1 = pz.w1;
    const T e00 = xw0 * ec[z0 + y0 + px.c0] + xw1 * ec[z0 + y0 + px.c1];
    const T e01 = xw0 * ec[z0 + y1 + px.c0] + xw1 * ec[z0 + y1 + px.c1];
    const T e10 = xw0 * ec[z1 + y0 + px.c0] + xw1 * ec[z1 + y0 + px.c1];
    const T e11 = xw0 * ec[z1 + y1 + px.c0] + xw1 * ec[z1 + y1 + px.c1];
    v += zw0 * (yw0 * e00 + yw1 * e01) + zw1 * (yw0 * e10 + yw1 * e11);
  }
  out[n] = v;
}

// Post-smoothing on a coarse level: w = x + omega D^-1 (b - A x) (the level's solution).
template <class T>
__global__ void mg_post_kernel(const MgLevelDev<T> L, const T* par, int l, const PcgScalars* sc) {
  if (sc->done) return;
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nn = (long long)L.nxn * L.nyn * L.nzn;
  if (n >= nn) return;
  int i, j, k;
  node_ijk(L, n, i, j, k);
  T y = T(0);
  mg_for_adjacent(L, i, j, k, [&](const T* row, long long n0, int) { y += mg_row_dot<T>(L, row, n0, L.x); });
  L.w[n] = L.x[n] + mg_omega<T>(par, l) * L.dinv[n] * (L.b[n] - y);
}

// Coarsest level: Chebyshev iteration of degree MG_COARSE_DEGREE for A x = b on
// [hi / 64, hi] inside one block of 1024 threads, with the element matrices and the vectors
// in shared memory; the result goes to w.
template <class T>
__global__ void __launch_bounds__(1024) mg_coarse_kernel(const MgLevelDev<T> L, const T* par, int l,
                                                         const PcgScalars* sc) {
  if (sc->done) return;
  extern __shared__ __align__(16) unsigned char mg_coarse_sh[];
  T* sh = reinterpret_cast<T*>(mg_coarse_sh);
  const int ne = L.nx * L.ny * L.nz;
  const int nn = L.nxn * L.nyn * L.nzn;
  T* sA = sh;               // 64 ne
  T* sd = sA + 64 * ne;     // direction
  T* sr = sd + nn;          // residual
  T* sx = sr + nn;          // solution
  for (int q = threadIdx.x; q < 64 * ne; q += blockDim.x) sA[q] = L.A[q];
  const T hi = par[l];
  const int n = threadIdx.x;  // one node per thread: the coarsest level has at most 512 nodes
  const bool own = n < nn;
  if (!(hi > T(0))) {
    if (own) L.w[n] = T(0);
    return;
  }
  const T lo = hi / T(64);
  const T theta = T(0.5) * (hi + lo), delta = T(0.5) * (hi - lo), sigma = theta / delta;
  const T dv = own ? L.dinv[n] : T(0);
  if (own) {
    const T r = L.b[n];
    const T d = dv * r / theta;
    sr[n] = r;
    sd[n] = d;
    sx[n] = d;
  }
  __syncthreads();
  int i = 0, j = 0, k = 0;
  const int sy = L.nxn, sz = L.nxn * L.nyn;
  if (own) {
    i = n % L.nxn;
    j = (n / L.nxn) % L.nyn;
    k = n / sz;
  }
  T rho = T(1) / sigma;
  for (int it = 1; it < MG_COARSE_DEGREE; ++it) {
    const T rho_new = T(1) / (T(2) * sigma - rho);
    const T c1 = rho_new * rho, c2 = T(2) * rho_new / delta;
    T y = T(0);
    if (own) {
      for (int e = 0; e < 8; ++e) {
        const int ex = e & 1, ey = (e >> 1) & 1, ez = e >> 2;
        const int I = i - 1 + ex, J = j - 1 + ey, K = k - 1 + ez;
        if (I < 0 || J < 0 || K < 0 || I >= L.nx || J >= L.ny || K >= L.nz) continue;
        const int c = (1 - ex) + 2 * (1 - ey) + 4 * (1 - ez);
        const T* row = sA + 64 * (I + L.nx * (J + L.ny * K)) + 8 * c;
        const int n0 = I + sy * (J + L.nyn * K);
        y += row[0] * sd[n0] + row[1] * sd[n0 + 1] + row[2] * sd[n0 + sy] + row[3] * sd[n0 + sy + 1] +
             row[4] * sd[n0 + sz] + row[5] * sd[n0 + sz + 1] + row[6] * sd[n0 + sz + sy] +
             row[7] * sd[n0 + sz + sy + 1];
      }
    }
    __syncthreads();
    if (own) {
      const T r = sr[n] - y;
      const T d = c1 * sd[n] + c2 * dv * r;
      sr[n] = r;
      sd[n] = d;
      sx[n] += d;
    }
    rho = rho_new;
    __syncthreads();
  }
  if (own) L.w[n] = sx[n];
}

// Prolongation into level 0: zq = zp + P e1 (d[1] from d[0]).
// (mg_prolong_kernel with base d[0] and out d[1].)

// ---------------------------------------------------------------------------
// Host.

// Shared memory of the coarsest solve in precision T.
static size_t coarse_smem_bytes(const MgLevel& co, size_t elem) { return ((size_t)64 * co.ne + 3 * (size_t)co.n) * elem; }
static constexpr size_t MG_COARSE_SMEM_MAX = 200 * 1024;

bool mg_prepare(qcad_mesh_s* m) {
  // charged gates: the hierarchy's level-0 kernels carry no Robin face term (Jacobi instead)
  if (m->has_robin) return false;
  if (m->mg) return hier(m)->ok;
  auto H = std::make_shared<MgHier>();
  m->mg = H;
  cudaStream_t s = m->stream;
  std::deque<MgLevel>& L = H->L;
  L.emplace_back();
  {
    MgLevel& l0 = L[0];
    l0.nx = m->nx;
    l0.ny = m->ny;
    l0.nz = m->nz;
    l0.xs[0] = m->xc;
    l0.xs[1] = m->yc;
    l0.xs[2] = m->zc;
  }
  for (;;) {
    MgLevel& f = L.back();
    f.n = (long long)(f.nx + 1) * (f.ny + 1) * (f.nz + 1);
    f.ne = (long long)f.nx * f.ny * f.nz;
    const bool can = f.nx >= 2 || f.ny >= 2 || f.nz >= 2;
    if (f.n <= MG_COARSE_NODES || !can || (int)L.size() >= MG_MAX_LEVELS) break;
    AxisMap ax[3] = {coarsen_axis(f.xs[0]), coarsen_axis(f.xs[1]), coarsen_axis(f.xs[2])};
    for (int a = 0; a < 3; ++a) {
      upload_vec(f.em[a], ax[a].em, s);
      upload_vec(f.pr[a], ax[a].pr, s);
      upload_vec(f.rs[a], ax[a].rs, s);
      upload_vec(f.ch[a], ax[a].ch, s);
    }
    L.emplace_back();
    MgLevel& c = L.back();
    c.nx = (int)ax[0].xc.size() - 1;
    c.ny = (int)ax[1].xc.size() - 1;
    c.nz = (int)ax[2].xc.size() - 1;
    for (int a = 0; a < 3; ++a) c.xs[a] = ax[a].xc;
  }
  const MgLevel& co = L.back();
  // usable when there is at least one coarse level and the coarsest fits one block's shared
  // memory in FP64 (so that both precisions can use the hierarchy)
  H->ok = L.size() >= 2 && co.n <= MG_COARSE_NODES && coarse_smem_bytes(co, sizeof(double)) <= MG_COARSE_SMEM_MAX;
  if (!H->ok) return false;
  for (size_t l = 0; l < L.size(); ++l) {
    MgLevel& v = L[l];
    v.mask.ensure((size_t)v.n + 64);
    MgLevelDev<float>& d = v.d32;
    d = MgLevelDev<float>{};
    d.nx = v.nx;
    d.ny = v.ny;
    d.nz = v.nz;
    d.nxn = v.nx + 1;
    d.nyn = v.ny + 1;
    d.nzn = v.nz + 1;
    d.mask = v.mask.as<unsigned char>();
    for (int a = 0; a < 3; ++a) {
      d.em[a] = v.em[a].as<MgElemMap>();
      d.pr[a] = v.pr[a].as<MgProl>();
      d.rs[a] = v.rs[a].as<MgRestr>();
      d.ch[a] = v.ch[a].as<MgChild>();
    }
    MgLevelDev<double>& e = v.d64;
    e = MgLevelDev<double>{};
    e.nx = d.nx, e.ny = d.ny, e.nz = d.nz, e.nxn = d.nxn, e.nyn = d.nyn, e.nzn = d.nzn;
    e.mask = d.mask;
    for (int a = 0; a < 3; ++a) e.em[a] = d.em[a], e.pr[a] = d.pr[a], e.rs[a] = d.rs[a], e.ch[a] = d.ch[a];
  }
  mg_mask0_kernel<<<blocks_for(L[0].n), MG_THREADS, 0, s>>>(m->g32.g, L[0].mask.as<unsigned char>());
  for (size_t l = 0; l + 1 < L.size(); ++l)
    mg_mask_coarsen_kernel<<<blocks_for(L[l + 1].n), MG_THREADS, 0, s>>>(L[l].d32, L[l + 1].d32,
                                                                          L[l + 1].mask.as<unsigned char>());
  // the largest coarsest level any mesh may have (checked above), so one setting serves all
  CK(cudaFuncSetAttribute(mg_coarse_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)MG_COARSE_SMEM_MAX));
  CK(cudaFuncSetAttribute(mg_coarse_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)MG_COARSE_SMEM_MAX));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return true;
}

// Operators and vectors of precision T on every coarse level (first use of that precision).
// Kernel arguments carry these pointers by value, so this runs before any V-cycle is captured.
template <class T>
static void mg_alloc(MgHier* H) {
  const int p = prec_index<T>();
  if (H->alloc[p]) return;
  std::deque<MgLevel>& L = H->L;
  for (size_t l = 1; l < L.size(); ++l) {
    MgLevel& v = L[l];
    v.A[p].ensure((size_t)64 * v.ne * sizeof(T) + 64);
    v.dinv[p].ensure((size_t)v.n * sizeof(T) + 64);
    v.b[p].ensure((size_t)v.n * sizeof(T) + 64);
    v.x[p].ensure((size_t)v.n * sizeof(T) + 64);
    v.w[p].ensure((size_t)v.n * sizeof(T) + 64);
    MgLevelDev<T>& d = level_dev<T>(v);
    d.A = v.A[p].template as<T>();
    d.dinv = v.dinv[p].template as<T>();
    d.b = v.b[p].template as<T>();
    d.x = v.x[p].template as<T>();
    d.w = v.w[p].template as<T>();
  }
  H->par[p].ensure(MG_MAX_LEVELS * sizeof(T) + 64);
  H->alloc[p] = true;
}

template <class T>
void mg_reserve(qcad_mesh_s* m) {
  mg_alloc<T>(hier(m));
}
template void mg_reserve<float>(qcad_mesh_s*);
template void mg_reserve<double>(qcad_mesh_s*);

void mg_invalidate(qcad_mesh_s* m) {
  if (m->mg) hier(m)->lin_ver[0] = hier(m)->lin_ver[1] = -1;
}

int mg_levels(qcad_mesh_s* m) { return (m->mg && hier(m)->ok) ? (int)hier(m)->L.size() : 0; }

template <class T> static const Grid<T>& mesh_grid(qcad_mesh_s* m);
template <> const Grid<double>& mesh_grid<double>(qcad_mesh_s* m) { return m->g64.g; }
template <> const Grid<float>& mesh_grid<float>(qcad_mesh_s* m) { return m->g32.g; }
template <class T> static PcgBufs<T>& mesh_bufs(qcad_mesh_s* m);
template <> PcgBufs<double>& mesh_bufs<double>(qcad_mesh_s* m) { return m->k64; }
template <> PcgBufs<float>& mesh_bufs<float>(qcad_mesh_s* m) { return m->k32; }
template <class T> static LaunchCfg mesh_cfg(qcad_mesh_s* m);
template <> LaunchCfg mesh_cfg<double>(qcad_mesh_s* m) { return m->cfg64; }
template <> LaunchCfg mesh_cfg<float>(qcad_mesh_s* m) { return m->cfg32; }

template <class T>
void mg_setup(qcad_mesh_s* m, cudaStream_t s, bool force) {
  MgHier* H = hier(m);
  const int p = prec_index<T>();
  mg_alloc<T>(H);
  if (!force && H->lin_ver[p] == m->lin_ver[p]) return;
  std::deque<MgLevel>& L = H->L;
  const PcgBufs<T>& k = mesh_bufs<T>(m);
  T* par = H->par[p].template as<T>();
  if (!H->stiff_ok[p]) {
    H->S1[p].ensure((size_t)64 * L[1].ne * sizeof(T) + 64);
    H->ra0[p].ensure((size_t)L[0].n * sizeof(T) + 64);
    mg_gersh0_kernel<T, true><<<blocks_for(L[0].n), MG_THREADS, 0, s>>>(
        mesh_grid<T>(m), nullptr, level_dev<T>(L[0]), k.dinv.template as<T>(), H->ra0[p].template as<T>(), nullptr);
    mg_galerkin0_kernel<T, true><<<blocks_for(L[1].ne, 128), 128, 0, s>>>(
        mesh_grid<T>(m), nullptr, nullptr, level_dev<T>(L[0]), level_dev<T>(L[1]), H->S1[p].template as<T>());
    note_launch(2);
    CK(cudaGetLastError());
    H->stiff_ok[p] = true;
  }
  CK(cudaMemsetAsync(par, 0, MG_MAX_LEVELS * sizeof(T), s));
  mg_gersh0_kernel<T, false><<<blocks_for(L[0].n), MG_THREADS, 0, s>>>(
      mesh_grid<T>(m), k.c.template as<T>(), level_dev<T>(L[0]), k.dinv.template as<T>(), H->ra0[p].template as<T>(),
      par);
  mg_galerkin0_kernel<T, false><<<blocks_for(L[1].ne, 128), 128, 0, s>>>(
      mesh_grid<T>(m), k.c.template as<T>(), H->S1[p].template as<T>(), level_dev<T>(L[0]), level_dev<T>(L[1]),
      L[1].A[p].template as<T>());
  for (size_t l = 1; l < L.size(); ++l) {
    if (l > 1)
      mg_galerkin_kernel<T><<<blocks_for(L[l].ne, 128), 128, 0, s>>>(level_dev<T>(L[l - 1]), level_dev<T>(L[l]),
                                                                     L[l].A[p].template as<T>());
    mg_diag_kernel<T><<<blocks_for(L[l].n), MG_THREADS, 0, s>>>(level_dev<T>(L[l]), L[l].dinv[p].template as<T>(),
                                                                par + l);
  }
  note_launch(2 + 2 * ((int)L.size() - 1) - 1);
  CK(cudaGetLastError());
  H->lin_ver[p] = m->lin_ver[p];
}
template void mg_setup<float>(qcad_mesh_s*, cudaStream_t, bool);
template void mg_setup<double>(qcad_mesh_s*, cudaStream_t, bool);

// V-cycle after the level-0 pre-smoothing (zp in d[0]): ends with z and the PCG bookkeeping.
template <class T>
static void enqueue_vcycle(qcad_mesh_s* m, const PcgVecs<T>& v, PcgScalars* sc, cudaStream_t s) {
  MgHier* H = hier(m);
  std::deque<MgLevel>& L = H->L;
  const int p = prec_index<T>();
  const T* par = H->par[p].template as<T>();
  const int nl = (int)L.size();
  launch_mg_resid0<T>(mesh_grid<T>(m), v, sc, mesh_cfg<T>(m), s);
  for (int l = 0; l + 1 < nl; ++l) {
    const T* wf = l == 0 ? v.w : L[l].w[p].template as<T>();
    note_launch(), mg_restrict_kernel<T><<<blocks_for(L[l + 1].n), MG_THREADS, 0, s>>>(
                       level_dev<T>(L[l]), wf, level_dev<T>(L[l + 1]), par, l + 1, sc);
    if (l + 1 < nl - 1)
      note_launch(), mg_resid_kernel<T><<<blocks_for(L[l + 1].n), MG_THREADS, 0, s>>>(level_dev<T>(L[l + 1]), sc);
  }
  const MgLevel& co = L[nl - 1];
  const int smem = (int)coarse_smem_bytes(co, sizeof(T));
  note_launch(), mg_coarse_kernel<T><<<1, 1024, smem, s>>>(level_dev<T>(L[nl - 1]), par, nl - 1, sc);
  for (int l = nl - 2; l >= 1; --l) {
    note_launch(), mg_prolong_kernel<T><<<blocks_for(L[l].n), MG_THREADS, 0, s>>>(
                       level_dev<T>(L[l]), L[l + 1].w[p].template as<T>(), level_dev<T>(L[l + 1]),
                       L[l].x[p].template as<T>(), L[l].x[p].template as<T>(), sc);
    note_launch(), mg_post_kernel<T><<<blocks_for(L[l].n), MG_THREADS, 0, s>>>(level_dev<T>(L[l]), par, l, sc);
  }
  note_launch(), mg_prolong_kernel<T><<<blocks_for(L[0].n), MG_THREADS, 0, s>>>(
                     level_dev<T>(L[0]), L[1].w[p].template as<T>(), level_dev<T>(L[1]), v.d[0], v.d[1], sc);
  launch_mg_post0<T>(mesh_grid<T>(m), v, sc, par, mesh_cfg<T>(m), s);
}

static int vec_grid(long long n) { return (int)std::min<long long>(4 * 152, std::max<long long>(1, (n + 255) / 256)); }

template <class T>
void mg_enqueue_init(qcad_mesh_s* m, const PcgVecs<T>& v, PcgScalars* sc, cudaStream_t s) {
  note_launch(), mg_pcg_init_kernel<T><<<vec_grid(m->n_nodes), 256, 0, s>>>(
                     (int)m->n_nodes, v, sc, hier(m)->par[prec_index<T>()].template as<T>());
  enqueue_vcycle<T>(m, v, sc, s);
}
template void mg_enqueue_init<float>(qcad_mesh_s*, const PcgVecs<float>&, PcgScalars*, cudaStream_t);
template void mg_enqueue_init<double>(qcad_mesh_s*, const PcgVecs<double>&, PcgScalars*, cudaStream_t);

template <class T>
void mg_enqueue_update(qcad_mesh_s* m, const PcgVecs<T>& v, PcgScalars* sc, cudaStream_t s) {
  note_launch(), mg_pcg_update_kernel<T><<<vec_grid(m->n_nodes), 256, 0, s>>>(
                     (int)m->n_nodes, v, sc, hier(m)->par[prec_index<T>()].template as<T>());
  enqueue_vcycle<T>(m, v, sc, s);
}
template void mg_enqueue_update<float>(qcad_mesh_s*, const PcgVecs<float>&, PcgScalars*, cudaStream_t);
template void mg_enqueue_update<double>(qcad_mesh_s*, const PcgVecs<double>&, PcgScalars*, cudaStream_t);

int mg_launches_per_iteration(qcad_mesh_s* m) {
  const int nl = mg_levels(m);
  // apply, update, resid0, (restrict + resid) per coarse level but the coarsest has no resid,
  // coarse solve, (prolong + post) per intermediate level, prolong0, post0
  return 2 + 1 + (nl - 1) + (nl - 2) + 1 + 2 * (nl - 2) + 2;
}

}  // namespace qcad
