// Geometric multigrid V-cycle preconditioner (see mg.h): hierarchy construction, Galerkin
// setup per FP32 linearization, and the V-cycle kernels of the coarse levels.
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

// Host side of one level.
struct MgLevel {
  int nx = 0, ny = 0, nz = 0;
  long long n = 0, ne = 0;
  std::vector<double> xs[3];  // node coordinates along x, y, z
  DevBuf A, dinv, mask, b, x, w;
  DevBuf em[3], pr[3], rs[3], ch[3];  // transfers to the next coarser level
  MgLevelDev dev{};
};

struct MgHier {
  std::deque<MgLevel> L;  // a deque: levels are created in place and never move
  DevBuf par;  // per level: Gershgorin bound hi of D^-1 J (float)
  bool ok = false;
  int lin_ver = -1;   // FP32 linearization the operators were built for
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

__device__ __forceinline__ void node_ijk(const MgLevelDev& L, long long n, int& i, int& j, int& k) {
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
__global__ void mg_mask_coarsen_kernel(const MgLevelDev F, const MgLevelDev C, unsigned char* cmask) {
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
__device__ __forceinline__ void mg_accum_row(float (&AE)[64], const float (&row)[8], int a, const float (&px)[4],
                                             const float (&py)[4], const float (&pz)[4]) {
  float u[8], t[8];
  // right multiplication by P, one axis at a time: t[C] = sum_b row[b] P[b][C]
#pragma unroll
  for (int yz = 0; yz < 4; ++yz) {
    const float r0 = row[2 * yz], r1 = row[2 * yz + 1];
    u[2 * yz] = r0 * px[0] + r1 * px[2];
    u[2 * yz + 1] = r0 * px[1] + r1 * px[3];
  }
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int x = 0; x < 2; ++x) {
      const float r0 = u[x + 4 * z], r1 = u[x + 2 + 4 * z];
      t[x + 4 * z] = r0 * py[0] + r1 * py[2];
      t[x + 2 + 4 * z] = r0 * py[1] + r1 * py[3];
    }
#pragma unroll
  for (int xy = 0; xy < 4; ++xy) {
    const float r0 = t[xy], r1 = t[xy + 4];
    u[xy] = r0 * pz[0] + r1 * pz[2];
    u[xy + 4] = r0 * pz[1] + r1 * pz[3];
  }
  // P[a][R] factors by selection (a is a runtime index; indexing the arrays with it would
  // move them to local memory)
  const bool ax = a & 1, ay = (a >> 1) & 1, az = a >> 2;
  const float qx[2] = {ax ? px[2] : px[0], ax ? px[3] : px[1]};
  const float qy[2] = {ay ? py[2] : py[0], ay ? py[3] : py[1]};
  const float qz[2] = {az ? pz[2] : pz[0], az ? pz[3] : pz[1]};
#pragma unroll
  for (int R = 0; R < 8; ++R) {
    const float pa = qx[R & 1] * qy[(R >> 1) & 1] * qz[R >> 2];
#pragma unroll
    for (int C = 0; C < 8; ++C) AE[8 * R + C] += pa * u[C];
  }
}

__device__ __forceinline__ void mg_store_masked(const MgLevelDev& Cl, int I, int J, int K, float (&AE)[64],
                                                float* out) {
  bool dm[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const long long nd = (I + (c & 1)) + (long long)Cl.nxn * ((J + ((c >> 1) & 1)) + (long long)Cl.nyn * (K + (c >> 2)));
    dm[c] = Cl.mask[nd] != 0;
  }
  float4* o = reinterpret_cast<float4*>(out);
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    float v[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int R = (4 * q + s) >> 3, C = (4 * q + s) & 7;
      v[s] = (dm[R] || dm[C]) ? 0.0f : AE[4 * q + s];
    }
    o[q] = make_float4(v[0], v[1], v[2], v[3]);
  }
}

// Row a of the fine-mesh element matrix of element (i, j, k) (stiffness from the 1D element
// matrices, mass term from the 8 quadrature coefficients c), with the columns of Dirichlet
// corners zeroed.
__device__ __forceinline__ void mg_fine_row(const Grid<float>& g, int i, int j, int k, const float (&c)[8],
                                            const bool (&dm)[8], int a, float (&row)[8]) {
  const float mxo = g.mx[3 * i + 2], kxo = g.kx[3 * i + 2];
  const float myo = g.my[3 * j + 2], kyo = g.ky[3 * j + 2];
  const float mzxo = g.mzx[3 * k + 2], mzyo = g.mzy[3 * k + 2], kzo = g.kzz[3 * k + 2];
  const int ax = a & 1, ay = (a >> 1) & 1, az = a >> 2;
  const float GA = GaussConst<float>::a(), GB = GaussConst<float>::b();
  float u[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float bq = ((q & 1) == ax ? GA : GB) * (((q >> 1) & 1) == ay ? GA : GB) * ((q >> 2) == az ? GA : GB);
    u[q] = c[q] * bq;
  }
  float mrow[8];
  tp_apply<float>(u, mrow, GA, GB);
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const int bx = b & 1, by = (b >> 1) & 1, bz = b >> 2;
    const float Mx = (bx == ax ? 2.0f : 1.0f) * mxo, Kx = (bx == ax ? -kxo : kxo);
    const float My = (by == ay ? 2.0f : 1.0f) * myo, Ky = (by == ay ? -kyo : kyo);
    const float Mzx = (bz == az ? 2.0f : 1.0f) * mzxo, Mzy = (bz == az ? 2.0f : 1.0f) * mzyo;
    const float Kz = (bz == az ? -kzo : kzo);
    const float v = Kx * My * Mzx + Mx * Ky * Mzy + Mx * My * Kz + mrow[b];
    row[b] = dm[b] ? 0.0f : v;
  }
}

// Level-1 element matrices from the mesh operator (FP32 coefficients c, 8 per element).
__global__ void __launch_bounds__(128) mg_galerkin0_kernel(const Grid<float> g, const float* __restrict__ coef,
                                                           const MgLevelDev F, const MgLevelDev Cl, float* Aout) {
  const long long E = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long ne = (long long)Cl.nx * Cl.ny * Cl.nz;
  if (E >= ne) return;
  const int I = (int)(E % Cl.nx);
  const long long r = E / Cl.nx;
  const int J = (int)(r % Cl.ny), K = (int)(r / Cl.ny);
  float AE[64];
#pragma unroll
  for (int q = 0; q < 64; ++q) AE[q] = 0.0f;
  const MgChild cx = F.ch[0][I], cy = F.ch[1][J], cz = F.ch[2][K];
  for (int k = cz.first; k < cz.first + cz.count; ++k)
    for (int j = cy.first; j < cy.first + cy.count; ++j)
      for (int i = cx.first; i < cx.first + cx.count; ++i) {
        const MgElemMap ex = F.em[0][i], ey = F.em[1][j], ez = F.em[2][k];
        const float px[4] = {ex.p00, ex.p01, ex.p10, ex.p11};
        const float py[4] = {ey.p00, ey.p01, ey.p10, ey.p11};
        const float pz[4] = {ez.p00, ez.p01, ez.p10, ez.p11};
        float c[8];
        load_c8<float>(coef, i + (long long)g.nx * (j + (long long)g.ny * k), c);
        bool dm[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
          dm[q] = F.mask[(i + (q & 1)) + (long long)F.nxn * ((j + ((q >> 1) & 1)) + (long long)F.nyn * (k + (q >> 2)))] != 0;
        for (int a = 0; a < 8; ++a) {
          if (dm[a]) continue;
          float row[8];
          mg_fine_row(g, i, j, k, c, dm, a, row);
          mg_accum_row(AE, row, a, px, py, pz);
        }
      }
  mg_store_masked(Cl, I, J, K, AE, Aout + 64 * E);
}

// Level l+1 element matrices from the stored level-l ones.
__global__ void __launch_bounds__(128) mg_galerkin_kernel(const MgLevelDev F, const MgLevelDev Cl, float* Aout) {
  const long long E = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long ne = (long long)Cl.nx * Cl.ny * Cl.nz;
  if (E >= ne) return;
  const int I = (int)(E % Cl.nx);
  const long long r = E / Cl.nx;
  const int J = (int)(r % Cl.ny), K = (int)(r / Cl.ny);
  float AE[64];
#pragma unroll
  for (int q = 0; q < 64; ++q) AE[q] = 0.0f;
  const MgChild cx = F.ch[0][I], cy = F.ch[1][J], cz = F.ch[2][K];
  for (int k = cz.first; k < cz.first + cz.count; ++k)
    for (int j = cy.first; j < cy.first + cy.count; ++j)
      for (int i = cx.first; i < cx.first + cx.count; ++i) {
        const MgElemMap ex = F.em[0][i], ey = F.em[1][j], ez = F.em[2][k];
        const float px[4] = {ex.p00, ex.p01, ex.p10, ex.p11};
        const float py[4] = {ey.p00, ey.p01, ey.p10, ey.p11};
        const float pz[4] = {ez.p00, ez.p01, ez.p10, ez.p11};
        const float4* Ae = reinterpret_cast<const float4*>(F.A + 64 * (i + (long long)F.nx * (j + (long long)F.ny * k)));
        for (int a = 0; a < 8; ++a) {
          const float4 r0 = __ldg(Ae + 2 * a), r1 = __ldg(Ae + 2 * a + 1);
          const float row[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
          mg_accum_row(AE, row, a, px, py, pz);
        }
      }
  mg_store_masked(Cl, I, J, K, AE, Aout + 64 * E);
}

// For every element E of level L that contains node (i, j, k): f(row of the node in E's matrix,
// E's first corner node, the node's corner in E).
template <class F>
__device__ __forceinline__ void mg_for_adjacent(const MgLevelDev& L, int i, int j, int k, F&& f) {
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

__device__ __forceinline__ float mg_row_dot(const MgLevelDev& L, const float* row, long long n0, const float* x) {
  const float4 r0 = __ldg(reinterpret_cast<const float4*>(row)), r1 = __ldg(reinterpret_cast<const float4*>(row) + 1);
  const long long sy = L.nxn, sz = (long long)L.nxn * L.nyn;
  return r0.x * x[n0] + r0.y * x[n0 + 1] + r0.z * x[n0 + sy] + r0.w * x[n0 + sy + 1] + r1.x * x[n0 + sz] +
         r1.y * x[n0 + sz + 1] + r1.z * x[n0 + sz + sy] + r1.w * x[n0 + sz + sy + 1];
}

__device__ __forceinline__ void mg_block_max(float v, float* dst) {
  __shared__ float red[32];
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL_MASK, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0f;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL_MASK, v, o));
    if (lane == 0 && v > 0.0f) atomicMax(reinterpret_cast<int*>(dst), __float_as_int(v));
  }
}

// Diagonal, D^-1 and the Gershgorin bound max_i sum_j |J_ij| / J_ii of a coarse level.
__global__ void mg_diag_kernel(const MgLevelDev L, float* dinv, float* par_l) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nn = (long long)L.nxn * L.nyn * L.nzn;
  float ratio = 0.0f;
  if (n < nn) {
    int i, j, k;
    node_ijk(L, n, i, j, k);
    float dg = 0.0f, ra = 0.0f;
    mg_for_adjacent(L, i, j, k, [&](const float* row, long long, int c) {
      dg += row[c];
#pragma unroll
      for (int q = 0; q < 8; ++q) ra += fabsf(row[q]);
    });
    const bool dir = L.mask[n] != 0 || !(dg > 0.0f);
    dinv[n] = dir ? 0.0f : 1.0f / dg;
    ratio = dir ? 0.0f : ra / dg;
  }
  mg_block_max(ratio, par_l);
}

// Gershgorin bound of D^-1 J on the mesh (rows of the element matrices rebuilt from the
// coefficients; Dirichlet rows are identity rows there, ratio 1).
__global__ void mg_gersh0_kernel(const Grid<float> g, const float* __restrict__ coef, const MgLevelDev F,
                                 const float* dinv0, float* par0) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nn = (long long)F.nxn * F.nyn * F.nzn;
  float ratio = 0.0f;
  if (n < nn) {
    int i, j, k;
    node_ijk(F, n, i, j, k);
    if (F.mask[n]) {
      ratio = 1.0f;
    } else {
      float ra = 0.0f;
      for (int e = 0; e < 8; ++e) {
        const int ex = e & 1, ey = (e >> 1) & 1, ez = e >> 2;
        const int I = i - 1 + ex, J = j - 1 + ey, K = k - 1 + ez;
        if (I < 0 || J < 0 || K < 0 || I >= F.nx || J >= F.ny || K >= F.nz) continue;
        const int a = (1 - ex) + 2 * (1 - ey) + 4 * (1 - ez);
        float c[8];
        load_c8<float>(coef, I + (long long)g.nx * (J + (long long)g.ny * K), c);
        bool dm[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
          dm[q] = F.mask[(I + (q & 1)) + (long long)F.nxn * ((J + ((q >> 1) & 1)) + (long long)F.nyn * (K + (q >> 2)))] != 0;
        float row[8];
        mg_fine_row(g, I, J, K, c, dm, a, row);
#pragma unroll
        for (int q = 0; q < 8; ++q) ra += fabsf(row[q]);
      }
      ratio = ra * dinv0[n];
    }
  }
  mg_block_max(ratio, par0);
}

// ---------------------------------------------------------------------------
// V-cycle kernels. Every kernel returns at once when the PCG has finished (sc->done), so the
// iterations captured after convergence cost a launch each and nothing more.

// PCG start with the multigrid preconditioner: x = 0, r = b, ||r||^2, and the level-0
// pre-smoothing zp = omega D^-1 r (into d[0]).
__global__ void mg_pcg_init_kernel(int n, PcgVecs<float> v, PcgScalars* sc, const float* par) {
  const float om = mg_omega(par, 0);
  float rr = 0.0f;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    const float r = v.b[idx];
    v.x[idx] = 0.0f;
    v.r[idx] = r;
    v.d[0][idx] = om * v.dinv[idx] * r;
    rr += r * r;
  }
  double s1[1] = {(double)rr};
  block_sum_atomic<1>(s1, &sc->rr[0]);
}

// PCG update (alpha = rz / pAp): x += alpha p, r -= alpha Ap, ||r||^2, then zp = omega D^-1 r.
__global__ void mg_pcg_update_kernel(int n, PcgVecs<float> v, PcgScalars* sc, const float* par) {
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
  const float alpha = (float)alpha_d;
  const float om = mg_omega(par, 0);
  const float* __restrict__ p = (t & 1) ? v.p[1] : v.p[0];
  float rr = 0.0f;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
    v.x[idx] += alpha * p[idx];
    const float r = v.r[idx] - alpha * v.Ap[idx];
    v.r[idx] = r;
    v.d[0][idx] = om * v.dinv[idx] * r;
    rr += r * r;
  }
  double s1[1] = {(double)rr};
  block_sum_atomic<1>(s1, &sc->rr[(t + 1) & 3]);
}

// Restriction to level l+1 of the fine residual wf: b = P^T wf on the coarse free nodes, and
// the coarse pre-smoothing x = omega D^-1 b.
__global__ void mg_restrict_kernel(const MgLevelDev F, const float* __restrict__ wf, const MgLevelDev C,
                                   const float* par, int lc, const PcgScalars* sc) {
  if (sc->done) return;
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nn = (long long)C.nxn * C.nyn * C.nzn;
  if (n >= nn) return;
  int I, J, K;
  node_ijk(C, n, I, J, K);
  float b = 0.0f;
  if (!C.mask[n]) {
    const MgRestr rx = F.rs[0][I], ry = F.rs[1][J], rz = F.rs[2][K];
    const int fx[3] = {rx.f0, rx.f1, rx.f2}, fy[3] = {ry.f0, ry.f1, ry.f2}, fz[3] = {rz.f0, rz.f1, rz.f2};
    const float wx[3] = {rx.w0, rx.w1, rx.w2}, wy[3] = {ry.w0, ry.w1, ry.w2}, wz[3] = {rz.w0, rz.w1, rz.w2};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (wz[c] == 0.0f) continue;
#pragma unroll
      for (int bb = 0; bb < 3; ++bb) {
        if (wy[bb] == 0.0f) continue;
        const long long base = (long long)F.nxn * (fy[bb] + (long long)F.nyn * fz[c]);
        const float wyz = wy[bb] * wz[c];
        b += wyz * (wx[0] * wf[base + fx[0]] + wx[1] * wf[base + fx[1]] + wx[2] * wf[base + fx[2]]);
      }
    }
  }
  C.b[n] = b;
  C.x[n] = mg_omega(par, lc) * C.dinv[n] * b;
}

// Residual after pre-smoothing on a coarse level: w = b - A x.
__global__ void mg_resid_kernel(const MgLevelDev L, const PcgScalars* sc) {
  if (sc->done) return;
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nn = (long long)L.nxn * L.nyn * L.nzn;
  if (n >= nn) return;
  int i, j, k;
  node_ijk(L, n, i, j, k);
  float y = 0.0f;
  mg_for_adjacent(L, i, j, k, [&](const float* row, long long n0, int) { y += mg_row_dot(L, row, n0, L.x); });
  L.w[n] = L.b[n] - y;
}

// Coarse correction of level l from the solution ec of level l+1: out = base + P ec on free
// nodes (base on Dirichlet nodes).
__global__ void mg_prolong_kernel(const MgLevelDev F, const float* __restrict__ ec, const MgLevelDev C,
                                  const float* base, float* out, const PcgScalars* sc) {
  if (sc->done) return;
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nn = (long long)F.nxn * F.nyn * F.nzn;
  if (n >= nn) return;
  float v = base[n];
  if (!F.mask[n]) {
    int i, j, k;
    node_ijk(F, n, i, j, k);
    const MgProl px = F.pr[0][i], py = F.pr[1][j], pz = F.pr[2][k];
    const long long sy = C.nxn, sz = (long long)C.nxn * C.nyn;
    const long long z0 = pz.c0 * sz, z1 = pz.c1 * sz, y0 = py.c0 * sy, y1 = py.c1 * sy;
    const float e00 = px.w0 * ec[z0 + y0 + px.c0] + px.w1 * ec[z0 + y0 + px.c1];
    const float e01 = px.w0 * ec[z0 + y1 + px.c0] + px.w1 * ec[z0 + y1 + px.c1];
    const float e10 = px.w0 * ec[z1 + y0 + px.c0] + px.w1 * ec[z1 + y0 + px.c1];
    const float e11 = px.w0 * ec[z1 + y1 + px.c0] + px.w1 * ec[z1 + y1 + px.c1];
    v += pz.w0 * (py.w0 * e00 + py.w1 * e01) + pz.w1 * (py.w0 * e10 + py.w1 * e11);
  }
  out[n] = v;
}

// Post-smoothing on a coarse level: w = x + omega D^-1 (b - A x) (the level's solution).
__global__ void mg_post_kernel(const MgLevelDev L, const float* par, int l, const PcgScalars* sc) {
  if (sc->done) return;
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nn = (long long)L.nxn * L.nyn * L.nzn;
  if (n >= nn) return;
  int i, j, k;
  node_ijk(L, n, i, j, k);
  float y = 0.0f;
  mg_for_adjacent(L, i, j, k, [&](const float* row, long long n0, int) { y += mg_row_dot(L, row, n0, L.x); });
  L.w[n] = L.x[n] + mg_omega(par, l) * L.dinv[n] * (L.b[n] - y);
}

// Coarsest level: Chebyshev iteration of degree MG_COARSE_DEGREE for A x = b on
// [hi / 64, hi] inside one block of 1024 threads, with the element matrices and the vectors
// in shared memory; the result goes to w.
__global__ void __launch_bounds__(1024) mg_coarse_kernel(const MgLevelDev L, const float* par, int l,
                                                         const PcgScalars* sc) {
  if (sc->done) return;
  extern __shared__ float sh[];
  const int ne = L.nx * L.ny * L.nz;
  const int nn = L.nxn * L.nyn * L.nzn;
  float* sA = sh;               // 64 ne
  float* sd = sA + 64 * ne;     // direction
  float* sr = sd + nn;          // residual
  float* sx = sr + nn;          // solution
  for (int q = threadIdx.x; q < 64 * ne; q += blockDim.x) sA[q] = L.A[q];
  const float hi = par[l];
  const int n = threadIdx.x;  // one node per thread: the coarsest level has at most 512 nodes
  const bool own = n < nn;
  if (!(hi > 0.0f)) {
    if (own) L.w[n] = 0.0f;
    return;
  }
  const float lo = hi / 64.0f;
  const float theta = 0.5f * (hi + lo), delta = 0.5f * (hi - lo), sigma = theta / delta;
  const float dv = own ? L.dinv[n] : 0.0f;
  if (own) {
    const float r = L.b[n];
    const float d = dv * r / theta;
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
  float rho = 1.0f / sigma;
  for (int it = 1; it < MG_COARSE_DEGREE; ++it) {
    const float rho_new = 1.0f / (2.0f * sigma - rho);
    const float c1 = rho_new * rho, c2 = 2.0f * rho_new / delta;
    float y = 0.0f;
    if (own) {
      for (int e = 0; e < 8; ++e) {
        const int ex = e & 1, ey = (e >> 1) & 1, ez = e >> 2;
        const int I = i - 1 + ex, J = j - 1 + ey, K = k - 1 + ez;
        if (I < 0 || J < 0 || K < 0 || I >= L.nx || J >= L.ny || K >= L.nz) continue;
        const int c = (1 - ex) + 2 * (1 - ey) + 4 * (1 - ez);
        const float* row = sA + 64 * (I + L.nx * (J + L.ny * K)) + 8 * c;
        const int n0 = I + sy * (J + L.nyn * K);
        y += row[0] * sd[n0] + row[1] * sd[n0 + 1] + row[2] * sd[n0 + sy] + row[3] * sd[n0 + sy + 1] +
             row[4] * sd[n0 + sz] + row[5] * sd[n0 + sz + 1] + row[6] * sd[n0 + sz + sy] +
             row[7] * sd[n0 + sz + sy + 1];
      }
    }
    __syncthreads();
    if (own) {
      const float r = sr[n] - y;
      const float d = c1 * sd[n] + c2 * dv * r;
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
  // usable when there is at least one coarse level and the coarsest fits one block's shared memory
  const size_t coarse_smem = ((size_t)64 * co.ne + 3 * (size_t)co.n) * sizeof(float);
  H->ok = L.size() >= 2 && co.n <= MG_COARSE_NODES && coarse_smem <= 200 * 1024;
  if (!H->ok) return false;
  for (size_t l = 0; l < L.size(); ++l) {
    MgLevel& v = L[l];
    v.mask.ensure((size_t)v.n + 64);
    if (l > 0) {
      v.A.ensure((size_t)64 * v.ne * sizeof(float) + 64);
      v.dinv.ensure((size_t)v.n * sizeof(float) + 64);
      v.b.ensure((size_t)v.n * sizeof(float) + 64);
      v.x.ensure((size_t)v.n * sizeof(float) + 64);
      v.w.ensure((size_t)v.n * sizeof(float) + 64);
    }
    MgLevelDev& d = v.dev;
    d.nx = v.nx;
    d.ny = v.ny;
    d.nz = v.nz;
    d.nxn = v.nx + 1;
    d.nyn = v.ny + 1;
    d.nzn = v.nz + 1;
    d.A = v.A.as<float>();
    d.dinv = v.dinv.as<float>();
    d.mask = v.mask.as<unsigned char>();
    d.b = v.b.as<float>();
    d.x = v.x.as<float>();
    d.w = v.w.as<float>();
    for (int a = 0; a < 3; ++a) {
      d.em[a] = v.em[a].as<MgElemMap>();
      d.pr[a] = v.pr[a].as<MgProl>();
      d.rs[a] = v.rs[a].as<MgRestr>();
      d.ch[a] = v.ch[a].as<MgChild>();
    }
  }
  H->par.ensure(MG_MAX_LEVELS * sizeof(float) + 64);
  mg_mask0_kernel<<<blocks_for(L[0].n), MG_THREADS, 0, s>>>(m->g32.g, L[0].mask.as<unsigned char>());
  for (size_t l = 0; l + 1 < L.size(); ++l)
    mg_mask_coarsen_kernel<<<blocks_for(L[l + 1].n), MG_THREADS, 0, s>>>(L[l].dev, L[l + 1].dev,
                                                                          L[l + 1].mask.as<unsigned char>());
  // the largest coarsest level any mesh may have (checked above), so one setting serves all
  CK(cudaFuncSetAttribute(mg_coarse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return true;
}

void mg_invalidate(qcad_mesh_s* m) {
  if (m->mg) hier(m)->lin_ver = -1;
}

int mg_levels(qcad_mesh_s* m) { return (m->mg && hier(m)->ok) ? (int)hier(m)->L.size() : 0; }

void mg_setup(qcad_mesh_s* m, cudaStream_t s, bool force) {
  MgHier* H = hier(m);
  if (!force && H->lin_ver == m->lin_ver[1]) return;
  std::deque<MgLevel>& L = H->L;
  const PcgBufs<float>& k = m->k32;
  float* par = H->par.as<float>();
  CK(cudaMemsetAsync(par, 0, MG_MAX_LEVELS * sizeof(float), s));
  mg_gersh0_kernel<<<blocks_for(L[0].n), MG_THREADS, 0, s>>>(m->g32.g, k.c.as<float>(), L[0].dev,
                                                             k.dinv.as<float>(), par);
  mg_galerkin0_kernel<<<blocks_for(L[1].ne, 128), 128, 0, s>>>(m->g32.g, k.c.as<float>(), L[0].dev, L[1].dev,
                                                          L[1].A.as<float>());
  for (size_t l = 1; l < L.size(); ++l) {
    if (l > 1)
      mg_galerkin_kernel<<<blocks_for(L[l].ne, 128), 128, 0, s>>>(L[l - 1].dev, L[l].dev, L[l].A.as<float>());
    mg_diag_kernel<<<blocks_for(L[l].n), MG_THREADS, 0, s>>>(L[l].dev, L[l].dinv.as<float>(), par + l);
  }
  note_launch(2 + 2 * ((int)L.size() - 1) - 1);
  CK(cudaGetLastError());
  H->lin_ver = m->lin_ver[1];
}

// V-cycle after the level-0 pre-smoothing (zp in d[0]): ends with z and the PCG bookkeeping.
static void enqueue_vcycle(qcad_mesh_s* m, const PcgVecs<float>& v, PcgScalars* sc, cudaStream_t s) {
  MgHier* H = hier(m);
  std::deque<MgLevel>& L = H->L;
  const float* par = H->par.as<float>();
  const int nl = (int)L.size();
  launch_mg_resid0(m->g32.g, v, sc, m->cfg32, s);
  for (int l = 0; l + 1 < nl; ++l) {
    const float* wf = l == 0 ? v.w : L[l].w.as<float>();
    note_launch(), mg_restrict_kernel<<<blocks_for(L[l + 1].n), MG_THREADS, 0, s>>>(L[l].dev, wf, L[l + 1].dev,
                                                                                      par, l + 1, sc);
    if (l + 1 < nl - 1) note_launch(), mg_resid_kernel<<<blocks_for(L[l + 1].n), MG_THREADS, 0, s>>>(L[l + 1].dev, sc);
  }
  const MgLevel& co = L[nl - 1];
  const int smem = (int)(((size_t)64 * co.ne + 3 * (size_t)co.n) * sizeof(float));
  note_launch(), mg_coarse_kernel<<<1, 1024, smem, s>>>(co.dev, par, nl - 1, sc);
  for (int l = nl - 2; l >= 1; --l) {
    note_launch(), mg_prolong_kernel<<<blocks_for(L[l].n), MG_THREADS, 0, s>>>(L[l].dev, L[l + 1].w.as<float>(),
                                                                                 L[l + 1].dev, L[l].x.as<float>(),
                                                                                 L[l].x.as<float>(), sc);
    note_launch(), mg_post_kernel<<<blocks_for(L[l].n), MG_THREADS, 0, s>>>(L[l].dev, par, l, sc);
  }
  note_launch(), mg_prolong_kernel<<<blocks_for(L[0].n), MG_THREADS, 0, s>>>(L[0].dev, L[1].w.as<float>(), L[1].dev,
                                                                              v.d[0], v.d[1], sc);
  launch_mg_post0(m->g32.g, v, sc, par, m->cfg32, s);
}

static int vec_grid(long long n) { return (int)std::min<long long>(4 * 152, std::max<long long>(1, (n + 255) / 256)); }

void mg_enqueue_init(qcad_mesh_s* m, const PcgVecs<float>& v, PcgScalars* sc, cudaStream_t s) {
  note_launch(), mg_pcg_init_kernel<<<vec_grid(m->n_nodes), 256, 0, s>>>((int)m->n_nodes, v, sc,
                                                                         hier(m)->par.as<float>());
  enqueue_vcycle(m, v, sc, s);
}

void mg_enqueue_update(qcad_mesh_s* m, const PcgVecs<float>& v, PcgScalars* sc, cudaStream_t s) {
  note_launch(), mg_pcg_update_kernel<<<vec_grid(m->n_nodes), 256, 0, s>>>((int)m->n_nodes, v, sc,
                                                                           hier(m)->par.as<float>());
  enqueue_vcycle(m, v, sc, s);
}

int mg_launches_per_iteration(qcad_mesh_s* m) {
  const int nl = mg_levels(m);
  // apply, update, resid0, (restrict + resid) per coarse level but the coarsest has no resid,
  // coarse solve, (prolong + post) per intermediate level, prolong0, post0
  return 2 + 1 + (nl - 1) + (nl - 2) + 1 + 2 * (nl - 2) + 2;
}

}  // namespace qcad
