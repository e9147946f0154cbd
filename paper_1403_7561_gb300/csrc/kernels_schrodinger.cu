// Effective-mass Schrodinger operators on the quantum subdomain and the dense
// block kernels of LOBPCG. Sec. II.B (Eqs. SchrodEqn, SchrodEqnWeakForm,
// Schrodinger3D) with the potential energy of Eq. SchrodPotEnergy (no V_xc).
#include <cuda_runtime.h>

#include "dfloat.cuh"

#include <cstdlib>
#include <cstring>
#include <type_traits>

#include <algorithm>

#include "qcad_host.h"
#include "qcad_internal.cuh"
#include "qcad_dense.h"

namespace qcad {

// H X and M X for nvec vectors in one z-march: field 0 = H (kinetic stencil
// with kappa_d = hbar^2/(2 m_d) plus the V mass term), field 1 = M (consistent
// mass). psi = 0 on the subdomain boundary: outputs there are zero.
template <class T>
struct HmOp {
  static constexpr int NF = 2;
  static constexpr bool STIFF = true;
  using ED = C8<T>;
  HmArgs<T> a;
  int vec;
  __device__ bool skip() const { return false; }
  __device__ void set_vec(int v) { vec = v; }
  __device__ T load(const Grid<T>&, int n, bool in, int, int, int) const {
    return in ? a.x[(long long)vec * a.ld + n] : T(0);
  }
  __device__ ED edata(const Grid<T>& g, int i, int j, int k) const {
    ED r;
    load_c8<T>(a.cV, i + g.nx * (j + g.ny * k), r.c);
    return r;
  }
  __device__ void elem(const Grid<T>& g, int i, int j, int k, const T* v, const ED& ed, T (*out)[8], bool) const {
    qp_mass<T>(v, ed.c, out[0]);
    const T wdet = g.hx[i] * g.hy[j] * g.hz[k] * T(0.125);
    T u[8];
    tp_apply(v, u, GaussConst<T>::a(), GaussConst<T>::b());
#pragma unroll
    for (int q = 0; q < 8; ++q) u[q] *= wdet;
    tp_apply(u, out[1], GaussConst<T>::a(), GaussConst<T>::b());
  }
  __device__ void node(const Grid<T>& g, int n, int i, int j, int k, T, T stiff, const T* mass) {
    const bool bd = grid_is_dir(g, i, j, k);
    const long long o = (long long)vec * a.ld + n;
    if (a.hx) a.hx[o] = bd ? T(0) : stiff + mass[0];
    if (a.mx) a.mx[o] = bd ? T(0) : mass[1];
  }
  __device__ void finish() {}
};

template <class T>
void launch_hm_apply(const Grid<T>& g, const HmArgs<T>& args, LaunchCfg cfg, cudaStream_t s) {
  if (cfg.variant >= 2) {
    launch_hm_apply_lin<T>(g, args, cfg, s);
    return;
  }
  HmOp<T> op = {};
  op.a = args;
  const int by = cfg.by == 4 ? 4 : 8;
  dim3 grid = march_grid(g.nxn, g.nyn, g.nzn, by, cfg.kchunk, args.nvec);
  if (by == 4)
    note_launch(), march_kernel<T, 4, HmOp<T>><<<grid, dim3(QCAD_BX, 4), 0, s>>>(g, op, cfg.kchunk);
  else
    note_launch(), march_kernel<T, 8, HmOp<T>><<<grid, dim3(QCAD_BX, 8), 0, s>>>(g, op, cfg.kchunk);
}
template void launch_hm_apply<float>(const Grid<float>&, const HmArgs<float>&, LaunchCfg, cudaStream_t);
template void launch_hm_apply<double>(const Grid<double>&, const HmArgs<double>&, LaunchCfg, cudaStream_t);

constexpr int DT = 256;
static int dblocks(long long n) {
  long long b = (n + DT - 1) / DT;
  return (int)(b < 152 * 8 ? (b > 0 ? b : 1) : 152 * 8);
}

// cV_q = (q phi_ref - chi - q phi(x_q)) * w|J| for every subdomain element (Eq. SchrodPotEnergy).
template <class T>
__global__ void potential_kernel(SubdomainMap sm, const double* phi, double V0, const double* hx,
                                 const double* hy, const double* hz, const double* vxq, T* cV, double* vmin) {
  const long long ne = (long long)sm.nxs * sm.nys * sm.nzs;
  double lo = 1e300;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x) {
    const int is = (int)(e % sm.nxs);
    const int js = (int)((e / sm.nxs) % sm.nys);
    const int ks = (int)(e / ((long long)sm.nxs * sm.nys));
    const int i = sm.i0 + is, j = sm.j0 + js, k = sm.k0 + ks;
    const long long n0 = i + sm.nxn * ((long long)j + (long long)sm.nyn * k);
    const long long px = 1, py = sm.nxn, pz = (long long)sm.nxn * sm.nyn;
    double v[8], q[8];
    v[0] = phi[n0];
    v[1] = phi[n0 + px];
    v[2] = phi[n0 + py];
    v[3] = phi[n0 + px + py];
    v[4] = phi[n0 + pz];
    v[5] = phi[n0 + pz + px];
    v[6] = phi[n0 + pz + py];
    v[7] = phi[n0 + pz + px + py];
    tp_apply(v, q, GaussConst<double>::a(), GaussConst<double>::b());
    const double wdet = hx[i] * hy[j] * hz[k] * 0.125;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const double V = V0 - q[s] + (vxq ? vxq[8 * e + s] : 0.0);
      lo = fmin(lo, V);
      cV[8 * e + s] = (T)(V * wdet);
    }
  }
  // min over the block via shuffles, then an atomic on the ordered bits of (V + offset)
  for (int o = 16; o > 0; o >>= 1) lo = fmin(lo, __shfl_xor_sync(FULL_MASK, lo, o));
  if ((threadIdx.x & 31) == 0 && lo < 1e299) {
    // vmin[0] holds the minimum shifted by +100 eV to stay non-negative
    atomicMin(reinterpret_cast<unsigned long long*>(vmin), (unsigned long long)__double_as_longlong(lo + 100.0));
  }
}

template <class T>
void launch_potential(const SubdomainMap& sm, const double* phi, double V0, const double* hx, const double* hy,
                      const double* hz, const double* vxq, T* cV, double* vmin, cudaStream_t s) {
  const long long ne = (long long)sm.nxs * sm.nys * sm.nzs;
  note_launch(), potential_kernel<T><<<dblocks(ne), DT, 0, s>>>(sm, phi, V0, hx, hy, hz, vxq, cV, vmin);
}
template void launch_potential<float>(const SubdomainMap&, const double*, double, const double*, const double*,
                                      const double*, const double*, float*, double*, cudaStream_t);
template void launch_potential<double>(const SubdomainMap&, const double*, double, const double*, const double*,
                                       const double*, const double*, double*, double*, cudaStream_t);

// Interior-DOF <-> full subdomain node vector (column-major blocks).
__global__ void pack_kernel(SubdomainMap sm, int nvec, double* full, long long ldf, double* dof, long long ldd,
                            int unpack) {
  const int nxi = sm.nxs - 1, nyi = sm.nys - 1, nzi = sm.nzs - 1;
  const long long nd = (long long)nxi * nyi * nzi;
  const long long total = nd * nvec;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int v = (int)(t / nd);
    const long long d = t % nd;
    const int a = (int)(d % nxi) + 1;
    const int b = (int)((d / nxi) % nyi) + 1;
    const int c = (int)(d / ((long long)nxi * nyi)) + 1;
    const long long f = a + (long long)(sm.nxs + 1) * (b + (long long)(sm.nys + 1) * c);
    if (unpack)
      full[v * ldf + f] = dof[v * ldd + d];
    else
      dof[v * ldd + d] = full[v * ldf + f];
  }
}

void launch_pack(const SubdomainMap& sm, int nvec, double* full, long long ldf, double* dof, long long ldd,
                 int unpack, cudaStream_t s) {
  const long long total = (long long)(sm.nxs - 1) * (sm.nys - 1) * (sm.nzs - 1) * nvec;
  note_launch(), pack_kernel<<<dblocks(total), DT, 0, s>>>(sm, nvec, full, ldf, dof, ldd, unpack);
}

// Double-float arithmetic for the FP64 phase's dense block products. This part runs FP32 at
// about 57 times its FP64 rate, so a product-accumulate of two FP64 values carried as
// unevaluated sums of two floats (hi + lo, a 48-bit significand) costs fewer cycles than one
// DFMA. The product is exact up to the dropped lo*lo term (Dekker's product through the fused
// multiply-add); the sum is Knuth's two-sum into the high word with the errors gathered in the
// low word. Relative error of a length-p dot product: about p * 2^-48.
__device__ __forceinline__ void df_split(double a, float& h, float& l) {
  h = __double2float_rn(a);
  l = __double2float_rn(a - (double)h);
}

__device__ __forceinline__ void df_mac(float& sh, float& sl, float ah, float al, float bh, float bl) {
  const float ph = ah * bh;
  float pl = fmaf(ah, bh, -ph);
  pl = fmaf(ah, bl, pl);
  pl = fmaf(al, bh, pl);
  const float t = sh + ph;
  const float bp = t - sh;
  const float e = (sh - (t - bp)) + (ph - bp);
  sh = t;
  sl += e + pl;
}

// Splits and joins of FP64 values go through the bit patterns (dfloat.cuh): the FP32<->FP64
// conversion instructions run on the FP64 pipe of this part (2 lanes per SM per clock), so
// converting in float arithmetic would cost more than the products themselves.
__device__ __forceinline__ void df_split_i(double a, float& h, float& l) {
  const dfl d = dfl_from_bits(a);
  h = d.h;
  l = d.l;
}
__device__ __forceinline__ double df_join(float h, float l) { return dfl_to_double(dfl(h, l)); }

// (ah, al) += (bh, bl) in double-float (Knuth's two-sum on the high words, low words summed).
__device__ __forceinline__ void df_acc(float& ah, float& al, float bh, float bl) {
  const float t = ah + bh;
  const float bp = t - ah;
  const float e = (ah - (t - bp)) + (bh - bp);
  ah = t;
  al += e + bl;
}

// G1 = A^T B1 and optionally G2 = A^T B2 (p x p each, row-major o = a*p + b) for column-major
// A (n x p, lda) and B1, B2 (n x p, ldb): the Gram matrices of the LOBPCG blocks. A block walks
// 32-row tiles of its share of the rows, copied asynchronously (double-buffered) into shared
// memory transposed ([row][column]); each thread owns a 4 x 4 tile of outputs (registers), sums
// a row tile in the storage precision and accumulates tiles in FP64. Every block writes its
// partial sums to its own slot of `part` (no atomics); gram_reduce_kernel adds the slots in a
// fixed order, so the result is deterministic.
constexpr int GR = 32;                   // rows per shared-memory tile
constexpr int GRAM_MAX_BLOCKS = 2 * 152;

// 4 consecutive values of a shared row (16-byte aligned for float, two 16-byte loads for double).
__device__ __forceinline__ void gram_ld4(const float* p, float* v) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void gram_ld4(const double* p, double* v) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// One element global -> shared, asynchronous; zero fill when !valid.
template <class T>
__device__ __forceinline__ void gram_cp(T* smem, const T* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? (int)sizeof(T) : 0;
  if constexpr (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(n) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}

// GC > 0: the row-group count G at compile time (FP32 storage takes one group), so that the row loop
// over a shared tile unrolls completely.
template <class T, int GC = 0>
__global__ void __launch_bounds__(512) gram_kernel(long long n, int p, int nb2, const T* A, long long lda,
                                                   const T* B1, const T* B2, long long ldb, double* part, int G_) {
  const int G = GC > 0 ? GC : G_;
  extern __shared__ __align__(16) unsigned char sh_raw[];
  T* sh = reinterpret_cast<T*>(sh_raw);      // two stages of GR x W
  const int q = p;
  const int qt = q * nb2;
  const int ta_n = (p + 3) / 4, tb_n = (qt + 3) / 4;
  const int pp = 4 * ta_n, qp = 4 * tb_n;
  const int W = pp + qp + 4;                 // shared row stride (multiple of 4): A | B1 | B2
  const int tid = threadIdx.x, nth = blockDim.x;
  // padding columns stay zero (the copies write only the real columns)
  for (int t = tid; t < 2 * GR * W; t += nth) sh[t] = T(0);
  __syncthreads();
  // G row groups of nt = ta_n * tb_n output tiles: group g takes the rows g, g + G, ... of each
  // shared tile, so that small products still occupy the block
  const int nt = ta_n * tb_n;
  const bool active = tid < G * nt;
  const int grp = active ? tid / nt : 0, tt = active ? tid % nt : 0;
  const int ta = tt / tb_n, tb = tt % tb_n;
  // across tiles: FP64 (double storage) or double-float on the FP32 pipes (float storage, where
  // an FP64 add per output and tile would cost more than the tile's products)
  double acc[16];
  float acch[16], accl[16];
#pragma unroll
  for (int s = 0; s < 16; ++s) {
    acc[s] = 0.0;
    acch[s] = 0.0f;
    accl[s] = 0.0f;
  }
  const long long ntiles = (n + GR - 1) / GR;
  auto issue = [&](long long tile, int stage) {
    if (tile < ntiles) {
      const long long r0 = tile * GR;
      T* st = sh + (size_t)stage * GR * W;
      for (int t = tid; t < (p + qt) * GR; t += nth) {
        const int col = t / GR, rr = t % GR;
        const long long row = r0 + rr;
        const bool ok = row < n;
        const T* src;
        int sc;
        if (col < p) {
          src = A + col * lda + (ok ? row : 0);
          sc = col;
        } else {
          const int bc = col - p;
          src = (bc < q ? B1 + bc * ldb : B2 + (bc - q) * ldb) + (ok ? row : 0);
          sc = pp + bc;
        }
        gram_cp<T>(st + rr * W + sc, src, ok);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  int stage = 0;
  issue(blockIdx.x, 0);
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    issue(tile + gridDim.x, stage ^ 1);  // next tile into the other stage
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    __syncthreads();
    if (active) {
      const T* st = sh + (size_t)stage * GR * W;
      T s16[16];
#pragma unroll
      for (int s = 0; s < 16; ++s) s16[s] = T(0);
#pragma unroll(GC > 0 ? GR / (GC > 0 ? GC : 1) : 4)
      for (int rr = grp; rr < GR; rr += G) {
        const T* row = st + rr * W;
        T av[4], bv[4];
        gram_ld4(row + 4 * ta, av);
        gram_ld4(row + pp + 4 * tb, bv);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) s16[4 * u + v] += av[u] * bv[v];
      }
#pragma unroll
      for (int s = 0; s < 16; ++s) {
        if constexpr (sizeof(T) == 4)
          df_acc(acch[s], accl[s], (float)s16[s], 0.0f);
        else
          acc[s] += (double)s16[s];
      }
    }
    __syncthreads();  // the stage is refilled by the next iteration's copies
    stage ^= 1;
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int s = 0; s < 16; ++s) acc[s] = df_join(acch[s], accl[s]);
  }
  // the groups' sums in a fixed order (the staging area is free now)
  __syncthreads();
  double* red = reinterpret_cast<double*>(sh_raw);  // [G][nt][16]
  if (active)
#pragma unroll
    for (int s = 0; s < 16; ++s) red[((size_t)grp * nt + tt) * 16 + s] = acc[s];
  __syncthreads();
  if (!active || grp != 0) return;
  for (int g2 = 1; g2 < G; ++g2)
#pragma unroll
    for (int s = 0; s < 16; ++s) acc[s] += red[((size_t)g2 * nt + tt) * 16 + s];
  // slot layout: product 0 (p*q) then product 1
  double* out = part + (size_t)blockIdx.x * p * qt;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int a = 4 * ta + u;
    if (a >= p) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int bc = 4 * tb + v;
      if (bc >= qt) continue;
      out[bc < q ? a * q + bc : p * q + a * q + (bc - q)] = acc[4 * u + v];
    }
  }
}

// Sum of the per-block partials in a fixed order: 32 outputs per block, 8 warps each summing
// every 8th partial, then the 8 sums in order.
__global__ void __launch_bounds__(256) gram_reduce_kernel(int nblk, int tot, int pq, const double* part, double* G1,
                                                          double* G2) {
  __shared__ double red[8][32];
  const int o = blockIdx.x * 32 + threadIdx.x;
  double s = 0.0;
  if (o < tot)
    for (int b = threadIdx.y; b < nblk; b += 8) s += part[(size_t)b * tot + o];
  red[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && o < tot) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w][threadIdx.x];
    if (o < pq)
      G1[o] = t;
    else
      G2[o - pq] = t;
  }
}

size_t gram_part_doubles(int p, int q) { return (size_t)GRAM_MAX_BLOCKS * p * 2 * q; }

// ---------------------------------------------------------------------------
// gram_kernel for FP64 blocks in double-float arithmetic: the double tile lands in shared
// memory as before, is split once into hi and lo float tiles, and each 32-row tile is summed in
// double-float before it is added to the FP64 accumulators.
// upper: only the output tiles on or above the diagonal of each product (p == q, q a multiple of
// 4); the entries below are left unwritten.
__global__ void __launch_bounds__(512) gram_df_kernel(long long n, int p, int nb2, const double* A, long long lda,
                                                      const double* B1, const double* B2, long long ldb,
                                                      double* part, int G, int upper) {
  extern __shared__ __align__(16) unsigned char sh_raw[];
  const int q = p;
  const int qt = q * nb2;
  const int ta_n = (p + 3) / 4, tb_n = (qt + 3) / 4;
  const int pp = 4 * ta_n, qp = 4 * tb_n;
  const int W = pp + qp + 4;
  double* sh = reinterpret_cast<double*>(sh_raw);                 // two stages of GR x W doubles
  float* fh = reinterpret_cast<float*>(sh + (size_t)2 * GR * W);  // GR x W hi words
  float* fl = fh + (size_t)GR * W;                                // GR x W lo words
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int t = tid; t < 2 * GR * W; t += nth) sh[t] = 0.0;
  __syncthreads();
  // G row groups of nt output tiles, as in gram_kernel
  const int tq = ta_n, tri = tq * (tq + 1) / 2;  // upper: tiles per product on or above its diagonal
  const int nt = upper ? nb2 * tri : ta_n * tb_n;
  const bool active = tid < G * nt;
  const int grp = active ? tid / nt : 0, tt = active ? tid % nt : 0;
  int ta, tb;
  if (upper) {
    const int k = tt / tri;
    int r = tt % tri, row = 0;
    while (r >= tq - row) {
      r -= tq - row;
      ++row;
    }
    ta = row;
    tb = k * tq + row + r;
  } else {
    ta = tt / tb_n;
    tb = tt % tb_n;
  }
  float acch[16], accl[16];  // double-float accumulation across tiles
#pragma unroll
  for (int s = 0; s < 16; ++s) {
    acch[s] = 0.0f;
    accl[s] = 0.0f;
  }
  const long long ntiles = (n + GR - 1) / GR;
  auto issue = [&](long long tile, int stage) {
    if (tile < ntiles) {
      const long long r0 = tile * GR;
      double* st = sh + (size_t)stage * GR * W;
      for (int t = tid; t < (p + qt) * GR; t += nth) {
        const int col = t / GR, rr = t % GR;
        const long long row = r0 + rr;
        const bool ok = row < n;
        const double* src;
        int sc;
        if (col < p) {
          src = A + col * lda + (ok ? row : 0);
          sc = col;
        } else {
          const int bc = col - p;
          src = (bc < q ? B1 + bc * ldb : B2 + (bc - q) * ldb) + (ok ? row : 0);
          sc = pp + bc;
        }
        gram_cp<double>(st + rr * W + sc, src, ok);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  int stage = 0;
  issue(blockIdx.x, 0);
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    issue(tile + gridDim.x, stage ^ 1);
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    __syncthreads();
    {
      const double* st = sh + (size_t)stage * GR * W;
      for (int t = tid; t < GR * W; t += nth) df_split_i(st[t], fh[t], fl[t]);
    }
    __syncthreads();
    if (active) {
      float sh16[16], sl16[16];
#pragma unroll
      for (int s = 0; s < 16; ++s) {
        sh16[s] = 0.0f;
        sl16[s] = 0.0f;
      }
#pragma unroll 2
      for (int rr = grp; rr < GR; rr += G) {
        float ah[4], al[4], bh[4], bl[4];
        gram_ld4(fh + rr * W + 4 * ta, ah);
        gram_ld4(fl + rr * W + 4 * ta, al);
        gram_ld4(fh + rr * W + pp + 4 * tb, bh);
        gram_ld4(fl + rr * W + pp + 4 * tb, bl);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) df_mac(sh16[4 * u + v], sl16[4 * u + v], ah[u], al[u], bh[v], bl[v]);
      }
#pragma unroll
      for (int s = 0; s < 16; ++s) df_acc(acch[s], accl[s], sh16[s], sl16[s]);
    }
    __syncthreads();
    stage ^= 1;
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  double acc[16];
#pragma unroll
  for (int s = 0; s < 16; ++s) acc[s] = df_join(acch[s], accl[s]);
  __syncthreads();
  double* red = reinterpret_cast<double*>(sh_raw);  // [G][nt][16]
  if (active)
#pragma unroll
    for (int s = 0; s < 16; ++s) red[((size_t)grp * nt + tt) * 16 + s] = acc[s];
  __syncthreads();
  if (!active || grp != 0) return;
  for (int g2 = 1; g2 < G; ++g2)
#pragma unroll
    for (int s = 0; s < 16; ++s) acc[s] += red[((size_t)g2 * nt + tt) * 16 + s];
  double* out = part + (size_t)blockIdx.x * p * qt;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int a = 4 * ta + u;
    if (a >= p) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int bc = 4 * tb + v;
      if (bc >= qt) continue;
      out[bc < q ? a * q + bc : p * q + a * q + (bc - q)] = acc[4 * u + v];
    }
  }
}

// Whether the FP64 phase's Gram and combine run in double-float (default) or in native FP64
// (environment QCAD_FP64_DENSE=native).
static bool dense_df() {
  static const bool df = [] {
    const char* e = std::getenv("QCAD_FP64_DENSE");
    return !(e && std::strcmp(e, "native") == 0);
  }();
  return df;
}

template <class T>
void launch_gram(long long n, int p, int q, const T* A, long long lda, const T* B1, const T* B2, long long ldb,
                 double* G1, double* G2, double* part, cudaStream_t s, bool upper) {
  (void)q;  // the products of LOBPCG are square: q == p
  const int nb2 = B2 ? 2 : 1;
  const int ta_n = (p + 3) / 4, tb_n = (p * nb2 + 3) / 4;
  // row groups (double storage): as many copies of the output tiles as fit 512 threads (at most
  // 8), so that the double-float products of small blocks occupy the block; with float storage a
  // tile's products are cheap next to the per-tile accumulation, so one group
  const int nt = ta_n * tb_n;
  const int G = sizeof(T) == 8 ? std::max(1, std::min(8, 512 / nt)) : 1;
  const int nth = std::min(512, std::max(256, ((G * nt + 31) / 32) * 32));
  const long long ntiles = (n + GR - 1) / GR;
  const int nblk = (int)std::max<long long>(1, std::min<long long>(GRAM_MAX_BLOCKS, ntiles));
  const size_t red = (size_t)G * nt * 16 * sizeof(double);  // the groups' sums, after the tiles
  const size_t shm = std::max(red, (size_t)2 * GR * (4 * ta_n + 4 * tb_n + 4) * sizeof(T));
  static bool attr = false;
  if (!attr)
    attr = cudaFuncSetAttribute(gram_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024) == cudaSuccess &&
           cudaFuncSetAttribute(gram_kernel<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024) ==
               cudaSuccess;
  if constexpr (std::is_same<T, double>::value) {
    if (dense_df()) {
      // the upper triangles only (the caller mirrors them), where the tiles align with the products
      const int up = (upper && p == q && p % 4 == 0) ? 1 : 0;
      const int nt_df = up ? nb2 * (ta_n * (ta_n + 1) / 2) : nt;
      const int G_df = std::max(1, std::min(8, 512 / nt_df));
      const int nth_df = std::min(512, std::max(256, ((G_df * nt_df + 31) / 32) * 32));
      const size_t red_df = (size_t)G_df * nt_df * 16 * sizeof(double);
      // two double stages plus the hi and lo float tiles
      const size_t shm_df =
          std::max(red_df, (size_t)2 * GR * (4 * ta_n + 4 * tb_n + 4) * (sizeof(double) + sizeof(float)));
      static bool attr_df = false;
      if (!attr_df)
        attr_df = cudaFuncSetAttribute(gram_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) ==
                  cudaSuccess;
      note_launch(), gram_df_kernel<<<nblk, nth_df, shm_df, s>>>(n, p, nb2, A, lda, B1, B2, ldb, part, G_df, up);
      const int tot = p * p * nb2;
      note_launch(), gram_reduce_kernel<<<(tot + 31) / 32, dim3(32, 8), 0, s>>>(nblk, tot, p * p, part, G1, G2);
      return;
    }
  }
  if (G == 1)
    note_launch(), gram_kernel<T, 1><<<nblk, nth, shm, s>>>(n, p, nb2, A, lda, B1, B2, ldb, part, G);
  else
    note_launch(), gram_kernel<T><<<nblk, nth, shm, s>>>(n, p, nb2, A, lda, B1, B2, ldb, part, G);
  const int tot = p * p * nb2;
  note_launch(), gram_reduce_kernel<<<(tot + 31) / 32, dim3(32, 8), 0, s>>>(nblk, tot, p * p, part, G1, G2);
}
template void launch_gram<float>(long long, int, int, const float*, long long, const float*, const float*, long long,
                                 double*, double*, double*, cudaStream_t, bool);
template void launch_gram<double>(long long, int, int, const double*, long long, const double*, const double*,
                                  long long, double*, double*, double*, cudaStream_t, bool);

// Row-wise block combination, safe in place: each row of A is read completely into
// registers by one thread before any output of the row is written. Y = A C with A n x p
// (lda), C p x q column-major (staged in shared memory with rows padded to a multiple of 4);
// output columns j < q1 go to Y1 (ldy), columns j >= q1 to Y2 (ldy). PMAX >= p.
// blockIdx.y selects one of several equally laid out block sets (A, Y1, Y2 offset by bstride
// elements each): LOBPCG combines the S, H S and M S blocks with one C in one launch.
template <class T, int PMAX>
__global__ void __launch_bounds__(256) combine_kernel(long long n, int p, int q, int q1, const T* A, long long lda,
                                                      const T* C, T* Y1, T* Y2, long long ldy, long long bstride) {
  extern __shared__ __align__(16) unsigned char sc_raw[];
  A += blockIdx.y * bstride;
  Y1 += blockIdx.y * bstride;
  Y2 += blockIdx.y * bstride;
  T* sC = reinterpret_cast<T*>(sc_raw);  // [q][pp]
  const int pp = (p + 3) & ~3;
  for (int t = threadIdx.x; t < pp * q; t += blockDim.x) {
    const int j = t / pp, i = t % pp;
    sC[t] = i < p ? C[j * p + i] : T(0);
  }
  __syncthreads();
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
    T a[PMAX];
#pragma unroll
    for (int i = 0; i < PMAX; ++i) a[i] = i < p ? A[i * lda + r] : T(0);
    for (int j = 0; j < q; ++j) {
      const T* cj = sC + j * pp;
      T s = T(0);
#pragma unroll
      for (int i = 0; i < PMAX; i += 4) {
        if (i < pp) {
          T c4[4];
          gram_ld4(cj + i, c4);  // 16-byte aligned: pp is a multiple of 4
          s += a[i] * c4[0] + a[i + 1] * c4[1];
          s += a[i + 2] * c4[2] + a[i + 3] * c4[3];
        }
      }
      if (j < q1)
        Y1[j * ldy + r] = s;
      else
        Y2[(j - q1) * ldy + r] = s;
    }
  }
}

// combine_kernel for FP64 blocks in double-float arithmetic: C is split into hi and lo float
// tables in shared memory, each thread splits its row of A once, and every output is a
// double-float dot product rounded to FP64 at the end. Four outputs are formed together so that
// four independent two-sum chains interleave.
template <int PMAX>
__global__ void __launch_bounds__(256, 2) combine_df_kernel(long long n, int p, int q, int q1, const double* A,
                                                         long long lda, const double* C, double* Y1, double* Y2,
                                                         long long ldy, long long bstride) {
  extern __shared__ __align__(16) unsigned char sc_raw[];
  A += blockIdx.y * bstride;
  Y1 += blockIdx.y * bstride;
  Y2 += blockIdx.y * bstride;
  const int pp = (p + 3) & ~3;
  const int qq = (q + 3) & ~3;
  float* sCh = reinterpret_cast<float*>(sc_raw);  // [qq][pp], zero beyond p and q
  float* sCl = sCh + (size_t)pp * qq;
  for (int t = threadIdx.x; t < pp * qq; t += blockDim.x) {
    const int j = t / pp, i = t % pp;
    df_split(i < p && j < q ? C[j * p + i] : 0.0, sCh[t], sCl[t]);
  }
  __syncthreads();
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
    float ah[PMAX], al[PMAX];
#pragma unroll
    for (int i = 0; i < PMAX; ++i) df_split_i(i < p ? A[i * lda + r] : 0.0, ah[i], al[i]);
    for (int j0 = 0; j0 < q; j0 += 4) {
      float sh[4] = {0.0f, 0.0f, 0.0f, 0.0f}, sl[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int i = 0; i < PMAX; i += 4) {
        if (i < pp) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            float ch[4], cl[4];  // 16-byte aligned loads: pp is a multiple of 4
            gram_ld4(sCh + (j0 + u) * pp + i, ch);
            gram_ld4(sCl + (j0 + u) * pp + i, cl);
#pragma unroll
            for (int w = 0; w < 4; ++w) df_mac(sh[u], sl[u], ah[i + w], al[i + w], ch[w], cl[w]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = j0 + u;
        if (j >= q) break;
        const double y = df_join(sh[u], sl[u]);
        if (j < q1)
          Y1[j * ldy + r] = y;
        else
          Y2[(j - q1) * ldy + r] = y;
      }
    }
  }
}

template <class T>
void launch_combine(long long n, int p, int q, int q1, const T* A, long long lda, const T* C, T* Y1, T* Y2,
                    long long ldy, cudaStream_t s, int nbase, long long bstride) {
  const size_t shm = (size_t)((p + 3) & ~3) * q * sizeof(T);
  const dim3 grid(dblocks(n), std::max(1, nbase));
  if constexpr (std::is_same<T, double>::value) {
    if (dense_df()) {  // hi and lo float tables, q padded to a multiple of 4
      const size_t shm_df = (size_t)((p + 3) & ~3) * ((q + 3) & ~3) * 2 * sizeof(float);
      if (p <= 16)
        note_launch(), combine_df_kernel<16><<<grid, 256, shm_df, s>>>(n, p, q, q1, A, lda, C, Y1, Y2, ldy, bstride);
      else if (p <= 32)
        note_launch(), combine_df_kernel<32><<<grid, 256, shm_df, s>>>(n, p, q, q1, A, lda, C, Y1, Y2, ldy, bstride);
      else if (p <= 48)
        note_launch(), combine_df_kernel<48><<<grid, 256, shm_df, s>>>(n, p, q, q1, A, lda, C, Y1, Y2, ldy, bstride);
      else
        note_launch(), combine_df_kernel<64><<<grid, 256, shm_df, s>>>(n, p, q, q1, A, lda, C, Y1, Y2, ldy, bstride);
      return;
    }
  }
  if (p <= 16)
    note_launch(), combine_kernel<T, 16><<<grid, 256, shm, s>>>(n, p, q, q1, A, lda, C, Y1, Y2, ldy, bstride);
  else if (p <= 32)
    note_launch(), combine_kernel<T, 32><<<grid, 256, shm, s>>>(n, p, q, q1, A, lda, C, Y1, Y2, ldy, bstride);
  else
    note_launch(), combine_kernel<T, 64><<<grid, 256, shm, s>>>(n, p, q, q1, A, lda, C, Y1, Y2, ldy, bstride);
}
template void launch_combine<float>(long long, int, int, int, const float*, long long, const float*, float*, float*,
                                    long long, cudaStream_t, int, long long);
template void launch_combine<double>(long long, int, int, int, const double*, long long, const double*, double*,
                                     double*, long long, cudaStream_t, int, long long);

// LOBPCG update of the block sets [X | W | P] (nb columns each, columns at stride ld; blockIdx.y
// selects S, H S or M S, bstride elements apart): with Z = [W P] (the nz = nuse - nb columns after
// X) and the first nb Ritz vectors' coefficients C (nuse x nb, column-major) split into the X rows
// Cx and the Z rows Cz,
//   P' = Z Cz   and   X' = X Cx + P'
// written in place over P (block 2) and X (block 0). This is X' = [X W P] C with the P' products
// shared, about half the products of forming X' and P' separately. Each row is read completely
// into registers before any output of the row is written; four outputs are formed together.
template <class T, int NBX, int NZX>
__global__ void __launch_bounds__(256) lobpcg_update_kernel(long long n, int nb, int nz, T* S, long long ld,
                                                            const T* C, long long bstride) {
  extern __shared__ __align__(16) unsigned char su_raw[];
  S += blockIdx.y * bstride;
  const int px = (nb + 3) & ~3, pz = (nz + 3) & ~3, nq = (nb + 3) & ~3, nuse = nb + nz;
  T* sCx = reinterpret_cast<T*>(su_raw);  // [nq][px], zero beyond nb
  T* sCz = sCx + (size_t)nq * px;         // [nq][pz], zero beyond nz
  for (int t = threadIdx.x; t < nq * px; t += blockDim.x) {
    const int j = t / px, i = t % px;
    sCx[t] = (i < nb && j < nb) ? C[j * nuse + i] : T(0);
  }
  for (int t = threadIdx.x; t < nq * pz; t += blockDim.x) {
    const int j = t / pz, i = t % pz;
    sCz[t] = (i < nz && j < nb) ? C[j * nuse + nb + i] : T(0);
  }
  __syncthreads();
  T* X = S;
  T* P = S + 2 * (long long)nb * ld;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
    T ax[NBX], az[NZX];
#pragma unroll
    for (int i = 0; i < NBX; ++i) ax[i] = i < nb ? X[i * ld + r] : T(0);
#pragma unroll
    for (int i = 0; i < NZX; ++i) az[i] = i < nz ? S[(nb + i) * ld + r] : T(0);
    for (int j0 = 0; j0 < nb; j0 += 4) {
      T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
      for (int i = 0; i < NZX; i += 4) {
        if (i < pz) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            T c4[4];
            gram_ld4(sCz + (j0 + u) * pz + i, c4);  // 16-byte aligned: pz is a multiple of 4
            acc[u] += az[i] * c4[0] + az[i + 1] * c4[1];
            acc[u] += az[i + 2] * c4[2] + az[i + 3] * c4[3];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (j0 + u < nb) P[(j0 + u) * ld + r] = acc[u];
#pragma unroll
      for (int i = 0; i < NBX; i += 4) {
        if (i < px) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            T c4[4];
            gram_ld4(sCx + (j0 + u) * px + i, c4);
            acc[u] += ax[i] * c4[0] + ax[i + 1] * c4[1];
            acc[u] += ax[i + 2] * c4[2] + ax[i + 3] * c4[3];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (j0 + u < nb) X[(j0 + u) * ld + r] = acc[u];
    }
  }
}

// lobpcg_update_kernel for FP64 blocks in double-float arithmetic (C split into hi and lo float
// tables, each row split once; X' continues P's unrounded double-float sums).
template <int NBX, int NZX>
__global__ void __launch_bounds__(256, (NBX <= 12 ? 2 : 1)) lobpcg_update_df_kernel(long long n, int nb, int nz, double* S,
                                                                long long ld, const double* C, long long bstride) {
  extern __shared__ __align__(16) unsigned char su_raw[];
  S += blockIdx.y * bstride;
  const int px = (nb + 3) & ~3, pz = (nz + 3) & ~3, nq = (nb + 3) & ~3, nuse = nb + nz;
  float* sCxh = reinterpret_cast<float*>(su_raw);  // [nq][px]
  float* sCxl = sCxh + (size_t)nq * px;
  float* sCzh = sCxl + (size_t)nq * px;            // [nq][pz]
  float* sCzl = sCzh + (size_t)nq * pz;
  // the next row of each thread, staged by cp.async while the current one is combined:
  // [NBX + NZX][blockDim.x] doubles (column-major over the threads: conflict-free accesses)
  double* stg = reinterpret_cast<double*>(su_raw + (((size_t)nq * (px + pz) * 2 * sizeof(float) + 15) & ~(size_t)15));
  for (int t = threadIdx.x; t < nq * px; t += blockDim.x) {
    const int j = t / px, i = t % px;
    df_split((i < nb && j < nb) ? C[j * nuse + i] : 0.0, sCxh[t], sCxl[t]);
  }
  for (int t = threadIdx.x; t < nq * pz; t += blockDim.x) {
    const int j = t / pz, i = t % pz;
    df_split((i < nz && j < nb) ? C[j * nuse + nb + i] : 0.0, sCzh[t], sCzl[t]);
  }
  __syncthreads();
  double* X = S;
  double* P = S + 2 * (long long)nb * ld;
  const int tid = threadIdx.x, bd = blockDim.x;
  const long long stride = (long long)gridDim.x * bd;
  auto prefetch = [&](long long row) {
    if (row < n) {
      for (int i = 0; i < nb; ++i) gram_cp<double>(stg + (size_t)i * bd + tid, X + i * ld + row, true);
      for (int i = 0; i < nz; ++i) gram_cp<double>(stg + (size_t)(NBX + i) * bd + tid, S + (nb + i) * ld + row, true);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  long long r = blockIdx.x * (long long)bd + tid;
  prefetch(r);
  for (; r < n; r += stride) {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    // this thread's staged row into registers (padding columns are zeros without a split: a zero
    // would take the FP64 conversion), then the next row's copies into the freed stage (issue is
    // in order, so they start after these reads have completed)
    float axh[NBX], axl[NBX], azh[NZX], azl[NZX];
#pragma unroll
    for (int i = 0; i < NBX; ++i) {
      axh[i] = axl[i] = 0.0f;
      if (i < nb) df_split_i(stg[(size_t)i * bd + tid], axh[i], axl[i]);
    }
#pragma unroll
    for (int i = 0; i < NZX; ++i) {
      azh[i] = azl[i] = 0.0f;
      if (i < nz) df_split_i(stg[(size_t)(NBX + i) * bd + tid], azh[i], azl[i]);
    }
    prefetch(r + stride);
    for (int j0 = 0; j0 < nb; j0 += 4) {
      float sh[4] = {0.0f, 0.0f, 0.0f, 0.0f}, sl[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int i = 0; i < NZX; i += 4) {
        if (i < pz) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            float ch[4], cl[4];
            gram_ld4(sCzh + (j0 + u) * pz + i, ch);
            gram_ld4(sCzl + (j0 + u) * pz + i, cl);
#pragma unroll
            for (int w = 0; w < 4; ++w) df_mac(sh[u], sl[u], azh[i + w], azl[i + w], ch[w], cl[w]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (j0 + u < nb) P[(j0 + u) * ld + r] = df_join(sh[u], sl[u]);
#pragma unroll
      for (int i = 0; i < NBX; i += 4) {
        if (i < px) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            float ch[4], cl[4];
            gram_ld4(sCxh + (j0 + u) * px + i, ch);
            gram_ld4(sCxl + (j0 + u) * px + i, cl);
#pragma unroll
            for (int w = 0; w < 4; ++w) df_mac(sh[u], sl[u], axh[i + w], axl[i + w], ch[w], cl[w]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (j0 + u < nb) X[(j0 + u) * ld + r] = df_join(sh[u], sl[u]);
    }
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <class T>
void launch_lobpcg_update(long long n, int nb, int nz, T* S, long long ld, const T* C, cudaStream_t s, int nbase,
                          long long bstride) {
  const int px = (nb + 3) & ~3, pz = (nz + 3) & ~3, nq = (nb + 3) & ~3;
  const dim3 grid(dblocks(n), std::max(1, nbase));
  const bool small = nb <= 12 && nz <= 24;
  if constexpr (std::is_same<T, double>::value) {
    if (dense_df()) {
      // persistent: one wave of resident blocks over the nbase block sets, each thread walking
      // rows with the next one staged in shared memory
      const size_t tab = (((size_t)nq * (px + pz) * 2 * sizeof(float) + 15) & ~(size_t)15);
      const size_t shm = tab + (size_t)(small ? 36 : 60) * 256 * sizeof(double);
      static bool attr = false;
      if (!attr)  // a failure shows as the launch's error, which the callers check
        attr = cudaFuncSetAttribute(lobpcg_update_df_kernel<12, 24>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    100 * 1024) == cudaSuccess &&
               cudaFuncSetAttribute(lobpcg_update_df_kernel<20, 40>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    150 * 1024) == cudaSuccess;
      const long long rows = (n + 255) / 256;
      const int per_sm = small ? 2 : 1;
      const int gx = (int)std::max<long long>(1, std::min<long long>(rows, (long long)152 * per_sm / std::max(1, nbase)));
      const dim3 pgrid(gx, std::max(1, nbase));
      if (small)
        note_launch(), lobpcg_update_df_kernel<12, 24><<<pgrid, 256, shm, s>>>(n, nb, nz, S, ld, C, bstride);
      else
        note_launch(), lobpcg_update_df_kernel<20, 40><<<pgrid, 256, shm, s>>>(n, nb, nz, S, ld, C, bstride);
      return;
    }
  }
  const size_t shm = (size_t)nq * (px + pz) * sizeof(T);
  if (small)
    note_launch(), lobpcg_update_kernel<T, 12, 24><<<grid, 256, shm, s>>>(n, nb, nz, S, ld, C, bstride);
  else
    note_launch(), lobpcg_update_kernel<T, 20, 40><<<grid, 256, shm, s>>>(n, nb, nz, S, ld, C, bstride);
}
template void launch_lobpcg_update<float>(long long, int, int, float*, long long, const float*, cudaStream_t, int,
                                          long long);
template void launch_lobpcg_update<double>(long long, int, int, double*, long long, const double*, cudaStream_t, int,
                                           long long);

template <class T>
__global__ void __launch_bounds__(256) move_cols_kernel(long long n, T* S, long long ld, const ColMoves mv,
                                                        long long bstride) {
  S += blockIdx.y * bstride;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
    T v[40];
#pragma unroll
    for (int t = 0; t < 40; ++t)
      if (t < mv.n) v[t] = S[mv.src[t] * ld + r];
#pragma unroll
    for (int t = 0; t < 40; ++t)
      if (t < mv.n) S[mv.dst[t] * ld + r] = v[t];
  }
}

template <class T>
void launch_move_cols(long long n, T* S, long long ld, const ColMoves& mv, cudaStream_t s, int nbase,
                      long long bstride) {
  if (mv.n <= 0 || mv.n > 40) return;  // the caller checks n <= 40
  note_launch(), move_cols_kernel<T><<<dim3(dblocks(n), std::max(1, nbase)), 256, 0, s>>>(n, S, ld, mv, bstride);
}
template void launch_move_cols<float>(long long, float*, long long, const ColMoves&, cudaStream_t, int, long long);
template void launch_move_cols<double>(long long, double*, long long, const ColMoves&, cudaStream_t, int, long long);

// R[:, j] = HX[:, j] - lam_j MX[:, j]; W[:, j] = dinv o R[:, j]; norms[2j] += |R_j|^2,
// norms[2j+1] += |MX_j|^2 (FP64 sums per thread, reduced per block, one atomic per block).
template <class T, int MB>
__global__ void __launch_bounds__(256, 2) residual_block_kernel(long long n, int m, const T* HX, const T* MX,
                                                             long long ld, const double* lam, const T* dinv, T* W,
                                                             double* norms) {
  // one pass over the rows for all m <= MB columns: each thread's sums for every column stay in
  // registers, then one block reduction and 2m atomics per block. A thread's sums (a few rows) and
  // the warp's reduction stay in the storage precision, the warps' partials are added in FP64: on
  // this part FP64 arithmetic and the FP32 to FP64 conversions run on the narrow FP64 pipe, which
  // per-element or per-lane FP64 work would make the bound of this kernel.
  __shared__ double red[2 * MB][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T r2[MB], m2[MB];
  T l[MB];
#pragma unroll
  for (int j = 0; j < MB; ++j) {
    r2[j] = T(0);
    m2[j] = T(0);
    l[j] = j < m ? (T)lam[j] : T(0);
  }
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
    const T dr = dinv ? dinv[r] : T(1);
#pragma unroll
    for (int j = 0; j < MB; ++j) {
      if (j < m) {
        const T mx = MX[j * ld + r];
        const T res = HX[j * ld + r] - l[j] * mx;
        W[j * ld + r] = dinv ? dr * res : res;
        r2[j] += res * res;
        m2[j] += mx * mx;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < MB; ++j) {
    if (j < m) {
      T a = r2[j], b = m2[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(FULL_MASK, a, o);
        b += __shfl_xor_sync(FULL_MASK, b, o);
      }
      if (lane == 0) {
        red[2 * j][warp] = (double)a;
        red[2 * j + 1][warp] = (double)b;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 * m) {
    double a = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += red[threadIdx.x][w];
    atomicAdd(norms + threadIdx.x, a);
  }
}

template <class T>
void launch_residual_block(long long n, int m, const T* HX, const T* MX, long long ld, const double* lam,
                           const T* dinv, T* W, double* norms, cudaStream_t s) {
  // one block per SM at least (the loads of a thread's rows are its only latency cover), up to
  // two resident blocks per SM with eight rows per thread or more (the reductions cost as much as
  // a few rows)
  const int nb = (int)std::max<long long>(std::min<long long>(152, (n + 255) / 256),
                                          std::min<long long>(2 * 152, (n + 2047) / 2048));
  if (m <= 12)
    note_launch(), residual_block_kernel<T, 12><<<nb, 256, 0, s>>>(n, m, HX, MX, ld, lam, dinv, W, norms);
  else
    note_launch(), residual_block_kernel<T, 20><<<nb, 256, 0, s>>>(n, m, HX, MX, ld, lam, dinv, W, norms);
}
template void launch_residual_block<float>(long long, int, const float*, const float*, long long, const double*,
                                           const float*, float*, double*, cudaStream_t);
template void launch_residual_block<double>(long long, int, const double*, const double*, long long, const double*,
                                            const double*, double*, double*, cudaStream_t);

// Block Chebyshev-Jacobi preconditioner of LOBPCG, column by column the recurrence of the
// PCG preconditioner: z = p(D^-1 H) D^-1 r on the interval [theta - delta, theta + delta]
// of D^-1 H. Init: w = r, d = D^-1 r / theta, z = d; step: w -= H d,
// d = c1 d + c2 D^-1 w, z += d. Elementwise, so z may alias r.
template <class T>
__global__ void cheb_block_init_kernel(long long n, int m, long long ld, const T* R, const T* dinv, T inv_theta,
                                       T* Wb, T* Db, T* Zb) {
  const long long tot = n * (long long)m;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const long long r = t % n, idx = (t / n) * ld + r;
    const T rv = R[idx];
    const T d = dinv[r] * rv * inv_theta;
    Wb[idx] = rv;
    Db[idx] = d;
    Zb[idx] = d;
  }
}
template <class T>
__global__ void cheb_block_step_kernel(long long n, int m, long long ld, const T* HD, const T* dinv, T c1, T c2,
                                       T* Wb, T* Db, T* Zb) {
  const long long tot = n * (long long)m;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const long long r = t % n, idx = (t / n) * ld + r;
    const T w = Wb[idx] - HD[idx];
    const T d = c1 * Db[idx] + c2 * dinv[r] * w;
    Wb[idx] = w;
    Db[idx] = d;
    Zb[idx] += d;
  }
}
template <class T>
void launch_cheb_block_init(long long n, int m, long long ld, const T* R, const T* dinv, double inv_theta, T* W,
                            T* D, T* Z, cudaStream_t s) {
  note_launch(), cheb_block_init_kernel<T><<<dblocks(n * m), DT, 0, s>>>(n, m, ld, R, dinv, (T)inv_theta, W, D, Z);
}
template <class T>
void launch_cheb_block_step(long long n, int m, long long ld, const T* HD, const T* dinv, double c1, double c2,
                            T* W, T* D, T* Z, cudaStream_t s) {
  note_launch(), cheb_block_step_kernel<T><<<dblocks(n * m), DT, 0, s>>>(n, m, ld, HD, dinv, (T)c1, (T)c2, W, D, Z);
}
template void launch_cheb_block_init<float>(long long, int, long long, const float*, const float*, double, float*,
                                            float*, float*, cudaStream_t);
template void launch_cheb_block_step<float>(long long, int, long long, const float*, const float*, double, double,
                                            float*, float*, float*, cudaStream_t);

// One power step for the largest eigenvalue of D^-1 H on the interior nodes (dinv > 0):
// vn = D^-1 H v, acc[0] += v.Hv, acc[1] += v.D v, acc[2] += |vn|^2.
template <class T>
__global__ void power_sub_kernel(long long n, const T* v, const T* Hv, const T* dinv, T* vn, double* acc) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
    const double di = (double)dinv[r];
    if (di > 0.0) {
      const double x = (double)v[r], y = (double)Hv[r], z = di * y;
      vn[r] = (T)z;
      a0 += x * y;
      a1 += x * x / di;
      a2 += z * z;
    } else {
      vn[r] = T(0);
    }
  }
  a0 = warp_sum(a0);
  a1 = warp_sum(a1);
  a2 = warp_sum(a2);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(acc, a0);
    atomicAdd(acc + 1, a1);
    atomicAdd(acc + 2, a2);
  }
}
template <class T>
void launch_power_sub(long long n, const T* v, const T* Hv, const T* dinv, T* vn, double* acc, cudaStream_t s) {
  note_launch(), power_sub_kernel<T><<<std::min(dblocks(n), 2 * 152), DT, 0, s>>>(n, v, Hv, dinv, vn, acc);
}
template void launch_power_sub<float>(long long, const float*, const float*, const float*, float*, double*,
                                      cudaStream_t);

// Counter-based pseudo-random start block (SplitMix64 finalizer of the index), interior nodes only.
template <class T>
__global__ void random_block_kernel(long long n, int m, long long ld, const unsigned char* interior, uint64_t seed,
                                    T* X) {
  const long long total = n * (long long)m;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long r = t % n;
    const int j = (int)(t / n);
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(t + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    X[j * ld + r] = interior[r] ? (T)u : T(0);
  }
}

// Smooth starting block: column j is the box mode sin(pi a x) sin(pi b y) sin(pi c z) (a, b, c =
// modes[j], x, y, z the node's fractional position in the nx x ny x nz-element box) plus eps times
// the random entries of random_block_kernel, on interior nodes.
template <class T>
__global__ void box_mode_block_kernel(long long n, int m, long long ld, int nx, int ny, int nz, BoxModes modes,
                                      double eps, const unsigned char* interior, uint64_t seed, T* X) {
  const long long total = n * (long long)m;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long r = t % n;
    const int j = (int)(t / n);
    const int i = (int)(r % (nx + 1)), jy = (int)((r / (nx + 1)) % (ny + 1)), k = (int)(r / ((long long)(nx + 1) * (ny + 1)));
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(t + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    // a starting guess: FP32 (the FP64 sine runs on the FP64 pipe)
    const float v = sinpif((float)(modes.a[j] * i) / nx) * sinpif((float)(modes.b[j] * jy) / ny) *
                    sinpif((float)(modes.c[j] * k) / nz);
    X[j * ld + r] = interior[r] ? (T)(v + eps * u) : T(0);
  }
}

template <class T>
void launch_box_mode_block(long long n, int m, long long ld, int nx, int ny, int nz, const BoxModes& modes, double eps,
                           const unsigned char* interior, uint64_t seed, T* X, cudaStream_t s) {
  note_launch(), box_mode_block_kernel<T><<<dblocks(n * m), DT, 0, s>>>(n, m, ld, nx, ny, nz, modes, eps, interior,
                                                                          seed, X);
}
template void launch_box_mode_block<float>(long long, int, long long, int, int, int, const BoxModes&, double,
                                           const unsigned char*, uint64_t, float*, cudaStream_t);

template <class T>
void launch_random_block(long long n, int m, long long ld, const unsigned char* interior, uint64_t seed, T* X,
                         cudaStream_t s) {
  note_launch(), random_block_kernel<T><<<dblocks(n * m), DT, 0, s>>>(n, m, ld, interior, seed, X);
}
template void launch_random_block<float>(long long, int, long long, const unsigned char*, uint64_t, float*,
                                         cudaStream_t);
template void launch_random_block<double>(long long, int, long long, const unsigned char*, uint64_t, double*,
                                          cudaStream_t);

}  // namespace qcad
