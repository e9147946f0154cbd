// Effective-mass Schrodinger operators on the quantum subdomain and the dense
// block kernels of LOBPCG. Sec. II.B (Eqs. SchrodEqn, SchrodEqnWeakForm,
// Schrodinger3D) with the potential energy of Eq. SchrodPotEnergy (no V_xc).
#include <cuda_runtime.h>

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
                                 const double* hy, const double* hz, T* cV, double* vmin) {
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
      const double V = V0 - q[s];
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
                      const double* hz, T* cV, double* vmin, cudaStream_t s) {
  const long long ne = (long long)sm.nxs * sm.nys * sm.nzs;
  note_launch(), potential_kernel<T><<<dblocks(ne), DT, 0, s>>>(sm, phi, V0, hx, hy, hz, cV, vmin);
}
template void launch_potential<float>(const SubdomainMap&, const double*, double, const double*, const double*,
                                      const double*, float*, double*, cudaStream_t);
template void launch_potential<double>(const SubdomainMap&, const double*, double, const double*, const double*,
                                       const double*, double*, double*, cudaStream_t);

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

// G[p x q] (+)= A^T B for column-major A (n x p, lda) and B (n x q, ldb). Each thread sums
// a 32-row tile in the storage precision T and accumulates tiles in FP64; blocks add
// their partials atomically. Output row-major (o = a*q + b); all uses are symmetric.
constexpr int GR = 32;
template <class T>
__global__ void __launch_bounds__(256) gram_kernel(long long n, int p, int q, const T* A, long long lda,
                                                   const T* B, long long ldb, double* G) {
  extern __shared__ __align__(16) unsigned char sh_raw[];
  T* sh = reinterpret_cast<T*>(sh_raw);
  T* sA = sh;             // [p][GR]
  T* sB = sh + p * GR;    // [q][GR]
  const int nout = p * q;
  const int per = (nout + blockDim.x - 1) / blockDim.x;
  double acc[16];
  for (int s = 0; s < 16; ++s) acc[s] = 0.0;
  for (long long r0 = (long long)blockIdx.x * GR; r0 < n; r0 += (long long)gridDim.x * GR) {
    __syncthreads();
    for (int t = threadIdx.x; t < (p + q) * GR; t += blockDim.x) {
      const int col = t / GR, rr = t % GR;
      const long long row = r0 + rr;
      T v = T(0);
      if (row < n) v = col < p ? A[col * lda + row] : B[(col - p) * ldb + row];
      sh[col * GR + rr] = v;
    }
    __syncthreads();
    for (int s = 0; s < per && s < 16; ++s) {
      const int o = threadIdx.x + s * blockDim.x;
      if (o < nout) {
        const int a = o / q, b = o % q;
        T sum = T(0);
#pragma unroll 8
        for (int rr = 0; rr < GR; ++rr) sum += sA[a * GR + rr] * sB[b * GR + rr];
        acc[s] += (double)sum;
      }
    }
  }
  for (int s = 0; s < per && s < 16; ++s) {
    const int o = threadIdx.x + s * blockDim.x;
    if (o < nout && acc[s] != 0.0) atomicAdd(G + o, acc[s]);
  }
}

template <class T>
void launch_gram(long long n, int p, int q, const T* A, long long lda, const T* B, long long ldb, double* G,
                 cudaStream_t s) {
  const int nb = dblocks((n + GR - 1) / GR * DT);
  const size_t shm = (size_t)(p + q) * GR * sizeof(T);
  note_launch(), gram_kernel<T><<<nb, 256, shm, s>>>(n, p, q, A, lda, B, ldb, G);
}
template void launch_gram<float>(long long, int, int, const float*, long long, const float*, long long, double*,
                                 cudaStream_t);
template void launch_gram<double>(long long, int, int, const double*, long long, const double*, long long, double*,
                                  cudaStream_t);

// Row-wise block combination, safe in place: each row is read completely by one thread
// before it is written. Y = A C with A n x p (lda), C p x q column-major; output
// columns j < q1 go to Y1 (ldy), columns j >= q1 to Y2 (ldy).
template <class T>
__global__ void combine_kernel(long long n, int p, int q, int q1, const T* A, long long lda, const T* C, T* Y1,
                               T* Y2, long long ldy) {
  extern __shared__ __align__(16) unsigned char sc_raw[];
  T* sC = reinterpret_cast<T*>(sc_raw);
  for (int t = threadIdx.x; t < p * q; t += blockDim.x) sC[t] = C[t];
  __syncthreads();
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
    T a[QCAD_DENSE_MAXP];
    for (int i = 0; i < p; ++i) a[i] = A[i * lda + r];
    for (int j = 0; j < q; ++j) {
      T s = T(0);
      for (int i = 0; i < p; ++i) s += a[i] * sC[j * p + i];
      if (j < q1)
        Y1[j * ldy + r] = s;
      else
        Y2[(j - q1) * ldy + r] = s;
    }
  }
}

template <class T>
void launch_combine(long long n, int p, int q, int q1, const T* A, long long lda, const T* C, T* Y1, T* Y2,
                    long long ldy, cudaStream_t s) {
  note_launch(), combine_kernel<T><<<dblocks(n), DT, (size_t)p * q * sizeof(T), s>>>(n, p, q, q1, A, lda, C, Y1, Y2,
                                                                                   ldy);
}
template void launch_combine<float>(long long, int, int, int, const float*, long long, const float*, float*, float*,
                                    long long, cudaStream_t);
template void launch_combine<double>(long long, int, int, int, const double*, long long, const double*, double*,
                                     double*, long long, cudaStream_t);

// R[:, j] = HX[:, j] - lam_j MX[:, j]; W[:, j] = dinv o R[:, j]; norms2[j] += |R_j|^2, mnorm2[j] += |MX_j|^2.
template <class T>
__global__ void residual_block_kernel(long long n, int m, const T* HX, const T* MX, long long ld, const double* lam,
                                      const T* dinv, T* W, double* norms) {
  for (int j = 0; j < m; ++j) {
    double r2 = 0.0, m2 = 0.0;
    const T l = (T)lam[j];
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n;
         r += (long long)gridDim.x * blockDim.x) {
      const T mx = MX[j * ld + r];
      const T res = HX[j * ld + r] - l * mx;
      W[j * ld + r] = dinv[r] * res;
      r2 += (double)res * (double)res;
      m2 += (double)mx * (double)mx;
    }
    r2 = warp_sum(r2);
    m2 = warp_sum(m2);
    if ((threadIdx.x & 31) == 0) {
      if (r2 != 0.0) atomicAdd(norms + 2 * j, r2);
      if (m2 != 0.0) atomicAdd(norms + 2 * j + 1, m2);
    }
  }
}

template <class T>
void launch_residual_block(long long n, int m, const T* HX, const T* MX, long long ld, const double* lam,
                           const T* dinv, T* W, double* norms, cudaStream_t s) {
  note_launch(), residual_block_kernel<T><<<dblocks(n), DT, 0, s>>>(n, m, HX, MX, ld, lam, dinv, W, norms);
}
template void launch_residual_block<float>(long long, int, const float*, const float*, long long, const double*,
                                           const float*, float*, double*, cudaStream_t);
template void launch_residual_block<double>(long long, int, const double*, const double*, long long, const double*,
                                            const double*, double*, double*, cudaStream_t);

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
