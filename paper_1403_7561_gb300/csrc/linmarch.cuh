// Plane-factorized z-march for the linear operators y = K v + M_c v (separable
// Q1 stiffness plus the 2x2x2 Gauss-point mass term with stored per-element
// coefficients c; Sec. II.A.3, Eq. PoissonWeakForm linearized).
//
// The element-gather skeleton (qcad_internal.cuh) evaluates the quadrature
// interpolation B x B x B of every element from its eight corners. Here the
// interpolation is factorized over the structured grid instead: along x and y
// it is done once per node plane and shared by the two element layers that
// touch the plane, and the transposed interpolation is applied to the sum of
// the two layers' contributions. With B = [[a, b], [b, a]] (a, b the Gauss
// weights of the linear shape functions), for the element column (i, j):
//   X_k(qx)      = sum_a B[a][qx] v(i + a, j, k)            (per node row)
//   U_k(qx, qy)  = sum_b B[b][qy] X_k(qx) of row j + b      (per plane)
//   u(q)         = sum_c B[c][qz] U_{k+c}(qx, qy),  w = c_q u  (per element)
//   W_k(qx, qy)  = sum_qz B[0][qz] w_layer k + B[1][qz] w_layer k-1
// and the node value is the xy-transpose of W_k gathered from the four
// element columns around the node. The stiffness is the separable 27-point
// stencil of the element-gather skeleton (z from registers, y from registers
// or shared memory, x by shuffles).
//
// Thread layout: a block is 32 lanes (x, one node column each, the outer two a
// halo) by BY warps; each thread holds R consecutive node rows, so a tile has
// BY*R rows of which the first and the last are a halo. Row exchanges between
// warps go through double-buffered shared memory with one barrier per node
// plane; X of plane k+2 is published one plane ahead so that the barrier also
// serves the next plane's interpolation. The element coefficients of layer
// k+2 are copied to shared memory with cp.async while layer k is computed
// (three stages, zero fill outside the mesh), so they occupy no registers.
#pragma once

#include <type_traits>

#include "qcad_internal.cuh"

namespace qcad {

__device__ __forceinline__ void lin_cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}
// One element (4 or 8 bytes) global -> shared, asynchronous.
template <class T>
__device__ __forceinline__ void lin_cp_async_elem(T* smem, const T* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void lin_cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void lin_cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// The eight coefficients of one element from its 16-byte chunks (chunk h of lane l
// at p[32 h]: lanes of a chunk are contiguous, so reads are free of bank conflicts).
template <class T>
__device__ __forceinline__ void lin_lds_c8(const uint4* p, T* c);
template <>
__device__ __forceinline__ void lin_lds_c8<float>(const uint4* p, float* c) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  const float4 b = *reinterpret_cast<const float4*>(p + 32);
  c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w;
  c[4] = b.x; c[5] = b.y; c[6] = b.z; c[7] = b.w;
}
template <>
__device__ __forceinline__ void lin_lds_c8<double>(const uint4* p, double* c) {
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const double2 a = *reinterpret_cast<const double2*>(p + 32 * h);
    c[2 * h] = a.x;
    c[2 * h + 1] = a.y;
  }
}

// Packed row-exchange values (one shared access per pair or quadruple).
template <class T>
struct alignas(2 * sizeof(T)) LinV2 {
  T x, y;
};
template <class T>
struct alignas(16) LinV4 {
  T x, y, z, w;
};

// Dynamic shared memory: the row-exchange buffers (two parities of X, the upper-row
// gather and the stiffness z stage), the chunk's plane tables, three planes of raw inputs,
// then NST coefficient stages.
template <class T, int BY, int R>
struct LinShape {
  static constexpr int TR = BY * R;                  // node rows of a tile (incl. two halo rows)
  static constexpr int NCH = (8 * sizeof(T)) / 16;   // 16-byte chunks of one element's coefficients
  static constexpr int NST = 3;                      // coefficient stages in flight
  static constexpr int ZMAX = 128;                   // longest z chunk (plane tables held in shared memory)
  static constexpr size_t xch_bytes = (size_t)2 * BY * 32 * (2 * sizeof(LinV2<T>) + 2 * sizeof(LinV4<T>));
  static constexpr size_t zt_bytes = (size_t)(ZMAX + 1) * 12 * sizeof(T);
  static constexpr size_t vst_bytes = (size_t)3 * 2 * TR * 32 * sizeof(T);  // 3 planes x 2 raw inputs
  static constexpr size_t dyn_bytes = xch_bytes + zt_bytes + vst_bytes + (size_t)NST * TR * NCH * 32 * 16;
};

// Launch geometry (kchunk at most LinShape::ZMAX): x tiles of 30 interior nodes, y tiles of
// BY*R - 2 interior rows,
// (vector, z chunk) pairs along z.
inline dim3 lin_grid(int nxn, int nyn, int nzn, int by, int r, int kchunk, int nvec = 1) {
  const int tr = by * r;
  return dim3((nxn + 29) / 30, (nyn + tr - 3) / (tr - 2), ((nzn + kchunk - 1) / kchunk) * nvec);
}

// Op: the linear ops of pcg_ops.cuh (lin_in, lin_out, lin_dir, skip, set_vec, finish, coeffs),
// or an op with SEPM = true (m_scale, lin_out2), which writes the operator with zero Dirichlet
// rows and, as a second output, the separable consistent mass (Schrodinger H and M).
// Loads are unpredicated: node indices are clamped into the mesh (and into the chunk's
// planes), and every value read outside the operator's support meets a zero table entry or
// a zero coefficient, so only finiteness of the input matters there.
template <class T, int BY, int R, class Op>
__device__ __forceinline__ void lin_body(const Grid<T>& g, const Op& op_in, int kchunk, int bx, int by, int bz,
                                         unsigned char* dyn) {
  using S = LinShape<T, BY, R>;
  constexpr int TR = S::TR, NCH = S::NCH, NST = S::NST;
  if (op_in.skip()) return;
  const int nch = (g.nzn + kchunk - 1) / kchunk;
  Op op = op_in;
  op.set_vec(bz / nch);
  // [relative plane parity][...][BY][32]: X (qx = 0, 1) of each warp's first row; upper-row
  // gather (qx = 0, 1) of each warp's last row; stiffness z stage (3 fields + pad) of the first
  // and of the last row
  LinV2<T>(*xch_x)[BY][32] = reinterpret_cast<LinV2<T>(*)[BY][32]>(dyn);
  LinV2<T>(*xch_y)[BY][32] = xch_x + 2;
  LinV4<T>(*xch_s)[2][BY][32] = reinterpret_cast<LinV4<T>(*)[2][BY][32]>(xch_y + 2);
  T* zts = reinterpret_cast<T*>(dyn + S::xch_bytes);  // plane tables of planes k0 .. k1-1
  T* vst = reinterpret_cast<T*>(dyn + S::xch_bytes + S::zt_bytes);  // [3 planes][2 inputs][TR][32]
  uint4* cst = reinterpret_cast<uint4*>(dyn + S::xch_bytes + S::zt_bytes + S::vst_bytes);

  const int lane = threadIdx.x, ty = threadIdx.y;
  // neighbour warps, clamped: the tile's halo rows read their own warp (their results are unused)
  const int tyu = min(ty + 1, BY - 1), tyd = max(ty - 1, 0);
  const int i = bx * 30 - 1 + lane;
  const int jb = by * (TR - 2) - 1 + ty * R;
  const int k0 = (bz % nch) * kchunk;
  const int k1 = min(k0 + kchunk, g.nzn);
  const int kmax = min(k1, g.nzn - 1);  // last plane the chunk reads
  const int plane = (int)g.plane;
  const T A = GaussConst<T>::a(), B = GaussConst<T>::b();
  const T* __restrict__ cg = op.coeffs();
  const bool dov = op.lin_dir();

  const bool iin = i >= 0 && i < g.nxn;
  const bool iel = i >= 0 && i < g.nx;
  const int ic = min(max(i, 0), g.nxn - 1);
  T cmx[3], ckx[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    cmx[s] = iin ? g.mx[3 * i + s] : T(0);
    ckx[s] = iin ? g.kx[3 * i + s] : T(0);
  }
  T cmy[R][3], cky[R][3];
  bool wr[R], eok[R], top[R], bnd[R];
  int nrow[R], crow[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int j = jb + r;
    const int row = ty * R + r;
    const bool nin = iin && j >= 0 && j < g.nyn;
    const int jc = min(max(j, 0), g.nyn - 1);
    eok[r] = iel && j >= 0 && j < g.ny;
    wr[r] = nin && lane >= 1 && lane <= 30 && row >= 1 && row <= TR - 2;
    nrow[r] = ic + g.nxn * jc;
    crow[r] = eok[r] ? i + g.nx * j : 0;
    top[r] = dov && nin && g.dir_top != nullptr && g.dir_top[nrow[r]] != 0;
    bnd[r] = dov && g.dir_boundary && (i == 0 || j == 0 || i == g.nx || j == g.ny);
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      cmy[r][s] = nin ? g.my[3 * j + s] : T(0);
      cky[r][s] = nin ? g.ky[3 * j + s] : T(0);
    }
  }
  const int eplane = g.nx * g.ny;

  // one copy group: the raw inputs of node plane vplane (if >= 0; clamped into the chunk's
  // planes) and the coefficients of element layer `layer`, zeros where the element does not
  // exist (outside the mesh in x or y, or the layer above the top plane); layers the chunk
  // does not use are skipped
  auto issue = [&](int layer, int vplane) {
    if (vplane >= 0) {
      T* vs = vst + (size_t)(vplane % 3) * (2 * TR * 32);
      const int off = min(vplane, kmax) * plane;
#pragma unroll
      for (int q = 0; q < Op::NIN; ++q) {
        const T* src = op.lin_src(q);
#pragma unroll
        for (int r = 0; r < R; ++r) lin_cp_async_elem<T>(vs + (q * TR + ty * R + r) * 32 + lane, src + nrow[r] + off);
      }
    }
    if (layer >= 0 && layer < k1) {
      uint4* st = cst + (size_t)(layer % NST) * (TR * NCH * 32);
      const bool lok = layer < g.nz;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const bool ok = eok[r] && lok;
        const T* src = ok ? cg + 8 * ((size_t)crow[r] + (size_t)eplane * layer) : cg;
        uint4* dst = st + ((ty * R + r) * NCH) * 32 + lane;
#pragma unroll
        for (int h = 0; h < NCH; ++h) lin_cp_async16(dst + 32 * h, src + h * (16 / sizeof(T)), ok);
      }
    }
    lin_cp_commit();
  };
  auto loadv = [&](int r, int k) -> T { return op.lin_in(nrow[r] + min(max(k, 0), kmax) * plane); };
  auto xinterp = [&](T v, T* x) {
    const T vr = __shfl_down_sync(FULL_MASK, v, 1);
    x[0] = A * v + B * vr;
    x[1] = B * v + A * vr;
  };
  auto uinterp = [&](const T* xj, const T* xj1, T* u) {
    u[0] = A * xj[0] + B * xj1[0];
    u[1] = A * xj[1] + B * xj1[1];
    u[2] = B * xj[0] + A * xj1[0];
    u[3] = B * xj[1] + A * xj1[1];
  };

  // ---- prologue: planes k0-1 .. k0+2, interpolations of planes k0-1 .. k0+1, carry of layer k0-1
  issue(k0 - 1, -1);
  issue(k0, k0 + 3);
  issue(k0 + 1, k0 + 4);
  T vm[R], vc[R], vp[R], vq[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    vm[r] = loadv(r, k0 - 1);
    vc[r] = loadv(r, k0);
    vp[r] = loadv(r, k0 + 1);
    vq[r] = loadv(r, k0 + 2);
  }
  T Um[R][4], Uc[R][4], Un[R][4];
  {
    T X0[R][2], X1[R][2], X2[R][2];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      xinterp(vm[r], X0[r]);
      xinterp(vc[r], X1[r]);
      xinterp(vp[r], X2[r]);
    }
    for (int q = ty * 32 + lane; q < 12 * (k1 - k0); q += 32 * BY) zts[q] = g.zt[12 * k0 + q];
    // the stiffness buffer of parity 1: the first march step writes parity 0
    LinV4<T>(*pro)[BY][32] = xch_s[1];
    pro[0][ty][lane] = LinV4<T>{X0[0][0], X0[0][1], X1[0][0], X1[0][1]};
    pro[1][ty][lane] = LinV4<T>{X2[0][0], X2[0][1], T(0), T(0)};
    __syncthreads();
    const LinV4<T> p0 = pro[0][tyu][lane], p1 = pro[1][tyu][lane];
    const T A0[2] = {p0.x, p0.y};
    const T A1[2] = {p0.z, p0.w};
    const T A2[2] = {p1.x, p1.y};
#pragma unroll
    for (int r = 0; r < R; ++r) {
      uinterp(X0[r], r + 1 < R ? X0[r + 1 < R ? r + 1 : r] : A0, Um[r]);
      uinterp(X1[r], r + 1 < R ? X1[r + 1 < R ? r + 1 : r] : A1, Uc[r]);
      uinterp(X2[r], r + 1 < R ? X2[r + 1 < R ? r + 1 : r] : A2, Un[r]);
    }
  }
  T carry[R][4];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) carry[r][q] = T(0);
  if (k0 > 0) {
    lin_cp_wait<2>();
    const uint4* st = cst + (size_t)((k0 - 1) % NST) * (TR * NCH * 32);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      T c[8];
      lin_lds_c8<T>(st + ((ty * R + r) * NCH) * 32 + lane, c);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const T w0 = c[q] * (A * Um[r][q] + B * Uc[r][q]);
        const T w1 = c[q + 4] * (B * Um[r][q] + A * Uc[r][q]);
        carry[r][q] = B * w0 + A * w1;
      }
    }
  }

  // ---- one node plane k; P is the parity of k - k0 (selects the exchange buffers)
  auto step = [&](int k, auto Pc) {
    constexpr int P = decltype(Pc)::value;
    issue(k + 2, k + 5);
    typename Op::Pre pre[R];
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (wr[r]) pre[r] = op.lin_pre(nrow[r] + k * plane);
    // X of plane k+2; the first row's is published for the warp below
    T Xq[R][2];
#pragma unroll
    for (int r = 0; r < R; ++r) xinterp(vq[r], Xq[r]);
    xch_x[P][ty][lane] = LinV2<T>{Xq[0][0], Xq[0][1]};
    // element layer k: the lower corners feed plane k, the upper ones are carried to k+1
    // (the wait also completes the raw inputs of plane k+3)
    lin_cp_wait<2>();
    const uint4* st = cst + (size_t)(k % NST) * (TR * NCH * 32);
    T Ylo[R][2], Yhi[R][2];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      T c[8];
      lin_lds_c8<T>(st + ((ty * R + r) * NCH) * 32 + lane, c);
      T W[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const T w0 = c[q] * (A * Uc[r][q] + B * Un[r][q]);
        const T w1 = c[q + 4] * (B * Uc[r][q] + A * Un[r][q]);
        W[q] = carry[r][q] + A * w0 + B * w1;
        carry[r][q] = B * w0 + A * w1;
      }
      Ylo[r][0] = A * W[0] + B * W[2];
      Ylo[r][1] = A * W[1] + B * W[3];
      Yhi[r][0] = B * W[0] + A * W[2];
      Yhi[r][1] = B * W[1] + A * W[3];
    }
    xch_y[P][ty][lane] = LinV2<T>{Yhi[R - 1][0], Yhi[R - 1][1]};
    // stiffness, z stage
    T z[12];
    {
      const LinV4<T>* zp = reinterpret_cast<const LinV4<T>*>(zts + 12 * (k - k0));
#pragma unroll
      for (int h = 0; h < 3; ++h) {
        const LinV4<T> t4 = zp[h];
        z[4 * h] = t4.x;
        z[4 * h + 1] = t4.y;
        z[4 * h + 2] = t4.z;
        z[4 * h + 3] = t4.w;
      }
    }
    T ax[R], ay[R], az[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      ax[r] = z[0] * vm[r] + z[1] * vc[r] + z[2] * vp[r];
      ay[r] = z[3] * vm[r] + z[4] * vc[r] + z[5] * vp[r];
      az[r] = z[6] * vm[r] + z[7] * vc[r] + z[8] * vp[r];
    }
    xch_s[P][0][ty][lane] = LinV4<T>{ax[0], ay[0], az[0], T(0)};
    if (R > 1) xch_s[P][1][ty][lane] = LinV4<T>{ax[R - 1], ay[R - 1], az[R - 1], T(0)};
    __syncthreads();
    // neighbours across warps: the row above the last row, the row below the first row
    constexpr int LAST = R > 1 ? 1 : 0;
    const LinV2<T> xa2 = xch_x[P][tyu][lane], yb2 = xch_y[P][tyd][lane];
    const LinV4<T> sa4 = xch_s[P][0][tyu][lane], sb4 = xch_s[P][LAST][tyd][lane];
    const T Xa[2] = {xa2.x, xa2.y};
    const T Yb[2] = {yb2.x, yb2.y};
    const T sa[3] = {sa4.x, sa4.y, sa4.z};
    const T sb[3] = {sb4.x, sb4.y, sb4.z};
    const bool pdir = dov && ((g.dir_bottom && k == 0) || (g.dir_boundary && (k == 0 || k == g.nz)));
    const bool ptop = k == g.nz;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      // mass: the own element row and the row below gathered, then x
      const T yl0 = Ylo[r][0] + (r > 0 ? Yhi[r > 0 ? r - 1 : 0][0] : Yb[0]);
      const T yl1 = Ylo[r][1] + (r > 0 ? Yhi[r > 0 ? r - 1 : 0][1] : Yb[1]);
      const T own = A * yl0 + B * yl1;
      const T nxt = B * yl0 + A * yl1;
      const T mass = own + __shfl_up_sync(FULL_MASK, nxt, 1);
      // stiffness, y then x stage
      const T axm = r > 0 ? ax[r > 0 ? r - 1 : 0] : sb[0], axp = r + 1 < R ? ax[r + 1 < R ? r + 1 : r] : sa[0];
      const T aym = r > 0 ? ay[r > 0 ? r - 1 : 0] : sb[1], ayp = r + 1 < R ? ay[r + 1 < R ? r + 1 : r] : sa[1];
      const T azm = r > 0 ? az[r > 0 ? r - 1 : 0] : sb[2], azp = r + 1 < R ? az[r + 1 < R ? r + 1 : r] : sa[2];
      const T c1 = cmy[r][0] * axm + cmy[r][1] * ax[r] + cmy[r][2] * axp;
      const T d = cky[r][0] * aym + cky[r][1] * ay[r] + cky[r][2] * ayp + cmy[r][0] * azm + cmy[r][1] * az[r] +
                  cmy[r][2] * azp;
      const T c1m = __shfl_up_sync(FULL_MASK, c1, 1);
      const T c1p = __shfl_down_sync(FULL_MASK, c1, 1);
      const T dm = __shfl_up_sync(FULL_MASK, d, 1);
      const T dp = __shfl_down_sync(FULL_MASK, d, 1);
      const T stiff = ckx[0] * c1m + ckx[1] * c1 + ckx[2] * c1p + cmx[0] * dm + cmx[1] * d + cmx[2] * dp;
      const bool isdir = pdir || bnd[r] || (ptop && top[r]);
      if constexpr (Op::SEPM) {
        // second output: the separable consistent mass Mx My Mz v (the x stage of c1 rescaled)
        const T mm = op.m_scale() * (cmx[0] * c1m + cmx[1] * c1 + cmx[2] * c1p);
        if (wr[r]) op.lin_out2(nrow[r] + k * plane, isdir ? T(0) : stiff + mass, isdir ? T(0) : mm);
      } else {
        const T y = isdir ? vc[r] : stiff + mass;
        if (wr[r]) op.lin_out(nrow[r] + k * plane, pre[r], vc[r], y);
      }
    }
    // interpolation of plane k+2 for the next layer, then shift the plane window (plane k+3
    // from its stage)
    const T* vs = vst + (size_t)((k + 3) % 3) * (2 * TR * 32);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const T x0 = vs[(ty * R + r) * 32 + lane];
      const T x1 = Op::NIN > 1 ? vs[(TR + ty * R + r) * 32 + lane] : T(0);
      const T vnew = op.lin_mix(x0, x1);
      T Uq[4];
      uinterp(Xq[r], r + 1 < R ? Xq[r + 1 < R ? r + 1 : r] : Xa, Uq);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        Uc[r][q] = Un[r][q];
        Un[r][q] = Uq[q];
      }
      vm[r] = vc[r];
      vc[r] = vp[r];
      vp[r] = vq[r];
      vq[r] = vnew;
    }
  };

  // ---- march over node planes k0 .. k1-1, two planes per trip (compile-time buffer parity)
  int k = k0;
  for (; k + 1 < k1; k += 2) {
    step(k, std::integral_constant<int, 0>());
    step(k + 1, std::integral_constant<int, 1>());
  }
  if (k < k1) step(k, std::integral_constant<int, 0>());
  lin_cp_wait<0>();
  op.finish();
}

// Resident blocks per SM the register allocation is held to: 32 warps per SM for FP32 with one
// row per thread, 20 with two, 16 (FP64, one row) and at least one block otherwise.
template <class T, int BY, int R>
constexpr int lin_min_blocks() {
  return sizeof(T) == 4 ? ((R == 1 ? 1024 : 640) / (32 * BY) > 0 ? (R == 1 ? 1024 : 640) / (32 * BY) : 1)
                        : (R == 1 && 512 / (32 * BY) > 0 ? 512 / (32 * BY) : 1);
}

template <class T, int BY, int R, class Op>
__global__ void __launch_bounds__(32 * BY, (lin_min_blocks<T, BY, R>()))
    lin_march_kernel(const Grid<T> g, const Op op_in, int kchunk) {
  extern __shared__ __align__(16) unsigned char lin_dyn[];
  lin_body<T, BY, R, Op>(g, op_in, kchunk, blockIdx.x, blockIdx.y, blockIdx.z, lin_dyn);
}

}  // namespace qcad
