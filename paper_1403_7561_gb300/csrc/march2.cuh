// FP32 z-marching skeleton with two x-adjacent nodes (and two elements) per
// thread, computed as packed pairs with the sm_100-family f32x2 FMA.
//
// Same discretization and gather scheme as march_kernel (qcad_internal.cuh):
// separable stiffness stencil, element Gauss-point mass term, planes k-1..k+1
// of the input in a shared ring, element corner outputs gathered along x by
// warp shuffles, along y through shared memory and along z by a register
// carry, next plane prefetched into registers. Here a warp row covers 64
// nodes: lane l holds nodes 2l and 2l+1 (a float2) and the elements whose
// left corner they are, so the two elements of a thread run through the
// Gauss-point interpolation, scaling and testing as one packed pair. The
// block's x stride is 60 nodes; lanes 0 and 31 are halo.
#pragma once

#include "qcad_internal.cuh"

namespace qcad {

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 bcast(float s) { return make_float2(s, s); }

// Packed version of tp_apply: [[a, b], [b, a]] along x, y, z on 8 corner pairs.
__device__ __forceinline__ void tp_apply2(const float2* in, float2* out, float a, float b) {
  const float2 A = bcast(a), B = bcast(b);
  float2 t[8], u[8];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    t[2 * p] = ffma2(A, in[2 * p], fmul2(B, in[2 * p + 1]));
    t[2 * p + 1] = ffma2(B, in[2 * p], fmul2(A, in[2 * p + 1]));
  }
#pragma unroll
  for (int z = 0; z < 2; ++z) {
#pragma unroll
    for (int x = 0; x < 2; ++x) {
      const int i0 = x + 4 * z, i1 = i0 + 2;
      u[i0] = ffma2(A, t[i0], fmul2(B, t[i1]));
      u[i1] = ffma2(B, t[i0], fmul2(A, t[i1]));
    }
  }
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    out[p] = ffma2(A, u[p], fmul2(B, u[p + 4]));
    out[p + 4] = ffma2(B, u[p], fmul2(A, u[p + 4]));
  }
}

// Element pair mass term: out = B (c o (B v)) for two elements at once.
__device__ __forceinline__ void qp_mass2(const float2* v, const float2* c, float2* out) {
  float2 u[8];
  tp_apply2(v, u, GaussConst<float>::a(), GaussConst<float>::b());
#pragma unroll
  for (int q = 0; q < 8; ++q) u[q] = fmul2(u[q], c[q]);
  tp_apply2(u, out, GaussConst<float>::a(), GaussConst<float>::b());
}

constexpr int PX = 60;  // x stride of a pair-tile (nodes written per warp row)

// Op (all FP32, one gathered field with the stiffness stencil) supplies:
//   bool skip(), void set_vec(int)
//   float load(n, in)                         input value at node n (0 when !in)
//   void edata(g, i, j, k, float (&c)[8])     the element's 8 quadrature coefficients
//   void node(g, n, i, j, k, vin, y)          writer epilogue for one node (y = J v before
//                                             the Dirichlet override, which the op applies)
//   void finish()
template <int BY, class Op>
__global__ void __launch_bounds__(32 * BY)
march2_kernel(const Grid<float> g, const Op op_in, int kchunk) {
  if (op_in.skip()) return;
  const int nch = (g.nzn + kchunk - 1) / kchunk;
  Op op = op_in;
  op.set_vec(blockIdx.z / nch);
  __shared__ float2 ring[4][BY][32];
  __shared__ float2 s1[BY][32];
  __shared__ float2 s2[BY][32];
  __shared__ float2 sax[BY][32];
  __shared__ float2 say[BY][32];
  __shared__ float2 sb[BY][32];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.x * PX - 2 + 2 * tx;  // first node of the pair; second is i + 1
  const int j = blockIdx.y * (BY - 2) - 1 + ty;
  const int k0 = (blockIdx.z % nch) * kchunk;
  const int k1 = min(k0 + kchunk, g.nzn);
  const int plane = (int)g.plane;
  const bool jin = (j >= 0 && j < g.nyn);
  const bool in0 = jin && i >= 0 && i < g.nxn;
  const bool in1 = jin && i + 1 >= 0 && i + 1 < g.nxn;
  const bool wrow = ty >= 1 && ty < BY - 1 && tx >= 1 && tx <= 30;
  const bool w0 = wrow && in0, w1 = wrow && in1;
  const bool ejin = (j >= 0 && j < g.ny) && ty < BY - 1;
  const bool eA = ejin && i >= 0 && i < g.nx;                // element i (left corner i)
  const bool eB = ejin && i + 1 >= 0 && i + 1 < g.nx && tx < 31;  // element i + 1 needs node i + 2
  const int typ = min(ty + 1, BY - 1), tym = max(ty - 1, 0);
  // 1D stencil rows: y coefficients shared by the pair, x coefficients per node
  float cmy[3] = {0, 0, 0}, cky[3] = {0, 0, 0};
  float2 kxp[3], mxp[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) {
    kxp[s] = make_float2(0.f, 0.f);
    mxp[s] = make_float2(0.f, 0.f);
  }
  if (jin) {
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      cmy[s] = g.my[3 * j + s];
      cky[s] = g.ky[3 * j + s];
    }
  }
  if (in0) {
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      kxp[s].x = g.kx[3 * i + s];
      mxp[s].x = g.mx[3 * i + s];
    }
  }
  if (in1) {
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      kxp[s].y = g.kx[3 * (i + 1) + s];
      mxp[s].y = g.mx[3 * (i + 1) + s];
    }
  }
  const int nij = (jin ? g.nxn * j : 0) + i;  // node index of the first node in plane 0 (valid when in0)
  auto load2 = [&](int k) -> float2 {
    const int b = nij + k * plane;
    return make_float2(in0 ? op.load(b, true) : 0.f, in1 ? op.load(b + 1, true) : 0.f);
  };
  // element pair coefficients (qp-major pairs)
  auto edata2 = [&](int k, float2* c) {
    float ca[8], cb[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) ca[q] = cb[q] = 0.f;
    if (eA && k < g.nz) op.edata(g, i, j, k, ca);
    if (eB && k < g.nz) op.edata(g, i + 1, j, k, cb);
#pragma unroll
    for (int q = 0; q < 8; ++q) c[q] = make_float2(ca[q], cb[q]);
  };
  // corners of the element pair from the ring: x0 corners are the own pair, x1 corners are
  // (own.y, next lane's .x)
  auto corners = [&](int ka, int kb, float2* v) {
    const float2 a0 = ring[ka & 3][ty][tx], a1 = ring[ka & 3][typ][tx];
    const float2 b0 = ring[kb & 3][ty][tx], b1 = ring[kb & 3][typ][tx];
    const float na0 = __shfl_down_sync(FULL_MASK, a0.x, 1), na1 = __shfl_down_sync(FULL_MASK, a1.x, 1);
    const float nb0 = __shfl_down_sync(FULL_MASK, b0.x, 1), nb1 = __shfl_down_sync(FULL_MASK, b1.x, 1);
    v[0] = a0;
    v[1] = make_float2(a0.y, na0);
    v[2] = a1;
    v[3] = make_float2(a1.y, na1);
    v[4] = b0;
    v[5] = make_float2(b0.y, nb0);
    v[6] = b1;
    v[7] = make_float2(b1.y, nb1);
  };
  // node-pair sums of one (y, z) corner class: (A.x0 + prev lane's B.x1, B.x0 + A.x1)
  auto xgather = [&](float2 x0, float2 x1) -> float2 {
    const float pb = __shfl_up_sync(FULL_MASK, x1.y, 1);
    return fadd2(x0, make_float2(tx > 0 ? pb : 0.f, x1.x));
  };
  const float2 zero2 = make_float2(0.f, 0.f);
  float2 carry = zero2;

  if (k0 > 0) ring[(k0 - 1) & 3][ty][tx] = load2(k0 - 1);
  ring[k0 & 3][ty][tx] = load2(k0);
  float2 vnext = (k0 + 1 < g.nzn) ? load2(k0 + 1) : zero2;
  float2 cnext[8];
  edata2(k0, cnext);
  __syncthreads();
  if (k0 > 0) {
    float2 v[8], c[8], out[8];
    corners(k0 - 1, k0, v);
    edata2(k0 - 1, c);
    qp_mass2(v, c, out);
    const float2 hy0 = xgather(out[4], out[5]);
    const float2 hy1 = xgather(out[6], out[7]);
    s2[ty][tx] = hy1;
    __syncthreads();
    carry = fadd2(hy0, ty > 0 ? s2[ty - 1][tx] : zero2);
  }
  for (int k = k0; k < k1; ++k) {
    const int kp = k + 1;
    ring[kp & 3][ty][tx] = vnext;
    float2 c[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) c[q] = cnext[q];
    if (k + 1 < k1) {
      vnext = (k + 2 < g.nzn) ? load2(k + 2) : zero2;
      edata2(k + 1, cnext);
    }
    __syncthreads();
    float2 out[8];
    {
      float2 v[8];
      corners(k, kp, v);
      qp_mass2(v, c, out);  // zero coefficients of invalid elements give zero outputs
    }
    const float2 ly0 = xgather(out[0], out[1]);
    const float2 ly1 = xgather(out[2], out[3]);
    const float2 hy0 = xgather(out[4], out[5]);
    const float2 hy1 = xgather(out[6], out[7]);
    s1[ty][tx] = ly1;
    s2[ty][tx] = hy1;
    const float2 vc = ring[k & 3][ty][tx];
    const float2 vm = (k > 0) ? ring[(k - 1) & 3][ty][tx] : zero2;
    const float2 vp = ring[kp & 3][ty][tx];
    const float* zx = g.mzx + 3 * k;
    const float* zy = g.mzy + 3 * k;
    const float* zz = g.kzz + 3 * k;
    const float2 ax = ffma2(bcast(zx[0]), vm, ffma2(bcast(zx[1]), vc, fmul2(bcast(zx[2]), vp)));
    const float2 ay = ffma2(bcast(zy[0]), vm, ffma2(bcast(zy[1]), vc, fmul2(bcast(zy[2]), vp)));
    const float2 bz = ffma2(bcast(zz[0]), vm, ffma2(bcast(zz[1]), vc, fmul2(bcast(zz[2]), vp)));
    sax[ty][tx] = ax;
    say[ty][tx] = ay;
    sb[ty][tx] = bz;
    __syncthreads();
    const float2 mass = fadd2(fadd2(ly0, ty > 0 ? s1[ty - 1][tx] : zero2), carry);
    carry = fadd2(hy0, ty > 0 ? s2[ty - 1][tx] : zero2);
    const float2 c1 = ffma2(bcast(cmy[0]), sax[tym][tx], ffma2(bcast(cmy[1]), ax, fmul2(bcast(cmy[2]), sax[typ][tx])));
    const float2 c2 = ffma2(bcast(cky[0]), say[tym][tx], ffma2(bcast(cky[1]), ay, fmul2(bcast(cky[2]), say[typ][tx])));
    const float2 c3 = ffma2(bcast(cmy[0]), sb[tym][tx], ffma2(bcast(cmy[1]), bz, fmul2(bcast(cmy[2]), sb[typ][tx])));
    const float2 d = fadd2(c2, c3);
    const float c1l = __shfl_up_sync(FULL_MASK, c1.y, 1), c1r = __shfl_down_sync(FULL_MASK, c1.x, 1);
    const float dl = __shfl_up_sync(FULL_MASK, d.y, 1), dr = __shfl_down_sync(FULL_MASK, d.x, 1);
    const float2 c1m = make_float2(c1l, c1.x), c1p = make_float2(c1.y, c1r);
    const float2 dm = make_float2(dl, d.x), dp = make_float2(d.y, dr);
    float2 y = ffma2(kxp[0], c1m, ffma2(kxp[1], c1, fmul2(kxp[2], c1p)));
    y = ffma2(mxp[0], dm, ffma2(mxp[1], d, ffma2(mxp[2], dp, y)));
    y = fadd2(y, mass);
    const int n0 = nij + k * plane;
    if (w0) op.node(g, n0, i, j, k, vc.x, y.x);
    if (w1) op.node(g, n0 + 1, i + 1, j, k, vc.y, y.y);
  }
  op.finish();
}

inline dim3 march2_grid(int nxn, int nyn, int nzn, int by, int kchunk, int nvec = 1) {
  return dim3((nxn + PX - 1) / PX, (nyn + by - 3) / (by - 2), ((nzn + kchunk - 1) / kchunk) * nvec);
}

}  // namespace qcad
