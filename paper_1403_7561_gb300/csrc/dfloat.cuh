// Double-float arithmetic on the FP32 pipes: a value is the unevaluated sum h + l of two floats
// (about 46 significant bits). The product uses Dekker's fused-multiply-add split, the sum Knuth's
// two-sum, each renormalized by a fast two-sum; relative error of a product or sum about 2^-46.
// On this part FP32 runs at 64 times the FP64 rate, so a double-float multiply-add (some twenty
// FP32 instructions) costs a third of an FP64 one. Conversions to and from FP64 go through the
// bit patterns (integer instructions), because the FP32<->FP64 conversion instructions run on the
// FP64 pipe.
//
// Used as the scalar type T of the plane-factorized z-march for the FP64 phase of the
// eigensolver's H and M applies (kernels_lin.cu).
#pragma once
#include <cuda_runtime.h>

#include "qcad_internal.cuh"

namespace qcad {

struct dfl {
  float h, l;
  __host__ __device__ dfl() : h(0.0f), l(0.0f) {}
  __host__ __device__ dfl(int v) : h((float)v), l(0.0f) {}
  __host__ __device__ dfl(float hh, float ll) : h(hh), l(ll) {}
  // host only: the split of a double by FP32 rounding (device code uses dfl_from_bits)
  __host__ dfl(double v) : h((float)v), l((float)(v - (double)(float)v)) {}
};

__device__ __forceinline__ dfl dfl_quick(float s, float e) {
  const float h = s + e;
  return dfl(h, e - (h - s));
}

__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  const float s = a.h + b.h;
  const float bb = s - a.h;
  float e = (a.h - (s - bb)) + (b.h - bb);
  e += a.l + b.l;
  return dfl_quick(s, e);
}
__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.h, -a.l); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return dfl_quick(p, e);
}
__device__ __forceinline__ dfl& operator+=(dfl& a, dfl b) { return a = a + b; }
__device__ __forceinline__ dfl& operator*=(dfl& a, dfl b) { return a = a * b; }

// Warp shuffles of both words (the built-in overloads stay visible beside these).
using ::__shfl_down_sync;
using ::__shfl_up_sync;
using ::__shfl_xor_sync;
__device__ __forceinline__ dfl __shfl_down_sync(unsigned mask, dfl v, unsigned d) {
  return dfl(::__shfl_down_sync(mask, v.h, d), ::__shfl_down_sync(mask, v.l, d));
}
__device__ __forceinline__ dfl __shfl_up_sync(unsigned mask, dfl v, unsigned d) {
  return dfl(::__shfl_up_sync(mask, v.h, d), ::__shfl_up_sync(mask, v.l, d));
}
__device__ __forceinline__ dfl __shfl_xor_sync(unsigned mask, dfl v, int d) {
  return dfl(::__shfl_xor_sync(mask, v.h, d), ::__shfl_xor_sync(mask, v.l, d));
}

// a = h + l for 2^-80 <= |a| < 2^127 by the bit pattern: h keeps the sign, exponent and top 23
// mantissa bits of a (truncation, exact), l the next 23 (bits 28..6), |a - h - l| <= 2^-46 |a|;
// below 2^-80 l is dropped, outside [2^-100, 2^127) (zero included) the FP64 conversion is used.
__device__ __forceinline__ dfl dfl_from_bits(double a) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(a);
  const unsigned hi32 = (unsigned)(u >> 32), lo32 = (unsigned)u;
  const int e = (int)((hi32 >> 20) & 0x7FF);
  const unsigned sgn = hi32 & 0x80000000u;
  if (e < 923 || e > 1150) return dfl(__double2float_rn(a), 0.0f);
  const float h = __uint_as_float(sgn | ((unsigned)(e - 896) << 23) | ((hi32 & 0xFFFFFu) << 3) | (lo32 >> 29));
  if (e < 943) return dfl(h, 0.0f);
  const float m = __uint_as_float(0x4B000000u | ((lo32 >> 6) & 0x7FFFFFu)) - 8388608.0f;
  return dfl(h, __uint_as_float(__float_as_uint(m * __uint_as_float((unsigned)(e - 942) << 23)) | sgn));
}

// The FP64 value of a float by its bit pattern (exact for normal floats and zero).
__device__ __forceinline__ double dfl_f2d(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned e = (u >> 23) & 0xFFu;
  if (e == 0u || e == 0xFFu) return (double)x;
  return __longlong_as_double((long long)(((unsigned long long)(u & 0x80000000u) << 32) |
                                          ((unsigned long long)(e + 896u) << 52) |
                                          ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

// h + l rounded to FP64 (one FP64 addition).
__device__ __forceinline__ double dfl_to_double(dfl a) { return dfl_f2d(a.h) + dfl_f2d(a.l); }

// The Gauss weights (1 +- 1/sqrt 3) / 2 of the linear shape functions as double-float pairs.
template <> struct GaussConst<dfl> {
  static __device__ __forceinline__ dfl a() { return dfl(0x1.93cd3ap-1f, 0x1.640cc8p-28f); }
  static __device__ __forceinline__ dfl b() { return dfl(0x1.b0cb18p-3f, -0x1.640cc8p-28f); }
};

}  // namespace qcad
