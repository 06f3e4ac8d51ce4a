// Double-float ("df64") arithmetic: a value is the unevaluated sum h + l of two
// FP32 numbers, |l| small against |h|.  The operator kernel instantiated with
// this type evaluates the FP64 operator to about 1e-14 relative accuracy using
// only FP32 instructions, which GB300 issues 62 times faster than FP64 ones.
//
// Building blocks are the error-free transformations of Dekker (1971) and
// Knuth: TwoProd through one FMA (p = a b, e = fma(a, b, -p) is exact), and
// TwoSum (s = a + b, e = (a - (s - bb)) + (b - bb), bb = s - a, is exact).  A
// product keeps the error of the high parts exactly and adds the cross terms
// a.h b.l + a.l b.h in FP32; a multiply-add keeps the rounding error of the
// high-part sum exactly and collects every error term in the low part, which is
// left unnormalised (it stays within a few ulps of h for the short sums of the
// sum factorization) and is folded into the high part on conversion.
#pragma once

#include <cuda_runtime.h>

namespace sem {
// The df type and its operations live in their own namespace so that only
// argument-dependent lookup finds them: unqualified fma / atomicAdd calls on
// double or float arguments elsewhere in namespace sem keep resolving to the
// CUDA built-ins (and never convert silently to df).
namespace dfx {

struct df {
  float h, l;
  df() = default;
  __host__ __device__ constexpr df(float hh, float ll) : h(hh), l(ll) {}
  __host__ __device__ explicit constexpr df(int z) : h((float)z), l(0.f) {}
  __host__ __device__ df(double x) {
    h = (float)x;
    l = (float)(x - (double)h);
  }
  __host__ __device__ explicit operator double() const { return (double)h + (double)l; }
};

// Metric storage of the df64 operator: the split pair of each FP64 metric value.
struct df_pair {
  float h, l;
};

__device__ __forceinline__ df operator*(df a, df b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
  return df(p, e);
}

__device__ __forceinline__ df& operator*=(df& a, df b) {
  a = a * b;
  return a;
}

// c + a b
__device__ __forceinline__ df fma(df a, df b, df c) {
  const float p = a.h * b.h;
  const float ep = fmaf(a.h, b.h, -p);
  const float s = c.h + p;
  const float bb = s - c.h;
  const float es = (c.h - (s - bb)) + (p - bb);
  const float cross = fmaf(a.h, b.l, a.l * b.h);
  return df(s, c.l + (es + (ep + cross)));
}

__device__ __forceinline__ df operator+(df a, df b) {
  const float s = a.h + b.h;
  const float bb = s - a.h;
  const float es = (a.h - (s - bb)) + (b.h - bb);
  return df(s, es + (a.l + b.l));
}

__device__ __forceinline__ df& operator+=(df& a, df b) {
  a = a + b;
  return a;
}

__device__ __forceinline__ df operator-(df a, df b) { return a + df(-b.h, -b.l); }

}  // namespace dfx
using dfx::df;
using dfx::df_pair;

// x as a float pair (h, l), h + l = x to about 2^-46 relative, with 32-bit
// integer and FP32 instructions only (FP64 instructions, conversions included,
// issue at a small fraction of the FP32 rate on GB300): h is x with its
// mantissa cut to 23 bits, l the next 23 bits, made exact as a float by the
// 2^23 exponent trick (the bits under the mantissa of 2^23, minus 2^23) and
// scaled by 2^(E - 1069) in two exact halves.  |x| below 2^-126 (no normal
// float) gives a signed zero, |x| from 2^128 on an infinity and a NaN a NaN;
// for |x| below 2^-80 l loses bits to FP32 underflow (absolute error below
// 2^-149).
#ifdef __CUDACC__
__device__ __forceinline__ df_pair split_pair(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int E = (int)((hi >> 20) & 0x7ffu);
  const unsigned sign = hi & 0x80000000u;
  if (E < 897) return df_pair{__uint_as_float(sign), 0.f};
  if (E > 1150) {
    const bool nan = E == 2047 && ((hi & 0xfffffu) | lo) != 0u;
    return df_pair{__uint_as_float(sign | 0x7f800000u | (nan ? 0x400000u : 0u)), 0.f};
  }
  const unsigned hb = sign | ((unsigned)(E - 896) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const float m = __uint_as_float(0x4b000000u | ((lo >> 6) & 0x7fffffu)) - 8388608.f;
  const int s = E - 1069, s1 = s >> 1, s2 = s - s1;  // both in [-86, 41]
  const float l = (m * __int_as_float((s1 + 127) << 23)) * __int_as_float((s2 + 127) << 23);
  return df_pair{__uint_as_float(hb), __uint_as_float(__float_as_uint(l) ^ sign)};
}

// Exact float -> double by integer operations (subnormal floats, below 1.2e-38,
// become zero).
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
  if (e == 0u) return __longlong_as_double((long long)sign);
  const unsigned long long d =
      sign | ((unsigned long long)(e - 127u + 1023u) << 52) | ((unsigned long long)(b & 0x7fffffu) << 29);
  return __longlong_as_double((long long)d);
}

// Float pair -> FP64 with one FP64 instruction (the addition).
__device__ __forceinline__ double df_to_double(df a) { return f2d_bits(a.h) + f2d_bits(a.l); }
#endif
}  // namespace sem
