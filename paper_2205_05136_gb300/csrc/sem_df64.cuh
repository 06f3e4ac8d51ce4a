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

// x as a float pair (h, l), h + l = x to about 2^-48 relative, with integer and
// FP32 instructions only (FP64 instructions, conversions included, issue at a
// small fraction of the FP32 rate on GB300): h is x with its mantissa cut to
// 23 bits, l the remaining 29 bits, m_low 2^(E - 1075), as a float (the one
// rounding).  Zeros, tiny (|x| < 2^-63), huge and non-finite values take FP64
// conversions instead.
#ifdef __CUDACC__
__device__ __forceinline__ df_pair split_pair(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ffull);
  if (E < 960 || E > 1150) {
    const float h = (float)x;
    return df_pair{h, (float)(x - (double)h)};
  }
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const unsigned hb = sign | ((unsigned)(E - 896) << 23) | (unsigned)((b >> 29) & 0x7fffffull);
  const float l = (float)(unsigned)(b & ((1ull << 29) - 1)) * __int_as_float((E - 948) << 23);
  return df_pair{__int_as_float((int)hb), sign ? -l : l};
}
#endif
}  // namespace sem
