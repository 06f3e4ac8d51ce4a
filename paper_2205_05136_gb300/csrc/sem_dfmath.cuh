// Double-float functions for the per-node ionic update (FP32-pipe arithmetic,
// about 1e-14 relative): exp, division and the conversions between FP64 and
// float pairs.  GB300 issues FP64 instructions (conversions included) at a
// small fraction of its FP32 rate, which bounds a per-node update in FP64.
//
// Methods:
//   - double-float arithmetic: Dekker (1971), error-free sums and products
//     (sem_df64.cuh);
//   - exp: Cody and Waite's argument reduction x = k ln2 + r, |r| <= ln2 / 2,
//     with ln2 split into three floats c1 + c2 + c3 such that k c1 and k c2 are
//     exact for |k| < 128 (k rounded by adding and subtracting 1.5 2^23); then
//     the Taylor series of exp(r) to r^13 / 13! (truncation below 1e-17 for
//     |r| <= 0.36) by Horner's rule: the terms from r^8 / 8! on are below
//     2^-25 and are summed in FP32, the others in double-float; and the exact
//     scaling by 2^k;
//   - division a / b: q1 ~ a.h / b.h, then one correction with the exact
//     residual a - q1 b (Dekker's division); the FP32 quotients are the fast
//     approximate ones, the correction absorbs their error.
#pragma once

#include "sem_df64.cuh"

namespace sem {

// Constants of dfexp, computed on the host (ionic_df_constants).
struct DfExpConst {
  float inv_ln2, c1, c2, c3;   // 1 / ln2; ln2 = c1 + c2 + c3 (c1, c2 with 16 significant bits)
  float th[14], tl[14];        // 1 / j! as the float pair th[j] + tl[j]
};

#ifdef __CUDACC__

// Renormalised pair (|l| at most half an ulp of h): Dekker's fast two-sum.
__device__ __forceinline__ df dfnorm(df a) {
  const float s = a.h + a.l;
  return df(s, a.l - (s - a.h));
}

__device__ __forceinline__ df dfneg(df a) { return df(-a.h, -a.l); }

// FP64 -> float pair with integer and FP32 instructions (split_pair).
__device__ __forceinline__ df dfd(double x) {
  const df_pair p = split_pair(x);
  return df(p.h, p.l);
}

// a / b.
__device__ __forceinline__ df dfdiv(df a, df b) {
  const float q1 = __fdividef(a.h, b.h);
  const df r = a - df(q1, 0.f) * b;
  const float q2 = __fdividef(r.h + r.l, b.h);
  return dfnorm(df(q1, q2));
}

// exp(x) for x <= 88; zero below -87 (the result would be a subnormal float).
__device__ __forceinline__ df dfexp(df x, const DfExpConst& K) {
  if (x.h < -87.f) return df(0.f, 0.f);
  const float k = (x.h * K.inv_ln2 + 12582912.f) - 12582912.f;  // nearest integer
  df r = x - df(k * K.c1, 0.f);  // k c1 and k c2 are exact products
  r = r - df(k * K.c2, 0.f);
  r = dfnorm(r - df(k * K.c3, 0.f));
  float tail = K.th[13];
#pragma unroll
  for (int j = 12; j >= 8; --j) tail = fmaf(tail, r.h, K.th[j]);
  df t = dfnorm(fma(df(tail, 0.f), r, df(K.th[7], K.tl[7])));
#pragma unroll
  for (int j = 6; j >= 0; --j) t = dfnorm(fma(t, r, df(K.th[j], K.tl[j])));
  const float s = __int_as_float(((int)k + 127) << 23);  // 2^k, |k| <= 126
  return df(t.h * s, t.l * s);
}

#endif  // __CUDACC__

}  // namespace sem
