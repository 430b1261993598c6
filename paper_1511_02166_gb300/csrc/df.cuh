// df.cuh -- double-float arithmetic: a value is an unevaluated sum hi + lo of two
// float32 (|lo| <= ulp(hi)/2), about 48 significant bits, evaluated entirely on
// the FP32 pipe.  On GB300 the FP64 pipe issues about 1/74 of the FP32 rate, so
// the mixed-precision path computes its FP64-class quantities this way.
//
// Building blocks (published error-free transformations):
//   two_sum       Knuth (TAOCP vol. 2), 6 flops, s + e = a + b exactly;
//   fast_two_sum  Dekker 1971, 3 flops, exact when |a| >= |b|;
//   two_prod      with a fused multiply-add, p + e = a * b exactly.
// Sums, products and quotients of pairs follow Dekker 1971 and Joldes, Muller and
// Popescu, "Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic" (ACM TOMS 2017): relative errors of a few 2^-48.
// Every float operation below uses the _rn intrinsics so that the compiler can
// neither contract nor reorder them.
//
// df_log is table driven (P. T. P. Tang, "Table-driven implementation of the
// logarithm function in IEEE floating-point arithmetic", ACM TOMS 1990):
// y = 2^e m, m in [1, 2), F = 1 + j/256 nearest to m, u = (m - F)/F with
// |u| <= 2^-9, log y = e ln 2 + log F + log1p(u), the series of log1p(u) summed
// in double-float up to u^2 and in float32 beyond.  df_atan2 reduces to
// t = min/max in [0, 1], a 33-entry table of atan(j/32), and the series of
// atan(d), d = (t - c)/(1 + t c), |d| <= 1/64.  The tables come from
// gen_df_tables.py (decimal arithmetic from the definitions).
#pragma once
#include <cuda_runtime.h>

#include "df_tables.cuh"

namespace panel {

struct df2 {
  float hi, lo;
};

__device__ __forceinline__ df2 mkdf(float h, float l = 0.0f) {
  df2 r;
  r.hi = h;
  r.lo = l;
  return r;
}

__device__ __forceinline__ df2 df_from_double(double x) {
  float h = __double2float_rn(x);
  float l = __double2float_rn(x - (double)h);
  return mkdf(h, l);
}
__device__ __forceinline__ double df_to_double(df2 a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df2 two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return mkdf(s, e);
}
__device__ __forceinline__ df2 fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return mkdf(s, e);
}
__device__ __forceinline__ df2 two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return mkdf(p, e);
}

__device__ __forceinline__ df2 df_neg(df2 a) { return mkdf(-a.hi, -a.lo); }

// Dekker's sum: error ~2^-47 (|a| + |b|); use when no cancellation matters
// relative to the result.
__device__ __forceinline__ df2 df_add(df2 a, df2 b) {
  df2 s = two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df2 df_sub(df2 a, df2 b) { return df_add(a, df_neg(b)); }
// Accurate sum: error ~3 2^-48 |a + b| even under cancellation.
__device__ __forceinline__ df2 df_add_acc(df2 a, df2 b) {
  df2 s = two_sum(a.hi, b.hi);
  df2 t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df2 df_sub_acc(df2 a, df2 b) { return df_add_acc(a, df_neg(b)); }
// a + f for a float f.
__device__ __forceinline__ df2 df_add_f(df2 a, float f) {
  df2 s = two_sum(a.hi, f);
  s.lo = __fadd_rn(s.lo, a.lo);
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df2 df_mul(df2 a, df2 b) {
  df2 p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
  p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df2 df_mul_f(df2 a, float b) {
  df2 p = two_prod(a.hi, b);
  p.lo = __fmaf_rn(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df2 df_sqr(df2 a) {
  df2 p = two_prod(a.hi, a.hi);
  p.lo = __fmaf_rn(__fmul_rn(2.0f, a.hi), a.lo, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
// 1/a: one Newton correction of the rounded float reciprocal.
__device__ __forceinline__ df2 df_rcp(df2 a) {
  float r = __frcp_rn(a.hi);
  float e = __fmaf_rn(-a.hi, r, 1.0f);
  e = __fmaf_rn(-a.lo, r, e);
  return fast_two_sum(r, __fmul_rn(r, e));
}
// a / b: quotient, remainder in double-float, corrected quotient.
__device__ __forceinline__ df2 df_div(df2 a, df2 b) {
  float rb = __frcp_rn(b.hi);
  float q1 = __fmul_rn(a.hi, rb);
  df2 p = df_mul_f(b, q1);
  df2 r = df_sub(a, p);
  float q2 = __fmul_rn(r.hi, rb);
  return fast_two_sum(q1, q2);
}
__device__ __forceinline__ df2 df_const(const float* c) { return mkdf(c[0], c[1]); }

// Natural logarithm of y > 0 (normal float range).  `tab` = kLogTable staged
// in shared memory.
__device__ __forceinline__ df2 df_log(df2 y, const float4* __restrict__ tab) {
  const int bits = __float_as_int(y.hi);
  const int e = ((bits >> 23) & 0xff) - 127;
  const float m = __int_as_float((bits & 0x007fffff) | 0x3f800000);  // [1, 2)
  const int j = __float2int_rn(__fmul_rn(__fsub_rn(m, 1.0f), 256.0f));  // 0..256
  const float F = __fadd_rn(1.0f, __fmul_rn((float)j, 0.00390625f));  // exact
  const float f = __fsub_rn(m, F);                                     // exact
  const float4 t = tab[j];
  const df2 u = df_mul_f(mkdf(t.z, t.w), f);  // f / F
  const df2 u2 = df_sqr(u);
  const float uh = u.hi;
  // u^3/3 - u^4/4 + u^5/5 - u^6/6 in float32 (below 2^-27 in magnitude)
  float tail = __fmaf_rn(uh, -0.16666667f, 0.2f);
  tail = __fmaf_rn(uh, tail, -0.25f);
  tail = __fmaf_rn(uh, tail, 0.33333334f);
  tail = __fmul_rn(__fmul_rn(__fmul_rn(uh, uh), uh), tail);
  df2 s = df_add(u, mkdf(-0.5f * u2.hi, -0.5f * u2.lo));  // u - u^2/2
  s = fast_two_sum(s.hi, __fadd_rn(s.lo, tail));
  s = df_add(s, mkdf(t.x, t.y));                         // + log F
  s = df_add(s, df_mul_f(df_const(kLn2), (float)e));    // + e ln 2
  // log(y.hi + y.lo) = log(y.hi) + y.lo / y.hi + O(2^-48)
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fmul_rn(y.lo, __frcp_rn(y.hi))));
}

// atan2(y, x) in (-pi, pi]; atan2(0, 0) = 0.  `atab` = kAtanTable in shared memory.
__device__ __forceinline__ df2 df_atan2(df2 y, df2 x, const float2* __restrict__ atab) {
  const bool sy = y.hi < 0.0f, sx = x.hi < 0.0f;
  const df2 ay = sy ? df_neg(y) : y;
  const df2 ax = sx ? df_neg(x) : x;
  const bool sw = ay.hi > ax.hi;
  const df2 num = sw ? ax : ay;
  const df2 den = sw ? ay : ax;
  if (den.hi == 0.0f) return mkdf(0.0f);
  const df2 t = df_div(num, den);                            // [0, 1]
  const int j = __float2int_rn(__fmul_rn(t.hi, 32.0f));      // 0..32
  const float c = __fmul_rn((float)j, 0.03125f);
  const df2 dn = df_add_f(t, -c);                            // t - c
  const df2 dd = df_add_f(df_mul_f(t, c), 1.0f);             // 1 + t c
  const df2 d = df_div(dn, dd);                              // |d| <= 1/64
  const df2 d2 = df_sqr(d);
  const df2 d3 = df_mul(df_mul(d2, d), df_const(kThird));    // d^3 / 3
  const float dh = d.hi, dh2 = __fmul_rn(dh, dh);
  // d^5/5 - d^7/7 in float32
  const float tail = __fmul_rn(__fmul_rn(__fmul_rn(dh2, dh2), dh),
                               __fmaf_rn(dh2, -0.14285715f, 0.2f));
  df2 a = df_sub(d, d3);
  a = fast_two_sum(a.hi, __fadd_rn(a.lo, tail));
  const float2 tb = atab[j];
  a = df_add(a, mkdf(tb.x, tb.y));
  if (sw) a = df_sub(df_const(kPiHalf), a);
  if (sx) a = df_sub(df_const(kPi), a);
  return sy ? df_neg(a) : a;
}

// Stage the lookup tables in shared memory (all threads of the block call it).
__device__ __forceinline__ void df_stage_tables(float4* s_log, float2* s_atan) {
  for (int k = threadIdx.x; k < 257; k += blockDim.x) s_log[k] = kLogTable[k];
  for (int k = threadIdx.x; k < 33; k += blockDim.x) s_atan[k] = kAtanTable[k];
}

}  // namespace panel
