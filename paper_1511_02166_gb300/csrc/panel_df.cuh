// panel_df.cuh -- the panel integral of Section 2 in double-float arithmetic.
//
// G(p; panel) = (1/2pi) * integral over the panel of log|p - s| ds, so that the
// matrix coefficient of Section 2 is A_ji = -G(x_{j+1/2}; panel i).  Two exact
// rearrangements of the printed closed form are used, both written around the
// panel midpoint c, with P = p - c, half-length L/2 and unit tangent t:
//
//  far field (|P| >= 4 L): the multipole series of the same integral,
//     G = (L/2pi) [ log|P| - sum_{n>=1} q^n T_n(cos 2phi) / (2n (2n+1)) ],
//     q = L^2 / (4 |P|^2), phi = angle(P) - angle(t), T_n Chebyshev polynomials;
//     q <= 1/64, so seven terms reach 2^-48; terms n = 1, 2 in double-float,
//     n >= 3 in float32 (their size keeps the float32 error below 2^-48).
//     One logarithm, no arctangent.
//  near field: with zeta = P.t, eta = P.n, r1^2 = (zeta + L/2)^2 + eta^2,
//     r2^2 = (zeta - L/2)^2 + eta^2 (distances to the two panel ends),
//     G = (1/2pi) [ zeta/2 (log r1^2 - log r2^2) + L/4 (log r1^2 + log r2^2)
//                   + eta theta - L ],  theta = atan2(L eta, |P|^2 - L^2/4),
//     which is the printed bracket (two logs, the two arctan2 merged into the
//     angle the panel subtends, in (-pi, pi)).  On the own panel P = 0 exactly
//     and G = (L/2pi)(log(L/2) - 1).
// Both branches agree with the printed form to rounding; the far-field form
// avoids the cancellation of the printed one when |P| >> L.
//
// P itself must be accurate relative to |P|, also when p sits a fraction of a
// short panel away from it.  Midpoints (which are also the control points) are
// therefore kept as three floats on fixed grids, x = h + m + l with h a
// multiple of 2^-12, m a multiple of 2^-35 (|m| <= 2^-13) and |l| <= 2^-36, so
// that differences of h and of m are exact in float32 and P is formed before
// any rounding to double-float.  This needs |x| < 1024.
#pragma once
#include "df.cuh"

namespace panel {

// Per-panel constants, structure of arrays in shared memory (stride `ld`).
enum PanelField {
  kCx = 0, kCy = 3, kTx = 6, kTy = 8, kL = 10, kLg = 12, kQ6 = 14, kQ20 = 16, kC2 = 18, kS2 = 20,
  kPanelFields = 22
};

// x = h + m + l on the grids 2^-12 and 2^-35 (|x| < 1024); FP64 arithmetic.
struct split3 {
  float h, m, l;
};
__device__ __forceinline__ split3 split_coord(double x) {
  const double h = rint(x * 4096.0) * (1.0 / 4096.0);
  const double r = x - h;
  const double m = rint(r * 34359738368.0) * (1.0 / 34359738368.0);
  split3 s;
  s.h = (float)h;
  s.m = (float)m;
  s.l = (float)(r - m);
  return s;
}
// (a - b) as a double-float, a and b split on the same grids.
__device__ __forceinline__ df2 split_diff(float ah, float am, float al, float bh, float bm,
                                          float bl) {
  const float dh = __fsub_rn(ah, bh);  // exact
  const float dm = __fsub_rn(am, bm);  // exact
  const float dl = __fsub_rn(al, bl);
  const df2 t = two_sum(dh, dm);
  return fast_two_sum(t.hi, __fadd_rn(t.lo, dl));
}

__device__ __forceinline__ df2 pf(const float* s, int ld, int field, int i) {
  return mkdf(s[field * ld + i], s[(field + 1) * ld + i]);
}
__device__ __forceinline__ void pf_store(float* s, int ld, int field, int i, double v) {
  df2 d = df_from_double(v);
  s[field * ld + i] = d.hi;
  s[(field + 1) * ld + i] = d.lo;
}

// Fill the per-panel constants of panel i from FP64 node coordinates
// (a = x_i, b = x_{i+1}).  c = midpoint, t = unit tangent, L = length,
// Lg = L/(2pi), Q6 = L^2/24, Q20 = L^4/320, (C2, S2) = (cos 2beta, sin 2beta).
__device__ __forceinline__ void panel_constants(float* s, int ld, int i, double ax, double ay,
                                                double bx, double by) {
  const double hx = bx - ax, hy = by - ay;
  const double L = sqrt(hx * hx + hy * hy);
  const double tx = hx / L, ty = hy / L;
  const double L2 = L * L;
  const split3 cx = split_coord(0.5 * (ax + bx)), cy = split_coord(0.5 * (ay + by));
  s[kCx * ld + i] = cx.h;
  s[(kCx + 1) * ld + i] = cx.m;
  s[(kCx + 2) * ld + i] = cx.l;
  s[kCy * ld + i] = cy.h;
  s[(kCy + 1) * ld + i] = cy.m;
  s[(kCy + 2) * ld + i] = cy.l;
  pf_store(s, ld, kTx, i, tx);
  pf_store(s, ld, kTy, i, ty);
  pf_store(s, ld, kL, i, L);
  pf_store(s, ld, kLg, i, L * 0.15915494309189533577);
  pf_store(s, ld, kQ6, i, L2 / 24.0);
  pf_store(s, ld, kQ20, i, L2 * L2 / 320.0);
  pf_store(s, ld, kC2, i, tx * tx - ty * ty);
  pf_store(s, ld, kS2, i, 2.0 * tx * ty);
}

// The split coordinates of a control point.
struct point3 {
  float xh, xm, xl, yh, ym, yl;
};
__device__ __forceinline__ point3 load_point(const float* s, int ld, int j) {
  point3 p;
  p.xh = s[kCx * ld + j];
  p.xm = s[(kCx + 1) * ld + j];
  p.xl = s[(kCx + 2) * ld + j];
  p.yh = s[kCy * ld + j];
  p.ym = s[(kCy + 1) * ld + j];
  p.yl = s[(kCy + 2) * ld + j];
  return p;
}
__device__ __forceinline__ point3 make_point(double x, double y) {
  const split3 a = split_coord(x), b = split_coord(y);
  point3 p;
  p.xh = a.h; p.xm = a.m; p.xl = a.l;
  p.yh = b.h; p.ym = b.m; p.yl = b.l;
  return p;
}

// P = p - c_i (exactly formed from the split coordinates) and |P|^2.
struct PairGeom {
  df2 px, py, px2, py2, rho2;
  float Lh;
  __device__ __forceinline__ bool far() const { return rho2.hi >= 16.0f * Lh * Lh; }
};
__device__ __forceinline__ PairGeom pair_geom(const point3& p, const float* __restrict__ s,
                                              int ld, int i) {
  PairGeom g;
  g.px = split_diff(p.xh, p.xm, p.xl, s[kCx * ld + i], s[(kCx + 1) * ld + i],
                    s[(kCx + 2) * ld + i]);
  g.py = split_diff(p.yh, p.ym, p.yl, s[kCy * ld + i], s[(kCy + 1) * ld + i],
                    s[(kCy + 2) * ld + i]);
  g.px2 = df_sqr(g.px);
  g.py2 = df_sqr(g.py);
  g.rho2 = df_add(g.px2, g.py2);
  g.Lh = s[kL * ld + i];
  return g;
}

// The far-field series of G(p; panel i) from the quantities of the pair that
// do not depend on the panel's orientation or length (they are the same for
// the pair seen from either end: P -> -P leaves them unchanged exactly):
// X + iY = P^2 (X = px^2 - py^2, Y = 2 px py), inv = 1/|P|^2, inv2 = inv^2,
// lgh = log|P|.  Term n = 1 in double-float, n = 2 in double-float within
// 32 panel lengths (q > 1/4096), n >= 3 in float32.
__device__ __forceinline__ df2 panel_G_far(const df2 X, const df2 Y, const df2 inv,
                                           const df2 inv2, const df2 lgh,
                                           const float* __restrict__ s, int ld, int i, float Lh) {
  const df2 Z = df_add(df_mul(pf(s, ld, kC2, i), X), df_mul(pf(s, ld, kS2, i), Y));
  const df2 cc = df_mul(Z, inv);  // cos 2phi
  const df2 t1 = df_mul(df_mul(pf(s, ld, kQ6, i), inv), cc);       // q c / 6
  const float q = __fmul_rn(__fmul_rn(0.25f * Lh, Lh), inv.hi);
  const float c = cc.hi;
  const float c2 = __fmul_rn(2.0f, c);
  const float T3 = __fmul_rn(c, __fsub_rn(__fmul_rn(__fmul_rn(4.0f, c), c), 3.0f));
  if (q <= 1.0f / 4096.0f) {
    // |P| >= 32 L: the n = 2 term (at most 3e-9 of the leading one) joins
    // the float32 tail, q^2 (T2/20 + q (T3/42 + q (T4/72 + ...)))
    const float T2 = __fsub_rn(__fmul_rn(c2, c), 1.0f);
    const float T4 = __fsub_rn(__fmul_rn(c2, T3), T2);
    const float T5 = __fsub_rn(__fmul_rn(c2, T4), T3);
    const float T6 = __fsub_rn(__fmul_rn(c2, T5), T4);
    const float T7 = __fsub_rn(__fmul_rn(c2, T6), T5);
    float tail = __fadd_rn(__fmul_rn(T6, 1.0f / 156.0f), __fmul_rn(__fmul_rn(q, T7), 1.0f / 210.0f));
    tail = __fadd_rn(__fmul_rn(T5, 1.0f / 110.0f), __fmul_rn(q, tail));
    tail = __fadd_rn(__fmul_rn(T4, 1.0f / 72.0f), __fmul_rn(q, tail));
    tail = __fadd_rn(__fmul_rn(T3, 1.0f / 42.0f), __fmul_rn(q, tail));
    tail = __fadd_rn(__fmul_rn(T2, 1.0f / 20.0f), __fmul_rn(q, tail));
    tail = __fmul_rn(tail, __fmul_rn(q, q));
    return df_mul(pf(s, ld, kLg, i), df_sub(lgh, df_add_f(t1, tail)));
  }
  df2 T2 = df_sqr(cc);
  T2.hi *= 2.0f;
  T2.lo *= 2.0f;
  T2 = df_add_f(T2, -1.0f);                                        // 2c^2 - 1
  const df2 t2 = df_mul(df_mul(pf(s, ld, kQ20, i), inv2), T2);     // q^2 T2 / 20
  // n >= 3 in float32: q^3 (T3/42 + q (T4/72 + q (T5/110 + q (T6/156 + q T7/210))))
  const float T4 = __fsub_rn(__fmul_rn(c2, T3), T2.hi);
  const float T5 = __fsub_rn(__fmul_rn(c2, T4), T3);
  const float T6 = __fsub_rn(__fmul_rn(c2, T5), T4);
  const float T7 = __fsub_rn(__fmul_rn(c2, T6), T5);
  float tail = __fadd_rn(__fmul_rn(T6, 1.0f / 156.0f), __fmul_rn(__fmul_rn(q, T7), 1.0f / 210.0f));
  tail = __fadd_rn(__fmul_rn(T5, 1.0f / 110.0f), __fmul_rn(q, tail));
  tail = __fadd_rn(__fmul_rn(T4, 1.0f / 72.0f), __fmul_rn(q, tail));
  tail = __fadd_rn(__fmul_rn(T3, 1.0f / 42.0f), __fmul_rn(q, tail));
  tail = __fmul_rn(tail, __fmul_rn(__fmul_rn(q, q), q));
  df2 S = df_add(t1, t2);
  S = fast_two_sum(S.hi, __fadd_rn(S.lo, tail));
  return df_mul(pf(s, ld, kLg, i), df_sub(lgh, S));
}

// G(p; panel i) in double-float for the control point p.  WHICH = 0: the far or
// the near form by |P| >= 4 L; 1: the far form; 2: the near form (the caller has
// made the choice with PairGeom::far).
template <int WHICH = 0>
__device__ __forceinline__ df2 panel_G_df(const PairGeom& gm, const float* __restrict__ s,
                                          int ld, int i, const float4* __restrict__ tlog,
                                          const float2* __restrict__ tatan) {
  const df2 px = gm.px, py = gm.py, px2 = gm.px2, py2 = gm.py2, rho2 = gm.rho2;
  const float Lh = gm.Lh;
  if (WHICH == 1 || (WHICH == 0 && gm.far())) {
    // ---- far field: multipole series about the panel midpoint ----
    const df2 X = df_sub(px2, py2);
    df2 Y = df_mul(px, py);
    Y.hi *= 2.0f;
    Y.lo *= 2.0f;
    const df2 inv = df_rcp(rho2);
    df2 lg = df_log(rho2, tlog);
    lg.hi *= 0.5f;
    lg.lo *= 0.5f;
    return panel_G_far(X, Y, inv, df_sqr(inv), lg, s, ld, i, Lh);
  }
  if (WHICH == 1) return mkdf(0.0f);
  // ---- near field: exact closed form in the panel frame ----
  const df2 tx = pf(s, ld, kTx, i), ty = pf(s, ld, kTy, i);
  const df2 L = pf(s, ld, kL, i);
  const df2 zeta = df_add(df_mul(px, tx), df_mul(py, ty));
  const df2 eta = df_sub(df_mul(py, tx), df_mul(px, ty));
  const df2 half = mkdf(0.5f * L.hi, 0.5f * L.lo);
  const df2 a1 = df_add(zeta, half), a2 = df_sub(zeta, half);
  const df2 eta2 = df_sqr(eta);
  const df2 l1 = df_log(df_add(df_sqr(a1), eta2), tlog);
  const df2 l2 = df_log(df_add(df_sqr(a2), eta2), tlog);
  const df2 quarterL2 = df_mul_f(pf(s, ld, kQ6, i), 6.0f);  // L^2 / 4
  const df2 th = df_atan2(df_mul(L, eta), df_sub(rho2, quarterL2), tatan);
  df2 br = df_mul(mkdf(0.5f * zeta.hi, 0.5f * zeta.lo), df_sub(l1, l2));
  br = df_add(br, df_mul(mkdf(0.25f * L.hi, 0.25f * L.lo), df_add(l1, l2)));
  br = df_add(br, df_mul(eta, th));
  br = df_sub(br, L);
  return df_mul(br, df_const(kInv2Pi));
}

__device__ __forceinline__ df2 panel_G_df(const point3& p, const float* __restrict__ s, int ld,
                                          int i, const float4* __restrict__ tlog,
                                          const float2* __restrict__ tatan) {
  return panel_G_df<0>(pair_geom(p, s, ld, i), s, ld, i, tlog, tatan);
}

}  // namespace panel
