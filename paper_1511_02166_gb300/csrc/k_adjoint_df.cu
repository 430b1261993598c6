// k_adjoint_df.cu -- the dM/dx contraction of the adjoint in double-float
// (mixed-precision path).
//
// dCl/dx_k = dCl/dx_k|_u + lambda^T (db/dx_k - (dM/dx_k) u) with M_ji = -G_ji,
// G(p; a, b) = (1/2pi) int_a^b log|p - s| ds (Section 2's panel integral), so
//   dCl/dx_k = (2/(v c)) (gamma_{k-1} t_{k-1} - gamma_k t_k)
//            + v/2 (-sin a, cos a) (lambda_{k-1} + lambda_k)
//            + 1/2 (lambda_{k-1} P_{k-1} + lambda_k P_k) + u_k A_k + u_{k-1} B_{k-1},
//   P_j = sum_i u_i dG_ji/dp,  A_i = sum_j lambda_j dG_ji/da,  B_i = sum_j lambda_j dG_ji/db.
// Per pair two gradients are evaluated (dG/da = -dG/dp - dG/db):
//
//  far field (|P| >= 4L, P = p - c, complex notation, Delta = b - a = L t,
//  u = Delta^2 / (4 P^2), |u| <= 1/64), from 2pi G = L Re H,
//  H = log P - sum_n u^n / (2n (2n+1)):
//     2pi dG/dp     = L conj(F1(u) / P),    F1(u) = 1 + u/3 + u^2/5 + ... = atanh(w)/w,
//     2pi dG/dDelta = t (log|P| + Re(log(1 - u))/2 + i Im F1(u)),
//     dG/db = -dG/dp / 2 + dG/dDelta;
//  u and the first-order terms in double-float, the terms of second and higher
//  order in u (below 5e-5 of the leading one) in float32; when every lane of a
//  warp has |P| >= 32 L (|u| <= 1/4096) only the leading terms L P / |P|^2 and
//  t log|P| are double-float and the whole series is float32.  A warp with a
//  near-field lane and every lane within 64 L takes the near-field form on all
//  lanes.  The caller's lanes must all call this function together (warp votes
//  pick the branches).
//  near field (panel frame: xi = (p-a).t, eta = (p-a).n, l1 = log|p-a|^2,
//  l2 = log|p-b|^2, theta the subtended angle):
//     2pi dG/dp = (l1 - l2)/2 t + theta n,
//     2pi dG/db = l2/2 t + ((l1 - l2)/2 eta - theta xi)/L n.
//  On the own panel theta (+-pi) cancels between the terms and is set to 0.
//  In every branch 2pi dG/db = R_t K - (2pi dG/dp)/2 with K = (K_r, K_i) in the
//  panel frame (R_t K = K_r t + K_i n): far field K = log|P| + Re log(1 - u)/2 +
//  i Im F1, near field K = (l2 + (l1 - l2)/2, ((l1 - l2)/2 eta - theta xi)/L +
//  theta/2).  So B_i = sum_j lambda_j dG_ji/db needs per pair only the two
//  scalars lambda_j K (t_i is the lane's own panel): B_i = R_t (sum lambda K) -
//  S_i / 2, rotated once per panel in FP64.
//
// Layout: one block per airfoil; each warp owns 32 consecutive columns (panels
// i, one per lane) and sweeps all rows j: S_i = sum_j lambda_j dG_ji/dp and B_i
// accumulate in the lane's registers (double-float; A_i = -S_i - B_i by
// translation invariance), the row sums P_j are warp-reduced and kept as one
// double-float partial per warp in shared memory, summed at the end
// (n <= kPartialsN).  Larger airfoils take k_adjoint_df_split: the panels are
// cut into chunks of 256, one block per (airfoil, chunk), and every term of the
// formula above is added into the caller's gradient buffer by FP64 atomics
// once per row window, column or node (a few per pair row, not per pair).
#include "panel_common.cuh"
#include "panel_df.cuh"

namespace panel {

// 2pi dG/dp and the panel-frame K of 2pi dG/db = R_t K - pi dG/dp for the pair
// (p; panel i).
__device__ __forceinline__ void panel_dG_df(const point3& p, const float* __restrict__ s, int ld,
                                            int i, bool self, const float4* __restrict__ tlog,
                                            const float2* __restrict__ tatan, df2& gpx, df2& gpy,
                                            df2& kr, df2& ki) {
  const df2 px = split_diff(p.xh, p.xm, p.xl, s[kCx * ld + i], s[(kCx + 1) * ld + i],
                            s[(kCx + 2) * ld + i]);
  const df2 py = split_diff(p.yh, p.ym, p.yl, s[kCy * ld + i], s[(kCy + 1) * ld + i],
                            s[(kCy + 2) * ld + i]);
  const df2 px2 = df_sqr(px), py2 = df_sqr(py);
  const df2 rho2 = df_add(px2, py2);
  const float Lh = s[kL * ld + i];
  const df2 L = pf(s, ld, kL, i);
  if (__all_sync(0xffffffffu, rho2.hi >= 1024.0f * Lh * Lh)) {
    // every lane of the warp at |P| >= 32 L (warp-uniform branch): |u| <= 1/4096,
    // the leading terms L P / |P|^2 and t log|P| in double-float, the whole
    // series in u in float32 (below 1/12288 of the leading term: ~3e-11 of it)
    const df2 inv = df_rcp(rho2);
    const df2 Li = df_mul(L, inv);
    gpx = df_mul(Li, px);
    gpy = df_mul(Li, py);
    df2 lg = df_log(rho2, tlog);
    lg.hi *= 0.5f;
    lg.lo *= 0.5f;
    const float pxh = px.hi, pyh = py.hi, invf = inv.hi;
    const float X = pxh * pxh - pyh * pyh, Y = 2.0f * pxh * pyh;
    const float q = 6.0f * s[kQ6 * ld + i] * invf;  // L^2 / (4 |P|^2)
    const float c2 = s[kC2 * ld + i], s2 = s[kS2 * ld + i];
    const float ur = q * (c2 * X + s2 * Y) * invf, ui = q * (s2 * X - c2 * Y) * invf;
    // F1 - 1 = u (1/3 + u (1/5 + u (1/7 + u / 9))): the u^5 term is below 1e-19
    float ar = (1.0f / 7.0f) + ur * (1.0f / 9.0f), ai = ui * (1.0f / 9.0f), tr;
    tr = (1.0f / 5.0f) + ur * ar - ui * ai; ai = ur * ai + ui * ar; ar = tr;
    tr = (1.0f / 3.0f) + ur * ar - ui * ai; ai = ur * ai + ui * ar; ar = tr;
    const float Fr = ur * ar - ui * ai, Fi = ur * ai + ui * ar;
    // -Re log(1 - u) = Re u (1 + u (1/2 + u (1/3 + u / 4)))
    float br = (1.0f / 3.0f) + ur * 0.25f, bi = ui * 0.25f;
    tr = 0.5f + ur * br - ui * bi; bi = ur * bi + ui * br; br = tr;
    tr = 1.0f + ur * br - ui * bi; bi = ur * bi + ui * br; br = tr;
    const float rl = ur * br - ui * bi;
    const float Lif = Li.hi;
    gpx = df_add_f(gpx, Lif * (Fr * pxh + Fi * pyh));
    gpy = df_add_f(gpy, Lif * (Fr * pyh - Fi * pxh));
    kr = df_add_f(lg, -0.5f * rl);
    ki = mkdf(Fi);
    return;
  }
  // A warp with a lane in the near field (|P| < 4 L) and every lane within 64 L
  // evaluates the closed form on all lanes (warp-uniform): its log difference
  // loses at most ~64x to cancellation (~1e-12 of the pair's value), and the
  // warp runs one branch instead of both.
  const bool near_all = __any_sync(0xffffffffu, rho2.hi < 16.0f * Lh * Lh) &&
                        __all_sync(0xffffffffu, rho2.hi < 4096.0f * Lh * Lh);
  if (!near_all && rho2.hi >= 16.0f * Lh * Lh) {
    const df2 X = df_sub(px2, py2);
    df2 Y = df_mul(px, py);
    Y.hi *= 2.0f;
    Y.lo *= 2.0f;
    const df2 c2 = pf(s, ld, kC2, i), s2 = pf(s, ld, kS2, i);
    const df2 inv = df_rcp(rho2);
    const df2 q = df_mul(df_mul_f(pf(s, ld, kQ6, i), 6.0f), inv);  // L^2 / (4 |P|^2)
    // u = q (cos 2beta + i sin 2beta) conj(P)^2 / |P|^2 in double-float
    const df2 ure = df_mul(q, df_mul(df_add(df_mul(c2, X), df_mul(s2, Y)), inv));
    const df2 uim = df_mul(q, df_mul(df_sub(df_mul(s2, X), df_mul(c2, Y)), inv));
    // the first-order terms in double-float, the rest (below 5e-5 of the leading
    // term) in float32 from the leading word of u:
    //   F1 - 1 = u/3 + u^2 (1/5 + u (1/7 + u (1/9 + u/11))),
    //   -Re log(1 - u) = Re u + Re u^2 (1/2 + u (1/3 + u (1/4 + u/5)))
    const float ur = ure.hi, ui = uim.hi;
    const float u2r = ur * ur - ui * ui, u2i = 2.0f * ur * ui;
    float ar = (1.0f / 9.0f) + ur * (1.0f / 11.0f), ai = ui * (1.0f / 11.0f), tr;
    tr = (1.0f / 7.0f) + ur * ar - ui * ai; ai = ur * ai + ui * ar; ar = tr;
    tr = (1.0f / 5.0f) + ur * ar - ui * ai; ai = ur * ai + ui * ar; ar = tr;
    const float hFr = u2r * ar - u2i * ai, hFi = u2r * ai + u2i * ar;
    float br = 0.25f + ur * 0.2f, bi = ui * 0.2f;
    tr = (1.0f / 3.0f) + ur * br - ui * bi; bi = ur * bi + ui * br; br = tr;
    tr = 0.5f + ur * br - ui * bi; bi = ur * bi + ui * br; br = tr;
    const float hL = u2r * br - u2i * bi;
    const df2 third = df_const(kThird);
    const df2 Fre = df_add_f(df_mul(ure, third), hFr);
    const df2 Fim = df_add_f(df_mul(uim, third), hFi);
    // 2pi dG/dp = L inv conj(F1) P
    const df2 fr = df_add_f(Fre, 1.0f);
    const df2 Li = df_mul(L, inv);
    gpx = df_mul(Li, df_add(df_mul(fr, px), df_mul(Fim, py)));
    gpy = df_mul(Li, df_sub(df_mul(fr, py), df_mul(Fim, px)));
    // K = log|P| + Re log(1 - u)/2 + i Im F1
    df2 lg = df_log(rho2, tlog);
    lg.hi *= 0.5f;
    lg.lo *= 0.5f;
    const df2 rl = df_add_f(ure, hL);  // -Re log(1 - u)
    kr = df_sub(lg, mkdf(0.5f * rl.hi, 0.5f * rl.lo));
    ki = Fim;
    return;
  }
  // near field, panel frame (n = t rotated by +90 degrees)
  const df2 tx = pf(s, ld, kTx, i), ty = pf(s, ld, kTy, i);
  const df2 zeta = df_add(df_mul(px, tx), df_mul(py, ty));
  const df2 eta = df_sub(df_mul(py, tx), df_mul(px, ty));
  const df2 half = mkdf(0.5f * L.hi, 0.5f * L.lo);
  const df2 xi = df_add(zeta, half);
  const df2 a2 = df_sub(zeta, half);
  const df2 eta2 = df_sqr(eta);
  const df2 l1 = df_log(df_add(df_sqr(xi), eta2), tlog);
  const df2 l2 = df_log(df_add(df_sqr(a2), eta2), tlog);
  df2 th = mkdf(0.0f);
  if (!self) {
    const df2 quarterL2 = df_mul_f(pf(s, ld, kQ6, i), 6.0f);
    th = df_atan2(df_mul(L, eta), df_sub(rho2, quarterL2), tatan);
  }
  df2 hd = df_sub(l1, l2);
  hd.hi *= 0.5f;
  hd.lo *= 0.5f;
  gpx = df_sub(df_mul(hd, tx), df_mul(th, ty));
  gpy = df_add(df_mul(hd, ty), df_mul(th, tx));
  const df2 cn = df_div(df_sub(df_mul(hd, eta), df_mul(th, xi)), L);
  // K = (l2/2, cn) + (hd, theta)/2: 2pi dG/dp is R_t (hd, theta)
  kr = df_add(mkdf(0.5f * l2.hi, 0.5f * l2.lo), mkdf(0.5f * hd.hi, 0.5f * hd.lo));
  ki = df_add(cn, mkdf(0.5f * th.hi, 0.5f * th.lo));
}

// acc += a b with the product's two parts added to an unnormalised pair (the
// low word collects the rounding errors of a window of terms; acc_norm
// renormalises it at the end of the window).
__device__ __forceinline__ void acc_add_prod(df2& acc, df2 a, df2 b) {
  df2 p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
  p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
  const df2 t = two_sum(acc.hi, p.hi);
  acc.hi = t.hi;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(t.lo, p.lo));
}
__device__ __forceinline__ void acc_norm(df2& acc) { acc = two_sum(acc.hi, acc.lo); }

__device__ __forceinline__ df2 shfl_xor_df(df2 a, int o) {
  return mkdf(__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o));
}

// Sums over the 32 lanes of a window of 4 rows: lane l holds v[t] (row t, its
// own column).  Two halving exchanges (offsets 16, 8: each lane keeps half of
// its rows and adds the partner's copy of them) and three butterflies (4, 2,
// 1) leave the full sum of row (l >> 3) in every lane of the group l >> 3: 6
// double-float additions per window instead of 20 for four warp reductions.
__device__ __forceinline__ df2 warp_rowsum4(const df2 (&v)[4], int lane) {
  const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0;
  df2 k0 = b4 ? v[2] : v[0], k1 = b4 ? v[3] : v[1];
  const df2 s0 = b4 ? v[0] : v[2], s1 = b4 ? v[1] : v[3];
  k0 = df_add(k0, shfl_xor_df(s0, 16));
  k1 = df_add(k1, shfl_xor_df(s1, 16));
  df2 k = b3 ? k1 : k0;
  k = df_add(k, shfl_xor_df(b3 ? k0 : k1, 8));
  k = df_add(k, shfl_xor_df(k, 4));
  k = df_add(k, shfl_xor_df(k, 2));
  k = df_add(k, shfl_xor_df(k, 1));
  return k;
}

__device__ __forceinline__ df2 warp_sum_df2(df2 a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    a = df_add(a, mkdf(__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)));
  return a;
}

constexpr int kPartialsN = 256;

__global__ void __launch_bounds__(256) k_adjoint_df(
    Batch bt, const double* __restrict__ u, const double* __restrict__ lambda,
    const double* __restrict__ alpha, const double* __restrict__ vinf,
    const double* __restrict__ chord, const double* __restrict__ grad_cl,
    double* __restrict__ grad, const int32_t* __restrict__ info, int lam_weighted) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int ld = bt.n_max;
  float4* tlog = reinterpret_cast<float4*>(smraw);        // 257
  float2* tatan = reinterpret_cast<float2*>(tlog + 257);  // 34
  double* xs = reinterpret_cast<double*>(tatan + 34);     // n_max
  double* ys = xs + ld;
  double* P = ys + ld;                                    // 2 n_max (FP64 row sums)
  double* Ac = P + 2 * ld;                                // 2 n_max
  double* Bc = Ac + 2 * ld;                               // 2 n_max
  float* lamh = reinterpret_cast<float*>(Bc + 2 * ld);    // n_max (lambda as float pairs)
  float* laml = lamh + ld;
  float* pc = laml + ld;                                  // kPanelFields * n_max
  float4* Pw = reinterpret_cast<float4*>(pc + kPanelFields * ld);  // 8 * n_max

  const int b = bt.order[blockIdx.x];
  const int n = airfoil_n(bt, b);
  double* gout = grad + 2 * bt.node_off[b];
  if ((info && info[b] != 0) || n > ld || n < 3) {
    for (int k = threadIdx.x; k < 2 * n; k += blockDim.x) gout[k] = nan("");
    return;
  }
  const double* nodes = bt.nodes + 2 * bt.node_off[b];
  const double* ub = u + vec_off(bt, b);
  const double* lb = lambda + vec_off(bt, b);
  df_stage_tables(tlog, tatan);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    xs[k] = nodes[2 * k];
    ys[k] = nodes[2 * k + 1];
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) Pw[w * ld + k] = make_float4(0, 0, 0, 0);
    const df2 l = df_from_double(lb[k]);
    lamh[k] = l.hi;
    laml[k] = l.lo;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const int k1 = (k + 1 == n) ? 0 : k + 1;
    panel_constants(pc, ld, k, xs[k], ys[k], xs[k1], ys[k1]);
  }
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int ncb = (n + 31) >> 5;
  for (int cb = warp; cb < ncb; cb += nw) {
    const int i = cb * 32 + lane;
    const bool ok = i < n;
    const int ii = ok ? i : n - 1;
    const df2 ui = ok ? df_from_double(ub[ii]) : mkdf(0.0f);
    df2 sSx = mkdf(0.0f), sSy = mkdf(0.0f), sKr = mkdf(0.0f), sKi = mkdf(0.0f);
    // rows in windows of 4: the lane's u_i dG/dp terms are shifted into rx/ry
    // (static register indices with a rolled loop) and reduced per window
    df2 rx[4], ry[4];
    for (int j0 = 0; j0 < n; j0 += 4) {
#pragma unroll 1
      for (int t = 0; t < 4; ++t) {
        const int j = j0 + t;
        df2 vx = mkdf(0.0f), vy = mkdf(0.0f);
        if (j < n) {
          const point3 pj = load_point(pc, ld, j);
          df2 gpx, gpy, kr, ki;
          panel_dG_df(pj, pc, ld, ii, ii == j, tlog, tatan, gpx, gpy, kr, ki);
          const df2 lj = mkdf(lamh[j], laml[j]);
          // S_i += lambda_j gp, sum lambda_j K (B_i = R_t sum lambda K - S_i / 2)
          acc_add_prod(sSx, lj, gpx);
          acc_add_prod(sSy, lj, gpy);
          acc_add_prod(sKr, lj, kr);
          acc_add_prod(sKi, lj, ki);
          if (ok) {
            vx = df_mul(ui, gpx);
            vy = df_mul(ui, gpy);
          }
        }
        rx[0] = rx[1]; rx[1] = rx[2]; rx[2] = rx[3]; rx[3] = vx;
        ry[0] = ry[1]; ry[1] = ry[2]; ry[2] = ry[3]; ry[3] = vy;
      }
      acc_norm(sSx);
      acc_norm(sSy);
      acc_norm(sKr);
      acc_norm(sKi);
      const df2 sx = warp_rowsum4(rx, lane), sy = warp_rowsum4(ry, lane);
      const int jr = j0 + (lane >> 3);
      if ((lane & 7) == 0 && jr < n) {
        const float4 q = Pw[warp * ld + jr];
        const df2 px = df_add(mkdf(q.x, q.y), sx), py = df_add(mkdf(q.z, q.w), sy);
        Pw[warp * ld + jr] = make_float4(px.hi, px.lo, py.hi, py.lo);
      }
    }
    if (ok) {
      // B_i = R_t K - S_i / 2 with the panel's FP64 unit tangent; A_i = -S_i - B_i
      const int i1 = (i + 1 == n) ? 0 : i + 1;
      const double hx = xs[i1] - xs[i], hy = ys[i1] - ys[i];
      const double Li = sqrt(hx * hx + hy * hy), tx = hx / Li, ty = hy / Li;
      const double Sx = df_to_double(sSx), Sy = df_to_double(sSy);
      const double Kr = df_to_double(sKr), Ki = df_to_double(sKi);
      const double bx = tx * Kr - ty * Ki - 0.5 * Sx, by = ty * Kr + tx * Ki - 0.5 * Sy;
      Ac[2 * i] = -(Sx + bx);
      Ac[2 * i + 1] = -(Sy + by);
      Bc[2 * i] = bx;
      Bc[2 * i + 1] = by;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    df2 sx = mkdf(0.0f), sy = mkdf(0.0f);
    for (int w = 0; w < nw; ++w) {
      const float4 q = Pw[w * ld + k];
      sx = df_add(sx, mkdf(q.x, q.y));
      sy = df_add(sy, mkdf(q.z, q.w));
    }
    P[2 * k] = df_to_double(sx);
    P[2 * k + 1] = df_to_double(sy);
  }
  __syncthreads();
  const double v = vinf ? vinf[b] : 1.0, c = chord ? chord[b] : 1.0;
  const double ca = cos(alpha[b]), sa = sin(alpha[b]);
  // se scales the explicit dCl/dx term, sl the lambda terms: the upstream
  // dL/dCl for both when lambda solves M^T lambda = dCl/du, or (w_cl, 1) when
  // lambda already carries the weights of a vector-Jacobian product
  const double se = grad_cl ? grad_cl[b] : (lam_weighted ? 0.0 : 1.0);
  const double sl = lam_weighted ? 1.0 : se;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const int km = (k == 0) ? n - 1 : k - 1;
    const int k1 = (k + 1 == n) ? 0 : k + 1;
    // unit tangents of panels k-1 and k from the FP64 nodes
    const double hkx = xs[k1] - xs[k], hky = ys[k1] - ys[k];
    const double hmx = xs[k] - xs[km], hmy = ys[k] - ys[km];
    const double Lk = sqrt(hkx * hkx + hky * hky), Lm = sqrt(hmx * hmx + hmy * hmy);
    const double ex = 2.0 / (v * c) * (ub[km] * hmx / Lm - ub[k] * hkx / Lk);
    const double ey = 2.0 / (v * c) * (ub[km] * hmy / Lm - ub[k] * hky / Lk);
    double gx = 0.5 * v * (-sa) * (lb[km] + lb[k]);
    double gy = 0.5 * v * ca * (lb[km] + lb[k]);
    gx += kInvTwoPi * (0.5 * (lb[km] * P[2 * km] + lb[k] * P[2 * k]) + ub[k] * Ac[2 * k] +
                       ub[km] * Bc[2 * km]);
    gy += kInvTwoPi * (0.5 * (lb[km] * P[2 * km + 1] + lb[k] * P[2 * k + 1]) +
                       ub[k] * Ac[2 * k + 1] + ub[km] * Bc[2 * km + 1]);
    gout[2 * k] = se * ex + sl * gx;
    gout[2 * k + 1] = se * ey + sl * gy;
  }
}

// ---------------------------------------------------------------------------
// Large airfoils (n > kPartialsN): block (x, y) takes the panels [256 y,
// 256 y + 256) of airfoil order[x] -- one 32-column block per warp -- against
// every control point.  Shared memory holds the control points of all rows,
// lambda, and the constants of the block's own panels only.  Rows are swept in
// windows of 32: each warp leaves its warp-reduced P_j partials in shared
// memory, one warp sums the eight and adds lambda_j P_j / 2 to nodes j and
// j + 1 of the gradient.  The caller's gradient rows are set to zero (or NaN for
// a failed airfoil) by k_adjoint_prepare first; every contribution goes in by
// an FP64 atomic add, so the summation order, and the last bits, vary between
// runs.
// ---------------------------------------------------------------------------
constexpr int kSplitChunk = 256;

__global__ void k_adjoint_prepare(Batch bt, double* __restrict__ grad,
                                  const int32_t* __restrict__ info) {
  const int b = bt.order[blockIdx.x];
  const int n = airfoil_n(bt, b);
  const bool bad = (info && info[b] != 0) || n > bt.n_max || n < 3;
  double* gout = grad + 2 * bt.node_off[b];
  for (int k = threadIdx.x; k < 2 * n; k += blockDim.x) gout[k] = bad ? nan("") : 0.0;
}

__global__ void __launch_bounds__(256) k_adjoint_df_split(
    Batch bt, const double* __restrict__ u, const double* __restrict__ lambda,
    const double* __restrict__ alpha, const double* __restrict__ vinf,
    const double* __restrict__ chord, const double* __restrict__ grad_cl,
    double* __restrict__ grad, const int32_t* __restrict__ info, int lam_weighted) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int ld = bt.n_max;
  float4* tlog = reinterpret_cast<float4*>(smraw);        // 257
  float2* tatan = reinterpret_cast<float2*>(tlog + 257);  // 34
  float4* win = reinterpret_cast<float4*>(tatan + 34);    // 8 warps x 32 rows
  // the current window's 32 rows, two buffers: control points (6 split
  // coordinates, stride 32) and lambda as a float pair
  float* wrow = reinterpret_cast<float*>(win + 8 * 32);   // 2 x 8 x 32
  float* cpc = wrow + 2 * 8 * 32;                         // kPanelFields * kSplitChunk

  const int b = bt.order[blockIdx.x];
  const int n = airfoil_n(bt, b);
  const int i0 = blockIdx.y * kSplitChunk;
  if ((info && info[b] != 0) || n > ld || n < 3 || i0 >= n) return;
  const double* nodes = bt.nodes + 2 * bt.node_off[b];
  const double* ub = u + vec_off(bt, b);
  const double* lb = lambda + vec_off(bt, b);
  double* gout = grad + 2 * bt.node_off[b];
  const int nc = min(kSplitChunk, n - i0);
  df_stage_tables(tlog, tatan);
  // the rows of window j0 into buffer (j0 / 32) & 1, a thread per row
  auto stage_rows = [&](int j0) {
    const int t = threadIdx.x, k = j0 + t;
    if (t < 32 && k < n) {
      float* w = wrow + ((j0 >> 5) & 1) * 256;
      const int k1 = (k + 1 == n) ? 0 : k + 1;
      const point3 c = make_point(0.5 * (nodes[2 * k] + nodes[2 * k1]),
                                  0.5 * (nodes[2 * k + 1] + nodes[2 * k1 + 1]));
      w[kCx * 32 + t] = c.xh;
      w[(kCx + 1) * 32 + t] = c.xm;
      w[(kCx + 2) * 32 + t] = c.xl;
      w[kCy * 32 + t] = c.yh;
      w[(kCy + 1) * 32 + t] = c.ym;
      w[(kCy + 2) * 32 + t] = c.yl;
      const df2 l = df_from_double(lb[k]);
      w[6 * 32 + t] = l.hi;
      w[7 * 32 + t] = l.lo;
    }
  };
  for (int k = threadIdx.x; k < nc; k += blockDim.x) {
    const int i = i0 + k, i1 = (i + 1 == n) ? 0 : i + 1;
    panel_constants(cpc, kSplitChunk, k, nodes[2 * i], nodes[2 * i + 1], nodes[2 * i1],
                    nodes[2 * i1 + 1]);
  }
  const double v = vinf ? vinf[b] : 1.0, c = chord ? chord[b] : 1.0;
  // se scales the explicit dCl/dx term, sl the lambda terms (as in k_adjoint_df)
  const double se = grad_cl ? grad_cl[b] : (lam_weighted ? 0.0 : 1.0);
  const double sl = lam_weighted ? 1.0 : se;
  const double w2pi = sl * kInvTwoPi;
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int il = 32 * warp + lane;  // column within the chunk
  const int i = i0 + il;
  const bool ok = il < nc;
  const bool warp_on = 32 * warp < nc;
  const int ic = ok ? il : 0;
  const df2 ui = ok ? df_from_double(ub[i]) : mkdf(0.0f);
  df2 sSx = mkdf(0.0f), sSy = mkdf(0.0f), sKr = mkdf(0.0f), sKi = mkdf(0.0f);
  for (int j0 = 0; j0 < n; j0 += 32) {
    const int jn = min(32, n - j0);
    stage_rows(j0);
    __syncthreads();
    const float* wr = wrow + ((j0 >> 5) & 1) * 256;
    if (warp_on) {
      df2 rx[4], ry[4];
      for (int t0 = 0; t0 < jn; t0 += 4) {
#pragma unroll 1
        for (int t = t0; t < t0 + 4; ++t) {
          const int j = j0 + t;
          df2 vx = mkdf(0.0f), vy = mkdf(0.0f);
          if (t < jn) {
            const point3 pj = load_point(wr, 32, t);
            df2 gpx, gpy, kr, ki;
            panel_dG_df(pj, cpc, kSplitChunk, ic, ok && i == j, tlog, tatan, gpx, gpy, kr, ki);
            const df2 lj = mkdf(wr[6 * 32 + t], wr[7 * 32 + t]);
            acc_add_prod(sSx, lj, gpx);
            acc_add_prod(sSy, lj, gpy);
            acc_add_prod(sKr, lj, kr);
            acc_add_prod(sKi, lj, ki);
            if (ok) {
              vx = df_mul(ui, gpx);
              vy = df_mul(ui, gpy);
            }
          }
          rx[0] = rx[1]; rx[1] = rx[2]; rx[2] = rx[3]; rx[3] = vx;
          ry[0] = ry[1]; ry[1] = ry[2]; ry[2] = ry[3]; ry[3] = vy;
        }
        acc_norm(sSx);
        acc_norm(sSy);
        acc_norm(sKr);
        acc_norm(sKi);
        const df2 sx = warp_rowsum4(rx, lane), sy = warp_rowsum4(ry, lane);
        const int tr = t0 + (lane >> 3);
        if ((lane & 7) == 0 && tr < jn) win[warp * 32 + tr] = make_float4(sx.hi, sx.lo, sy.hi, sy.lo);
      }
    } else if (lane < jn) {
      win[warp * 32 + lane] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    __syncthreads();
    if (warp == 0 && lane < jn) {
      df2 sx = mkdf(0.0f), sy = mkdf(0.0f);
#pragma unroll
      for (int w = 0; w < 8; ++w) {
        const float4 q = win[w * 32 + lane];
        sx = df_add(sx, mkdf(q.x, q.y));
        sy = df_add(sy, mkdf(q.z, q.w));
      }
      // lambda_j P_j / 2 belongs to the nodes j and j + 1 (the ends of panel j)
      const int j = j0 + lane, j1 = (j + 1 == n) ? 0 : j + 1;
      const double f = 0.5 * w2pi * lb[j];
      const double px = f * df_to_double(sx), py = f * df_to_double(sy);
      atomicAdd(&gout[2 * j], px);
      atomicAdd(&gout[2 * j + 1], py);
      atomicAdd(&gout[2 * j1], px);
      atomicAdd(&gout[2 * j1 + 1], py);
    }
    __syncthreads();
  }
  if (ok) {
    // u_i A_i belongs to node i (start of panel i), u_i B_i to node i + 1
    const int i1 = (i + 1 == n) ? 0 : i + 1;
    const double f = w2pi * ub[i];
    // B_i = R_t K - S_i / 2 with the panel's FP64 unit tangent; A_i = -S_i - B_i
    const double hx = nodes[2 * i1] - nodes[2 * i], hy = nodes[2 * i1 + 1] - nodes[2 * i + 1];
    const double Li = sqrt(hx * hx + hy * hy), tx = hx / Li, ty = hy / Li;
    const double Sx = df_to_double(sSx), Sy = df_to_double(sSy);
    const double Kr = df_to_double(sKr), Ki = df_to_double(sKi);
    const double bx = tx * Kr - ty * Ki - 0.5 * Sx, by = ty * Kr + tx * Ki - 0.5 * Sy;
    atomicAdd(&gout[2 * i], -f * (Sx + bx));
    atomicAdd(&gout[2 * i + 1], -f * (Sy + by));
    atomicAdd(&gout[2 * i1], f * bx);
    atomicAdd(&gout[2 * i1 + 1], f * by);
  }
  if (blockIdx.y == 0) {
    // the terms that need no pair sums, once per node
    const double ca = cos(alpha[b]), sa = sin(alpha[b]);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const int km = (k == 0) ? n - 1 : k - 1;
      const int k1 = (k + 1 == n) ? 0 : k + 1;
      const double hkx = nodes[2 * k1] - nodes[2 * k], hky = nodes[2 * k1 + 1] - nodes[2 * k + 1];
      const double hmx = nodes[2 * k] - nodes[2 * km], hmy = nodes[2 * k + 1] - nodes[2 * km + 1];
      const double Lk = sqrt(hkx * hkx + hky * hky), Lm = sqrt(hmx * hmx + hmy * hmy);
      const double ex = 2.0 / (v * c) * (ub[km] * hmx / Lm - ub[k] * hkx / Lk);
      const double ey = 2.0 / (v * c) * (ub[km] * hmy / Lm - ub[k] * hky / Lk);
      const double bx = 0.5 * v * (-sa) * (lb[km] + lb[k]);
      const double by = 0.5 * v * ca * (lb[km] + lb[k]);
      atomicAdd(&gout[2 * k], se * ex + sl * bx);
      atomicAdd(&gout[2 * k + 1], se * ey + sl * by);
    }
  }
}

size_t adjoint_df_smem(int n_max) {
  if (n_max > kPartialsN)
    return 257 * 16 + 34 * 8 + 8 * 32 * 16 + 2 * 8 * 32 * 4 +
           (size_t)kPanelFields * kSplitChunk * 4;
  return 257 * 16 + 34 * 8 + (size_t)n_max * 8 * 8 + (size_t)n_max * 4 * 2 +
         (size_t)kPanelFields * n_max * 4 + (size_t)8 * n_max * 16;
}

cudaError_t launch_adjoint_df(const Batch& bt, const double* u, const double* lambda,
                              const double* alpha, const double* vinf, const double* chord,
                              const double* grad_cl, double* grad, const int32_t* info,
                              cudaStream_t s, bool lam_weighted) {
  const size_t smem = adjoint_df_smem(bt.n_max);
  cudaError_t e;
  if (bt.n_max <= kPartialsN) {
    e = ensure_smem(k_adjoint_df, smem);
    if (e != cudaSuccess) return e;
    k_adjoint_df<<<bt.B, 256, smem, s>>>(bt, u, lambda, alpha, vinf, chord, grad_cl, grad, info,
                                         lam_weighted ? 1 : 0);
  } else {
    e = ensure_smem(k_adjoint_df_split, smem);
    if (e != cudaSuccess) return e;
    k_adjoint_prepare<<<bt.B, 256, 0, s>>>(bt, grad, info);
    const dim3 grid(bt.B, (bt.n_max + kSplitChunk - 1) / kSplitChunk);
    k_adjoint_df_split<<<grid, 256, smem, s>>>(bt, u, lambda, alpha, vinf, chord, grad_cl, grad,
                                               info, lam_weighted ? 1 : 0);
  }
  return cudaGetLastError();
}

}  // namespace panel
