// k_viscous.cu -- the viscous correction of Section 2: Thwaites's laminar
// boundary-layer method on the inviscid surface speed, giving the momentum
// thickness, skin friction, laminar separation and the drag (the paper names
// Thwaites's method for the drag and validates it on a circular cylinder; the
// optimisation of Section 3 maximises lift over drag).  FP64 throughout: the
// work is O(n) per airfoil against the O(n^2) assembly.
//
// The paper prints no formulas; the textbook method is used and the choices it
// leaves open are the library's:
//   U_j = |gamma_j| / v_inf at control point j (lengths in chords, speeds in v_inf);
//   stagnation point between control points j and j+1 for the first j with
//   gamma_j > 0 >= gamma_{j+1}, at the linear zero of gamma along the surface
//   (distance d_j = (L_j + L_{j+1}) / 2); the upper surface marches through
//   control points j, j-1, .., 0, the lower through j+1, .., n-1 (j+1 left out
//   when gamma_{j+1} = 0), each ending at the trailing-edge node half a panel
//   beyond its last control point at that point's speed;
//   theta^2 U^6 = (0.45 / Re) int U^5 ds with U linear between consecutive
//   points (each piece integrated exactly), theta^2 = 0.075 / (Re U'(0)) at the
//   stagnation point; lambda = Re theta^2 dU/ds with the derivative of the
//   quadratic through a point and its neighbours (one-sided at the ends);
//   Cebeci-Bradshaw fits l(lambda), H(lambda) with lambda clamped to
//   [-0.09, 0.1]; laminar separation at the first control point with
//   lambda < -0.09 (or U = 0), past which the wall shear is zero and H keeps its
//   separation value while theta follows the same integral; cf = 2 l U /
//   (Re theta); Cd_f = sum of cf integrated along the freestream direction
//   (trapezoid); Cd by Squire and Young, 2 theta U^((H + 5) / 2) per surface at
//   the trailing edge.
//
// One warp per surface, two per airfoil.  A surface is marched in chunks of 32
// points, one per lane: every per-point quantity except the integral needs only
// the point and its neighbours (shuffles); the integral is a warp prefix sum
// with a carry between chunks, and the separation point is the first lane of a
// ballot.
#include "panel_common.cuh"

namespace panel {

namespace {

constexpr double kLambdaSep = -0.09;
constexpr double kLambdaMax = 0.1;

__device__ __forceinline__ void shear_shape(double lam, double& l, double& H) {
  lam = fmin(fmax(lam, kLambdaSep), kLambdaMax);
  if (lam >= 0.0) {
    l = 0.22 + 1.57 * lam - 1.8 * lam * lam;
    H = 2.61 - 3.75 * lam + 5.24 * lam * lam;
  } else {
    l = 0.22 + 1.402 * lam + 0.018 * lam / (lam + 0.107);
    H = 2.088 + 0.0731 / (lam + 0.14);
  }
}

// One airfoil's surface geometry and speeds, in chords and v_inf.
struct Foil {
  const double* x;  // nodes [n][2]
  const double* g;  // gamma [n]
  int n;
  double inv_c, inv_v;

  __device__ __forceinline__ double q(int j) const { return g[j] * inv_v; }
  __device__ __forceinline__ double px(int k) const { return x[2 * (k == n ? 0 : k)] * inv_c; }
  __device__ __forceinline__ double py(int k) const {
    return x[2 * (k == n ? 0 : k) + 1] * inv_c;
  }
  __device__ __forceinline__ double len(int j) const {
    return hypot(px(j + 1) - px(j), py(j + 1) - py(j));
  }
  __device__ __forceinline__ double mx(int j) const { return 0.5 * (px(j) + px(j + 1)); }
  __device__ __forceinline__ double my(int j) const { return 0.5 * (py(j) + py(j + 1)); }
};

// One surface: marching point 0 is the stagnation point, 1..K control points
// first, first + step, .., K+1 the trailing edge (at control point K's speed).
struct Surface {
  int K, first, step;
  double h1;        // distance from the stagnation point to marching point 1
  double p0x, p0y;  // stagnation point
  __device__ __forceinline__ int cp(int k) const { return first + step * (k - 1); }
};

__device__ __forceinline__ double warp_incl_scan(double v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Marches one surface with one warp, 32 points per chunk.  Every lane holds
// its point's speed U, panel length L, step h and position P; the neighbours'
// values come by shuffles, across chunk boundaries from carries (previous
// chunk) or a direct evaluation (lane 31's next point).  Returns on every lane
// the surface's Squire-Young and friction drag terms and its separating
// control point (-1 if none).
__device__ void march_surface(const Foil& F, const Surface& S, double Re, double ex, double ey,
                              int lane, double* __restrict__ theta_out,
                              double* __restrict__ cf_out, double& cd_s, double& cdf_s,
                              int& sep) {
  const unsigned full = 0xffffffffu;
  const int K = S.K;
  // carries: values of points base-1 (and base-2 for U) of the previous chunk
  double cI = 0.0, cU1 = 0.0, cU2 = 0.0, cL = 0.0, cH = 0.0, cLam = 0.0, cCf = 0.0;
  double cPx = S.p0x, cPy = S.p0y;
  bool separated = false;
  int e = K + 1;
  cd_s = 0.0;
  cdf_s = 0.0;
  for (int base = 1; base <= K + 1; base += 32) {
    const int k = base + lane;
    const bool live = k <= K + 1;
    const int c = S.cp(k < K ? k : K);
    const double Uo = fabs(F.q(c));
    const double Lo = F.len(c);
    const double Pxo = (k == K + 1) ? F.px(0) : F.mx(c);
    const double Pyo = (k == K + 1) ? F.py(0) : F.my(c);
    double Lprev = __shfl_up_sync(full, Lo, 1);
    double Uprev = __shfl_up_sync(full, Uo, 1);
    double Uprev2 = __shfl_up_sync(full, Uo, 2);
    double Pxp = __shfl_up_sync(full, Pxo, 1);
    double Pyp = __shfl_up_sync(full, Pyo, 1);
    if (lane == 0) {
      Lprev = cL;
      Uprev = cU1;
      Uprev2 = cU2;
      Pxp = cPx;
      Pyp = cPy;
    } else if (lane == 1) {
      Uprev2 = cU1;
    }
    const double hk = (k == 1) ? S.h1 : (k == K + 1 ? 0.5 * Lo : 0.5 * (Lprev + Lo));
    double hprev = __shfl_up_sync(full, hk, 1);
    if (lane == 0) hprev = cH;
    double Unext = __shfl_down_sync(full, Uo, 1);
    double hnext = __shfl_down_sync(full, hk, 1);
    if (lane == 31 && k < K) {
      const int cn = S.cp(k + 1);
      Unext = fabs(F.q(cn));
      hnext = 0.5 * (Lo + F.len(cn));
    }
    // Thwaites's integral: U linear on [k-1, k]
    double g = 0.0;
    if (live) {
      const double a = Uprev, a2 = a * a, b2 = Uo * Uo;
      g = hk * (a2 * a2 * a + a2 * a2 * Uo + a2 * a * b2 + a2 * b2 * Uo + a * b2 * b2 +
                b2 * b2 * Uo) / 6.0;
    }
    const double I = cI + warp_incl_scan(g, lane);
    double dUk = 0.0;
    if (k < K) {
      dUk = (hk * hk * (Unext - Uo) + hnext * hnext * (Uo - Uprev)) / (hk * hnext * (hk + hnext));
    } else if (k == K) {
      if (K >= 2) {
        const double a = hprev, b = hk;
        dUk = Uprev2 * b / (a * (a + b)) - Uprev * (a + b) / (a * b) +
              Uo * (a + 2.0 * b) / (b * (a + b));
      } else {
        dUk = (Uo - Uprev) / hk;
      }
    }
    double th2, lam;
    if (Uo == 0.0) {
      th2 = INFINITY;
      lam = -INFINITY;
    } else {
      const double U3 = Uo * Uo * Uo;
      th2 = 0.45 * I / (Re * (U3 * U3));
      lam = Re * th2 * dUk;
    }
    // the trailing edge takes control point K's lambda
    double lam_prev = __shfl_up_sync(full, lam, 1);
    if (lane == 0) lam_prev = cLam;
    if (k == K + 1) lam = lam_prev;
    // laminar separation: the first control point with lambda < -0.09
    const unsigned m = __ballot_sync(full, live && k <= K && !(lam >= kLambdaSep));
    if (!separated && m) e = base + __ffs(m) - 1;
    const bool sep_k = (separated || m) && k >= e;
    double l, H;
    shear_shape(sep_k ? kLambdaSep : lam, l, H);
    const double th = sqrt(th2);
    const double cfk = (live && !sep_k) ? 2.0 * l * Uo / (Re * th) : 0.0;
    double cf_prev = __shfl_up_sync(full, cfk, 1);
    if (lane == 0) cf_prev = cCf;
    double term = 0.0;
    if (live) term = 0.5 * (cf_prev + cfk) * ((Pxo - Pxp) * ex + (Pyo - Pyp) * ey);
    cdf_s += warp_sum(term);
    if (live && k <= K) {
      if (theta_out) theta_out[c] = th;
      if (cf_out) cf_out[c] = cfk;
    }
    if (k == K + 1) cd_s = 2.0 * th * pow(Uo, 0.5 * (H + 5.0));
    separated = separated || m;
    cI = __shfl_sync(full, I, 31);
    cU1 = __shfl_sync(full, Uo, 31);
    cU2 = __shfl_sync(full, Uo, 30);
    cL = __shfl_sync(full, Lo, 31);
    cH = __shfl_sync(full, hk, 31);
    cLam = __shfl_sync(full, lam, 31);
    cCf = __shfl_sync(full, cfk, 31);
    cPx = __shfl_sync(full, Pxo, 31);
    cPy = __shfl_sync(full, Pyo, 31);
  }
  cd_s = __shfl_sync(full, cd_s, K % 32);
  sep = (e <= K) ? S.cp(e) : -1;
}

}  // namespace

// Two airfoils per block of four warps: warp 2a marches airfoil a's upper
// surface, warp 2a+1 its lower surface; the pair's sums meet in shared memory.
__global__ void __launch_bounds__(128) k_viscous(Batch bt, const double* __restrict__ u,
                                                 const double* __restrict__ alpha,
                                                 const double* __restrict__ vinf,
                                                 const double* __restrict__ chord,
                                                 const double* __restrict__ reynolds,
                                                 const int32_t* __restrict__ info,
                                                 const double* __restrict__ cl,
                                                 double* __restrict__ ld,
                                                 double* __restrict__ cd,
                                                 double* __restrict__ cd_f,
                                                 double* __restrict__ theta,
                                                 double* __restrict__ cf,
                                                 int32_t* __restrict__ sep) {
  __shared__ double s_cd[4], s_cdf[4];
  __shared__ int s_sep[4], s_ok[4];
  const int wib = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int b = blockIdx.x * 2 + (wib >> 1);
  const int side = wib & 1;
  const bool have = b < bt.B;
  double cd_s = 0.0, cdf_s = 0.0;
  int sep_s = -2;
  bool ok = false;
  int n = 0;
  double* th_b = nullptr;
  double* cf_b = nullptr;
  if (have) {
    n = airfoil_n(bt, b);
    const int64_t o0 = bt.node_off[b];
    th_b = theta ? theta + o0 : nullptr;
    cf_b = cf ? cf + o0 : nullptr;
    const double Re = reynolds[b];
    const Foil F{bt.nodes + 2 * o0, u + vec_off(bt, b), n, 1.0 / (chord ? chord[b] : 1.0),
                 1.0 / (vinf ? vinf[b] : 1.0)};
    // stagnation point: the first j with q_j > 0 >= q_{j+1}
    int j = -1;
    ok = !(info && info[b] != 0) && n >= 3 && Re > 0.0 && Re < INFINITY;
    if (ok) {
      for (int base = 0; base < n - 1; base += 32) {
        const int i = base + lane;
        const bool hit = i < n - 1 && F.q(i) > 0.0 && F.q(i + 1) <= 0.0;
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (m) {
          j = base + __ffs(m) - 1;
          break;
        }
      }
      ok = j >= 0;
    }
    int skip = 0;
    if (ok) {
      skip = F.q(j + 1) == 0.0;
      ok = j + 1 + skip < n;
    }
    if (ok) {
      const double qj = F.q(j), qj1 = F.q(j + 1);
      const double f = qj / (qj - qj1);
      const double Lj = F.len(j), Lj1 = F.len(j + 1);
      const double dj = 0.5 * (Lj + Lj1);
      const double t = f * dj;
      double p0x, p0y;
      if (t <= 0.5 * Lj) {
        const double r = t / (0.5 * Lj);
        p0x = F.mx(j) + r * (F.px(j + 1) - F.mx(j));
        p0y = F.my(j) + r * (F.py(j + 1) - F.my(j));
      } else {
        const double r = (t - 0.5 * Lj) / (0.5 * Lj1);
        p0x = F.px(j + 1) + r * (F.mx(j + 1) - F.px(j + 1));
        p0y = F.py(j + 1) + r * (F.my(j + 1) - F.py(j + 1));
      }
      const double a = alpha[b];
      const double ex = cos(a), ey = sin(a);
      if (side == 0) {
        const Surface S{j + 1, j, -1, f * dj, p0x, p0y};
        march_surface(F, S, Re, ex, ey, lane, th_b, cf_b, cd_s, cdf_s, sep_s);
      } else {
        const double h1 = skip ? 0.5 * (Lj1 + F.len(j + 2)) : (1.0 - f) * dj;
        const Surface S{n - 1 - j - skip, j + 1 + skip, 1, h1, p0x, p0y};
        march_surface(F, S, Re, ex, ey, lane, th_b, cf_b, cd_s, cdf_s, sep_s);
        if (skip && lane == 0) {
          // control point j+1 is the stagnation point itself
          const double U1 = fabs(F.q(j + 2));
          if (th_b) th_b[j + 1] = sqrt(0.075 / (Re * (U1 / h1)));
          if (cf_b) cf_b[j + 1] = 0.0;
        }
      }
    } else if (side == 0) {
      for (int i = lane; i < n; i += 32) {
        if (th_b) th_b[i] = nan("");
        if (cf_b) cf_b[i] = nan("");
      }
    }
  }
  if (lane == 0) {
    s_cd[wib] = cd_s;
    s_cdf[wib] = cdf_s;
    s_sep[wib] = sep_s;
    s_ok[wib] = ok;
  }
  __syncthreads();
  if (have && side == 0 && lane == 0) {
    if (s_ok[wib]) {
      const double cdv = s_cd[wib] + s_cd[wib + 1];
      cd[b] = cdv;
      if (cd_f) cd_f[b] = s_cdf[wib] + s_cdf[wib + 1];
      if (ld) ld[b] = cl[b] / cdv;
      if (sep) {
        sep[2 * b] = s_sep[wib];
        sep[2 * b + 1] = s_sep[wib + 1];
      }
    } else {
      cd[b] = nan("");
      if (cd_f) cd_f[b] = nan("");
      if (ld) ld[b] = nan("");
      if (sep) sep[2 * b] = sep[2 * b + 1] = -2;
    }
  }
}

cudaError_t launch_viscous(const Batch& bt, const double* u, const double* alpha,
                           const double* vinf, const double* chord, const double* reynolds,
                           const int32_t* info, const double* cl, double* ld, double* cd,
                           double* cd_f, double* theta, double* cf, int32_t* sep,
                           cudaStream_t s) {
  k_viscous<<<(bt.B + 1) / 2, 128, 0, s>>>(
      bt, u, alpha, vinf, chord, reynolds, info, cl, ld, cd, cd_f, theta, cf, sep);
  return cudaGetLastError();
}

}  // namespace panel
