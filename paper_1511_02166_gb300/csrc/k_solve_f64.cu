// k_solve_f64.cu -- plain FP64 path: LU with partial pivoting and solve.
//
// One block per airfoil works on its (n+1)^2 matrix in global memory (the
// FP64 matrix of a 200-panel airfoil, 323 KB, does not fit in shared memory).
// Right-looking elimination: pivot = largest |a_rk| (lowest row on ties, as in
// the oracle), physical row swap, multipliers, rank-1 update; then P b,
// forward substitution with the unit-lower factor and back substitution.
// This is the "plain all-FP64 per-airfoil" baseline; it does no refinement.
#include "panel_common.cuh"

namespace panel {

// Pivot search over rows k..m-1 of column k by warp 0; result in *s_piv.
__device__ __forceinline__ void pivot_search_f64(const double* F, int m, int k, int* s_piv) {
  if (threadIdx.x < 32) {
    double best = -1.0;
    int bi = k;
    for (int r = k + threadIdx.x; r < m; r += 32) {
      double v = fabs(F[(int64_t)r * m + k]);
      if (v > best) { best = v; bi = r; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double ov = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (threadIdx.x == 0) *s_piv = bi;
  }
}

// Factor F (m x m, row-major, global) in place; returns 0 or k+1 for a zero pivot.
__device__ int lu_factor_f64(double* F, int32_t* piv, int m, int* s_piv) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = 0; k < m; ++k) {
    pivot_search_f64(F, m, k, s_piv);
    __syncthreads();
    const int p = *s_piv;
    const double akk = F[(int64_t)p * m + k];
    if (akk == 0.0) return k + 1;  // uniform across the block
    if (threadIdx.x == 0) piv[k] = p;
    if (p != k) {
      for (int c = threadIdx.x; c < m; c += blockDim.x) {
        double t = F[(int64_t)k * m + c];
        F[(int64_t)k * m + c] = F[(int64_t)p * m + c];
        F[(int64_t)p * m + c] = t;
      }
    }
    __syncthreads();
    const double inv = 1.0 / akk;
    for (int r = k + 1 + threadIdx.x; r < m; r += blockDim.x) F[(int64_t)r * m + k] *= inv;
    __syncthreads();
    for (int r = k + 1 + warp; r < m; r += nw) {
      const double l = F[(int64_t)r * m + k];
      double* fr = F + (int64_t)r * m;
      const double* fk = F + (int64_t)k * m;
      for (int c = k + 1 + lane; c < m; c += 32) fr[c] = fma(-l, fk[c], fr[c]);
    }
    __syncthreads();
  }
  return 0;
}

// x <- (P^T L U)^{-1} x, i.e. solve M x = b with the factors; x in shared memory.
__device__ void lu_solve_f64(const double* F, const int32_t* piv, int m, double* x) {
  if (threadIdx.x == 0)
    for (int k = 0; k < m; ++k) {
      int p = piv[k];
      if (p != k) { double t = x[k]; x[k] = x[p]; x[p] = t; }
    }
  __syncthreads();
  for (int k = 0; k < m; ++k) {  // unit lower
    const double xk = x[k];
    for (int r = k + 1 + threadIdx.x; r < m; r += blockDim.x) x[r] = fma(-F[(int64_t)r * m + k], xk, x[r]);
    __syncthreads();
  }
  for (int k = m - 1; k >= 0; --k) {  // upper
    if (threadIdx.x == 0) x[k] /= F[(int64_t)k * m + k];
    __syncthreads();
    const double xk = x[k];
    for (int r = threadIdx.x; r < k; r += blockDim.x) x[r] = fma(-F[(int64_t)r * m + k], xk, x[r]);
    __syncthreads();
  }
}

// y <- M^{-T} y with M = P^T L U:  U^T z = y, L^T w = z, y = P^T w.
__device__ void lu_solve_transposed_f64(const double* F, const int32_t* piv, int m, double* y) {
  for (int k = 0; k < m; ++k) {  // U^T is lower triangular
    if (threadIdx.x == 0) y[k] /= F[(int64_t)k * m + k];
    __syncthreads();
    const double yk = y[k];
    for (int r = k + 1 + threadIdx.x; r < m; r += blockDim.x) y[r] = fma(-F[(int64_t)k * m + r], yk, y[r]);
    __syncthreads();
  }
  for (int k = m - 1; k >= 0; --k) {  // L^T unit upper
    const double yk = y[k];
    for (int r = threadIdx.x; r < k; r += blockDim.x) y[r] = fma(-F[(int64_t)k * m + r], yk, y[r]);
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = m - 1; k >= 0; --k) {
      int p = piv[k];
      if (p != k) { double t = y[k]; y[k] = y[p]; y[p] = t; }
    }
  __syncthreads();
}

// g = dCl/du: g_i = 2 |h_i| / (v_inf c) for the strengths, 0 for C.
__device__ void cl_sensitivity_f64(const double* nodes, int n, double v, double c, double* g) {
  const int m = n + 1;
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    if (k < n) {
      int k1 = (k + 1 == n) ? 0 : k + 1;
      double hx = nodes[2 * k1] - nodes[2 * k], hy = nodes[2 * k1 + 1] - nodes[2 * k + 1];
      g[k] = 2.0 * sqrt(hx * hx + hy * hy) / (v * c);
    } else {
      g[k] = 0.0;
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) k_solve_f64(Batch bt, const double* __restrict__ A,
                                                   double* __restrict__ LU, int32_t* __restrict__ piv,
                                                   const double* __restrict__ rhs,
                                                   const double* __restrict__ vinf,
                                                   const double* __restrict__ chord,
                                                   double* __restrict__ u, double* __restrict__ lambda,
                                                   int32_t* __restrict__ info,
                                                   int32_t* __restrict__ iters) {
  extern __shared__ double x[];
  __shared__ int s_piv;
  const int b = bt.order[blockIdx.x];
  const int n = airfoil_n(bt, b);
  const int m = n + 1;
  if (info[b] != 0) return;
  if (n > bt.n_max) {
    if (threadIdx.x == 0) info[b] = PANEL_INFO_TOO_LARGE;
    return;
  }
  const double* Ab = A + bt.mat_off[b];
  double* F = LU + bt.mat_off[b];
  int32_t* pv = piv + vec_off(bt, b);
  const int64_t mm = (int64_t)m * m;
  for (int64_t e = threadIdx.x; e < mm; e += blockDim.x) F[e] = Ab[e];
  __syncthreads();
  int st = lu_factor_f64(F, pv, m, &s_piv);
  if (st != 0) {
    if (threadIdx.x == 0) { info[b] = st; if (iters) iters[b] = 0; }
    return;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < m; k += blockDim.x) x[k] = rhs[vec_off(bt, b) + k];
  __syncthreads();
  lu_solve_f64(F, pv, m, x);
  for (int k = threadIdx.x; k < m; k += blockDim.x) u[vec_off(bt, b) + k] = x[k];
  if (threadIdx.x == 0 && iters) iters[b] = 0;
  if (lambda) {
    __syncthreads();
    cl_sensitivity_f64(bt.nodes + 2 * bt.node_off[b], n, vinf ? vinf[b] : 1.0,
                       chord ? chord[b] : 1.0, x);
    lu_solve_transposed_f64(F, pv, m, x);
    for (int k = threadIdx.x; k < m; k += blockDim.x) lambda[vec_off(bt, b) + k] = x[k];
  }
}

cudaError_t launch_solve_f64(const Batch& bt, const double* A, double* LU, int32_t* piv,
                             const double* rhs, const double* vinf, const double* chord, double* u,
                             double* lambda, int32_t* info, int32_t* iters, cudaStream_t s) {
  size_t smem = (size_t)(bt.n_max + 1) * sizeof(double);
  k_solve_f64<<<bt.B, 256, smem, s>>>(bt, A, LU, piv, rhs, vinf, chord, u, lambda, info, iters);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Adjoint contraction (plain FP64)
// ---------------------------------------------------------------------------
//
// With G(p; a, b) = (1/2pi) int_a^b log|p - s| ds, M_ji = -G(x_{j+1/2}; x_i, x_{i+1}),
// in the frame t = (b-a)/L, n = t rotated by +90 degrees, xi = (p-a).t,
// eta = (p-a).n, l1 = log|p-a|^2, l2 = log|p-b|^2, theta the subtended angle:
//   2pi dG/dp = (l1 - l2)/2 t + theta n
//   2pi dG/db = l2/2 t + ((l1 - l2)/2 eta - theta xi)/L n
//   dG/da     = -dG/dp - dG/db            (translation invariance)
// and dCl/dx_k = dCl/dx_k|_u + lambda^T (db/dx_k - (dM/dx_k) u) becomes
//   (2/(v c)) (gamma_{k-1} t_{k-1} - gamma_k t_k)
//   + v/2 (-sin a, cos a) (lambda_{k-1} + lambda_k)
//   + 1/2 (lambda_{k-1} P_{k-1} + lambda_k P_k) + u_k Acol_k + u_{k-1} Bcol_{k-1}
// with P_j = sum_i u_i dG_ji/dp, Acol_i = sum_j lambda_j dG_ji/da,
// Bcol_i = sum_j lambda_j dG_ji/db (indices mod n).  On the own panel (i = j)
// theta is ambiguous (+-pi); it cancels between the terms, so it is set to 0.
__global__ void __launch_bounds__(256) k_adjoint_f64(
    Batch bt, const double* __restrict__ LU, const int32_t* __restrict__ piv,
    const double* __restrict__ u, const double* __restrict__ lambda_in,
    double* __restrict__ lambda_out, const double* __restrict__ alpha,
    const double* __restrict__ vinf, const double* __restrict__ chord,
    const double* __restrict__ grad_cl, double* __restrict__ grad,
    const int32_t* __restrict__ info) {
  extern __shared__ double sm[];
  const int b = bt.order[blockIdx.x];
  const int n = airfoil_n(bt, b);
  const int m = n + 1;
  const int nm = bt.n_max;
  double* gout = grad + 2 * bt.node_off[b];
  if ((info && info[b] != 0) || n > nm || n < 3) {
    for (int k = threadIdx.x; k < 2 * n; k += blockDim.x) gout[k] = nan("");
    return;
  }
  double* xs = sm;
  double* ys = xs + nm;
  double* txs = ys + nm;
  double* tys = txs + nm;
  double* Ls = tys + nm;
  double* lam = Ls + nm;      // m
  double* uu = lam + nm + 1;  // m
  double* P = uu + nm + 1;    // 2n
  double* Ac = P + 2 * nm;    // 2n
  double* Bc = Ac + 2 * nm;   // 2n
  const double* nodes = bt.nodes + 2 * bt.node_off[b];
  const double v = vinf ? vinf[b] : 1.0, c = chord ? chord[b] : 1.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    xs[k] = nodes[2 * k];
    ys[k] = nodes[2 * k + 1];
  }
  for (int k = threadIdx.x; k < m; k += blockDim.x) uu[k] = u[vec_off(bt, b) + k];
  for (int k = threadIdx.x; k < 2 * n; k += blockDim.x) P[k] = 0.0;
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    int k1 = (k + 1 == n) ? 0 : k + 1;
    double hx = xs[k1] - xs[k], hy = ys[k1] - ys[k];
    double L = sqrt(hx * hx + hy * hy);
    txs[k] = hx / L;
    tys[k] = hy / L;
    Ls[k] = L;
  }
  if (lambda_in) {
    for (int k = threadIdx.x; k < m; k += blockDim.x) lam[k] = lambda_in[vec_off(bt, b) + k];
    __syncthreads();
  } else {
    cl_sensitivity_f64(nodes, n, v, c, lam);
    lu_solve_transposed_f64(LU + bt.mat_off[b], piv + vec_off(bt, b), m, lam);
    for (int k = threadIdx.x; k < m; k += blockDim.x) lambda_out[vec_off(bt, b) + k] = lam[k];
  }
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int ncb = (n + 31) >> 5;
  for (int cb = warp; cb < ncb; cb += nw) {
    const int i = cb * 32 + lane;
    const bool ok = i < n;
    const int ii = ok ? i : 0;
    const double ax = xs[ii], ay = ys[ii], tx = txs[ii], ty = tys[ii], L = Ls[ii];
    const double ui = ok ? uu[ii] : 0.0;
    double sAx = 0, sAy = 0, sBx = 0, sBy = 0;
    for (int j = 0; j < n; ++j) {
      const int j1 = (j + 1 == n) ? 0 : j + 1;
      const double px = 0.5 * (xs[j] + xs[j1]), py = 0.5 * (ys[j] + ys[j1]);
      double dx = px - ax, dy = py - ay;
      double xi = dx * tx + dy * ty;
      double eta = dy * tx - dx * ty;
      double xl = xi - L;
      double l1 = log(xi * xi + eta * eta);
      double l2 = log(xl * xl + eta * eta);
      double th = (i == j) ? 0.0 : atan2(eta * L, xi * xl + eta * eta);
      double hd = 0.5 * (l1 - l2);
      // dG/dp and dG/db (without the 1/2pi), in global coordinates
      double gpx = hd * tx - th * ty, gpy = hd * ty + th * tx;
      double cn = (hd * eta - th * xi) / L;
      double gbx = 0.5 * l2 * tx - cn * ty, gby = 0.5 * l2 * ty + cn * tx;
      const double lj = lam[j];
      sAx += lj * (-gpx - gbx);
      sAy += lj * (-gpy - gby);
      sBx += lj * gbx;
      sBy += lj * gby;
      double rx = warp_sum(ok ? ui * gpx : 0.0);
      double ry = warp_sum(ok ? ui * gpy : 0.0);
      if (lane == 0) {
        atomicAdd(&P[2 * j], rx);
        atomicAdd(&P[2 * j + 1], ry);
      }
    }
    if (ok) {
      Ac[2 * i] = sAx;
      Ac[2 * i + 1] = sAy;
      Bc[2 * i] = sBx;
      Bc[2 * i + 1] = sBy;
    }
  }
  __syncthreads();
  const double ca = cos(alpha[b]), sa = sin(alpha[b]);
  const double gscale = grad_cl ? grad_cl[b] : 1.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const int km = (k == 0) ? n - 1 : k - 1;
    double gx = 2.0 / (v * c) * (uu[km] * txs[km] - uu[k] * txs[k]);
    double gy = 2.0 / (v * c) * (uu[km] * tys[km] - uu[k] * tys[k]);
    gx += 0.5 * v * (-sa) * (lam[km] + lam[k]);
    gy += 0.5 * v * ca * (lam[km] + lam[k]);
    gx += kInvTwoPi * (0.5 * (lam[km] * P[2 * km] + lam[k] * P[2 * k]) + uu[k] * Ac[2 * k] +
                       uu[km] * Bc[2 * km]);
    gy += kInvTwoPi * (0.5 * (lam[km] * P[2 * km + 1] + lam[k] * P[2 * k + 1]) +
                       uu[k] * Ac[2 * k + 1] + uu[km] * Bc[2 * km + 1]);
    gout[2 * k] = gscale * gx;
    gout[2 * k + 1] = gscale * gy;
  }
}

size_t adjoint_f64_smem(int n_max) { return (size_t)(13 * n_max + 2) * sizeof(double); }

cudaError_t launch_adjoint_f64(const Batch& bt, const double* LU, const int32_t* piv,
                               const double* u, const double* lambda_in, double* lambda_out,
                               const double* alpha, const double* vinf, const double* chord,
                               const double* grad_cl, double* grad, const int32_t* info,
                               cudaStream_t s) {
  size_t smem = adjoint_f64_smem(bt.n_max);
  cudaError_t e = ensure_smem(k_adjoint_f64, smem);
  if (e != cudaSuccess) return e;
  k_adjoint_f64<<<bt.B, 256, smem, s>>>(bt, LU, piv, u, lambda_in, lambda_out, alpha, vinf, chord,
                                        grad_cl, grad, info);
  return cudaGetLastError();
}

}  // namespace panel
