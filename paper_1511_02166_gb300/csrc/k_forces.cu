// k_forces.cu -- Cp and lift from the panel strengths, FP64 warp reductions.
//
// The paper reports C_L (Section 2, Figure 2) without writing the formula;
// with the printed system the unknown gamma_j is the surface speed at the
// control point (the sheet jump, zero flow inside the body), so
//   Cp_j = 1 - (gamma_j / v_inf)^2,   Cl = 2 sum_i gamma_i |h_i| / (v_inf c)
// (Kutta-Joukowski with circulation sum gamma_i |h_i|), and, as a check,
// the pressure force F = -sum_j Cp_j n_j |h_j| with outward n_j = (h_y, -h_x)/|h_j|:
//   Cl_p = (-F_x sin a + F_y cos a) / c,  Cd_p = (F_x cos a + F_y sin a) / c.
#include "panel_common.cuh"

namespace panel {

// One warp per airfoil.
__global__ void __launch_bounds__(256) k_forces(Batch bt, const double* __restrict__ u,
                                                const double* __restrict__ alpha,
                                                const double* __restrict__ vinf,
                                                const double* __restrict__ chord,
                                                const int32_t* __restrict__ info,
                                                double* __restrict__ cp, double* __restrict__ cl,
                                                double* __restrict__ cl_p,
                                                double* __restrict__ cd_p) {
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= bt.B) return;
  const int b = w;
  const int n = airfoil_n(bt, b);
  const double* x = bt.nodes + 2 * bt.node_off[b];
  const double* g = u + vec_off(bt, b);
  double* cpb = cp + bt.node_off[b];
  if ((info && info[b] != 0) || n < 3) {
    for (int j = lane; j < n; j += 32) cpb[j] = nan("");
    if (lane == 0) {
      cl[b] = nan("");
      if (cl_p) cl_p[b] = nan("");
      if (cd_p) cd_p[b] = nan("");
    }
    return;
  }
  const double v = vinf ? vinf[b] : 1.0, c = chord ? chord[b] : 1.0;
  double circ = 0.0, fx = 0.0, fy = 0.0;
  for (int j = lane; j < n; j += 32) {
    const int j1 = (j + 1 == n) ? 0 : j + 1;
    const double hx = x[2 * j1] - x[2 * j], hy = x[2 * j1 + 1] - x[2 * j + 1];
    const double L = sqrt(hx * hx + hy * hy);
    const double gj = g[j];
    const double q = gj / v;
    const double cpj = 1.0 - q * q;
    cpb[j] = cpj;
    circ = fma(gj, L, circ);
    fx = fma(-cpj, hy, fx);
    fy = fma(cpj, hx, fy);
  }
  circ = warp_sum(circ);
  fx = warp_sum(fx);
  fy = warp_sum(fy);
  if (lane == 0) {
    const double a = alpha[b];
    cl[b] = 2.0 * circ / (v * c);
    if (cl_p) cl_p[b] = (-fx * sin(a) + fy * cos(a)) / c;
    if (cd_p) cd_p[b] = (fx * cos(a) + fy * sin(a)) / c;
  }
}

cudaError_t launch_forces(const Batch& bt, const double* u, const double* alpha,
                          const double* vinf, const double* chord, const int32_t* info,
                          double* cp, double* cl, double* cl_p, double* cd_p, cudaStream_t s) {
  const int wpb = 8;
  const int grid = (bt.B + wpb - 1) / wpb;
  k_forces<<<grid, wpb * 32, 0, s>>>(bt, u, alpha, vinf, chord, info, cp, cl, cl_p, cd_p);
  return cudaGetLastError();
}

// Polar: with the basis solutions u_y (right-hand side v m_y) and u_x (-v m_x)
// of the same factored system, u(alpha) = cos(alpha) u_y + sin(alpha) u_x by
// linearity, so Cl(alpha) = cos(alpha) Cl_y + sin(alpha) Cl_x.  One warp per
// airfoil of this call (size order); cl is [B][K] by airfoil index.
__global__ void __launch_bounds__(256) k_polar_cl(Batch bt, const double* __restrict__ uy,
                                                  const double* __restrict__ ux,
                                                  const double* __restrict__ vinf,
                                                  const double* __restrict__ chord, int K,
                                                  const double* __restrict__ alphas,
                                                  const int32_t* __restrict__ info,
                                                  double* __restrict__ cl) {
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= bt.B) return;
  const int b = bt.order[w];
  const int n = airfoil_n(bt, b);
  double* out = cl + (int64_t)b * K;
  if ((info && info[b] != 0) || n < 3 || n > bt.n_max) {
    for (int k = lane; k < K; k += 32) out[k] = nan("");
    return;
  }
  const double* x = bt.nodes + 2 * bt.node_off[b];
  const double* gy = uy + vec_off(bt, b);
  const double* gx = ux + vec_off(bt, b);
  double cy = 0.0, cx = 0.0;
  for (int j = lane; j < n; j += 32) {
    const int j1 = (j + 1 == n) ? 0 : j + 1;
    const double hx = x[2 * j1] - x[2 * j], hy = x[2 * j1 + 1] - x[2 * j + 1];
    const double L = sqrt(hx * hx + hy * hy);
    cy = fma(gy[j], L, cy);
    cx = fma(gx[j], L, cx);
  }
  cy = warp_sum(cy);
  cx = warp_sum(cx);
  const double v = vinf ? vinf[b] : 1.0, c = chord ? chord[b] : 1.0;
  const double f = 2.0 / (v * c);
  for (int k = lane; k < K; k += 32) {
    const double al = alphas[(int64_t)b * K + k];
    out[k] = f * (cos(al) * cy + sin(al) * cx);
  }
}

cudaError_t launch_polar_cl(const Batch& bt, const double* uy, const double* ux,
                            const double* vinf, const double* chord, int K, const double* alphas,
                            const int32_t* info, double* cl, cudaStream_t s) {
  const int wpb = 8;
  const int grid = (bt.B + wpb - 1) / wpb;
  k_polar_cl<<<grid, wpb * 32, 0, s>>>(bt, uy, ux, vinf, chord, K, alphas, info, cl);
  return cudaGetLastError();
}

}  // namespace panel
