// k_assemble_f64.cu -- plain FP64 assembly of the bordered panel system.
//
// Section 2 of the paper: A_ji = -F_i(x_{j+1/2}) / gamma_i with the closed-form
// panel integral, the C column of ones, the Kutta row gamma_0 + gamma_{n-1} = 0
// and b_j = v_inf (y_{j+1/2} cos a - x_{j+1/2} sin a).  The printed integral
// uses two log and two atan2 per pair; here the two atan2 of one pair are
// combined into one (their difference is the angle the panel subtends, always
// inside (-pi, pi)), which leaves two log and one atan2 in native FP64.
#include "panel_common.cuh"

namespace panel {

// (1/2pi) * integral over the panel a->b of log|p - s| ds, in the panel frame
// xi = (p-a).t, eta = (p-a).n (n = t rotated by +90 degrees), L = |b-a|:
//   G = (1/2pi) [ xi/2 log r1^2 - (xi-L)/2 log r2^2 + eta*theta - L ],
//   theta = atan2(eta L, xi (xi - L) + eta^2).
__device__ __forceinline__ double panel_G_f64(double px, double py, double ax, double ay,
                                              double tx, double ty, double L) {
  double dx = px - ax, dy = py - ay;
  double xi = dx * tx + dy * ty;
  double eta = dy * tx - dx * ty;
  double xl = xi - L;
  double r1 = xi * xi + eta * eta;
  double r2 = xl * xl + eta * eta;
  double th = atan2(eta * L, xi * xl + eta * eta);
  return kInvTwoPi * (0.5 * xi * log(r1) - 0.5 * xl * log(r2) + eta * th - L);
}

__global__ void __launch_bounds__(256) k_assemble_f64(Batch bt, const double* __restrict__ alpha,
                                                      const double* __restrict__ vinf,
                                                      double* __restrict__ A,
                                                      double* __restrict__ rhs,
                                                      int32_t* __restrict__ info) {
  extern __shared__ double sm[];
  const int b = bt.order[blockIdx.x];
  const int n = airfoil_n(bt, b);
  const int m = n + 1;
  double* xs = sm;                 // nodes
  double* ys = xs + bt.n_max;
  double* txs = ys + bt.n_max;     // unit tangents of the panels
  double* tys = txs + bt.n_max;
  double* Ls = tys + bt.n_max;     // panel lengths
  double* mxs = Ls + bt.n_max;     // control points
  double* mys = mxs + bt.n_max;
  double* scratch = mys + bt.n_max;

  const double* nodes = bt.nodes + 2 * bt.node_off[b];
  if (n > bt.n_max) {
    if (threadIdx.x == 0) info[b] = PANEL_INFO_TOO_LARGE;
    return;
  }
  int st = load_and_check_geometry(nodes, n, xs, ys, scratch);
  if (threadIdx.x == 0) info[b] = st;
  if (st != 0) return;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    int k1 = (k + 1 == n) ? 0 : k + 1;
    double hx = xs[k1] - xs[k], hy = ys[k1] - ys[k];
    double L = sqrt(hx * hx + hy * hy);
    txs[k] = hx / L;
    tys[k] = hy / L;
    Ls[k] = L;
    mxs[k] = 0.5 * (xs[k] + xs[k1]);
    mys[k] = 0.5 * (ys[k] + ys[k1]);
  }
  __syncthreads();

  const double v = vinf ? vinf[b] : 1.0;
  const double ca = cos(alpha[b]), sa = sin(alpha[b]);
  double* Ab = A + bt.mat_off[b];
  double* rb = rhs + vec_off(bt, b);
  for (int j = threadIdx.x; j < m; j += blockDim.x)
    rb[j] = (j < n) ? v * (mys[j] * ca - mxs[j] * sa) : 0.0;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = warp; j < m; j += nw) {
    double* row = Ab + (int64_t)j * m;
    if (j < n) {
      const double px = mxs[j], py = mys[j];
      for (int i = lane; i < n; i += 32)
        row[i] = -panel_G_f64(px, py, xs[i], ys[i], txs[i], tys[i], Ls[i]);
      if (lane == 0) row[n] = 1.0;
    } else {
      for (int i = lane; i < m; i += 32) row[i] = (i == 0 || i == n - 1) ? 1.0 : 0.0;
    }
  }
}

size_t assemble_f64_smem(int n_max) { return (size_t)(7 * n_max + 32) * sizeof(double); }

cudaError_t launch_assemble_f64(const Batch& bt, const double* alpha, const double* vinf,
                                double* A, double* rhs, int32_t* info, cudaStream_t s) {
  size_t smem = assemble_f64_smem(bt.n_max);
  cudaError_t e = ensure_smem(k_assemble_f64, smem);
  if (e != cudaSuccess) return e;
  k_assemble_f64<<<bt.B, 256, smem, s>>>(bt, alpha, vinf, A, rhs, info);
  return cudaGetLastError();
}

}  // namespace panel
