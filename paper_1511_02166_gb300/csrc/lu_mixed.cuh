// lu_mixed.cuh -- declarations shared by the FP32 factorisations of the
// mixed-precision path (k_solve_mixed.cu: one block per airfoil; k_lu_large.cu:
// the step-synchronous blocked factor of large airfoils) and the refinement.
#pragma once
#include "panel_common.cuh"

namespace panel {

constexpr int kSmemM = 230;  // largest m = n + 1 factored in shared memory
constexpr int kGjM = 288;    // m up to this: Gauss-Jordan inverse (k_gj_mixed.cu)
constexpr int kLargeM = 640; // m above this takes the step-synchronous blocked factor
constexpr int kNB = 32;      // panel width
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

struct SolveArgs {
  Batch bt;
  const float* A_hi;
  const float* A_lo;
  float* LU;
  int32_t* piv;
  const double* rhs;
  const double* vinf;
  const double* chord;
  double* u;         // forward solution (may be NULL: no forward system)
  double* lam;       // transposed solution (may be NULL: no transposed system)
  int max_iter;
  double tol;
  int32_t* info;
  int32_t* iters;
  int inverse;       // m <= kGjM: Gauss-Jordan inverse (k_gj_mixed.cu) instead of the LU
  int n_cap;         // the caller's n_max (bt.n_max may be lowered to size a kernel)
  int rhs_kind;      // forward right-hand side: 0 rhs, 1 v m_y, 2 -v m_x (polar basis)
  int ir_shape;      // refinement block shape: 0 by size, 1..4 = 128x8, 256x4, 512x2, 1024x1
  // Transposed right-hand side of a vector-Jacobian product (vjp != 0):
  // w_cl[b] dCl/du + w_u + w_cp dCp/du (each may be NULL = 0), with the
  // strengths u_in of the forward solution; vjp == 0 is dCl/du alone.
  int vjp;
  const double* w_cl;
  const double* w_u;   // [sum m_b], packed like u (gamma, C)
  const double* w_cp;  // [sum n_b], packed like the nodes
  const double* u_in;  // [sum m_b]
};

__device__ __forceinline__ double block_absmax_d(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = 0.0;
  const int nw = blockDim.x >> 5;
  for (int w = 0; w < nw; ++w) r = fmax(r, red[w]);
  __syncthreads();
  return r;
}

// border scale s = mean |A_jj| over the influence block (hi plane)
__device__ __forceinline__ double border_scale(const float* Ah, int n, int m, double* red) {
  double sdiag = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) sdiag += fabs((double)Ah[j * m + j]);
  return block_sum(sdiag, red) / n;
}

// ---------------------------------------------------------------------------
// Inverted diagonal blocks, in place, one warp per 32 x 32 block (lane j =
// column j of the inverse).  X = L_dd^{-1} (unit lower) replaces the part
// below the diagonal row by row (row i is written after every lane has read
// it); Y = U_dd^{-1} (upper) replaces the rest row by row from the bottom.
// invert_block takes one kb x kb block (kb <= 32) at B with row stride ld,
// called by all lanes of one warp.
// ---------------------------------------------------------------------------
__device__ inline void invert_block(float* B, int ld, int kb) {
  const int j = threadIdx.x & 31;
  // X[i][j] = -(L[i][j] + sum_{j<k<i} L[i][k] X[k][j]),  i > j
  for (int i = 1; i < kb; ++i) {
    float x = 0.0f;
    if (j < i) {
      x = -B[i * ld + j];
      for (int k = j + 1; k < i; ++k) x = fmaf(-B[i * ld + k], B[k * ld + j], x);
    }
    __syncwarp();
    if (j < i) B[i * ld + j] = x;
    __syncwarp();
  }
  // Y[i][j] = -(sum_{i<k<=j} U[i][k] Y[k][j]) / U[i][i] (i < j), Y[j][j] = 1/U[j][j]
  for (int i = kb - 1; i >= 0; --i) {
    float y = 0.0f;
    const float uii = B[i * ld + i];
    if (j == i) {
      y = 1.0f / uii;
    } else if (j > i && j < kb) {
      float acc = 0.0f;
      for (int k = i + 1; k <= j; ++k) acc = fmaf(B[i * ld + k], B[k * ld + j], acc);
      y = -acc / uii;
    }
    __syncwarp();
    if (j >= i && j < kb) B[i * ld + j] = y;
    __syncwarp();
  }
}

__device__ inline void invert_diagonal_blocks(float* F, int ld, int m) {
  const int warp = threadIdx.x >> 5;
  const int nb = (m + 31) >> 5;
  for (int d = warp; d < nb; d += kWarps) {
    const int k0 = 32 * d;
    invert_block(F + k0 * ld + k0, ld, min(32, m - k0));
  }
}

cudaError_t launch_lu_large(const SolveArgs& a, cudaStream_t s);
cudaError_t launch_gj_mixed(const SolveArgs& a, cudaStream_t s);
long long set_wait_limit(long long polls);
size_t lu_large_min_m();

}  // namespace panel
