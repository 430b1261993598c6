// lu_mixed.cuh -- declarations shared by the FP32 factorisations of the
// mixed-precision path (k_solve_mixed.cu: one block per airfoil; k_lu_large.cu:
// the step-synchronous blocked factor of large airfoils) and the refinement.
#pragma once
#include "panel_common.cuh"

namespace panel {

constexpr int kSmemM = 230;  // largest m = n + 1 of a Gauss-Jordan inverse in shared memory
constexpr int kGjM = 288;    // m up to this: Gauss-Jordan inverse (k_gj_mixed.cu)
constexpr int kLargeM = 640; // m above this takes the step-synchronous blocked factor
constexpr int kSmemLuM = 224; // m up to this: LU with the whole matrix in shared memory
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
  int lu_kind;       // LU of m <= kSmemLuM: 0/2 whole matrix in shared memory, 1 through L2
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
// Inverted diagonal blocks, in place: X = L_dd^{-1} (unit lower) replaces the
// part below the diagonal, Y = U_dd^{-1} (upper) the rest.  Each is one warp's
// work, lane j computing column j of the inverse in registers by substitution
// against the unit vector e_j, right-looking: once entry k of the column is
// final, it is multiplied into every later entry (L: rows below k, U: rows
// above k) at once, so each step is 31 independent FMAs on broadcast loads
// instead of a dependent dot product.  The two parts read and write disjoint
// entries (strictly below / on and above the diagonal): two warps may do them
// at the same time.  Every index into the register column is a compile-time
// constant (fully unrolled loops); kb <= 32 is the block size, B its first
// element, ld the row stride, all lanes of the warp call.
// ---------------------------------------------------------------------------
__device__ inline void invert_lower_unit(float* B, int ld, int kb) {
  const int j = threadIdx.x & 31;
  float acc[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) acc[i] = (i == j) ? 1.0f : 0.0f;
#pragma unroll
  for (int k = 0; k < 31; ++k) {
    if (k < kb) {
      const float xk = acc[k];  // X[k][j], final
#pragma unroll
      for (int i = k + 1; i < 32; ++i)
        if (i < kb) acc[i] = fmaf(-B[i * ld + k], xk, acc[i]);
    }
  }
  __syncwarp();
#pragma unroll
  for (int i = 1; i < 32; ++i)
    if (i < kb && j < i) B[i * ld + j] = acc[i];
  __syncwarp();
}

__device__ inline void invert_upper(float* B, int ld, int kb) {
  const int j = threadIdx.x & 31;
  float acc[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) acc[i] = (i == j) ? 1.0f : 0.0f;
#pragma unroll
  for (int k = 31; k >= 0; --k) {
    if (k < kb) {
      const float yk = acc[k] / B[k * ld + k];  // Y[k][j], final
      acc[k] = yk;
#pragma unroll
      for (int i = 0; i < k; ++i) acc[i] = fmaf(-B[i * ld + k], yk, acc[i]);
    }
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < 32; ++i)
    if (i < kb && j >= i && j < kb) B[i * ld + j] = acc[i];
  __syncwarp();
}

__device__ inline void invert_block(float* B, int ld, int kb) {
  invert_lower_unit(B, ld, kb);
  invert_upper(B, ld, kb);
}

cudaError_t launch_lu_large(const SolveArgs& a, cudaStream_t s);
cudaError_t launch_gj_mixed(const SolveArgs& a, cudaStream_t s);
long long set_wait_limit(long long polls);
size_t lu_large_min_m();

}  // namespace panel
