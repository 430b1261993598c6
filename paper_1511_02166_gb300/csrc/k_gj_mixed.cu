// k_gj_mixed.cu -- FP32 inverse of the bordered system for airfoils with
// m = n + 1 <= kGjM (mixed-precision path): blocked Gauss-Jordan elimination in
// place, one block of 256 threads per airfoil, the matrix in shared memory
// (m <= kSmemM) or in the caller's LU buffer (through L2).  Used with
// PANEL_INVERSE only; by default the LU of k_solve_mixed.cu takes every size.
//
// For each block column K = [k0, k0 + 32) of the rescaled matrix A:
//   1. warp 0 inverts the diagonal block D = A[K][K] in place by Gauss-Jordan
//      with partial pivoting over the rows of K (exchanges inside K only);
//   2. row block:     A[K][j]  <- D'^{-1} (P_K A)[K][j]        (j outside K)
//   3. the rest:      A[i][j]  <- A[i][j] - A[i][K] A[K][j]    (i, j outside K)
//   4. column block:  A[i][K]  <- -A[i][K] D'^{-1}             (i outside K)
//   5. A[K][K] <- D'^{-1}
// with D' = P_K D.  Exchanging rows of K before K is eliminated is the same as
// exchanging them in the original matrix, so the result is X = (P A)^{-1} with
// P the product of all exchanges (stored as sequential exchanges in piv, like
// an LU's, but as -(row + 1): the sign tells the refinement which layout the
// factor buffer holds), and A^{-1} = X P.  The refinement then applies X with one
// matrix-vector product per correction (forward) or one with X^T (transposed)
// instead of two triangular sweeps of m/32 dependent steps.
//
// Pivoting only inside the 32-row diagonal blocks: for the logarithmic
// single-layer collocation matrices of Section 2 (bordered by the Kutta row and
// the C column) partial pivoting over whole columns exchanges almost nothing,
// and the refinement with the double-float residual converges in as few steps
// from this inverse as from a partially pivoted LU.  An exactly zero pivot
// sets info[b] = its index + 1.
#include "lu_mixed.cuh"

namespace panel {

constexpr int kGB = 32;   // block width
constexpr int kLdB = 36;  // row stride of the block copies (16-byte rows)

struct GjShared {
  float Dv[kGB * kLdB];  // the diagonal block, inverted in place
  float Dt[kGB * kLdB];  // its transpose
  int sp[kGB];           // the block's exchanges, sequential
  int pk[kGB];           // their composition: row t of P_K D is row pk[t] of D
  int flag;              // 0, or q + 1 for an exactly zero pivot at block column q
  double red[32];
};

// Warp 0: Gauss-Jordan with partial pivoting on the kb x kb block Dv (zero
// padded to 32 x 32); lane = column.  Returns 0 or q + 1 (uniform).
__device__ int gj_block(GjShared& sh, int kb, int lane) {
  float* Dv = sh.Dv;
  for (int q = 0; q < kb; ++q) {
    const float v = (lane >= q && lane < kb) ? fabsf(Dv[lane * kLdB + q]) : -1.0f;
    // |x| bit patterns are monotone; +1 so that 0 means "no candidate" (and NaN)
    const unsigned key = (v >= 0.0f) ? __float_as_uint(v) + 1u : 0u;
    const unsigned mx = __reduce_max_sync(0xffffffffu, key);
    if (mx <= 1u) return q + 1;
    const int p = __ffs(__ballot_sync(0xffffffffu, key == mx)) - 1;  // lowest row on ties
    if (lane == 0) sh.sp[q] = p;
    if (p != q) {
      const float t = Dv[q * kLdB + lane];
      Dv[q * kLdB + lane] = Dv[p * kLdB + lane];
      Dv[p * kLdB + lane] = t;
    }
    __syncwarp();
    const float inv = 1.0f / Dv[q * kLdB + q];
    const float rq = (lane == q) ? inv : Dv[q * kLdB + lane] * inv;
    for (int r = 0; r < kb; ++r) {
      if (r == q) continue;
      const float f = Dv[r * kLdB + q];
      __syncwarp();
      Dv[r * kLdB + lane] = (lane == q) ? -f * inv : fmaf(-f, rq, Dv[r * kLdB + lane]);
    }
    __syncwarp();
    Dv[q * kLdB + lane] = rq;
    __syncwarp();
  }
  if (lane == 0) {
    for (int t = 0; t < kGB; ++t) sh.pk[t] = t;
    for (int q = 0; q < kb; ++q) {
      const int p = sh.sp[q];
      const int t = sh.pk[q];
      sh.pk[q] = sh.pk[p];
      sh.pk[p] = t;
    }
  }
  for (int r = 0; r < kGB; ++r) sh.Dt[lane * kLdB + r] = Dv[r * kLdB + lane];
  __syncwarp();
  return 0;
}

// A[i][j] -= A[i][K] A[K][j] for i, j outside K: warp tiles of 8 rows x 128
// columns (4 per lane), indices mapped around the block K.
__device__ __forceinline__ void gj_update(float* A, int ld, int m, int k0, int kb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int mo = m - kb;  // rows / columns outside K
  const int nr = (mo + 7) >> 3, nc = (mo + 127) >> 7;
  for (int tile = warp; tile < nr * nc; tile += kWarps) {
    const int rr0 = 8 * (tile / nc);
    const int cc0 = 128 * (tile % nc) + lane;
    int ri[8], cj[4];
    bool rok[8], cok[4];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int rr = rr0 + a;
      rok[a] = rr < mo;
      ri[a] = rok[a] ? ((rr < k0) ? rr : rr + kb) : 0;
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int cc = cc0 + 32 * t;
      cok[t] = cc < mo;
      cj[t] = cok[t] ? ((cc < k0) ? cc : cc + kb) : 0;
    }
    // the rank-kb product is summed on its own and subtracted once: entries of
    // A can be much larger than the update, and 32 roundings at |A| would cost
    // the inverse several times its attainable accuracy
    float acc[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int t = 0; t < 4; ++t) acc[a][t] = 0.0f;
#pragma unroll 2
    for (int q = 0; q < kb; ++q) {
      float lv[8], uv[4];
#pragma unroll
      for (int a = 0; a < 8; ++a) lv[a] = A[ri[a] * ld + k0 + q];
#pragma unroll
      for (int t = 0; t < 4; ++t) uv[t] = A[(k0 + q) * ld + cj[t]];
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int t = 0; t < 4; ++t) acc[a][t] = fmaf(lv[a], uv[t], acc[a][t]);
    }
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (rok[a] && cok[t]) A[ri[a] * ld + cj[t]] -= acc[a][t];
  }
}

template <bool SMEM>
__global__ void __launch_bounds__(kThreads, SMEM ? 1 : 2) k_gj_mixed(SolveArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ GjShared sh;
  const Batch& bt = a.bt;
  const int b = bt.order[blockIdx.x];
  const int n = airfoil_n(bt, b);
  const int m = n + 1;
  if (a.info[b] != 0) return;
  if (!a.inverse || m > (SMEM ? kSmemM : kGjM) || (!SMEM && m <= kSmemM)) return;
  if (n > a.n_cap) {
    if (threadIdx.x == 0) a.info[b] = PANEL_INFO_TOO_LARGE;
    return;
  }
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t moff = bt.mat_off[b];
  const float* Ah = a.A_hi + moff;
  float* G = a.LU + moff;
  const int ld = SMEM ? (m | 1) : m;
  float* A = SMEM ? reinterpret_cast<float*>(smraw) : G;
  const float sf = (float)border_scale(Ah, n, m, sh.red);
  for (int r = warp; r < m; r += kWarps)
    for (int c = lane; c < m; c += 32) {
      const float v = Ah[r * m + c];
      A[r * ld + c] = ((c == n && r < n) || r == n) ? v * sf : v;
    }
  int32_t* gpiv = a.piv + vec_off(bt, b);
  for (int k0 = 0; k0 < m; k0 += kGB) {
    const int kb = min(kGB, m - k0);
    __syncthreads();
    for (int e = tid; e < kGB * kGB; e += kThreads) {
      const int r = e >> 5, c = e & 31;
      sh.Dv[r * kLdB + c] = (r < kb && c < kb) ? A[(k0 + r) * ld + k0 + c] : 0.0f;
    }
    __syncthreads();
    if (warp == 0) {
      const int f = gj_block(sh, kb, lane);
      if (lane == 0) sh.flag = f;
    }
    __syncthreads();
    if (sh.flag) {
      if (tid == 0) {
        a.info[b] = k0 + sh.flag;
        if (a.iters) a.iters[b] = 0;
      }
      return;
    }
    // the exchanges, tagged as belonging to an inverse: -(row + 1)
    if (tid < kb) gpiv[k0 + tid] = -(k0 + sh.sp[tid]) - 1;
    // row block: a thread per column j outside K
    for (int jj = tid; jj < m - kb; jj += kThreads) {
      const int j = (jj < k0) ? jj : jj + kb;
      float col[kGB];
#pragma unroll
      for (int q = 0; q < kGB; ++q) col[q] = (q < kb) ? A[(k0 + sh.pk[q]) * ld + j] : 0.0f;
#pragma unroll 4
      for (int t = 0; t < kGB; ++t) {
        const float4* dr = reinterpret_cast<const float4*>(sh.Dv + t * kLdB);
        float acc = 0.0f;
#pragma unroll
        for (int q4 = 0; q4 < kGB / 4; ++q4) {
          const float4 d = dr[q4];
          acc = fmaf(d.x, col[4 * q4], acc);
          acc = fmaf(d.y, col[4 * q4 + 1], acc);
          acc = fmaf(d.z, col[4 * q4 + 2], acc);
          acc = fmaf(d.w, col[4 * q4 + 3], acc);
        }
        if (t < kb) A[(k0 + t) * ld + j] = acc;
      }
    }
    __syncthreads();
    gj_update(A, ld, m, k0, kb);
    __syncthreads();
    // column block: a thread per row i outside K; then the block itself
    for (int ii = tid; ii < m - kb; ii += kThreads) {
      const int i = (ii < k0) ? ii : ii + kb;
      float row[kGB];
#pragma unroll
      for (int q = 0; q < kGB; ++q) row[q] = (q < kb) ? A[i * ld + k0 + q] : 0.0f;
#pragma unroll 4
      for (int t = 0; t < kGB; ++t) {
        const float4* dc = reinterpret_cast<const float4*>(sh.Dt + t * kLdB);
        float acc = 0.0f;
#pragma unroll
        for (int q4 = 0; q4 < kGB / 4; ++q4) {
          const float4 d = dc[q4];
          acc = fmaf(d.x, row[4 * q4], acc);
          acc = fmaf(d.y, row[4 * q4 + 1], acc);
          acc = fmaf(d.z, row[4 * q4 + 2], acc);
          acc = fmaf(d.w, row[4 * q4 + 3], acc);
        }
        if (t < kb) A[i * ld + k0 + t] = -acc;
      }
    }
    for (int e = tid; e < kb * kb; e += kThreads) {
      const int r = e / kb, c = e % kb;
      A[(k0 + r) * ld + k0 + c] = sh.Dv[r * kLdB + c];
    }
  }
  if (SMEM) {
    __syncthreads();
    for (int r = warp; r < m; r += kWarps)
      for (int c = lane; c < m; c += 32) G[r * m + c] = A[r * ld + c];
  }
}

size_t gj_smem_bytes(int n_max) {
  const size_t mf = (size_t)min(n_max + 1, kSmemM);
  return mf * (mf | 1) * 4;
}

cudaError_t launch_gj_mixed(const SolveArgs& a, cudaStream_t s) {
  const Batch& bt = a.bt;
  if (!a.inverse) return cudaSuccess;  // the LU takes every airfoil
  const size_t smem = gj_smem_bytes(bt.n_max);
  cudaError_t e = ensure_smem(k_gj_mixed<true>, smem);
  if (e != cudaSuccess) return e;
  k_gj_mixed<true><<<bt.B, kThreads, smem, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (bt.n_max + 1 > kSmemM) {
    k_gj_mixed<false><<<bt.B, kThreads, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace panel
