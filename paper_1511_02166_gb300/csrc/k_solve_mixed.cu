// k_solve_mixed.cu -- FP32 LU with partial pivoting + double-float iterative
// refinement for the bordered panel system (the mixed-precision path).
//
// The factor is of the rescaled matrix Mt = S_r M S_c, where S_c multiplies the
// C column and S_r the Kutta row by s = mean |A_jj| (the self-influence scale);
// this balances the border against the influence coefficients and lowers the
// condition number seen by the FP32 factor.  Refinement (Wilkinson/Moler):
//   x_0 = solve(b);  r_k = b - M x_k  with products and sums exact to ~2^-70
//   against the stored planes A_hi + A_lo;  x_{k+1} = x_k + solve(r_k), until
//   |dx|_inf <= tol |x|_inf.  The transposed system M^T lambda = g (g = dCl/du)
//   is refined in the same kernel.
//
// Two kernels:
//  k_lu_mixed  one block per airfoil.  For m <= kSmemM the matrix is copied
//    into shared memory (cp.async) and factored there; beyond, it is factored
//    in place in the caller's LU buffer.  Right-looking, panels of 32 columns:
//    in the shared-memory variant thread t keeps row t of the panel in 32
//    registers (shifted left after every column, so that no register index is
//    dynamic and the loop stays rolled); per column one shuffle argmax per warp,
//    two block barriers, the pivot row broadcast through shared memory.  Then
//    the panel's row exchanges are applied to the other columns, U12 =
//    L11^{-1} A12 is formed (a column per lane) and A22 -= L21 U12 runs as a
//    register-tiled rank-32 update (8 rows x 4 columns per thread).  Finally
//    the 32 x 32 diagonal blocks of L and U are replaced by their inverses, so
//    that the triangular solves below are matrix-vector products.  The stored
//    LU buffer therefore holds this library-internal layout.
//  k_ir_mixed  one small block per airfoil (many per SM): triangular solves
//    with the stored factor (read through L1/L2) and the refinement residuals
//    (one pass over the rows for M u, one over the columns for M^T lambda).
#include "df.cuh"
#include "lu_mixed.cuh"

namespace panel {

// ---------------------------------------------------------------------------
// Pieces shared by both factorisations (all indices fit in 32 bits)
// ---------------------------------------------------------------------------
// Apply the exchanges ipiv[k0..k0+kb) to every column outside [k0, k0+kb).
__device__ __forceinline__ void apply_panel_swaps(float* F, int ld, int m, int k0, int kb,
                                                  const int* ipiv) {
  for (int c = threadIdx.x; c < m; c += kThreads) {
    if (c >= k0 && c < k0 + kb) continue;
    for (int k = k0; k < k0 + kb; ++k) {
      const int p = ipiv[k];
      if (p != k) {
        const float t = F[k * ld + c];
        F[k * ld + c] = F[p * ld + c];
        F[p * ld + c] = t;
      }
    }
  }
}

// U12 = L11^{-1} A12 (L11 unit lower kb x kb), one column per lane.  The base
// of L11 goes through an opaque move per column block so that its loads are
// not hoisted out of the loop.
__device__ __forceinline__ void panel_trsm(float* F, int ld, int m, int k0, int kb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int k1 = k0 + kb;
  for (int cb = k1 + 32 * warp; cb < m; cb += kThreads) {
    const int c = cb + lane;
    const bool ok = c < m;
    int lbase;
    asm volatile("mov.b32 %0, %1;" : "=r"(lbase) : "r"(k0 * ld + k0));
    const float* L11 = F + lbase;
    float col[kNB];
#pragma unroll
    for (int t = 0; t < kNB; ++t) col[t] = (ok && t < kb) ? F[(k0 + t) * ld + c] : 0.0f;
#pragma unroll
    for (int t = 1; t < kNB; ++t) {
      float acc = col[t];
#pragma unroll
      for (int q = 0; q < kNB; ++q)
        if (q < t) acc = fmaf(-L11[t * ld + q], col[q], acc);
      col[t] = acc;
    }
#pragma unroll
    for (int t = 0; t < kNB; ++t)
      if (ok && t < kb) F[(k0 + t) * ld + c] = col[t];
  }
}

// A22 -= L21 U12 over rows/columns [k1, m): warp tiles of 8 rows x 128 columns.
__device__ __forceinline__ void panel_gemm(float* F, int ld, int m, int k0, int kb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int k1 = k0 + kb;
  const int rows = m - k1;
  const int nr = (rows + 7) >> 3;
  const int nc = (rows + 127) >> 7;
  for (int tile = warp; tile < nr * nc; tile += kWarps) {
    const int r0 = k1 + 8 * (tile / nc);
    const int cb = k1 + 128 * (tile % nc) + lane;
    float acc[8][4];
    bool cok[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) cok[t] = cb + 32 * t < m;
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int t = 0; t < 4; ++t)
        acc[a][t] = (r0 + a < m && cok[t]) ? F[(r0 + a) * ld + cb + 32 * t] : 0.0f;
#pragma unroll 2
    for (int q = 0; q < kb; ++q) {
      float lv[8], uv[4];
#pragma unroll
      for (int a = 0; a < 8; ++a) lv[a] = (r0 + a < m) ? F[(r0 + a) * ld + k0 + q] : 0.0f;
#pragma unroll
      for (int t = 0; t < 4; ++t) uv[t] = cok[t] ? F[(k0 + q) * ld + cb + 32 * t] : 0.0f;
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int t = 0; t < 4; ++t) acc[a][t] = fmaf(-lv[a], uv[t], acc[a][t]);
    }
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (r0 + a < m && cok[t]) F[(r0 + a) * ld + cb + 32 * t] = acc[a][t];
  }
}

// ---------------------------------------------------------------------------
// LU with partial pivoting, factor in shared memory, m <= kThreads rows:
// thread t owns row t of the current panel in registers.
// Returns 0 or k+1 for an exactly zero pivot (uniform over the block).
// ---------------------------------------------------------------------------
__device__ int lu_rowpanel(float* F, int ld, int m, int* ipiv, float* prow, float* krow,
                           unsigned long long* cand) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const bool has = t < m;
  for (int k0 = 0; k0 < m; k0 += kNB) {
    const int kb = min(kNB, m - k0);
    float a[kNB];
#pragma unroll
    for (int q = 0; q < kNB; ++q) a[q] = (has && q < kb) ? F[t * ld + k0 + q] : 0.0f;
    for (int q = 0; q < kb; ++q) {
      const int k = k0 + q;
      float4* pr = reinterpret_cast<float4*>(prow + (q & 1) * kNB);
      float4* kr = reinterpret_cast<float4*>(krow + (q & 1) * kNB);
      // warp argmax of |a_tk| over rows t >= k, ties to the lowest row: the key
      // is the float's bit pattern + 1 (monotone for |x|; 0 marks no candidate)
      const unsigned key = (has && t >= k) ? __float_as_uint(fabsf(a[0])) + 1u : 0u;
      const unsigned mx = __reduce_max_sync(0xffffffffu, key);
      const unsigned win = __ffs(__ballot_sync(0xffffffffu, key == mx)) - 1;
      if (lane == 0)
        cand[(q & 1) * kWarps + warp] =
            ((unsigned long long)mx << 32) | (unsigned)(0x7fffffff - (warp * 32 + (int)win));
      __syncthreads();
      unsigned long long best = 0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) best = max(best, cand[(q & 1) * kWarps + w]);
      if ((unsigned)(best >> 32) <= 1u) return k + 1;  // no candidate or |pivot| = 0
      const int p = 0x7fffffff - (int)(best & 0xffffffffu);
      if (t == p) {
#pragma unroll
        for (int c = 0; c < kNB / 4; ++c)
          pr[c] = make_float4(a[4 * c], a[4 * c + 1], a[4 * c + 2], a[4 * c + 3]);
      }
      if (t == k) {
#pragma unroll
        for (int c = 0; c < kNB / 4; ++c)
          kr[c] = make_float4(a[4 * c], a[4 * c + 1], a[4 * c + 2], a[4 * c + 3]);
        ipiv[k] = p;
      }
      __syncthreads();
      if (p != k) {
        if (t == k || t == p) {
          const float4* src = (t == k) ? pr : kr;
#pragma unroll
          for (int c = 0; c < kNB / 4; ++c) {
            const float4 v = src[c];
            a[4 * c] = v.x;
            a[4 * c + 1] = v.y;
            a[4 * c + 2] = v.z;
            a[4 * c + 3] = v.w;
          }
        }
        // exchange the already finished multipliers of rows k and p
        if (warp == 0 && lane < q) {
          const float x = F[k * ld + k0 + lane];
          F[k * ld + k0 + lane] = F[p * ld + k0 + lane];
          F[p * ld + k0 + lane] = x;
        }
      }
      const float* pv = prow + (q & 1) * kNB;
      // row k is final within the panel: U[k][k..k0+kb)
      if (warp == kWarps - 1 && lane < kb - q) F[k * ld + k + lane] = pv[lane];
      if (has && t > k) {
        const float l = a[0] * __frcp_rn(pv[0]);
        F[t * ld + k] = l;
#pragma unroll
        for (int c = 0; c < kNB / 4; ++c) {
          const float4 v = pr[c];
          if (c > 0) a[4 * c - 1] = fmaf(-l, v.x, a[4 * c]);
          a[4 * c] = fmaf(-l, v.y, a[4 * c + 1]);
          a[4 * c + 1] = fmaf(-l, v.z, a[4 * c + 2]);
          a[4 * c + 2] = fmaf(-l, v.w, a[4 * c + 3]);
        }
        a[kNB - 1] = 0.0f;
      }
    }
    __syncthreads();
    apply_panel_swaps(F, ld, m, k0, kb, ipiv);
    __syncthreads();
    if (k0 + kb >= m) break;
    panel_trsm(F, ld, m, k0, kb);
    __syncthreads();
    panel_gemm(F, ld, m, k0, kb);
    __syncthreads();
  }
  return 0;
}


// ---------------------------------------------------------------------------
// The LU kernel, factor in shared memory (m <= kSmemM)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 1) k_lu_mixed(SolveArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const Batch& bt = a.bt;
  const int b = bt.order[blockIdx.x];
  const int n = airfoil_n(bt, b);
  const int m = n + 1;
  if (a.info[b] != 0) return;
  if (m > kSmemM) return;  // taken by k_lu_global
  if (n > bt.n_max) {
    if (threadIdx.x == 0) a.info[b] = PANEL_INFO_TOO_LARGE;
    return;
  }
  double* red = reinterpret_cast<double*>(smraw);      // 32
  int* ipiv = reinterpret_cast<int*>(red + 32);         // n_max + 1
  float* prow = reinterpret_cast<float*>(
      (reinterpret_cast<uintptr_t>(ipiv + bt.n_max + 1) + 15) & ~(uintptr_t)15);  // 2 kNB
  float* krow = prow + 2 * kNB;                                                    // 2 kNB
  unsigned long long* cand = reinterpret_cast<unsigned long long*>(krow + 2 * kNB);  // 2 kWarps
  float* F = reinterpret_cast<float*>(cand + 2 * kWarps);

  const int64_t moff = bt.mat_off[b];
  const float* Ah = a.A_hi + moff;
  const int ld = m | 1;
  const float sf = (float)border_scale(Ah, n, m, red);

  // copy the hi plane asynchronously into shared memory, rescale the border
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int rr = warp; rr < m; rr += kWarps)
    for (int cc = lane; cc < m; cc += 32) {
      const unsigned dst = (unsigned)__cvta_generic_to_shared(F + rr * ld + cc);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(Ah + rr * m + cc));
    }
  asm volatile("cp.async.wait_all;\n" ::);
  __syncthreads();
  for (int j = threadIdx.x; j < m; j += kThreads) {
    if (j < n) F[j * ld + n] *= sf;
    F[n * ld + j] *= sf;
  }
  __syncthreads();
  const int st = lu_rowpanel(F, ld, m, ipiv, prow, krow, cand);
  if (st != 0) {
    if (threadIdx.x == 0) {
      a.info[b] = st;
      if (a.iters) a.iters[b] = 0;
    }
    return;
  }
  invert_diagonal_blocks(F, ld, m);
  __syncthreads();
  int32_t* gpiv = a.piv + vec_off(bt, b);
  for (int k = threadIdx.x; k < m; k += kThreads) gpiv[k] = ipiv[k];
  float* G = a.LU + moff;
  for (int rr = warp; rr < m; rr += kWarps)
    for (int cc = lane; cc < m; cc += 32) G[rr * m + cc] = F[rr * ld + cc];
}

size_t lu_mixed_smem(int n_max) {
  const int mf = n_max + 1;
  size_t bytes = 32 * 8 + (size_t)(n_max + 1) * 4 + 16 + 4 * kNB * 4 + 2 * kWarps * 8;
  bytes = (bytes + 15) & ~(size_t)15;
  return bytes + (size_t)mf * (size_t)(mf | 1) * 4;
}

// ---------------------------------------------------------------------------
// The LU kernel, factor in global memory (m > kSmemM): blocked right-looking
// with the current panel of NB columns staged in shared memory (rows spread
// over the threads), the row exchanges, U12 and the rank-NB update applied to
// the factor in the caller's LU buffer through L2.  Shared memory stays small
// (the panel plus a 128-column slab of U12), so several airfoils share an SM
// and hide each other's latencies.
// ---------------------------------------------------------------------------
template <int NB>
__global__ void __launch_bounds__(kThreads, 2) k_lu_global(SolveArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int LDP = NB + 1;
  constexpr int CW = 128;  // GEMM column slab
  const Batch& bt = a.bt;
  const int b = bt.order[blockIdx.x];
  const int n = airfoil_n(bt, b);
  const int m = n + 1;
  if (a.info[b] != 0) return;
  if (m <= kSmemM && !a.force_global) return;  // taken by k_lu_mixed
  if (n > a.n_cap) {
    if (threadIdx.x == 0) a.info[b] = PANEL_INFO_TOO_LARGE;
    return;
  }
  if (m > kLargeM) return;  // taken by the blocked factor (k_lu_large.cu)
  const int mv = bt.n_max + 1;
  float* P = reinterpret_cast<float*>(smraw);           // mv x LDP panel
  float* U = P + mv * LDP;                              // NB x CW slab of U12
  double* red = reinterpret_cast<double*>(
      (reinterpret_cast<uintptr_t>(U + NB * CW) + 15) & ~(uintptr_t)15);  // 32
  unsigned long long* cand = reinterpret_cast<unsigned long long*>(red + 32);  // kWarps
  int* ipiv = reinterpret_cast<int*>(cand + kWarps);    // mv

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t moff = bt.mat_off[b];
  const float* Ah = a.A_hi + moff;
  float* F = a.LU + moff;
  const float sf = (float)border_scale(Ah, n, m, red);
  for (int rr = warp; rr < m; rr += kWarps)
    for (int cc = lane; cc < m; cc += 32) {
      const float v = Ah[rr * m + cc];
      F[rr * m + cc] = ((cc == n && rr < n) || rr == n) ? v * sf : v;
    }
  __syncthreads();

  for (int k0 = 0; k0 < m; k0 += NB) {
    const int kb = min(NB, m - k0);
    const int rows = m - k0;
    // ---- stage the panel ----
    for (int r = warp; r < rows; r += kWarps)
      if (lane < kb) P[r * LDP + lane] = F[(k0 + r) * m + k0 + lane];
    __syncthreads();
    // ---- factor the panel (rows over the threads) ----
    for (int q = 0; q < kb; ++q) {
      unsigned bk = 0;
      int br = 0x7fffffff;
      for (int r = q + tid; r < rows; r += kThreads) {
        const unsigned key = __float_as_uint(fabsf(P[r * LDP + q])) + 1u;
        if (key > bk) { bk = key; br = r; }
      }
      const unsigned mx = __reduce_max_sync(0xffffffffu, bk);
      const unsigned rmin = __reduce_min_sync(0xffffffffu, bk == mx ? (unsigned)br : 0xffffffffu);
      if (lane == 0) cand[warp] = ((unsigned long long)mx << 32) | (0x7fffffffu - rmin);
      __syncthreads();
      unsigned long long best = 0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) best = max(best, cand[w]);
      if ((unsigned)(best >> 32) <= 1u) {
        if (tid == 0) {
          a.info[b] = k0 + q + 1;
          if (a.iters) a.iters[b] = 0;
        }
        return;
      }
      const int p = (int)(0x7fffffffu - (unsigned)(best & 0xffffffffu));
      if (p != q && tid < kb) {
        const float t = P[q * LDP + tid];
        P[q * LDP + tid] = P[p * LDP + tid];
        P[p * LDP + tid] = t;
      }
      if (tid == 0) ipiv[k0 + q] = k0 + p;
      __syncthreads();
      const float inv = 1.0f / P[q * LDP + q];
      for (int r = q + 1 + tid; r < rows; r += kThreads) {
        const float l = P[r * LDP + q] * inv;
        P[r * LDP + q] = l;
        for (int c = q + 1; c < kb; ++c) P[r * LDP + c] = fmaf(-l, P[q * LDP + c], P[r * LDP + c]);
      }
      __syncthreads();
    }
    // ---- write the panel back, exchange rows outside it ----
    for (int r = warp; r < rows; r += kWarps)
      if (lane < kb) F[(k0 + r) * m + k0 + lane] = P[r * LDP + lane];
    for (int c = tid; c < m; c += kThreads) {
      if (c >= k0 && c < k0 + kb) continue;
      for (int k = k0; k < k0 + kb; ++k) {
        const int pk = ipiv[k];
        if (pk != k) {
          const float t = F[k * m + c];
          F[k * m + c] = F[pk * m + c];
          F[pk * m + c] = t;
        }
      }
    }
    __syncthreads();
    const int k1 = k0 + kb;
    if (k1 >= m) break;
    // ---- U12 = L11^{-1} A12, a column per lane, shifted registers ----
    for (int cb = k1 + 32 * warp; cb < m; cb += kThreads) {
      const int c = cb + lane;
      const bool ok = c < m;
      float col[NB];
#pragma unroll
      for (int t = 0; t < NB; ++t) col[t] = (ok && t < kb) ? F[(k0 + t) * m + c] : 0.0f;
      for (int q = 0; q < kb; ++q) {
        const float x = col[0];
        if (ok) F[(k0 + q) * m + c] = x;
#pragma unroll
        for (int t = 1; t < NB; ++t) {
          const float l = (q + t < kb) ? P[(q + t) * LDP + q] : 0.0f;
          col[t - 1] = fmaf(-l, x, col[t]);
        }
        col[NB - 1] = 0.0f;
      }
    }
    __syncthreads();
    // ---- A22 -= L21 U12, 128-column slabs of U12 staged in shared memory ----
    const int nrt = (m - k1 + 7) >> 3;
    for (int cc = k1; cc < m; cc += CW) {
      for (int t = warp; t < kb; t += kWarps)
#pragma unroll
        for (int j = 0; j < CW / 32; ++j) {
          const int c = cc + lane + 32 * j;
          U[t * CW + lane + 32 * j] = (c < m) ? F[(k0 + t) * m + c] : 0.0f;
        }
      __syncthreads();
      for (int rt = warp; rt < nrt; rt += kWarps) {
        const int r0 = k1 + 8 * rt;
        float acc[8][4];
#pragma unroll
        for (int aa = 0; aa < 8; ++aa)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int r = r0 + aa, c = cc + lane + 32 * j;
            acc[aa][j] = (r < m && c < m) ? F[r * m + c] : 0.0f;
          }
#pragma unroll 4
        for (int q = 0; q < kb; ++q) {
          float lv[8], uv[4];
#pragma unroll
          for (int aa = 0; aa < 8; ++aa) lv[aa] = (r0 + aa < m) ? P[(r0 + aa - k0) * LDP + q] : 0.0f;
#pragma unroll
          for (int j = 0; j < 4; ++j) uv[j] = U[q * CW + lane + 32 * j];
#pragma unroll
          for (int aa = 0; aa < 8; ++aa)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[aa][j] = fmaf(-lv[aa], uv[j], acc[aa][j]);
        }
#pragma unroll
        for (int aa = 0; aa < 8; ++aa)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int r = r0 + aa, c = cc + lane + 32 * j;
            if (r < m && c < m) F[r * m + c] = acc[aa][j];
          }
      }
      __syncthreads();
    }
  }
  invert_diagonal_blocks(F, m, m);
  __syncthreads();
  int32_t* gpiv = a.piv + vec_off(bt, b);
  for (int k = tid; k < m; k += kThreads) gpiv[k] = ipiv[k];
}

template <int NB>
size_t lu_global_smem(int n_max) {
  const size_t mv = (size_t)n_max + 1;
  size_t bytes = mv * (NB + 1) * 4 + (size_t)NB * 128 * 4;
  bytes = (bytes + 15) & ~(size_t)15;
  return bytes + 32 * 8 + kWarps * 8 + mv * 4;
}

// ---------------------------------------------------------------------------
// Triangular solves with the stored factor (global memory, ld = m, diagonal
// blocks inverted), on a float vector y in shared memory; `t32` is a 32-float
// shared scratch.  Every 32-row block takes two block barriers and all eight
// warps: a warp owns 4 rows of the block and reduces across its lanes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// y <- L^{-1} y then U^{-1} y, left-looking: the rows of block d read their
// own contiguous segments L[i][0..k0) (coalesced across the lanes).
__device__ void lu_apply_inverse(const float* __restrict__ F, int m, float* y, float* t32) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k0 = 0; k0 < m; k0 += 32) {
    const int kb = min(32, m - k0);
    for (int q = warp; q < kb; q += kWarps) {
      const int i = k0 + q;
      const float* row = F + i * m;
      float acc = 0.0f;
      for (int k = lane; k < k0; k += 32) acc = fmaf(__ldg(row + k), y[k], acc);
      acc = warp_sum_f(acc);
      if (lane == 0) t32[q] = y[i] - acc;
    }
    __syncthreads();
    for (int q = warp; q < kb; q += kWarps) {
      const int i = k0 + q;
      // z_i = t_i + sum_{k<i} X[i][k] t_k  (X unit lower, stored below the diagonal)
      float v = (lane < q) ? __ldg(F + i * m + k0 + lane) * t32[lane] : 0.0f;
      v = warp_sum_f(v);
      if (lane == 0) y[i] = t32[q] + v;
    }
    __syncthreads();
  }
  for (int k0 = ((m - 1) >> 5) << 5; k0 >= 0; k0 -= 32) {
    const int kb = min(32, m - k0);
    for (int q = warp; q < kb; q += kWarps) {
      const int i = k0 + q;
      const float* row = F + i * m;
      float acc = 0.0f;
      for (int k = k0 + kb + lane; k < m; k += 32) acc = fmaf(__ldg(row + k), y[k], acc);
      acc = warp_sum_f(acc);
      if (lane == 0) t32[q] = y[i] - acc;
    }
    __syncthreads();
    for (int q = warp; q < kb; q += kWarps) {
      const int i = k0 + q;
      // x_i = sum_{k>=i} Y[i][k] t_k  (Y upper with diagonal)
      float v = (lane >= q && lane < kb) ? __ldg(F + i * m + k0 + lane) * t32[lane] : 0.0f;
      v = warp_sum_f(v);
      if (lane == 0) y[i] = v;
    }
    __syncthreads();
  }
}

// y <- U^{-T} y then L^{-T} y.  Right-looking updates (a thread per row r reads
// U[k][r], coalesced across r); the diagonal products are split over the warps.
__device__ void lu_apply_inverse_transposed(const float* __restrict__ F, int m, float* y,
                                            float* t32) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k0 = 0; k0 < m; k0 += 32) {
    const int kb = min(32, m - k0);
    if (threadIdx.x < 32) t32[lane] = (lane < kb) ? y[k0 + lane] : 0.0f;
    __syncthreads();
    for (int q = warp; q < kb; q += kWarps) {
      // z_i = sum_{k<=i} Y[k][i] t_k
      const int i = k0 + q;
      float v = (lane <= q) ? __ldg(F + (k0 + lane) * m + i) * t32[lane] : 0.0f;
      v = warp_sum_f(v);
      if (lane == 0) y[i] = v;
    }
    __syncthreads();
    for (int r = k0 + kb + threadIdx.x; r < m; r += kThreads) {
      float acc = y[r];
#pragma unroll 8
      for (int t = 0; t < kb; ++t) acc = fmaf(-__ldg(F + (k0 + t) * m + r), y[k0 + t], acc);
      y[r] = acc;
    }
    __syncthreads();
  }
  for (int k0 = ((m - 1) >> 5) << 5; k0 >= 0; k0 -= 32) {
    const int kb = min(32, m - k0);
    if (threadIdx.x < 32) t32[lane] = (lane < kb) ? y[k0 + lane] : 0.0f;
    __syncthreads();
    for (int q = warp; q < kb; q += kWarps) {
      // z_i = t_i + sum_{k>i} X[k][i] t_k
      const int i = k0 + q;
      float v = (lane > q && lane < kb) ? __ldg(F + (k0 + lane) * m + i) * t32[lane] : 0.0f;
      v = warp_sum_f(v);
      if (lane == 0) y[i] = t32[q] + v;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < k0; r += kThreads) {
      float acc = y[r];
#pragma unroll 8
      for (int t = 0; t < kb; ++t) acc = fmaf(-__ldg(F + (k0 + t) * m + r), y[k0 + t], acc);
      y[r] = acc;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Double-float residuals against the stored planes
// ---------------------------------------------------------------------------
// Accumulator for sum_k (h_k + l_k)(xh_k + xl_k) with error ~2^-70 sum|p|:
// s1 collects the exact leading products h*xh through two_sum (their rounding
// errors go to s2), s2 (double-float) collects the ~2^-24 terms (the two_prod
// error of h*xh, h*xl, l*xh) and s3 (float) the ~2^-48 terms (the errors of
// h*xl and l*xh, and l*xl).  Every product is exact via two_prod.
struct ResAcc {
  float s1, s3;
  df2 s2;
};
__device__ __forceinline__ void resacc_init(ResAcc& a) {
  a.s1 = 0.0f;
  a.s3 = 0.0f;
  a.s2 = mkdf(0.0f);
}
__device__ __forceinline__ void resacc_add(ResAcc& a, float h, float l, float xh, float xl) {
  const df2 p1 = two_prod(h, xh);
  const df2 p2 = two_prod(h, xl);
  const df2 p3 = two_prod(l, xh);
  const df2 t = two_sum(a.s1, p1.hi);
  a.s1 = t.hi;
  a.s2 = df_add_f(a.s2, t.lo);
  a.s2 = df_add_f(a.s2, p1.lo);
  a.s2 = df_add_f(a.s2, p2.hi);
  a.s2 = df_add_f(a.s2, p3.hi);
  a.s3 = __fadd_rn(a.s3, __fadd_rn(__fadd_rn(p2.lo, p3.lo), __fmul_rn(l, xl)));
}
__device__ __forceinline__ void resacc_merge(ResAcc& a, const ResAcc& b) {
  const df2 t = two_sum(a.s1, b.s1);
  a.s1 = t.hi;
  a.s2 = df_add_f(a.s2, t.lo);
  a.s2 = df_add(a.s2, b.s2);
  a.s3 = __fadd_rn(a.s3, b.s3);
}
__device__ __forceinline__ ResAcc warp_sum_res(ResAcc a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ResAcc b;
    b.s1 = __shfl_xor_sync(0xffffffffu, a.s1, o);
    b.s2.hi = __shfl_xor_sync(0xffffffffu, a.s2.hi, o);
    b.s2.lo = __shfl_xor_sync(0xffffffffu, a.s2.lo, o);
    b.s3 = __shfl_xor_sync(0xffffffffu, a.s3, o);
    resacc_merge(a, b);
  }
  return a;
}
// c - acc in FP64 (c is FP64).
__device__ __forceinline__ double resacc_sub_from(double c, const ResAcc& a) {
  return ((c - (double)a.s1) - ((double)a.s2.hi + (double)a.s2.lo)) - (double)a.s3;
}

// r_j = b_j - sum_i M_ji x_i for all rows j; x given as float pairs (xh, xl).
// A warp takes two rows at a time and issues all loads of a 256-column chunk
// before accumulating.
__device__ void residual_rows(const float* __restrict__ Ah, const float* __restrict__ Al, int m,
                              const float* xh, const float* xl, const double* b, double* r) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j0 = 2 * warp; j0 < m; j0 += 2 * kWarps) {
    ResAcc acc0, acc1;
    resacc_init(acc0);
    resacc_init(acc1);
    const bool two = j0 + 1 < m;
    for (int c0 = 0; c0 < m; c0 += 256) {
      float h0[8], l0[8], h1[8], l1[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int c = c0 + lane + 32 * t;
        const bool ok = c < m;
        h0[t] = ok ? __ldg(Ah + j0 * m + c) : 0.0f;
        l0[t] = ok ? __ldg(Al + j0 * m + c) : 0.0f;
        h1[t] = (ok && two) ? __ldg(Ah + (j0 + 1) * m + c) : 0.0f;
        l1[t] = (ok && two) ? __ldg(Al + (j0 + 1) * m + c) : 0.0f;
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int c = c0 + lane + 32 * t;
        if (c < m) {
          const float xa = xh[c], xb = xl[c];
          resacc_add(acc0, h0[t], l0[t], xa, xb);
          resacc_add(acc1, h1[t], l1[t], xa, xb);
        }
      }
    }
    acc0 = warp_sum_res(acc0);
    acc1 = warp_sum_res(acc1);
    if (lane == 0) {
      r[j0] = resacc_sub_from(b[j0], acc0);
      if (two) r[j0 + 1] = resacc_sub_from(b[j0 + 1], acc1);
    }
  }
}

// r_i = g_i - sum_j M_ji x_j for all columns i: each warp owns 32 consecutive
// columns (one per lane) and walks all rows, 8 rows of loads in flight.
__device__ void residual_cols(const float* __restrict__ Ah, const float* __restrict__ Al, int m,
                              const float* xh, const float* xl, const double* g, double* r) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int cb = 32 * warp; cb < m; cb += kThreads) {
    const int c = cb + lane;
    const bool ok = c < m;
    ResAcc acc;
    resacc_init(acc);
    for (int jb = 0; jb < m; jb += 8) {
      float h[8], l[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int j = jb + q;
        h[q] = (ok && j < m) ? __ldg(Ah + j * m + c) : 0.0f;
        l[q] = (ok && j < m) ? __ldg(Al + j * m + c) : 0.0f;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (jb + q < m) resacc_add(acc, h[q], l[q], xh[jb + q], xl[jb + q]);
    }
    if (ok) r[c] = resacc_sub_from(g[c], acc);
  }
}

// ---------------------------------------------------------------------------
// The refinement kernel: forward and/or transposed system of one airfoil
// ---------------------------------------------------------------------------
struct IrSystem {
  double* x;   // m  current solution
  double* r;   // m  residual
  double* bb;  // m  right-hand side
  float* xh;   // m
  float* xl;   // m
};

__global__ void __launch_bounds__(kThreads, 3) k_ir_mixed(SolveArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const Batch& bt = a.bt;
  const int b = bt.order[blockIdx.x];
  const int n = airfoil_n(bt, b);
  const int m = n + 1;
  if (a.info[b] != 0 || n > bt.n_max) return;
  const int mv = bt.n_max + 1;
  double* red = reinterpret_cast<double*>(smraw);  // 32
  IrSystem sys[2];
  double* dp = red + 32;
  for (int q = 0; q < 2; ++q) {
    sys[q].x = dp;
    sys[q].r = dp + mv;
    sys[q].bb = dp + 2 * mv;
    dp += 3 * mv;
  }
  float* y = reinterpret_cast<float*>(dp);  // m
  float* fp = y + mv;
  for (int q = 0; q < 2; ++q) {
    sys[q].xh = fp;
    sys[q].xl = fp + mv;
    fp += 2 * mv;
  }
  int* perm = reinterpret_cast<int*>(fp);  // m
  float* t32 = reinterpret_cast<float*>(perm + mv);  // 32

  const int64_t moff = bt.mat_off[b];
  const float* Ah = a.A_hi + moff;
  const float* Al = a.A_lo + moff;
  const float* F = a.LU + moff;
  const int32_t* gpiv = a.piv + vec_off(bt, b);
  const double s = border_scale(Ah, n, m, red);
  const bool act0 = a.u != nullptr, act1 = a.lam != nullptr;

  // right-hand sides: b, and g = dCl/du = 2 |h_k| / (v c) (0 for C)
  const double* nd = bt.nodes + 2 * bt.node_off[b];
  const double v = a.vinf ? a.vinf[b] : 1.0, cc = a.chord ? a.chord[b] : 1.0;
  for (int k = threadIdx.x; k < m; k += kThreads) {
    if (act0) sys[0].bb[k] = a.rhs[vec_off(bt, b) + k];
    if (act1) {
      double g = 0.0;
      if (k < n) {
        const int k1 = (k + 1 == n) ? 0 : k + 1;
        const double hx = nd[2 * k1] - nd[2 * k], hy = nd[2 * k1 + 1] - nd[2 * k + 1];
        g = 2.0 * sqrt(hx * hx + hy * hy) / (v * cc);
      }
      sys[1].bb[k] = g;
    }
    for (int q = 0; q < 2; ++q) {
      sys[q].x[k] = 0.0;
      sys[q].r[k] = sys[q].bb[k];
    }
  }
  // row permutation of the factor: P y = y[perm]
  if (threadIdx.x == 0) {
    for (int k = 0; k < m; ++k) perm[k] = k;
    for (int k = 0; k < m; ++k) {
      const int p = gpiv[k];
      const int t = perm[k];
      perm[k] = perm[p];
      perm[p] = t;
    }
  }
  __syncthreads();

  bool active[2] = {act0, act1};
  bool conv[2] = {!act0, !act1};
  int it = 0;
  for (;; ++it) {
    for (int q = 0; q < 2; ++q) {
      if (!active[q] || conv[q]) continue;
      IrSystem& S = sys[q];
      if (q == 0) {
        // y = P S_r r;  solve;  dx = S_c y
        for (int k = threadIdx.x; k < m; k += kThreads) {
          const int src = perm[k];
          y[k] = (float)((src == n) ? S.r[src] * s : S.r[src]);
        }
        __syncthreads();
        lu_apply_inverse(F, m, y, t32);
      } else {
        // z = Mt^{-T} S_c r;  dlambda = S_r P^T z
        for (int k = threadIdx.x; k < m; k += kThreads)
          y[k] = (float)((k == n) ? S.r[k] * s : S.r[k]);
        __syncthreads();
        lu_apply_inverse_transposed(F, m, y, t32);
      }
      double dmax = 0.0;
      for (int k = threadIdx.x; k < m; k += kThreads) {
        const int dst = (q == 0) ? k : perm[k];
        const double d = (dst == n) ? (double)y[k] * s : (double)y[k];
        S.x[dst] += d;
        dmax = fmax(dmax, fabs(d));
      }
      __syncthreads();
      double xmax = 0.0;
      for (int k = threadIdx.x; k < m; k += kThreads) xmax = fmax(xmax, fabs(S.x[k]));
      dmax = block_absmax_d(dmax, red);
      xmax = block_absmax_d(xmax, red);
      if (it >= 1 && dmax <= a.tol * xmax) conv[q] = true;
    }
    if ((conv[0] && conv[1]) || it >= a.max_iter) break;
    for (int q = 0; q < 2; ++q) {
      if (!active[q] || conv[q]) continue;
      for (int k = threadIdx.x; k < m; k += kThreads) {
        const df2 d = df_from_double(sys[q].x[k]);
        sys[q].xh[k] = d.hi;
        sys[q].xl[k] = d.lo;
      }
    }
    __syncthreads();
    if (active[0] && !conv[0]) residual_rows(Ah, Al, m, sys[0].xh, sys[0].xl, sys[0].bb, sys[0].r);
    if (active[1] && !conv[1]) residual_cols(Ah, Al, m, sys[1].xh, sys[1].xl, sys[1].bb, sys[1].r);
    __syncthreads();
  }
  for (int k = threadIdx.x; k < m; k += kThreads) {
    if (act0) a.u[vec_off(bt, b) + k] = sys[0].x[k];
    if (act1) a.lam[vec_off(bt, b) + k] = sys[1].x[k];
  }
  if (threadIdx.x == 0) {
    if (a.iters && act0) a.iters[b] = it;
    if (!(conv[0] && conv[1])) a.info[b] = PANEL_INFO_NOCONV;
  }
}

size_t ir_mixed_smem(int n_max) {
  const size_t mv = (size_t)n_max + 1;
  return 32 * 8 + 6 * mv * 8 + 5 * mv * 4 + mv * 4 + 32 * 4 + 16;
}

static SolveArgs make_args(const Batch& bt, const float* A_hi, const float* A_lo, float* LU,
                           int32_t* piv, const double* rhs, const double* vinf,
                           const double* chord, double* u, double* lam, int max_iter, double tol,
                           int32_t* info, int32_t* iters) {
  SolveArgs a;
  a.bt = bt;
  a.A_hi = A_hi;
  a.A_lo = A_lo;
  a.LU = LU;
  a.piv = piv;
  a.rhs = rhs;
  a.vinf = vinf;
  a.chord = chord;
  a.u = u;
  a.lam = lam;
  a.max_iter = max_iter;
  a.tol = tol;
  a.info = info;
  a.iters = iters;
  a.force_global = 0;
  a.n_cap = bt.n_max;
  return a;
}

// Factor every airfoil (shared-memory kernel for m <= kSmemM, global beyond).
constexpr size_t kMaxSmem = 232448;
cudaError_t launch_lu_mixed(const Batch& bt, const float* A_hi, float* LU, int32_t* piv,
                            int32_t* info, int32_t* iters, bool force_global, cudaStream_t s) {
  SolveArgs a = make_args(bt, A_hi, nullptr, LU, piv, nullptr, nullptr, nullptr, nullptr,
                          nullptr, 0, 0.0, info, iters);
  a.force_global = force_global ? 1 : 0;
  cudaError_t e;
  if (bt.n_max + 1 > kLargeM) {
    e = launch_lu_large(a, s);
    if (e != cudaSuccess) return e;
  }
  if (bt.n_max + 1 > kSmemM || force_global) {
    SolveArgs g = a;
    g.bt.n_max = min(bt.n_max, kLargeM - 1);
    const size_t smem = lu_global_smem<32>(g.bt.n_max);
    e = ensure_smem(k_lu_global<32>, smem);
    if (e != cudaSuccess) return e;
    k_lu_global<32><<<bt.B, kThreads, smem, s>>>(g);
    e = cudaGetLastError();
    if (e != cudaSuccess || force_global) return e;
  }
  Batch bs = bt;
  bs.n_max = min(bt.n_max, kSmemM - 1);
  a.bt = bs;
  const size_t smem = lu_mixed_smem(bs.n_max);
  e = ensure_smem(k_lu_mixed, smem);
  if (e != cudaSuccess) return e;
  k_lu_mixed<<<bt.B, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

// Refine the forward (u) and/or transposed (lam) systems with the stored factor.
cudaError_t launch_ir_mixed(const Batch& bt, const float* A_hi, const float* A_lo,
                            const float* LU, const int32_t* piv, const double* rhs,
                            const double* vinf, const double* chord, double* u, double* lam,
                            int max_iter, double tol, int32_t* info, int32_t* iters,
                            cudaStream_t s) {
  SolveArgs a = make_args(bt, A_hi, A_lo, const_cast<float*>(LU), const_cast<int32_t*>(piv),
                          rhs, vinf, chord, u, lam, max_iter, tol, info, iters);
  const size_t smem = ir_mixed_smem(bt.n_max);
  cudaError_t e = ensure_smem(k_ir_mixed, smem);
  if (e != cudaSuccess) return e;
  k_ir_mixed<<<bt.B, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace panel
