// k_solve_mixed.cu -- FP32 LU with partial pivoting + double-float iterative
// refinement for the bordered panel system (the mixed-precision path).
//
// The factor is of the rescaled matrix Mt = S_r M S_c, where S_c multiplies the
// C column and S_r the Kutta row by s = mean |A_jj| (the self-influence scale);
// this balances the border against the influence coefficients and lowers the
// condition number seen by the FP32 factor.  Refinement (Wilkinson/Moler):
//   x_0 = solve(b);  r_k = b - M x_k  in double-float from the stored planes
//   A_hi + A_lo;  x_{k+1} = x_k + solve(r_k), until |dx|_inf <= tol |x|_inf.
// The transposed system M^T lambda = g (g = dCl/du) is refined the same way.
//
// Factorisation: right-looking, panels of NB = 32 columns.  SMEM = true (the
// whole m x m factor in shared memory, m <= kSmemM): thread t keeps row t of
// the panel in 32 registers; per column one shuffle argmax per warp, the warp
// winners meet in shared memory, the pivot row is broadcast through shared
// memory and every row below updates its registers (two block barriers per
// column).  SMEM = false (factor in the caller's LU buffer in global memory,
// any m): the panel lives in memory and every warp runs the pivot search.
// After a panel, its row exchanges are applied to the other columns,
// U12 = L11^{-1} A12 is formed (a column per thread) and A22 -= L21 U12 runs as
// a register-tiled rank-32 update (8 rows x 4 columns per thread, columns
// lane-interleaved so that shared-memory loads are conflict-free).
#include "df.cuh"
#include "panel_common.cuh"

namespace panel {

constexpr int kSmemM = 230;  // largest m = n + 1 factored in shared memory
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
  double* out;       // u (forward) or lambda (transposed)
  int max_iter;
  double tol;
  int32_t* info;
  int32_t* iters;
  int trans;         // 0: M x = b, 1: M^T x = g (reuses the factor in LU/piv)
};

// ---------------------------------------------------------------------------
// block-level helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_absmax_d(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = 0.0;
  for (int w = 0; w < kWarps; ++w) r = fmax(r, red[w]);
  __syncthreads();
  return r;
}

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
// of L11 is passed through an opaque move each column block, so that the 496
// loads of L11 are not hoisted out of the loop into registers.
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
                           float* cand_v, int* cand_i) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const bool has = t < m;
  for (int k0 = 0; k0 < m; k0 += kNB) {
    const int kb = min(kNB, m - k0);
    float a[kNB];
#pragma unroll
    for (int q = 0; q < kNB; ++q) a[q] = (has && q < kb) ? F[t * ld + k0 + q] : 0.0f;
#pragma unroll
    for (int q = 0; q < kNB; ++q) {
      if (q < kb) {
        const int k = k0 + q;
        float v = (has && t >= k) ? fabsf(a[q]) : -1.0f;
        int vi = t;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float ov = __shfl_xor_sync(0xffffffffu, v, o);
          const int oi = __shfl_xor_sync(0xffffffffu, vi, o);
          if (ov > v || (ov == v && oi < vi)) { v = ov; vi = oi; }
        }
        if (lane == 0) {
          cand_v[warp] = v;
          cand_i[warp] = vi;
        }
        __syncthreads();
        float best = -1.0f;
        int p = k;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
          const float cv = cand_v[w];
          const int ci = cand_i[w];
          if (cv > best || (cv == best && ci < p)) { best = cv; p = ci; }
        }
        if (best <= 0.0f) return k + 1;
        if (t == p) {
#pragma unroll
          for (int c = 0; c < kNB; ++c) prow[c] = a[c];
        }
        if (t == k) {
#pragma unroll
          for (int c = 0; c < kNB; ++c) krow[c] = a[c];
          ipiv[k] = p;
        }
        __syncthreads();
        if (t == k && p != k) {
#pragma unroll
          for (int c = 0; c < kNB; ++c) a[c] = prow[c];
        }
        if (t == p && p != k) {
#pragma unroll
          for (int c = 0; c < kNB; ++c) a[c] = krow[c];
        }
        if (has && t > k) {
          const float l = a[q] / prow[q];
          a[q] = l;
#pragma unroll
          for (int c = q + 1; c < kNB; ++c) a[c] = fmaf(-l, prow[c], a[c]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kNB; ++q)
      if (has && q < kb) F[t * ld + k0 + q] = a[q];
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
// LU with partial pivoting, factor in global memory (any m).
// ---------------------------------------------------------------------------
__device__ int lu_blocked(float* F, int ld, int m, int* ipiv) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k0 = 0; k0 < m; k0 += kNB) {
    const int kb = min(kNB, m - k0);
    for (int k = k0; k < k0 + kb; ++k) {
      float best = -1.0f;
      int bi = k;
      for (int r = k + lane; r < m; r += 32) {
        const float v = fabsf(F[r * ld + k]);
        if (v > best) { best = v; bi = r; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      const int p = bi;
      if (best <= 0.0f) return k + 1;
      __syncthreads();  // everyone has read column k before rows move
      if (p != k && threadIdx.x < kb) {
        const int c = k0 + threadIdx.x;
        const float tt = F[k * ld + c];
        F[k * ld + c] = F[p * ld + c];
        F[p * ld + c] = tt;
      }
      if (threadIdx.x == 0) ipiv[k] = p;
      __syncthreads();
      const float inv = 1.0f / F[k * ld + k];
      const int c = k0 + lane;
      const float fkc = (lane < kb && c > k) ? F[k * ld + c] : 0.0f;
      for (int r = k + 1 + warp; r < m; r += kWarps) {
        const float l = F[r * ld + k] * inv;
        __syncwarp();
        if (lane < kb && c > k) F[r * ld + c] = fmaf(-l, fkc, F[r * ld + c]);
        if (c == k) F[r * ld + k] = l;
      }
      __syncthreads();
    }
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
// Triangular solves with the factor, on a float vector y (shared memory).
// Blocks of 32 rows: warp 0 solves the diagonal block with shuffles, then all
// threads update the rows below (or above) with that block.
// ---------------------------------------------------------------------------
// y <- L^{-1} y (unit lower) then U^{-1} y.
__device__ void lu_apply_inverse(const float* F, int ld, int m, float* y) {
  const int lane = threadIdx.x & 31;
  for (int k0 = 0; k0 < m; k0 += 32) {
    const int kb = min(32, m - k0);
    if (threadIdx.x < 32) {
      float v = (lane < kb) ? y[k0 + lane] : 0.0f;
      for (int t = 0; t < kb; ++t) {
        const float yt = __shfl_sync(0xffffffffu, v, t);
        if (lane > t && lane < kb) v = fmaf(-F[(k0 + lane) * ld + k0 + t], yt, v);
      }
      if (lane < kb) y[k0 + lane] = v;
    }
    __syncthreads();
    for (int r = k0 + kb + threadIdx.x; r < m; r += kThreads) {
      float s = y[r];
      for (int t = 0; t < kb; ++t) s = fmaf(-F[r * ld + k0 + t], y[k0 + t], s);
      y[r] = s;
    }
    __syncthreads();
  }
  for (int k1 = m; k1 > 0; k1 -= 32) {
    const int k0 = max(0, k1 - 32);
    const int kb = k1 - k0;
    if (threadIdx.x < 32) {
      float v = (lane < kb) ? y[k0 + lane] : 0.0f;
      for (int t = kb - 1; t >= 0; --t) {
        float vt = (lane == t) ? v / F[(k0 + t) * ld + k0 + t] : v;
        const float yt = __shfl_sync(0xffffffffu, vt, t);
        if (lane == t) v = vt;
        if (lane < t) v = fmaf(-F[(k0 + lane) * ld + k0 + t], yt, v);
      }
      if (lane < kb) y[k0 + lane] = v;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < k0; r += kThreads) {
      float s = y[r];
      for (int t = 0; t < kb; ++t) s = fmaf(-F[r * ld + k0 + t], y[k0 + t], s);
      y[r] = s;
    }
    __syncthreads();
  }
}

// y <- U^{-T} y (lower, non-unit) then L^{-T} y (unit upper).
__device__ void lu_apply_inverse_transposed(const float* F, int ld, int m, float* y) {
  const int lane = threadIdx.x & 31;
  for (int k0 = 0; k0 < m; k0 += 32) {
    const int kb = min(32, m - k0);
    if (threadIdx.x < 32) {
      float v = (lane < kb) ? y[k0 + lane] : 0.0f;
      for (int t = 0; t < kb; ++t) {
        float vt = (lane == t) ? v / F[(k0 + t) * ld + k0 + t] : v;
        const float yt = __shfl_sync(0xffffffffu, vt, t);
        if (lane == t) v = vt;
        if (lane > t && lane < kb) v = fmaf(-F[(k0 + t) * ld + k0 + lane], yt, v);
      }
      if (lane < kb) y[k0 + lane] = v;
    }
    __syncthreads();
    for (int r = k0 + kb + threadIdx.x; r < m; r += kThreads) {
      float s = y[r];
      for (int t = 0; t < kb; ++t) s = fmaf(-F[(k0 + t) * ld + r], y[k0 + t], s);
      y[r] = s;
    }
    __syncthreads();
  }
  for (int k1 = m; k1 > 0; k1 -= 32) {
    const int k0 = max(0, k1 - 32);
    const int kb = k1 - k0;
    if (threadIdx.x < 32) {
      float v = (lane < kb) ? y[k0 + lane] : 0.0f;
      for (int t = kb - 1; t >= 0; --t) {
        const float yt = __shfl_sync(0xffffffffu, v, t);
        if (lane < t) v = fmaf(-F[(k0 + t) * ld + k0 + lane], yt, v);
      }
      if (lane < kb) y[k0 + lane] = v;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < k0; r += kThreads) {
      float s = y[r];
      for (int t = 0; t < kb; ++t) s = fmaf(-F[(k0 + t) * ld + r], y[k0 + t], s);
      y[r] = s;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Double-float residuals against the stored planes
// ---------------------------------------------------------------------------
__device__ __forceinline__ df2 warp_sum_df(df2 a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    df2 b = mkdf(__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o));
    a = df_add(a, b);
  }
  return a;
}

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
// Each warp takes two rows at a time and issues all loads of a 256-column chunk
// before accumulating, to keep enough bytes in flight.
__device__ void residual_rows(const float* __restrict__ Ah, const float* __restrict__ Al, int m,
                              const float* xh, const float* xl, const double* b, double* r) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j0 = 2 * warp; j0 < m; j0 += 2 * kWarps) {
    const bool two = j0 + 1 < m;
    ResAcc acc0, acc1;
    resacc_init(acc0);
    resacc_init(acc1);
    for (int c0 = 0; c0 < m; c0 += 256) {
      float h0[8], l0[8], h1[8], l1[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int c = c0 + lane + 32 * q;
        const bool ok = c < m;
        h0[q] = ok ? __ldg(Ah + j0 * m + c) : 0.0f;
        l0[q] = ok ? __ldg(Al + j0 * m + c) : 0.0f;
        h1[q] = (ok && two) ? __ldg(Ah + (j0 + 1) * m + c) : 0.0f;
        l1[q] = (ok && two) ? __ldg(Al + (j0 + 1) * m + c) : 0.0f;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int c = c0 + lane + 32 * q;
        if (c < m) {
          resacc_add(acc0, h0[q], l0[q], xh[c], xl[c]);
          resacc_add(acc1, h1[q], l1[q], xh[c], xl[c]);
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

// r_i = g_i - sum_j M_ji x_j for all columns i.  Warps own 32-column blocks and
// a share of the rows; partial sums meet in `part` ([kParts][m] accumulators).
constexpr int kParts = 4;
__host__ __device__ __forceinline__ int parts_for(int m) {
  const int ncb = (m + 31) >> 5;
  const int q = kWarps / ncb;
  return q < 1 ? 1 : (q > kParts ? kParts : q);
}
// Entries of `part` needed by any m <= mv (nparts(m) * m is at most 512 when
// nparts(m) > 1).
__host__ __device__ __forceinline__ int parts_entries(int mv) {
  const int a = 4 * mv < 512 ? 4 * mv : 512;
  const int b = parts_for(mv) * mv;
  return a > b ? a : b;
}
__device__ void residual_cols(const float* __restrict__ Ah, const float* __restrict__ Al, int m,
                              const float* xh, const float* xl, const double* g, double* r,
                              float4* part) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ncb = (m + 31) >> 5;
  const int nparts = parts_for(m);
  for (int task = warp; task < ncb * nparts; task += kWarps) {
    const int cb = task % ncb, pt = task / ncb;
    const int c = cb * 32 + lane;
    const int j0 = (int)((int64_t)m * pt / nparts), j1 = (int)((int64_t)m * (pt + 1) / nparts);
    ResAcc acc;
    resacc_init(acc);
    if (c < m) {
      for (int jb = j0; jb < j1; jb += 8) {
        float h[8], l[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int j = jb + q;
          h[q] = (j < j1) ? __ldg(Ah + j * m + c) : 0.0f;
          l[q] = (j < j1) ? __ldg(Al + j * m + c) : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (jb + q < j1) resacc_add(acc, h[q], l[q], xh[jb + q], xl[jb + q]);
      }
      part[pt * m + c] = make_float4(acc.s1, acc.s2.hi, acc.s2.lo, acc.s3);
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < m; c += kThreads) {
    ResAcc acc;
    resacc_init(acc);
    for (int pt = 0; pt < nparts; ++pt) {
      const float4 q = part[pt * m + c];
      ResAcc b;
      b.s1 = q.x;
      b.s2 = mkdf(q.y, q.z);
      b.s3 = q.w;
      resacc_merge(acc, b);
    }
    r[c] = resacc_sub_from(g[c], acc);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// The kernel
// ---------------------------------------------------------------------------
template <bool SMEM>
__global__ void __launch_bounds__(kThreads, 1) k_solve_mixed(SolveArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const Batch& bt = a.bt;
  const int b = bt.order[blockIdx.x];
  const int n = airfoil_n(bt, b);
  const int m = n + 1;
  if (a.info[b] != 0) return;
  // each airfoil is taken by exactly one of the two variants
  if (SMEM != (m <= kSmemM)) return;
  if (n > bt.n_max) {
    if (threadIdx.x == 0) a.info[b] = PANEL_INFO_TOO_LARGE;
    return;
  }
  // shared layout: vectors first, the factor (SMEM) last
  double* x = reinterpret_cast<double*>(smraw);   // m
  double* r = x + bt.n_max + 1;                    // m
  double* bb = r + bt.n_max + 1;                   // m (rhs of this system)
  float* y = reinterpret_cast<float*>(bb + bt.n_max + 1);  // m
  float* xh = y + bt.n_max + 1;                    // m
  float* xl = xh + bt.n_max + 1;                   // m
  int* ipiv = reinterpret_cast<int*>(xl + bt.n_max + 1);   // m
  int* perm = ipiv + bt.n_max + 1;                 // m
  float4* part = reinterpret_cast<float4*>(
      (reinterpret_cast<uintptr_t>(perm + bt.n_max + 1) + 15) & ~(uintptr_t)15);
  double* red = reinterpret_cast<double*>(part + parts_entries(bt.n_max + 1));  // 32
  float* prow = reinterpret_cast<float*>(red + 32);  // kNB
  float* krow = prow + kNB;                          // kNB
  float* cand_v = krow + kNB;                        // kWarps
  int* cand_i = reinterpret_cast<int*>(cand_v + kWarps);  // kWarps
  float* Fs = reinterpret_cast<float*>(cand_i + kWarps);

  const int64_t moff = bt.mat_off[b];
  const float* Ah = a.A_hi + moff;
  const float* Al = a.A_lo + moff;
  const int ld = SMEM ? (m | 1) : m;
  float* F = SMEM ? Fs : (a.LU + moff);
  int32_t* gpiv = a.piv + vec_off(bt, b);

  // border scale s = mean |A_jj| over the influence block (from the hi plane)
  double sdiag = 0.0;
  for (int j = threadIdx.x; j < n; j += kThreads) sdiag += fabs((double)Ah[j * m + j]);
  const double s = block_sum(sdiag, red) / n;
  const float sf = (float)s;

  if (!a.trans) {
    // load the hi plane, rescale the border, factor
    {
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      for (int rr = warp; rr < m; rr += kWarps)
        for (int c0 = 0; c0 < m; c0 += 256) {
          float v[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int cc = c0 + lane + 32 * q;
            v[q] = cc < m ? Ah[rr * m + cc] : 0.0f;
          }
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int cc = c0 + lane + 32 * q;
            if (cc < m) F[rr * ld + cc] = ((cc == n && rr < n) || rr == n) ? v[q] * sf : v[q];
          }
        }
    }
    __syncthreads();
    const int st = SMEM ? lu_rowpanel(F, ld, m, ipiv, prow, krow, cand_v, cand_i)
                        : lu_blocked(F, ld, m, ipiv);
    if (st != 0) {
      if (threadIdx.x == 0) {
        a.info[b] = st;
        if (a.iters) a.iters[b] = 0;
      }
      return;
    }
    for (int k = threadIdx.x; k < m; k += kThreads) gpiv[k] = ipiv[k];
    if (SMEM && a.LU) {
      float* G = a.LU + moff;
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      for (int rr = warp; rr < m; rr += kWarps)
        for (int cc = lane; cc < m; cc += 32) G[rr * m + cc] = F[rr * ld + cc];
    }
    for (int k = threadIdx.x; k < m; k += kThreads) bb[k] = a.rhs[vec_off(bt, b) + k];
  } else {
    // reuse the stored factor
    if (SMEM) {
      const float* G = a.LU + moff;
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      for (int rr = warp; rr < m; rr += kWarps)
        for (int c0 = 0; c0 < m; c0 += 256) {
          float v[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int cc = c0 + lane + 32 * q;
            v[q] = cc < m ? G[rr * m + cc] : 0.0f;
          }
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int cc = c0 + lane + 32 * q;
            if (cc < m) F[rr * ld + cc] = v[q];
          }
        }
    }
    for (int k = threadIdx.x; k < m; k += kThreads) ipiv[k] = gpiv[k];
    // g = dCl/du: 2 |h_k| / (v c) for the strengths, 0 for C
    const double* nd = bt.nodes + 2 * bt.node_off[b];
    const double v = a.vinf ? a.vinf[b] : 1.0, c = a.chord ? a.chord[b] : 1.0;
    for (int k = threadIdx.x; k < m; k += kThreads) {
      if (k < n) {
        const int k1 = (k + 1 == n) ? 0 : k + 1;
        const double hx = nd[2 * k1] - nd[2 * k], hy = nd[2 * k1 + 1] - nd[2 * k + 1];
        bb[k] = 2.0 * sqrt(hx * hx + hy * hy) / (v * c);
      } else {
        bb[k] = 0.0;
      }
    }
  }
  // row permutation of the factor: P y = y[perm]
  if (threadIdx.x == 0) {
    for (int k = 0; k < m; ++k) perm[k] = k;
    for (int k = 0; k < m; ++k) {
      const int p = ipiv[k];
      const int t = perm[k];
      perm[k] = perm[p];
      perm[p] = t;
    }
  }
  for (int k = threadIdx.x; k < m; k += kThreads) {
    x[k] = 0.0;
    r[k] = bb[k];
  }
  __syncthreads();

  int it = 0;
  bool conv = false;
  for (;; ++it) {
    if (!a.trans) {
      // y = P S_r r;  solve;  dx = S_c y
      for (int k = threadIdx.x; k < m; k += kThreads) {
        const int src = perm[k];
        const double v = (src == n) ? r[src] * s : r[src];
        y[k] = (float)v;
      }
      __syncthreads();
      lu_apply_inverse(F, ld, m, y);
    } else {
      // z = Mt^{-T} S_c r;  lambda update = S_r P^T z
      for (int k = threadIdx.x; k < m; k += kThreads) y[k] = (float)((k == n) ? r[k] * s : r[k]);
      __syncthreads();
      lu_apply_inverse_transposed(F, ld, m, y);
    }
    double dmax = 0.0, xmax = 0.0;
    if (!a.trans) {
      for (int k = threadIdx.x; k < m; k += kThreads) {
        const double d = (k == n) ? (double)y[k] * s : (double)y[k];
        x[k] += d;
        dmax = fmax(dmax, fabs(d));
        xmax = fmax(xmax, fabs(x[k]));
      }
    } else {
      // y holds the permuted solution: lambda[perm[k]] += y[k] (S_r on row n)
      for (int k = threadIdx.x; k < m; k += kThreads) {
        const int dst = perm[k];
        const double d = (dst == n) ? (double)y[k] * s : (double)y[k];
        x[dst] += d;
        dmax = fmax(dmax, fabs(d));
      }
      __syncthreads();
      for (int k = threadIdx.x; k < m; k += kThreads) xmax = fmax(xmax, fabs(x[k]));
    }
    dmax = block_absmax_d(dmax, red);
    xmax = block_absmax_d(xmax, red);
    if (it >= 1 && dmax <= a.tol * xmax) { conv = true; break; }
    if (it >= a.max_iter) break;
    // residual against the double-float matrix
    for (int k = threadIdx.x; k < m; k += kThreads) {
      const df2 d = df_from_double(x[k]);
      xh[k] = d.hi;
      xl[k] = d.lo;
    }
    __syncthreads();
    if (!a.trans) residual_rows(Ah, Al, m, xh, xl, bb, r);
    else residual_cols(Ah, Al, m, xh, xl, bb, r, part);
    __syncthreads();
  }
  double* out = a.out + vec_off(bt, b);
  for (int k = threadIdx.x; k < m; k += kThreads) out[k] = x[k];
  if (threadIdx.x == 0) {
    if (a.iters && !a.trans) a.iters[b] = it;
    if (!conv) a.info[b] = PANEL_INFO_NOCONV;
  }
}

size_t solve_mixed_smem(int n_max, bool smem_factor, int m_factor) {
  const size_t mv = (size_t)n_max + 1;
  size_t bytes = mv * 8 * 3 + mv * 4 * 3 + mv * 4 * 2 + 16 + (size_t)parts_entries((int)mv) * 16 +
                 32 * 8 + 2 * kNB * 4 + 2 * kWarps * 4;
  bytes = (bytes + 15) & ~(size_t)15;
  if (smem_factor) bytes += (size_t)m_factor * (size_t)(m_factor | 1) * 4;
  return bytes;
}

cudaError_t launch_solve_mixed(const Batch& bt, const float* A_hi, const float* A_lo, float* LU,
                               int32_t* piv, const double* rhs, const double* vinf,
                               const double* chord, double* out, int max_iter, double tol,
                               int32_t* info, int32_t* iters, int trans, cudaStream_t s) {
  SolveArgs a;
  a.bt = bt;
  a.A_hi = A_hi;
  a.A_lo = A_lo;
  a.LU = LU;
  a.piv = piv;
  a.rhs = rhs;
  a.vinf = vinf;
  a.chord = chord;
  a.out = out;
  a.max_iter = max_iter;
  a.tol = tol;
  a.info = info;
  a.iters = iters;
  a.trans = trans;
  const int mmax = bt.n_max + 1;
  if (mmax > kSmemM) {  // airfoils with m > kSmemM: factor in global memory
    const size_t smem = solve_mixed_smem(bt.n_max, false, 0);
    cudaError_t e = cudaFuncSetAttribute(k_solve_mixed<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_solve_mixed<false><<<bt.B, kThreads, smem, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // airfoils with m <= kSmemM: factor in shared memory
  Batch bs = bt;
  bs.n_max = min(bt.n_max, kSmemM - 1);
  a.bt = bs;
  const size_t smem = solve_mixed_smem(bs.n_max, true, bs.n_max + 1);
  cudaError_t e = cudaFuncSetAttribute(k_solve_mixed<true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_solve_mixed<true><<<bt.B, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace panel
