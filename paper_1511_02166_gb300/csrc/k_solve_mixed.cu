// k_solve_mixed.cu -- FP32 LU with partial pivoting + double-float iterative
// refinement for the bordered panel system (the mixed-precision path).
//
// The factor is of the rescaled matrix Mt = S_r M S_c, where S_c multiplies the
// C column and S_r the Kutta row by s = mean |A_jj| (the self-influence scale);
// this balances the border against the influence coefficients and lowers the
// condition number seen by the FP32 factor.  Refinement (Wilkinson/Moler):
//   x_0 = solve(b);  r_k = b - M x_k  with products and sums exact to ~2^-70
//   against the stored planes A_hi + A_lo;  x_{k+1} = x_k + solve(r_k), until
//   |dx|_inf <= tol |x|_inf, or until the contraction of the last two
//   corrections predicts the next one below that.  The transposed system
//   M^T lambda = g (g = dCl/du) is refined in the same kernel.
//
// The FP32 factor depends on the size m = n + 1 and the launch's choices:
//   PANEL_INVERSE, m <= kGjM (288)   explicit inverse by blocked Gauss-Jordan
//                                    (k_gj_mixed.cu); a correction is one GEMV;
//   m <= kSmemLuM (224)              k_lu_smem below: LU with the whole matrix in
//                                    shared memory (by size, PANEL_TUNE_LU(2)),
//                                    or k_lu_global (PANEL_TUNE_LU(1));
//   m <= kLargeM (640)               k_lu_global below: one block per airfoil,
//                                    blocked right-looking LU, the trailing
//                                    matrix in the caller's LU buffer through L2;
//   m > kLargeM                      the step-synchronous blocked LU
//                                    (k_lu_large.cu, k_update_tc.cu).
// All LU variants pivot inside the current diagonal block and replace the
// 32 x 32 diagonal blocks of L and U by their inverses, so that the triangular
// solves below are sequences of matrix-vector products.  The LU buffer
// therefore holds a library-internal layout (an inverse, or an LU with
// inverted diagonal blocks: row-major up to kLargeM, above it the tiled layout
// of the blocked factor, tl_layout.cuh).
//  k_ir_mixed  one block per airfoil: the corrections with the stored factor
//    (read through L1/L2) and the refinement residuals (for m <= kFuseM one
//    pass over the matrix for both systems, else one over the rows for M u and
//    one over the columns for M^T lambda).
#include <type_traits>

#include "df.cuh"
#include "tl_layout.cuh"

namespace panel {

// ---------------------------------------------------------------------------
// LU with partial pivoting of one kb x kb diagonal block (kb <= 32) by one
// warp, register-resident: lane r holds row r (x = its NB columns); rows keep
// their lanes and `pos` tracks their current position, so an exchange of
// positions q and p is bookkeeping plus one ipiv entry.  The pivot of column
// q is the largest |x_q| among the rows not yet pivotal (the lowest position
// among equal maxima).  The loop is not unrolled (the single warp would run
// thousands of straight-line instructions once each, fetched from beyond the
// instruction cache); instead the columns rotate through the registers: at
// step q the current column is x[0], the later ones x[1 .. NB-1-q], and the
// finished entries of the earlier columns x[NB-q ..]; each step retires x[0]
// (the multiplier, or the U entry of a pivotal row) to x[NB-1] and shifts the
// rest down, so every register index is a constant and after NB steps the
// columns are back in order.  The reciprocal of the pivot is the correctly
// rounded one (the same value as 1 / p).  ipiv[q] receives base + the position of column
// q's pivot row.  On return `fz` is 0, or q + 1 for the first exactly zero (or
// NaN) pivot column q, after which the block is left as it stands.
// ---------------------------------------------------------------------------
template <int NB>
__device__ __forceinline__ void warp_block_lu(float (&x)[NB], int& pos, bool& done, int& fz,
                                              int kb, int* ipiv, int base) {
  const int lane = threadIdx.x & 31;
  // every step is straight-line code: the warp-uniform conditions (the step is
  // inside the block, no zero pivot so far) act as predicates, not branches
#pragma unroll 1
  for (int q = 0; q < NB; ++q) {
    const bool act = q < kb && fz == 0;
    const float v = (act && !done) ? fabsf(x[0]) : -1.0f;
    const unsigned key = (v >= 0.0f) ? __float_as_uint(v) + 1u : 0u;  // |x| bits are monotone
    const unsigned mx = __reduce_max_sync(0xffffffffu, key);
    const bool ok = act && mx > 1u;  // a nonzero pivot (mx <= 1: zero or NaN column)
    if (act && !ok) fz = q + 1;
    // the lowest current position among the maxima
    const unsigned pm = __reduce_min_sync(0xffffffffu, (ok && key == mx) ? (unsigned)pos : 0xffu);
    const int pl = (__ffs(__ballot_sync(0xffffffffu, ok && key == mx && pos == (int)pm)) - 1) & 31;
    const int ql = __ffs(__ballot_sync(0xffffffffu, ok && pos == q)) - 1;  // the row now at q
    if (ok && lane == 0) ipiv[q] = base + (int)pm;
    if (ok && lane == ql) pos = (int)pm;
    if (ok && lane == pl) {
      pos = q;
      done = true;
    }
    const float inv = __frcp_rn(__shfl_sync(0xffffffffu, x[0], pl));
    const float l = x[0] * inv;
    const bool elim = ok && !done;
#pragma unroll
    for (int t = 1; t < NB; ++t) {
      const float uc = __shfl_sync(0xffffffffu, x[t], pl);
      x[t] = (elim && t < NB - q) ? fmaf(-l, uc, x[t]) : x[t];  // a later column
    }
    const float out = elim ? l : x[0];
#pragma unroll
    for (int t = 0; t < NB - 1; ++t) x[t] = x[t + 1];
    x[NB - 1] = out;
  }
}

// ---------------------------------------------------------------------------
// The LU kernel, factor in global memory (kSmemLuM < m <= kLargeM, or every
// m <= kLargeM with PANEL_TUNE_LU(1)): blocked right-looking
// with the current panel of NB columns staged in shared memory (rows spread
// over the threads), the row exchanges, U12 and the rank-NB update applied to
// the factor in the caller's LU buffer through L2.  Shared memory stays small
// (the panel plus a 128-column slab of U12), so several airfoils share an SM
// and hide each other's latencies.
// ---------------------------------------------------------------------------
// A22 -= L21 U12 over the columns [cc, cc + 32 J) of the staged U12 slab: warp
// w takes the 8-row tiles w, w + 8, ...; lane l the columns cc + l + 32 j.
template <int J, int LDP, int CW>
__device__ __forceinline__ void update_tiles(float* __restrict__ F, const float* __restrict__ P,
                                             const float* __restrict__ U, int m, int k0, int k1,
                                             int kb, int cc, int nrt) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int rt = warp; rt < nrt; rt += kWarps) {
    const int r0 = k1 + 8 * rt;
    float acc[8][J];
#pragma unroll
    for (int aa = 0; aa < 8; ++aa)
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int r = r0 + aa, c = cc + lane + 32 * j;
        acc[aa][j] = (r < m && c < m) ? F[r * m + c] : 0.0f;
      }
#pragma unroll 4
    for (int q = 0; q < kb; ++q) {
      float lv[8], uv[J];
#pragma unroll
      for (int aa = 0; aa < 8; ++aa) lv[aa] = (r0 + aa < m) ? P[(r0 + aa - k0) * LDP + q] : 0.0f;
#pragma unroll
      for (int j = 0; j < J; ++j) uv[j] = U[q * CW + lane + 32 * j];
#pragma unroll
      for (int aa = 0; aa < 8; ++aa)
#pragma unroll
        for (int j = 0; j < J; ++j) acc[aa][j] = fmaf(-lv[aa], uv[j], acc[aa][j]);
    }
#pragma unroll
    for (int aa = 0; aa < 8; ++aa)
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int r = r0 + aa, c = cc + lane + 32 * j;
        if (r < m && c < m) F[r * m + c] = acc[aa][j];
      }
  }
}

template <int NB>
__global__ void __launch_bounds__(kThreads, 3) k_lu_global(SolveArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int LDP = NB + 1;
  constexpr int CW = 128;  // GEMM column slab
  const Batch& bt = a.bt;
  const int b = bt.order[blockIdx.x];
  const int n = airfoil_n(bt, b);
  const int m = n + 1;
  if (a.info[b] != 0) return;
  if (m <= kGjM && a.inverse) return;  // taken by k_gj_mixed
  if (n > a.n_cap) {
    if (threadIdx.x == 0) a.info[b] = PANEL_INFO_TOO_LARGE;
    return;
  }
  if (m > kLargeM) return;  // taken by the blocked factor (k_lu_large.cu)
  if (m <= kSmemLuM && a.lu_kind != 1) return;  // taken by k_lu_smem
  const int mv = bt.n_max + 1;
  float* P = reinterpret_cast<float*>(smraw);           // mv x LDP panel
  float* U = P + mv * LDP;                              // NB x CW slab of U12
  double* red = reinterpret_cast<double*>(
      (reinterpret_cast<uintptr_t>(U + NB * CW) + 15) & ~(uintptr_t)15);  // 32
  unsigned long long* cand = reinterpret_cast<unsigned long long*>(red + 32);  // kWarps
  int* ipiv = reinterpret_cast<int*>(cand + kWarps);    // mv
  int* bperm = ipiv + mv;  // NB: final row q of the block = row k0 + bperm[q] before its exchanges

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
    // ---- factor the panel: LU of the diagonal block by warp 0 (pivot search
    // inside the block's rows, lane = column), then L21 = A21 U11^{-1} with a
    // thread per row below the block ----
    if (warp == 0) {
      // register-resident: lane r holds row r of the diagonal block (x[t] =
      // column t); rows keep their lanes and pos tracks their current position,
      // so an exchange of positions q and p is bookkeeping plus one ipiv entry
      float x[NB];
#pragma unroll
      for (int t = 0; t < NB; ++t) x[t] = (lane < kb && t < kb) ? P[lane * LDP + t] : 0.0f;
      int pos = lane;
      bool done = lane >= kb;  // already a pivot row (or outside the block)
      int fz = 0;
      warp_block_lu<NB>(x, pos, done, fz, kb, ipiv + k0, k0);
      __syncwarp();
      if (lane < kb) {
#pragma unroll
        for (int t = 0; t < NB; ++t)
          if (t < kb) P[pos * LDP + t] = x[t];
        bperm[pos] = lane;
      }
      __syncwarp();
      if (lane == 0) cand[0] = (unsigned long long)fz;
      if (lane < kb && fz == 0) red[lane] = (double)(1.0f / P[lane * LDP + lane]);
    }
    __syncthreads();
    if (cand[0] != 0ull) {
      if (tid == 0) {
        a.info[b] = k0 + (int)cand[0];
        if (a.iters) a.iters[b] = 0;
      }
      return;
    }
    if (rows > kb) {  // then kb == NB
      for (int r = kb + tid; r < rows; r += kThreads) {
        float x[NB];
#pragma unroll
        for (int t = 0; t < NB; ++t) x[t] = P[r * LDP + t];
        // right-looking: once x_q is final it goes into every later column
        // (the same terms in the same order as the row's dot products)
#pragma unroll
        for (int q = 0; q < NB; ++q) {
          x[q] *= (float)red[q];
#pragma unroll
          for (int t = q + 1; t < NB; ++t) x[t] = fmaf(-x[q], P[q * LDP + t], x[t]);
        }
#pragma unroll
        for (int t = 0; t < NB; ++t) P[r * LDP + t] = x[t];
      }
      __syncthreads();
    }
    // ---- write the panel back, exchange rows outside it ----
    for (int r = warp; r < rows; r += kWarps)
      if (lane < kb) F[(k0 + r) * m + k0 + lane] = P[r * LDP + lane];
    // the exchanges of this block's rows: composed into bperm, all loads of a
    // column in flight at once; the columns right of the panel read their rows
    // through bperm in the U12 solve below instead
    for (int c = tid; c < k0; c += kThreads) {
      float v[NB];
#pragma unroll
      for (int q = 0; q < NB; ++q) v[q] = (q < kb) ? F[(k0 + bperm[q]) * m + c] : 0.0f;
#pragma unroll
      for (int q = 0; q < NB; ++q)
        if (q < kb) F[(k0 + q) * m + c] = v[q];
    }
    __syncthreads();
    const int k1 = k0 + kb;
    if (k1 >= m) break;
    // ---- U12 = L11^{-1} A12, a column per lane, unrolled forward substitution
    // (here kb == NB: a panel with columns right of it is full) ----
    for (int cb = k1 + 32 * warp; cb < m; cb += kThreads) {
      const int c = cb + lane;
      const bool ok = c < m;
      float col[NB];
#pragma unroll
      for (int t = 0; t < NB; ++t) col[t] = ok ? F[(k0 + bperm[t]) * m + c] : 0.0f;
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        const float x = col[q];
        if (ok) F[(k0 + q) * m + c] = x;
#pragma unroll
        for (int t = q + 1; t < NB; ++t) col[t] = fmaf(-P[t * LDP + q], x, col[t]);
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
      // register tiles 8 rows x 32 J columns, J = 1..4 by the width of the slab
      const int J = min(CW / 32, (m - cc + 31) >> 5);
      if (J == 4)
        update_tiles<4, LDP, CW>(F, P, U, m, k0, k1, kb, cc, nrt);
      else if (J == 3)
        update_tiles<3, LDP, CW>(F, P, U, m, k0, k1, kb, cc, nrt);
      else if (J == 2)
        update_tiles<2, LDP, CW>(F, P, U, m, k0, k1, kb, cc, nrt);
      else
        update_tiles<1, LDP, CW>(F, P, U, m, k0, k1, kb, cc, nrt);
      __syncthreads();
    }
  }
  // the diagonal blocks inverted in shared memory (the panel and slab buffers
  // are free now: a 32 x LDP slot per warp), then written back
  {
    float* S = P + warp * (NB * LDP);
    const int nb = (m + NB - 1) / NB;
    for (int d = warp; d < nb; d += kWarps) {
      const int d0 = NB * d, kbd = min(NB, m - d0);
      for (int r = 0; r < kbd; ++r)
        if (lane < kbd) S[r * LDP + lane] = F[(d0 + r) * m + d0 + lane];
      __syncwarp();
      invert_block(S, LDP, kbd);
      for (int r = 0; r < kbd; ++r)
        if (lane < kbd) F[(d0 + r) * m + d0 + lane] = S[r * LDP + lane];
      __syncwarp();
    }
  }
  __syncthreads();
  int32_t* gpiv = a.piv + vec_off(bt, b);
  for (int k = tid; k < m; k += kThreads) gpiv[k] = ipiv[k];
}

// ---------------------------------------------------------------------------
// The LU kernel with the whole matrix in shared memory (3 <= m <= kSmemLuM):
// one block of 512 threads per airfoil and per SM.  The algorithm and the
// factor's layout are those of k_lu_global (32-column panels, the pivot search
// inside the diagonal block, register LU of the diagonal block by one warp, L21
// by a thread per row, the block's exchanges composed, U12 by a thread per
// column, the rank-32 update in 8 x 32J register tiles accumulated in the same
// order, the 32 x 32 diagonal blocks inverted at the end), so the two kernels
// store the same factor bit for bit.  Here every step works on the scaled
// matrix staged once in shared memory (odd row stride: conflict-free columns)
// and the factor goes to the caller's buffer once: one read of the hi plane and
// one write of the factor per airfoil.  Since one airfoil has the SM to itself,
// the steps are arranged to keep its warps busy:
//   A  L21 (threads 0..255, one row each, also kept transposed in LT so that the
//      update reads eight rows' multipliers with two broadcast vector loads)
//      and U12 (threads 256..511, one column each) at once, then the exchanges
//      on the columns left of the panel;
//   B  the update of the next panel's 32 columns;
//   C  warp 0 factors the next diagonal block (look-ahead) while warps 1..15
//      update the remaining columns.
// ---------------------------------------------------------------------------
constexpr int kSmemLuThreads = 512;
constexpr int kSmemLuWarps = kSmemLuThreads / 32;
static_assert(kSmemLuM <= 256, "k_lu_smem moves rows of at most 8 x 32 columns");
static_assert(kSmemLuM - 32 <= kSmemLuThreads / 2, "a thread per row / column in phase A");

// A22 -= L21 U12 on rows [r0, r0 + 8) x columns cc + lane + 32 j (j < J): the
// multipliers of the 8 rows from LT (panel column q at LT[q ldt + r - k1]),
// U12 from the matrix rows k0..k0 + kb.
template <int J>
__device__ __forceinline__ void smem_update_tile(float* __restrict__ F, int ld,
                                                 const float* __restrict__ LT, int ldt, int m,
                                                 int k0, int k1, int kb, int r0, int cc) {
  const int lane = threadIdx.x & 31;
  float acc[8][J];
#pragma unroll
  for (int aa = 0; aa < 8; ++aa)
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int r = r0 + aa, c = cc + lane + 32 * j;
      acc[aa][j] = (r < m && c < m) ? F[r * ld + c] : 0.0f;
    }
  const float* lt = LT + (r0 - k1);
#pragma unroll 4
  for (int q = 0; q < kb; ++q) {
    const float4 la = *reinterpret_cast<const float4*>(lt + q * ldt);
    const float4 lb = *reinterpret_cast<const float4*>(lt + q * ldt + 4);
    const float lv[8] = {la.x, la.y, la.z, la.w, lb.x, lb.y, lb.z, lb.w};
    float uv[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int c = cc + lane + 32 * j;
      uv[j] = (c < m) ? F[(k0 + q) * ld + c] : 0.0f;
    }
#pragma unroll
    for (int aa = 0; aa < 8; ++aa)
#pragma unroll
      for (int j = 0; j < J; ++j) acc[aa][j] = fmaf(-lv[aa], uv[j], acc[aa][j]);
  }
#pragma unroll
  for (int aa = 0; aa < 8; ++aa)
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int r = r0 + aa, c = cc + lane + 32 * j;
      if (r < m && c < m) F[r * ld + c] = acc[aa][j];
    }
}

// Update tasks of 8 rows x 32 J columns over the columns [c0, c1) of the rows
// [k1, m), distributed over the warps w0 .. kSmemLuWarps - 1.
__device__ __forceinline__ void smem_update(float* F, int ld, const float* LT, int ldt, int m,
                                            int k0, int k1, int kb, int c0, int c1, int w0,
                                            int cw) {
  const int warp = threadIdx.x >> 5;
  if (warp < w0 || c1 <= c0) return;
  const int nrt = (m - k1 + 7) >> 3, ncs = (c1 - c0 + cw - 1) / cw;
  for (int task = warp - w0; task < nrt * ncs; task += kSmemLuWarps - w0) {
    const int r0 = k1 + 8 * (task / ncs), cc = c0 + cw * (task % ncs);
    const int J = min(cw / 32, (min(c1, m) - cc + 31) >> 5);
    if (J >= 4)
      smem_update_tile<4>(F, ld, LT, ldt, m, k0, k1, kb, r0, cc);
    else if (J == 3)
      smem_update_tile<3>(F, ld, LT, ldt, m, k0, k1, kb, r0, cc);
    else if (J == 2)
      smem_update_tile<2>(F, ld, LT, ldt, m, k0, k1, kb, r0, cc);
    else
      smem_update_tile<1>(F, ld, LT, ldt, m, k0, k1, kb, r0, cc);
  }
}

// LU of the diagonal block at (k0, k0), kb x kb, by the calling warp: the block
// rows in their final order, the pivots in ipiv[k0 ..], the composed exchanges
// in bperm, 1 / U_tt in red, and in *fz 0 or the first zero pivot column + 1.
__device__ __forceinline__ void smem_diag_lu(float* F, int ld, int k0, int kb, int* ipiv,
                                             int* bperm, double* red,
                                             unsigned long long* fzp) {
  constexpr int NB = 32;
  const int lane = threadIdx.x & 31;
  float* P = F + k0 * ld + k0;
  float x[NB];
#pragma unroll
  for (int t = 0; t < NB; ++t) x[t] = (lane < kb && t < kb) ? P[lane * ld + t] : 0.0f;
  int pos = lane;
  bool done = lane >= kb;
  int fz = 0;
  warp_block_lu<NB>(x, pos, done, fz, kb, ipiv + k0, k0);
  __syncwarp();
  if (lane < kb) {
#pragma unroll
    for (int t = 0; t < NB; ++t)
      if (t < kb) P[pos * ld + t] = x[t];
    bperm[pos] = lane;
  }
  __syncwarp();
  if (lane == 0) *fzp = (unsigned long long)fz;
  if (lane < kb && fz == 0) red[lane] = (double)(1.0f / P[lane * ld + lane]);
}

__global__ void __launch_bounds__(kSmemLuThreads, 1) k_lu_smem(SolveArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int NB = 32;
  const Batch& bt = a.bt;
  const int b = bt.order[blockIdx.x];
  const int n = airfoil_n(bt, b);
  const int m = n + 1;
  if (a.info[b] != 0) return;
  if (m <= kGjM && a.inverse) return;  // taken by k_gj_mixed
  if (n > a.n_cap) {
    if (threadIdx.x == 0) a.info[b] = PANEL_INFO_TOO_LARGE;
    return;
  }
  if (m > kSmemLuM || a.lu_kind == 1) return;  // taken by k_lu_global or the blocked factor
  const int ld = m | 1;
  const int mv = bt.n_max + 1;
  const int ldv = mv | 1;
  const int ldt = (mv + 7) & ~7;
  float* F = reinterpret_cast<float*>(smraw);  // m x ld
  float* LT = reinterpret_cast<float*>(
      (reinterpret_cast<uintptr_t>(F + (size_t)mv * ldv) + 15) & ~(uintptr_t)15);  // NB x ldt
  double* red = reinterpret_cast<double*>(LT + NB * ldt);                          // 32
  unsigned long long* cand = reinterpret_cast<unsigned long long*>(red + 32);      // 1
  int* ipiv = reinterpret_cast<int*>(cand + 2);                                    // mv
  int* bperm = ipiv + mv;                                                          // NB

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t moff = bt.mat_off[b];
  const float* Ah = a.A_hi + moff;
  // the hi plane in by asynchronous copies (every element of the thread in
  // flight at once; rows of stride m are only 4-byte aligned), a warp per row
  for (int rr = warp; rr < m; rr += kSmemLuWarps)
    for (int cc = lane; cc < m; cc += 32) {
      const unsigned dst = (unsigned)__cvta_generic_to_shared(F + rr * ld + cc);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(Ah + rr * m + cc)
                   : "memory");
    }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  const float sf = (float)border_scale(Ah, n, m, red);
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  // the C column and the Kutta row scaled by sf
  for (int k = tid; k < m; k += kSmemLuThreads) {
    F[n * ld + k] *= sf;
    if (k < n) F[k * ld + n] *= sf;
  }
  __syncthreads();
  if (warp == 0) smem_diag_lu(F, ld, 0, min(NB, m), ipiv, bperm, red, cand);
  __syncthreads();

  for (int k0 = 0;; k0 += NB) {
    if (cand[0] != 0ull) {
      if (tid == 0) {
        a.info[b] = k0 + (int)cand[0];
        if (a.iters) a.iters[b] = 0;
      }
      return;
    }
    const int kb = min(NB, m - k0);
    const int k1 = k0 + kb;
    const float* P = F + k0 * ld + k0;
    // ---- A: L21 = A21 U11^{-1} (also into LT), then the exchanges on the
    // columns left of the panel (threads 0..255); U12 = L11^{-1} A12 with the
    // rows read through the exchanges (threads 256..511) ----
    if (tid < kSmemLuThreads / 2) {
      const int r = k1 + tid;
      if (r < m) {  // then kb == NB
        float x[NB];
#pragma unroll
        for (int t = 0; t < NB; ++t) x[t] = F[r * ld + k0 + t];
        // right-looking: once x_q is final it goes into every later column
        // (the same terms in the same order as the row's dot products)
#pragma unroll
        for (int q = 0; q < NB; ++q) {
          x[q] *= (float)red[q];
#pragma unroll
          for (int t = q + 1; t < NB; ++t) x[t] = fmaf(-x[q], P[q * ld + t], x[t]);
        }
#pragma unroll
        for (int t = 0; t < NB; ++t) {
          F[r * ld + k0 + t] = x[t];
          LT[t * ldt + tid] = x[t];
        }
      }
      for (int c = tid; c < k0; c += kSmemLuThreads / 2) {
        float v[NB];
#pragma unroll
        for (int q = 0; q < NB; ++q) v[q] = (q < kb) ? F[(k0 + bperm[q]) * ld + c] : 0.0f;
#pragma unroll
        for (int q = 0; q < NB; ++q)
          if (q < kb) F[(k0 + q) * ld + c] = v[q];
      }
    } else {
      const int c = k1 + tid - kSmemLuThreads / 2;
      if (c < m) {  // then kb == NB
        float col[NB];
#pragma unroll
        for (int t = 0; t < NB; ++t) col[t] = F[(k0 + bperm[t]) * ld + c];
#pragma unroll
        for (int q = 0; q < NB; ++q) {
          const float x = col[q];
          F[(k0 + q) * ld + c] = x;
#pragma unroll
          for (int t = q + 1; t < NB; ++t) col[t] = fmaf(-P[t * ld + q], x, col[t]);
        }
      }
    }
    __syncthreads();
    if (k1 >= m) break;
    const int kb2 = min(NB, m - k1);
    // ---- B: the next panel's columns [k1, k1 + kb2) ----
    smem_update(F, ld, LT, ldt, m, k0, k1, kb, k1, k1 + kb2, 0, 32);
    __syncthreads();
    // ---- C: the next diagonal block (warp 0) | the remaining columns ----
    if (warp == 0)
      smem_diag_lu(F, ld, k1, kb2, ipiv, bperm, red, cand);
    else
      smem_update(F, ld, LT, ldt, m, k0, k1, kb, k1 + kb2, m, 1, 128);
    __syncthreads();
  }
  // the 32 x 32 diagonal blocks inverted in place, a warp per triangle
  {
    const int nb = (m + NB - 1) / NB;
    for (int t = warp; t < 2 * nb; t += kSmemLuWarps) {
      const int d0 = NB * (t >> 1), kbd = min(NB, m - d0);
      if (t & 1)
        invert_upper(F + d0 * ld + d0, ld, kbd);
      else
        invert_lower_unit(F + d0 * ld + d0, ld, kbd);
    }
  }
  __syncthreads();
  float* G = a.LU + moff;
  for (int rr = warp; rr < m; rr += kSmemLuWarps)
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int cc = lane + 32 * u;
      if (cc < m) G[rr * m + cc] = F[rr * ld + cc];
    }
  int32_t* gpiv = a.piv + vec_off(bt, b);
  for (int k = tid; k < m; k += kSmemLuThreads) gpiv[k] = ipiv[k];
}

size_t lu_smem_smem(int n_max) {
  const size_t mv = (size_t)n_max + 1, ldv = mv | 1, ldt = (mv + 7) & ~(size_t)7;
  const size_t bytes = (mv * ldv * 4 + 15) & ~(size_t)15;
  return bytes + 32 * ldt * 4 + 32 * 8 + 16 + mv * 4 + 32 * 4;
}

template <int NB>
size_t lu_global_smem(int n_max) {
  const size_t mv = (size_t)n_max + 1;
  size_t bytes = mv * (NB + 1) * 4 + (size_t)NB * 128 * 4;
  bytes = (bytes + 15) & ~(size_t)15;
  return bytes + 32 * 8 + kWarps * 8 + mv * 4 + NB * 4;
}

// ---------------------------------------------------------------------------
// Triangular solves with the stored factor (global memory, the 32 x 32
// diagonal blocks inverted) on float vectors in shared memory: the forward
// system y <- U^{-1} L^{-1} y and the transposed system z <- L^{-T} U^{-T} z,
// one of them or both at once.  Both go over the 32-row groups of the factor
// top-down (L, U^T) and then bottom-up (U, L^T), two block barriers per group:
//   phase A  forward: t_i = y_i - (row i of L or U outside the group) . y, a
//            warp per row, lanes along the row (left-looking, coalesced);
//            transposed: the previous group's columns of U^T (rows of U), or
//            of L^T, applied to the rest of z, a thread per column
//            (right-looking, coalesced across the threads); the group's own
//            entries go to its 32-float scratch instead of z;
//   phase B  the group's diagonal block: y_i = sum X_iq t_q (a warp per row),
//            z_i = sum X_qi t_q (a warp per column).
// Solving both systems, every warp takes its share of both in each phase (the
// two share the barriers, and a warp done with its forward rows goes on to its
// transposed columns while others are still loading); each system's
// arithmetic is the same as when it is solved alone.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float sum8(const float (&a)[8]) {
  return ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
}

// One lane's shares of sum_{k in [k0, k1)} row[k] y[k] (k = lane + 32 t) for
// two rows r0 and r1 (r1 only if `two`) over the same columns, with eight
// independent partial sums per row, so that up to sixteen loads are in flight
// per lane (a long row is otherwise a chain of dependent round trips to L2);
// the last (< 256) columns take one masked pass.
__device__ __forceinline__ float2 row_dot2(const float* __restrict__ r0,
                                           const float* __restrict__ r1, bool two,
                                           const float* y, int k0, int k1, int lane) {
  float a[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  float b[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  int k = k0 + lane;
  for (; k + 7 * 32 < k1; k += 8 * 32) {
    float u[8], v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      u[t] = __ldg(r0 + k + 32 * t);
      v[t] = two ? __ldg(r1 + k + 32 * t) : 0.0f;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const float yy = y[k + 32 * t];
      a[t] = fmaf(u[t], yy, a[t]);
      b[t] = fmaf(v[t], yy, b[t]);
    }
  }
  if (k < k1) {
    float u[8], v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const bool ok = k + 32 * t < k1;
      u[t] = ok ? __ldg(r0 + k + 32 * t) : 0.0f;
      v[t] = (ok && two) ? __ldg(r1 + k + 32 * t) : 0.0f;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      if (k + 32 * t < k1) {
        const float yy = y[k + 32 * t];
        a[t] = fmaf(u[t], yy, a[t]);
        b[t] = fmaf(v[t], yy, b[t]);
      }
    }
  }
  return make_float2(sum8(a), sum8(b));
}

// The factor of an airfoil of at most kLargeM - 1 panels: row-major, ld m,
// groups of 32 rows from row 0.
struct RmFactor {
  const float* F;
  int m;
  __device__ int groups() const { return (m + 31) >> 5; }
  __device__ int k0(int d) const { return 32 * d; }
  __device__ int kb(int d) const { return min(32, m - 32 * d); }
  // lane shares of row i . y (and of row i1 . y if `two`) over the columns
  // before / after group d
  __device__ float2 dot_left(int i, int i1, bool two, int d, const float* y, int lane) const {
    return row_dot2(F + (int64_t)i * m, F + (int64_t)i1 * m, two, y, 0, 32 * d, lane);
  }
  __device__ float2 dot_right(int i, int i1, bool two, int d, const float* y, int lane) const {
    return row_dot2(F + (int64_t)i * m, F + (int64_t)i1 * m, two, y, 32 * d + kb(d), m, lane);
  }
  // row i's entries in the columns of group d
  __device__ const float* diag_row(int d, int i) const { return F + (int64_t)i * m + 32 * d; }
  // z_r -= sum_t M[k0 + t][r] z_{k0 + t} (group d's rows) for the columns r after
  // group d; those of group d + 1 go to nx.  Thread tid of nth.
  __device__ void update_right(int d, float* z, float* nx, int tid, int nth) const {
    const int k0 = 32 * d, kb = this->kb(d), c0 = k0 + kb;
    for (int r = c0 + tid; r < m; r += nth) {
      float acc = z[r];
#pragma unroll 8
      for (int t = 0; t < kb; ++t) acc = fmaf(-__ldg(F + (int64_t)(k0 + t) * m + r), z[k0 + t], acc);
      if (r < c0 + 32)
        nx[r - c0] = acc;
      else
        z[r] = acc;
    }
  }
  // the same for the columns before group d; those of group d - 1 go to nx
  __device__ void update_left(int d, float* z, float* nx, int tid, int nth) const {
    const int k0 = 32 * d, kb = this->kb(d);
    for (int r = tid; r < k0; r += nth) {
      float acc = z[r];
#pragma unroll 8
      for (int t = 0; t < kb; ++t) acc = fmaf(-__ldg(F + (int64_t)(k0 + t) * m + r), z[k0 + t], acc);
      if (r >= k0 - 32)
        nx[r - (k0 - 32)] = acc;
      else
        z[r] = acc;
    }
  }
};

// The factor of an airfoil of more than kLargeM - 1 panels, in the layout the
// blocked LU (k_lu_large.cu) leaves: the tiled layout of tl_layout.cuh with
// every full tile in row chunks.  Block row 0 (the first e rows) is row-major
// (ld m); in block row I >= 1 the columns below e sit in the ragged tile (I, 0)
// (row-major, ld e, split at the head) and column e + 32 ch + c of row rr at
// tile(I, 1) + 4096 ch + 32 rr + c: a row is a run of 32-float chunks 4096
// floats apart.  The 32-row groups follow the tiles: ceil(e / 32) groups in
// block row 0, then four per full block row, and the diagonal blocks inverted
// are those of these groups.  In the transposed updates of block row I >= 1
// the threads of a warp take the 32 columns of one chunk.
struct CrFactor;
// The ragged tile (I, 0) of block row I >= 1: element (rr, c), c < e, is float
// rr e + c of the tile, which sits at span(I) up to the head and after the full
// tiles beyond it.
struct CrRag {
  const float* p;  // the block row's span
  int hh, e;
  int64_t jump;    // the full tiles' floats
  __device__ CrRag(const float* F, const TlGeom& g, int I)
      : p(F + g.span(I)), hh(g.head(I)), e(g.e), jump((int64_t)(g.T - 1) * kTlTile) {}
  __device__ float operator()(int rr, int c) const {
    const int idx = rr * e + c;
    return __ldg(p + (idx < hh ? (int64_t)idx : idx + jump));
  }
};

// sum_{ch in [c0, c1)} p[4096 ch] yy[32 ch] (one lane's share of a chunked row:
// p and yy already offset by the lane) for two rows p0 and p1 (p1 only if
// `two`), as row_dot2.
__device__ __forceinline__ float2 chunk_dot2(const float* __restrict__ p0,
                                             const float* __restrict__ p1, bool two,
                                             const float* yy, int c0, int c1) {
  float a[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  float b[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  int ch = c0;
  for (; ch + 7 < c1; ch += 8) {
    float u[8], v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      u[t] = __ldg(p0 + (int64_t)(ch + t) * kTlChunk);
      v[t] = two ? __ldg(p1 + (int64_t)(ch + t) * kTlChunk) : 0.0f;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const float y = yy[32 * (ch + t)];
      a[t] = fmaf(u[t], y, a[t]);
      b[t] = fmaf(v[t], y, b[t]);
    }
  }
  if (ch < c1) {
    float u[8], v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const bool ok = ch + t < c1;
      u[t] = ok ? __ldg(p0 + (int64_t)(ch + t) * kTlChunk) : 0.0f;
      v[t] = (ok && two) ? __ldg(p1 + (int64_t)(ch + t) * kTlChunk) : 0.0f;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      if (ch + t < c1) {
        const float y = yy[32 * (ch + t)];
        a[t] = fmaf(u[t], y, a[t]);
        b[t] = fmaf(v[t], y, b[t]);
      }
    }
  }
  return make_float2(sum8(a), sum8(b));
}

struct CrFactor {
  const float* F;  // the airfoil's matrix
  TlGeom g;
  int m;
  int G0;          // groups of block row 0
  int nch;         // chunks of a full block row: 4 (T - 1)
  __device__ void init(const float* F_, int m_, int64_t moff) {
    F = F_;
    m = m_;
    g.init(m_, moff);
    G0 = (g.e + 31) >> 5;
    nch = 4 * (g.T - 1);
  }
  __device__ int groups() const { return G0 + nch; }
  __device__ int k0(int d) const { return d < G0 ? 32 * d : g.e + 32 * (d - G0); }
  __device__ int kb(int d) const { return d < G0 ? min(32, g.e - 32 * d) : 32; }
  // row rr of block row I >= 1: its chunk 0 (add 4096 ch + the column in the chunk)
  __device__ const float* chunk_row(int I, int rr) const {
    return F + g.tile(I, 1) + (int64_t)rr * kTlC;
  }
  // rows i and i1 (i1 only if `two`) of group d, as RmFactor
  __device__ float2 dot_left(int i, int i1, bool two, int d, const float* y, int lane) const {
    if (d < G0) return row_dot2(F + (int64_t)i * m, F + (int64_t)i1 * m, two, y, 0, 32 * d, lane);
    const int e = g.e, I = 1 + ((i - e) >> 7), rr = (i - e) & (kTlB - 1), rr1 = (i1 - e) & (kTlB - 1);
    const CrRag rag(F, g, I);
    float v = 0.0f, w = 0.0f;
#pragma unroll
    for (int t = 0; t < kTlB / 32; ++t) {
      const int c = lane + 32 * t;
      if (c < e) {
        v = fmaf(rag(rr, c), y[c], v);
        if (two) w = fmaf(rag(rr1, c), y[c], w);
      }
    }
    const float2 p = chunk_dot2(chunk_row(I, rr) + lane, chunk_row(I, rr1) + lane, two,
                                y + e + lane, 0, d - G0);
    return make_float2(v + p.x, w + p.y);
  }
  __device__ float2 dot_right(int i, int i1, bool two, int d, const float* y, int lane) const {
    if (d < G0)
      return row_dot2(F + (int64_t)i * m, F + (int64_t)i1 * m, two, y, k0(d) + kb(d), m, lane);
    const int e = g.e, I = 1 + ((i - e) >> 7), rr = (i - e) & (kTlB - 1), rr1 = (i1 - e) & (kTlB - 1);
    return chunk_dot2(chunk_row(I, rr) + lane, chunk_row(I, rr1) + lane, two, y + e + lane,
                      d - G0 + 1, nch);
  }
  __device__ const float* diag_row(int d, int i) const {
    if (d < G0) return F + (int64_t)i * m + 32 * d;
    const int h = d - G0, rr = (i - g.e) & (kTlB - 1);
    return chunk_row(1 + (h >> 2), rr) + (int64_t)h * kTlChunk;
  }
  __device__ void update_right(int d, float* z, float* nx, int tid, int nth) const {
    const int k0 = this->k0(d), kb = this->kb(d), c0 = k0 + kb;
    const int c1 = c0 + this->kb(d + 1);  // end of group d + 1 (d + 1 < groups())
    if (d < G0) {
      for (int r = c0 + tid; r < m; r += nth) {
        float acc = z[r];
#pragma unroll 16
        for (int t = 0; t < kb; ++t)
          acc = fmaf(-__ldg(F + (int64_t)(k0 + t) * m + r), z[k0 + t], acc);
        if (r < c1)
          nx[r - c0] = acc;
        else
          z[r] = acc;
      }
    } else {
      const int h = d - G0, e = g.e;
      const float* p = chunk_row(1 + (h >> 2), 32 * (h & 3));  // row k0 of the group
      for (int c = 32 * (h + 1) + tid; c < 32 * nch; c += nth) {
        const float* pc = p + (int64_t)(c >> 5) * kTlChunk + (c & 31);
        float acc = z[e + c];
#pragma unroll 16
        for (int t = 0; t < 32; ++t) acc = fmaf(-__ldg(pc + t * kTlC), z[k0 + t], acc);
        if (e + c < c1)
          nx[e + c - c0] = acc;
        else
          z[e + c] = acc;
      }
    }
  }
  __device__ void update_left(int d, float* z, float* nx, int tid, int nth) const {
    const int k0 = this->k0(d), kb = this->kb(d);
    const int p0 = this->k0(d - 1);  // start of group d - 1 (d >= 1)
    if (d < G0) {
      for (int r = tid; r < k0; r += nth) {
        float acc = z[r];
#pragma unroll 16
        for (int t = 0; t < kb; ++t)
          acc = fmaf(-__ldg(F + (int64_t)(k0 + t) * m + r), z[k0 + t], acc);
        if (r >= p0)
          nx[r - p0] = acc;
        else
          z[r] = acc;
      }
    } else {
      const int h = d - G0, I = 1 + (h >> 2), rr0 = 32 * (h & 3), e = g.e;
      // columns below e: the ragged tile (I, 0)
      const CrRag rag(F, g, I);
      for (int r = tid; r < e; r += nth) {
        float acc = z[r];
#pragma unroll 16
        for (int t = 0; t < 32; ++t) acc = fmaf(-rag(rr0 + t, r), z[k0 + t], acc);
        if (r >= p0)
          nx[r - p0] = acc;
        else
          z[r] = acc;
      }
      // columns e .. k0 - 1: the chunks before the group's
      const float* p = chunk_row(I, rr0);
      for (int c = tid; c < 32 * h; c += nth) {
        const float* pc = p + (int64_t)(c >> 5) * kTlChunk + (c & 31);
        float acc = z[e + c];
#pragma unroll 16
        for (int t = 0; t < 32; ++t) acc = fmaf(-__ldg(pc + t * kTlC), z[k0 + t], acc);
        if (e + c >= p0)
          nx[e + c - p0] = acc;
        else
          z[e + c] = acc;
      }
    }
  }
};

// FWD: y <- U^{-1} L^{-1} y (scratch ty); TRN: z <- L^{-T} U^{-T} z (scratch tz).
template <bool FWD, bool TRN, class Fac>
__device__ void lu_sweeps(const Fac& f, float* y, float* z, float* ty, float* tz) {
  static_assert(FWD || TRN, "a system to solve");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  const int tid = (int)threadIdx.x, nt = (int)blockDim.x;
  const int G = f.groups();
  for (int d = 0; d < G; ++d) {
    const int k0 = f.k0(d), kb = f.kb(d);
    if (FWD) {
      // rows q and q + nw of the group together
      for (int q = warp; q < kb; q += 2 * nw) {
        const int i = k0 + q, q1 = q + nw;
        const bool two = q1 < kb;
        const float2 p = f.dot_left(i, two ? k0 + q1 : i, two, d, y, lane);
        const float acc = warp_sum_f(p.x), acc1 = warp_sum_f(p.y);
        if (lane == 0) {
          ty[q] = y[i] - acc;
          if (two) ty[q1] = y[k0 + q1] - acc1;
        }
      }
    }
    if (TRN) {
      if (d == 0) {
        if (tid < 32) tz[tid] = (tid < kb) ? z[k0 + tid] : 0.0f;
      } else {
        f.update_right(d - 1, z, tz, tid, nt);
      }
    }
    __syncthreads();
    if (FWD) {
      for (int q = warp; q < kb; q += nw) {
        const int i = k0 + q;
        // y_i = t_i + sum_{k<i} X[i][k] t_k  (X unit lower, stored below the diagonal)
        float v = (lane < q) ? __ldg(f.diag_row(d, i) + lane) * ty[lane] : 0.0f;
        v = warp_sum_f(v);
        if (lane == 0) y[i] = ty[q] + v;
      }
    }
    if (TRN) {
      for (int q = warp; q < kb; q += nw) {
        // z_i = sum_{k<=i} Y[k][i] t_k  (Y upper with diagonal)
        const int i = k0 + q;
        float v = (lane <= q) ? __ldg(f.diag_row(d, k0 + lane) + q) * tz[lane] : 0.0f;
        v = warp_sum_f(v);
        if (lane == 0) z[i] = v;
      }
    }
    __syncthreads();
  }
  for (int d = G - 1; d >= 0; --d) {
    const int k0 = f.k0(d), kb = f.kb(d);
    if (FWD) {
      for (int q = warp; q < kb; q += 2 * nw) {
        const int i = k0 + q, q1 = q + nw;
        const bool two = q1 < kb;
        const float2 p = f.dot_right(i, two ? k0 + q1 : i, two, d, y, lane);
        const float acc = warp_sum_f(p.x), acc1 = warp_sum_f(p.y);
        if (lane == 0) {
          ty[q] = y[i] - acc;
          if (two) ty[q1] = y[k0 + q1] - acc1;
        }
      }
    }
    if (TRN) {
      if (d == G - 1) {
        if (tid < 32) tz[tid] = (tid < kb) ? z[k0 + tid] : 0.0f;
      } else {
        f.update_left(d + 1, z, tz, tid, nt);
      }
    }
    __syncthreads();
    if (FWD) {
      for (int q = warp; q < kb; q += nw) {
        const int i = k0 + q;
        // y_i = sum_{k>=i} Y[i][k] t_k  (Y upper with diagonal)
        float v = (lane >= q && lane < kb) ? __ldg(f.diag_row(d, i) + lane) * ty[lane] : 0.0f;
        v = warp_sum_f(v);
        if (lane == 0) y[i] = v;
      }
    }
    if (TRN) {
      for (int q = warp; q < kb; q += nw) {
        // z_i = t_i + sum_{k>i} X[k][i] t_k  (X unit lower, stored below the diagonal)
        const int i = k0 + q;
        float v = (lane > q && lane < kb) ? __ldg(f.diag_row(d, k0 + lane) + q) * tz[lane] : 0.0f;
        v = warp_sum_f(v);
        if (lane == 0) z[i] = tz[q] + v;
      }
    }
    __syncthreads();
  }
}

// The forward system (fw), the transposed one (tr) or both; ty, tz: 32 floats
// each.  Both at once (COMBINE) or one after the other.
template <bool COMBINE, class Fac>
__device__ void lu_solve(const Fac& f, bool fw, bool tr, float* y, float* z, float* ty,
                         float* tz) {
  if (COMBINE && fw && tr) {
    lu_sweeps<true, true>(f, y, z, ty, tz);
    return;
  }
  if (fw) lu_sweeps<true, false>(f, y, z, ty, tz);
  if (tr) lu_sweeps<false, true>(f, y, z, ty, tz);
}

// ---------------------------------------------------------------------------
// Double-float residuals against the stored planes
// ---------------------------------------------------------------------------
// Accumulator for sum_k (h_k + l_k)(xh_k + xl_k) with error ~2^-70 sum|p|:
// s1 collects the exact leading products h*xh through two_sum (their rounding
// errors go to s2), s2 (double-float) collects the ~2^-24 terms (the two_prod
// error of h*xh, h*xl, l*xh), summed error-free into one float per entry
// first, and s3 (float) the ~2^-48 terms (the errors of h*xl, l*xh and of
// that sum, and l*xl).  Every product is exact via two_prod.
// Corrections with the Gauss-Jordan inverse X = (P Mt)^{-1}: y <- X y (rows
// over the warps, 4 rows per pass, lanes along the row) and y <- X^T y (the
// rows split into 8 ranges, one per warp, a column per lane, partial sums in
// `part`, 8 x m floats).  `w` is an m-float shared scratch.
__device__ void gj_apply(const float* __restrict__ X, int m, float* y, float* w) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i0 = 4 * warp; i0 < m; i0 += 4 * (int)(blockDim.x >> 5)) {
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int k = lane; k < m; k += 32) {
      const float yk = y[k];
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (i0 + r < m) acc[r] = fmaf(__ldg(X + (i0 + r) * m + k), yk, acc[r]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float v = warp_sum_f(acc[r]);
      if (lane == 0 && i0 + r < m) w[i0 + r] = v;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < m; k += (int)blockDim.x) y[k] = w[k];
  __syncthreads();
}

__device__ void gj_apply_transposed(const float* __restrict__ X, int m, float* y, float* part) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rows = (m + (int)(blockDim.x >> 5) - 1) / (int)(blockDim.x >> 5);
  const int k0 = warp * rows, k1 = min(m, k0 + rows);
  for (int cb = 0; cb < m; cb += 32) {
    const int i = cb + lane;
    float acc = 0.0f;
    if (i < m) {
#pragma unroll 4
      for (int k = k0; k < k1; ++k) acc = fmaf(__ldg(X + k * m + i), y[k], acc);
    }
    if (i < m) part[warp * m + i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += (int)blockDim.x) {
    float v = 0.0f;
#pragma unroll
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += part[w * m + i];
    y[i] = v;
  }
  __syncthreads();
}

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
  // the four ~2^-24 terms summed error-free (u, v, w) before the one
  // double-float addition; the three sums' errors are ~2^-48 terms
  const df2 u = two_sum(t.lo, p1.lo);
  const df2 v = two_sum(p2.hi, p3.hi);
  const df2 w = two_sum(u.hi, v.hi);
  a.s2 = df_add_f(a.s2, w.hi);
  const float e1 = __fadd_rn(__fadd_rn(u.lo, v.lo), w.lo);
  const float e2 = __fadd_rn(__fadd_rn(p2.lo, p3.lo), __fmul_rn(l, xl));
  a.s3 = __fadd_rn(a.s3, __fadd_rn(e1, e2));
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

// The first residual of the refinement only has to carry the ~1e-4 error of
// the float32 solve to the next correction: a double-float sum of the products
// (each exact to ~2^-48 of itself, the sum to ~2^-44 of sum |p|) suffices there.
struct LiteAcc {
  df2 s;
};
__device__ __forceinline__ void resacc_init(LiteAcc& a) { a.s = mkdf(0.0f); }
__device__ __forceinline__ void resacc_add(LiteAcc& a, float h, float l, float xh, float xl) {
  const df2 p = two_prod(h, xh);
  const float e = __fmaf_rn(h, xl, __fmaf_rn(l, xh, p.lo));
  a.s = df_add(a.s, mkdf(p.hi, e));
}
__device__ __forceinline__ void resacc_merge(LiteAcc& a, const LiteAcc& b) { a.s = df_add(a.s, b.s); }
__device__ __forceinline__ LiteAcc warp_sum_res(LiteAcc a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    LiteAcc b;
    b.s.hi = __shfl_xor_sync(0xffffffffu, a.s.hi, o);
    b.s.lo = __shfl_xor_sync(0xffffffffu, a.s.lo, o);
    resacc_merge(a, b);
  }
  return a;
}
__device__ __forceinline__ double resacc_sub_from(double c, const LiteAcc& a) {
  return c - ((double)a.s.hi + (double)a.s.lo);
}

// r_j = b_j - sum_i M_ji x_i for all rows j; x given as float pairs (xh, xl).
// A warp takes two rows at a time and issues all loads of a 256-column chunk
// before accumulating.
template <class Acc, class Rhs, class RT>
__device__ void residual_rows(const float* __restrict__ Ah, const float* __restrict__ Al, int m,
                              const float* xh, const float* xl, const Rhs& b, RT* r) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j0 = 2 * warp; j0 < m; j0 += 2 * (int)(blockDim.x >> 5)) {
    Acc acc0, acc1;
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
      b.store(r, j0, resacc_sub_from(b(j0), acc0));
      if (two) b.store(r, j0 + 1, resacc_sub_from(b(j0 + 1), acc1));
    }
  }
}

// r_i = g_i - sum_j M_ji x_j for all columns i: each warp owns 32 consecutive
// columns (one per lane) and walks all rows, 8 rows of loads in flight.
template <class Acc, class Rhs, class RT>
__device__ void residual_cols(const float* __restrict__ Ah, const float* __restrict__ Al, int m,
                              const float* xh, const float* xl, const Rhs& g, RT* r) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int cb = 32 * warp; cb < m; cb += (int)blockDim.x) {
    const int c = cb + lane;
    const bool ok = c < m;
    Acc acc;
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
    if (ok) g.store(r, c, resacc_sub_from(g(c), acc));
  }
}

// Both residuals in one pass over the matrix (m <= kFuseM), each entry loaded
// once: warp w takes the rows j = w, w + 8, ...; lane l owns the columns
// c = l + 32 t.  The row sums (forward system, x) are reduced across the warp
// per row; the column sums (transposed system, lam) stay in per-lane
// accumulators and are merged across the warps through `part` ((int)(blockDim.x >> 5) x m).
constexpr int kFuseM = 288;
constexpr int kFuseT = (kFuseM + 31) / 32;
static_assert(kFuseM <= kLargeM, "KEEP launches never hold a blocked (tiled) factor");
template <class Acc, int FT = kFuseT, class Rhs, class RT>
__device__ void residual_both(const float* __restrict__ Ah, const float* __restrict__ Al, int m,
                              const float* xh, const float* xl, const float* yh, const float* yl,
                              const Rhs& b, const Rhs& g, RT* rf, RT* rt, Acc* part) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Acc cacc[FT];
#pragma unroll
  for (int t = 0; t < FT; ++t) resacc_init(cacc[t]);
  for (int j = warp; j < m; j += (int)(blockDim.x >> 5)) {
    float h[FT], l[FT];
#pragma unroll
    for (int t = 0; t < FT; ++t) {
      const int c = lane + 32 * t;
      const bool ok = c < m;
      h[t] = ok ? __ldg(Ah + j * m + c) : 0.0f;
      l[t] = ok ? __ldg(Al + j * m + c) : 0.0f;
    }
    const float yjh = yh[j], yjl = yl[j];
    Acc racc;
    resacc_init(racc);
#pragma unroll
    for (int t = 0; t < FT; ++t) {
      const int c = lane + 32 * t;
      if (c < m) {
        resacc_add(racc, h[t], l[t], xh[c], xl[c]);
        resacc_add(cacc[t], h[t], l[t], yjh, yjl);
      }
    }
    racc = warp_sum_res(racc);
    if (lane == 0) b.store(rf, j, resacc_sub_from(b(j), racc));
  }
#pragma unroll
  for (int t = 0; t < FT; ++t) {
    const int c = lane + 32 * t;
    if (c < m) part[warp * m + c] = cacc[t];
  }
  __syncthreads();
  for (int c = threadIdx.x; c < m; c += (int)blockDim.x) {
    Acc acc = part[c];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) resacc_merge(acc, part[w * m + c]);
    g.store(rt, c, resacc_sub_from(g(c), acc));
  }
}

// ---------------------------------------------------------------------------
// The refinement kernel: forward and/or transposed system of one airfoil
// ---------------------------------------------------------------------------
// Where the refinement keeps its vectors.  Launches of small airfoils
// (n_max + 1 <= kFuseM, KEEP) hold x, the residual r and the right-hand side
// in shared memory as doubles.  The others, whose shared memory bounds the
// airfoils per SM, keep x in the caller's output array, the residual as the
// float the correction solve takes (component n already times s) and evaluate
// the right-hand side where it is needed, once per row or column of a
// residual pass.
template <class RT>
struct IrSystem {
  double* x;   // m  current solution
  RT* r;       // m  residual
  float* xh;   // m  x as float pairs for the residual
  float* xl;   // m
};

// A stored right-hand side (KEEP): the residual is kept as is.
struct SmemRhs {
  const double* bb;
  __device__ double operator()(int k) const { return bb[k]; }
  __device__ void store(double* r, int k, double v) const { r[k] = v; }
};

// Right-hand side of system q (0: M u = b, 1: M^T lambda = g), evaluated; the
// residual is stored as the correction solve's float input.
struct IrRhs {
  const double* rhs;   // forward right-hand side (rhs_kind 0), at the airfoil's offset
  const double* nd;    // the airfoil's nodes
  const double* w_u;   // vector-Jacobian weights at the airfoil's offsets (or NULL)
  const double* w_cp;
  const double* u_in;
  double w_cl;
  int n, q, rhs_kind, vjp;
  double v, cc, s;
  __device__ double operator()(int k) const { return eval(k); }
  __device__ double eval(int k) const {
    if (q == 0) {
      if (rhs_kind == 0) return rhs[k];
      // the basis right-hand sides of a polar: b(alpha) = cos(alpha) b_y +
      // sin(alpha) b_x with b_y = v m_y, b_x = -v m_x (m the control point)
      if (k >= n) return 0.0;
      const int k1 = (k + 1 == n) ? 0 : k + 1;
      return (rhs_kind == 1) ? 0.5 * v * (nd[2 * k + 1] + nd[2 * k1 + 1])
                                : -0.5 * v * (nd[2 * k] + nd[2 * k1]);
    }
    double g = 0.0;
    if (k < n) {
      const int k1 = (k + 1 == n) ? 0 : k + 1;
      const double hx = nd[2 * k1] - nd[2 * k], hy = nd[2 * k1 + 1] - nd[2 * k + 1];
      g = 2.0 * sqrt(hx * hx + hy * hy) / (v * cc);  // dCl/dgamma_k
    }
    if (vjp) {
      // dL/du for L = w_cl Cl + w_u . u + w_cp . Cp, Cp_k = 1 - (gamma_k / v)^2
      g *= w_cl;
      if (w_u) g += w_u[k];
      if (w_cp && k < n) g += w_cp[k] * (-2.0 * u_in[k] / (v * v));
    }
    return g;
  }
  __device__ float scaled(int k, double r) const { return (float)((k == n) ? r * s : r); }
  __device__ void store(float* r, int k, double v) const { r[k] = scaled(k, v); }
};

// The float input of the correction solve from a residual component.
__device__ __forceinline__ float solve_input(double r, int k, int n, double s) {
  return (float)((k == n) ? r * s : r);
}
__device__ __forceinline__ float solve_input(float r, int, int, double) { return r; }

__device__ __forceinline__ int gpiv_first(const SolveArgs& a, int b) {
  return a.piv[vec_off(a.bt, b)];
}

// NT threads, MINB blocks per SM (see launch_ir_kernel).
template <int NT, int MINB, int FT, bool KEEP>
__global__ void __launch_bounds__(NT, MINB) k_ir_mixed(SolveArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const Batch& bt = a.bt;
  const int b = bt.order[blockIdx.x];
  const int n = airfoil_n(bt, b);
  const int m = n + 1;
  if (a.info[b] != 0 || n > bt.n_max) return;
  const int mv = bt.n_max + 1;
  using RT = typename std::conditional<KEEP, double, float>::type;
  double* red = reinterpret_cast<double*>(smraw);  // 32
  IrSystem<RT> sys[2];
  double* dp = red + 32;
  double* bbs = dp;  // KEEP: x, r, bb of both systems (6 m doubles)
  if (KEEP) {
    for (int q = 0; q < 2; ++q) {
      sys[q].x = dp;
      sys[q].r = reinterpret_cast<RT*>(dp + mv);
      dp += 2 * mv;
    }
    bbs = dp;
    dp += 2 * mv;
  }
  float* y = reinterpret_cast<float*>(dp);  // m
  float* fp = y + mv;
  for (int q = 0; q < 2; ++q) {
    sys[q].xh = fp;
    sys[q].xl = fp + mv;
    fp += 2 * mv;
    if (!KEEP) {
      sys[q].r = reinterpret_cast<RT*>(fp);
      fp += mv;
    }
  }
  int* perm = reinterpret_cast<int*>(fp);  // m
  float* t32 = reinterpret_cast<float*>(perm + mv);  // 32
  // per-warp partial sums: of the inverse's products (floats, m <= kGjM), or of
  // the fused residual pass (ResAcc, launches with n_max + 1 <= kFuseM)
  float* part = reinterpret_cast<float*>(
      (reinterpret_cast<uintptr_t>(t32 + 32) + 15) & ~(uintptr_t)15);
  // The corrections: the forward one in y, the transposed one in z, which is
  // the transposed system's float copy of lambda (rewritten from lambda before
  // it is read again); the transposed sweeps' 32-float group scratch is `red`
  // (free while the sweeps run).
  float* z = sys[1].xh;
  float* t32z = reinterpret_cast<float*>(red);
  // the factor buffer holds an inverse (exchanges stored as -(row + 1)) or an LU
  const bool gj = gpiv_first(a, b) < 0;

  const int64_t moff = bt.mat_off[b];
  const float* Ah = a.A_hi + moff;
  const float* Al = a.A_lo + moff;
  const float* F = a.LU + moff;
  // above kLargeM - 1 panels: the blocked factor's tiled layout (never in a
  // KEEP launch: n_max + 1 <= kFuseM there)
  const bool cr = !KEEP && !gj && m > kLargeM;
  CrFactor crf;
  if constexpr (!KEEP) {
    if (cr) crf.init(F, m, moff);
  }
  const int32_t* gpiv = a.piv + vec_off(bt, b);
  const double s = border_scale(Ah, n, m, red);
  const bool act0 = a.u != nullptr, act1 = a.lam != nullptr;
  // the fused residual pass needs `part`, allocated when the launch's n_max fits
  const bool fuse = bt.n_max + 1 <= kFuseM;

  // right-hand sides: b, and g = dCl/du = 2 |h_k| / (v c) (0 for C); x = 0, r = b
  IrRhs rhs[2];
  for (int q = 0; q < 2; ++q) {
    const int64_t vo = vec_off(bt, b);
    rhs[q].rhs = (a.rhs_kind == 0 && a.rhs) ? a.rhs + vo : nullptr;
    rhs[q].nd = bt.nodes + 2 * bt.node_off[b];
    rhs[q].w_u = a.w_u ? a.w_u + vo : nullptr;
    rhs[q].w_cp = a.w_cp ? a.w_cp + bt.node_off[b] : nullptr;
    rhs[q].u_in = a.u_in ? a.u_in + vo : nullptr;
    rhs[q].w_cl = a.w_cl ? a.w_cl[b] : 0.0;
    rhs[q].n = n;
    rhs[q].q = q;
    rhs[q].rhs_kind = a.rhs_kind;
    rhs[q].vjp = a.vjp;
    rhs[q].v = a.vinf ? a.vinf[b] : 1.0;
    rhs[q].cc = a.chord ? a.chord[b] : 1.0;
    rhs[q].s = s;
  }
  SmemRhs srhs[2];
  srhs[0].bb = bbs;
  srhs[1].bb = bbs + mv;
  if (!KEEP) {
    sys[0].x = act0 ? a.u + vec_off(bt, b) : nullptr;
    sys[1].x = act1 ? a.lam + vec_off(bt, b) : nullptr;
  }
  for (int k = threadIdx.x; k < m; k += (int)blockDim.x) {
    for (int q = 0; q < 2; ++q) {
      if (!(q == 0 ? act0 : act1)) continue;
      const double bk = rhs[q].eval(k);
      sys[q].x[k] = 0.0;
      if constexpr (KEEP) {
        bbs[q * mv + k] = bk;
        sys[q].r[k] = bk;
      } else {
        sys[q].r[k] = rhs[q].scaled(k, bk);
      }
    }
  }
  // row permutation of the factor: P y = y[perm]
  if (threadIdx.x == 0) {
    for (int k = 0; k < m; ++k) perm[k] = k;
    for (int k = 0; k < m; ++k) {
      const int p = gj ? -gpiv[k] - 1 : gpiv[k];
      const int t = perm[k];
      perm[k] = perm[p];
      perm[p] = t;
    }
  }
  __syncthreads();

  bool active[2] = {act0, act1};
  bool conv[2] = {!act0, !act1};
  double dprev[2] = {0.0, 0.0};  // size of the previous correction
  int it = 0;
  for (;; ++it) {
    const bool run0 = active[0] && !conv[0], run1 = active[1] && !conv[1];
    // the corrections' right-hand sides: y = P S_r r (forward system; then
    // dx = S_c y) and z = S_c r (transposed system; then dlambda = S_r P^T z)
    for (int k = threadIdx.x; k < m; k += (int)blockDim.x) {
      if (run0) {
        const int src = perm[k];
        y[k] = solve_input(sys[0].r[src], src, n, s);
      }
      if (run1) z[k] = solve_input(sys[1].r[k], k, n, s);
    }
    __syncthreads();
    if (gj) {
      if (run0) gj_apply(F, m, y, part);
      if (run1) gj_apply_transposed(F, m, z, part);
    } else if constexpr (!KEEP) {
      if (cr)
        lu_solve<true>(crf, run0, run1, y, z, t32, t32z);
      else
        lu_solve<true>(RmFactor{F, m}, run0, run1, y, z, t32, t32z);
    } else {
      lu_solve<false>(RmFactor{F, m}, run0, run1, y, z, t32, t32z);
    }
    for (int q = 0; q < 2; ++q) {
      if (!(q == 0 ? run0 : run1)) continue;
      IrSystem<RT>& S = sys[q];
      const float* w = (q == 0) ? y : z;
      double dmax = 0.0;
      for (int k = threadIdx.x; k < m; k += (int)blockDim.x) {
        const int dst = (q == 0) ? k : perm[k];
        const double d = (dst == n) ? (double)w[k] * s : (double)w[k];
        S.x[dst] += d;
        dmax = fmax(dmax, fabs(d));
      }
      __syncthreads();
      double xmax = 0.0;
      for (int k = threadIdx.x; k < m; k += (int)blockDim.x) xmax = fmax(xmax, fabs(S.x[k]));
      dmax = block_absmax_d(dmax, red);
      xmax = block_absmax_d(xmax, red);
      // Converged when the correction just applied is below tol |x|, or when
      // the contraction seen over the last two corrections (rho = |d_k| /
      // |d_{k-1}| <= 1/8) predicts the next one, |d_k| rho, below tol |x|: the
      // error left in x_{k+1} is about that next correction.
      // (the correction of iteration 1 comes from the double-float residual,
      // so the first test waits for iteration 2)
      if (it >= 2 && dmax <= a.tol * xmax) conv[q] = true;
      if (it >= 2 && dmax <= 0.125 * dprev[q] && dmax * (dmax / dprev[q]) <= a.tol * xmax)
        conv[q] = true;
      dprev[q] = dmax;
    }
    if ((conv[0] && conv[1]) || it >= a.max_iter) break;
    for (int q = 0; q < 2; ++q) {
      if (!active[q] || conv[q]) continue;
      for (int k = threadIdx.x; k < m; k += (int)blockDim.x) {
        const df2 d = df_from_double(sys[q].x[k]);
        sys[q].xh[k] = d.hi;
        sys[q].xl[k] = d.lo;
      }
    }
    __syncthreads();
    const bool both = active[0] && !conv[0] && active[1] && !conv[1];
    auto residuals = [&](const auto& R0, const auto& R1) {
      if (it == 0) {
        if (both && fuse) {
          residual_both<LiteAcc, FT>(Ah, Al, m, sys[0].xh, sys[0].xl, sys[1].xh, sys[1].xl, R0,
                                     R1, sys[0].r, sys[1].r, reinterpret_cast<LiteAcc*>(part));
        } else {
          if (active[0] && !conv[0])
            residual_rows<LiteAcc>(Ah, Al, m, sys[0].xh, sys[0].xl, R0, sys[0].r);
          if (active[1] && !conv[1])
            residual_cols<LiteAcc>(Ah, Al, m, sys[1].xh, sys[1].xl, R1, sys[1].r);
        }
      } else if (both && fuse) {
        residual_both<ResAcc, FT>(Ah, Al, m, sys[0].xh, sys[0].xl, sys[1].xh, sys[1].xl, R0, R1,
                                  sys[0].r, sys[1].r, reinterpret_cast<ResAcc*>(part));
      } else {
        if (active[0] && !conv[0])
          residual_rows<ResAcc>(Ah, Al, m, sys[0].xh, sys[0].xl, R0, sys[0].r);
        if (active[1] && !conv[1])
          residual_cols<ResAcc>(Ah, Al, m, sys[1].xh, sys[1].xl, R1, sys[1].r);
      }
    };
    if constexpr (KEEP)
      residuals(srhs[0], srhs[1]);
    else
      residuals(rhs[0], rhs[1]);
    __syncthreads();
  }
  if (KEEP) {
    for (int k = threadIdx.x; k < m; k += (int)blockDim.x) {
      if (act0) a.u[vec_off(bt, b) + k] = sys[0].x[k];
      if (act1) a.lam[vec_off(bt, b) + k] = sys[1].x[k];
    }
  }
  if (threadIdx.x == 0) {
    if (a.iters && act0) a.iters[b] = it;
    if (!(conv[0] && conv[1])) a.info[b] = PANEL_INFO_NOCONV;
  }
}

// `part` (per-warp partial sums) serves the fused residual pass of launches with
// n_max + 1 <= kFuseM (nt/32 x m accumulators) and, in any launch, the
// Gauss-Jordan products of airfoils with m <= kGjM (nt/32 x m floats): the
// factor of a refinement launch may hold inverses whatever its n_max.
size_t ir_mixed_smem(int n_max, int nt) {
  const size_t mv = (size_t)n_max + 1;
  const size_t part = (mv <= (size_t)kFuseM) ? (size_t)(nt / 32) * mv * sizeof(ResAcc)
                                             : (size_t)(nt / 32) * kGjM * sizeof(float);
  // x, r and the right-hand side of both systems as doubles (KEEP), or r as floats
  const size_t vecs = (mv <= (size_t)kFuseM) ? 6 * mv * 8 + 5 * mv * 4 : 7 * mv * 4;
  return 32 * 8 + vecs + mv * 4 + 32 * 4 + 32 + part;
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
  a.inverse = 0;
  a.n_cap = bt.n_max;
  a.rhs_kind = 0;
  a.ir_shape = 0;
  a.lu_kind = 0;
  a.vjp = 0;
  a.w_cl = a.w_u = a.w_cp = a.u_in = nullptr;
  return a;
}

// Factor every airfoil: with `inverse` the Gauss-Jordan inverse for m <= kGjM;
// otherwise the one-block LU with the whole matrix in shared memory for m <=
// kSmemLuM (lu_kind 0 or 2) or in the LU buffer through L2 (lu_kind 1, and
// every m up to kLargeM); the step-synchronous blocked LU beyond.
cudaError_t launch_lu_mixed(const Batch& bt, const float* A_hi, float* LU, int32_t* piv,
                            int32_t* info, int32_t* iters, bool inverse, cudaStream_t s,
                            int lu_kind) {
  SolveArgs a = make_args(bt, A_hi, nullptr, LU, piv, nullptr, nullptr, nullptr, nullptr,
                          nullptr, 0, 0.0, info, iters);
  a.inverse = inverse ? 1 : 0;
  a.lu_kind = lu_kind;
  cudaError_t e;
  if (bt.n_max + 1 > kLargeM) {
    e = launch_lu_large(a, s);
    if (e != cudaSuccess) return e;
  }
  if (!inverse && lu_kind != 1) {
    // airfoils up to kSmemLuM unknowns with the whole matrix in shared memory
    SolveArgs h = a;
    h.bt.n_max = min(bt.n_max, kSmemLuM - 1);
    const size_t hs = lu_smem_smem(h.bt.n_max);
    e = ensure_smem(k_lu_smem, hs);
    if (e != cudaSuccess) return e;
    k_lu_smem<<<bt.B, kSmemLuThreads, hs, s>>>(h);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if ((bt.n_max + 1 > kSmemLuM || lu_kind == 1) && (bt.n_max + 1 > kGjM || !inverse)) {
    SolveArgs g = a;
    g.bt.n_max = min(bt.n_max, kLargeM - 1);
    const size_t smem = lu_global_smem<32>(g.bt.n_max);
    e = ensure_smem(k_lu_global<32>, smem);
    if (e != cudaSuccess) return e;
    k_lu_global<32><<<bt.B, kThreads, smem, s>>>(g);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return launch_gj_mixed(a, s);
}

// lambda of a vector-Jacobian product: M^T lambda = w_cl dCl/du + w_u +
// w_cp dCp/du (refined), with the forward strengths u.
// Blocks of 128 threads, 8 per SM, while the shared memory of 8 fits in the SM's
// 228 KB (1 KB of it reserved per block; m <= 204) and the batch fills 8 blocks
// on every SM: more airfoils in flight to hide the latency of the dependent
// sweeps (a smaller batch is better served by more warps per airfoil).  Then 256
// threads, 4 per SM up to kFuseM unknowns (a few spilled registers), and above
// it the most warps per airfoil that shared memory allows: 4 x 256, 2 x 512 or
// 1 x 1024 threads (3 x 256 is the autotuner's fifth shape).
// FT: columns per lane of the fused residual pass (ceil(n_max + 1 / 32) at most;
// fewer registers for the smaller airfoils of the 128-thread shape, m <= 204).
template <int NT, int MINB, int FT = kFuseT>
static cudaError_t launch_ir_shape(const SolveArgs& a, cudaStream_t s) {
  const size_t smem = ir_mixed_smem(a.bt.n_max, NT);
  if (a.bt.n_max + 1 <= kFuseM) {
    const cudaError_t e = ensure_smem(k_ir_mixed<NT, MINB, FT, true>, smem);
    if (e != cudaSuccess) return e;
    k_ir_mixed<NT, MINB, FT, true><<<a.bt.B, NT, smem, s>>>(a);
  } else {
    const cudaError_t e = ensure_smem(k_ir_mixed<NT, MINB, FT, false>, smem);
    if (e != cudaSuccess) return e;
    k_ir_mixed<NT, MINB, FT, false><<<a.bt.B, NT, smem, s>>>(a);
  }
  return cudaGetLastError();
}

static cudaError_t launch_ir_kernel(const SolveArgs& a, cudaStream_t s) {
  const int n_max = a.bt.n_max;
  auto fits = [&](int nt, int blocks) {
    return (size_t)blocks * (ir_mixed_smem(n_max, nt) + 1024) <= 233472;
  };
  // an explicit shape (autotuning), when one block of it fits the shared memory
  switch (a.ir_shape) {
    case 1:
      if (fits(128, 1) && n_max + 1 <= 7 * 32) return launch_ir_shape<128, 8, 7>(a, s);
      break;
    case 2:
      if (fits(kThreads, 1)) return launch_ir_shape<kThreads, 4>(a, s);
      break;
    case 3:
      if (fits(512, 1)) return launch_ir_shape<512, 2>(a, s);
      break;
    case 4:
      if (fits(1024, 1)) return launch_ir_shape<1024, 1>(a, s);
      break;
    case 5:
      if (fits(kThreads, 1)) return launch_ir_shape<kThreads, 3>(a, s);
      break;
    default:
      break;
  }
  if (fits(128, 8) && n_max + 1 <= 7 * 32 && a.bt.B >= 8 * sm_count())
    return launch_ir_shape<128, 8, 7>(a, s);
  if (n_max + 1 <= kFuseM || fits(kThreads, 4)) return launch_ir_shape<kThreads, 4>(a, s);
  if (fits(512, 2)) return launch_ir_shape<512, 2>(a, s);
  return launch_ir_shape<1024, 1>(a, s);
}

cudaError_t launch_ir_vjp(const Batch& bt, const float* A_hi, const float* A_lo,
                          const float* LU, const int32_t* piv, const double* vinf,
                          const double* chord, const double* u, const double* w_cl,
                          const double* w_u, const double* w_cp, double* lam, int max_iter,
                          double tol, int32_t* info, cudaStream_t s) {
  SolveArgs a = make_args(bt, A_hi, A_lo, const_cast<float*>(LU), const_cast<int32_t*>(piv),
                          nullptr, vinf, chord, nullptr, lam, max_iter, tol, info, nullptr);
  a.vjp = 1;
  a.w_cl = w_cl;
  a.w_u = w_u;
  a.w_cp = w_cp;
  a.u_in = u;
  return launch_ir_kernel(a, s);
}

// Refine the forward (u) and/or transposed (lam) systems with the stored factor.
cudaError_t launch_ir_mixed(const Batch& bt, const float* A_hi, const float* A_lo,
                            const float* LU, const int32_t* piv, const double* rhs,
                            const double* vinf, const double* chord, double* u, double* lam,
                            int max_iter, double tol, int32_t* info, int32_t* iters,
                            cudaStream_t s, int rhs_kind, int ir_shape) {
  SolveArgs a = make_args(bt, A_hi, A_lo, const_cast<float*>(LU), const_cast<int32_t*>(piv),
                          rhs, vinf, chord, u, lam, max_iter, tol, info, iters);
  a.rhs_kind = rhs_kind;
  a.ir_shape = ir_shape;
  return launch_ir_kernel(a, s);
}

}  // namespace panel
