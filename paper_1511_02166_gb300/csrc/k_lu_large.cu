// k_lu_large.cu -- FP32 LU of large airfoils (m = n + 1 > kLargeM) for the
// mixed-precision path: blocked right-looking elimination, step-synchronous
// across the batch, so that each block column is spread over many blocks
// instead of one block per airfoil.
//
// The factor is kept in the tiled layout of tl_layout.cuh while the steps run
// (a ragged first block of e rows, then 128-row blocks), so that the tensor
// memory access unit can move whole 128 x 32 chunks.  Launches:
//   k_large_init      the scaled hi plane into the factor buffer, tiled;
//   per block K = 0 .. T-1:
//     k_large_diag    one block per airfoil: LU of the diagonal block in
//                     shared memory, with the pivot search restricted to its
//                     rows; its row exchanges are applied to the rest of
//                     those rows;
//     k_large_trsm    U12 = L11^{-1} A12 (stored transposed, the tensor cores'
//                     K-major B operand) and L21 = A21 U11^{-1}: the two
//                     triangles of the diagonal block are inverted in shared
//                     memory, then 128-wide slabs are multiplied by them;
//     k_update_tc     A22 -= L21 U12 on the tcgen05 tensor cores, operands
//                     loaded by TMA, A22 updated by TMA reduce-add
//                     (k_update_tc.cu);
//   k_tl_untranspose  the U tiles back from their transposed order to row
//                     chunks, one block per tile, in place;
//   k_large_finish    the 32 x 32 diagonal blocks of L and U of the first block
//                     row inverted in place (k_large_diag inverts those of the
//                     full diagonal tiles).
// The per-airfoil kernels take gridDim.y blocks per airfoil striding over
// slabs / tiles / rows, so a batch of few airfoils still fills the GPU.
//
// Pivoting.  The system is the collocation matrix of the logarithmic
// single-layer kernel (Section 2) bordered by the Kutta row and the C column
// (rescaled by s = mean |A_jj|).  For this family partial pivoting over the
// whole column exchanges almost nothing (only the first and the bordered last
// rows), and LU with no exchanges at all shows element growth ~1.3 at
// n = 2048.  Restricting the search to the diagonal block keeps every
// exchange inside the block's rows -- which is what lets L21 be a plain
// triangular solve over all rows in parallel -- and the refinement with the
// double-float residual takes the result to the same tolerance (it converges
// in as few steps as with full partial pivoting).  An exactly zero pivot still
// sets info[b] = its index + 1.
//
// The finished factor: P A = L U in the caller's LU buffer in the tiled layout
// with every full tile in row chunks (tl_layout.cuh), pivots as sequential
// exchanges, and the 32 x 32 diagonal blocks of L and U that follow the tiles
// replaced by their inverses; the refinement (k_solve_mixed.cu) reads it in
// that layout.
#include <atomic>

#include "tl_layout.cuh"

namespace panel {

constexpr int kBW = kTlB;     // block size
constexpr int kLdD = kBW + 1;

size_t lu_large_min_m() { return kLargeM + 1; }

__device__ __forceinline__ bool large_live(const SolveArgs& a, int b, int& n, int& m) {
  n = airfoil_n(a.bt, b);
  m = n + 1;
  return m > kLargeM && n <= a.bt.n_max && a.info[b] == 0;
}

// Scaled copy A_hi -> LU (border row and column times s) into the tiled
// layout.  Block y of gridDim.y takes block rows blockIdx.y, + gridDim.y, ...;
// the writes run along the tiled order (consecutive threads, consecutive
// floats) and the reads along rows of A_hi within 32-column chunks.
constexpr int kInitThreads = 256;
__global__ void __launch_bounds__(kInitThreads) k_large_init(SolveArgs a) {
  __shared__ double red[32];
  const Batch& bt = a.bt;
  const int b = bt.order[blockIdx.x];
  const int n = airfoil_n(bt, b), m = n + 1;
  if (m <= kLargeM || a.info[b] != 0) return;
  if (n > bt.n_max) {
    if (blockIdx.y == 0 && threadIdx.x == 0) a.info[b] = PANEL_INFO_TOO_LARGE;
    return;
  }
  const int64_t moff = bt.mat_off[b];
  const float* Ah = a.A_hi + moff;
  float* F = a.LU + moff;
  TlGeom g;
  g.init(m, moff);
  const float sf = (float)border_scale(Ah, n, m, red);
  auto scaled = [&](int r, int c) {
    const float v = Ah[(int64_t)r * m + c];
    return ((c == n && r < n) || r == n) ? v * sf : v;
  };
  constexpr int kU = 8;  // loads in flight per thread
  for (int I = blockIdx.y; I < g.T; I += gridDim.y) {
    const int r0 = g.start(I);
    if (I == 0) {  // row-major rows 0..e-1, kU loads in flight per thread
      for (int r = 0; r < g.e; ++r) {
        for (int c0 = threadIdx.x; c0 < m; c0 += kU * kInitThreads) {
          float v[kU];
#pragma unroll
          for (int i = 0; i < kU; ++i) {
            const int c = c0 + i * kInitThreads;
            v[i] = (c < m) ? scaled(r, c) : 0.0f;
          }
#pragma unroll
          for (int i = 0; i < kU; ++i) {
            const int c = c0 + i * kInitThreads;
            if (c < m) F[(int64_t)r * m + c] = v[i];
          }
        }
      }
      continue;
    }
    // a warp reads two whole rows of a tile (2 x 512 contiguous bytes of A_hi)
    // and writes them as 128-byte rows of the tile's four chunks
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    static_assert(kU == 8 && kInitThreads == 256, "8 warps x 2 rows x 4 chunks");
    for (int J = 1; J < g.T; ++J) {
      float* Tt = F + g.tile(I, J);
      const int c0 = g.start(J);
      for (int rb = 2 * warp; rb < kTlB; rb += 16) {
        float v[kU];
#pragma unroll
        for (int i = 0; i < kU; ++i) v[i] = scaled(r0 + rb + (i >> 2), c0 + 32 * (i & 3) + lane);
#pragma unroll
        for (int i = 0; i < kU; ++i) Tt[(i & 3) * kTlChunk + (rb + (i >> 2)) * kTlC + lane] = v[i];
      }
    }
    // the ragged tile (I, 0), kU loads in flight per thread
    for (int p0 = 0; p0 < kTlB * g.e; p0 += kU * kInitThreads) {
      float v[kU];
#pragma unroll
      for (int i = 0; i < kU; ++i) {
        const int p = p0 + i * kInitThreads + threadIdx.x;
        v[i] = (p < kTlB * g.e) ? scaled(r0 + p / g.e, p % g.e) : 0.0f;
      }
#pragma unroll
      for (int i = 0; i < kU; ++i) {
        const int p = p0 + i * kInitThreads + threadIdx.x;
        if (p < kTlB * g.e) F[g.rag(I, p / g.e, p % g.e)] = v[i];
      }
    }
  }
}

// One triangle of a 32 x 32 diagonal block inverted (the unit lower one, or
// the upper one; they touch disjoint entries, so two warps may work on one
// block at once), in a call of its own, so that its 32-register columns do
// not weigh on the register allocation of the LU around it.
__device__ __noinline__ void invert_triangle32(float* B, int ld, bool lower) {
  if (lower)
    invert_lower_unit(B, ld, 32);
  else
    invert_upper(B, ld, 32);
}

// LU of the diagonal block K with partial pivoting inside the block.
__global__ void __launch_bounds__(256, 3) k_large_diag(SolveArgs a, int K) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float* D = reinterpret_cast<float*>(smraw);          // kBW x kLdD
  float* rows4 = D + kBW * kLdD;                       // 2 x 4 x 32: the warps' candidate rows
  unsigned* red = reinterpret_cast<unsigned*>(rows4 + 256);  // 2 x 4 x 2: their keys, positions
  int* sp = reinterpret_cast<int*>(red + 16);          // kBW
  const Batch& bt = a.bt;
  const int b = bt.order[blockIdx.x];
  int n, m;
  if (!large_live(a, b, n, m)) return;
  TlGeom g;
  g.init(m, bt.mat_off[b]);
  if (K >= g.T) return;
  const int k0 = g.start(K), kb = g.size(K);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float* F = a.LU + bt.mat_off[b];
  // the diagonal block: rows of block row 0 (row-major), or the full tile (K, K)
  float* Td = (K == 0) ? F : F + g.tile(K, K);
  auto dpos = [&](int r, int c) {
    return (K == 0) ? (int64_t)r * m + c : (int64_t)((c >> 5) << 12) + r * 32 + (c & 31);
  };
  for (int e = tid; e < kBW * kBW; e += 256) {
    const int r = e >> 7, c = e & 127;
    D[r * kLdD + c] = (r < kb && c < kb) ? Td[dpos(r, c)] : 0.0f;
  }
  __syncthreads();
  // Blocked in panels of 32 columns.  Per panel: warps 0-3 factor the panel
  // (rows c0..kb-1) column by column with partial pivoting over those rows,
  // thread t holding row c0 + t of the panel in registers; rows keep their
  // threads and `pos` tracks their current position, so an exchange is
  // bookkeeping plus one sp entry.  Per column, one 128-thread barrier: each
  // warp finds its candidate (largest |x|, the lowest position among equal
  // maxima) and puts its key, position and whole row in shared memory (two
  // buffers, alternating by column); after the barrier every thread picks the
  // pivot among the four and reads its row; the rank-1 update in registers.  The step loop is rolled, the columns
  // rotating through the registers (x[0] is the current one) so that every
  // register index is a constant; each finished entry goes to the row's own
  // place in D (by original row), and the rows are written back in their final
  // order at the end.  Then the whole block applies the panel's exchanges to
  // the other columns, solves U12 = L11^{-1} A12 (a thread per column) and
  // updates the trailing block in 4 x 4 register tiles.
  __shared__ int zero_pivot;
  if (tid == 0) zero_pivot = -1;
  __syncthreads();
  for (int c0 = 0; c0 < kb; c0 += 32) {
    const int w = min(32, kb - c0);
    if (warp < 4) {
      const int nrow = kb - c0;  // rows taking part: c0 .. kb-1
      float x[32];
#pragma unroll
      for (int t = 0; t < 32; ++t)
        x[t] = (tid < nrow && t < w) ? D[(c0 + tid) * kLdD + c0 + t] : 0.0f;
      int pos = tid;
      bool done = tid >= nrow;
      int fz = -1;
#pragma unroll 1
      for (int q = 0; q < 32; ++q) {
        const bool act = q < w && fz < 0;  // uniform over the 128 threads
        const float v = (act && !done) ? fabsf(x[0]) : -1.0f;
        const unsigned key = (v >= 0.0f) ? __float_as_uint(v) + 1u : 0u;
        const unsigned wm = __reduce_max_sync(0xffffffffu, key);
        const unsigned wp = __reduce_min_sync(0xffffffffu, key == wm ? (unsigned)pos : 0xffffu);
        float* slot = rows4 + (q & 1) * 128;
        unsigned* rk = red + (q & 1) * 8;
        if (key == wm && pos == (int)wp) {  // the warp's candidate (one lane)
#pragma unroll
          for (int t = 0; t < 32; t += 4)
            *reinterpret_cast<float4*>(slot + warp * 32 + t) =
                make_float4(x[t], x[t + 1], x[t + 2], x[t + 3]);
        }
        if (lane == 0) {
          rk[warp] = wm;
          rk[4 + warp] = wp;
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
        unsigned mx = rk[0], pm = rk[4];
        int ww = 0;
#pragma unroll
        for (int k = 1; k < 4; ++k) {
          const unsigned kk = rk[k], pk = rk[4 + k];
          if (kk > mx || (kk == mx && pk < pm)) {
            mx = kk;
            pm = pk;
            ww = k;
          }
        }
        const bool ok = act && mx > 1u;  // mx <= 1: exactly zero (or NaN) column
        if (act && !ok) fz = q;
        const bool piv = ok && key == mx && pos == (int)pm;
        if (ok && tid == 0) sp[c0 + q] = c0 + (int)pm;
        if (ok && pos == q && !piv) pos = (int)pm;
        if (piv) {
          pos = q;
          done = true;
        }
        // the pivot row, four columns at a time straight into the update
        const float* prow = slot + ww * 32;
        const float4 f0 = *reinterpret_cast<const float4*>(prow);
        const bool elim = ok && !done;
        const float l = x[0] * __frcp_rn(f0.x);
        const float le = elim ? l : 0.0f;
        x[1] = fmaf(-le, f0.y, x[1]);
        x[2] = fmaf(-le, f0.z, x[2]);
        x[3] = fmaf(-le, f0.w, x[3]);
#pragma unroll
        for (int t = 4; t < 32; t += 4) {
          const float4 r4 = *reinterpret_cast<const float4*>(prow + t);
          x[t] = fmaf(-le, r4.x, x[t]);
          x[t + 1] = fmaf(-le, r4.y, x[t + 1]);
          x[t + 2] = fmaf(-le, r4.z, x[t + 2]);
          x[t + 3] = fmaf(-le, r4.w, x[t + 3]);
        }
        if (tid < nrow && q < w) D[(c0 + tid) * kLdD + c0 + q] = elim ? l : x[0];
#pragma unroll
        for (int t = 0; t < 31; ++t) x[t] = x[t + 1];
        x[31] = 0.0f;
      }
      if (fz >= 0 && tid == 0) zero_pivot = c0 + fz;
      asm volatile("bar.sync 1, 128;" ::: "memory");
      // the panel's rows in their final order
#pragma unroll
      for (int t = 0; t < 32; ++t) x[t] = (tid < nrow && t < w) ? D[(c0 + tid) * kLdD + c0 + t] : 0.0f;
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (tid < nrow) {
#pragma unroll
        for (int t = 0; t < 32; ++t)
          if (t < w) D[(c0 + pos) * kLdD + c0 + t] = x[t];
      }
    }
    __syncthreads();
    if (zero_pivot >= 0) {  // uniform exit
      if (tid == 0) {
        a.info[b] = k0 + zero_pivot + 1;
        if (a.iters) a.iters[b] = 0;
      }
      return;
    }
    // the panel's exchanges, in order, on the block's other columns
    for (int c = tid; c < kb; c += 256) {
      if (c >= c0 && c < c0 + w) continue;
      for (int q = c0; q < c0 + w; ++q) {
        const int p = sp[q];
        if (p != q) {
          const float t = D[q * kLdD + c];
          D[q * kLdD + c] = D[p * kLdD + c];
          D[p * kLdD + c] = t;
        }
      }
    }
    __syncthreads();
    const int c1 = c0 + w;
    if (c1 >= kb) break;
    // U12 = L11^{-1} A12 on rows c0..c1-1, columns c1..kb-1 (unit lower L11;
    // here w == 32): a thread per column in registers, right-looking
    for (int c = c1 + tid; c < kb; c += 256) {
      float col[32];
#pragma unroll
      for (int t = 0; t < 32; ++t) col[t] = D[(c0 + t) * kLdD + c];
#pragma unroll
      for (int q = 0; q < 32; ++q)
#pragma unroll
        for (int t = q + 1; t < 32; ++t) col[t] = fmaf(-D[(c0 + t) * kLdD + c0 + q], col[q], col[t]);
#pragma unroll
      for (int t = 1; t < 32; ++t) D[(c0 + t) * kLdD + c] = col[t];
    }
    __syncthreads();
    // trailing block: rows and columns c1..kb-1, D -= L21 U12, 4 x 4 per task
    const int nr = kb - c1, nb4 = (nr + 3) >> 2;
    for (int task = tid; task < nb4 * nb4; task += 256) {
      const int r0 = c1 + 4 * (task / nb4), cc0 = c1 + 4 * (task % nb4);
      float acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) acc[i][jj] = 0.0f;
      for (int t = 0; t < w; ++t) {
        float av[4], bw[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) av[i] = (r0 + i < kb) ? D[(r0 + i) * kLdD + c0 + t] : 0.0f;
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) bw[jj] = (cc0 + jj < kb) ? D[(c0 + t) * kLdD + cc0 + jj] : 0.0f;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) acc[i][jj] = fmaf(av[i], bw[jj], acc[i][jj]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
          if (r0 + i < kb && cc0 + jj < kb) D[(r0 + i) * kLdD + cc0 + jj] -= acc[i][jj];
    }
    __syncthreads();
  }
  if (K >= 1) {
    // A full diagonal tile leaves with its four 32 x 32 diagonal blocks of L and
    // U inverted in place, the form the refinement takes; k_trsm_tc reads them
    // as the diagonal blocks of its triangular inverse.  (Block row 0's, which
    // the step-0 solve still needs as they are, are inverted by k_large_finish.)
    const int warp = tid >> 5, q = warp & 3;  // warps 0-3: L, warps 4-7: U of block q
    invert_triangle32(D + 32 * q * kLdD + 32 * q, kLdD, warp < 4);
    __syncthreads();
  }
  for (int e = tid; e < kBW * kBW; e += 256) {
    const int r = e >> 7, c = e & 127;
    if (r < kb && c < kb) Td[dpos(r, c)] = D[r * kLdD + c];
  }
  int32_t* gpiv = a.piv + vec_off(bt, b);
  if (tid < kb) gpiv[k0 + tid] = k0 + sp[tid];
  // the exchanges made (usually a few), in order, as a list
  int* ex = sp + kBW;  // 2 x kBW ints after the pivots
  __shared__ int nex;
  if (tid == 0) {
    int k = 0;
    for (int q = 0; q < kb; ++q)
      if (sp[q] != q) {
        ex[2 * k] = q;
        ex[2 * k + 1] = sp[q];
        ++k;
      }
    nex = k;
  }
  __syncthreads();
  // ... applied to the columns outside the block (block row K: the finished L
  // to the left, A12 to the right, both untransposed here)
  // exchange by exchange, each thread's columns (at most 9: m <= 2049) all in
  // flight at once
  constexpr int kXc = (PANEL_N_MAX + 1 + 255) / 256;
  for (int x = 0; x < nex; ++x) {
    const int ra = k0 + ex[2 * x], rb = k0 + ex[2 * x + 1];
    float va[kXc], vb[kXc];
#pragma unroll
    for (int j = 0; j < kXc; ++j) {
      const int c = tid + 256 * j;
      const bool on = c < m && (c < k0 || c >= k0 + kb);
      va[j] = on ? F[g.off(ra, c, false)] : 0.0f;
      vb[j] = on ? F[g.off(rb, c, false)] : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < kXc; ++j) {
      const int c = tid + 256 * j;
      if (c < m && (c < k0 || c >= k0 + kb)) {
        F[g.off(ra, c, false)] = vb[j];
        F[g.off(rb, c, false)] = va[j];
      }
    }
  }
}

size_t large_diag_smem() { return (size_t)kBW * kLdD * 4 + 256 * 4 + 16 * 4 + 3 * kBW * 4; }

// U12 = L11^{-1} A12 and L21 = A21 U11^{-1} as products with the explicit
// inverses of the two triangles of the factored diagonal block K.  Per block:
//   1. the block D = L11 \ U11 is staged (a ragged block of e < 128 rows is
//      completed by the identity, whose inverse it leaves alone); thread
//      j < 128 forms column j of L11^{-1} (forward substitution on e_j), thread
//      128 + i row i of U11^{-1} (from X U = I, so each row needs only its own
//      earlier entries); four partial sums per dot product keep the chains
//      short;
//   2. tasks 0..ns-1 are the tiles (K, J > K) of A12, tasks ns..2ns-1 the tiles
//      (I > K, K) of A21 (every block after the first is 128 wide): the tile is
//      staged in shared memory and multiplied by the inverse, 8 x 8 outputs per
//      thread, written straight back to the factor -- U12 transposed (K >= 1),
//      L21 as it is.
// Li holds L11^{-1} transposed (Li[k][t] = (L11^{-1})[t][k]) and Ui holds
// U11^{-1} by rows, both with an odd row stride (conflict-free while they are
// formed); the slab has 16-byte rows for vector reads.
constexpr int kLdI = kBW + 1;
constexpr int kLdX = kBW + 4;

__global__ void __launch_bounds__(256) k_large_trsm(SolveArgs a, int K) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float* X = reinterpret_cast<float*>(smraw);  // kBW x kLdX: D (stride kLdI), then the slab
  float* Li = X + kBW * kLdX;                  // kBW x kLdI
  float* Ui = Li + kBW * kLdI;                 // kBW x kLdI
  float* dinv = Ui + kBW * kLdI;               // kBW
  const Batch& bt = a.bt;
  const int b = bt.order[blockIdx.x];
  int n, m;
  if (!large_live(a, b, n, m)) return;
  TlGeom g;
  g.init(m, bt.mat_off[b]);
  if (K >= g.T - 1) return;  // the last block has no trailing matrix
  const int k0 = g.start(K), kb = g.size(K);
  const int tid = threadIdx.x;
  float* F = a.LU + bt.mat_off[b];
  float* D = X;
  for (int e = tid; e < kBW * kBW; e += 256) {
    const int r = e / kBW, c = e % kBW;
    D[r * kLdI + c] = (r < kb && c < kb) ? F[g.off(k0 + r, k0 + c, false)]
                                         : (r == c ? 1.0f : 0.0f);
  }
  __syncthreads();
  if (tid < kBW) dinv[tid] = 1.0f / D[tid * kLdI + tid];
  __syncthreads();
  // Only the first kb rows and columns of the inverses are used (the products
  // below run over k < kb; X is zero beyond); their entries at t >= kb are zero.
  if (tid < kb) {
    // column j of L11^{-1}: x_j = 1, x_t = -sum_{j <= q < t} L[t][q] x_q
    const int j = tid;
    float* x = Li + j * kLdI;
    for (int t = 0; t < j; ++t) x[t] = 0.0f;
    for (int t = kb; t < kBW; ++t) x[t] = 0.0f;
    x[j] = 1.0f;
    for (int t = j + 1; t < kb; ++t) {
      const float* Lt = D + t * kLdI;
      float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
      int q = j;
      for (; q + 3 < t; q += 4) {
        s0 = fmaf(Lt[q], x[q], s0);
        s1 = fmaf(Lt[q + 1], x[q + 1], s1);
        s2 = fmaf(Lt[q + 2], x[q + 2], s2);
        s3 = fmaf(Lt[q + 3], x[q + 3], s3);
      }
      for (; q < t; ++q) s0 = fmaf(Lt[q], x[q], s0);
      x[t] = -((s0 + s1) + (s2 + s3));
    }
  } else if (tid >= kBW && tid - kBW < kb) {
    // row i of U11^{-1}: y_i = 1 / U_ii, y_t = -(sum_{i <= q < t} y_q U[q][t]) / U_tt
    const int i = tid - kBW;
    float* y = Ui + i * kLdI;
    for (int t = 0; t < i; ++t) y[t] = 0.0f;
    for (int t = kb; t < kBW; ++t) y[t] = 0.0f;
    y[i] = dinv[i];
    for (int t = i + 1; t < kb; ++t) {
      float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
      int q = i;
      for (; q + 3 < t; q += 4) {
        s0 = fmaf(y[q], D[q * kLdI + t], s0);
        s1 = fmaf(y[q + 1], D[(q + 1) * kLdI + t], s1);
        s2 = fmaf(y[q + 2], D[(q + 2) * kLdI + t], s2);
        s3 = fmaf(y[q + 3], D[(q + 3) * kLdI + t], s3);
      }
      for (; q < t; ++q) s0 = fmaf(y[q], D[q * kLdI + t], s0);
      y[t] = -((s0 + s1) + (s2 + s3)) * dinv[t];
    }
  }
  const int ns = g.T - 1 - K;
  const int tx = tid & 15, ty = tid >> 4;
  // The task's tile is read into registers one task ahead (64 values per
  // thread; element e = tid + 256 i is (k, c) = (e / 128, e % 128) of A12 or
  // (r, k) of A21), so that its loads overlap the previous task's products.
  constexpr int kPre = kBW * 128 / 256;
  float pre[kPre];
  auto fetch = [&](int task) {
    const bool cols = task < ns;
    const int JI = K + 1 + (cols ? task : task - ns);
    const int base = g.start(JI);
    const float* Tt = (K == 0) ? nullptr : F + (cols ? g.tile(K, JI) : g.tile(JI, K));
#pragma unroll
    for (int i = 0; i < kPre; ++i) {
      const int e = tid + 256 * i, hi7 = e >> 7, lo7 = e & 127;
      float v = 0.0f;
      if (cols) {  // A12[k0 + k][base + c], k = hi7, c = lo7
        if (hi7 < kb)
          v = (K == 0) ? F[(int64_t)hi7 * m + base + lo7]
                       : Tt[((lo7 >> 5) << 12) + hi7 * 32 + (lo7 & 31)];
      } else {     // A21[base + r][k0 + k], r = hi7, k = lo7
        if (lo7 < kb)
          v = (K == 0) ? F[g.rag(JI, hi7, lo7)] : Tt[((lo7 >> 5) << 12) + hi7 * 32 + (lo7 & 31)];
      }
      pre[i] = v;
    }
  };
  if ((int)blockIdx.y < 2 * ns) fetch(blockIdx.y);
  for (int task = blockIdx.y; task < 2 * ns; task += gridDim.y) {
    const bool cols = task < ns;
    const int JI = K + 1 + (cols ? task : task - ns);  // the tile column J or row I
    const int base = g.start(JI);
    // the tile: (K, J) of A12 or (I, K) of A21; at K = 0 block row 0 (row-major)
    // and the ragged tiles (I, 0)
    float* Tt = (K == 0) ? nullptr : F + (cols ? g.tile(K, JI) : g.tile(JI, K));
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kPre; ++i) {
      const int e = tid + 256 * i, hi7 = e >> 7, lo7 = e & 127;
      // X[k][c] = A12[k0 + k][base + c], or X[k][r] = A21[base + r][k0 + k]
      if (cols)
        X[hi7 * kLdX + lo7] = pre[i];
      else
        X[lo7 * kLdX + hi7] = pre[i];
    }
    __syncthreads();
    if (task + (int)gridDim.y < 2 * ns) fetch(task + gridDim.y);
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
    // rows 4ty.., 64+4ty.. and columns 4tx.., 64+4tx.. of the 128 x 128 result
    if (cols) {
      // U12[t][c] = sum_k (L11^{-1})[t][k] X[k][c]
#pragma unroll 2
      for (int k = 0; k < kb; ++k) {
        const float* lk = Li + k * kLdI;
        float av[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          av[i] = lk[4 * ty + i];
          av[i + 4] = lk[64 + 4 * ty + i];
        }
        const float4 b0 = *reinterpret_cast<const float4*>(X + k * kLdX + 4 * tx);
        const float4 b1 = *reinterpret_cast<const float4*>(X + k * kLdX + 64 + 4 * tx);
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
      }
      if (K == 0) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int t = (i < 4) ? 4 * ty + i : 64 + 4 * ty + i - 4;
          if (t >= kb) continue;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int c = (j < 4) ? 4 * tx + j : 64 + 4 * tx + j - 4;
            F[(int64_t)t * m + base + c] = acc[i][j];
          }
        }
      } else {
        // U12 of tile (K, J) goes back transposed (chunks of 32 rows of U12,
        // column by column): staged as X[c][t], then written in storage order
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int t = (i < 4) ? 4 * ty + i : 64 + 4 * ty + i - 4;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int c = (j < 4) ? 4 * tx + j : 64 + 4 * tx + j - 4;
            X[c * kLdX + t] = acc[i][j];
          }
        }
        __syncthreads();
        for (int p = tid; p < kTlTile; p += 256) {
          const int c = (p & 4095) >> 5, t = ((p >> 12) << 5) + (p & 31);
          Tt[p] = X[c * kLdX + t];
        }
      }
    } else {
      // L21[r][t] = sum_k X[k][r] (U11^{-1})[k][t]
#pragma unroll 2
      for (int k = 0; k < kb; ++k) {
        const float4 a0 = *reinterpret_cast<const float4*>(X + k * kLdX + 4 * ty);
        const float4 a1 = *reinterpret_cast<const float4*>(X + k * kLdX + 64 + 4 * ty);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float* uk = Ui + k * kLdI;
        float bv[8];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          bv[j] = uk[4 * tx + j];
          bv[j + 4] = uk[64 + 4 * tx + j];
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
      }
      // L21 staged as X[r][t], then written in storage order
      __syncthreads();
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = (i < 4) ? 4 * ty + i : 64 + 4 * ty + i - 4;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int t = (j < 4) ? 4 * tx + j : 64 + 4 * tx + j - 4;
          X[r * kLdX + t] = acc[i][j];
        }
      }
      __syncthreads();
      if (K == 0) {
        for (int p = tid; p < kTlB * kb; p += 256) {
          const int r = p / kb, t = p - r * kb;
          F[g.rag(JI, r, t)] = X[r * kLdX + t];
        }
      } else {
        for (int p = tid; p < kTlTile; p += 256) {
          const int r = (p & 4095) >> 5, t = ((p >> 12) << 5) + (p & 31);
          Tt[p] = X[r * kLdX + t];
        }
      }
    }
  }
}

size_t large_trsm_smem() {
  return ((size_t)kBW * kLdX + 2 * (size_t)kBW * kLdI + kBW) * 4;
}

// The U tiles (I, J > I) back from their transposed order to row chunks, in
// place, so that every full tile of the finished factor has the same order.
// The 32 x 32 block (R, C) of a transposed tile (U rows 32 R .., columns
// 32 C ..) is stored column by column at R 4096 + C 1024; in row chunks it is
// stored row by row at C 4096 + R 1024.  A block takes one tile: it stages the
// 64 KB in shared memory (the 32-float columns padded to 33 floats against bank
// conflicts) and writes them back in the new order.  Grid: x = the launch
// position of the airfoil, y = the tile, counted by J then I (tile (I, J) is
// number (J - 1)(J - 2) / 2 + I - 1).
constexpr int kUtThreads = 256;
constexpr size_t kUtSmem = (size_t)16 * 32 * 33 * sizeof(float);

__global__ void __launch_bounds__(kUtThreads, 3) k_tl_untranspose(SolveArgs a) {
  extern __shared__ __align__(16) float S[];
  const Batch& bt = a.bt;
  const int b = bt.order[blockIdx.x];
  int n, m;
  if (!large_live(a, b, n, m)) return;
  TlGeom g;
  g.init(m, bt.mat_off[b]);
  int k = blockIdx.y, J = 2;
  while (J < g.T && k >= J - 1) {
    k -= J - 1;
    ++J;
  }
  if (J >= g.T) return;
  float* t = a.LU + bt.mat_off[b] + g.tile(1 + k, J);
  const float4* t4 = reinterpret_cast<const float4*>(t);
#pragma unroll 8
  for (int p4 = threadIdx.x; p4 < kTlTile / 4; p4 += kUtThreads) {
    const float4 v = t4[p4];
    // floats 4 p4 .. 4 p4 + 3: rows (4 p4) % 32 .. of column (4 p4) / 32
    float* d = S + ((4 * p4) >> 5) * 33 + ((4 * p4) & 31);
    d[0] = v.x;
    d[1] = v.y;
    d[2] = v.z;
    d[3] = v.w;
  }
  __syncthreads();
#pragma unroll 8
  for (int p = threadIdx.x; p < kTlTile; p += kUtThreads) {
    const int C = p >> 12, r = (p >> 5) & 127, c = p & 31;
    t[p] = S[(((r >> 5) * 4 + C) * 32 + c) * 33 + (r & 31)];
  }
}

// The 32 x 32 diagonal blocks of L and U of the first block row inverted in
// place, the form the refinement's triangular sweeps take: ceil(e / 32) blocks
// (row-major, row stride m; the last one e - 32 floor((e - 1) / 32) wide).
// The full diagonal tiles' four blocks each are inverted by k_large_diag.
// Each warp stages a block in shared memory, inverts both triangles there and
// writes the block back.
__global__ void __launch_bounds__(256) k_large_finish(SolveArgs a) {
  __shared__ float S[8][32 * 33];
  const Batch& bt = a.bt;
  const int b = bt.order[blockIdx.x];
  int n, m;
  if (!large_live(a, b, n, m)) return;
  float* F = a.LU + bt.mat_off[b];
  TlGeom g;
  g.init(m, bt.mat_off[b]);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int G0 = (g.e + 31) >> 5;
  float* W = S[warp];
  for (int d = blockIdx.y * 8 + warp; d < G0; d += 8 * (int)gridDim.y) {
    float* B = F + (int64_t)(32 * d) * m + 32 * d;
    const int ld = m, kb = min(32, g.e - 32 * d);
    float v[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) v[r] = (r < kb && lane < kb) ? B[(int64_t)r * ld + lane] : 0.0f;
#pragma unroll
    for (int r = 0; r < 32; ++r) W[r * 33 + lane] = v[r];
    __syncwarp();
    invert_block(W, 33, kb);
    for (int r = 0; r < kb; ++r)
      if (lane < kb) B[(int64_t)r * ld + lane] = W[r * 33 + lane];
    __syncwarp();
  }
}

// Polls of each pipeline wait in k_update_tc before it gives up (a wait that
// runs out marks the airfoil PANEL_INFO_DEVICE_TIMEOUT instead of hanging).
// The default is far above any wait of a working pipeline; panel_debug_wait_limit
// lowers it to exercise that path.
constexpr long long kDefaultWaitLimit = 1ll << 22;
static std::atomic<long long> g_wait_limit{kDefaultWaitLimit};

long long set_wait_limit(long long polls) {
  return g_wait_limit.exchange(polls > 0 ? polls : kDefaultWaitLimit);
}

// gridDim.y per airfoil: enough blocks for ~`per_sm` per SM over the whole batch.
static int split_for(int B, int per_airfoil_max, int per_sm = 4) {
  const int sms = sm_count() > 0 ? sm_count() : 152;
  const int want = (per_sm * sms + B - 1) / max(B, 1);
  return max(1, min(want, per_airfoil_max));
}

cudaError_t launch_lu_large(const SolveArgs& a, cudaStream_t s) {
  const Batch& bt = a.bt;
  const int B = bt.B, m_max = bt.n_max + 1;
  if (B == 0 || m_max <= kLargeM) return cudaSuccess;
  if (B > 65535) return cudaErrorInvalidValue;
  const int T_max = (m_max + kTlB - 1) / kTlB;
  cudaError_t e;
  UpdateMap tmap;
  e = make_update_map(a.LU, (uint64_t)B * (uint64_t)m_max * (uint64_t)m_max, &tmap);
  if (e != cudaSuccess) return e;
  e = ensure_smem(k_large_diag, large_diag_smem());
  if (e != cudaSuccess) return e;
  e = ensure_smem(k_large_trsm, large_trsm_smem());
  if (e != cudaSuccess) return e;
  e = ensure_update_smem();
  if (e != cudaSuccess) return e;
  e = ensure_smem(k_tl_untranspose, kUtSmem);
  if (e != cudaSuccess) return e;
  const long long spin = g_wait_limit.load();
  // a block per block row: the work of one block is at most 128 rows of the
  // largest airfoil, so the batch's last wave stays short
  k_large_init<<<dim3(B, T_max), kInitThreads, 0, s>>>(a);
  for (int K = 0; K < T_max; ++K) {
    k_large_diag<<<B, 256, large_diag_smem(), s>>>(a, K);
    const int ns = T_max - 1 - K;  // blocks after K in the largest airfoil
    if (ns <= 0) break;
    if (K == 0) {
      k_large_trsm<<<dim3(B, split_for(B, 2 * ns)), 256, large_trsm_smem(), s>>>(a, K);
    } else {
      e = launch_trsm_tc(a, tmap, K, split_for(B, ns, 1), spin, s);
      if (e != cudaSuccess) return e;
    }
    e = launch_update_tc(a, tmap, K, split_for(B, ns * ns, 1), spin, s);
    if (e != cudaSuccess) return e;
  }
  const int tiles = (T_max - 1) * (T_max - 2) / 2;  // U tiles of the largest airfoil
  if (tiles > 0) k_tl_untranspose<<<dim3(B, tiles), kUtThreads, kUtSmem, s>>>(a);
  k_large_finish<<<dim3(B, 1), 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace panel
