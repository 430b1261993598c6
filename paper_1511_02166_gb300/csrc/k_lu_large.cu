// k_lu_large.cu -- FP32 LU of large airfoils (m = n + 1 > kLargeM) for the
// mixed-precision path: blocked right-looking elimination, step-synchronous
// across the batch, so that each block column is spread over many blocks
// instead of one block per airfoil.
//
// Per block column k0 (kBW = 128 wide) three launches:
//   k_large_diag    one block per airfoil: LU of the kBW x kBW diagonal block D
//                   in shared memory, with the pivot search restricted to the
//                   rows of D; its row exchanges are applied to the rest of
//                   those rows.
//   k_large_trsm    U12 = L11^{-1} A12 and L21 = A21 U11^{-1}: the two
//                   triangles of the diagonal block are inverted in shared
//                   memory, then 128-wide slabs are multiplied by them.
//   k_update_tc     A22 -= L21 U12 in 128 x 128 tiles on the tcgen05 tensor
//                   cores (k_update_tc.cu).
// Each of the three takes gridDim.y blocks per airfoil striding over its
// slabs / tiles, so a batch of few airfoils still fills the GPU.
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
// The finished factor has the layout of the one-block kernels: P A = L U in
// the caller's LU buffer (ld = m), pivots as sequential exchanges, and the
// 32 x 32 diagonal blocks of L and U replaced by their inverses.
#include <atomic>

#include "lu_mixed.cuh"

namespace panel {

constexpr int kBW = 128;      // block column width
constexpr int kLdD = kBW + 1;

size_t lu_large_min_m() { return kLargeM + 1; }

__device__ __forceinline__ bool large_live(const SolveArgs& a, int b, int& n, int& m) {
  n = airfoil_n(a.bt, b);
  m = n + 1;
  return m > kLargeM && n <= a.bt.n_max && a.info[b] == 0;
}

// Scaled copy A_hi -> LU (border row and column times s); rows strided over
// gridDim.y blocks per airfoil.
__global__ void __launch_bounds__(256) k_large_init(SolveArgs a) {
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
  const float sf = (float)border_scale(Ah, n, m, red);
  for (int r = blockIdx.y; r < m; r += gridDim.y) {
    const float* src = Ah + r * m;
    float* dst = F + r * m;
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
      const float v = src[c];
      dst[c] = ((c == n && r < n) || r == n) ? v * sf : v;
    }
  }
}

// LU of the diagonal block with partial pivoting inside the block.
__global__ void __launch_bounds__(256) k_large_diag(SolveArgs a, int k0) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float* D = reinterpret_cast<float*>(smraw);          // kBW x kLdD
  int* sp = reinterpret_cast<int*>(D + kBW * kLdD);    // kBW
  const Batch& bt = a.bt;
  const int b = bt.order[blockIdx.x];
  int n, m;
  if (!large_live(a, b, n, m) || k0 >= m) return;
  const int kb = min(kBW, m - k0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float* F = a.LU + bt.mat_off[b];
  for (int e = tid; e < kBW * kBW; e += 256) {
    const int r = e / kBW, c = e % kBW;
    D[r * kLdD + c] = (r < kb && c < kb) ? F[(k0 + r) * m + k0 + c] : 0.0f;
  }
  __syncthreads();
  for (int q = 0; q < kb; ++q) {
    if (warp == 0) {
      // argmax |D[r][q]| over the rows q..kb-1, lowest row on ties
      float bv = -1.0f;
      int br = kBW;
#pragma unroll
      for (int t = 0; t < kBW / 32; ++t) {
        const int r = lane + 32 * t;
        const float v = (r >= q && r < kb) ? fabsf(D[r * kLdD + q]) : -1.0f;
        if (v > bv) {
          bv = v;
          br = r;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int orr = __shfl_xor_sync(0xffffffffu, br, o);
        if (ov > bv || (ov == bv && orr < br)) {
          bv = ov;
          br = orr;
        }
      }
      if (lane == 0) sp[q] = (br < kb) ? br : q;
    }
    __syncthreads();
    const int p = sp[q];
    if (!(fabsf(D[p * kLdD + q]) > 0.0f)) {  // exact zero (or NaN) pivot: uniform exit
      if (tid == 0) {
        a.info[b] = k0 + q + 1;
        if (a.iters) a.iters[b] = 0;
      }
      return;
    }
    if (p != q && tid < kBW) {
      const float t = D[q * kLdD + tid];
      D[q * kLdD + tid] = D[p * kLdD + tid];
      D[p * kLdD + tid] = t;
    }
    __syncthreads();
    const float inv = 1.0f / D[q * kLdD + q];
    for (int r = q + 1 + warp; r < kb; r += 8) {
      const float l = D[r * kLdD + q] * inv;
      for (int c = q + 1 + lane; c < kb; c += 32)
        D[r * kLdD + c] = fmaf(-l, D[q * kLdD + c], D[r * kLdD + c]);
      __syncwarp();
      if (lane == 0) D[r * kLdD + q] = l;
    }
    __syncthreads();
  }
  for (int e = tid; e < kb * kb; e += 256) {
    const int r = e / kb, c = e % kb;
    F[(k0 + r) * m + k0 + c] = D[r * kLdD + c];
  }
  int32_t* gpiv = a.piv + vec_off(bt, b);
  if (tid < kb) gpiv[k0 + tid] = k0 + sp[tid];
  // the same exchanges, in order, on the columns outside the block
  for (int c = tid; c < m; c += 256) {
    if (c >= k0 && c < k0 + kb) continue;
    for (int q = 0; q < kb; ++q) {
      const int p = sp[q];
      if (p != q) {
        float* x = F + (k0 + q) * m + c;
        float* y = F + (k0 + p) * m + c;
        const float t = *x;
        *x = *y;
        *y = t;
      }
    }
  }
}

size_t large_diag_smem() { return (size_t)kBW * kLdD * 4 + kBW * 4; }

// U12 = L11^{-1} A12 and L21 = A21 U11^{-1} as products with the explicit
// inverses of the two triangles of the factored diagonal block.  Per block:
//   1. the block D = L11 \ U11 is staged; thread j < 128 forms column j of
//      L11^{-1} (forward substitution on e_j), thread 128 + i row i of
//      U11^{-1} (from X U = I, so each row needs only its own earlier
//      entries); four partial sums per dot product keep the chains short;
//   2. tasks 0..ns-1 are 128-column slabs of A12, tasks ns..2ns-1 128-row
//      slabs of A21: the slab is staged in shared memory and multiplied by the
//      inverse, 8 x 8 outputs per thread, written straight back to the factor.
// Li holds L11^{-1} transposed (Li[k][t] = (L11^{-1})[t][k]) and Ui holds
// U11^{-1} by rows, both with an odd row stride (conflict-free while they are
// formed); the slab has 16-byte rows for vector reads.
constexpr int kLdI = kBW + 1;
constexpr int kLdX = kBW + 4;

__global__ void __launch_bounds__(256) k_large_trsm(SolveArgs a, int k0) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float* X = reinterpret_cast<float*>(smraw);  // kBW x kLdX: D (stride kLdI), then the slab
  float* Li = X + kBW * kLdX;                  // kBW x kLdI
  float* Ui = Li + kBW * kLdI;                 // kBW x kLdI
  float* dinv = Ui + kBW * kLdI;               // kBW
  const Batch& bt = a.bt;
  const int b = bt.order[blockIdx.x];
  int n, m;
  if (!large_live(a, b, n, m)) return;
  const int k1 = k0 + kBW;  // a block column narrower than kBW is the last one
  if (k1 >= m) return;
  const int tid = threadIdx.x;
  float* F = a.LU + bt.mat_off[b];
  float* D = X;
  for (int e = tid; e < kBW * kBW; e += 256) {
    const int r = e / kBW, c = e % kBW;
    D[r * kLdI + c] = F[(k0 + r) * m + k0 + c];
  }
  __syncthreads();
  if (tid < kBW) dinv[tid] = 1.0f / D[tid * kLdI + tid];
  __syncthreads();
  if (tid < kBW) {
    // column j of L11^{-1}: x_j = 1, x_t = -sum_{j <= q < t} L[t][q] x_q
    const int j = tid;
    float* x = Li + j * kLdI;
    for (int t = 0; t < j; ++t) x[t] = 0.0f;
    x[j] = 1.0f;
    for (int t = j + 1; t < kBW; ++t) {
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
  } else {
    // row i of U11^{-1}: y_i = 1 / U_ii, y_t = -(sum_{i <= q < t} y_q U[q][t]) / U_tt
    const int i = tid - kBW;
    float* y = Ui + i * kLdI;
    for (int t = 0; t < i; ++t) y[t] = 0.0f;
    y[i] = dinv[i];
    for (int t = i + 1; t < kBW; ++t) {
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
  const int rest = m - k1, ns = (rest + 127) >> 7;
  const int tx = tid & 15, ty = tid >> 4;
  for (int task = blockIdx.y; task < 2 * ns; task += gridDim.y) {
    const bool cols = task < ns;
    const int base = k1 + (cols ? task : task - ns) * 128;
    const int cnt = min(128, m - base);
    __syncthreads();
    if (cols) {
      // X[k][c] = A12[k0 + k][base + c]
      for (int e = tid; e < kBW * 128; e += 256) {
        const int k = e >> 7, c = e & 127;
        X[k * kLdX + c] = (c < cnt) ? F[(k0 + k) * m + base + c] : 0.0f;
      }
    } else {
      // X[k][r] = A21[base + r][k0 + k]
      for (int e = tid; e < 128 * kBW; e += 256) {
        const int r = e / kBW, k = e % kBW;
        X[k * kLdX + r] = (r < cnt) ? F[(base + r) * m + k0 + k] : 0.0f;
      }
    }
    __syncthreads();
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
    // rows 4ty.., 64+4ty.. and columns 4tx.., 64+4tx.. of the 128 x 128 result
    if (cols) {
      // U12[t][c] = sum_k (L11^{-1})[t][k] X[k][c]
#pragma unroll 2
      for (int k = 0; k < kBW; ++k) {
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
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int t = (i < 4) ? 4 * ty + i : 64 + 4 * ty + i - 4;
        float* row = F + (k0 + t) * m + base;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int c = (j < 4) ? 4 * tx + j : 64 + 4 * tx + j - 4;
          if (c < cnt) row[c] = acc[i][j];
        }
      }
    } else {
      // L21[r][t] = sum_k X[k][r] (U11^{-1})[k][t]
#pragma unroll 2
      for (int k = 0; k < kBW; ++k) {
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
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = (i < 4) ? 4 * ty + i : 64 + 4 * ty + i - 4;
        if (r >= cnt) continue;
        float* row = F + (base + r) * m + k0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int t = (j < 4) ? 4 * tx + j : 64 + 4 * tx + j - 4;
          row[t] = acc[i][j];
        }
      }
    }
  }
}

size_t large_trsm_smem() {
  return ((size_t)kBW * kLdX + 2 * (size_t)kBW * kLdI + kBW) * 4;
}

__global__ void __launch_bounds__(256) k_large_finish(SolveArgs a) {
  const Batch& bt = a.bt;
  const int b = bt.order[blockIdx.x];
  int n, m;
  if (!large_live(a, b, n, m)) return;
  invert_diagonal_blocks(a.LU + bt.mat_off[b], m, m);
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

// gridDim.y per airfoil: enough blocks for ~4 per SM over the whole batch.
static int split_for(int B, int per_airfoil_max) {
  const int want = (4 * 152 + B - 1) / max(B, 1);
  return max(1, min(want, per_airfoil_max));
}

cudaError_t launch_lu_large(const SolveArgs& a, cudaStream_t s) {
  const Batch& bt = a.bt;
  const int B = bt.B, m_max = bt.n_max + 1;
  if (B == 0 || m_max <= kLargeM) return cudaSuccess;
  cudaError_t e;
  e = ensure_smem(k_large_diag, large_diag_smem());
  if (e != cudaSuccess) return e;
  e = ensure_smem(k_large_trsm, large_trsm_smem());
  if (e != cudaSuccess) return e;
  e = ensure_smem(k_update_tc, update_tc_smem());
  if (e != cudaSuccess) return e;
  const long long spin = g_wait_limit.load();
  k_large_init<<<dim3(B, split_for(B, 64)), 256, 0, s>>>(a);
  for (int k0 = 0; k0 < m_max; k0 += kBW) {
    k_large_diag<<<B, 256, large_diag_smem(), s>>>(a, k0);
    const int rest = m_max - (k0 + kBW);
    if (rest <= 0) break;
    const int ns = (rest + 127) / 128;
    k_large_trsm<<<dim3(B, split_for(B, 2 * ns)), 256, large_trsm_smem(), s>>>(a, k0);
    k_update_tc<<<dim3(B, split_for(B, ns * ns)), 288, update_tc_smem(), s>>>(a, k0, spin);
  }
  k_large_finish<<<B, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace panel
