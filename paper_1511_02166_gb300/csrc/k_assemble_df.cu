// k_assemble_df.cu -- mixed-precision assembly: the bordered system of Section 2
// in double-float, stored as two float32 planes A = A_hi + A_lo.
//
// One block per airfoil (launched in size order).  Prologue: validate the
// geometry (FP64), build the per-panel constants in shared memory and stage the
// log/atan tables.  Main loop: pairs (j, i) in row-major order, consecutive
// threads on consecutive columns, so each warp writes contiguous runs of both
// planes.  The right-hand side phi_v(x_{j+1/2}) is FP64.
#include "panel_common.cuh"
#include "panel_df.cuh"

namespace panel {

__global__ void __launch_bounds__(256) k_assemble_df(Batch bt, const double* __restrict__ alpha,
                                                     const double* __restrict__ vinf,
                                                     float* __restrict__ A_hi,
                                                     float* __restrict__ A_lo,
                                                     double* __restrict__ rhs,
                                                     int32_t* __restrict__ info, int rounds) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int ld = bt.n_max;
  float4* tlog = reinterpret_cast<float4*>(smraw);                   // 257
  float2* tatan = reinterpret_cast<float2*>(tlog + 257);             // 33 (+1 pad)
  double* xs = reinterpret_cast<double*>(tatan + 34);                // n_max
  double* ys = xs + ld;                                              // n_max
  double* scratch = ys + ld;                                         // 32
  float* pc = reinterpret_cast<float*>(scratch + 32);                // 20 * n_max

  const int b = bt.order[blockIdx.x];
  const int n = airfoil_n(bt, b);
  const int m = n + 1;
  if (n > ld) {
    if (threadIdx.x == 0) info[b] = PANEL_INFO_TOO_LARGE;
    return;
  }
  const double* nodes = bt.nodes + 2 * bt.node_off[b];
  const int st = load_and_check_geometry(nodes, n, xs, ys, scratch);
  if (threadIdx.x == 0) info[b] = st;
  if (st != 0) return;
  df_stage_tables(tlog, tatan);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const int k1 = (k + 1 == n) ? 0 : k + 1;
    panel_constants(pc, ld, k, xs[k], ys[k], xs[k1], ys[k1]);
  }
  const double v = vinf ? vinf[b] : 1.0;
  const double ca = cos(alpha[b]), sa = sin(alpha[b]);
  double* rb = rhs + vec_off(bt, b);
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    if (j < n) {
      const int j1 = (j + 1 == n) ? 0 : j + 1;
      rb[j] = v * (0.5 * (ys[j] + ys[j1]) * ca - 0.5 * (xs[j] + xs[j1]) * sa);
    } else {
      rb[j] = 0.0;
    }
  }
  __syncthreads();

  const int64_t base = bt.mat_off[b];
  float* Ah = A_hi + base;
  float* Al = A_lo + base;
  // border: C column of ones and the Kutta row (gamma_0 + gamma_{n-1} = 0)
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    if (j < n) {
      Ah[(int64_t)j * m + n] = 1.0f;
      Al[(int64_t)j * m + n] = 0.0f;
    }
    Ah[(int64_t)n * m + j] = (j == 0 || j == n - 1) ? 1.0f : 0.0f;
    Al[(int64_t)n * m + j] = 0.0f;
  }
  // pairs (j, i), j, i < n, row-major over the threads of the block, in rounds of
  // `rounds` pairs per thread: the far-field pairs are evaluated at once, the
  // near-field ones (|P| < 4 L) queued and then evaluated by all threads
  // together, so that no warp runs both forms for a mix of its lanes
  // (rounds == 0: both forms inline, for the largest airfoils, whose one block
  // per SM cannot afford the barriers)
  int* queue = reinterpret_cast<int*>(pc + kPanelFields * ld);  // blockDim.x * rounds
  int* qn = queue + blockDim.x * rounds;
  const int stride = blockDim.x;
  const int dj = stride / n, di = stride % n;
  int j = threadIdx.x / n, i = threadIdx.x % n;
  point3 pj = load_point(pc, ld, j < n ? j : 0);
  if (rounds == 0) {
    while (j < n) {
      const df2 g = panel_G_df<0>(pair_geom(pj, pc, ld, i), pc, ld, i, tlog, tatan);
      const int64_t e = (int64_t)j * m + i;
      Ah[e] = -g.hi;
      Al[e] = -g.lo;
      const int jo = j;
      i += di;
      j += dj;
      if (i >= n) {
        i -= n;
        ++j;
      }
      if (j != jo && j < n) pj = load_point(pc, ld, j);
    }
    return;
  }
  const int np = n * n;
  for (int p0 = 0; p0 < np; p0 += stride * rounds) {
    if (threadIdx.x == 0) *qn = 0;
    __syncthreads();
    for (int r = 0; r < rounds && j < n; ++r) {
      const PairGeom gm = pair_geom(pj, pc, ld, i);
      if (gm.far()) {
        const df2 g = panel_G_df<1>(gm, pc, ld, i, tlog, tatan);
        const int64_t e = (int64_t)j * m + i;
        Ah[e] = -g.hi;
        Al[e] = -g.lo;
      } else {
        queue[atomicAdd(qn, 1)] = j * n + i;
      }
      const int jo = j;
      i += di;
      j += dj;
      if (i >= n) {
        i -= n;
        ++j;
      }
      if (j != jo && j < n) pj = load_point(pc, ld, j);
    }
    __syncthreads();
    const int cnt = *qn;
    for (int t = threadIdx.x; t < cnt; t += stride) {
      const int pq = queue[t];
      const int jq = pq / n, iq = pq - jq * n;
      const PairGeom gm = pair_geom(load_point(pc, ld, jq), pc, ld, iq);
      const df2 g = panel_G_df<2>(gm, pc, ld, iq, tlog, tatan);
      const int64_t e = (int64_t)jq * m + iq;
      Ah[e] = -g.hi;
      Al[e] = -g.lo;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// The same matrix with each far-field pair's shared work done once for both
// of its entries.  For the control points c_j, c_i (the panel midpoints) the
// entries (j, i) and (i, j) have P = c_j - c_i and -P: |P|^2, 1/|P|^2, log|P|
// and P^2 are the same for both, exactly (the split coordinates make -P the
// exact negation of P); only the panel's orientation, length and scale differ
// (panel_G_far).  A warp takes a 32 x 32 tile of rows j and columns i (lane =
// column) and its mirror tile: the entry (j, i) is written with the warp's
// lanes on consecutive columns, the mirror entry (i, j) down a column.  Near
// pairs (either direction may be near on its own) take the closed form of
// panel_G_df.  Every entry is computed by the same operations as in
// k_assemble_df, so the two kernels give the same matrix bit for bit.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_assemble_df_sym(Batch bt, const double* __restrict__ alpha,
                                                         const double* __restrict__ vinf,
                                                         float* __restrict__ A_hi,
                                                         float* __restrict__ A_lo,
                                                         double* __restrict__ rhs,
                                                         int32_t* __restrict__ info) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int ld = bt.n_max;
  float4* tlog = reinterpret_cast<float4*>(smraw);                   // 257
  float2* tatan = reinterpret_cast<float2*>(tlog + 257);             // 33 (+1 pad)
  double* xs = reinterpret_cast<double*>(tatan + 34);                // n_max
  double* ys = xs + ld;                                              // n_max
  double* scratch = ys + ld;                                         // 32
  float* pc = reinterpret_cast<float*>(scratch + 32);                // kPanelFields * n_max

  const int b = bt.order[blockIdx.x];
  const int n = airfoil_n(bt, b);
  const int m = n + 1;
  if (n > ld) {
    if (threadIdx.x == 0) info[b] = PANEL_INFO_TOO_LARGE;
    return;
  }
  const double* nodes = bt.nodes + 2 * bt.node_off[b];
  const int st = load_and_check_geometry(nodes, n, xs, ys, scratch);
  if (threadIdx.x == 0) info[b] = st;
  if (st != 0) return;
  df_stage_tables(tlog, tatan);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const int k1 = (k + 1 == n) ? 0 : k + 1;
    panel_constants(pc, ld, k, xs[k], ys[k], xs[k1], ys[k1]);
  }
  const double v = vinf ? vinf[b] : 1.0;
  const double ca = cos(alpha[b]), sa = sin(alpha[b]);
  double* rb = rhs + vec_off(bt, b);
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    if (j < n) {
      const int j1 = (j + 1 == n) ? 0 : j + 1;
      rb[j] = v * (0.5 * (ys[j] + ys[j1]) * ca - 0.5 * (xs[j] + xs[j1]) * sa);
    } else {
      rb[j] = 0.0;
    }
  }
  __syncthreads();

  const int64_t base = bt.mat_off[b];
  float* Ah = A_hi + base;
  float* Al = A_lo + base;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    if (j < n) {
      Ah[(int64_t)j * m + n] = 1.0f;
      Al[(int64_t)j * m + n] = 0.0f;
    }
    Ah[(int64_t)n * m + j] = (j == 0 || j == n - 1) ? 1.0f : 0.0f;
    Al[(int64_t)n * m + j] = 0.0f;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nt = (n + 31) >> 5;
  for (int t = warp; t < nt * nt; t += nw) {
    const int bj = t / nt, bi = t - bj * nt;
    if (bj > bi) continue;
    const int i = 32 * bi + lane;
    const bool iok = i < n;
    const int ii = iok ? i : n - 1;
    const float Li = pc[kL * ld + ii];
    const int jn = min(32, n - 32 * bj);
    for (int r = 0; r < jn; ++r) {
      const int j = 32 * bj + r;
      const PairGeom gm = pair_geom(load_point(pc, ld, j), pc, ld, ii);  // P = c_j - c_i
      if (bj == bi) {  // the diagonal tile: every pair from its own row
        if (iok) {
          const df2 g = panel_G_df<0>(gm, pc, ld, ii, tlog, tatan);
          Ah[(int64_t)j * m + i] = -g.hi;
          Al[(int64_t)j * m + i] = -g.lo;
        }
        continue;
      }
      const float Lj = pc[kL * ld + j];
      const bool far_ji = gm.rho2.hi >= 16.0f * Li * Li;  // entry (j, i), panel i
      const bool far_ij = gm.rho2.hi >= 16.0f * Lj * Lj;  // entry (i, j), panel j
      df2 g_ji, g_ij;
      if (__any_sync(0xffffffffu, far_ji || far_ij)) {
        const df2 X = df_sub(gm.px2, gm.py2);
        df2 Y = df_mul(gm.px, gm.py);
        Y.hi *= 2.0f;
        Y.lo *= 2.0f;
        const df2 inv = df_rcp(gm.rho2);
        const df2 inv2 = df_sqr(inv);
        df2 lg = df_log(gm.rho2, tlog);
        lg.hi *= 0.5f;
        lg.lo *= 0.5f;
        g_ji = panel_G_far(X, Y, inv, inv2, lg, pc, ld, ii, Li);
        g_ij = panel_G_far(X, Y, inv, inv2, lg, pc, ld, j, Lj);
      }
      if (!far_ji) g_ji = panel_G_df<2>(gm, pc, ld, ii, tlog, tatan);
      if (!far_ij) {
        PairGeom gr = gm;  // the pair seen from c_i: -P
        gr.px = df_neg(gm.px);
        gr.py = df_neg(gm.py);
        gr.Lh = Lj;
        g_ij = panel_G_df<2>(gr, pc, ld, j, tlog, tatan);
      }
      if (iok) {
        Ah[(int64_t)j * m + i] = -g_ji.hi;
        Al[(int64_t)j * m + i] = -g_ji.lo;
        Ah[(int64_t)i * m + j] = -g_ij.hi;
        Al[(int64_t)i * m + j] = -g_ij.lo;
      }
    }
  }
}

// Pairs per thread between two near-field passes (the queue holds 256 x rounds
// pair indices, 16 KB); 0 above 1024 panels: there the panel constants take
// most of the shared memory, one block fits an SM, and the barriers of the
// deferred pass cost more than the mixed branches (C5 assembly 36 -> 49 ms).
// `sel` (the PANEL_TUNE_ROUNDS field of the flags) overrides it: 1 inline, 2..5
// rounds of 4, 8, 16 or 32 pairs; 0 keeps the default.
static int assemble_rounds(int n_max, int sel) {
  static const int kSel[6] = {-1, 0, 4, 8, 16, 32};
  if (sel >= 1 && sel <= 5) return kSel[sel];
  return n_max <= 1024 ? 16 : 0;
}
// sel 6 (or the choice by size above 1024 panels): k_assemble_df_sym
static bool assemble_sym(int n_max, int sel) { return sel == 6 || (sel == 0 && n_max > 1024); }

static size_t assemble_df_smem(int n_max, int rounds) {
  return 257 * 16 + 34 * 8 + (size_t)(2 * n_max + 32) * 8 + (size_t)kPanelFields * n_max * 4 +
         ((size_t)256 * rounds + 1) * 4;
}

cudaError_t launch_assemble_df(const Batch& bt, const double* alpha, const double* vinf,
                               float* A_hi, float* A_lo, double* rhs, int32_t* info,
                               cudaStream_t s, int rounds_sel) {
  if (assemble_sym(bt.n_max, rounds_sel)) {
    const size_t smem = assemble_df_smem(bt.n_max, 0);
    cudaError_t e = ensure_smem(k_assemble_df_sym, smem);
    if (e != cudaSuccess) return e;
    // 16 warps: one block fills an SM's shared memory above 1024 panels
    k_assemble_df_sym<<<bt.B, 512, smem, s>>>(bt, alpha, vinf, A_hi, A_lo, rhs, info);
    return cudaGetLastError();
  }
  int rounds = assemble_rounds(bt.n_max, rounds_sel);
  // a requested queue that does not fit the shared memory falls back to the default
  if (assemble_df_smem(bt.n_max, rounds) > 232448) rounds = assemble_rounds(bt.n_max, 0);
  const size_t smem = assemble_df_smem(bt.n_max, rounds);
  cudaError_t e = ensure_smem(k_assemble_df, smem);
  if (e != cudaSuccess) return e;
  k_assemble_df<<<bt.B, 256, smem, s>>>(bt, alpha, vinf, A_hi, A_lo, rhs, info, rounds);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Diagnostic evaluation of the double-float primitives on arrays (panel_df_eval)
// ---------------------------------------------------------------------------
__global__ void k_df_eval(int op, int count, const double* __restrict__ a,
                          const double* __restrict__ b, double* __restrict__ out) {
  __shared__ float4 tlog[257];
  __shared__ float2 tatan[34];
  __shared__ float pc[kPanelFields * 256];  // 22.5 KB
  df_stage_tables(tlog, tatan);
  __syncthreads();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  if (op == 0) {
    out[k] = df_to_double(df_log(df_from_double(a[k]), tlog));
  } else if (op == 1) {
    out[k] = df_to_double(df_atan2(df_from_double(a[k]), df_from_double(b[k]), tatan));
  } else {
    // op 2: A coefficient -G for control point a[2k..] and panel b[4k..4k+3]
    const int t = threadIdx.x;
    panel_constants(pc, 256, t, b[4 * k], b[4 * k + 1], b[4 * k + 2], b[4 * k + 3]);
    const df2 g = panel_G_df(make_point(a[2 * k], a[2 * k + 1]), pc, 256, t, tlog, tatan);
    out[k] = -df_to_double(g);
  }
}

cudaError_t launch_df_eval(int op, int count, const double* a, const double* b, double* out,
                           cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  k_df_eval<<<(count + 255) / 256, 256, 0, s>>>(op, count, a, b, out);
  return cudaGetLastError();
}

}  // namespace panel
