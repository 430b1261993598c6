// capi.cu -- the extern "C" entry points declared in include/panel.h.
//
// Host-side argument validation, then stream-ordered kernel launches.  No
// allocation, no synchronisation.
#include <algorithm>
#include <numeric>
#include <vector>

#include "panel_common.cuh"

namespace panel {
cudaError_t launch_assemble_f64(const Batch&, const double*, const double*, double*, double*,
                                int32_t*, cudaStream_t);
cudaError_t launch_solve_f64(const Batch&, const double*, double*, int32_t*, const double*,
                             const double*, const double*, double*, double*, int32_t*, int32_t*,
                             cudaStream_t);
cudaError_t launch_adjoint_f64(const Batch&, const double*, const int32_t*, const double*,
                               const double*, double*, const double*, const double*,
                               const double*, const double*, double*, const int32_t*,
                               cudaStream_t);
cudaError_t launch_forces(const Batch&, const double*, const double*, const double*,
                          const double*, const int32_t*, double*, double*, double*, double*,
                          cudaStream_t);
cudaError_t launch_assemble_df(const Batch&, const double*, const double*, float*, float*,
                               double*, int32_t*, cudaStream_t, int rounds_sel = 0);
cudaError_t launch_lu_mixed(const Batch&, const float*, float*, int32_t*, int32_t*, int32_t*,
                            bool, cudaStream_t, int lu_kind = 0);
cudaError_t launch_ir_mixed(const Batch&, const float*, const float*, const float*,
                            const int32_t*, const double*, const double*, const double*, double*,
                            double*, int, double, int32_t*, int32_t*, cudaStream_t,
                            int rhs_kind = 0, int ir_shape = 0);
cudaError_t launch_ga_sample(int, int, int, const double*, const double*, double*, cudaStream_t);
cudaError_t launch_ga_step(int, int, int, double, double, const double*, const double*,
                           const double*, const double*, const double*, const double*, double*,
                           cudaStream_t);
int ga_max_tournament();
cudaError_t launch_ga_genome_grad(int, int, int, const double*, double, const double*,
                                  const double*, double*, double*, cudaStream_t);
cudaError_t launch_polar_cl(const Batch&, const double*, const double*, const double*,
                            const double*, int, const double*, const int32_t*, double*,
                            cudaStream_t);
cudaError_t launch_df_eval(int, int, const double*, const double*, double*, cudaStream_t);
cudaError_t launch_viscous(const Batch&, const double*, const double*, const double*,
                           const double*, const double*, const int32_t*, const double*, double*,
                           double*, double*, double*, double*, int32_t*, cudaStream_t);
size_t adjoint_df_smem(int n_max);
constexpr size_t kMaxDynSmem = 232448;
cudaError_t launch_adjoint_df(const Batch&, const double*, const double*, const double*,
                              const double*, const double*, const double*, double*,
                              const int32_t*, cudaStream_t, bool lam_weighted = false);
long long set_wait_limit(long long polls);
cudaError_t launch_ir_vjp(const Batch&, const float*, const float*, const float*,
                          const int32_t*, const double*, const double*, const double*,
                          const double*, const double*, const double*, double*, int, double,
                          int32_t*, cudaStream_t);
}  // namespace panel

using panel::Batch;

namespace {

int mode_of(int flags) {
  const int m = flags & (PANEL_FP64 | PANEL_MIXED);
  if (m == PANEL_FP64 || m == PANEL_MIXED) return m;
  return 0;
}

int tune_ir(int flags) { return (flags >> PANEL_TUNE_IR_SHIFT) & 7; }
int tune_rounds(int flags) { return (flags >> PANEL_TUNE_ROUNDS_SHIFT) & 7; }
int tune_lu(int flags) { return (flags >> PANEL_TUNE_LU_SHIFT) & 3; }

bool flags_ok(int flags) {
  const int known = PANEL_FP64 | PANEL_MIXED | PANEL_WITH_ADJOINT | PANEL_FACTOR_ONLY |
                    PANEL_REUSE_FACTOR | PANEL_INVERSE | (7 << PANEL_TUNE_IR_SHIFT) |
                    (7 << PANEL_TUNE_ROUNDS_SHIFT) | (3 << PANEL_TUNE_LU_SHIFT);
  if (tune_ir(flags) > 5 || tune_rounds(flags) > 6 || tune_lu(flags) > 2) return false;
  if (mode_of(flags) == 0 || (flags & ~known) != 0) return false;
  const int stage = flags & (PANEL_FACTOR_ONLY | PANEL_REUSE_FACTOR);
  if (stage == (PANEL_FACTOR_ONLY | PANEL_REUSE_FACTOR)) return false;
  if ((flags & PANEL_INVERSE) && mode_of(flags) != PANEL_MIXED) return false;
  return stage == 0 || mode_of(flags) == PANEL_MIXED;
}

Batch make_batch(int B, int n_max, const double* nodes, const int64_t* node_offsets,
                 const int64_t* mat_offsets, const int32_t* order) {
  Batch b;
  b.B = B;
  b.n_max = n_max;
  b.nodes = nodes;
  b.node_off = node_offsets;
  b.mat_off = mat_offsets;
  b.order = order;
  return b;
}

int status_of(cudaError_t e) { return e == cudaSuccess ? PANEL_OK : PANEL_ECUDA; }

}  // namespace

extern "C" {

const char* panel_strerror(int status) {
  switch (status) {
    case PANEL_OK: return "ok";
    case PANEL_EINVAL: return "invalid argument";
    case PANEL_ENOTSUP: return "size or mode not supported";
    case PANEL_ECUDA: return "CUDA launch failed";
    case PANEL_ESCRATCH:
      return "batch too large for the static work array of panel_solve_noalloc "
             "(PANEL_NOALLOC_SCRATCH_BYTES)";
    default: return "unknown panel status";
  }
}

int64_t panel_debug_wait_limit(int64_t polls) { return panel::set_wait_limit(polls); }

const char* panel_version(void) { return "panel-gb300 0.1 (sm_103a)"; }

int panel_plan(int B, const int64_t* node_offsets, int64_t* mat_offsets, int32_t* order,
               int32_t* n_max) {
  if (B < 0 || !node_offsets || !mat_offsets || !order || !n_max) return PANEL_EINVAL;
  int64_t nm = 0;
  mat_offsets[0] = 0;
  for (int b = 0; b < B; ++b) {
    const int64_t n = node_offsets[b + 1] - node_offsets[b];
    if (n < 0) return PANEL_EINVAL;
    if (n > PANEL_N_MAX) return PANEL_ENOTSUP;
    nm = std::max(nm, n);
    mat_offsets[b + 1] = mat_offsets[b] + (n + 1) * (n + 1);
  }
  std::vector<int32_t> idx(B);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t c) {
    return (node_offsets[a + 1] - node_offsets[a]) > (node_offsets[c + 1] - node_offsets[c]);
  });
  std::copy(idx.begin(), idx.end(), order);
  *n_max = (int32_t)std::max<int64_t>(nm, 3);
  return PANEL_OK;
}

size_t panel_workspace_size(int B, const int64_t* node_offsets, int flags) {
  const size_t bad = (size_t)-1;
  if (B < 0 || (B > 0 && !node_offsets)) return bad;
  const int mode = flags & (PANEL_FP64 | PANEL_MIXED);
  if (mode != PANEL_FP64 && mode != PANEL_MIXED) return bad;
  size_t mat = 0, vec = 0;
  for (int b = 0; b < B; ++b) {
    const int64_t n = node_offsets[b + 1] - node_offsets[b];
    if (n < 0 || n > PANEL_N_MAX) return bad;
    mat += (size_t)(n + 1) * (size_t)(n + 1);
    vec += (size_t)(n + 1);
  }
  // planes + factor: FP64 plane and FP64 factor, or two FP32 planes and an FP32 factor
  const size_t mat_bytes = (mode == PANEL_FP64) ? mat * (8 + 8) : mat * (4 + 4 + 4);
  // pivots (i32), rhs and lambda (f64)
  return mat_bytes + vec * (4 + 8 + 8);
}

int panel_assemble(int B, int n_max, int flags, const double* nodes, const int64_t* node_offsets,
                   const int64_t* mat_offsets, const int32_t* order, const double* alpha,
                   const double* vinf, double* A64, float* A_hi, float* A_lo, double* rhs,
                   int32_t* info, void* stream) {
  if (B < 0 || n_max < 3 || n_max > PANEL_N_MAX || !flags_ok(flags)) return PANEL_EINVAL;
  if (B == 0) return PANEL_OK;
  if (!nodes || !node_offsets || !mat_offsets || !order || !alpha || !rhs || !info)
    return PANEL_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  Batch bt = make_batch(B, n_max, nodes, node_offsets, mat_offsets, order);
  if (mode_of(flags) == PANEL_FP64) {
    if (!A64 || A_hi || A_lo) return PANEL_EINVAL;
    return status_of(panel::launch_assemble_f64(bt, alpha, vinf, A64, rhs, info, s));
  }
  if (!A_hi || !A_lo) return PANEL_EINVAL;
  return status_of(
      panel::launch_assemble_df(bt, alpha, vinf, A_hi, A_lo, rhs, info, s, tune_rounds(flags)));
}

int panel_solve(int B, int n_max, int flags, const double* nodes, const int64_t* node_offsets,
                const int64_t* mat_offsets, const int32_t* order, const double* A64,
                const float* A_hi, const float* A_lo, void* LU, int32_t* piv,
                const double* rhs, const double* vinf, const double* chord, double* u,
                double* lambda, int max_iter, double tol, int32_t* info, int32_t* iters,
                void* stream) {
  if (B < 0 || n_max < 3 || n_max > PANEL_N_MAX || !flags_ok(flags)) return PANEL_EINVAL;
  if (B == 0) return PANEL_OK;
  const bool factor_only = (flags & PANEL_FACTOR_ONLY) != 0;
  const bool reuse = (flags & PANEL_REUSE_FACTOR) != 0;
  if (!node_offsets || !mat_offsets || !order || !piv || !info) return PANEL_EINVAL;
  if (!factor_only && (!rhs || !u)) return PANEL_EINVAL;
  const bool adj = (flags & PANEL_WITH_ADJOINT) != 0;
  if (adj && (!lambda || !nodes)) return PANEL_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  Batch bt = make_batch(B, n_max, nodes, node_offsets, mat_offsets, order);
  if (mode_of(flags) == PANEL_FP64) {
    if (!A64 || !LU) return PANEL_EINVAL;
    return status_of(panel::launch_solve_f64(bt, A64, (double*)LU, piv, rhs, vinf, chord, u,
                                             adj ? lambda : nullptr, info, iters, s));
  }
  if (!A_hi || !A_lo || !LU || max_iter < 0 || !(tol > 0.0)) return PANEL_EINVAL;
  cudaError_t e = cudaSuccess;
  if (!reuse)
    e = panel::launch_lu_mixed(bt, A_hi, (float*)LU, piv, info, iters,
                               (flags & PANEL_INVERSE) != 0, s, tune_lu(flags));
  if (e == cudaSuccess && !factor_only)
    e = panel::launch_ir_mixed(bt, A_hi, A_lo, (const float*)LU, piv, rhs, vinf, chord, u,
                               adj ? lambda : nullptr, max_iter, tol, info, iters, s, 0,
                               tune_ir(flags));
  return status_of(e);
}

int panel_polar(int B, int n_max, int flags, const double* nodes, const int64_t* node_offsets,
                const int64_t* mat_offsets, const int32_t* order, const float* A_hi,
                const float* A_lo, const void* LU, const int32_t* piv, const double* vinf,
                const double* chord, int K, const double* alphas, double* u_y, double* u_x,
                double* cl, int max_iter, double tol, int32_t* info, int32_t* iters,
                void* stream) {
  if (B < 0 || n_max < 3 || n_max > PANEL_N_MAX || K < 0) return PANEL_EINVAL;
  if (mode_of(flags) == PANEL_FP64) return PANEL_ENOTSUP;
  if (mode_of(flags) != PANEL_MIXED || (flags & ~PANEL_MIXED) != 0) return PANEL_EINVAL;
  if (B == 0) return PANEL_OK;
  if (!nodes || !node_offsets || !mat_offsets || !order || !A_hi || !A_lo || !LU || !piv ||
      !u_y || !u_x || !info || (K > 0 && (!alphas || !cl)) || max_iter < 0 || !(tol > 0.0))
    return PANEL_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  Batch bt = make_batch(B, n_max, nodes, node_offsets, mat_offsets, order);
  cudaError_t e = panel::launch_ir_mixed(bt, A_hi, A_lo, (const float*)LU, piv, nullptr, vinf,
                                         chord, u_y, nullptr, max_iter, tol, info, iters, s, 1);
  if (e == cudaSuccess)
    e = panel::launch_ir_mixed(bt, A_hi, A_lo, (const float*)LU, piv, nullptr, vinf, chord,
                               u_x, nullptr, max_iter, tol, info, iters, s, 2);
  if (e == cudaSuccess && K > 0)
    e = panel::launch_polar_cl(bt, u_y, u_x, vinf, chord, K, alphas, info, cl, s);
  return status_of(e);
}

int panel_vjp(int B, int n_max, int flags, const double* nodes, const int64_t* node_offsets,
              const int64_t* mat_offsets, const int32_t* order, const float* A_hi,
              const float* A_lo, const void* LU, const int32_t* piv, const double* u,
              const double* alpha, const double* vinf, const double* chord, const double* w_cl,
              const double* w_u, const double* w_cp, double* lambda, double* grad_nodes,
              int max_iter, double tol, int32_t* info, void* stream) {
  if (B < 0 || n_max < 3 || n_max > PANEL_N_MAX) return PANEL_EINVAL;
  if (mode_of(flags) == PANEL_FP64) return PANEL_ENOTSUP;
  if (mode_of(flags) != PANEL_MIXED || (flags & ~PANEL_MIXED) != 0) return PANEL_EINVAL;
  if (B == 0) return PANEL_OK;
  if (!nodes || !node_offsets || !mat_offsets || !order || !A_hi || !A_lo || !LU || !piv ||
      !u || !alpha || !lambda || !grad_nodes || !info || max_iter < 0 || !(tol > 0.0))
    return PANEL_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  Batch bt = make_batch(B, n_max, nodes, node_offsets, mat_offsets, order);
  cudaError_t e = panel::launch_ir_vjp(bt, A_hi, A_lo, (const float*)LU, piv, vinf, chord, u,
                                       w_cl, w_u, w_cp, lambda, max_iter, tol, info, s);
  if (e != cudaSuccess) return status_of(e);
  if (panel::adjoint_df_smem(n_max) > panel::kMaxDynSmem) return PANEL_ENOTSUP;
  return status_of(panel::launch_adjoint_df(bt, u, lambda, alpha, vinf, chord, w_cl,
                                            grad_nodes, info, s, true));
}

int panel_ga_sample(int B, int P, int n, const double* ctrl_x, const double* genome,
                    double* nodes, void* stream) {
  if (B < 0 || B > 65535 * 64 || P < 4 || n < 3 || n > PANEL_N_MAX) return PANEL_EINVAL;
  if (B == 0) return PANEL_OK;
  if (!ctrl_x || !genome || !nodes) return PANEL_EINVAL;
  return status_of(panel::launch_ga_sample(B, P, n, ctrl_x, genome, nodes, (cudaStream_t)stream));
}

int panel_ga_genome_grad(int B, int P, int n, const double* grad_nodes, double lr,
                         const double* lo, const double* hi, double* genome, double* grad_genome,
                         void* stream) {
  if (B < 0 || P < 4 || n < 3 || n > PANEL_N_MAX || !(lr == lr)) return PANEL_EINVAL;
  if (B == 0) return PANEL_OK;
  if (!grad_nodes || (!grad_genome && lr == 0.0)) return PANEL_EINVAL;
  if (lr != 0.0 && (!lo || !hi || !genome)) return PANEL_EINVAL;
  return status_of(panel::launch_ga_genome_grad(B, P, n, grad_nodes, lr, lo, hi, genome,
                                                grad_genome, (cudaStream_t)stream));
}

int panel_ga_step(int B, int P, int k, double p, double pm, const double* lo, const double* hi,
                  const double* sigma, const double* genome_in, const double* fitness,
                  const double* rand, double* genome_out, void* stream) {
  if (B < 0 || (B & 1) || P < 2 || k < 1 || k > panel::ga_max_tournament() || !(p >= 0.0) ||
      !(p <= 1.0) || !(pm >= 0.0) || !(pm <= 1.0))
    return PANEL_EINVAL;
  if (B == 0) return PANEL_OK;
  if (!lo || !hi || !sigma || !genome_in || !fitness || !rand || !genome_out ||
      genome_in == genome_out)
    return PANEL_EINVAL;
  return status_of(panel::launch_ga_step(B, P, k, p, pm, lo, hi, sigma, genome_in, fitness, rand,
                                         genome_out, (cudaStream_t)stream));
}

int panel_forces(int B, const double* nodes, const int64_t* node_offsets, const double* u,
                 const double* alpha, const double* vinf, const double* chord,
                 const int32_t* info, double* cp, double* cl, double* cl_p, double* cd_p,
                 void* stream) {
  if (B < 0) return PANEL_EINVAL;
  if (B == 0) return PANEL_OK;
  if (!nodes || !node_offsets || !u || !alpha || !cp || !cl) return PANEL_EINVAL;
  Batch bt = make_batch(B, 0, nodes, node_offsets, nullptr, nullptr);
  return status_of(panel::launch_forces(bt, u, alpha, vinf, chord, info, cp, cl, cl_p, cd_p,
                                        (cudaStream_t)stream));
}

int panel_viscous(int B, const double* nodes, const int64_t* node_offsets, const double* u,
                  const double* alpha, const double* vinf, const double* chord,
                  const double* reynolds, const int32_t* info, const double* cl, double* ld,
                  double* cd, double* cd_f, double* theta, double* cf, int32_t* sep,
                  void* stream) {
  if (B < 0) return PANEL_EINVAL;
  if (B == 0) return PANEL_OK;
  if (!nodes || !node_offsets || !u || !alpha || !reynolds || !cd || (ld && !cl))
    return PANEL_EINVAL;
  Batch bt = make_batch(B, 0, nodes, node_offsets, nullptr, nullptr);
  return status_of(panel::launch_viscous(bt, u, alpha, vinf, chord, reynolds, info, cl, ld, cd,
                                         cd_f, theta, cf, sep, (cudaStream_t)stream));
}

int panel_adjoint(int B, int n_max, int flags, const double* nodes, const int64_t* node_offsets,
                  const int64_t* mat_offsets, const int32_t* order, const double* A64,
                  const float* A_hi, const float* A_lo, const void* LU, const int32_t* piv,
                  const double* u, const double* lambda_in, double* lambda_out,
                  const double* alpha, const double* vinf, const double* chord,
                  const double* grad_cl, double* grad_nodes, int max_iter, double tol,
                  int32_t* info, void* stream) {
  if (B < 0 || n_max < 3 || n_max > PANEL_N_MAX || !flags_ok(flags)) return PANEL_EINVAL;
  if (B == 0) return PANEL_OK;
  if (!nodes || !node_offsets || !mat_offsets || !order || !u || !alpha || !grad_nodes)
    return PANEL_EINVAL;
  if (!lambda_in && (!lambda_out || !LU || !piv)) return PANEL_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  Batch bt = make_batch(B, n_max, nodes, node_offsets, mat_offsets, order);
  if (mode_of(flags) == PANEL_FP64) {
    return status_of(panel::launch_adjoint_f64(bt, (const double*)LU, piv, u, lambda_in,
                                               lambda_out, alpha, vinf, chord, grad_cl,
                                               grad_nodes, info, s));
  }
  (void)A64;
  if (!A_hi || !A_lo || !info) return PANEL_EINVAL;
  const double* lam = lambda_in;
  if (!lam) {
    if (max_iter < 0 || !(tol > 0.0)) return PANEL_EINVAL;
    cudaError_t e = panel::launch_ir_mixed(bt, A_hi, A_lo, (const float*)LU, piv, nullptr, vinf,
                                           chord, nullptr, lambda_out, max_iter, tol, info,
                                           nullptr, s);
    if (e != cudaSuccess) return PANEL_ECUDA;
    lam = lambda_out;
  }
  // the double-float contraction keeps ~160 B per panel in shared memory; for
  // larger airfoils the FP64 contraction is used
  if (panel::adjoint_df_smem(n_max) <= panel::kMaxDynSmem)
    return status_of(panel::launch_adjoint_df(bt, u, lam, alpha, vinf, chord, grad_cl,
                                              grad_nodes, info, s));
  return status_of(panel::launch_adjoint_f64(bt, nullptr, nullptr, u, lam, nullptr, alpha, vinf,
                                             chord, grad_cl, grad_nodes, info, s));
}

int panel_df_eval(int op, int count, const double* a, const double* b, double* out,
                  void* stream) {
  if (op < 0 || op > 2 || count < 0) return PANEL_EINVAL;
  if (count == 0) return PANEL_OK;
  if (!a || !out || (op >= 1 && !b)) return PANEL_EINVAL;
  return status_of(panel::launch_df_eval(op, count, a, b, out, (cudaStream_t)stream));
}

}  // extern "C"
