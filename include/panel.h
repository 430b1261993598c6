/*
 * panel.h -- C ABI of the batched 2D panel solver for NVIDIA GB300 (sm_103a).
 *
 * The library evaluates a batch of airfoils with the constant-strength vortex,
 * stream-function panel method of Section 2 of Einkemmer, "Evaluation of the
 * Intel Xeon Phi 7120 and NVIDIA K80 as Accelerators for Two-Dimensional Panel
 * Codes" (arXiv 1511.02166):
 *
 *   panel_assemble  dense influence matrix (panel integral F_i of Section 2,
 *                   collocation at x_{j+1/2}), the C column, the Kutta row
 *                   gamma_0 + gamma_{n-1} = 0 and the right-hand side
 *                   phi_v(x_{j+1/2}) = v_inf (y cos a - x sin a);
 *   panel_solve     LU with partial pivoting and triangular solves (Section 3
 *                   names LU as the solver), with iterative refinement in the
 *                   mixed-precision mode;
 *   panel_forces    Cp at the control points and the lift coefficient
 *                   (Section 2, Figure 2 report C_L);
 *   panel_viscous   Thwaites's boundary layer on the surface speed: momentum
 *                   thickness, skin friction, separation and the drag
 *                   (Section 2's viscous correction);
 *   panel_adjoint   dCl/d(node coordinates) by a transposed solve with the
 *                   stored LU and a contraction with dM/dx (the method has no
 *                   gradient in the paper; the formulas are the chain rule of
 *                   the same panel integral).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Batch layout.  Airfoil b has n_b = node_offsets[b+1] - node_offsets[b] >= 3
 *   distinct nodes x_0..x_{n_b-1} (counter-clockwise, x_0 at the trailing edge;
 *   the closing node x_{n_b} = x_0 is implied, Section 2 / Figure 1), stored as
 *   nodes[2*(node_offsets[b] + k) + {0,1}] (float64 x, y).  The bordered system
 *   has m_b = n_b + 1 unknowns u = (gamma_0..gamma_{n_b-1}, C).
 *   Vectors of length m_b are packed at vec offset node_offsets[b] + b.
 *   Matrices are m_b x m_b row-major at element offset mat_offsets[b], where
 *   mat_offsets is the exclusive prefix sum of m_b^2 (panel_plan fills it).
 * Memory.  Every pointer argument of the compute entry points is DEVICE memory
 *   owned by the caller (e.g. allocated by torch); the library allocates
 *   nothing, never synchronises the stream and launches only on `stream`
 *   (a cudaStream_t; NULL means the legacy default stream).
 * Errors.  The return value is a call-level status (panel_status): argument
 *   errors are detected on the host before anything is launched; a launch
 *   failure returns PANEL_ECUDA.  Per-airfoil problems are written to info[b]
 *   on the device: 0 ok; k > 0 the k-th pivot of the LU was exactly zero;
 *   -1 fewer than 3 nodes; -2 clockwise or zero signed area; -3 a zero-length
 *   panel; -4 a non-finite coordinate or one with magnitude >= 1024; -5 refinement did not converge within
 *   max_iter (mixed mode; the last iterate is still written); -6 n_b larger
 *   than the n_max passed to the call (nothing is written for that airfoil).
 * Precision modes (flags).
 *   PANEL_FP64   plain path: FP64 assembly (native log/atan2), FP64 LU with
 *                partial pivoting, FP64 triangular solves, no refinement.
 *   PANEL_MIXED  GB300 path: the matrix is assembled in double-float (pairs of
 *                FP32, about 48 significant bits) into two FP32 planes
 *                A = A_hi + A_lo; the LU factor is FP32 (of A_hi, with the C
 *                column and Kutta row rescaled); the solution is refined with
 *                double-float residuals b - (A_hi + A_lo) u until
 *                |du|_inf <= tol |u|_inf.  u and all reported outputs are FP64.
 */
#ifndef PANEL_H
#define PANEL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PANEL_OK = 0,
  PANEL_EINVAL = 1,   /* bad argument: size, NULL pointer, flag combination  */
  PANEL_ENOTSUP = 2,  /* size beyond what the library supports (n_b > PANEL_N_MAX) */
  PANEL_ECUDA = 3,    /* a CUDA launch or device query failed                 */
  PANEL_ESCRATCH = 4  /* panel_solve_noalloc: the batch's factor and pivots do
                         not fit PANEL_NOALLOC_SCRATCH_BYTES                   */
} panel_status;

#define PANEL_FP64 0x1
#define PANEL_MIXED 0x2
/* panel_solve: also solve the transposed system M^T lambda = dCl/du for unit
 * upstream gradient (used later by panel_adjoint), sharing the residual passes. */
#define PANEL_WITH_ADJOINT 0x10
/* panel_solve, PANEL_MIXED only: factor (LU, piv, info) and stop ... */
#define PANEL_FACTOR_ONLY 0x20
/* ... or skip the factorisation and refine with the LU/piv of an earlier call
 * (the same matrix planes), e.g. for another right-hand side. */
#define PANEL_REUSE_FACTOR 0x40
/* panel_solve, PANEL_MIXED only: for airfoils with n_b < 288, store the
 * explicit inverse of the (rescaled) system, computed by blocked Gauss-Jordan
 * elimination, instead of the default LU; each refinement correction is then
 * one matrix-vector product instead of two triangular sweeps, at three times
 * the factorisation flops.  Which is faster depends on n_b and on the batch
 * (the autotuner in solver.py picks).  A later PANEL_REUSE_FACTOR call
 * recognises either layout by itself. */
#define PANEL_INVERSE 0x80

/* Launch-shape fields of the flags of panel_assemble and panel_solve (the
 * values an autotuner searches; 0 keeps the library's choice by size).  They
 * change how the work is laid out on the GPU, not what is computed: results
 * agree to rounding.
 *   PANEL_TUNE_IR(s), s = 1..5: the refinement (panel_solve, PANEL_MIXED) runs
 *     blocks of 128 threads (8 per SM; airfoils of at most 223 panels), 256
 *     (4 per SM), 512 (2 per SM), 1024 (1 per SM) or 256 threads (3 per SM); a
 *     shape whose shared memory does not fit the airfoils' size falls back to
 *     the choice by size.
 *   PANEL_TUNE_ROUNDS(r), r = 1..6: the double-float assembly (panel_assemble,
 *     PANEL_MIXED) evaluates near-field pairs inline with the far-field ones
 *     (1) or queues them and evaluates them together after every 4, 8, 16 or
 *     32 pairs per thread (2..5), or (6, the choice by size above 1024 panels)
 *     evaluates each pair of control points once for both of its entries,
 *     sharing the far field's orientation-free terms.  All give the same
 *     matrix.
 *   PANEL_TUNE_LU(k), k = 1..2: the FP32 LU (panel_solve, PANEL_MIXED, without
 *     PANEL_INVERSE) of airfoils with n_b < 224 keeps the trailing matrix in
 *     the LU buffer through L2, several airfoils per SM (1), or the whole
 *     matrix in shared memory, one airfoil per SM (2, the choice by size).
 *     The two compute the same factor (the same operations in the same order).
 * Other values are rejected (PANEL_EINVAL). */
#define PANEL_TUNE_IR_SHIFT 8
#define PANEL_TUNE_ROUNDS_SHIFT 12
#define PANEL_TUNE_LU_SHIFT 16
#define PANEL_TUNE_IR(s) ((s) << PANEL_TUNE_IR_SHIFT)
#define PANEL_TUNE_ROUNDS(r) ((r) << PANEL_TUNE_ROUNDS_SHIFT)
#define PANEL_TUNE_LU(k) ((k) << PANEL_TUNE_LU_SHIFT)

/* Largest panel count per airfoil the library accepts. */
#define PANEL_N_MAX 2048

/* Per-airfoil status codes written to info[b]. */
#define PANEL_INFO_FEW_NODES (-1)
#define PANEL_INFO_ORIENTATION (-2)
#define PANEL_INFO_ZERO_PANEL (-3)
#define PANEL_INFO_NONFINITE (-4)
#define PANEL_INFO_NOCONV (-5)
#define PANEL_INFO_TOO_LARGE (-6) /* n_b exceeds the n_max given to the call */
/* A bounded device-side wait (tensor-core completion) ran out; the airfoil's
 * factor is incomplete.  Not expected in operation: it turns a stalled
 * pipeline into an error instead of a hang. */
#define PANEL_INFO_DEVICE_TIMEOUT (-7)

/*
 * panel_plan (HOST memory only, no GPU work).
 * From host node_offsets[B+1] compute mat_offsets[B+1] (exclusive prefix sum
 * of (n_b+1)^2), order[B] (airfoil indices by decreasing n_b, ties by index:
 * the launch order of the persistent kernels) and *n_max.  Returns PANEL_EINVAL
 * for B < 0, decreasing offsets or NULL pointers, PANEL_ENOTSUP if some
 * n_b > PANEL_N_MAX.  Airfoils with n_b < 3 are accepted here and flagged in
 * info[b] by panel_assemble.
 */
int panel_plan(int B, const int64_t* node_offsets, int64_t* mat_offsets, int32_t* order,
               int32_t* n_max);

/*
 * panel_workspace_size (HOST memory only, no GPU work).
 * Bytes of the device arrays the calls below need besides their inputs and
 * outputs, for a batch with host node_offsets[B+1] and the precision flag in
 * `flags` (PANEL_FP64 or PANEL_MIXED): the matrix plane(s) (A64, or A_hi and
 * A_lo) and the factor buffer (sum m_b^2 elements each, m_b = n_b + 1), the
 * pivots, the right-hand side and lambda (sum m_b each).  The library allocates
 * nothing: the caller provides these as separate arrays with the layouts given
 * at each call, and this is their total, for budgeting device memory.  Returns
 * 0 for B == 0 and (size_t)-1 for B < 0, a NULL pointer, decreasing offsets,
 * n_b > PANEL_N_MAX or a bad flag.
 */
size_t panel_workspace_size(int B, const int64_t* node_offsets, int flags);

/*
 * panel_assemble -- Section 2: influence matrix, C column, Kutta row, rhs.
 *   nodes [sum n_b][2] f64, node_offsets [B+1] i64, mat_offsets [B+1] i64,
 *   order [B] i32 (from panel_plan), alpha [B] f64 (radians),
 *   vinf [B] f64 or NULL (1.0).
 *   PANEL_FP64:  A64 [sum m_b^2] f64 receives M; A_hi/A_lo must be NULL.
 *   PANEL_MIXED: A_hi, A_lo [sum m_b^2] f32 receive M = A_hi + A_lo;
 *                A64 may be NULL.
 *   rhs [sum m_b] f64 receives b (b_n = 0 for the Kutta row);
 *   info [B] i32 receives 0 or a geometry code (the matrix of a rejected
 *   airfoil is left unwritten).
 */
int panel_assemble(int B, int n_max, int flags, const double* nodes, const int64_t* node_offsets,
                   const int64_t* mat_offsets, const int32_t* order, const double* alpha,
                   const double* vinf, double* A64, float* A_hi, float* A_lo, double* rhs,
                   int32_t* info, void* stream);

/*
 * panel_solve -- LU with partial pivoting and solve (Section 3), refined in
 * PANEL_MIXED mode.
 *   PANEL_FP64:  reads A64; LU [sum m_b^2] f64 receives the factors (L unit
 *                lower, U upper, row-major, in one array); no refinement.
 *   PANEL_MIXED: reads A_hi, A_lo; LU [sum m_b^2] f32 receives the FP32
 *                factors of the rescaled matrix in a library-internal layout
 *                (row-major L\U with every 32 x 32 diagonal block of L and of
 *                U replaced by its inverse), used by the refinement and by
 *                panel_adjoint.
 *   piv [sum m_b] i32 receives the pivot rows (LAPACK style, 0-based).
 *   rhs [sum m_b] f64; u [sum m_b] f64 receives (gamma, C).
 *   lambda [sum m_b] f64 or NULL: with PANEL_WITH_ADJOINT receives the
 *   solution of M^T lambda = g, g_i = 2 |h_i| / (v_inf c) (i < n_b), g_n = 0,
 *   i.e. dCl/du for unit upstream gradient; needs nodes, vinf and chord.
 *   max_iter >= 0 refinement steps at most, tol > 0 stopping threshold on
 *   |du|_inf / |u|_inf (ignored by PANEL_FP64).
 *   info [B] i32: airfoils with info[b] != 0 on entry are skipped; on exit
 *   k > 0 for a zero pivot, PANEL_INFO_NOCONV if not converged.
 *   iters [B] i32 or NULL receives the refinement steps taken.
 */
int panel_solve(int B, int n_max, int flags, const double* nodes, const int64_t* node_offsets,
                const int64_t* mat_offsets, const int32_t* order, const double* A64,
                const float* A_hi, const float* A_lo, void* LU, int32_t* piv,
                const double* rhs, const double* vinf, const double* chord, double* u,
                double* lambda, int max_iter, double tol, int32_t* info, int32_t* iters,
                void* stream);

/*
 * panel_forces -- Cp_j = 1 - (gamma_j / v_inf)^2 at the control points,
 * Cl = 2 sum_i gamma_i |h_i| / (v_inf c) (Kutta-Joukowski), and the
 * pressure-integrated Cl_p, Cd_p with outward normals (h_y, -h_x)/|h|.
 *   u [sum m_b] f64 from panel_solve; alpha [B] f64; vinf, chord [B] f64 or
 *   NULL (1.0); cp [sum n_b] f64; cl [B] f64; cl_p, cd_p [B] f64 or NULL.
 *   Airfoils with info[b] != 0 get NaN outputs (info may be NULL).
 *   FP64 throughout (warp-shuffle reductions).
 */
int panel_forces(int B, const double* nodes, const int64_t* node_offsets, const double* u,
                 const double* alpha, const double* vinf, const double* chord,
                 const int32_t* info, double* cp, double* cl, double* cl_p, double* cd_p,
                 void* stream);

/*
 * panel_viscous -- the viscous correction of Section 2 (Thwaites's laminar
 * boundary-layer method on the inviscid surface speed; the paper names the
 * method for the drag and prints no formulas, the textbook ones are used):
 *   U_j = |gamma_j| / v_inf at the control points; the stagnation point lies
 *   between control points j and j+1 for the first j with gamma_j > 0 >=
 *   gamma_{j+1} (linear zero of gamma); the upper surface runs through control
 *   points j..0, the lower through j+1..n-1, each to the trailing edge;
 *   theta^2 U^6 = (0.45 / Re) int U^5 ds (U piecewise linear, lengths in chords),
 *   lambda = Re theta^2 dU/ds, Thwaites's shear and shape functions l, H
 *   (Cebeci-Bradshaw fits, lambda clamped to [-0.09, 0.1]); laminar separation
 *   at the first control point with lambda < -0.09, past which the wall shear
 *   is zero and H keeps its separation value while theta follows the integral.
 *   u [sum m_b] f64 from panel_solve; alpha [B] f64; vinf, chord [B] f64 or NULL
 *   (1.0); reynolds [B] f64, Re = v_inf c / nu.
 *   Outputs: cd [B] f64 profile drag by Squire and Young,
 *   sum over both surfaces of 2 theta U^((H + 5) / 2) at the trailing edge;
 *   cd_f [B] f64 or NULL, skin-friction drag (cf = 2 l U / (Re theta)
 *   integrated along the freestream direction); theta [sum n_b] f64 or NULL,
 *   momentum thickness / c at the control points; cf [sum n_b] f64 or NULL,
 *   skin-friction coefficient at the control points; sep [B][2] i32 or NULL,
 *   the separating control point of the upper and lower surface (-1: attached
 *   to the trailing edge); ld [B] f64 or NULL, the lift-to-drag ratio
 *   cl[b] / cd[b] (cl [B] f64 from panel_forces, required with ld; the fitness
 *   of Section 3's optimisation).  Airfoils with info[b] != 0, no stagnation
 *   point, or Re not positive and finite get NaN outputs and sep = -2.  FP64;
 *   one warp per surface (prefix sums for the integral).
 */
int panel_viscous(int B, const double* nodes, const int64_t* node_offsets, const double* u,
                  const double* alpha, const double* vinf, const double* chord,
                  const double* reynolds, const int32_t* info, const double* cl, double* ld,
                  double* cd, double* cd_f, double* theta, double* cf, int32_t* sep,
                  void* stream);

/*
 * panel_adjoint -- grad_nodes = grad_cl[b] * dCl/d(nodes of airfoil b).
 *   dCl/dx_k = dCl/dx_k|_u + lambda^T (db/dx_k - (dM/dx_k) u),  M^T lambda = dCl/du.
 *   If lambda_in is non-NULL it holds lambda from panel_solve(PANEL_WITH_ADJOINT);
 *   otherwise lambda is solved here from LU/piv (and refined against the
 *   matrix in PANEL_MIXED mode) into lambda_out (required then, [sum m_b] f64).
 *   The contraction re-evaluates the panel-integral derivatives per pair
 *   (two per pair: with respect to the control point and to the panel end).
 *   grad_cl [B] f64 upstream gradient (NULL means 1); grad_nodes [sum n_b][2]
 *   f64 output.  info [B] i32 (in/out): airfoils with info[b] != 0 are skipped
 *   (gradient set to NaN); the refinement of lambda may set PANEL_INFO_NOCONV.
 */
int panel_adjoint(int B, int n_max, int flags, const double* nodes, const int64_t* node_offsets,
                  const int64_t* mat_offsets, const int32_t* order, const double* A64,
                  const float* A_hi, const float* A_lo, const void* LU, const int32_t* piv,
                  const double* u, const double* lambda_in, double* lambda_out,
                  const double* alpha, const double* vinf, const double* chord,
                  const double* grad_cl, double* grad_nodes, int max_iter, double tol,
                  int32_t* info, void* stream);

/*
 * panel_polar -- Cl at K angles of attack per airfoil from one factorisation
 * (PANEL_MIXED only; PANEL_FP64 returns PANEL_ENOTSUP).
 *   The right-hand side of Section 2's system is linear in (cos a, sin a):
 *   b(a) = cos(a) b_y + sin(a) b_x with b_y,j = v m_j,y and b_x,j = -v m_j,x
 *   (m_j the control point, 0 in the Kutta row), so the strengths are
 *   u(a) = cos(a) u_y + sin(a) u_x and Cl(a) = cos(a) Cl_y + sin(a) Cl_x.
 *   The call refines the two basis systems against the matrix planes with the
 *   factor (LU, piv) stored by an earlier panel_solve of the same planes (e.g.
 *   with PANEL_FACTOR_ONLY), then combines them.
 *   alphas [B][K] f64 radians by airfoil index; u_y, u_x [sum m_b] f64
 *   outputs packed like u; cl [B][K] f64 output (NaN where info[b] != 0).
 *   vinf, chord as in panel_solve.  info / iters as in panel_solve (iters is
 *   that of the second basis system).  K = 0 solves the basis only.
 */
int panel_polar(int B, int n_max, int flags, const double* nodes, const int64_t* node_offsets,
                const int64_t* mat_offsets, const int32_t* order, const float* A_hi,
                const float* A_lo, const void* LU, const int32_t* piv, const double* vinf,
                const double* chord, int K, const double* alphas, double* u_y, double* u_x,
                double* cl, int max_iter, double tol, int32_t* info, int32_t* iters,
                void* stream);

/*
 * panel_vjp -- vector-Jacobian product of the strengths, Cp and Cl with
 * respect to the node coordinates (PANEL_MIXED only; PANEL_FP64 returns
 * PANEL_ENOTSUP): grad_nodes = dL/dx for
 *   L = sum_b w_cl[b] Cl_b + sum_j w_u[j] u_j + sum_j w_cp[j] Cp_j,
 *   u = (gamma, C) per airfoil as solved by panel_solve, Cp_j = 1 - (gamma_j / v)^2
 *   (Section 2's strengths and Cp, as panel_forces).
 *   lambda solves M^T lambda = dL/du (refined with the stored factor LU/piv of
 *   an earlier panel_solve of the same matrix planes), then
 *   dL/dx_k = w_cl dCl/dx_k|_u + lambda^T (db/dx_k - (dM/dx_k) u), with the pair
 *   derivatives of panel_adjoint.
 *   u [sum m_b] the solved strengths; w_cl [B] (NULL = 0); w_u [sum m_b] packed
 *   like u and w_cp [sum n_b] packed like the nodes (NULL = 0); lambda
 *   [sum m_b] f64 output;
 *   grad_nodes [sum n_b][2] f64 output (NaN where info[b] != 0).
 */
int panel_vjp(int B, int n_max, int flags, const double* nodes, const int64_t* node_offsets,
              const int64_t* mat_offsets, const int32_t* order, const float* A_hi,
              const float* A_lo, const void* LU, const int32_t* piv, const double* u,
              const double* alpha, const double* vinf, const double* chord, const double* w_cl,
              const double* w_u, const double* w_cp, double* lambda, double* grad_nodes,
              int max_iter, double tol, int32_t* info, void* stream);

/*
 * Genetic algorithm around the evaluator (the genetic optimisation of
 * Section 2; the paper leaves the spline, the sampling, k, p and the mutation
 * unspecified -- the choices below are this library's).
 *
 * panel_ga_sample -- nodes of B airfoils from their B-spline genomes.
 *   The airfoil is a clamped uniform cubic B-spline over P >= 4 control points
 *   with x coordinates ctrl_x [P] shared by the population (trailing edge,
 *   upper surface, leading edge, lower surface, trailing edge) and y
 *   coordinates genome [B][P].  Node i of n is the curve at
 *   t_i = (1 - cos(pi i / n_u)) / 4 for i <= n_u = ceil(n/2), else
 *   1/2 + (1 - cos(pi (i - n_u) / (n - n_u))) / 4.  nodes [B*n][2] f64 output
 *   (airfoil b at rows b n .. b n + n - 1, the layout panel_plan expects with
 *   node_offsets[b] = b n).  B <= 65535 * 64.
 *
 * panel_ga_step -- one generation: genome_out [B][P] from genome_in [B][P]
 *   and fitness [B] (higher is better, NaN never preferred), B even, by
 *   B/2 x (two tournaments of size k <= 16 accepting the j-th ranked
 *   candidate with probability p (1-p)^j, one-point crossover into two
 *   children, per child a mutation with probability pm of one gene by
 *   sigma_g (2u - 1), clamped to [lo_g, hi_g]).  Every random number is an
 *   input: rand [B/2][4k + 5] uniform in [0, 1), per pair: k candidate draws
 *   and k - 1 acceptance draws per tournament, the crossover point, then per
 *   child the mutation decision, gene and amount.  lo, hi, sigma [P].
 *
 * panel_ga_genome_grad -- genome gradient of a loss L from its node gradient
 *   (gradient-refined GA steps; e.g. L = Cl with grad_nodes from panel_adjoint):
 *   the nodes of panel_ga_sample have y_i = sum_r N_r(t_i) g_r with x fixed, so
 *   dL/dg_r = sum_i N_r(t_i) dL/dy_i.  grad_nodes [B*n][2] f64 (only the y
 *   components are read); grad_genome [B][P] f64 output or NULL; with lr != 0
 *   the genome [B][P] (in/out) takes the ascent step g <- clamp(g + lr dL/dg,
 *   lo, hi) (lo, hi [P]) for every gene whose dL/dg is finite; a gene with a
 *   non-finite gradient (e.g. an airfoil whose solve failed, whose node
 *   gradients panel_adjoint sets to NaN) keeps its value.  Sums in node order
 *   (deterministic).
 */
int panel_ga_genome_grad(int B, int P, int n, const double* grad_nodes, double lr,
                         const double* lo, const double* hi, double* genome, double* grad_genome,
                         void* stream);
int panel_ga_sample(int B, int P, int n, const double* ctrl_x, const double* genome,
                    double* nodes, void* stream);
int panel_ga_step(int B, int P, int k, double p, double pm, const double* lo, const double* hi,
                  const double* sigma, const double* genome_in, const double* fitness,
                  const double* rand, double* genome_out, void* stream);

/*
 * panel_df_eval -- diagnostic: evaluate the double-float primitives of the
 * PANEL_MIXED assembly on `count` device inputs (results rounded to f64):
 *   op 0: out[k] = log(a[k])                      (a[k] > 0)
 *   op 1: out[k] = atan2(a[k], b[k])
 *   op 2: out[k] = A coefficient -G of Section 2 for the control point
 *         (a[2k], a[2k+1]) and the panel (b[4k], b[4k+1]) -> (b[4k+2], b[4k+3]).
 * Inputs are rounded to double-float first.  Used by the tests to compare the
 * emulated arithmetic with FP64.
 */
int panel_df_eval(int op, int count, const double* a, const double* b, double* out,
                  void* stream);

/*
 * panel_debug_wait_limit (HOST, diagnostic) -- the number of polls after which
 * a pipeline wait inside the tensor-core trailing update of the large-airfoil
 * factor (n_b >= 640, PANEL_MIXED) gives up.  A wait that runs out stops the
 * airfoil's factorisation: the kernel waits for the tensor-core operations it
 * has already issued, releases its tensor memory, writes
 * info[b] = PANEL_INFO_DEVICE_TIMEOUT and returns, and the later stages skip
 * that airfoil.  The default (2^22 polls, far above any wait of a working
 * pipeline) turns a stalled pipeline into that error instead of a hang; a test
 * lowers it to exercise the error path.  polls <= 0 restores the default.
 * Returns the previous limit.  The value is process-wide and read when a
 * panel_solve call launches its kernels (not synchronised with calls in flight
 * on other host threads).  Not part of the paper's method.
 */
int64_t panel_debug_wait_limit(int64_t polls);

/*
 * panel_solve_noalloc -- panel_solve for callers that cannot allocate device
 * memory.  The paper has no counterpart: this is a memory-management variant
 * of panel_solve, not a step of the method.
 *
 * Who needs it.  panel_solve takes two work arrays from the caller, the factor
 * buffer LU and the pivots piv.  A caller that cannot call cudaMalloc (or any
 * allocator) -- a plug-in that runs inside a host application which owns every
 * device allocation, a real-time loop that must not allocate once it runs, a
 * binding from a language without a device allocator -- cannot provide them.
 * This entry point keeps both in one fixed-size array of device memory that
 * the library itself declares (file scope, static): the CUDA runtime sets it
 * aside on each GPU when the library's device code is loaded there, and it
 * stays reserved on that GPU until the process exits.  The call allocates
 * nothing (no cudaMalloc, no cudaFree, no allocating library routine) and runs
 * the same kernels as panel_solve on the given stream.
 *
 * Arguments are those of panel_solve without LU and piv, plus
 *   node_offsets_host [B+1] i64 in HOST memory, equal to the device array
 *   node_offsets: the library sums the work array sizes on the host before
 *   launching anything.  mat_offsets must be panel_plan's for the same offsets.
 *   flags: PANEL_FP64 or PANEL_MIXED, optionally with PANEL_WITH_ADJOINT (and
 *   PANEL_INVERSE in PANEL_MIXED mode); PANEL_FACTOR_ONLY and
 *   PANEL_REUSE_FACTOR are rejected (the factor does not outlive the call).
 *   n_max must bound every n_b (PANEL_EINVAL otherwise).
 * Limit.  The factor (sum m_b^2 elements of 4 bytes in PANEL_MIXED mode, 8 in
 *   PANEL_FP64 mode) and, 256-byte aligned after it, the pivots (sum m_b int32)
 *   must fit PANEL_NOALLOC_SCRATCH_BYTES (32 MiB: e.g. about 200 airfoils of 200
 *   panels in PANEL_MIXED mode, or one of 2048); a larger batch returns
 *   PANEL_ESCRATCH before anything is launched.  Split larger populations into
 *   several calls, or use panel_solve.
 * Sharing.  Every call on a GPU uses the same array, which keeps the last
 *   call's factor and pivots; each call writes all it reads, so nothing needs
 *   to be cleared between calls.  Calls whose kernels overlap on the GPU (on
 *   different streams, or from different host threads) race on the array and
 *   give wrong results: order them on one stream, or synchronise between them.
 * Set-up.  The first call on each device (the current device of the calling
 *   thread) looks up the array's device address (cudaGetSymbolAddress) and
 *   caches it; make that first call before any stream capture on that device.
 *   A failed look-up returns PANEL_ECUDA.
 */
#define PANEL_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int panel_solve_noalloc(int B, int n_max, int flags, const int64_t* node_offsets_host,
                        const double* nodes, const int64_t* node_offsets,
                        const int64_t* mat_offsets, const int32_t* order, const double* A64,
                        const float* A_hi, const float* A_lo, const double* rhs,
                        const double* vinf, const double* chord, double* u, double* lambda,
                        int max_iter, double tol, int32_t* info, int32_t* iters, void* stream);

/* Human-readable name of a panel_status value (static string). */
const char* panel_strerror(int status);

/* Library version string. */
const char* panel_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PANEL_H */
