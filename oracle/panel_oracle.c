/*
 * panel_oracle.c -- FP64 CPU oracle for the batched 2D panel method.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only tests/, the smoke check in
 * __graft_entry__.py and the CPU-baseline leg of bench.py load this file.
 * The CUDA library shares no code with it.
 *
 * It is a plain, slow, obviously-checkable restatement of the method in
 * Section 2 of Einkemmer, "Evaluation of the Intel Xeon Phi 7120 and NVIDIA
 * K80 as Accelerators for Two-Dimensional Panel Codes" (arXiv 1511.02166):
 *
 *   geometry   nodes x_0..x_{n-1}, closing node x_n = x_0, trailing edge at x_0,
 *              h_i = x_{i+1} - x_i, control points x_{j+1/2} = (x_j + x_{j+1})/2
 *              (Section 2, Figure 1);
 *   influence  the closed-form panel integral F_i(x) with two logarithms and two
 *              arctan2 per panel, evaluated literally as printed (Section 2);
 *   system     sum_i A_ji gamma_i + C = phi_v(x_{j+1/2}) with A_ji = -F_i/gamma_i,
 *              phi_v(x) = v_inf (y cos(alpha) - x sin(alpha)), plus the Kutta
 *              condition gamma_0 = -gamma_{n-1} written as an extra row, giving
 *              an (n+1) x (n+1) system in u = (gamma_0..gamma_{n-1}, C) (Section 2);
 *   solve      LU with partial pivoting (ties go to the lowest row), then forward
 *              and back substitution (Section 3 names LU as the solver), then two
 *              steps of iterative refinement whose residual b - M x is accumulated
 *              in long double: the result is the solution of the FP64-assembled
 *              system to about 1e-15, so the FP64 LU's own rounding error
 *              (condition number x 1e-16, which reaches 1e-10 for some 500-panel
 *              airfoils) does not enter comparisons;
 *   forces     surface speed |gamma_j|, Cp_j = 1 - (gamma_j / v_inf)^2,
 *              Cl = 2 sum_i gamma_i |h_i| / (v_inf c) (Kutta-Joukowski), and the
 *              pressure-integrated Cl_p, Cd_p.  The paper reports C_L without a
 *              formula (Section 2, Figure 2 tables); these are the textbook ones.
 *   gradient   dCl/d(node coordinates) by forward-mode dual numbers pushed
 *              through the same influence formula and a re-solve with the LU,
 *              one tangent per coordinate (O(n^3) per airfoil by design).
 *
 * Arithmetic is in `real`: IEEE double by default.  The same source compiled
 * with -DORACLE_LONG_DOUBLE computes in long double (80-bit on x86-64, 128-bit
 * on aarch64) and serves as the reference where the system is so ill
 * conditioned that the FP64 evaluation itself is off by more than the
 * comparison tolerance (some perturbed 500-panel airfoils: the FP64 entries are
 * right to 1e-16, their solution only to ~1e-9).  Inputs and outputs are double
 * in both builds.  No fast-math, no blocking or reordering beyond the
 * definitions.  Batch entry points run airfoils in parallel with OpenMP; each
 * airfoil is computed serially.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifdef ORACLE_LONG_DOUBLE
typedef long double real;
#define R_LOG logl
#define R_ATAN2 atan2l
#define R_SQRT sqrtl
#define R_FABS fabsl
#define R_COS cosl
#define R_SIN sinl
#else
typedef double real;
#define R_LOG log
#define R_ATAN2 atan2
#define R_SQRT sqrt
#define R_FABS fabs
#define R_COS cos
#define R_SIN sin
#endif

static const real TWO_PI = 6.283185307179586476925286766559L;

/* 1 for the long double build, 0 for the double build. */
int oracle_is_extended(void) { return sizeof(real) > sizeof(double); }

/* ------------------------------------------------------------------------ */
/* Geometry (Section 2, Figure 1)                                           */
/* ------------------------------------------------------------------------ */

/* Node i of an n-node airfoil with the closing convention x_n = x_0. */
static void node(const double *nodes, int n, int i, real *x, real *y) {
  int k = i % n;
  *x = nodes[2 * k];
  *y = nodes[2 * k + 1];
}

/* Signed polygon area (shoelace); positive for counter-clockwise nodes. */
double oracle_signed_area(int n, const double *nodes) {
  real a = 0.0;
  for (int i = 0; i < n; ++i) {
    real x0, y0, x1, y1;
    node(nodes, n, i, &x0, &y0);
    node(nodes, n, i + 1, &x1, &y1);
    a += x0 * y1 - x1 * y0;
  }
  return (double)(0.5 * a);
}

/* ------------------------------------------------------------------------ */
/* Panel integral F_i (Section 2), literally as printed                     */
/* ------------------------------------------------------------------------ */

/*
 * F_i(p) / gamma_i for the panel from a = x_i to b = x_{i+1}:
 *
 *   (1/2pi)(1/|h|) [ 1/2 <p-a,h> log|p-a|^2 - 1/2 <p-b,h> log|p-b|^2
 *                    - I atan2(I, <p-a,h>) + I atan2(I, <p-b,h>) - |h|^2 ]
 *
 * with h = b - a, I = <h_perp, p-a>, h_perp = (h_y, -h_x) (outward for
 * counter-clockwise nodes, |h_perp| = |h|).
 */
static real panel_integral(real px, real py, real ax, real ay, real bx, real by) {
  real hx = bx - ax, hy = by - ay;
  real hn = R_SQRT(hx * hx + hy * hy);
  real dax = px - ax, day = py - ay; /* p - x_i     */
  real dbx = px - bx, dby = py - by; /* p - x_{i+1} */
  real dot_a = dax * hx + day * hy;  /* <p - x_i, h>     */
  real dot_b = dbx * hx + dby * hy;  /* <p - x_{i+1}, h> */
  real I = hy * dax - hx * day;      /* <h_perp, p - x_i> */
  real ra2 = dax * dax + day * day;
  real rb2 = dbx * dbx + dby * dby;
  real bracket = 0.5 * dot_a * R_LOG(ra2) - 0.5 * dot_b * R_LOG(rb2) -
                 I * R_ATAN2(I, dot_a) + I * R_ATAN2(I, dot_b) - hn * hn;
  return bracket / (hn * TWO_PI);
}

double oracle_panel_integral(double px, double py, double ax, double ay, double bx,
                             double by) {
  return (double)panel_integral(px, py, ax, ay, bx, by);
}

/* A_ji = -F_i(x_{j+1/2}) / gamma_i: the coefficient of gamma_i in row j. */
static real influence(const double *nodes, int n, int j, int i) {
  real xj, yj, xj1, yj1, xa, ya, xb, yb;
  node(nodes, n, j, &xj, &yj);
  node(nodes, n, j + 1, &xj1, &yj1);
  node(nodes, n, i, &xa, &ya);
  node(nodes, n, i + 1, &xb, &yb);
  real px = 0.5 * (xj + xj1), py = 0.5 * (yj + yj1);
  return -panel_integral(px, py, xa, ya, xb, yb);
}

/* ------------------------------------------------------------------------ */
/* Bordered system (Section 2): rows 0..n-1 collocation, row n Kutta        */
/* ------------------------------------------------------------------------ */

/*
 * M is (n+1) x (n+1), row-major.  Unknowns u = (gamma_0 .. gamma_{n-1}, C).
 *   M[j][i] = A_ji, M[j][n] = 1, b_j = phi_v(x_{j+1/2})           (j < n)
 *   M[n][0] = M[n][n-1] = 1, all other M[n][*] = 0, b_n = 0         (Kutta)
 */
static void assemble(int n, const double *nodes, real alpha, real vinf, real *M, real *b) {
  int m = n + 1;
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < n; ++i) M[j * m + i] = influence(nodes, n, j, i);
    M[j * m + n] = 1.0;
    real xj, yj, xj1, yj1;
    node(nodes, n, j, &xj, &yj);
    node(nodes, n, j + 1, &xj1, &yj1);
    real px = 0.5 * (xj + xj1), py = 0.5 * (yj + yj1);
    b[j] = vinf * (py * R_COS(alpha) - px * R_SIN(alpha));
  }
  for (int i = 0; i < m; ++i) M[n * m + i] = 0.0;
  M[n * m + 0] = 1.0;
  M[n * m + (n - 1)] = 1.0;
  b[n] = 0.0;
}

void oracle_assemble(int n, const double *nodes, double alpha, double vinf, double *M,
                     double *b) {
  int m = n + 1;
  real *Mr = (real *)malloc(sizeof(real) * (size_t)m * m);
  real *br = (real *)malloc(sizeof(real) * (size_t)m);
  assemble(n, nodes, alpha, vinf, Mr, br);
  for (size_t k = 0; k < (size_t)m * m; ++k) M[k] = (double)Mr[k];
  for (int k = 0; k < m; ++k) b[k] = (double)br[k];
  free(Mr);
  free(br);
}

/* ------------------------------------------------------------------------ */
/* Dense LU with partial pivoting (Doolittle, in place, row-major)          */
/* ------------------------------------------------------------------------ */

/* piv[k] = row exchanged with row k at step k.  Returns 0, or k+1 if the
 * k-th pivot is exactly zero (LAPACK convention; factorisation stops). */
static int lu_factor(int m, real *A, int *piv) {
  for (int k = 0; k < m; ++k) {
    int p = k;
    real best = R_FABS(A[k * m + k]);
    for (int r = k + 1; r < m; ++r) {
      real v = R_FABS(A[r * m + k]);
      if (v > best) { best = v; p = r; }
    }
    piv[k] = p;
    if (best == 0.0) return k + 1;
    if (p != k) {
      for (int c = 0; c < m; ++c) {
        real t = A[k * m + c];
        A[k * m + c] = A[p * m + c];
        A[p * m + c] = t;
      }
    }
    for (int r = k + 1; r < m; ++r) {
      real l = A[r * m + k] / A[k * m + k];
      A[r * m + k] = l;
      for (int c = k + 1; c < m; ++c) A[r * m + c] -= l * A[k * m + c];
    }
  }
  return 0;
}

/* Solve (LU) x = P b in place given the factors of lu_factor. */
static void lu_solve(int m, const real *LU, const int *piv, real *x) {
  for (int k = 0; k < m; ++k) {
    int p = piv[k];
    if (p != k) { real t = x[k]; x[k] = x[p]; x[p] = t; }
  }
  for (int r = 1; r < m; ++r)
    for (int c = 0; c < r; ++c) x[r] -= LU[r * m + c] * x[c];
  for (int r = m - 1; r >= 0; --r) {
    for (int c = r + 1; c < m; ++c) x[r] -= LU[r * m + c] * x[c];
    x[r] /= LU[r * m + r];
  }
}

/* Solve M^T y = g in place given the factors of lu_factor. */
static void lu_solve_transposed(int m, const real *LU, const int *piv, real *y) {
  /* M = P^T L U  =>  M^T = U^T L^T P.  Solve U^T z = g, L^T w = z, y = P^T w. */
  for (int r = 0; r < m; ++r) {
    for (int c = 0; c < r; ++c) y[r] -= LU[c * m + r] * y[c];
    y[r] /= LU[r * m + r];
  }
  for (int r = m - 1; r >= 0; --r)
    for (int c = r + 1; c < m; ++c) y[r] -= LU[c * m + r] * y[c];
  for (int k = m - 1; k >= 0; --k) {
    int p = piv[k];
    if (p != k) { real t = y[k]; y[k] = y[p]; y[p] = t; }
  }
}

/* x += M^{-1} (b - M x), the residual accumulated in long double, `steps` times. */
static void refine(int m, const real *M, const real *LU, const int *piv, const real *b, real *x,
                   int steps) {
  real *r = (real *)malloc(sizeof(real) * (size_t)m);
  for (int s = 0; s < steps; ++s) {
    for (int i = 0; i < m; ++i) {
      long double acc = b[i];
      for (int j = 0; j < m; ++j) acc -= (long double)M[i * m + j] * (long double)x[j];
      r[i] = (real)acc;
    }
    lu_solve(m, LU, piv, r);
    for (int i = 0; i < m; ++i) x[i] += r[i];
  }
  free(r);
}

/* double-array wrappers of the LU routines (for the library-comparison pins) */
int oracle_lu_factor(int m, double *A, int *piv) {
  real *Ar = (real *)malloc(sizeof(real) * (size_t)m * m);
  for (size_t k = 0; k < (size_t)m * m; ++k) Ar[k] = A[k];
  int info = lu_factor(m, Ar, piv);
  for (size_t k = 0; k < (size_t)m * m; ++k) A[k] = (double)Ar[k];
  free(Ar);
  return info;
}

static void solve_wrapper(int m, const double *LU, const int *piv, double *x, int transposed) {
  real *Lr = (real *)malloc(sizeof(real) * (size_t)m * m);
  real *xr = (real *)malloc(sizeof(real) * (size_t)m);
  for (size_t k = 0; k < (size_t)m * m; ++k) Lr[k] = LU[k];
  for (int k = 0; k < m; ++k) xr[k] = x[k];
  if (transposed) lu_solve_transposed(m, Lr, piv, xr);
  else lu_solve(m, Lr, piv, xr);
  for (int k = 0; k < m; ++k) x[k] = (double)xr[k];
  free(Lr);
  free(xr);
}
void oracle_lu_solve(int m, const double *LU, const int *piv, double *x) {
  solve_wrapper(m, LU, piv, x, 0);
}
void oracle_lu_solve_transposed(int m, const double *LU, const int *piv, double *y) {
  solve_wrapper(m, LU, piv, y, 1);
}

/* ------------------------------------------------------------------------ */
/* Forces (Section 2 reports C_L; formulas are the textbook ones)           */
/* ------------------------------------------------------------------------ */

/*
 * gamma = u[0..n-1].  Outputs cp[n] and out3 = (Cl, Cl_p, Cd_p):
 *   Cp_j  = 1 - (gamma_j / v_inf)^2                 at the control points
 *   Cl    = 2 sum_i gamma_i |h_i| / (v_inf c)       (Kutta-Joukowski)
 *   F     = -sum_j Cp_j n_j |h_j|,  n_j = (h_y, -h_x)/|h_j| (outward)
 *   Cl_p  = (-F_x sin a + F_y cos a)/c,  Cd_p = (F_x cos a + F_y sin a)/c
 */
static void forces(int n, const double *nodes, const real *u, real alpha, real vinf, real chord,
                   double *cp, double *out3) {
  real circ = 0.0, fx = 0.0, fy = 0.0;
  for (int j = 0; j < n; ++j) {
    real xa, ya, xb, yb;
    node(nodes, n, j, &xa, &ya);
    node(nodes, n, j + 1, &xb, &yb);
    real hx = xb - xa, hy = yb - ya;
    real len = R_SQRT(hx * hx + hy * hy);
    real g = u[j];
    real c = 1.0 - (g / vinf) * (g / vinf);
    if (cp) cp[j] = (double)c;
    circ += g * len;
    fx -= c * hy;    /* -Cp * n_x * |h| with n_x |h| = h_y  */
    fy -= c * (-hx); /* -Cp * n_y * |h| with n_y |h| = -h_x */
  }
  out3[0] = (double)(2.0 * circ / (vinf * chord));
  out3[1] = (double)((-fx * R_SIN(alpha) + fy * R_COS(alpha)) / chord);
  out3[2] = (double)((fx * R_COS(alpha) + fy * R_SIN(alpha)) / chord);
}

void oracle_forces(int n, const double *nodes, const double *u, double alpha, double vinf,
                   double chord, double *cp, double *out3) {
  real *ur = (real *)malloc(sizeof(real) * (size_t)(n + 1));
  for (int k = 0; k <= n; ++k) ur[k] = u[k];
  forces(n, nodes, ur, alpha, vinf, chord, cp, out3);
  free(ur);
}

/* ------------------------------------------------------------------------ */
/* One airfoil, end to end                                                  */
/* ------------------------------------------------------------------------ */

/*
 * Assemble, factor, solve (refined) and reduce one airfoil.  u[n+1] = (gamma,
 * C), cp[n] (may be NULL), out3 = (Cl, Cl_p, Cd_p) (may be NULL).
 * Returns 0, a negative geometry code (-1: n < 3, -2: clockwise or zero area),
 * or k+1 for a zero pivot at step k.
 */
int oracle_evaluate(int n, const double *nodes, double alpha, double vinf, double chord,
                    double *u, double *cp, double *out3) {
  if (n < 3) return -1;
  if (!(oracle_signed_area(n, nodes) > 0.0)) return -2;
  int m = n + 1;
  real *M = (real *)malloc(sizeof(real) * (size_t)m * m);
  real *LU = (real *)malloc(sizeof(real) * (size_t)m * m);
  real *b = (real *)malloc(sizeof(real) * (size_t)m);
  real *x = (real *)malloc(sizeof(real) * (size_t)m);
  int *piv = (int *)malloc(sizeof(int) * (size_t)m);
  assemble(n, nodes, alpha, vinf, M, b);
  memcpy(LU, M, sizeof(real) * (size_t)m * m);
  int info = lu_factor(m, LU, piv);
  if (info == 0) {
    memcpy(x, b, sizeof(real) * (size_t)m);
    lu_solve(m, LU, piv, x);
    refine(m, M, LU, piv, b, x, 2);
    for (int k = 0; k < m; ++k) u[k] = (double)x[k];
    if (cp || out3) {
      double tmp[3];
      forces(n, nodes, x, alpha, vinf, chord, cp, out3 ? out3 : tmp);
    }
  }
  free(M);
  free(LU);
  free(b);
  free(x);
  free(piv);
  return info;
}

/* ------------------------------------------------------------------------ */
/* Forward-mode dual numbers for the gradient oracle                        */
/* ------------------------------------------------------------------------ */

typedef struct { real v, d; } dual;

static dual dadd(dual a, dual b) { dual r = {a.v + b.v, a.d + b.d}; return r; }
static dual dsub(dual a, dual b) { dual r = {a.v - b.v, a.d - b.d}; return r; }
static dual dmul(dual a, dual b) { dual r = {a.v * b.v, a.d * b.v + a.v * b.d}; return r; }
static dual dscale(real s, dual a) { dual r = {s * a.v, s * a.d}; return r; }
static dual ddiv(dual a, dual b) {
  dual r = {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)};
  return r;
}
static dual dlog(dual a) { dual r = {R_LOG(a.v), a.d / a.v}; return r; }
static dual dsqrt(dual a) {
  real s = R_SQRT(a.v);
  dual r = {s, a.d / (2.0 * s)};
  return r;
}
static dual datan2(dual y, dual x) {
  dual r = {R_ATAN2(y.v, x.v), (x.v * y.d - y.v * x.d) / (x.v * x.v + y.v * y.v)};
  return r;
}

/* The same printed panel integral as panel_integral, in dual numbers. */
static dual panel_integral_dual(dual px, dual py, dual ax, dual ay, dual bx, dual by) {
  dual hx = dsub(bx, ax), hy = dsub(by, ay);
  dual hn = dsqrt(dadd(dmul(hx, hx), dmul(hy, hy)));
  dual dax = dsub(px, ax), day = dsub(py, ay);
  dual dbx = dsub(px, bx), dby = dsub(py, by);
  dual dot_a = dadd(dmul(dax, hx), dmul(day, hy));
  dual dot_b = dadd(dmul(dbx, hx), dmul(dby, hy));
  dual I = dsub(dmul(hy, dax), dmul(hx, day));
  dual ra2 = dadd(dmul(dax, dax), dmul(day, day));
  dual rb2 = dadd(dmul(dbx, dbx), dmul(dby, dby));
  dual t1 = dscale(0.5, dmul(dot_a, dlog(ra2)));
  dual t2 = dscale(0.5, dmul(dot_b, dlog(rb2)));
  dual t3 = dmul(I, datan2(I, dot_a));
  dual t4 = dmul(I, datan2(I, dot_b));
  dual bracket = dsub(dadd(dsub(dsub(t1, t2), t3), t4), dmul(hn, hn));
  return ddiv(bracket, dscale(TWO_PI, hn));
}

/* Value-and-tangent check hook: the dual integral with a tangent seed on the
 * six inputs (dp = d/ds of (px,py,ax,ay,bx,by)).  out2 = (value, derivative). */
void oracle_panel_integral_dual(const double *in6, const double *seed6, double *out2) {
  dual v[6];
  for (int k = 0; k < 6; ++k) { v[k].v = in6[k]; v[k].d = seed6[k]; }
  dual r = panel_integral_dual(v[0], v[1], v[2], v[3], v[4], v[5]);
  out2[0] = (double)r.v;
  out2[1] = (double)r.d;
}

/* Node i (closing convention) as a dual number, tangent 1 on coordinate
 * `coord` of node `k`. */
static void node_dual(const double *nodes, int n, int i, int k, int coord, dual *x, dual *y) {
  int ii = i % n;
  x->v = nodes[2 * ii];
  y->v = nodes[2 * ii + 1];
  x->d = (ii == k && coord == 0) ? 1.0 : 0.0;
  y->d = (ii == k && coord == 1) ? 1.0 : 0.0;
}

/*
 * Vector-Jacobian product for one airfoil by forward tangents: the gradient
 * with respect to the node coordinates of
 *   L = w_cl Cl + sum_j w_u[j] u_j + sum_j w_cp[j] Cp_j
 * with u = (gamma_0 .. gamma_{n-1}, C) (w_u of length n + 1, w_cp of length n,
 * either may be NULL = 0), through
 *   M du/ds = db/ds - (dM/ds) u,   dCl/ds = 2/(v_inf c) sum_i (du_i/ds |h_i| + u_i d|h_i|/ds),
 *   dCp_j/ds = -2 gamma_j dgamma_j/ds / v_inf^2,
 * for each of the 2n coordinates s, reusing the LU of M.  dM/ds is formed
 * entry by entry from the dual panel integral; entries that do not involve
 * node k (neither the control point nor the panel touches it) have zero
 * derivative and are skipped.  grad[2k+c] = dL/d(x_k)_c.  Returns the LU info
 * (0 on success) or a negative geometry code.
 */
static int vjp_nodes(int n, const double *nodes, double alpha, double vinf, double chord,
                     double w_cl, const double *w_u, const double *w_cp, int node_stride,
                     double *grad);

int oracle_vjp(int n, const double *nodes, double alpha, double vinf, double chord, double w_cl,
               const double *w_u, const double *w_cp, double *grad) {
  return vjp_nodes(n, nodes, alpha, vinf, chord, w_cl, w_u, w_cp, 1, grad);
}

/* The same product for the nodes k = 0, s, 2s, ... only (s = node_stride >= 1;
 * the other entries of grad are left untouched).  Each node's two tangents are
 * independent of the others', so the cost is the assembly, LU and solve of M
 * plus a part proportional to the nodes computed. */
static int vjp_nodes(int n, const double *nodes, double alpha, double vinf, double chord,
                     double w_cl, const double *w_u, const double *w_cp, int node_stride,
                     double *grad) {
  if (n < 3) return -1;
  if (!(oracle_signed_area(n, nodes) > 0.0)) return -2;
  int m = n + 1;
  real *M = (real *)malloc(sizeof(real) * (size_t)m * m);
  real *LU = (real *)malloc(sizeof(real) * (size_t)m * m);
  real *b = (real *)malloc(sizeof(real) * (size_t)m);
  real *u = (real *)malloc(sizeof(real) * (size_t)m);
  real *r = (real *)malloc(sizeof(real) * (size_t)m);
  int *piv = (int *)malloc(sizeof(int) * (size_t)m);
  const real ra = alpha, rv = vinf, rc = chord;
  assemble(n, nodes, ra, rv, M, b);
  memcpy(LU, M, sizeof(real) * (size_t)m * m);
  int info = lu_factor(m, LU, piv);
  if (info == 0) {
    memcpy(u, b, sizeof(real) * (size_t)m);
    lu_solve(m, LU, piv, u);
    refine(m, M, LU, piv, b, u, 2);
    for (int k = 0; k < n; k += node_stride) {
      for (int coord = 0; coord < 2; ++coord) {
        for (int j = 0; j < m; ++j) r[j] = 0.0;
        for (int j = 0; j < n; ++j) {
          int row_touches = (j % n == k) || ((j + 1) % n == k);
          dual xj, yj, xj1, yj1;
          node_dual(nodes, n, j, k, coord, &xj, &yj);
          node_dual(nodes, n, j + 1, k, coord, &xj1, &yj1);
          dual px = dscale(0.5, dadd(xj, xj1)), py = dscale(0.5, dadd(yj, yj1));
          /* right-hand side phi_v(x_{j+1/2}) */
          real dbj = rv * (py.d * R_COS(ra) - px.d * R_SIN(ra));
          real dMu = 0.0;
          for (int i = 0; i < n; ++i) {
            int col_touches = (i % n == k) || ((i + 1) % n == k);
            if (!row_touches && !col_touches) continue;
            dual xa, ya, xb, yb;
            node_dual(nodes, n, i, k, coord, &xa, &ya);
            node_dual(nodes, n, i + 1, k, coord, &xb, &yb);
            dual f = panel_integral_dual(px, py, xa, ya, xb, yb);
            dMu += (-f.d) * u[i]; /* d A_ji / ds * gamma_i */
          }
          r[j] = dbj - dMu;
        }
        r[n] = 0.0; /* the Kutta row is constant */
        lu_solve(m, LU, piv, r);
        real dcl = 0.0;
        for (int i = 0; i < n; ++i) {
          dual xa, ya, xb, yb;
          node_dual(nodes, n, i, k, coord, &xa, &ya);
          node_dual(nodes, n, i + 1, k, coord, &xb, &yb);
          dual hx = dsub(xb, xa), hy = dsub(yb, ya);
          dual len = dsqrt(dadd(dmul(hx, hx), dmul(hy, hy)));
          dcl += r[i] * len.v + u[i] * len.d;
        }
        real dl = (real)w_cl * 2.0 * dcl / (rv * rc);
        for (int j = 0; j < m; ++j)
          if (w_u) dl += (real)w_u[j] * r[j];
        for (int j = 0; j < n; ++j)
          if (w_cp) dl += (real)w_cp[j] * (-2.0 * u[j] * r[j] / (rv * rv));
        grad[2 * k + coord] = (double)dl;
      }
    }
  }
  free(M);
  free(LU);
  free(b);
  free(u);
  free(r);
  free(piv);
  return info;
}

/* dCl/d(node coordinates): the product above with w_cl = 1 alone. */
int oracle_cl_gradient(int n, const double *nodes, double alpha, double vinf, double chord,
                       double *grad) {
  return oracle_vjp(n, nodes, alpha, vinf, chord, 1.0, NULL, NULL, grad);
}

/* ------------------------------------------------------------------------ */
/* Ragged batches (airfoils are independent; OpenMP across airfoils)        */
/* ------------------------------------------------------------------------ */

/*
 * Airfoil b has n_b = offsets[b+1] - offsets[b] nodes starting at
 * nodes[2*offsets[b]].  Outputs are packed the same way: u at
 * u[offsets[b] + b .. + n_b] (n_b + 1 values), cp at cp[offsets[b] ..],
 * cl/clp/cdp/info at [b].  vinf/chord/clp/cdp/cp may be NULL (defaults 1).
 * nthreads <= 0 uses the OpenMP default.
 */
void oracle_evaluate_batch(int B, const double *nodes, const int64_t *offsets,
                           const double *alpha, const double *vinf, const double *chord,
                           double *u, double *cp, double *cl, double *clp, double *cdp,
                           int32_t *info, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
  for (int b = 0; b < B; ++b) {
    int64_t off = offsets[b];
    int n = (int)(offsets[b + 1] - off);
    double out3[3] = {NAN, NAN, NAN};
    double v = vinf ? vinf[b] : 1.0, c = chord ? chord[b] : 1.0;
    int st = oracle_evaluate(n, nodes + 2 * off, alpha[b], v, c, u + off + b,
                             cp ? cp + off : NULL, out3);
    cl[b] = out3[0];
    if (clp) clp[b] = out3[1];
    if (cdp) cdp[b] = out3[2];
    info[b] = st;
  }
}

/* dCl/d(nodes) for a ragged batch; grad packed like nodes ([sum n_b][2]). */
void oracle_cl_gradient_batch(int B, const double *nodes, const int64_t *offsets,
                              const double *alpha, const double *vinf, const double *chord,
                              double *grad, int32_t *info, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
  for (int b = 0; b < B; ++b) {
    int64_t off = offsets[b];
    int n = (int)(offsets[b + 1] - off);
    double v = vinf ? vinf[b] : 1.0, c = chord ? chord[b] : 1.0;
    info[b] = oracle_cl_gradient(n, nodes + 2 * off, alpha[b], v, c, grad + 2 * off);
  }
}

/* dCl/d(nodes) of the nodes k = 0, s, 2s, ... of every airfoil (grad packed like
 * the nodes; the other entries are left untouched): a bounded sample of the
 * gradient's work for timing the oracle on large airfoils. */
void oracle_cl_gradient_strided_batch(int B, const double *nodes, const int64_t *offsets,
                                      const double *alpha, const double *vinf, const double *chord,
                                      int node_stride, double *grad, int32_t *info, int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
  for (int b = 0; b < B; ++b) {
    int64_t off = offsets[b];
    int n = (int)(offsets[b + 1] - off);
    double v = vinf ? vinf[b] : 1.0, c = chord ? chord[b] : 1.0;
    info[b] = vjp_nodes(n, nodes + 2 * off, alpha[b], v, c, 1.0, NULL, NULL,
                        node_stride < 1 ? 1 : node_stride, grad + 2 * off);
  }
}

/* Number of OpenMP threads a parallel region would use. */
int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
