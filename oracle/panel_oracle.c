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
 *              and back substitution (Section 3 names LU as the solver);
 *   forces     surface speed |gamma_j|, Cp_j = 1 - (gamma_j / v_inf)^2,
 *              Cl = 2 sum_i gamma_i |h_i| / (v_inf c) (Kutta-Joukowski), and the
 *              pressure-integrated Cl_p, Cd_p.  The paper reports C_L without a
 *              formula (Section 2, Figure 2 tables); these are the textbook ones.
 *   gradient   dCl/d(node coordinates) by forward-mode dual numbers pushed
 *              through the same influence formula and a re-solve with the LU,
 *              one tangent per coordinate (O(n^3) per airfoil by design).
 *
 * Everything is IEEE double, no fast-math, no blocking or reordering beyond the
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

static const double TWO_PI = 6.283185307179586476925286766559;

/* ------------------------------------------------------------------------ */
/* Geometry (Section 2, Figure 1)                                           */
/* ------------------------------------------------------------------------ */

/* Node i of an n-node airfoil with the closing convention x_n = x_0. */
static void node(const double *nodes, int n, int i, double *x, double *y) {
  int k = i % n;
  *x = nodes[2 * k];
  *y = nodes[2 * k + 1];
}

/* Signed polygon area (shoelace); positive for counter-clockwise nodes. */
double oracle_signed_area(int n, const double *nodes) {
  double a = 0.0;
  for (int i = 0; i < n; ++i) {
    double x0, y0, x1, y1;
    node(nodes, n, i, &x0, &y0);
    node(nodes, n, i + 1, &x1, &y1);
    a += x0 * y1 - x1 * y0;
  }
  return 0.5 * a;
}

/* ------------------------------------------------------------------------ */
/* Panel integral F_i (Section 2), literally as printed                     */
/* ------------------------------------------------------------------------ */

/*
 * Returns F_i(p) / gamma_i for the panel from a = x_i to b = x_{i+1}:
 *
 *   (1/2pi)(1/|h|) [ 1/2 <p-a,h> log|p-a|^2 - 1/2 <p-b,h> log|p-b|^2
 *                    - I atan2(I, <p-a,h>) + I atan2(I, <p-b,h>) - |h|^2 ]
 *
 * with h = b - a, I = <h_perp, p-a>, h_perp = (h_y, -h_x) (outward for
 * counter-clockwise nodes, |h_perp| = |h|).
 */
double oracle_panel_integral(double px, double py, double ax, double ay, double bx,
                             double by) {
  double hx = bx - ax, hy = by - ay;
  double hn = sqrt(hx * hx + hy * hy);
  double dax = px - ax, day = py - ay; /* p - x_i     */
  double dbx = px - bx, dby = py - by; /* p - x_{i+1} */
  double dot_a = dax * hx + day * hy;  /* <p - x_i, h>     */
  double dot_b = dbx * hx + dby * hy;  /* <p - x_{i+1}, h> */
  double I = hy * dax - hx * day;      /* <h_perp, p - x_i> */
  double ra2 = dax * dax + day * day;
  double rb2 = dbx * dbx + dby * dby;
  double bracket = 0.5 * dot_a * log(ra2) - 0.5 * dot_b * log(rb2) - I * atan2(I, dot_a) +
                   I * atan2(I, dot_b) - hn * hn;
  return bracket / (hn * TWO_PI);
}

/* A_ji = -F_i(x_{j+1/2}) / gamma_i: the coefficient of gamma_i in row j. */
static double influence(const double *nodes, int n, int j, int i) {
  double xj, yj, xj1, yj1, xa, ya, xb, yb;
  node(nodes, n, j, &xj, &yj);
  node(nodes, n, j + 1, &xj1, &yj1);
  node(nodes, n, i, &xa, &ya);
  node(nodes, n, i + 1, &xb, &yb);
  double px = 0.5 * (xj + xj1), py = 0.5 * (yj + yj1);
  return -oracle_panel_integral(px, py, xa, ya, xb, yb);
}

/* ------------------------------------------------------------------------ */
/* Bordered system (Section 2): rows 0..n-1 collocation, row n Kutta        */
/* ------------------------------------------------------------------------ */

/*
 * M is (n+1) x (n+1), row-major.  Unknowns u = (gamma_0 .. gamma_{n-1}, C).
 *   M[j][i] = A_ji, M[j][n] = 1, b_j = phi_v(x_{j+1/2})           (j < n)
 *   M[n][0] = M[n][n-1] = 1, all other M[n][*] = 0, b_n = 0         (Kutta)
 */
void oracle_assemble(int n, const double *nodes, double alpha, double vinf, double *M,
                     double *b) {
  int m = n + 1;
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < n; ++i) M[j * m + i] = influence(nodes, n, j, i);
    M[j * m + n] = 1.0;
    double xj, yj, xj1, yj1;
    node(nodes, n, j, &xj, &yj);
    node(nodes, n, j + 1, &xj1, &yj1);
    double px = 0.5 * (xj + xj1), py = 0.5 * (yj + yj1);
    b[j] = vinf * (py * cos(alpha) - px * sin(alpha));
  }
  for (int i = 0; i < m; ++i) M[n * m + i] = 0.0;
  M[n * m + 0] = 1.0;
  M[n * m + (n - 1)] = 1.0;
  b[n] = 0.0;
}

/* ------------------------------------------------------------------------ */
/* Dense LU with partial pivoting (Doolittle, in place, row-major)          */
/* ------------------------------------------------------------------------ */

/* piv[k] = row exchanged with row k at step k.  Returns 0, or k+1 if the
 * k-th pivot is exactly zero (LAPACK convention; factorisation stops). */
int oracle_lu_factor(int m, double *A, int *piv) {
  for (int k = 0; k < m; ++k) {
    int p = k;
    double best = fabs(A[k * m + k]);
    for (int r = k + 1; r < m; ++r) {
      double v = fabs(A[r * m + k]);
      if (v > best) { best = v; p = r; }
    }
    piv[k] = p;
    if (best == 0.0) return k + 1;
    if (p != k) {
      for (int c = 0; c < m; ++c) {
        double t = A[k * m + c];
        A[k * m + c] = A[p * m + c];
        A[p * m + c] = t;
      }
    }
    for (int r = k + 1; r < m; ++r) {
      double l = A[r * m + k] / A[k * m + k];
      A[r * m + k] = l;
      for (int c = k + 1; c < m; ++c) A[r * m + c] -= l * A[k * m + c];
    }
  }
  return 0;
}

/* Solve (LU) x = P b in place given the factors of oracle_lu_factor. */
void oracle_lu_solve(int m, const double *LU, const int *piv, double *x) {
  for (int k = 0; k < m; ++k) {
    int p = piv[k];
    if (p != k) { double t = x[k]; x[k] = x[p]; x[p] = t; }
  }
  for (int r = 1; r < m; ++r)
    for (int c = 0; c < r; ++c) x[r] -= LU[r * m + c] * x[c];
  for (int r = m - 1; r >= 0; --r) {
    for (int c = r + 1; c < m; ++c) x[r] -= LU[r * m + c] * x[c];
    x[r] /= LU[r * m + r];
  }
}

/* Solve (LU)^T y = g, i.e. M^T y = g, given the factors of oracle_lu_factor. */
void oracle_lu_solve_transposed(int m, const double *LU, const int *piv, double *y) {
  /* M = P^T L U  =>  M^T = U^T L^T P.  Solve U^T z = g, L^T w = z, y = P^T w. */
  for (int r = 0; r < m; ++r) {
    for (int c = 0; c < r; ++c) y[r] -= LU[c * m + r] * y[c];
    y[r] /= LU[r * m + r];
  }
  for (int r = m - 1; r >= 0; --r)
    for (int c = r + 1; c < m; ++c) y[r] -= LU[c * m + r] * y[c];
  for (int k = m - 1; k >= 0; --k) {
    int p = piv[k];
    if (p != k) { double t = y[k]; y[k] = y[p]; y[p] = t; }
  }
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
void oracle_forces(int n, const double *nodes, const double *u, double alpha, double vinf,
                   double chord, double *cp, double *out3) {
  double circ = 0.0, fx = 0.0, fy = 0.0;
  for (int j = 0; j < n; ++j) {
    double xa, ya, xb, yb;
    node(nodes, n, j, &xa, &ya);
    node(nodes, n, j + 1, &xb, &yb);
    double hx = xb - xa, hy = yb - ya;
    double len = sqrt(hx * hx + hy * hy);
    double g = u[j];
    double c = 1.0 - (g / vinf) * (g / vinf);
    if (cp) cp[j] = c;
    circ += g * len;
    fx -= c * hy;   /* -Cp * n_x * |h| with n_x |h| = h_y  */
    fy -= c * (-hx); /* -Cp * n_y * |h| with n_y |h| = -h_x */
  }
  out3[0] = 2.0 * circ / (vinf * chord);
  out3[1] = (-fx * sin(alpha) + fy * cos(alpha)) / chord;
  out3[2] = (fx * cos(alpha) + fy * sin(alpha)) / chord;
}

/* ------------------------------------------------------------------------ */
/* One airfoil, end to end                                                  */
/* ------------------------------------------------------------------------ */

/*
 * Assemble, factor, solve and reduce one airfoil.  u[n+1] = (gamma, C),
 * cp[n] (may be NULL), out3 = (Cl, Cl_p, Cd_p) (may be NULL).
 * Returns 0, a negative geometry code (-1: n < 3, -2: clockwise or zero area),
 * or k+1 for a zero pivot at step k.
 */
int oracle_evaluate(int n, const double *nodes, double alpha, double vinf, double chord,
                    double *u, double *cp, double *out3) {
  if (n < 3) return -1;
  if (!(oracle_signed_area(n, nodes) > 0.0)) return -2;
  int m = n + 1;
  double *M = (double *)malloc(sizeof(double) * (size_t)m * m);
  int *piv = (int *)malloc(sizeof(int) * (size_t)m);
  oracle_assemble(n, nodes, alpha, vinf, M, u);
  int info = oracle_lu_factor(m, M, piv);
  if (info == 0) {
    oracle_lu_solve(m, M, piv, u);
    if (cp || out3) {
      double tmp[3];
      oracle_forces(n, nodes, u, alpha, vinf, chord, cp, out3 ? out3 : tmp);
    }
  }
  free(M);
  free(piv);
  return info;
}

/* ------------------------------------------------------------------------ */
/* Forward-mode dual numbers for the gradient oracle                        */
/* ------------------------------------------------------------------------ */

typedef struct { double v, d; } dual;

static dual dc(double v) { dual r = {v, 0.0}; return r; }
static dual dadd(dual a, dual b) { dual r = {a.v + b.v, a.d + b.d}; return r; }
static dual dsub(dual a, dual b) { dual r = {a.v - b.v, a.d - b.d}; return r; }
static dual dmul(dual a, dual b) { dual r = {a.v * b.v, a.d * b.v + a.v * b.d}; return r; }
static dual dscale(double s, dual a) { dual r = {s * a.v, s * a.d}; return r; }
static dual ddiv(dual a, dual b) {
  dual r = {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)};
  return r;
}
static dual dlog(dual a) { dual r = {log(a.v), a.d / a.v}; return r; }
static dual dsqrt(dual a) {
  double s = sqrt(a.v);
  dual r = {s, a.d / (2.0 * s)};
  return r;
}
static dual datan2(dual y, dual x) {
  dual r = {atan2(y.v, x.v), (x.v * y.d - y.v * x.d) / (x.v * x.v + y.v * y.v)};
  return r;
}

/* The same printed panel integral as oracle_panel_integral, in dual numbers. */
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
  out2[0] = r.v;
  out2[1] = r.d;
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
 * dCl/d(node coordinates) for one airfoil by forward tangents:
 *   M du/ds = db/ds - (dM/ds) u,   dCl/ds = 2/(v_inf c) sum_i (du_i/ds |h_i| + u_i d|h_i|/ds)
 * for each of the 2n coordinates s, reusing the LU of M.  dM/ds is formed
 * entry by entry from the dual panel integral; entries that do not involve
 * node k (neither the control point nor the panel touches it) have zero
 * derivative and are skipped.  grad[2k+c] = dCl/d(x_k)_c.  Returns the LU info
 * (0 on success) or a negative geometry code.
 */
int oracle_cl_gradient(int n, const double *nodes, double alpha, double vinf, double chord,
                       double *grad) {
  if (n < 3) return -1;
  if (!(oracle_signed_area(n, nodes) > 0.0)) return -2;
  int m = n + 1;
  double *M = (double *)malloc(sizeof(double) * (size_t)m * m);
  double *u = (double *)malloc(sizeof(double) * (size_t)m);
  double *r = (double *)malloc(sizeof(double) * (size_t)m);
  int *piv = (int *)malloc(sizeof(int) * (size_t)m);
  oracle_assemble(n, nodes, alpha, vinf, M, u);
  int info = oracle_lu_factor(m, M, piv);
  if (info == 0) {
    oracle_lu_solve(m, M, piv, u);
    for (int k = 0; k < n; ++k) {
      for (int coord = 0; coord < 2; ++coord) {
        for (int j = 0; j < m; ++j) r[j] = 0.0;
        for (int j = 0; j < n; ++j) {
          int row_touches = (j % n == k) || ((j + 1) % n == k);
          dual xj, yj, xj1, yj1;
          node_dual(nodes, n, j, k, coord, &xj, &yj);
          node_dual(nodes, n, j + 1, k, coord, &xj1, &yj1);
          dual px = dscale(0.5, dadd(xj, xj1)), py = dscale(0.5, dadd(yj, yj1));
          /* right-hand side phi_v(x_{j+1/2}) */
          double dbj = vinf * (py.d * cos(alpha) - px.d * sin(alpha));
          double dMu = 0.0;
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
        oracle_lu_solve(m, M, piv, r);
        double dcl = 0.0;
        for (int i = 0; i < n; ++i) {
          dual xa, ya, xb, yb;
          node_dual(nodes, n, i, k, coord, &xa, &ya);
          node_dual(nodes, n, i + 1, k, coord, &xb, &yb);
          dual hx = dsub(xb, xa), hy = dsub(yb, ya);
          dual len = dsqrt(dadd(dmul(hx, hx), dmul(hy, hy)));
          dcl += r[i] * len.v + u[i] * len.d;
        }
        grad[2 * k + coord] = 2.0 * dcl / (vinf * chord);
      }
    }
  }
  free(M);
  free(u);
  free(r);
  free(piv);
  return info;
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

/* Number of OpenMP threads a parallel region would use. */
int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
