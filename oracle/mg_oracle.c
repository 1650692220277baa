/*
 * mg_oracle.c -- plain, slow, obviously-correct FP64 CPU multigrid (the oracle).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the CPU-baseline
 * leg of bench.py.  The CUDA solver never includes, links or calls it.
 *
 * What it follows (J. T. Wallis, "Methods toward better Multigrid Solver
 * Convergence", 2008):
 *   - the problem: Poisson / anisotropic / mapped-coordinate diffusion operators
 *     ("Introduction / Motivation": gravity Poisson problem, grid transformed to
 *     the unit square; "Anisotropies": -alpha u_xx - beta u_yy);
 *   - the smoothers: preconditioned Richardson x <- x - omega C^{-1}(A x - b)
 *     ("Smoothers") with the choices of C of "The choice of C": Jacobi (C = D),
 *     Gauss-Seidel (here in red-black order), and the tridiagonal line
 *     preconditioner TRI along x or y (here in Jacobi and zebra orders);
 *   - the multigrid algorithm MG(l, u, g) of "The Multigrid Technique": pre-
 *     smoothing, restriction of the defect, recursive coarse solves starting
 *     from zero, correction u + omega_l P e, post-smoothing, and A_1^{-1} g on
 *     the coarsest grid; the cycle is the F-cycle named in the abstract.
 * Where the paper is silent the readings are: rediscretised coarse operators
 * (edge weights coarsened by a harmonic mean along the edge, injection across
 * and a factor 1/4 for h -> 2h; cell coefficients averaged over children),
 * full-weighting restriction, bilinear/trilinear prolongation, red-before-black
 * (even lines before odd lines) in every smoothing step, and stopping on the
 * relative 2-norm residual ||b - A x|| / ||b|| over the unknowns.
 *
 * Plain loops, no blocking, no fusion: each function is one step of the method.
 */
#include "mg_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef OR_THREADED
#include <omp.h>
#endif

/* The timed CPU baseline builds this file a second time with -fopenmp -DOR_THREADED: the
 * loops marked OR_PAR_ROWS then run their grid rows (and the line loops their lines) on all
 * host cores.  Every node's arithmetic is the same in both builds, and each marked loop writes
 * only its own nodes from values no other iteration of it writes (one colour of red-black
 * Gauss-Seidel reads only the other colour; lines of one zebra colour are independent), so
 * the two builds give identical results.  Sums over the grid (norms) stay serial. */
#ifdef OR_THREADED
#define OR_PAR_ROWS _Pragma("omp parallel for collapse(2) schedule(static)")
#else
#define OR_PAR_ROWS
#endif

typedef struct {
  int dim, n[3], per, kind;
  double h[3], c[3];
  double *sx, *sy, *sz, *k;   /* owned copies of the coefficients of this level */
  double *ex, *ey, *ez;       /* OR_EDGE: per-node weights of the +x, +y, +z edges */
  double *st9;                /* Galerkin coarse levels (2-D): the 9-point stencil of every node,
                                 st9[9 p + 3 (b + 1) + (a + 1)] = A(p, p + (a, b)); NULL otherwise */
  double *u, *g, *r;          /* work vectors of this level (full node arrays) */
  long nsmooth;
} lev_t;

struct or_hier {
  int L;
  lev_t lev[OR_MAXLEV + 1];   /* lev[1] coarsest ... lev[L] finest */
  int smoother, nu1, nu2, coarse_mode, coarse_sweeps, dense_max;
  double omega, omega_corr;
  int adaptive_corr;
  int galerkin;
  /* coarsest-grid direct solver */
  int nc;                     /* number of coarsest unknowns */
  size_t *cidx;               /* node index of each coarsest unknown */
  double *chol;               /* dense Cholesky factor (row-major lower), or NULL -> CG */
  long ncoarse;
};

/* ------------------------------------------------------------------------- */
/* grid helpers                                                              */
/* ------------------------------------------------------------------------- */

static size_t nodes(const lev_t *v) { return (size_t)v->n[0] * v->n[1] * v->n[2]; }
static size_t nid(const lev_t *v, int i, int j, int k) { return ((size_t)k * v->n[1] + j) * v->n[0] + i; }
static int ywrap(const lev_t *v, int j) {
  if (!v->per) return j;
  return ((j % v->n[1]) + v->n[1]) % v->n[1];
}
static int is_unk(const lev_t *v, int i, int j, int k) {
  if (i < 1 || i > v->n[0] - 2) return 0;
  if (!v->per && (j < 1 || j > v->n[1] - 2)) return 0;
  if (v->dim == 3 && (k < 1 || k > v->n[2] - 2)) return 0;
  return 1;
}
/* u at node (i,j,k); Dirichlet nodes read as zero */
static double val(const lev_t *v, const double *u, int i, int j, int k) {
  j = ywrap(v, j);
  return is_unk(v, i, j, k) ? u[nid(v, i, j, k)] : 0.0;
}
static int ncells_y(const lev_t *v) { return v->per ? v->n[1] : v->n[1] - 1; }
static double kcell(const lev_t *v, int i, int j, int k) {
  j = ywrap(v, j);
  return v->k[((size_t)k * ncells_y(v) + j) * (v->n[0] - 1) + i];
}

/* Edge weights.  For the cell-coefficient kind -div(k grad u) the weight of an
 * edge is the mean of the cells touching it divided by h^2 (finite-volume flux
 * over the dual face); it is linear in k. */
static double wx_edge(const lev_t *v, int i, int j, int k) { /* (i,j,k)-(i+1,j,k) */
  if (v->kind == OR_EDGE) return v->ex[nid(v, i, j, k)];
  if (v->kind == OR_CONST) return v->c[0];
  if (v->kind == OR_SEPARABLE) return v->sx[i];
  if (v->dim == 2) return (kcell(v, i, j - 1, 0) + kcell(v, i, j, 0)) / (2.0 * v->h[0] * v->h[0]);
  return (kcell(v, i, j - 1, k - 1) + kcell(v, i, j, k - 1) + kcell(v, i, j - 1, k) + kcell(v, i, j, k)) /
         (4.0 * v->h[0] * v->h[0]);
}
static double wy_edge(const lev_t *v, int i, int j, int k) { /* (i,j,k)-(i,j+1,k) */
  if (v->kind == OR_EDGE) return v->ey[nid(v, i, j, k)];
  if (v->kind == OR_CONST) return v->c[1];
  if (v->kind == OR_SEPARABLE) return v->sy[i];
  if (v->dim == 2) return (kcell(v, i - 1, j, 0) + kcell(v, i, j, 0)) / (2.0 * v->h[1] * v->h[1]);
  return (kcell(v, i - 1, j, k - 1) + kcell(v, i, j, k - 1) + kcell(v, i - 1, j, k) + kcell(v, i, j, k)) /
         (4.0 * v->h[1] * v->h[1]);
}
static double wz_edge(const lev_t *v, int i, int j, int k) { /* (i,j,k)-(i,j,k+1) */
  if (v->kind == OR_EDGE) return v->ez[nid(v, i, j, k)];
  if (v->kind == OR_CONST) return v->c[2];
  if (v->kind == OR_SEPARABLE) return v->sz[i];
  return (kcell(v, i - 1, j - 1, k) + kcell(v, i, j - 1, k) + kcell(v, i - 1, j, k) + kcell(v, i, j, k)) /
         (4.0 * v->h[2] * v->h[2]);
}

/* (A u)_p = sum over the edges at p of w_e (u_p - u_q); on a Galerkin level the sum over the
 * 9-point stencil, sum_{a,b} A(p, p + (a, b)) u_{p + (a, b)} */
static double apply_at(const lev_t *v, const double *u, int i, int j, int k) {
  if (v->st9) {
    const double *a9 = v->st9 + 9 * nid(v, i, j, k);
    double s9 = 0.0;
    for (int b = -1; b <= 1; ++b)
      for (int a = -1; a <= 1; ++a) s9 += a9[3 * (b + 1) + (a + 1)] * val(v, u, i + a, j + b, k);
    return s9;
  }
  double up = u[nid(v, i, j, k)], s = 0.0;
  s += wx_edge(v, i - 1, j, k) * (up - val(v, u, i - 1, j, k));
  s += wx_edge(v, i, j, k) * (up - val(v, u, i + 1, j, k));
  s += wy_edge(v, i, ywrap(v, j - 1), k) * (up - val(v, u, i, j - 1, k));
  s += wy_edge(v, i, j, k) * (up - val(v, u, i, j + 1, k));
  if (v->dim == 3) {
    s += wz_edge(v, i, j, k - 1) * (up - val(v, u, i, j, k - 1));
    s += wz_edge(v, i, j, k) * (up - val(v, u, i, j, k + 1));
  }
  return s;
}
/* D_p = sum of the weights of the edges at p (Dirichlet edges included) */
static double diag_at(const lev_t *v, int i, int j, int k) {
  if (v->st9) return v->st9[9 * nid(v, i, j, k) + 4];
  double s = wx_edge(v, i - 1, j, k) + wx_edge(v, i, j, k) + wy_edge(v, i, ywrap(v, j - 1), k) + wy_edge(v, i, j, k);
  if (v->dim == 3) s += wz_edge(v, i, j, k - 1) + wz_edge(v, i, j, k);
  return s;
}

#define FOR_NODES(v) \
  for (int k = 0; k < (v)->n[2]; ++k) \
    for (int j = 0; j < (v)->n[1]; ++j) \
      for (int i = 0; i < (v)->n[0]; ++i)

/* ------------------------------------------------------------------------- */
/* operator, defect, norm                                                    */
/* ------------------------------------------------------------------------- */

static void lev_apply(const lev_t *v, const double *u, double *Au) {
  OR_PAR_ROWS
  FOR_NODES(v) Au[nid(v, i, j, k)] = is_unk(v, i, j, k) ? apply_at(v, u, i, j, k) : 0.0;
}
static void lev_defect(const lev_t *v, const double *u, const double *g, double *r) {
  OR_PAR_ROWS
  FOR_NODES(v) {
    size_t p = nid(v, i, j, k);
    r[p] = is_unk(v, i, j, k) ? g[p] - apply_at(v, u, i, j, k) : 0.0;
  }
}
static double lev_norm2(const lev_t *v, const double *x) {
  double s = 0.0;
  FOR_NODES(v) if (is_unk(v, i, j, k)) { double t = x[nid(v, i, j, k)]; s += t * t; }
  return sqrt(s);
}

/* ------------------------------------------------------------------------- */
/* smoothers: x <- x + omega C^{-1} (b - A x)   (section "Smoothers")        */
/* ------------------------------------------------------------------------- */

/* Thomas algorithm for a tridiagonal system lo[i] x[i-1] + di[i] x[i] + up[i] x[i+1] = d[i] */
void or_thomas(int m, const double *lo, const double *di, const double *up, const double *d, double *x) {
  double *cp = (double *)malloc(sizeof(double) * (size_t)m), *dp = (double *)malloc(sizeof(double) * (size_t)m);
  cp[0] = up[0] / di[0];
  dp[0] = d[0] / di[0];
  for (int i = 1; i < m; ++i) {
    double den = di[i] - lo[i] * cp[i - 1];
    cp[i] = up[i] / den;
    dp[i] = (d[i] - lo[i] * dp[i - 1]) / den;
  }
  x[m - 1] = dp[m - 1];
  for (int i = m - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
  free(cp);
  free(dp);
}

/* Cyclic tridiagonal system: rows t = 0..m-1 with lo[t] x_{t-1} + di[t] x_t + up[t] x_{t+1} = d[t],
 * indices modulo m (lo[0] couples to x_{m-1}, up[m-1] to x_0), m >= 3.  Sherman-Morrison: with
 * gamma = -di[0], A = T + u v^T where T is A without its two corners and with di[0] - gamma and
 * di[m-1] - up[m-1] lo[0] / gamma on the diagonal, u = (gamma, 0, .., 0, up[m-1]),
 * v = (1, 0, .., 0, lo[0] / gamma); then x = y - (v.y / (1 + v.z)) z with T y = d, T z = u. */
void or_cyclic_thomas(int m, const double *lo, const double *di, const double *up, const double *d, double *x) {
  double *l2 = (double *)malloc(sizeof(double) * (size_t)m), *d2 = (double *)malloc(sizeof(double) * (size_t)m);
  double *u2 = (double *)malloc(sizeof(double) * (size_t)m), *uu = (double *)calloc((size_t)m, sizeof(double));
  double *y = (double *)malloc(sizeof(double) * (size_t)m), *z = (double *)malloc(sizeof(double) * (size_t)m);
  double alpha = up[m - 1], beta = lo[0], gamma = -di[0];
  for (int t = 0; t < m; ++t) { l2[t] = lo[t]; d2[t] = di[t]; u2[t] = up[t]; }
  l2[0] = 0.0;
  u2[m - 1] = 0.0;
  d2[0] = di[0] - gamma;
  d2[m - 1] = di[m - 1] - alpha * beta / gamma;
  uu[0] = gamma;
  uu[m - 1] = alpha;
  or_thomas(m, l2, d2, u2, d, y);
  or_thomas(m, l2, d2, u2, uu, z);
  double fac = (y[0] + beta / gamma * y[m - 1]) / (1.0 + z[0] + beta / gamma * z[m - 1]);
  for (int t = 0; t < m; ++t) x[t] = y[t] - fac * z[t];
  free(l2); free(d2); free(u2); free(uu); free(y); free(z);
}

/* Jacobi, C = D: every unknown is corrected from the same old iterate */
static void sweep_jacobi(const lev_t *v, double *u, const double *g, double omega, double *r) {
  lev_defect(v, u, g, r);
  OR_PAR_ROWS
  FOR_NODES(v) if (is_unk(v, i, j, k)) u[nid(v, i, j, k)] += omega * r[nid(v, i, j, k)] / diag_at(v, i, j, k);
}

/* Gauss-Seidel in red-black order: red = (i+j+k) even.  One colour at a time,
 * each unknown corrected with the current iterate. */
static void halfsweep_rb(const lev_t *v, double *u, const double *g, double omega, int colour) {
  OR_PAR_ROWS
  FOR_NODES(v) {
    if (!is_unk(v, i, j, k) || ((i + j + k) & 1) != colour) continue;
    size_t p = nid(v, i, j, k);
    u[p] += omega * (g[p] - apply_at(v, u, i, j, k)) / diag_at(v, i, j, k);
  }
}

/* Gauss-Seidel on a Galerkin level (9-point stencil): nodes of one of the four colours
 * (i mod 2, j mod 2) = (ci, cj) at a time, each corrected with the current iterate.  Nodes of one
 * colour lie two apart and do not couple, and the two colours with i + j even (odd) together
 * make up the red (black) nodes of the red-black order; on a 5-point level the four-colour
 * order is the red-black one. */
static void quartersweep(const lev_t *v, double *u, const double *g, double omega, int ci, int cj) {
  OR_PAR_ROWS
  FOR_NODES(v) {
    if (!is_unk(v, i, j, k) || (i & 1) != ci || (j & 1) != cj) continue;
    size_t p = nid(v, i, j, k);
    u[p] += omega * (g[p] - apply_at(v, u, i, j, k)) / diag_at(v, i, j, k);
  }
}

/* One line of the TRI preconditioner: C restricted to the line is the
 * tridiagonal part of A along the line (diagonal D plus the couplings to the
 * line neighbours).  dir 0: line along x at (j,k); dir 1: line along y at (i,k).
 * Solves C_line delta = r_line and adds omega * delta. */
static void line_update(const lev_t *v, double *u, const double *r, double omega, int dir, int a, int b,
                        double *lo, double *di, double *up, double *rhs, double *dx) {
  int m;
  if (dir == 0) { /* x-line: j = a, k = b, unknowns i = 1..n0-2 */
    m = v->n[0] - 2;
    for (int t = 0; t < m; ++t) {
      int i = t + 1;
      di[t] = diag_at(v, i, a, b);
      lo[t] = (t > 0) ? -wx_edge(v, i - 1, a, b) : 0.0;
      up[t] = (t < m - 1) ? -wx_edge(v, i, a, b) : 0.0;
      rhs[t] = r[nid(v, i, a, b)];
    }
    or_thomas(m, lo, di, up, rhs, dx);
    for (int t = 0; t < m; ++t) u[nid(v, t + 1, a, b)] += omega * dx[t];
  } else if (v->per) { /* periodic y-line: i = a, k = b, every row j = 0..n1-1; cyclic system */
    m = v->n[1];
    for (int j = 0; j < m; ++j) {
      di[j] = diag_at(v, a, j, b);
      lo[j] = -wy_edge(v, a, ywrap(v, j - 1), b);   /* the edge to row j-1 (row 0: to row n1-1) */
      up[j] = -wy_edge(v, a, j, b);                  /* the edge to row j+1 (row n1-1: to row 0) */
      rhs[j] = r[nid(v, a, j, b)];
    }
    or_cyclic_thomas(m, lo, di, up, rhs, dx);
    for (int j = 0; j < m; ++j) u[nid(v, a, j, b)] += omega * dx[j];
  } else { /* y-line: i = a, k = b, unknowns j = 1..n1-2 */
    m = v->n[1] - 2;
    for (int t = 0; t < m; ++t) {
      int j = t + 1;
      di[t] = diag_at(v, a, j, b);
      lo[t] = (t > 0) ? -wy_edge(v, a, j - 1, b) : 0.0;
      up[t] = (t < m - 1) ? -wy_edge(v, a, j, b) : 0.0;
      rhs[t] = r[nid(v, a, j, b)];
    }
    or_thomas(m, lo, di, up, rhs, dx);
    for (int t = 0; t < m; ++t) u[nid(v, a, t + 1, b)] += omega * dx[t];
  }
}

/* every line of direction dir in planes kz0..kz1 whose colour matches (colour < 0: every line) */
static void update_lines(const lev_t *v, double *u, const double *r, double omega, int dir, int colour, int kz0,
                         int kz1) {
#ifdef OR_THREADED
#pragma omp parallel
#endif
  {
    int len = v->n[dir];
    double *lo = (double *)malloc(sizeof(double) * len), *di = (double *)malloc(sizeof(double) * len);
    double *up = (double *)malloc(sizeof(double) * len), *rhs = (double *)malloc(sizeof(double) * len);
    double *dx = (double *)malloc(sizeof(double) * len);
    if (dir == 0) {
      int j0 = v->per ? 0 : 1, j1 = v->per ? v->n[1] - 1 : v->n[1] - 2;
#ifdef OR_THREADED
#pragma omp for collapse(2) schedule(static)
#endif
      for (int k = kz0; k <= kz1; ++k)
        for (int j = j0; j <= j1; ++j)
          if (colour < 0 || ((j + k) & 1) == colour) line_update(v, u, r, omega, 0, j, k, lo, di, up, rhs, dx);
    } else {
#ifdef OR_THREADED
#pragma omp for collapse(2) schedule(static)
#endif
      for (int k = kz0; k <= kz1; ++k)
        for (int i = 1; i <= v->n[0] - 2; ++i)
          if (colour < 0 || ((i + k) & 1) == colour) line_update(v, u, r, omega, 1, i, k, lo, di, up, rhs, dx);
    }
    free(lo); free(di); free(up); free(rhs); free(dx);
  }
}

/* line smoothers: zebra = 0 -> line Jacobi (all lines from the old iterate);
 * zebra = 1 -> lines of one parity of the orthogonal index sum at a time */
static void sweep_line(const lev_t *v, double *u, const double *g, double omega, int dir, int zebra, int first,
                       double *r) {
  int kz0 = (v->dim == 3) ? 1 : 0, kz1 = (v->dim == 3) ? v->n[2] - 2 : 0;
  int ncol = zebra ? 2 : 1;
  for (int pass = 0; pass < ncol; ++pass) {
    int colour = zebra ? ((first + pass) & 1) : -1;
    lev_defect(v, u, g, r);
    update_lines(v, u, r, omega, dir, colour, kz0, kz1);
  }
}

/* `sweeps` smoothing steps; order OR_RED_FIRST: red (even) colour / even lines
 * first, OR_BLACK_FIRST: the reverse.  Jacobi-type smoothers have no order. */
static void lev_smooth(or_hier *H, lev_t *v, double *u, const double *g, int sweeps, int order) {
  for (int s = 0; s < sweeps; ++s) {
    int first = (order == OR_RED_FIRST) ? 0 : 1;
    switch (H->smoother) {
      case OR_JACOBI: sweep_jacobi(v, u, g, H->omega, v->r); break;
      case OR_RBGS:
        if (v->st9) {
          /* red = colours (0,0), (1,1), black = (1,0), (0,1); the black-first order is the exact
           * reverse of the red-first one, so the transposed cycle stays the adjoint */
          static const int seq[4][2] = {{0, 0}, {1, 1}, {1, 0}, {0, 1}};
          for (int q = 0; q < 4; ++q) {
            const int *c = seq[first ? 3 - q : q];
            quartersweep(v, u, g, H->omega, c[0], c[1]);
          }
          break;
        }
        halfsweep_rb(v, u, g, H->omega, first);
        halfsweep_rb(v, u, g, H->omega, 1 - first);
        break;
      case OR_LINE_X: sweep_line(v, u, g, H->omega, 0, 0, first, v->r); break;
      case OR_LINE_Y: sweep_line(v, u, g, H->omega, 1, 0, first, v->r); break;
      case OR_ZEBRA_X: sweep_line(v, u, g, H->omega, 0, 1, first, v->r); break;
      case OR_ZEBRA_Y: sweep_line(v, u, g, H->omega, 1, 1, first, v->r); break;
      /* ADI / GSADI (sections "The choice of C" and "Coordinate systems": TRIx then TRIy, GSTRIx
       * then GSTRIy): the x-line sweep then the y-line sweep.  The transposed cycle (BLACK_FIRST)
       * runs the composition in reverse order, each zebra part with its colours reversed. */
      case OR_ADI:
        sweep_line(v, u, g, H->omega, first ? 1 : 0, 0, first, v->r);
        sweep_line(v, u, g, H->omega, first ? 0 : 1, 0, first, v->r);
        break;
      case OR_GSADI:
        sweep_line(v, u, g, H->omega, first ? 1 : 0, 1, first, v->r);
        sweep_line(v, u, g, H->omega, first ? 0 : 1, 1, first, v->r);
        break;
    }
    v->nsmooth++;
  }
}

/* ------------------------------------------------------------------------- */
/* grid transfers                                                            */
/* ------------------------------------------------------------------------- */

/* 1-D full-weighting stencil [1/4 1/2 1/4] */
static double w1(int a) { return a == 0 ? 0.5 : 0.25; }

/* full weighting R: g_c(I) = sum_{a in {-1,0,1}^d} prod w1(a) r_f(2I + a) */
static void lev_restrict(const lev_t *f, const lev_t *c, const double *rf, double *gc) {
  OR_PAR_ROWS
  FOR_NODES(c) {
    size_t P = nid(c, i, j, k);
    gc[P] = 0.0;
    if (!is_unk(c, i, j, k)) continue;
    double s = 0.0;
    int c0 = (f->dim == 3) ? -1 : 0, c1 = (f->dim == 3) ? 1 : 0;
    for (int cz = c0; cz <= c1; ++cz)
      for (int b = -1; b <= 1; ++b)
        for (int a = -1; a <= 1; ++a) {
          double wt = w1(a) * w1(b) * (f->dim == 3 ? w1(cz) : 1.0);
          s += wt * val(f, rf, 2 * i + a, 2 * j + b, 2 * k + cz);
        }
    gc[P] = s;
  }
}

/* bilinear / trilinear interpolation P = 2^d R^T, added with weight w:
 * u_f(i) += w * sum over coarse nodes I with |2I - i| <= 1 of prod 2 w1(2I - i) e_c(I) */
static void lev_prolong_add(const lev_t *f, const lev_t *c, const double *ec, double *uf, double w) {
  OR_PAR_ROWS
  FOR_NODES(f) {
    if (!is_unk(f, i, j, k)) continue;
    double s = 0.0;
    int c0 = (f->dim == 3) ? -1 : 0, c1 = (f->dim == 3) ? 1 : 0;
    for (int cz = c0; cz <= c1; ++cz) {
      int kk = k + cz;
      if (f->dim == 3 && (kk & 1)) continue;
      for (int b = -1; b <= 1; ++b) {
        int jj = ywrap(f, j + b);
        if (jj & 1) continue;
        for (int a = -1; a <= 1; ++a) {
          int ii = i + a;
          if (ii & 1) continue;
          double wt = 2.0 * w1(a) * 2.0 * w1(b) * (f->dim == 3 ? 2.0 * w1(cz) : 1.0);
          s += wt * val(c, ec, ii / 2, jj / 2, f->dim == 3 ? kk / 2 : 0);
        }
      }
    }
    uf[nid(f, i, j, k)] += w * s;
  }
}

/* ------------------------------------------------------------------------- */
/* coarse operators by rediscretisation                                      */
/* ------------------------------------------------------------------------- */

static double harm(double a, double b) { return 2.0 * a * b / (a + b); }
/* the same, 0 for an edge that does not exist on the finer grid (both weights 0) */
static double harm0(double a, double b) { return a + b > 0.0 ? 2.0 * a * b / (a + b) : 0.0; }

static int coarsen(const lev_t *f, lev_t *c) {
  memset(c, 0, sizeof(*c));
  c->dim = f->dim;
  c->per = f->per;
  c->kind = f->kind;
  for (int d = 0; d < 3; ++d) c->h[d] = 2.0 * f->h[d];
  /* x (and z) Dirichlet: n = 2m + 1 -> m + 1 ; periodic y: n = 2m -> m */
  if ((f->n[0] - 1) % 2 || f->n[0] < 5) return OR_EINVAL;
  c->n[0] = (f->n[0] - 1) / 2 + 1;
  if (f->per) {
    if (f->n[1] % 2 || f->n[1] < 4) return OR_EINVAL;
    c->n[1] = f->n[1] / 2;
  } else {
    if ((f->n[1] - 1) % 2 || f->n[1] < 5) return OR_EINVAL;
    c->n[1] = (f->n[1] - 1) / 2 + 1;
  }
  if (f->dim == 3) {
    if ((f->n[2] - 1) % 2 || f->n[2] < 5) return OR_EINVAL;
    c->n[2] = (f->n[2] - 1) / 2 + 1;
  } else {
    c->n[2] = 1;
  }
  if (f->kind == OR_CONST) {
    for (int d = 0; d < 3; ++d) c->c[d] = 0.25 * f->c[d];
  } else if (f->kind == OR_SEPARABLE) {
    int n0 = c->n[0];
    c->sx = (double *)calloc((size_t)n0, sizeof(double));
    c->sy = (double *)calloc((size_t)n0, sizeof(double));
    c->sz = (double *)calloc((size_t)n0, sizeof(double));
    if (!c->sx || !c->sy || !c->sz) return OR_ENOMEM;
    for (int I = 0; I < n0 - 1; ++I) c->sx[I] = 0.25 * harm(f->sx[2 * I], f->sx[2 * I + 1]);
    for (int I = 0; I < n0; ++I) {
      c->sy[I] = 0.25 * f->sy[2 * I];
      c->sz[I] = 0.25 * f->sz[2 * I];
    }
  } else if (f->kind == OR_EDGE) {
    /* the same rule edge by edge: a coarse edge spans two fine edges in series (harmonic mean),
     * and takes the fine line through its end nodes (injection across), times 1/4 */
    size_t N = nodes(c);
    c->ex = (double *)calloc(N, sizeof(double));
    c->ey = (double *)calloc(N, sizeof(double));
    c->ez = (double *)calloc(N, sizeof(double));
    if (!c->ex || !c->ey || !c->ez) return OR_ENOMEM;
    FOR_NODES(c) {
      size_t P = nid(c, i, j, k);
      int kk = (c->dim == 3) ? 2 * k : 0;
      if (i < c->n[0] - 1)
        c->ex[P] = 0.25 * harm0(f->ex[nid(f, 2 * i, 2 * j, kk)], f->ex[nid(f, 2 * i + 1, 2 * j, kk)]);
      if (c->per || j < c->n[1] - 1)
        c->ey[P] = 0.25 * harm0(f->ey[nid(f, 2 * i, 2 * j, kk)], f->ey[nid(f, 2 * i, 2 * j + 1, kk)]);
      if (c->dim == 3 && k < c->n[2] - 1)
        c->ez[P] = 0.25 * harm0(f->ez[nid(f, 2 * i, 2 * j, kk)], f->ez[nid(f, 2 * i, 2 * j, kk + 1)]);
    }
  } else {
    int cx = c->n[0] - 1, cy = ncells_y(c), cz = (c->dim == 3) ? c->n[2] - 1 : 1;
    c->k = (double *)calloc((size_t)cx * cy * cz, sizeof(double));
    if (!c->k) return OR_ENOMEM;
    for (int K = 0; K < cz; ++K)
      for (int J = 0; J < cy; ++J)
        for (int I = 0; I < cx; ++I) {
          double s = 0.0;
          int nz = (c->dim == 3) ? 2 : 1;
          for (int z = 0; z < nz; ++z)
            for (int b = 0; b < 2; ++b)
              for (int a = 0; a < 2; ++a) s += kcell(f, 2 * I + a, 2 * J + b, (c->dim == 3) ? 2 * K + z : 0);
          c->k[((size_t)K * cy + J) * cx + I] = s / (nz * 4.0);
        }
  }
  return OR_OK;
}

/* A(p, p + (a, b)) of level v at unknown p = (i, j), 0 when p + (a, b) is not an unknown */
static double a_entry(const lev_t *v, int i, int j, int a, int b) {
  if (!is_unk(v, i + a, j + b, 0)) return 0.0;
  if (v->st9) return v->st9[9 * nid(v, i, j, 0) + 3 * (b + 1) + (a + 1)];
  if (a == 0 && b == 0) return diag_at(v, i, j, 0);
  if (b == 0) return -(a > 0 ? wx_edge(v, i, j, 0) : wx_edge(v, i - 1, j, 0));
  if (a == 0) return -(b > 0 ? wy_edge(v, i, j, 0) : wy_edge(v, i, j - 1, 0));
  return 0.0;
}

/* Galerkin coarse operator A_c = R A P (2-D, y not periodic), R full weighting and P = 4 R^T
 * bilinear interpolation over the unknowns: for every coarse unknown P and offset (al, be),
 *   A_c(P, P + (al, be)) = sum_p R(P, p) sum_q A(p, q) P(q, P + (al, be)),
 * p over the fine unknowns with |p - 2P| <= 1 (weights w1 x w1), q over the fine stencil of p,
 * and P(q, Q) = (2 w1(q_x - 2 Q_x)) (2 w1(q_y - 2 Q_y)) when |q - 2Q| <= 1 in both directions
 * (0 otherwise, and 0 when Q is not an unknown).  The coarse stencil reaches one coarse node
 * in each direction: 9 points. */
static int galerkin_coarse(const lev_t *f, lev_t *c) {
  c->st9 = (double *)calloc(9 * nodes(c), sizeof(double));
  if (!c->st9) return OR_ENOMEM;
  for (int J = 1; J < c->n[1] - 1; ++J)
    for (int I = 1; I < c->n[0] - 1; ++I) {
      double *out = c->st9 + 9 * nid(c, I, J, 0);
      for (int be = -1; be <= 1; ++be)
        for (int al = -1; al <= 1; ++al) {
          const int QI = I + al, QJ = J + be;
          if (!is_unk(c, QI, QJ, 0)) continue;
          double s = 0.0;
          for (int pb = -1; pb <= 1; ++pb)
            for (int pa = -1; pa <= 1; ++pa) {
              const int pi = 2 * I + pa, pj = 2 * J + pb;
              if (!is_unk(f, pi, pj, 0)) continue;
              double t = 0.0;
              for (int qb = -1; qb <= 1; ++qb)
                for (int qa = -1; qa <= 1; ++qa) {
                  const int qi = pi + qa, qj = pj + qb;
                  const int dx = qi - 2 * QI, dy = qj - 2 * QJ;
                  if (dx < -1 || dx > 1 || dy < -1 || dy > 1) continue;
                  t += a_entry(f, pi, pj, qa, qb) * (2.0 * w1(dx)) * (2.0 * w1(dy));
                }
              s += w1(pa) * w1(pb) * t;
            }
          out[3 * (be + 1) + (al + 1)] = s;
        }
    }
  return OR_OK;
}

/* ------------------------------------------------------------------------- */
/* coarsest grid: u = A_1^{-1} g                                             */
/* ------------------------------------------------------------------------- */

static int setup_coarse(or_hier *H) {
  lev_t *v = &H->lev[1];
  int nc = 0;
  FOR_NODES(v) if (is_unk(v, i, j, k)) nc++;
  H->nc = nc;
  H->cidx = (size_t *)malloc(sizeof(size_t) * (size_t)(nc > 0 ? nc : 1));
  if (!H->cidx) return OR_ENOMEM;
  int t = 0;
  FOR_NODES(v) if (is_unk(v, i, j, k)) H->cidx[t++] = nid(v, i, j, k);
  H->chol = NULL;
  if (H->coarse_mode != OR_COARSE_EXACT || nc > H->dense_max) return OR_OK;
  /* assemble the dense matrix column by column: column c = A e_c */
  double *A = (double *)calloc((size_t)nc * nc, sizeof(double));
  double *e = (double *)calloc(nodes(v), sizeof(double)), *Ae = (double *)calloc(nodes(v), sizeof(double));
  if (!A || !e || !Ae) return OR_ENOMEM;
  for (int c = 0; c < nc; ++c) {
    e[H->cidx[c]] = 1.0;
    lev_apply(v, e, Ae);
    for (int r = 0; r < nc; ++r) A[(size_t)r * nc + c] = Ae[H->cidx[r]];
    e[H->cidx[c]] = 0.0;
  }
  /* Cholesky A = L L^T, L stored in the lower triangle */
  for (int j = 0; j < nc; ++j) {
    double s = A[(size_t)j * nc + j];
    for (int q = 0; q < j; ++q) s -= A[(size_t)j * nc + q] * A[(size_t)j * nc + q];
    if (!(s > 0.0)) { free(A); free(e); free(Ae); return OR_EINVAL; }
    double ljj = sqrt(s);
    A[(size_t)j * nc + j] = ljj;
    for (int i = j + 1; i < nc; ++i) {
      double t2 = A[(size_t)i * nc + j];
      for (int q = 0; q < j; ++q) t2 -= A[(size_t)i * nc + q] * A[(size_t)j * nc + q];
      A[(size_t)i * nc + j] = t2 / ljj;
    }
  }
  H->chol = A;
  free(e);
  free(Ae);
  return OR_OK;
}

static void coarse_cg(or_hier *H, const double *g, double *u) {
  lev_t *v = &H->lev[1];
  size_t N = nodes(v);
  double *r = (double *)calloc(N, sizeof(double)), *p = (double *)calloc(N, sizeof(double));
  double *Ap = (double *)calloc(N, sizeof(double));
  memset(u, 0, N * sizeof(double));
  FOR_NODES(v) if (is_unk(v, i, j, k)) { size_t q = nid(v, i, j, k); r[q] = g[q]; p[q] = g[q]; }
  double rr = 0.0;
  for (size_t q = 0; q < N; ++q) rr += r[q] * r[q];
  double stop = 1e-28 * rr;
  for (int it = 0; it < 20 * H->nc + 100 && rr > stop && rr > 0.0; ++it) {
    lev_apply(v, p, Ap);
    double pAp = 0.0;
    for (size_t q = 0; q < N; ++q) pAp += p[q] * Ap[q];
    double alpha = rr / pAp, rr2 = 0.0;
    for (size_t q = 0; q < N; ++q) { u[q] += alpha * p[q]; r[q] -= alpha * Ap[q]; rr2 += r[q] * r[q]; }
    double beta = rr2 / rr;
    for (size_t q = 0; q < N; ++q) p[q] = r[q] + beta * p[q];
    rr = rr2;
  }
  free(r); free(p); free(Ap);
}

void or_coarse_solve(or_hier *H, const double *g, double *u) {
  lev_t *v = &H->lev[1];
  H->ncoarse++;
  if (H->coarse_mode == OR_COARSE_SMOOTH) {
    lev_smooth(H, v, u, g, H->coarse_sweeps, OR_RED_FIRST);
    return;
  }
  memset(u, 0, nodes(v) * sizeof(double));
  if (H->nc == 0) return;
  if (!H->chol) { coarse_cg(H, g, u); return; }
  int nc = H->nc;
  const double *L = H->chol;
  double *y = (double *)malloc(sizeof(double) * (size_t)nc);
  for (int i = 0; i < nc; ++i) { /* L y = g */
    double s = g[H->cidx[i]];
    for (int q = 0; q < i; ++q) s -= L[(size_t)i * nc + q] * y[q];
    y[i] = s / L[(size_t)i * nc + i];
  }
  for (int i = nc - 1; i >= 0; --i) { /* L^T x = y */
    double s = y[i];
    for (int q = i + 1; q < nc; ++q) s -= L[(size_t)q * nc + i] * y[q];
    y[i] = s / L[(size_t)i * nc + i];
  }
  for (int i = 0; i < nc; ++i) u[H->cidx[i]] = y[i];
  free(y);
}

/* ------------------------------------------------------------------------- */
/* the cycle                                                                 */
/* ------------------------------------------------------------------------- */

/* Adaptive weight of the coarse-grid correction (section "Multigrid", the omega_l chosen to
 * minimise the error in the energy norm).  With u* = A^-1 g, the corrected iterate
 * u + w P e has energy error ||u* - u - w P e||_A^2, a quadratic in w whose minimum is at
 * w = (A (u* - u), P e) / (A P e, P e) = (d, P e) / (A P e, P e) with d = g - A u, the
 * defect of the iterate before the correction.  Reading: the printed formula writes the
 * restriction symbol and mixes the iterate superscripts; the operator applied to the coarse
 * correction can only be the interpolation P (it maps level l-1 to level l), so that is the
 * formula taken.  Inner products run over the unknowns of level l. */
double or_adaptive_omega(const or_hier *H, int l, const double *u, const double *g, const double *e) {
  const lev_t *v = &H->lev[l], *c = &H->lev[l - 1];
  size_t n = nodes(v);
  double *pe = (double *)calloc(n, sizeof(double));
  double *ape = (double *)calloc(n, sizeof(double));
  double *d = (double *)calloc(n, sizeof(double));
  lev_prolong_add(v, c, e, pe, 1.0);   /* P e (zero on the Dirichlet nodes) */
  lev_apply(v, pe, ape);               /* A P e */
  lev_defect(v, u, g, d);              /* d = g - A u */
  double num = 0.0, den = 0.0;
  FOR_NODES(v) if (is_unk(v, i, j, k)) {
    size_t p = nid(v, i, j, k);
    num += d[p] * pe[p];
    den += ape[p] * pe[p];
  }
  free(pe);
  free(ape);
  free(d);
  return den > 0.0 ? num / den : 1.0;
}

/* MG(l, u, g) with the F-cycle recursion: the coarse problem is solved by an
 * F-cycle started from zero followed by a V-cycle (skipped when the coarse grid
 * is the coarsest, whose direct solve is already exact); a V-cycle recurses
 * once.  Both smoothing phases sweep red (even lines) first.
 * transposed = 1 runs the steps in reverse order with each replaced by its
 * transpose: pre- and post-smoothing exchange roles (nu2 sweeps before, nu1
 * after), every sweep runs its colours in reverse (black first), and the coarse
 * "F then V" becomes "V^T then F^T"; one such cycle is the adjoint iteration
 * lambda + M^T (g - A lambda). */
void or_cycle(or_hier *H, int l, double *u, const double *g, int type, int transposed) {
  lev_t *v = &H->lev[l];
  if (l == 1) { or_coarse_solve(H, g, u); return; }
  lev_t *c = &H->lev[l - 1];
  int npre = transposed ? H->nu2 : H->nu1, npost = transposed ? H->nu1 : H->nu2;
  int order = transposed ? OR_BLACK_FIRST : OR_RED_FIRST;
  lev_smooth(H, v, u, g, npre, order);
  lev_defect(v, u, g, v->r);                 /* d_l = g_l - A_l u_l */
  lev_restrict(v, c, v->r, c->g);            /* g_{l-1} = R d_l */
  memset(c->u, 0, nodes(c) * sizeof(double)); /* u_{l-1}^0 = 0 */
  if (type == OR_CYCLE_F) {
    int first = transposed ? OR_CYCLE_V : OR_CYCLE_F, second = transposed ? OR_CYCLE_F : OR_CYCLE_V;
    or_cycle(H, l - 1, c->u, c->g, first, transposed);
    if (l - 1 > 1) or_cycle(H, l - 1, c->u, c->g, second, transposed);
  } else {
    or_cycle(H, l - 1, c->u, c->g, OR_CYCLE_V, transposed);
  }
  double w = H->adaptive_corr ? or_adaptive_omega(H, l, u, g, c->u) : H->omega_corr;
  lev_prolong_add(v, c, c->u, u, w);          /* u + omega_l P u_{l-1} */
  lev_smooth(H, v, u, g, npost, order);
}

/* Nested-iteration start vector (section "Start-Vector Choice": begin the solution on the
 * coarsest level and work up to the finest).  Reading: the right-hand side is restricted to
 * every level by full weighting (its Dirichlet entries taken as 0), the coarsest level is
 * solved exactly, and on each finer level the bilinear / trilinear interpolation of the
 * coarser solution is improved by ncyc F-cycles.  x receives the finest-level result. */
void or_fmg_start(or_hier *H, const double *b, double *x, int ncyc) {
  int L = H->L;
  double **bl = (double **)calloc((size_t)L + 1, sizeof(double *));
  lev_t *vL = &H->lev[L];
  bl[L] = (double *)calloc(nodes(vL), sizeof(double));
  FOR_NODES(vL) if (is_unk(vL, i, j, k)) bl[L][nid(vL, i, j, k)] = b[nid(vL, i, j, k)];
  for (int l = L; l > 1; --l) {
    bl[l - 1] = (double *)calloc(nodes(&H->lev[l - 1]), sizeof(double));
    lev_restrict(&H->lev[l], &H->lev[l - 1], bl[l], bl[l - 1]);
  }
  double *xc = (double *)calloc(nodes(&H->lev[1]), sizeof(double));
  or_coarse_solve(H, bl[1], xc);
  for (int l = 2; l <= L; ++l) {
    double *xf = (double *)calloc(nodes(&H->lev[l]), sizeof(double));
    lev_prolong_add(&H->lev[l], &H->lev[l - 1], xc, xf, 1.0);
    for (int q = 0; q < ncyc; ++q) or_cycle(H, l, xf, bl[l], OR_CYCLE_F, 0);
    free(xc);
    xc = xf;
  }
  memcpy(x, xc, nodes(vL) * sizeof(double));
  free(xc);
  for (int l = 1; l <= L; ++l) free(bl[l]);
  free(bl);
}

int or_solve(or_hier *H, const double *b, double *x, double tol, int maxit, int transposed, double *hist,
             int hist_cap, int *cycles, double *relres) {
  lev_t *v = &H->lev[H->L];
  FOR_NODES(v) if (!is_unk(v, i, j, k)) x[nid(v, i, j, k)] = 0.0;
  double nb = lev_norm2(v, b);
  *cycles = 0;
  if (nb == 0.0) {
    memset(x, 0, nodes(v) * sizeof(double));
    *relres = 0.0;
    if (hist && hist_cap > 0) hist[0] = 0.0;
    return OR_OK;
  }
  for (int it = 0;; ++it) {
    lev_defect(v, x, b, v->r);
    double rr = lev_norm2(v, v->r) / nb;
    if (hist && it < hist_cap) hist[it] = rr;
    *relres = rr;
    *cycles = it;
    if (!isfinite(rr)) return OR_EDIVERGED;
    if (rr <= tol) return OR_OK;
    if (it >= maxit) return OR_ENOCONV;
    or_cycle(H, H->L, x, b, OR_CYCLE_F, transposed);
  }
}

/* ------------------------------------------------------------------------- */
/* gradient of a loss through A(k) u = f with respect to the cell field k      */
/* dL/dk_c = -lambda^T (dA/dk_c) u = -sum over edges e touching cell c of      */
/*           (dw_e/dk_c) (u_p - u_q)(lambda_p - lambda_q)                      */
/* ------------------------------------------------------------------------- */

static double edge_term(const lev_t *v, const double *u, const double *l, int i0, int j0, int k0, int i1, int j1,
                        int k1) {
  double du = val(v, u, i0, j0, k0) - val(v, u, i1, j1, k1);
  double dl = val(v, l, i0, j0, k0) - val(v, l, i1, j1, k1);
  return du * dl;
}

void or_grad_k(const or_hier *H, const double *u, const double *lam, double *dk) {
  const lev_t *v = &H->lev[H->L];
  int cx = v->n[0] - 1, cy = ncells_y(v), cz = (v->dim == 3) ? v->n[2] - 1 : 1;
  for (int k = 0; k < cz; ++k)
    for (int j = 0; j < cy; ++j)
      for (int i = 0; i < cx; ++i) {
        double s = 0.0;
        if (v->dim == 2) {
          double ax = 1.0 / (2.0 * v->h[0] * v->h[0]), ay = 1.0 / (2.0 * v->h[1] * v->h[1]);
          s += ax * edge_term(v, u, lam, i, j, 0, i + 1, j, 0);         /* bottom x-edge */
          s += ax * edge_term(v, u, lam, i, j + 1, 0, i + 1, j + 1, 0); /* top x-edge */
          s += ay * edge_term(v, u, lam, i, j, 0, i, j + 1, 0);         /* left y-edge */
          s += ay * edge_term(v, u, lam, i + 1, j, 0, i + 1, j + 1, 0); /* right y-edge */
        } else {
          double ax = 1.0 / (4.0 * v->h[0] * v->h[0]), ay = 1.0 / (4.0 * v->h[1] * v->h[1]);
          double az = 1.0 / (4.0 * v->h[2] * v->h[2]);
          for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
              s += ax * edge_term(v, u, lam, i, j + a, k + b, i + 1, j + a, k + b);
              s += ay * edge_term(v, u, lam, i + a, j, k + b, i + a, j + 1, k + b);
              s += az * edge_term(v, u, lam, i + a, j + b, k, i + a, j + b, k + 1);
            }
        }
        dk[((size_t)k * cy + j) * cx + i] = -s;
      }
}

/* ------------------------------------------------------------------------- */
/* construction and small accessors                                          */
/* ------------------------------------------------------------------------- */

static void free_level(lev_t *v) {
  free(v->sx); free(v->sy); free(v->sz); free(v->k);
  free(v->ex); free(v->ey); free(v->ez); free(v->st9);
  free(v->u); free(v->g); free(v->r);
  memset(v, 0, sizeof(*v));
}

void or_destroy(or_hier *H) {
  if (!H) return;
  for (int l = 1; l <= H->L; ++l) free_level(&H->lev[l]);
  free(H->cidx);
  free(H->chol);
  free(H);
}

int or_create(const or_config *cfg, or_hier **out) {
  *out = NULL;
  if (cfg->dim != 2 && cfg->dim != 3) return OR_EINVAL;
  if (cfg->levels < 1 || cfg->levels > OR_MAXLEV) return OR_EINVAL;
  if (cfg->smoother < OR_JACOBI || cfg->smoother > OR_GSADI) return OR_EINVAL;
  if (cfg->periodic_y && cfg->n[1] < 4 && (cfg->smoother == OR_LINE_Y || cfg->smoother == OR_ZEBRA_Y ||
                                            cfg->smoother == OR_ADI || cfg->smoother == OR_GSADI))
    return OR_EINVAL;   /* cyclic line systems need >= 3 rows on every level */
  if (cfg->n[0] < 3 || cfg->n[1] < (cfg->periodic_y ? 2 : 3) || (cfg->dim == 3 && cfg->n[2] < 3)) return OR_EINVAL;
  if (cfg->periodic_y && (cfg->n[1] % 2)) return OR_EINVAL;
  or_hier *H = (or_hier *)calloc(1, sizeof(or_hier));
  if (!H) return OR_ENOMEM;
  H->L = cfg->levels;
  H->smoother = cfg->smoother;
  H->omega = cfg->omega;
  H->nu1 = cfg->nu1;
  H->nu2 = cfg->nu2;
  H->omega_corr = cfg->omega_corr;
  H->adaptive_corr = cfg->adaptive_corr ? 1 : 0;
  H->galerkin = cfg->galerkin ? 1 : 0;
  /* Galerkin coarse operators: 2-D, y not periodic, point smoothers (the 9-point stencils have
   * no tridiagonal line part in the paper's sense) */
  if (H->galerkin && (cfg->dim != 2 || cfg->periodic_y || (cfg->smoother != OR_JACOBI && cfg->smoother != OR_RBGS))) {
    or_destroy(H);
    return OR_EINVAL;
  }
  H->coarse_mode = cfg->coarse_mode;
  H->coarse_sweeps = cfg->coarse_sweeps;
  H->dense_max = cfg->dense_max > 0 ? cfg->dense_max : 1024;
  lev_t *f = &H->lev[H->L];
  f->dim = cfg->dim;
  f->per = cfg->periodic_y ? 1 : 0;
  f->kind = cfg->kind;
  f->n[0] = cfg->n[0];
  f->n[1] = cfg->n[1];
  f->n[2] = (cfg->dim == 3) ? cfg->n[2] : 1;
  for (int d = 0; d < 3; ++d) { f->h[d] = cfg->h[d]; f->c[d] = cfg->c[d]; }
  int n0 = f->n[0];
  if (cfg->kind == OR_SEPARABLE) {
    f->sx = (double *)calloc((size_t)n0, sizeof(double));
    f->sy = (double *)calloc((size_t)n0, sizeof(double));
    f->sz = (double *)calloc((size_t)n0, sizeof(double));
    if (!f->sx || !f->sy || !f->sz) { or_destroy(H); return OR_ENOMEM; }
    memcpy(f->sx, cfg->sx, sizeof(double) * (size_t)(n0 - 1));
    memcpy(f->sy, cfg->sy, sizeof(double) * (size_t)n0);
    if (cfg->dim == 3) memcpy(f->sz, cfg->sz, sizeof(double) * (size_t)n0);
  } else if (cfg->kind == OR_CELL) {
    size_t nk = (size_t)(n0 - 1) * ncells_y(f) * (cfg->dim == 3 ? f->n[2] - 1 : 1);
    f->k = (double *)malloc(sizeof(double) * nk);
    if (!f->k) { or_destroy(H); return OR_ENOMEM; }
    memcpy(f->k, cfg->k, sizeof(double) * nk);
  } else if (cfg->kind == OR_EDGE) {
    size_t N = nodes(f);
    if (!cfg->ex || !cfg->ey || (cfg->dim == 3 && !cfg->ez)) { or_destroy(H); return OR_EINVAL; }
    f->ex = (double *)calloc(N, sizeof(double));
    f->ey = (double *)calloc(N, sizeof(double));
    f->ez = (double *)calloc(N, sizeof(double));
    if (!f->ex || !f->ey || !f->ez) { or_destroy(H); return OR_ENOMEM; }
    memcpy(f->ex, cfg->ex, sizeof(double) * N);
    memcpy(f->ey, cfg->ey, sizeof(double) * N);
    if (cfg->dim == 3) memcpy(f->ez, cfg->ez, sizeof(double) * N);
  } else if (cfg->kind != OR_CONST) {
    or_destroy(H);
    return OR_EINVAL;
  }
  for (int l = H->L - 1; l >= 1; --l) {
    int st = coarsen(&H->lev[l + 1], &H->lev[l]);
    if (!st && H->galerkin) st = galerkin_coarse(&H->lev[l + 1], &H->lev[l]);
    if (st) { or_destroy(H); return st; }
  }
  for (int l = 1; l <= H->L; ++l) {
    lev_t *v = &H->lev[l];
    size_t N = nodes(v);
    v->u = (double *)calloc(N, sizeof(double));
    v->g = (double *)calloc(N, sizeof(double));
    v->r = (double *)calloc(N, sizeof(double));
    if (!v->u || !v->g || !v->r) { or_destroy(H); return OR_ENOMEM; }
  }
  int st = setup_coarse(H);
  if (st) { or_destroy(H); return st; }
  *out = H;
  return OR_OK;
}

int or_levels(const or_hier *H) { return H->L; }
void or_level_dims(const or_hier *H, int l, int n[3]) {
  for (int d = 0; d < 3; ++d) n[d] = H->lev[l].n[d];
}
size_t or_level_nodes(const or_hier *H, int l) { return nodes(&H->lev[l]); }
int or_level_unknowns(const or_hier *H, int l) {
  const lev_t *v = &H->lev[l];
  int c = 0;
  FOR_NODES(v) if (is_unk(v, i, j, k)) c++;
  return c;
}
void or_level_coeffs(const or_hier *H, int l, double *out) {
  const lev_t *v = &H->lev[l];
  if (v->kind == OR_CONST) { for (int d = 0; d < 3; ++d) out[d] = v->c[d]; return; }
  if (v->kind == OR_EDGE) {   /* ex, ey, ez back to back */
    size_t N = nodes(v);
    memcpy(out, v->ex, sizeof(double) * N);
    memcpy(out + N, v->ey, sizeof(double) * N);
    memcpy(out + 2 * N, v->ez, sizeof(double) * N);
    return;
  }
  if (v->kind == OR_SEPARABLE) {
    int n0 = v->n[0];
    memcpy(out, v->sx, sizeof(double) * (size_t)n0);
    memcpy(out + n0, v->sy, sizeof(double) * (size_t)n0);
    memcpy(out + 2 * n0, v->sz, sizeof(double) * (size_t)n0);
    return;
  }
  size_t nk = (size_t)(v->n[0] - 1) * ncells_y(v) * (v->dim == 3 ? v->n[2] - 1 : 1);
  memcpy(out, v->k, sizeof(double) * nk);
}
void or_apply(const or_hier *H, int l, const double *u, double *Au) { lev_apply(&H->lev[l], u, Au); }
int or_level_stencil(const or_hier *H, int l, double *out) {
  const lev_t *v = &H->lev[l];
  if (!v->st9) return OR_EINVAL;
  memcpy(out, v->st9, sizeof(double) * 9 * nodes(v));
  return OR_OK;
}
int or_threads(void) {
#ifdef OR_THREADED
  return omp_get_max_threads();
#else
  return 1;
#endif
}
void or_diag(const or_hier *H, int l, double *D) {
  const lev_t *v = &H->lev[l];
  FOR_NODES(v) D[nid(v, i, j, k)] = is_unk(v, i, j, k) ? diag_at(v, i, j, k) : 0.0;
}
void or_defect(const or_hier *H, int l, const double *u, const double *g, double *r) {
  lev_defect(&H->lev[l], u, g, r);
}
double or_norm2(const or_hier *H, int l, const double *x) { return lev_norm2(&H->lev[l], x); }
void or_smooth(or_hier *H, int l, double *u, const double *g, int sweeps, int order) {
  lev_smooth(H, &H->lev[l], u, g, sweeps, order);
}
void or_restrict(const or_hier *H, int lf, const double *rf, double *gc) {
  lev_restrict(&H->lev[lf], &H->lev[lf - 1], rf, gc);
}
void or_prolong_add(const or_hier *H, int lf, const double *ec, double *uf, double w) {
  lev_prolong_add(&H->lev[lf], &H->lev[lf - 1], ec, uf, w);
}
void or_counts(const or_hier *H, long *smooth_sweeps, long *coarse_solves) {
  for (int l = 1; l <= H->L; ++l) smooth_sweeps[l - 1] = H->lev[l].nsmooth;
  *coarse_solves = H->ncoarse;
}
void or_reset_counts(or_hier *H) {
  for (int l = 1; l <= H->L; ++l) H->lev[l].nsmooth = 0;
  H->ncoarse = 0;
}
