/*
 * mg_oracle.h -- plain FP64 CPU reference implementation ("the oracle") of the
 * multigrid F-cycle with preconditioned-Richardson smoothers studied in
 * J. T. Wallis, "Methods toward better Multigrid Solver Convergence" (2008).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the solver library may include, link or
 * call this code; only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code with the CUDA path.
 *
 * Conventions (all levels):
 *   - vertex-centred grid, node (i,j,k) stored at ((k*n1 + j)*n0 + i), x fastest;
 *   - Dirichlet nodes (i = 0, n0-1; j = 0, n1-1 unless y is periodic; k = 0,
 *     n2-1 in 3D) are not unknowns and read as 0;
 *   - y may be periodic (the theta direction of a mapped annulus/cylinder);
 *   - the operator is edge based: (A u)_p = sum_{edges e=(p,q)} w_e (u_p - u_q);
 *   - level 1 is the coarsest grid and level L the finest (paper, section
 *     "The Multigrid Technique", algorithm MG(l, u, g)).
 */
#ifndef MG_ORACLE_H
#define MG_ORACLE_H
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_CONST = 0, OR_SEPARABLE = 1, OR_CELL = 2, OR_EDGE = 3 };
enum { OR_JACOBI = 0, OR_RBGS = 1, OR_LINE_X = 2, OR_LINE_Y = 3, OR_ZEBRA_X = 4, OR_ZEBRA_Y = 5,
       OR_ADI = 6,     /* alternating directions: x-line Jacobi sweep, then y-line Jacobi sweep */
       OR_GSADI = 7 }; /* zebra x-line Gauss-Seidel, then zebra y-line Gauss-Seidel */
enum { OR_RED_FIRST = 0, OR_BLACK_FIRST = 1 };
enum { OR_CYCLE_F = 0, OR_CYCLE_V = 1 };
enum { OR_COARSE_EXACT = 0, OR_COARSE_SMOOTH = 1 };
enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2, OR_ENOCONV = 4, OR_EDIVERGED = 5 };

#define OR_MAXLEV 16

typedef struct {
  int dim;            /* 2 or 3 */
  int n[3];           /* nodes per direction on the finest grid (n[2] ignored in 2D) */
  int periodic_y;     /* 1: y direction periodic with n[1] distinct nodes */
  int kind;           /* OR_CONST / OR_SEPARABLE / OR_CELL / OR_EDGE */
  double h[3];        /* mesh widths (used by OR_CELL) */
  double c[3];        /* OR_CONST: edge weight per direction */
  const double *sx;   /* OR_SEPARABLE: sx[i] = weight of x-edge (i, i+1), length n0-1 */
  const double *sy;   /* OR_SEPARABLE: sy[i] = weight of every y-edge at x-index i, length n0 */
  const double *sz;   /* OR_SEPARABLE: sz[i] = weight of every z-edge at x-index i, length n0 */
  const double *k;    /* OR_CELL: per-cell coefficient, (n0-1) x ncy [x (n2-1)], x fastest;
                         ncy = n1 if periodic_y else n1-1 */
  int levels;         /* number of grids L (>= 1) */
  int smoother;       /* OR_JACOBI ... OR_GSADI */
  double omega;       /* smoother damping / relaxation parameter */
  int nu1, nu2;       /* pre- and post-smoothing steps */
  double omega_corr;  /* omega_l of the coarse-grid correction */
  int coarse_mode;    /* OR_COARSE_EXACT (direct / CG) or OR_COARSE_SMOOTH */
  int coarse_sweeps;  /* sweeps used by OR_COARSE_SMOOTH */
  int dense_max;      /* largest coarsest-grid unknown count solved by dense Cholesky */
  int adaptive_corr;  /* 1: omega_l of every correction chosen to minimise the energy norm of
                         the error (or_adaptive_omega); omega_corr is then ignored */
  const double *ex;   /* OR_EDGE: full node arrays, x fastest: ex[p] = weight of the edge from node */
  const double *ey;   /* p to its +x neighbour, ey[p] to +y (periodic: the last row's edge wraps to */
  const double *ez;   /* row 0), ez[p] to +z (3-D); entries with no such edge are ignored */
  int galerkin;       /* 1: every coarse operator is the Galerkin product R A P of the next finer
                         one (a 9-point stencil; 2-D, y not periodic, Jacobi or Gauss-Seidel, the
                         latter in four colours (i mod 2, j mod 2) on those levels) */
} or_config;

typedef struct or_hier or_hier;

int    or_create(const or_config *cfg, or_hier **out);
void   or_destroy(or_hier *H);
int    or_levels(const or_hier *H);
void   or_level_dims(const or_hier *H, int l, int n[3]);
size_t or_level_nodes(const or_hier *H, int l);
int    or_level_unknowns(const or_hier *H, int l);
/* coefficient data of level l: CONST -> c[3]; SEPARABLE -> sx,sy,sz; CELL -> k, h */
void   or_level_coeffs(const or_hier *H, int l, double *out);

void or_apply(const or_hier *H, int l, const double *u, double *Au);
void or_diag(const or_hier *H, int l, double *D);
void or_defect(const or_hier *H, int l, const double *u, const double *g, double *r);
double or_norm2(const or_hier *H, int l, const double *v);
void or_smooth(or_hier *H, int l, double *u, const double *g, int sweeps, int order);
void or_restrict(const or_hier *H, int lf, const double *rf, double *gc);
void or_prolong_add(const or_hier *H, int lf, const double *ec, double *uf, double w);
void or_coarse_solve(or_hier *H, const double *g, double *u);
void or_cycle(or_hier *H, int l, double *u, const double *g, int type, int transposed);
/* energy-optimal correction weight at level l >= 2 for iterate u, right-hand side g and
 * coarse correction e: (g - A u, P e) / (A P e, P e); 1 when P e = 0 */
double or_adaptive_omega(const or_hier *H, int l, const double *u, const double *g, const double *e);
/* nested-iteration start vector: coarsest level exact, then on each finer level the
 * interpolated coarser solution improved by ncyc F-cycles (section "Start-Vector Choice") */
void or_fmg_start(or_hier *H, const double *b, double *x, int ncyc);
int  or_solve(or_hier *H, const double *b, double *x, double tol, int maxit, int transposed,
              double *hist, int hist_cap, int *cycles, double *relres);
void or_grad_k(const or_hier *H, const double *u, const double *lam, double *dk);
void or_thomas(int m, const double *lo, const double *di, const double *up,
               const double *d, double *x);
/* cyclic tridiagonal solve (indices modulo m: lo[0] couples to x[m-1], up[m-1] to x[0]), m >= 3 */
void or_cyclic_thomas(int m, const double *lo, const double *di, const double *up,
                      const double *d, double *x);
void or_counts(const or_hier *H, long *smooth_sweeps, long *coarse_solves);
/* Galerkin levels: the 9-point stencil of every node, out[9 p + 3 (b + 1) + (a + 1)] =
 * A(p, p + (a, b)); OR_EINVAL on a level without one */
int  or_level_stencil(const or_hier *H, int l, double *out);
/* threads the grid loops run on: 1, or the OpenMP thread count of the threaded build */
int  or_threads(void);
void or_reset_counts(or_hier *H);

#ifdef __cplusplus
}
#endif
#endif
