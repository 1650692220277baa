/*
 * mg.h -- C ABI of the GB300 geometric multigrid solver.
 *
 * The solver computes the method of J. T. Wallis, "Methods toward better
 * Multigrid Solver Convergence" (2008): the F-cycle (abstract; section "The
 * Multigrid Technique", algorithm MG(l, u, g)) with preconditioned-Richardson
 * smoothers x <- x - omega C^{-1}(A x - b) (section "Smoothers", choices of C
 * in "The choice of C") for the Poisson-type problems of sections
 * "Introduction / Motivation" and "Anisotropies": 5-point (2-D) / 7-point
 * (3-D) operators with constant, separable (mapped polar / cylindrical),
 * per-cell (-div(k grad u)) or per-edge coefficients, zero Dirichlet data,
 * optionally periodic in y.
 *
 * Conventions
 *   - Every array argument is a DEVICE pointer to a full node array (Dirichlet
 *     nodes included), contiguous, x fastest: (n1, n0) in 2-D, (n2, n1, n0) in
 *     3-D.  Entries at Dirichlet nodes of right-hand sides are ignored; those of
 *     solutions are written as 0.  Cell arrays are (ncy, n0-1) / (n2-1, ncy, n0-1)
 *     with ncy = n1 if y is periodic else n1-1.
 *   - Level 1 is the coarsest grid and level L the finest, as in the paper.
 *   - Every call is stream-ordered on mg_params.stream (a cudaStream_t).  A
 *     solve (mg_solve, mg_solve_host, mg_solve_adjoint) is one CUDA graph
 *     launch: the convergence test runs on the device after every cycle and
 *     ends a device-side loop, and the host synchronises the stream once, when
 *     the solve is over (MG_FLAG_NO_GRAPH: launched kernel by kernel, and the
 *     host then reads the residual norm once per cycle).
 *   - Memory: the caller allocates the workspace (mg_workspace_bytes) and all
 *     argument arrays; the library allocates only the opaque context on the
 *     host and its CUDA graph.  The library never calls cudaMalloc.
 *   - Sizes: at most 2^34 nodes, and at most 131,072 unknowns along x and
 *     along y (the block partial sums of the reductions).
 *   - Errors: every call returns an mg_status; no exception crosses the ABI.
 *     MG_EINVAL is returned before any launch for bad arguments; CUDA failures
 *     give MG_ECUDA with the text in mg_last_error().
 */
#ifndef MG_H
#define MG_H
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_ctx mg_ctx;

typedef enum {
  MG_OK = 0,
  MG_EINVAL = 1,     /* bad argument (sizes, levels, null pointer, workspace too small) */
  MG_ENOMEM = 2,     /* host allocation of the context failed */
  MG_ECUDA = 3,      /* a CUDA call failed; see mg_last_error */
  MG_ENOCONV = 4,    /* max_cycles reached before the tolerance; x holds the last iterate */
  MG_EDIVERGED = 5,  /* the residual norm became non-finite */
  MG_ETIMEOUT = 6,   /* a bounded device wait gave up; the output is not the solution */
  MG_EBOUNDS = 7     /* the checking build (-DMG_DEBUG, see mg_debug_build): a device-side check
                        found an out-of-range node index; the access was skipped (no fault), the
                        site is in mg_last_error, and the result of the call is not valid */
} mg_status;

/* Choice of C in x <- x + omega C^{-1} (b - A x) (section "The choice of C"). */
typedef enum {
  MG_JACOBI = 0,   /* C = D, damped by omega                                              */
  MG_RBGS = 1,     /* Gauss-Seidel / SOR in red-black order (red: i+j+k even, first)       */
  MG_LINE_X = 2,   /* TRIx: C = tridiagonal part of A along x lines, all lines at once       */
  MG_LINE_Y = 3,   /* TRIy: the same along y lines (the paper's "virtually transposed" TRI) */
  MG_ZEBRA_X = 4,  /* GSTRIx: x lines in two colours by parity of (j + k), even first       */
  MG_ZEBRA_Y = 5,  /* GSTRIy: y lines in two colours by parity of (i + k), even first       */
  MG_ADI = 6,      /* ADI: a TRIx sweep then a TRIy sweep (sections "The choice of C",
                      "Coordinate systems"); the transposed cycle runs y then x               */
  MG_GSADI = 7     /* GSADI: a GSTRIx sweep then a GSTRIy sweep; transposed: y then x, each
                      with its colours reversed.  y-lines across a periodic y are cyclic
                      tridiagonal systems: solved by cyclic reduction with wrapped indices
                      (lines of 4 to 2048 unknowns), else Thomas with Sherman-Morrison      */
} mg_smoother;

typedef enum { MG_COEF_CONST = 0, MG_COEF_SEPARABLE = 1, MG_COEF_CELL = 2, MG_COEF_EDGE = 3 } mg_coef_kind;

/* MG_FP64: every step in double precision.
 * MG_MIXED: iterative refinement -- the FP64 defect r = b - A x drives one or
 * more single-precision F-cycles (smoothing, restriction, prolongation in
 * FP32; the coarsest-grid solve in FP64) whose correction is added to x in FP64. */
typedef enum { MG_FP64 = 0, MG_MIXED = 1 } mg_precision;

#define MG_FLAG_NO_GRAPH 1u   /* launch the cycle kernel by kernel instead of as a CUDA graph */
#define MG_FLAG_TIMING   2u   /* record CUDA events around every finest-level smoothing launch */
#define MG_FLAG_NO_FUSED_COARSE 4u  /* run every grid with per-step kernels (no single-CTA coarse cycle) */
#define MG_FLAG_NO_FUSED_SWEEP  8u  /* 2-D: red-black half-sweep kernels and a separate defect / restriction */
#define MG_FLAG_NO_TMA          16u /* 2-D FP32 red-black sweeps: register-marching kernel instead of the
                                       TMA-fed one (same arithmetic, same results) */
#define MG_FLAG_FMG_START       32u /* ignore the caller's x: start from nested iteration (Wallis 2008,
                                       section "Start-Vector Choice"): b restricted to every level, the
                                       coarsest level solved exactly, then on each finer level the
                                       interpolated solution improved by one F-cycle.  Its cycles are
                                       not counted in mg_report.cycles.  MG_MIXED runs it in FP32 */
#define MG_FLAG_ADAPTIVE_CORR   64u /* every coarse-grid correction added with the weight that minimises
                                       the energy norm of the error (Wallis 2008, section "Multigrid"):
                                       omega_l = (g - A u, P e) / (A P e, P e) on the iterate u before
                                       the correction; omega_corr is ignored */
#define MG_FLAG_GALERKIN        256u /* coarse operators by the Galerkin product A_{l-1} = R A_l P (full
                                       weighting R, bilinear P) instead of rediscretisation: 9-point
                                       stencils below the finest grid.  2-D, y not periodic, MG_JACOBI
                                       or MG_RBGS (on the 9-point levels Gauss-Seidel runs in four
                                       colours (i mod 2, j mod 2): (0,0), (1,1), (1,0), (0,1), the
                                       transposed cycle in the reverse order), coarsest grid of at
                                       most 4096 unknowns, not with MG_FLAG_ADAPTIVE_CORR; otherwise
                                       MG_EINVAL.  The single-CTA coarse cycle is not used */
#define MG_FLAG_FP64_DEFECT     512u /* MG_MIXED: keep the refinement loop's defect r = b - A x in FP64.
                                       By default, in 2-D with constant or separable coefficients, that
                                       defect (the start vector's included) is evaluated in float-float
                                       arithmetic (each FP64 operand split into two floats, error-free
                                       FP32 sums and products; about 2^-46 of |b| + |A||x| in error
                                       instead of 2^-53).  The kernel
                                       also sums (|b| + |A||x|)^2; the loop stops on that residual only
                                       when it is below the tolerance by the error estimate E = 2^-46
                                       times the root of that sum, moves to FP64 defects when E is half
                                       the tolerance or more, when the residual is within 10 E of the
                                       tolerance or when a step cuts it by less than half, and the
                                       reported relative residual is the FP64 one of the result */
#define MG_FLAG_NO_PDL          1024u /* graphs keep ordinary dependencies between kernels (by default the
                                       kernel-to-kernel edges of the solve's graphs are programmatic: a
                                       kernel's launch overlaps its predecessor's end and waits for its
                                       completion before reading) -- results do not depend on it */
#define MG_FLAG_TEST_BOUNDS     2048u /* test hook of the checking build (mg_debug_build() == 1): each
                                       solve starts with one device-side bounds check of the index one
                                       past the finest grid's last node (nothing is accessed there), so
                                       that it returns MG_EBOUNDS with the context still usable; the
                                       normal build returns MG_EINVAL for this flag */
#define MG_FLAG_TRACE           4096u /* per-kernel trace: solves run one graph launch per refinement
                                       step / cycle from the host, with an event after every kernel;
                                       mg_trace_report gives the time per kernel and level (slower than
                                       the device-side loop: for profiling) */
#define MG_FLAG_TEST_WAIT_TIMEOUT 128u /* test hook, never for production: in each solve one copy of the
                                       first single-precision TMA sweep is left out, so that the compute
                                       warps' bounded waits run out (about a second) and the solve returns
                                       MG_ETIMEOUT with the context still usable */

typedef struct {
  int dim;                /* 2 or 3 */
  int n[3];               /* finest-grid nodes per direction: 2^m + 1, or 2^m in periodic y */
  int periodic_y;         /* 1: y is periodic (n[1] distinct nodes) */
  int levels;             /* number of grids L, 1 <= L <= max for n */
  mg_smoother smoother;
  double omega;           /* smoother damping / SOR parameter */
  int nu1, nu2;           /* pre- and post-smoothing steps */
  double omega_corr;      /* omega_l of the correction u + omega_l P e (fixed) */
  mg_precision precision;
  int max_cycles;         /* F-cycles (FP64) or refinement steps (MG_MIXED) */
  int inner_cycles;       /* MG_MIXED: single-precision F-cycles per refinement step (>= 1) */
  void *stream;           /* cudaStream_t; NULL = legacy default stream */
  unsigned flags;         /* MG_FLAG_* */
  int coarse_cut_nodes;   /* grids with at most this many nodes run inside the single-CTA coarse
                             cycle (0: 5000 for 3-D single precision, 1200 otherwise; it must also
                             fit in shared memory) -- a tuning knob of the autotuner */
  int sweep_rows;         /* rows one CTA marches through in the fused 2-D red-black sweeps of
                             single precision (0: from the occupancy) -- a tuning knob; results do
                             not depend on it */
  int tile_nodes;         /* 2-D grids with at most this many nodes smooth with the one-pass tile
                             kernels instead of the row-streaming ones (0: 1050625 = 1025^2,
                             -1: never) -- a tuning knob; results do not depend on it */
} mg_params;

typedef struct {
  mg_coef_kind kind;
  double h[3];            /* mesh widths; MG_COEF_CELL forms weights from them */
  double c[3];            /* MG_COEF_CONST: edge weight per direction (e.g. eps/h^2, 1/h^2) */
  const double *sx;       /* MG_COEF_SEPARABLE (device): weight of x-edge (i, i+1), length n0-1 */
  const double *sy;       /* MG_COEF_SEPARABLE (device): weight of the y-edges at x-index i, length n0 */
  const double *sz;       /* MG_COEF_SEPARABLE (device): weight of the z-edges at x-index i (3-D) */
  const double *k;        /* MG_COEF_CELL (device): coefficient per cell of -div(k grad u) */
  /* MG_COEF_EDGE (device): full node arrays of the finest grid, x fastest (the layout of b):
     ex[p] = weight of the edge from node p to its +x neighbour, ey[p] to +y (periodic y: the
     last row's edge wraps to row 0), ez[p] to +z (3-D only; may be NULL in 2-D).  Entries of
     edges that do not exist are ignored; every edge touching an unknown must weigh > 0.  Any
     symmetric 5-/7-point operator in edge form, e.g. a grid refined in two directions or a
     mapped geometry whose weights vary in both directions (section "Anisotropies").  Coarse
     weights: harmonic mean of the two fine edges along a coarse edge, times 1/4.  y-line
     smoothing keeps its y-lines (no axis swap). */
  const double *ex, *ey, *ez;
} mg_coeffs;

typedef struct {
  int cycles;             /* F-cycles (or refinement steps) performed */
  double relres;          /* ||b - A x||_2 / ||b||_2 over the unknowns, in FP64, at return */
  double rate;            /* (relres / relres_0)^(1/cycles) */
  mg_status status;
  double *history;        /* HOST array, relres before each cycle and at return; may be NULL */
  int history_cap;
  double seconds;         /* wall time of the call (host clock, after the final sync) */
} mg_report;

/* Workspace size in bytes for these parameters and coefficient kind.  Returns 0
 * for invalid parameters. */
size_t mg_workspace_bytes(const mg_params *p, const mg_coeffs *k);

/* a1: build the level hierarchy (coarsened coefficients, diagonal inverses, the
 * dense inverse of the coarsest operator, the CUDA graph of one cycle) inside
 * the caller's workspace (device memory, >= mg_workspace_bytes, 256-byte
 * aligned).  The coefficient arrays are copied; the caller may free them after
 * the call returns.  On success *out owns a host context; free it with
 * mg_destroy.  Sections "The Multigrid Technique" (A_l, S_l, P, R, A_1^{-1})
 * and "The choice of C" (preconditioner memory set up before iterating). */
mg_status mg_setup(const mg_params *p, const mg_coeffs *k, void *workspace, size_t ws_bytes, mg_ctx **out);

/* Solve A x = b by F-cycles until ||b - A x|| / ||b|| <= tol or max_cycles.
 * b: device, read-only.  x: device, in = start vector, out = solution (start
 * vector choice: section "Start-Vector Choice").  rep may be NULL.
 * Returns MG_OK, MG_ENOCONV (x = last iterate) or MG_EDIVERGED. */
mg_status mg_solve(mg_ctx *c, const double *b, double *x, double tol, mg_report *rep);

/* mg_solve with b and x in HOST memory (pageable or pinned): b and the start
 * vector are copied straight into the solver's finest-level buffers, the
 * solution is copied back into x before the call returns.  The copies are
 * stream-ordered on mg_params.stream; the call is synchronous. */
mg_status mg_solve_host(mg_ctx *c, const double *b_host, double *x_host, double tol, mg_report *rep);

/* Adjoint solve A^T lambda = g with the transposed F-cycle M^T (steps of the
 * cycle in reverse order, each transposed).  Same conventions as mg_solve. */
mg_status mg_solve_adjoint(mg_ctx *c, const double *g, double *lambda, double tol, mg_report *rep);

/* ---- Batched solves -------------------------------------------------------------
 * The paper solves one problem at a time; solving many independent problems together
 * is an addition of this library.  Each instance has its own context (its own sizes,
 * coefficients, smoother, precision and max_cycles) and its own b / x (device
 * pointers, layout as for mg_solve).  A batch runs in one of two forms, on the first
 * context's stream, with one host synchronisation per solve:
 *   - persistent (MG_BATCH_PERSISTENT): ONE cooperative kernel launch solves every
 *     instance.  Each instance is owned by a team of CTAs (sized in proportion to its
 *     grid; instances beyond the resident CTA count are dealt to teams in turn) that runs
 *     the instance's whole mixed-precision solve -- copy in, FP32 F-cycles, FP64 defect
 *     and update, the convergence test, copy out -- from a step program, with a team
 *     barrier between steps (grids up to 129^2 run on the team's first CTA alone).
 *     Every barrier wait is bounded (about a second): a team whose wait runs out stops,
 *     and its instances report MG_ETIMEOUT.  Covers contexts that are 2-D, y not
 *     periodic, constant or separable coefficients, MG_MIXED with inner_cycles = 1,
 *     MG_JACOBI / MG_RBGS / MG_LINE_X / MG_ZEBRA_X (and MG_LINE_Y / MG_ZEBRA_Y with
 *     constant coefficients, which run as x-lines of the axis-swapped problem), without
 *     MG_FLAG_GALERKIN, MG_FLAG_FMG_START or MG_FLAG_ADAPTIVE_CORR, with a coarsest grid
 *     of at most 4096 unknowns.  Its tables live in the contexts' workspaces.
 *   - graph (MG_BATCH_GRAPH): ONE CUDA graph launch with an independent branch per
 *     instance (copy in, initial check, a device-side loop to that instance's own test,
 *     copy out), for any contexts.
 *   MG_BATCH_AUTO: the qualifying instances whose finest grid has at most 100,000 nodes (up to
 *     257^2) in one persistent launch, then the others in one graph launch (an instance with a
 *     large grid solves faster as graph branches spread over the whole GPU than as a team of
 *     a few CTAs).
 *
 * mg_batch_create / mg_batch_create_ex: builds the batch for count contexts and their
 *   b[i] / x[i] (host arrays of device pointers; the pointer values are kept).  The
 *   contexts, b[i] and x[i] must stay valid until mg_batch_destroy.  MG_EINVAL for a
 *   NULL argument, count < 1, a context used twice, contexts on different devices, a
 *   context made with MG_FLAG_NO_GRAPH or MG_FLAG_TIMING, or MG_BATCH_PERSISTENT for
 *   contexts it does not cover.  The batch uses no device memory of its own (each
 *   instance works in its context's workspace); it owns a small pinned host buffer for
 *   the tolerance and the per-instance reports.  A context in a persistent batch may
 *   still be solved on its own.
 * mg_batch_solve: solves every instance to ||b_i - A_i x_i|| / ||b_i|| <= tol from
 *   the start vectors in x[i]; reps (NULL, or count reports) receives each instance's
 *   report.  Returns MG_OK when every instance converged, else the status of the
 *   first instance (in index order) that did not (MG_ENOCONV, MG_EDIVERGED,
 *   MG_ETIMEOUT); the x[i] hold each instance's last iterate either way (not for an
 *   instance that reports MG_ETIMEOUT).
 * mg_batch_info: *persistent = the number of instances the persistent launch solves (0: the
 *   graph alone), with its CTA and team counts.
 * mg_solve_batched: create (MG_BATCH_AUTO), solve and destroy in one call (the batch is
 *   built on every call; keep a batch to solve the same set repeatedly). */
typedef struct mg_batch mg_batch;
#define MG_BATCH_AUTO 0
#define MG_BATCH_GRAPH 1
#define MG_BATCH_PERSISTENT 2
mg_status mg_batch_create(mg_ctx *const *cs, int count, const double *const *b, double *const *x, mg_batch **out);
mg_status mg_batch_create_ex(mg_ctx *const *cs, int count, const double *const *b, double *const *x, int mode,
                             mg_batch **out);
mg_status mg_batch_info(const mg_batch *bt, int *persistent, int *ctas, int *teams);
mg_status mg_batch_solve(mg_batch *bt, double tol, mg_report *reps);
void mg_batch_destroy(mg_batch *bt);
mg_status mg_solve_batched(mg_ctx *const *cs, int count, const double *const *b, double *const *x, double tol,
                           mg_report *reps);

/* MG_COEF_CELL only: dk[c] = -sum over the edges e of cell c of
 * (d w_e / d k_c) (u_p - u_q)(lambda_p - lambda_q), i.e. dL/dk for a loss L
 * whose gradient in u is A^T lambda.  dk: device cell array, overwritten. */
mg_status mg_grad_coeff(mg_ctx *c, const double *u, const double *lambda, double *dk);

/* Au = A_l u on level l (1..L).  u, Au: device node arrays of level l. */
mg_status mg_apply(mg_ctx *c, int level, const double *u, double *Au);

/* ||b - A_l u||_2 over the unknowns of level l (1..L; MG_MIXED contexts: level L only), the
 * stopping quantity of the solve (section "Smoothers": the defect A x - b that C^{-1}
 * acts on).  u, b: device node arrays of level l (Dirichlet entries ignored); out: device
 * pointer to one double.  The reduction is deterministic (fixed-order partial sums held
 * in the context's workspace). */
mg_status mg_residual_norm(mg_ctx *c, int level, const double *u, const double *b, double *out);

/* ||b - A u||_2 over the unknowns of one grid, without a context and without allocating.
 * The paper has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc (for instance code whose device memory is owned entirely by another
 * allocator or a fixed budget, or code running while its stream is being captured),
 * and so cannot allocate the workspace mg_setup needs.
 *   p: dim, n, periodic_y and stream are used (levels, smoother etc. are ignored);
 *   k: MG_COEF_CONST or MG_COEF_SEPARABLE (MG_COEF_CELL returns MG_EINVAL);
 *   u, b: device node arrays in the compact caller layout, read in place -- the
 *         Dirichlet entries of u must hold 0; out: device pointer to one double.
 * The per-block partial sums live in a file-scope __device__ array of 65,568 doubles
 * (~512 KB) that every GPU touched by the library holds until the process exits.  One
 * partial sum covers at least 32 x-unknowns of a row, so a grid is accepted when it has at
 * most MG_NOALLOC_MAX_NODES nodes AND at most MG_NOALLOC_MAX_XUNKNOWNS unknowns along x
 * (n[0] - 2); any other grid returns MG_EINVAL before anything is launched.  The first
 * call on a device looks up that array's device address (cudaGetSymbolAddress) with the
 * device current; make that first call before any stream capture.  The call is
 * stream-ordered and asynchronous: *out is ready once p->stream has synchronised.  All
 * calls share the one array, so calls that overlap on the GPU (other streams, other host
 * threads) race; each call writes every slot it later reads, nothing has to be cleared
 * between calls. */
#define MG_NOALLOC_MAX_NODES 2147483647LL
#define MG_NOALLOC_MAX_XUNKNOWNS (32LL * 65536)
mg_status mg_residual_norm_noalloc(const mg_params *p, const mg_coeffs *k, const double *u, const double *b,
                                   double *out);

/* Level geometry: nodes per direction of level l. */
mg_status mg_level_dims(const mg_ctx *c, int level, int n[3]);

/* Single steps of the cycle, for testing.  Arguments are FP64 node arrays of the given
 * level in the caller layout, device pointers, out-of-place outputs.  Each step runs the
 * kernels the cycle runs on that level, in the context's precision: FP64 contexts compute
 * in FP64; MG_MIXED contexts round the inputs to FP32, compute in FP32 (the coarsest solve
 * excepted, which is FP64 in both) and widen the outputs to FP64.  MG_ETIMEOUT if a
 * bounded device wait gave up.
 *   mg_step_smooth:   out = S^sweeps(u, g) with colour order 0 = red first, 1 = black first
 *   mg_step_defect:   r = g - A_l u
 *   mg_step_restrict: gc = R r            (level = fine level, >= 2)
 *   mg_step_prolong:  u_out = u + w P ec  (level = fine level, >= 2)
 *   mg_step_coarse:   u = A_1^{-1} g
 *   mg_step_cycle:    x_out = one F-cycle (transposed = 1: one transposed cycle) from x
 *   mg_step_descend:  the first half of a visit of level l >= 2 in algorithm MG(l, u, g)
 *                     (section "The Multigrid Technique"): u_out = S^nu1(u, g) (transposed:
 *                     nu2 sweeps, colours reversed), then gc = R (g - A_l u_out) on level
 *                     l-1.  u == NULL starts the sweeps from zero, as on the first visit
 *                     of a coarse level.  The fused kernels the cycle uses here (sweeps with
 *                     the defect and restriction, the streamed defect + restriction) run.
 *   mg_step_ascend:   the second half: u_out = S^nu2(u + omega_l P ec, g) (transposed:
 *                     nu1 sweeps, colours reversed), ec on level l-1, omega_l as the
 *                     context's cycle takes it; the correction is folded into the first
 *                     fused red-black sweep where the cycle folds it. */
mg_status mg_step_smooth(mg_ctx *c, int level, const double *u, const double *g, double *out, int sweeps, int order);
mg_status mg_step_defect(mg_ctx *c, int level, const double *u, const double *g, double *r);
mg_status mg_step_restrict(mg_ctx *c, int level, const double *r, double *gc);
mg_status mg_step_prolong(mg_ctx *c, int level, const double *ec, const double *u, double *u_out, double w);
mg_status mg_step_coarse(mg_ctx *c, const double *g, double *u);
mg_status mg_step_cycle(mg_ctx *c, const double *x, const double *b, double *x_out, int transposed);
mg_status mg_step_descend(mg_ctx *c, int level, const double *u, const double *g, double *u_out, double *gc,
                          int transposed);
mg_status mg_step_ascend(mg_ctx *c, int level, const double *ec, const double *u, const double *g, double *u_out,
                         int transposed);
/* MG_MIXED contexts: the refinement loop's defect r = (float)(b - A x) of the finest grid, as the
 * solve's loop first computes it (float-float or FP64, see MG_FLAG_FP64_DEFECT), widened to FP64
 * into r (caller layout); *sq (host, may be NULL) receives the sum of its squares.  MG_EINVAL for
 * FP64 contexts. */
mg_status mg_step_outer_defect(mg_ctx *c, const double *x, const double *b, double *r, double *sq);

/* Mean duration (ms) of the finest-level smoothing launches recorded since the
 * last call (MG_FLAG_TIMING), their count, and the mean algorithmic bytes of one
 * such launch: per unknown, read u and g and write u (3 words), 2 words for a sweep
 * whose iterate starts at zero, plus one read of the coarse correction (per coarse
 * unknown) for a sweep that folds it in.  Resets the record. */
mg_status mg_kernel_timing(mg_ctx *c, double *mean_ms, int *launches, double *bytes_per_launch);

/* Number of kernels the library launched since the context was created. */
long long mg_launch_count(const mg_ctx *c);

void mg_destroy(mg_ctx *c);
const char *mg_status_str(mg_status s);
const char *mg_last_error(const mg_ctx *c);

/* Contexts made with MG_FLAG_TRACE: the trace gathered by the solves since the last report, as
 * text, one line per kernel launcher and level ("name level launches total_ms", the most
 * expensive first; a kernel's time is the time between the events after it and after the kernel
 * before it, launch latency included).  Writes the full length + 1 to *len (may be NULL); with
 * buf (host) non-NULL also writes at most cap bytes (NUL-terminated) there and clears the trace.
 * MG_EINVAL for contexts without the flag. */
mg_status mg_trace_report(mg_ctx *c, char *buf, size_t cap, size_t *len);

/* 1 for the checking build of this library (compiled with -DMG_DEBUG: every kernel checks the
 * node indices of its global accesses against the level's arrays, skips an access out of range
 * and records its site; each call that synchronises then returns MG_EBOUNDS), 0 for the normal
 * build, whose kernels carry no checks. */
int mg_debug_build(void);

#ifdef __cplusplus
}
#endif
#endif
