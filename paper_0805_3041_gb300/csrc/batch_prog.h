// batch_prog.h -- the persistent batched solve: step codes and the device tables it reads.
//
// One cooperative launch solves many independent problems.  Each instance is owned by a team
// of CTAs (a team may take several instances in turn); the team executes the instance's step
// program -- the mixed-precision refinement loop around FP32 F-cycles, the convergence test,
// the copies in and out -- with a team barrier after each step.  Steps on small grids are run
// by the team's first CTA alone ("solo"), with block barriers only.  All tables live in the
// instances' own workspaces; the launch allocates nothing.
#pragma once

#include "mg_internal.cuh"

namespace mg {

enum BatchOp {
  BP_PACK = 1,      // x64 <- caller x, b64 <- caller b (transposed for axis-swapped instances)
  BP_NORM_B = 2,    // scal[0] = ||b64||^2 over the unknowns
  BP_DEFECT64 = 3,  // g_L = (float)(b64 - A x64), scal[1] = sum of its squares
  BP_CHECK = 4,     // convergence test (a = 1: initial); the loop ends at the program's BP_UNPACK
  BP_ZERO = 5,      // u_l[a] = 0
  BP_RB = 6,        // red-black half sweep of colour a on u_l[b], in place
  BP_JAC = 7,       // u_l[b >> 4] = Jacobi step from u_l[b & 15]
  BP_XLINE = 8,     // x-line sweep: a = zebra | colour << 1; b = src | dst << 4 (zebra: src == dst)
  BP_DEFECT = 9,    // r_l = g_l - A u_l[a]
  BP_RESTRICT = 10, // g_{l-1} = R r_l
  BP_PROLONG = 11,  // u_l[a] += omega_l P u_{l-1}[b]
  BP_COARSE = 12,   // u_1[a] = A_1^{-1} g_1
  BP_COPY = 13,     // u_l[b] = u_l[a]
  BP_UPDATE = 14,   // x64 += u_L[a]
  BP_JUMP = 15,     // continue at step a
  BP_UNPACK = 16,   // caller x <- x64 (0 when b = 0)
  BP_END = 17
};
// bit of the op code: the step runs on the team's first CTA alone
constexpr int BP_SOLO = 1 << 8;

// one FP32 level of one instance
struct BatchLev {
  Lev<float> L;
  float *u[2], *g, *r;
};

// one instance: where its data and program are, and how it reports
struct BatchInst {
  int L;                       // levels
  const BatchLev *lev;         // lev[l - 1] = level l
  const int4 *prog;            // step program
  int plen;
  Lev<double> F64;             // finest level in FP64 (geometry and FP64 coefficients)
  int kind;                    // coefficient kind (K_CONST or K_SEP)
  double *x64, *b64;           // FP64 iterate and right-hand side (internal layout)
  const double *bcall;         // caller's b and x (compact layout, device)
  double *xcall;
  int swap;                    // caller layout is the transpose of the internal one
  int n0c, n1c;                // caller's node counts along x and y
  const double *Ainv;          // coarsest grid: dense inverse over its unknowns
  const long long *cidx;
  int nc;
  double *scal;                // [0] ||b||^2, [1] ||r||^2
  double *hrow;                // report row (mapped pinned host memory): as ints, [0] steps done, [1] status
                               // (0 ok, 4 no convergence, 5 diverged), [2] 0, [3] the launch's epoch once
                               // the instance is done; as doubles, [2] ||b||^2, [3 + k] the relative
                               // residual before step k and at the end
  int *st;                     // the context's loop state: [2] is set when a bounded wait gave up
  const double *tol;           // device scalar
  int maxit;
  float omega, omega_corr;
  int fail_arrival;            // test hook: the team's last CTA leaves at its first team barrier
};

// one team: CTAs [cta0, cta0 + size), instances inst[first .. first + count) in turn
struct BatchTeam {
  int cta0, size, first, count;
  unsigned *bar;               // barrier counter (zero before the launch)
  double *part;                // 2 * size partial sums (double-buffered reductions)
};

// launch the persistent batched solve: grid = number of CTAs, every team's CTAs resident
// (cooperative launch); teams / insts / order: device tables; epoch: written into each report
// row whose instance finishes, so that the host can tell finished rows from stale ones
cudaError_t launch_batch(cudaStream_t s, int grid, const BatchTeam *teams, int nteams, const BatchInst *insts,
                         const int *order, int epoch, long long *counter);
// resident CTAs of the batch kernel per SM
int batch_ctas_per_sm();
constexpr int kBatchThreads = 256;

}  // namespace mg
