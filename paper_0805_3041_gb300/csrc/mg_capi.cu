// mg_capi.cu -- host side of the solver: parameter checks, workspace layout,
// set-up of the level hierarchy, the F-cycle schedule (captured as a CUDA graph)
// and the C ABI declared in include/mg.h.
//
// The cycle follows Wallis (2008), section "The Multigrid Technique",
// algorithm MG(l, u, g), run as the F-cycle of the abstract: F(l) = pre-smooth,
// restrict the defect, F(l-1) from zero then V(l-1), correct with omega_l P e,
// post-smooth; V(l) recurses once; level 1 is solved directly.  The transposed
// cycle (adjoint solves) runs the same steps in reverse order, each transposed.
#include <chrono>
#include <cmath>
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/mg.h"
#include "coarse_prog.h"
#include "batch_prog.h"
#define MG_FILE_ID 13   // bounds-check sites (-DMG_DEBUG)
#include "mg_internal.cuh"

using namespace mg;

static const int MAXLEV = 16;

// ---------------------------------------------------------------------------------------
// workspace layout
// ---------------------------------------------------------------------------------------
struct Bump {
  char *base;
  size_t off;
  template <typename T>
  T *take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T *p = base ? (T *)(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

template <typename T>
struct LevData {
  T *u[2] = {nullptr, nullptr};
  T *g = nullptr, *r = nullptr;
  T *sx = nullptr, *sy = nullptr, *sz = nullptr, *sdinv = nullptr;
  T *k = nullptr, *ndinv = nullptr;
  T *ex = nullptr, *ey = nullptr, *ez = nullptr;
  T *t = nullptr;   // third line-solve scratch array (y-lines across a periodic y)
  T *dg = nullptr, *enw = nullptr;   // Galerkin levels: diagonal and -x+y weights (ex, ey, ez: +x, +y, +x+y)
};

struct LevGeom {
  int n[3];
  long long pitch, plane, count;   // elements per row / plane / array
  double c[3], d, dinv;            // CONST
  double ax, ay, az, h[3];         // CELL
};

struct mg_ctx {
  mg_params P;
  mg_coeffs K;
  int L;
  int kind;
  bool galerkin = false;   // MG_FLAG_GALERKIN: levels below the finest hold R A P (K_NINE)
  bool ff = false;         // MG_MIXED: the refinement loop's defect in float-float (kernels_ff.cu)
  LevGeom geo[MAXLEV + 1];
  LevData<double> d64[MAXLEV + 1];
  LevData<float> d32[MAXLEV + 1];
  bool mixed;
  // finest FP64 vectors of the mixed form
  double *x64 = nullptr, *b64 = nullptr;
  double *x64b = nullptr;       // float-float contexts: the second buffer of the fused update (st[7]: current)
  // scratch for reductions and scalars
  double *partials = nullptr;
  double *scal = nullptr;       // [0] bsq, [1] sq, [2] relres, [3] scratch, [4] tol, [5] float-float error scale, [8] omega
  double *hist = nullptr;       // device history, max_cycles + 2
  double *grad_tmp = nullptr;   // CELL gradient: padded dk
  // coarsest grid
  int nc = 0;
  long long *cidx = nullptr;
  int *cmap = nullptr;
  double *Ainv = nullptr, *gjcol = nullptr;
  // coarsest grids above the dense limit: conjugate gradients (FP64 x, r, p, A p on level 1)
  bool cg_mode = false;
  double *cgw = nullptr;
  int cg_max_it = 0;
  // single-CTA coarse kernel: every grid <= lcut in shared memory (lcut = 0: not used)
  int lcut = 0;
  void *slev = nullptr;            // device table of shared-memory level views
  int4 *prog = nullptr;            // device programs
  int prog_off[9] = {0}, prog_len[9] = {0};
  int prog_used = 0;               // int4 entries of prog taken by the coarse programs
  long long *cidx_s = nullptr;     // coarsest unknowns in the compact shared-memory layout
  size_t csk_smem = 0;
  // y-line smoothers run as x-line smoothers on the axis-swapped problem: internal node
  // (i, j, k) is the caller's (j, i, k); only the copies in and out see the difference
  bool swap = false;
  // bookkeeping
  int cur[MAXLEV + 1];          // current u buffer per level (schedule state)
  long long launches = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  cudaStream_t cap2 = nullptr;  // captures the body of a device-side solve loop
  int dev = 0;                  // the device the context was set up on
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};   // forward / transposed cycle + check
  cudaGraphExec_t lexec[2] = {nullptr, nullptr};   // whole solve: device-side WHILE loop
  long long loop_init_kernels[2] = {0, 0}, loop_body_kernels[2] = {0, 0};
  unsigned *oob = nullptr;                         // device bounds word (-DMG_DEBUG build's checks)
  int *st = nullptr;                               // device loop state: [0] cycles done, [1] status, [2] a wait
                                                   // gave up, [4] CG, [5] test hook, [6] FP64 outer defects
  unsigned *cnt = nullptr;                         // device: block counter of last-block reductions (zero at rest)
  long long graph_kernels[2] = {0, 0};
  double *h_relres = nullptr;   // pinned
  // timing of finest-level smoothing launches
  std::vector<cudaEvent_t> ev;  // pool: [0, 2048) direct launches, [2048, 4096) forward graph,
                                // [4096, 6144) transposed graph
  int ev_used = 0;
  int ev_graph_n[2] = {0, 0};
  double t_sum_ms = 0.0;
  double t_sum_bytes = 0.0;
  long long t_count = 0;
  std::vector<double> ev_bytes;   // algorithmic bytes of the launch opened by each pool event
  std::string err;
  // MG_FLAG_TRACE: event marks after every kernel of a refinement step / cycle (the forward
  // schedule in marks [0, kTraceMarks), the transposed one after it), and the sums per kernel
  // and level since the last report
  Tracer tracer;
  std::vector<cudaEvent_t> tr_ev;
  std::vector<const char *> tr_label;
  std::vector<int> tr_lev;
  int tr_n[2] = {0, 0};
  long long tr_steps = 0, tr_unread = 0;   // harvested schedules, marks whose time could not be read
  std::map<std::pair<std::string, int>, std::pair<long long, double>> tr_sum;
};
static const int kTraceMarks = 2048;

// Error estimate of the float-float outer defect relative to the norm of |b| + |A||x| (which
// that kernel also returns).  Each operand carries 47 significant bits, so a node's error is a
// few 2^-46 of its terms; measured over whole grids the norm of the error was 0.15 (isotropic
// 4097^2 benchmark), 0.19 (lines with eps = 1e3) and 0.5 (eps = 1e-3) of 2^-46 times that
// norm.  The loop stops on the float-float residual only below the tolerance by this estimate
// E.  It moves to FP64 defects when E is half the tolerance or more (the float-float residual
// could never decide), within kFFSwitch * E of the tolerance, or when a step cuts the residual
// by less than half: once the defect's error is a sizeable part of the residual the FP32 cycle
// is driven by that error, whose smooth part it amplifies (on the eps = 1e3 lines, E = 3.7 tol,
// the loop stalled at a true residual of 30 times the defect's error).  The FP64 residual
// computed afterwards is the one reported.
static const double kFFErr = 0x1p-46;
static const double kFFSwitch = 10.0;

// NVTX ranges name the phases of the cycle (solve, refinement step, each level's descending
// and ascending half, the coarse cycle in one CTA, the coarsest solve) for profilers.  They are
// pushed on the host around the launches: kernel by kernel (MG_FLAG_NO_GRAPH) they bracket
// the phase's kernels on a timeline; in the graph form they bracket the capture.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  NvtxRange(const char *what, int level) {
    char buf[64];
    snprintf(buf, sizeof buf, "level %d: %s", level, what);
    nvtxRangePushA(buf);
  }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// the operator form of level l: the context's coefficient kind, or K_NINE on Galerkin coarse levels
static int lev_kind(const mg_ctx *c, int l) { return (c->galerkin && l < c->L) ? K_NINE : c->kind; }

// rows padded to 128 elements: the marching kernels read 128-column strips with vector loads
static size_t padded_pitch(int n0) { return (size_t)((n0 + 127) / 128) * 128; }

static int coarsen_dims(const int nf[3], int dim, int per, int nc[3]) {
  if ((nf[0] - 1) % 2 || nf[0] < 5) return 0;
  nc[0] = (nf[0] - 1) / 2 + 1;
  if (per) {
    if (nf[1] % 2 || nf[1] < 4) return 0;
    nc[1] = nf[1] / 2;
  } else {
    if ((nf[1] - 1) % 2 || nf[1] < 5) return 0;
    nc[1] = (nf[1] - 1) / 2 + 1;
  }
  if (dim == 3) {
    if ((nf[2] - 1) % 2 || nf[2] < 5) return 0;
    nc[2] = (nf[2] - 1) / 2 + 1;
  } else {
    nc[2] = 1;
  }
  return 1;
}

static const long long kDenseCoarseMax = 4096;   // coarsest unknowns solved with a dense inverse

// line smoothers: the single-CTA coarse kernel keeps a third scratch array per level for their
// line steps (cyclic reduction over all lines, or the cyclic Thomas solve)
static bool line_smoother(const mg_params &P) {
  return P.smoother == MG_LINE_X || P.smoother == MG_LINE_Y || P.smoother == MG_ZEBRA_X ||
         P.smoother == MG_ZEBRA_Y || P.smoother == MG_ADI || P.smoother == MG_GSADI;
}

static mg_status check_params(const mg_params *p, const mg_coeffs *k) {
  if (!p || !k) return MG_EINVAL;
  if (p->dim != 2 && p->dim != 3) return MG_EINVAL;
  if (p->levels < 1 || p->levels > MAXLEV) return MG_EINVAL;
  if (p->smoother < MG_JACOBI || p->smoother > MG_GSADI) return MG_EINVAL;
  if (p->nu1 < 0 || p->nu2 < 0 || p->nu1 + p->nu2 < 1) return MG_EINVAL;
  if (p->precision != MG_FP64 && p->precision != MG_MIXED) return MG_EINVAL;
  if (p->max_cycles < 0 || p->sweep_rows < 0 || p->tile_nodes < -1) return MG_EINVAL;
  if (k->kind < MG_COEF_CONST || k->kind > MG_COEF_EDGE) return MG_EINVAL;
  if (k->kind == MG_COEF_EDGE && (!k->ex || !k->ey || (p->dim == 3 && !k->ez))) return MG_EINVAL;
  if (k->kind == MG_COEF_SEPARABLE && (!k->sx || !k->sy || (p->dim == 3 && !k->sz))) return MG_EINVAL;
  if (k->kind == MG_COEF_CELL && !k->k) return MG_EINVAL;
  int n[3] = {p->n[0], p->n[1], p->dim == 3 ? p->n[2] : 1};
  if (n[0] < 3 || n[1] < (p->periodic_y ? 2 : 3) || (p->dim == 3 && n[2] < 3)) return MG_EINVAL;
  if (p->periodic_y && (n[1] % 2)) return MG_EINVAL;
  if ((long long)n[0] * n[1] * n[2] > (1LL << 34)) return MG_EINVAL;
  // the reductions keep one partial sum per block of 32 unknowns of a row (4096 partials for the
  // adaptive weight's), on either axis (y-line smoothers may swap them)
  if (!norm_shape_ok(n[0] - 2, 4096) || !norm_shape_ok(n[1] - 2, 4096)) return MG_EINVAL;
  for (int l = 1; l < p->levels; ++l) {
    int c[3];
    if (!coarsen_dims(n, p->dim, p->periodic_y, c)) return MG_EINVAL;
    memcpy(n, c, sizeof(n));
  }
  // coarsest grid: a dense inverse up to kDenseCoarseMax unknowns, conjugate gradients above
  long long nc = (long long)(n[0] - 2) * (p->periodic_y ? n[1] : n[1] - 2) * (p->dim == 3 ? n[2] - 2 : 1);
  if (nc > (1LL << 26)) return MG_EINVAL;
  // Galerkin coarse operators: 2-D, y not periodic, point smoothers, the dense coarsest solve,
  // the fixed correction weight
  if ((p->flags & MG_FLAG_GALERKIN) &&
      (p->dim != 2 || p->periodic_y || (p->smoother != MG_JACOBI && p->smoother != MG_RBGS) ||
       nc > kDenseCoarseMax || (p->flags & MG_FLAG_ADAPTIVE_CORR)))
    return MG_EINVAL;
#ifndef MG_DEBUG
  if (p->flags & MG_FLAG_TEST_BOUNDS) return MG_EINVAL;   // the probe needs the checking build
#endif
  return MG_OK;
}

// Fill geometry; with ws == nullptr only sizes are computed.  Returns total bytes.
// y-line smoothing on the unswapped problem (separable or edge coefficients, periodic y, ADI /
// GSADI): the line kernels keep three scratch arrays per level
static bool ylines_unswapped(const mg_ctx *c) {
  const int sm = c->P.smoother;
  return !c->swap && (sm == MG_LINE_Y || sm == MG_ZEBRA_Y || sm == MG_ADI || sm == MG_GSADI);
}

static size_t layout(mg_ctx *c, char *ws) {
  const mg_params &P = c->P;
  Bump b{ws, 0};
  int n[3] = {P.n[0], P.n[1], P.dim == 3 ? P.n[2] : 1};
  double h[3] = {c->K.h[0], c->K.h[1], c->K.h[2]};
  for (int l = c->L; l >= 1; --l) {
    LevGeom &g = c->geo[l];
    memcpy(g.n, n, sizeof(n));
    g.pitch = (long long)padded_pitch(n[0]);
    g.plane = g.pitch * n[1];
    g.count = g.plane * n[2];
    memcpy(g.h, h, sizeof(h));
    if (l > 1) {
      int cn[3];
      coarsen_dims(n, P.dim, P.periodic_y, cn);
      memcpy(n, cn, sizeof(n));
      for (int d = 0; d < 3; ++d) h[d] *= 2.0;
    }
  }
  for (int l = c->L; l >= 1; --l) {
    LevGeom &g = c->geo[l];
    size_t cnt = (size_t)g.count, n0 = (size_t)g.n[0];
    LevData<double> &D = c->d64[l];
    // FP64 coefficient data on every level (set-up and the FP64 coarsest solve use it)
    if (c->kind == K_SEP) {
      D.sx = b.take<double>(n0);
      D.sy = b.take<double>(n0);
      D.sz = b.take<double>(n0);
      D.sdinv = b.take<double>(n0);
    } else if (c->kind == K_CELL) {
      D.k = b.take<double>(cnt);
      D.ndinv = b.take<double>(cnt);
    } else if (c->kind == K_EDGE) {
      D.ex = b.take<double>(cnt);
      D.ey = b.take<double>(cnt);
      if (P.dim == 3) D.ez = b.take<double>(cnt);
      D.ndinv = b.take<double>(cnt);
    }
    if (lev_kind(c, l) == K_NINE) {
      D.dg = b.take<double>(cnt);
      D.ex = b.take<double>(cnt);
      D.ey = b.take<double>(cnt);
      D.ez = b.take<double>(cnt);
      D.enw = b.take<double>(cnt);
      D.ndinv = b.take<double>(cnt);
    }
    if (!c->mixed) {
      D.u[0] = b.take<double>(cnt);
      D.u[1] = b.take<double>(cnt);
      D.g = b.take<double>(cnt);
      D.r = b.take<double>(cnt);
      if (ylines_unswapped(c)) D.t = b.take<double>(cnt);
    } else {
      LevData<float> &F = c->d32[l];
      F.u[0] = b.take<float>(cnt);
      F.u[1] = b.take<float>(cnt);
      F.g = b.take<float>(cnt);
      F.r = b.take<float>(cnt);
      if (ylines_unswapped(c)) F.t = b.take<float>(cnt);
      if (c->kind == K_SEP) {
        F.sx = b.take<float>(n0);
        F.sy = b.take<float>(n0);
        F.sz = b.take<float>(n0);
        F.sdinv = b.take<float>(n0);
      } else if (c->kind == K_CELL) {
        F.k = b.take<float>(cnt);
        F.ndinv = b.take<float>(cnt);
      } else if (c->kind == K_EDGE) {
        F.ex = b.take<float>(cnt);
        F.ey = b.take<float>(cnt);
        if (P.dim == 3) F.ez = b.take<float>(cnt);
        F.ndinv = b.take<float>(cnt);
      }
      if (lev_kind(c, l) == K_NINE) {
        F.dg = b.take<float>(cnt);
        F.ex = b.take<float>(cnt);
        F.ey = b.take<float>(cnt);
        F.ez = b.take<float>(cnt);
        F.enw = b.take<float>(cnt);
        F.ndinv = b.take<float>(cnt);
      }
    }
  }
  size_t fine = (size_t)c->geo[c->L].count;
  if (c->mixed) {
    c->x64 = b.take<double>(fine);
    if (c->ff) c->x64b = b.take<double>(fine);
    c->b64 = b.take<double>(fine);
    // FP64 scratch of the finest level for mg_apply and the gradient
    c->d64[c->L].u[0] = b.take<double>(fine);
    c->d64[c->L].g = b.take<double>(fine);
    c->d64[c->L].r = b.take<double>(fine);
  }
  if (c->kind == K_CELL) c->grad_tmp = b.take<double>(fine);
  c->partials = b.take<double>((size_t)norm_parts_count());
  c->scal = b.take<double>(16);
  c->hist = b.take<double>((size_t)P.max_cycles + 2);
  c->st = b.take<int>(8);
  c->oob = b.take<unsigned>(4);
  c->cnt = b.take<unsigned>(8);
  // coarsest grid
  const LevGeom &g1 = c->geo[1];
  long long nc = (long long)(g1.n[0] - 2) * (P.periodic_y ? g1.n[1] : g1.n[1] - 2) * (P.dim == 3 ? g1.n[2] - 2 : 1);
  c->nc = (int)nc;
  c->cidx = b.take<long long>((size_t)nc);
  c->cmap = b.take<int>((size_t)g1.count);
  c->cg_mode = nc > kDenseCoarseMax;
  if (c->cg_mode) {
    c->cgw = b.take<double>(4 * (size_t)g1.count);
    c->cg_max_it = (int)std::min<long long>(20000, 2 * nc);
  } else {
    c->Ainv = b.take<double>((size_t)nc * nc);
    c->gjcol = b.take<double>((size_t)nc);
  }
  // single-CTA coarse kernel: deepest level whose grids (and all coarser) fit in shared memory
  c->lcut = 0;
  if (!(P.flags & MG_FLAG_NO_FUSED_COARSE) && !c->cg_mode && !c->galerkin) {
    size_t es = c->mixed ? 4 : 8, total = 0;
    size_t arrays = 4 + (c->kind == K_CELL ? 2 : c->kind == K_EDGE ? (P.dim == 3 ? 4 : 3) : 0) +
                    (line_smoother(P) ? 1 : 0);
    // FP64 runs at 2 FMA/clk/SM: keep the one-SM part small.  In 2-D the 65^2 level is faster on the
    // tile and line kernels too (4097^2 RB-GS solve 7.21 against 7.24 ms, annulus GSADI 19.9 against
    // 20.9); a 3-D 17^3 level (4913 nodes) stays in the one-CTA program
    long long cap = (c->mixed && P.dim == 3) ? 5000 : 1200;
    if (P.coarse_cut_nodes > 0) cap = P.coarse_cut_nodes;
    for (int l = 1; l <= c->L; ++l) {
      long long nodes = (long long)c->geo[l].n[0] * c->geo[l].n[1] * c->geo[l].n[2];
      total += arrays * (size_t)((nodes + 3) / 4 * 4) * es;
      if (total > 190 * 1024 || nodes > cap) break;   // + ~21 KB of static shared memory
      c->lcut = l;
    }
    if (c->lcut < 2) c->lcut = 0;
  }
  c->slev = b.take<char>((size_t)(MAXLEV + 1) * 512);
  c->prog = b.take<int4>(32768);
  c->cidx_s = b.take<long long>((size_t)nc);
  return b.off + 256;
}

template <typename T>
static Lev<T> make_lev(const mg_ctx *c, int l) {
  const LevGeom &g = c->geo[l];
  Lev<T> L;
  memset(&L, 0, sizeof(L));
  L.dim = c->P.dim;
  L.n0 = g.n[0];
  L.n1 = g.n[1];
  L.n2 = g.n[2];
  L.per = c->P.periodic_y ? 1 : 0;
  L.pitch = g.pitch;
  L.plane = g.plane;
  L.cx = (T)g.c[0];
  L.cy = (T)g.c[1];
  L.cz = (T)g.c[2];
  L.d = (T)g.d;
  L.dinv = (T)g.dinv;
  L.ax = (T)g.ax;
  L.ay = (T)g.ay;
  L.az = (T)g.az;
  L.oob = c->oob;
  return L;
}
static Lev<double> lev64(const mg_ctx *c, int l) {
  Lev<double> L = make_lev<double>(c, l);
  const LevData<double> &D = c->d64[l];
  L.sx = D.sx; L.sy = D.sy; L.sz = D.sz; L.sdinv = D.sdinv;
  L.k = D.k; L.ndinv = D.ndinv;
  L.ex = D.ex; L.ey = D.ey; L.ez = D.ez;
  L.dg = D.dg; L.enw = D.enw;
  return L;
}
// Line smoothers along y on constant or cell coefficients are run along x on the
// axis-swapped problem (contiguous lines; the x-line kernel keeps a line in shared
// memory).  Separable and edge coefficients keep their y-line kernel.
static void apply_swap(mg_ctx *c) {
  mg_params &P = c->P;
  bool yline = P.smoother == MG_LINE_Y || P.smoother == MG_ZEBRA_Y;
  if (!yline || c->kind == K_SEP || c->kind == K_EDGE || P.periodic_y) return;
  c->swap = true;
  int t = P.n[0];
  P.n[0] = P.n[1];
  P.n[1] = t;
  double a = c->K.c[0];
  c->K.c[0] = c->K.c[1];
  c->K.c[1] = a;
  a = c->K.h[0];
  c->K.h[0] = c->K.h[1];
  c->K.h[1] = a;
  P.smoother = P.smoother == MG_LINE_Y ? MG_LINE_X : MG_ZEBRA_X;
}

// caller layout <-> internal padded layout (transposing when the axes are swapped)
static void pack_in(mg_ctx *c, const Launch &lc, const Lev<double> &L, const double *src, double *dst, int zb) {
  if (c->swap) launch_pack_swapped<double>(lc, L, src, dst, zb);
  else launch_pack<double>(lc, L, src, dst, zb);
}
static void unpack_out(mg_ctx *c, const Launch &lc, const Lev<double> &L, const double *src, double *dst,
                       double scale) {
  if (c->swap) launch_unpack_swapped<double>(lc, L, src, dst, scale);
  else launch_unpack<double>(lc, L, src, dst, scale);
}

static Lev<float> lev32(const mg_ctx *c, int l) {
  Lev<float> L = make_lev<float>(c, l);
  const LevData<float> &D = c->d32[l];
  L.sx = D.sx; L.sy = D.sy; L.sz = D.sz; L.sdinv = D.sdinv;
  L.k = D.k; L.ndinv = D.ndinv;
  L.ex = D.ex; L.ey = D.ey; L.ez = D.ez;
  L.dg = D.dg; L.enw = D.enw;
  return L;
}
template <typename T> struct LevOf;
template <> struct LevOf<double> {
  static Lev<double> get(const mg_ctx *c, int l) { return lev64(c, l); }
  static LevData<double> &data(mg_ctx *c, int l) { return c->d64[l]; }
};
template <> struct LevOf<float> {
  static Lev<float> get(const mg_ctx *c, int l) { return lev32(c, l); }
  static LevData<float> &data(mg_ctx *c, int l) { return c->d32[l]; }
};

#define CK(call)                                                         \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) {                                             \
      c->err = std::string(#call) + ": " + cudaGetErrorString(e_);       \
      return MG_ECUDA;                                                   \
    }                                                                    \
  } while (0)

#ifdef MG_DEBUG
// Source file of a bounds-check site id (the MG_FILE_ID of each translation unit).
static const char *site_file(unsigned id) {
  static const char *names[] = {"?", "kernels_point.cu", "kernels_transfer.cu", "kernels_line.cu",
                                "kernels_coarse.cu", "kernels_fast.cu", "kernels_xline.cu", "kernels_march.cu",
                                "kernels_tma.cu", "noalloc.cu", "kernels_cg.cu", "kernels_batch.cu",
                                "kernels_ff.cu", "mg_capi.cu", "?", "mg_internal.cuh"};
  return id < 16 ? names[id] : "?";
}
#endif

// After the context's stream has been synchronised: a failed launch, and in the -DMG_DEBUG
// build a device-side bounds check that failed since the last call (the word is cleared).
static mg_status last_launch(mg_ctx *c) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    c->err = std::string("kernel launch: ") + cudaGetErrorString(e);
    return MG_ECUDA;
  }
#ifdef MG_DEBUG
  unsigned site = 0;
  e = cudaMemcpy(&site, c->oob, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && site) e = cudaMemset(c->oob, 0, sizeof(unsigned));
  if (e != cudaSuccess) {
    c->err = std::string("bounds word: ") + cudaGetErrorString(e);
    return MG_ECUDA;
  }
  if (site) {
    c->err = std::string("device bounds check failed at ") + site_file(site >> 16) + ":" +
             std::to_string(site & 0xffffu) + " (access skipped)";
    return MG_EBOUNDS;
  }
#endif
  return MG_OK;
}

// ---------------------------------------------------------------------------------------
// the cycle schedule
// ---------------------------------------------------------------------------------------
// MG_FLAG_ADAPTIVE_CORR: the coarse correction is scaled by its energy-optimal weight
// before it is added, which is then added with weight 1
static bool adaptive_corr(const mg_ctx *c) { return (c->P.flags & MG_FLAG_ADAPTIVE_CORR) != 0; }
static double corr_weight(const mg_ctx *c) { return adaptive_corr(c) ? 1.0 : c->P.omega_corr; }

struct Sched {
  mg_ctx *c;
  Launch lc;
  bool timing;
  int ev_base = 0;      // first event of this schedule's range in the pool
  int *ev_next = nullptr;
  bool loop = false;    // emitting into a device-side solve loop: end cycles with launch_step_end
  cudaGraphConditionalHandle loop_h = 0;
};

// unknowns of level l (periodic y: every row is unknown)
static double level_unknowns(const mg_ctx *c, int l) {
  const LevGeom &g = c->geo[l];
  return (double)(g.n[0] - 2) * (c->P.periodic_y ? g.n[1] : g.n[1] - 2) * (c->P.dim == 3 ? g.n[2] - 2 : 1);
}

static void record_event(Sched &S, double bytes = 0.0) {
  mg_ctx *c = S.c;
  if (!S.timing || !S.ev_next) return;
  int idx = S.ev_base + *S.ev_next;
  if (*S.ev_next >= 2046 || idx >= (int)c->ev.size()) return;
  c->ev_bytes[idx] = bytes;
  // "external" so that a stream capture turns the record into an event-record node
  cudaEventRecordWithFlags(c->ev[idx], S.lc.s, cudaEventRecordExternal);
  ++*S.ev_next;
}

// One fused 2-D red-black sweep in FP32 through the TMA-fed kernel, where it applies.
template <typename T>
static bool sweep_tma(Sched &, const Lev<T> &, const T *, const T *, T *, T, int, int, const Lev<T> *, const T *, T) {
  return false;
}
template <>
bool sweep_tma<float>(Sched &S, const Lev<float> &L, const float *u, const float *g, float *out, float om, int order,
                      int mode, const Lev<float> *Cp, const float *ec, float oc) {
  mg_ctx *c = S.c;
  if (c->P.flags & MG_FLAG_NO_TMA) return false;
  return launch_rb2d_tma(S.lc, L, c->kind, u, g, out, om, order, mode, Cp, ec, oc, c->st + 2, c->P.sweep_rows,
                         (c->P.flags & MG_FLAG_TEST_WAIT_TIMEOUT) ? c->st + 5 : nullptr);
}

// The fused defect + restriction in FP32 through the TMA-fed kernel, where it applies.
template <typename T>
static bool defect_restrict_tma(Sched &, const Lev<T> &, const Lev<T> &, const T *, const T *, T *) {
  return false;
}
template <>
bool defect_restrict_tma<float>(Sched &S, const Lev<float> &L, const Lev<float> &C, const float *u, const float *g,
                                float *gc) {
  mg_ctx *c = S.c;
  if (c->P.flags & MG_FLAG_NO_TMA) return false;
  return launch_defect_restrict_tma(S.lc, L, C, c->kind, u, g, gc, c->st + 2, 0);
}

// `sweeps` smoothing steps on level l.  With ec != nullptr the coarse-grid correction
// u += omega_l P ec is applied first -- folded into the first fused red-black sweep when
// there is one, as its own kernel otherwise.
template <typename T>
static void smooth(Sched &S, int l, const T *g, int sweeps, int order, bool zero_start, const Lev<T> *Cp = nullptr,
                   const T *ec = nullptr) {
  mg_ctx *c = S.c;
  LevData<T> &D = LevOf<T>::data(c, l);
  Lev<T> L = LevOf<T>::get(c, l);
  T om = (T)c->P.omega, oc = (T)corr_weight(c);
  int &cur = c->cur[l];
  bool jac = c->P.smoother == MG_JACOBI;
  bool line = c->P.smoother >= MG_LINE_X;
  const int kind = lev_kind(c, l);
  bool rb2d = c->P.smoother == MG_RBGS && c->P.dim == 2 && !(c->P.flags & MG_FLAG_NO_FUSED_SWEEP) && kind != K_NINE;
  if (ec && !(rb2d && sweeps > 0)) {
    launch_prolong_add<T>(S.lc, L, *Cp, ec, D.u[cur], oc);
    ec = nullptr;
  }
  if (sweeps <= 0) {
    if (zero_start) cudaMemsetAsync(D.u[cur], 0, sizeof(T) * (size_t)c->geo[l].count, S.lc.s);
    return;
  }
  bool fine = (l == c->L) && S.timing;
  int odd_guard = 0;
  if (zero_start && !jac && !rb2d) cudaMemsetAsync(D.u[cur], 0, sizeof(T) * (size_t)c->geo[l].count, S.lc.s);
  // algorithmic bytes of one sweep: read u and g, write u (2 arrays when the iterate starts
  // at zero and is not read; plus one read of the coarse correction when it is folded in)
  const double es = sizeof(T), unk = level_unknowns(c, l);
  for (int s = 0; s < sweeps; ++s) {
    if (fine && S.ev_next && *S.ev_next < 2046) {
      bool zero = zero_start && s == 0 && (jac || rb2d);
      bool fold = rb2d && ec && s == 0;
      double bytes = es * unk * (zero ? 2.0 : 3.0) + (fold ? es * level_unknowns(c, l - 1) : 0.0);
      record_event(S, bytes);
      odd_guard = 1;
    }
    if (jac) {
      if (zero_start && s == 0) launch_jacobi_zero<T>(L, kind, S.lc, g, D.u[1 - cur], om);
      else launch_jacobi<T>(S.lc, L, kind, D.u[cur], g, D.u[1 - cur], om);
      cur = 1 - cur;
    } else if (rb2d) {
      int mode = (zero_start && s == 0) ? 1 : (ec && s == 0) ? 2 : 0;
      // small grids: one pass over tiles (launch latency bound), two sweeps per pass where
      // two remain (not on a timed finest level); large: row streaming
      const long long tile_max = c->P.tile_nodes == 0 ? 1050625 : c->P.tile_nodes < 0 ? -1 : c->P.tile_nodes;
      const bool small = tile_max >= 0 && (long long)L.n0 * L.n1 <= tile_max;
      if (small && sweeps - s >= 2 && !fine) {
        launch_rb2d_2<T>(S.lc, L, c->kind, D.u[cur], g, D.u[1 - cur], om, order, mode, Cp, ec, oc);
        cur = 1 - cur;
        ++s;   // the second sweep of the pair
        continue;
      }
      if (small || (!sweep_tma<T>(S, L, D.u[cur], g, D.u[1 - cur], om, order, mode, Cp, ec, oc) &&
                    !launch_rb2d_march<T>(S.lc, L, c->kind, D.u[cur], g, D.u[1 - cur], om, order, mode, Cp, ec,
                                          oc)))
        launch_rb2d<T>(S.lc, L, c->kind, D.u[cur], g, D.u[1 - cur], om, order, mode, Cp, ec, oc);
      cur = 1 - cur;
    } else if (!line && kind == K_NINE) {
      // Gauss-Seidel on a Galerkin level: four colours, red (0,0), (1,1) then black (1,0), (0,1);
      // order 1 runs the exact reverse
      static const int seq[4][2] = {{0, 0}, {1, 1}, {1, 0}, {0, 1}};
      for (int q = 0; q < 4; ++q) {
        const int *cc = seq[order ? 3 - q : q];
        launch_gs9_colour<T>(S.lc, L, D.u[cur], g, om, cc[0], cc[1]);
      }
    } else if (!line) {
      int first = order;
      launch_rb_half<T>(S.lc, L, kind, D.u[cur], g, om, first);
      launch_rb_half<T>(S.lc, L, kind, D.u[cur], g, om, 1 - first);
    } else {
      // one line sweep in direction dir: line Jacobi out of place, or zebra (both colours) in place.
      // x lines up to 4096 unknowns: the x-line kernels (one CTA or one warp a line, partition + PCR);
      // y lines and longer x lines: launch_line (y-line kernels by length, else one thread a line)
      auto line_pass = [&](int dir, bool zebra) {
        bool fast = dir == 0 && !(c->P.flags & MG_FLAG_NO_FUSED_SWEEP) && L.n0 - 2 <= 4096;
        if (zebra) {
          for (int col = 0; col < 2; ++col) {
            int colour = col == 0 ? order : 1 - order;
            if (!(fast && launch_xline<T>(S.lc, L, c->kind, 1, colour, D.u[cur], g, D.u[cur], om)))
              launch_line<T>(S.lc, L, c->kind, dir, 1, colour, D.u[cur], g, D.u[cur], om, D.r, D.u[1 - cur], D.t);
          }
        } else {
          if (!(fast && launch_xline<T>(S.lc, L, c->kind, 0, 0, D.u[cur], g, D.u[1 - cur], om)))
            launch_line<T>(S.lc, L, c->kind, dir, 0, 0, D.u[cur], g, D.u[1 - cur], om, D.r, D.u[1 - cur], D.t);
          cur = 1 - cur;
        }
      };
      const int sm = c->P.smoother;
      if (sm == MG_ADI || sm == MG_GSADI) {
        // x lines then y lines; the transposed cycle (order 1) runs the composition reversed
        const int d0 = order ? 1 : 0;
        line_pass(d0, sm == MG_GSADI);
        line_pass(1 - d0, sm == MG_GSADI);
      } else {
        line_pass((sm == MG_LINE_X || sm == MG_ZEBRA_X) ? 0 : 1, sm == MG_ZEBRA_X || sm == MG_ZEBRA_Y);
      }
    }
    if (fine && odd_guard) {
      record_event(S);
      odd_guard = 0;
    }
  }
}

// u_1 = A_1^{-1} g: the dense inverse, or conjugate gradients to 1e-14 above the dense limit
template <typename T>
static void coarse_solve_into(mg_ctx *c, const Launch &lc, const T *g, T *u) {
  if (c->cg_mode)
    launch_coarse_cg<T>(lc, lev64(c, 1), c->kind, g, u, c->cgw, c->partials, c->cg_max_it, 1e-14, c->st + 4);
  else
    launch_coarse_apply<T>(lc, c->Ainv, c->cidx, c->nc, g, u);
}
template <typename T>
static void coarse_solve(Sched &S, const T *g) {
  NvtxRange nr("coarsest solve");
  mg_ctx *c = S.c;
  c->tracer.level = 1;
  LevData<T> &D = LevOf<T>::data(c, 1);
  coarse_solve_into<T>(c, S.lc, g, D.u[c->cur[1]]);
}

// Programs of the single-CTA coarse kernel: 0..3 run the whole cycle on the finest grid
// (when every grid fits in shared memory), 4..7 the coarse correction below lcut + 1.
static int prog_id_fine(int zero, int tr) { return zero * 2 + tr; }
static int prog_id_sub(int type, int tr) { return 4 + type * 2 + tr; }
static const int PROG_FMG = 8;   // nested iteration on levels 1..lcut

template <typename T>
static void launch_csk(Sched &S, int pid, const T *g_in, const T *u_in, T *u_out) {
  NvtxRange nr("coarse grids in one CTA");
  mg_ctx *c = S.c;
  c->tracer.level = c->lcut;
  launch_coarse_cycle<T>(S.lc, c->P.dim, c->kind, c->slev, c->prog + c->prog_off[pid], c->prog_len[pid], c->lcut,
                         g_in, u_in, u_out, c->Ainv, c->cidx_s, c->nc, (T)c->P.omega, (T)corr_weight(c),
                         c->csk_smem, c->P.smoother > MG_RBGS || adaptive_corr(c));
}

// Host-side builder of the coarse programs: mirrors smooth() and cycle() step by step,
// tracking which of the two u buffers of each level is current.
struct ProgBuilder {
  const mg_ctx *c;
  std::vector<int4> ops;
  int cur[MAXLEV + 1] = {0};
  explicit ProgBuilder(const mg_ctx *cc) : c(cc) {}
  void op(int code, int lev, int a, int b) { ops.push_back(make_int4(code, lev, a, b)); }
  // descriptor of `sweeps` red-black sweeps starting with colour `order` (CP_RB_HALF)
  static int rb_desc(int sweeps, int order, bool zero) { return order | (zero ? 2 : 0) | ((2 * sweeps - 1) << 2); }
  void smooth(int l, int sweeps, int order, bool zero) {
    int &cu = cur[l];
    int sm = c->P.smoother;
    if (sweeps <= 0) {
      if (zero) op(CP_ZERO_U, l, cu, 0);
      return;
    }
    if (sm == MG_JACOBI) {
      for (int s = 0; s < sweeps; ++s) {
        op(CP_JACOBI, l, (zero && s == 0) ? -1 : cu, 1 - cu);
        cu = 1 - cu;
      }
      return;
    }
    if (sm == MG_RBGS) {   // all 2 * sweeps half sweeps in one step
      op(CP_RB_HALF, l, rb_desc(sweeps, order, zero), cu);
      return;
    }
    if (zero) op(CP_ZERO_U, l, cu, 0);
    auto pass = [&](int dir, bool zebra) {
      if (zebra) {
        int bufs = cu | (cu << 4) | ((1 - cu) << 8);
        op(CP_LINE, l, dir | 2 | (order << 2), bufs);
        op(CP_LINE, l, dir | 2 | ((1 - order) << 2), bufs);
      } else {
        op(CP_LINE, l, dir, cu | ((1 - cu) << 4) | ((1 - cu) << 8));
        cu = 1 - cu;
      }
    };
    for (int s = 0; s < sweeps; ++s) {
      if (sm == MG_ADI || sm == MG_GSADI) {   // x then y lines (reversed in the transposed cycle)
        const int d0 = order ? 1 : 0;
        pass(d0, sm == MG_GSADI);
        pass(1 - d0, sm == MG_GSADI);
      } else {
        pass((sm == MG_LINE_X || sm == MG_ZEBRA_X) ? 0 : 1, sm == MG_ZEBRA_X || sm == MG_ZEBRA_Y);
      }
    }
  }
  void cycle(int l, int type, int tr, bool zero) {
    if (l == 1) {
      op(CP_COARSE, 1, cur[1], 0);
      return;
    }
    int npre = tr ? c->P.nu2 : c->P.nu1, npost = tr ? c->P.nu1 : c->P.nu2, order = tr ? 1 : 0;
    smooth(l, npre, order, zero);
    op(CP_DEFECT, l, cur[l], 1);   // defect and its restriction in one step
    cur[l - 1] = 0;
    if (type == 0) {
      cycle(l - 1, tr ? 1 : 0, tr, true);
      if (l - 1 > 1) cycle(l - 1, tr ? 0 : 1, tr, false);
    } else {
      cycle(l - 1, 1, tr, true);
    }
    if (adaptive_corr(c)) {   // the correction with its own weight
      op(CP_ADAPT, l, cur[l], cur[l - 1]);
      smooth(l, npost, order, false);
    } else if (c->P.smoother == MG_RBGS && npost > 0) {   // correction and post-smoothing in one step
      op(CP_PROLONG, l, cur[l], cur[l - 1] | ((rb_desc(npost, order, false) + 1) << 1));
    } else {
      op(CP_PROLONG, l, cur[l], cur[l - 1]);
      smooth(l, npost, order, false);
    }
  }
  // coarse correction at level lc requested by a type-`type` cycle at lc + 1
  void sub(int lc, int type, int tr) {
    op(CP_LOAD_G, lc, 0, 0);
    cur[lc] = 0;
    if (type == 0) {
      cycle(lc, tr ? 1 : 0, tr, true);
      if (lc > 1) cycle(lc, tr ? 0 : 1, tr, false);
    } else {
      cycle(lc, 1, tr, true);
    }
    op(CP_STORE_U, lc, cur[lc], 0);
  }
  // nested iteration on levels 1..lc: g_lc loaded and restricted down to level 1, solved
  // there, then on each finer level the interpolated solution improved by one F-cycle
  void fmg(int lc) {
    op(CP_LOAD_G, lc, 0, 0);
    for (int l = lc; l > 1; --l) op(CP_RESTRICT, l, 1, 0);
    cur[1] = 0;
    op(CP_COARSE, 1, 0, 0);
    for (int l = 2; l <= lc; ++l) {
      cur[l] = 0;
      op(CP_INTERP, l, 0, cur[l - 1]);
      cycle(l, 0, 0, false);
    }
    op(CP_STORE_U, lc, cur[lc], 0);
  }
  // one F-cycle on the finest grid L (= lc)
  void fine(int L, int zero, int tr) {
    op(CP_LOAD_G, L, 0, 0);
    if (!zero) op(CP_LOAD_U, L, 0, 0);
    cur[L] = 0;
    cycle(L, 0, tr, zero != 0);
    op(CP_STORE_U, L, cur[L], 0);
  }
};

// Adaptive correction weight at level l (Wallis 2008, section "Multigrid": omega_l that
// minimises the energy norm of the error): P e into r_l, omega = (g - A u, P e) / (A P e, P e),
// then the coarse correction e scaled by omega in place, so that the correction added next
// (with weight 1) is omega P e.
template <typename T>
static void emit_adapt(Sched &S, int l, const T *g) {
  mg_ctx *c = S.c;
  LevData<T> &D = LevOf<T>::data(c, l), &Dc = LevOf<T>::data(c, l - 1);
  Lev<T> L = LevOf<T>::get(c, l), Lc = LevOf<T>::get(c, l - 1);
  T *e = Dc.u[c->cur[l - 1]];
  launch_interp<T>(S.lc, L, Lc, e, D.r);
  launch_corr_weight<T>(S.lc, L, c->kind, D.u[c->cur[l]], g, D.r, c->partials, norm_parts_count(), c->cnt,
                        c->scal + 8);
  launch_scale_by<T>(S.lc, e, (long long)c->geo[l - 1].count, c->scal + 8);
}

// The descending half of a visit of level l >= 2: the pre-smoothing sweeps on (u = current
// buffer of level l, g), then g_{l-1} = R (g - A u) into the coarse level's g.  Small 2-D
// red-black grids run both sweeps, the defect and the restriction in one pass.
template <typename T>
static void descend(Sched &S, int l, const T *g, int transposed, bool zero_start) {
  NvtxRange nr("pre-smoothing, defect, restriction", l);
  mg_ctx *c = S.c;
  c->tracer.level = l;
  LevData<T> &D = LevOf<T>::data(c, l);
  LevData<T> &Dc = LevOf<T>::data(c, l - 1);
  Lev<T> L = LevOf<T>::get(c, l), Lc = LevOf<T>::get(c, l - 1);
  int npre = transposed ? c->P.nu2 : c->P.nu1;
  int order = transposed ? 1 : 0;
  const long long tile_max = c->P.tile_nodes == 0 ? 1050625 : c->P.tile_nodes < 0 ? -1 : c->P.tile_nodes;
  const bool fused2d = c->P.dim == 2 && !(c->P.flags & MG_FLAG_NO_FUSED_SWEEP) && lev_kind(c, l) != K_NINE;
  if (fused2d && c->P.smoother == MG_RBGS && npre == 2 && tile_max >= 0 && (long long)L.n0 * L.n1 <= tile_max &&
      !(S.timing && l == c->L)) {
    // small grid: both pre-smoothing sweeps, the defect and the restriction in one pass
    int &cu = c->cur[l];
    launch_rb2d_2_dr<T>(S.lc, L, Lc, c->kind, D.u[cu], g, D.u[1 - cu], (T)c->P.omega, order, zero_start ? 1 : 0,
                        Dc.g);
    cu = 1 - cu;
  } else if (fused2d) {
    smooth<T>(S, l, g, npre, order, zero_start);
    if (!defect_restrict_tma<T>(S, L, Lc, D.u[c->cur[l]], g, Dc.g))
      launch_defect_restrict2d<T>(S.lc, L, Lc, c->kind, D.u[c->cur[l]], g, Dc.g);
  } else {
    smooth<T>(S, l, g, npre, order, zero_start);
    launch_defect<T>(S.lc, L, lev_kind(c, l), D.u[c->cur[l]], g, D.r);
    launch_restrict<T>(S.lc, L, Lc, D.r, Dc.g);
  }
}

// The ascending half of a visit of level l >= 2: the coarse correction (current buffer of
// level l-1) added with omega_l (energy-optimal with MG_FLAG_ADAPTIVE_CORR), then the
// post-smoothing sweeps; the correction is folded into the first fused red-black sweep.
template <typename T>
static void ascend(Sched &S, int l, const T *g, int transposed) {
  NvtxRange nr("correction, post-smoothing", l);
  mg_ctx *c = S.c;
  c->tracer.level = l;
  LevData<T> &Dc = LevOf<T>::data(c, l - 1);
  Lev<T> Lc = LevOf<T>::get(c, l - 1);
  int npost = transposed ? c->P.nu1 : c->P.nu2;
  int order = transposed ? 1 : 0;
  if (adaptive_corr(c)) emit_adapt<T>(S, l, g);
  smooth<T>(S, l, g, npost, order, false, &Lc, Dc.u[c->cur[l - 1]]);
}

// One cycle at level l on (u = current buffer of level l, g).  type 0 = F, 1 = V.
template <typename T>
static void cycle(Sched &S, int l, const T *g, int type, int transposed, bool zero_start) {
  mg_ctx *c = S.c;
  if (l == 1) {
    coarse_solve<T>(S, g);
    return;
  }
  LevData<T> &Dc = LevOf<T>::data(c, l - 1);
  descend<T>(S, l, g, transposed, zero_start);
  c->cur[l - 1] = 0;
  if (l - 1 == c->lcut) {
    // the whole coarse correction below level l in one single-CTA launch
    launch_csk<T>(S, prog_id_sub(type, transposed), Dc.g, nullptr, Dc.u[0]);
  } else if (type == 0) {
    int first = transposed ? 1 : 0, second = transposed ? 0 : 1;
    cycle<T>(S, l - 1, Dc.g, first, transposed, true);
    if (l - 1 > 1) cycle<T>(S, l - 1, Dc.g, second, transposed, false);
  } else {
    cycle<T>(S, l - 1, Dc.g, 1, transposed, true);
  }
  ascend<T>(S, l, g, transposed);
}

// Ensure the finest level's current buffer is buffer 0 at the end of a cycle.
template <typename T>
static void finest_to_zero(Sched &S) {
  mg_ctx *c = S.c;
  int L = c->L;
  if (c->cur[L] != 0) {
    LevData<T> &D = LevOf<T>::data(c, L);
    cudaMemcpyAsync(D.u[0], D.u[1], sizeof(T) * (size_t)c->geo[L].count, cudaMemcpyDeviceToDevice, S.lc.s);
    c->cur[L] = 0;
  }
}

// Nested iteration (Wallis 2008, section "Start-Vector Choice") on the levels of precision T:
// g of the finest level holds the right-hand side (zero on the boundary); it is restricted
// level by level into g of every coarser level, the coarsest level is solved exactly, and on
// each finer level l the interpolated coarse solution (u_l = P u_{l-1}) is improved by one
// F-cycle with g_l.  The cycle at level l overwrites g only below l, so each level's
// restricted right-hand side is still in place when its turn comes.  Levels 1..lcut run as
// one single-CTA launch.  Afterwards buffer 0 of the finest level holds the start vector.
template <typename T>
static void emit_fmg(Sched &S) {
  mg_ctx *c = S.c;
  const int L = c->L, lo = c->lcut >= 2 ? c->lcut : 1;
  for (int l = L; l > lo; --l)
    launch_restrict<T>(S.lc, LevOf<T>::get(c, l), LevOf<T>::get(c, l - 1), LevOf<T>::data(c, l).g,
                       LevOf<T>::data(c, l - 1).g);
  for (int l = 1; l <= lo; ++l) c->cur[l] = 0;
  if (lo == 1) coarse_solve<T>(S, LevOf<T>::data(c, 1).g);
  else launch_csk<T>(S, PROG_FMG, LevOf<T>::data(c, lo).g, nullptr, LevOf<T>::data(c, lo).u[0]);
  for (int l = lo + 1; l <= L; ++l) {
    LevData<T> &D = LevOf<T>::data(c, l), &Dc = LevOf<T>::data(c, l - 1);
    cudaMemsetAsync(D.u[0], 0, sizeof(T) * (size_t)c->geo[l].count, S.lc.s);
    launch_prolong_add<T>(S.lc, LevOf<T>::get(c, l), LevOf<T>::get(c, l - 1), Dc.u[c->cur[l - 1]], D.u[0], T(1));
    c->cur[l] = 0;
    cycle<T>(S, l, D.g, 0, 0, false);
  }
  finest_to_zero<T>(S);
}

// MG_FLAG_FMG_START: the start vector of a solve from nested iteration, in place of the
// caller's x (the packed b already sits in the finest-level buffers).  FP64 contexts run it
// on the FP64 levels; MG_MIXED contexts run it on the FP32 levels from (float) b and widen
// the result into x.  The operator is symmetric, so an adjoint solve uses the same start.
static void emit_fmg_start(Sched &S) {
  mg_ctx *c = S.c;
  const int L = c->L;
  if (c->mixed) {
    Lev<double> F64 = lev64(c, L);
    cudaMemsetAsync(c->x64, 0, sizeof(double) * (size_t)c->geo[L].count, S.lc.s);
    // g32 = (float)(b - A 0) = (float) b
    launch_defect64_to32(S.lc, F64, c->kind, c->x64, c->b64, c->d32[L].g, c->partials, norm_parts_count(),
                         c->scal + 1);
    emit_fmg<float>(S);
    launch_ir_update(S.lc, F64, c->x64, c->d32[L].u[0]);
  } else {
    emit_fmg<double>(S);
  }
}

// FP64 form: one F-cycle on the finest level followed by the residual check.
static void emit_fp64_cycle(Sched &S, int transposed) {
  NvtxRange nr("F-cycle");
  mg_ctx *c = S.c;
  int L = c->L;
  c->cur[L] = 0;
  if (c->lcut == L) launch_csk<double>(S, prog_id_fine(0, transposed), c->d64[L].g, c->d64[L].u[0], c->d64[L].u[0]);
  else cycle<double>(S, L, c->d64[L].g, 0, transposed, false);
  finest_to_zero<double>(S);
  c->tracer.level = L;
  launch_defect_norm<double>(S.lc, lev64(c, L), c->kind, c->d64[L].u[0], c->d64[L].g, c->partials,
                             norm_parts_count(), c->scal + 1);
  if (S.loop) launch_step_end(S.lc, S.loop_h, c->scal + 1, c->scal + 0, c->hist, c->st, c->scal + 4,
                              c->P.max_cycles, 0);
  else launch_relres(S.lc, c->scal + 1, c->scal + 0, nullptr, 0, c->scal + 2);
}

// Mixed form: FP32 inner F-cycles on r32 from zero, FP64 update, FP64 defect and check.
static void emit_mixed_step(Sched &S, int transposed) {
  NvtxRange nr("refinement step: FP32 F-cycle, update, outer defect");
  mg_ctx *c = S.c;
  int L = c->L;
  for (int q = 0; q < c->P.inner_cycles; ++q) {
    c->cur[L] = 0;
    if (c->lcut == L)
      launch_csk<float>(S, prog_id_fine(q == 0 ? 1 : 0, transposed), c->d32[L].g, c->d32[L].u[0], c->d32[L].u[0]);
    else
      cycle<float>(S, L, c->d32[L].g, 0, transposed, q == 0);
    finest_to_zero<float>(S);
  }
  c->tracer.level = L;
  // float-float contexts: the update x += c fused into the outer defect (double-buffered iterate);
  // otherwise the update, then the FP64 defect
  const bool ff = c->ff && launch_defect_ff(S.lc, lev64(c, L), c->kind, c->x64, c->x64b, c->b64, c->d32[L].g,
                                            c->partials, norm_parts_count(), c->scal + 1, c->scal + 5, c->st + 6,
                                            c->d32[L].u[0], c->st + 7);
  if (!ff) {
    launch_ir_update(S.lc, lev64(c, L), c->x64, c->d32[L].u[0]);
    launch_defect64_to32(S.lc, lev64(c, L), c->kind, c->x64, c->b64, c->d32[L].g, c->partials, norm_parts_count(),
                         c->scal + 1);
  }
  if (S.loop) launch_step_end(S.lc, S.loop_h, c->scal + 1, c->scal + 0, c->hist, c->st, c->scal + 4,
                              c->P.max_cycles, 0, ff ? c->scal + 5 : nullptr, kFFErr, kFFSwitch);
  else launch_relres(S.lc, c->scal + 1, c->scal + 0, nullptr, 0, c->scal + 2);
}

// The start vector's defect of a mixed solve, into the FP32 right-hand side of the first
// refinement step: in float-float arithmetic where the loop's defects are (with its error
// estimate, which the stopping test uses as in the loop: a start that passes it is confirmed by
// the FP64 defect after the loop), else in FP64.  Returns whether the float-float form ran.
static bool start_defect(mg_ctx *c, const Launch &lc) {
  const int L = c->L;
  const Lev<double> F64 = lev64(c, L);
  if (c->ff && launch_defect_ff(lc, F64, c->kind, c->x64, nullptr, c->b64, c->d32[L].g, c->partials,
                                norm_parts_count(), c->scal + 1, c->scal + 5, c->st + 6, nullptr, nullptr))
    return true;
  launch_defect64_to32(lc, F64, c->kind, c->x64, c->b64, c->d32[L].g, c->partials, norm_parts_count(), c->scal + 1);
  return false;
}

// Initial check of a device-side solve: ||b||^2, the defect of the start vector, and the
// loop condition (the packed b and x already sit in the finest-level buffers).
static void emit_solve_init(Sched &S) {
  mg_ctx *c = S.c;
  int L = c->L;
  Lev<double> F64 = lev64(c, L);
  if (c->P.flags & MG_FLAG_FMG_START) emit_fmg_start(S);
  if (c->mixed) {
    launch_norm_parts<double>(S.lc, F64, c->b64, c->partials, norm_parts_count(), c->scal + 0);
    const bool ff = start_defect(c, S.lc);
    launch_step_end(S.lc, S.loop_h, c->scal + 1, c->scal + 0, c->hist, c->st, c->scal + 4, c->P.max_cycles, 1,
                    ff ? c->scal + 5 : nullptr, kFFErr, kFFSwitch);
    return;
  }
  launch_norm_parts<double>(S.lc, F64, c->d64[L].g, c->partials, norm_parts_count(), c->scal + 0);
  launch_defect_norm<double>(S.lc, F64, c->kind, c->d64[L].u[0], c->d64[L].g, c->partials, norm_parts_count(),
                             c->scal + 1);
  launch_step_end(S.lc, S.loop_h, c->scal + 1, c->scal + 0, c->hist, c->st, c->scal + 4, c->P.max_cycles, 1);
}

// Kernel-to-kernel edges of a captured graph become programmatic dependencies: the next kernel's
// launch may overlap the end of the previous one, whose completion and writes it then waits for
// (MG_PDL_WAIT, the first statement of every kernel here).  An edge the driver refuses to convert
// keeps its ordinary form.  MG_FLAG_NO_PDL leaves every edge ordinary.
static void make_programmatic(const mg_ctx *c, cudaGraph_t g) {
  if (c->P.flags & MG_FLAG_NO_PDL) return;
  size_t n = 0;
  if (cudaGraphGetEdges(g, nullptr, nullptr, nullptr, &n) != cudaSuccess || n == 0) {
    cudaGetLastError();
    return;
  }
  std::vector<cudaGraphNode_t> from(n), to(n);
  std::vector<cudaGraphEdgeData> ed(n);
  if (cudaGraphGetEdges(g, from.data(), to.data(), ed.data(), &n) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  for (size_t q = 0; q < n; ++q) {
    cudaGraphNodeType tf, tt;
    if (cudaGraphNodeGetType(from[q], &tf) != cudaSuccess || cudaGraphNodeGetType(to[q], &tt) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (tf != cudaGraphNodeTypeKernel || tt != cudaGraphNodeTypeKernel || ed[q].type != cudaGraphDependencyTypeDefault ||
        ed[q].from_port != cudaGraphKernelNodePortDefault)
      continue;
    cudaGraphEdgeData pe;
    memset(&pe, 0, sizeof(pe));
    pe.from_port = cudaGraphKernelNodePortProgrammatic;
    pe.type = cudaGraphDependencyTypeProgrammatic;
    if (cudaGraphRemoveDependencies(g, &from[q], &to[q], &ed[q], 1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (cudaGraphAddDependencies(g, &from[q], &to[q], &pe, 1) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphAddDependencies(g, &from[q], &to[q], &ed[q], 1);   // back to the ordinary edge
      cudaGetLastError();
    }
  }
}

// Into the graph that stream s is capturing: the initial check, then a WHILE node whose
// body is one cycle (FP64) or refinement step (MG_MIXED) ending in the convergence test,
// which sets the loop condition on the device.  The body is captured on c->cap2.  The
// kernel counts of the initial part and of one body go to init_k / body_k.
static cudaError_t capture_loop(mg_ctx *c, cudaStream_t s, int transposed, long long *init_k, long long *body_k) {
  cudaGraph_t graph = nullptr;
  cudaGraphConditionalHandle h;
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t *deps = nullptr;
  size_t ndeps = 0;
  long long before = c->launches;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &graph, &deps, nullptr, &ndeps);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, graph, 0, 0);
  if (e == cudaSuccess) {
    Sched S{c, Launch{s, &c->launches}, false};
    S.loop = true;
    S.loop_h = h;
    emit_solve_init(S);
    e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &graph, &deps, nullptr, &ndeps);
  }
  cudaGraphNode_t cnode;
  cudaGraphNodeParams cp = {};
  if (e == cudaSuccess) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&cnode, graph, deps, nullptr, ndeps, &cp);
  }
  if (e == cudaSuccess)
    e = cudaStreamUpdateCaptureDependencies(s, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e == cudaSuccess) {
    *init_k = c->launches - before;
    e = cudaStreamBeginCaptureToGraph(c->cap2, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      long long b0 = c->launches;
      Sched S{c, Launch{c->cap2, &c->launches}, false};
      S.loop = true;
      S.loop_h = h;
      if (c->mixed) emit_mixed_step(S, transposed);
      else emit_fp64_cycle(S, transposed);
      *body_k = c->launches - b0;
      cudaGraph_t bout = cp.conditional.phGraph_out[0];
      e = cudaStreamEndCapture(c->cap2, &bout);
      if (e == cudaSuccess) make_programmatic(c, cp.conditional.phGraph_out[0]);
    }
  }
  if (e == cudaSuccess && c->mixed && c->ff) {
    // the loop stopped on the float-float defect: the iterate back into x64, and the FP64
    // residual of the result, reported
    long long f0 = c->launches;
    Launch lc{s, &c->launches};
    launch_x_settle(lc, c->x64, c->x64b, (long long)c->geo[c->L].count, c->st + 7);
    launch_defect64_to32(lc, lev64(c, c->L), c->kind, c->x64, c->b64, c->d32[c->L].g, c->partials,
                         norm_parts_count(), c->scal + 1);
    launch_final_check(lc, c->scal + 1, c->scal + 0, c->hist, c->st, c->scal + 4);
    e = cudaGetLastError();
    *init_k += c->launches - f0;
  }
  c->launches = before;
  return e;
}

// The whole solve as one graph (capture_loop on the context's own capture stream).  One
// launch and one synchronisation per solve.
static mg_status build_loop_graph(mg_ctx *c, int transposed) {
  if (c->lexec[transposed]) return MG_OK;
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = capture_loop(c, c->cap, transposed, &c->loop_init_kernels[transposed],
                               &c->loop_body_kernels[transposed]);
  cudaError_t e2 = cudaStreamEndCapture(c->cap, &graph);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) make_programmatic(c, graph);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&c->lexec[transposed], graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    c->err = std::string("solve-loop graph: ") + cudaGetErrorString(e);
    cudaGetLastError();
    c->lexec[transposed] = nullptr;
    return MG_ECUDA;
  }
  return MG_OK;
}

// MG_FLAG_TRACE: the marks of one step schedule (direction t) start with an unlabelled mark;
// every launch through lc then adds one
static void trace_begin(mg_ctx *c, Launch &lc, int t, bool capture) {
  if (!(c->P.flags & MG_FLAG_TRACE)) return;
  Tracer &tr = c->tracer;
  tr.capture = capture;
  tr.ev = c->tr_ev.data() + t * kTraceMarks;
  tr.label = c->tr_label.data() + t * kTraceMarks;
  tr.lev = c->tr_lev.data() + t * kTraceMarks;
  tr.cap = kTraceMarks;
  tr.n = 0;
  tr.level = c->L;
  tr.mark(lc.s, nullptr);
  lc.tr = &tr;
}
static void trace_end(mg_ctx *c, int t) {
  if (c->P.flags & MG_FLAG_TRACE) c->tr_n[t] = c->tracer.n;
}
// after the step ran (stream synchronised): the time between consecutive marks goes to the kernel
// that ends at the later one
static void trace_harvest(mg_ctx *c, int t) {
  if (!(c->P.flags & MG_FLAG_TRACE)) return;
  const int b = t * kTraceMarks;
  ++c->tr_steps;
  for (int i = 1; i < c->tr_n[t]; ++i) {
    const char *lab = c->tr_label[b + i];
    float ms = 0.f;
    if (!lab) continue;
    if (cudaEventElapsedTime(&ms, c->tr_ev[b + i - 1], c->tr_ev[b + i]) != cudaSuccess) {
      ++c->tr_unread;
      continue;
    }
    auto &e = c->tr_sum[{std::string(lab), c->tr_lev[b + i]}];
    e.first += 1;
    e.second += ms;
  }
  cudaGetLastError();
}

static mg_status build_graph(mg_ctx *c, int transposed) {
  if (c->gexec[transposed]) return MG_OK;
  bool timing = (c->P.flags & MG_FLAG_TIMING) != 0;
  c->ev_graph_n[transposed] = 0;
  Sched S{c, Launch{c->cap, &c->launches}, timing, 2048 * (1 + transposed), &c->ev_graph_n[transposed]};
  long long before = c->launches;
  CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
  trace_begin(c, S.lc, transposed, true);
  if (c->mixed) emit_mixed_step(S, transposed);
  else emit_fp64_cycle(S, transposed);
  trace_end(c, transposed);
  cudaGraph_t graph;
  cudaError_t e = cudaStreamEndCapture(c->cap, &graph);
  if (e != cudaSuccess) {
    c->err = std::string("graph capture: ") + cudaGetErrorString(e);
    cudaGetLastError();
    return MG_ECUDA;
  }
  c->graph_kernels[transposed] = c->launches - before;
  c->launches = before;
  make_programmatic(c, graph);
  e = cudaGraphInstantiate(&c->gexec[transposed], graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    c->err = std::string("graph instantiate: ") + cudaGetErrorString(e);
    c->gexec[transposed] = nullptr;
    return MG_ECUDA;
  }
  return MG_OK;
}

// ---------------------------------------------------------------------------------------
// set-up
// ---------------------------------------------------------------------------------------
static mg_status setup_levels(mg_ctx *c) {
  Launch lc{c->stream, &c->launches};
  const mg_params &P = c->P;
  int L = c->L;
  CK(cudaMemsetAsync(c->st, 0, sizeof(int) * 8, c->stream));   // loop state and the device-wait flag
  CK(cudaMemsetAsync(c->oob, 0, sizeof(unsigned) * 4, c->stream));
  CK(cudaMemsetAsync(c->cnt, 0, sizeof(unsigned) * 8, c->stream));
  // geometry constants per level
  for (int l = L; l >= 1; --l) {
    LevGeom &g = c->geo[l];
    double scale = std::ldexp(1.0, -2 * (L - l));   // CONST weights: 1/4 per coarsening
    for (int d = 0; d < 3; ++d) g.c[d] = c->K.c[d] * scale;
    if (P.dim == 2) g.c[2] = 0.0;
    g.d = 2.0 * (g.c[0] + g.c[1] + g.c[2]);
    g.dinv = 1.0 / g.d;
    double f = (P.dim == 2) ? 0.5 : 0.25;
    g.ax = f / (g.h[0] * g.h[0]);
    g.ay = f / (g.h[1] * g.h[1]);
    g.az = (P.dim == 3) ? f / (g.h[2] * g.h[2]) : 0.0;
  }
  // coefficient arrays
  if (c->kind == K_SEP) {
    LevData<double> &F = c->d64[L];
    int n0 = c->geo[L].n[0];
    CK(cudaMemsetAsync(F.sx, 0, sizeof(double) * n0, c->stream));
    CK(cudaMemsetAsync(F.sz, 0, sizeof(double) * n0, c->stream));
    CK(cudaMemcpyAsync(F.sx, c->K.sx, sizeof(double) * (n0 - 1), cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(F.sy, c->K.sy, sizeof(double) * n0, cudaMemcpyDeviceToDevice, c->stream));
    if (P.dim == 3) CK(cudaMemcpyAsync(F.sz, c->K.sz, sizeof(double) * n0, cudaMemcpyDeviceToDevice, c->stream));
    for (int l = L; l > 1; --l) {
      LevData<double> &A = c->d64[l], &B = c->d64[l - 1];
      launch_coarsen_sep(lc, A.sx, A.sy, A.sz, c->geo[l].n[0], B.sx, B.sy, B.sz, c->geo[l - 1].n[0]);
    }
    for (int l = L; l >= 1; --l) {
      LevData<double> &A = c->d64[l];
      launch_sep_dinv(lc, A.sx, A.sy, A.sz, c->geo[l].n[0], P.dim, A.sdinv);
    }
  } else if (c->kind == K_CELL) {
    for (int l = L; l >= 1; --l) CK(cudaMemsetAsync(c->d64[l].k, 0, sizeof(double) * c->geo[l].count, c->stream));
    if (c->swap) launch_cell_pack_swapped(lc, lev64(c, L), c->K.k, c->d64[L].k);
    else launch_cell_pack(lc, lev64(c, L), c->K.k, c->d64[L].k);
    for (int l = L; l > 1; --l) launch_coarsen_cell(lc, lev64(c, l), lev64(c, l - 1), c->d64[l].k, c->d64[l - 1].k);
    for (int l = L; l >= 1; --l) {
      CK(cudaMemsetAsync(c->d64[l].ndinv, 0, sizeof(double) * c->geo[l].count, c->stream));
      launch_cell_dinv(lc, lev64(c, l), c->d64[l].ndinv);
    }
  } else if (c->kind == K_EDGE) {
    for (int l = L; l >= 1; --l) {
      LevData<double> &A = c->d64[l];
      size_t bytes = sizeof(double) * (size_t)c->geo[l].count;
      for (double *p : {A.ex, A.ey, A.ez, A.ndinv})
        if (p) CK(cudaMemsetAsync(p, 0, bytes, c->stream));
    }
    Lev<double> F = lev64(c, L);
    LevData<double> &A = c->d64[L];
    launch_pack<double>(lc, F, c->K.ex, A.ex, 0);
    launch_pack<double>(lc, F, c->K.ey, A.ey, 0);
    if (P.dim == 3) launch_pack<double>(lc, F, c->K.ez, A.ez, 0);
    for (int l = L; l > 1; --l) {
      LevData<double> &Fd = c->d64[l], &Cd = c->d64[l - 1];
      launch_coarsen_edge(lc, lev64(c, l), lev64(c, l - 1), Fd.ex, Fd.ey, Fd.ez, Cd.ex, Cd.ey, Cd.ez);
    }
    for (int l = L; l >= 1; --l) launch_edge_dinv(lc, lev64(c, l), c->d64[l].ndinv);
  }
  // Galerkin: every coarser operator is R A P of the next finer one (9-point stencils)
  if (c->galerkin)
    for (int l = L - 1; l >= 1; --l) {
      LevData<double> &Cd = c->d64[l];
      launch_rap(lc, lev64(c, l + 1), lev_kind(c, l + 1), lev64(c, l), Cd.dg, Cd.ex, Cd.ey, Cd.ez, Cd.enw, Cd.ndinv);
    }
  // work vectors start at zero (Dirichlet nodes stay zero for good)
  for (int l = L; l >= 1; --l) {
    size_t cnt = (size_t)c->geo[l].count;
    if (!c->mixed) {
      LevData<double> &D = c->d64[l];
      for (double *p : {D.u[0], D.u[1], D.g, D.r}) CK(cudaMemsetAsync(p, 0, sizeof(double) * cnt, c->stream));
    } else {
      LevData<float> &D = c->d32[l];
      for (float *p : {D.u[0], D.u[1], D.g, D.r}) CK(cudaMemsetAsync(p, 0, sizeof(float) * cnt, c->stream));
      if (c->kind == K_SEP) {
        size_t n0 = (size_t)c->geo[l].n[0];
        launch_to_float(lc, c->d64[l].sx, D.sx, (long long)n0);
        launch_to_float(lc, c->d64[l].sy, D.sy, (long long)n0);
        launch_to_float(lc, c->d64[l].sz, D.sz, (long long)n0);
        launch_to_float(lc, c->d64[l].sdinv, D.sdinv, (long long)n0);
      } else if (c->kind == K_CELL) {
        launch_to_float(lc, c->d64[l].k, D.k, (long long)cnt);
        launch_to_float(lc, c->d64[l].ndinv, D.ndinv, (long long)cnt);
      } else if (c->kind == K_EDGE) {
        launch_to_float(lc, c->d64[l].ex, D.ex, (long long)cnt);
        launch_to_float(lc, c->d64[l].ey, D.ey, (long long)cnt);
        if (P.dim == 3) launch_to_float(lc, c->d64[l].ez, D.ez, (long long)cnt);
        launch_to_float(lc, c->d64[l].ndinv, D.ndinv, (long long)cnt);
      }
      if (lev_kind(c, l) == K_NINE) {
        const LevData<double> &S = c->d64[l];
        for (int q = 0; q < 6; ++q) {
          const double *src[6] = {S.dg, S.ex, S.ey, S.ez, S.enw, S.ndinv};
          float *dst[6] = {D.dg, D.ex, D.ey, D.ez, D.enw, D.ndinv};
          launch_to_float(lc, src[q], dst[q], (long long)cnt);
        }
      }
    }
  }
  if (c->mixed) {
    size_t fine = (size_t)c->geo[L].count;
    for (double *p : {c->x64, c->b64, c->d64[L].u[0], c->d64[L].g, c->d64[L].r})
      CK(cudaMemsetAsync(p, 0, sizeof(double) * fine, c->stream));
    if (c->x64b) CK(cudaMemsetAsync(c->x64b, 0, sizeof(double) * fine, c->stream));   // Dirichlet nodes stay 0
  }
  // coarsest grid: unknown index maps (built on the host: O(nodes of the coarsest grid))
  {
    const LevGeom &g = c->geo[1];
    std::vector<long long> cidx;
    std::vector<int> cmap((size_t)g.count, -1);
    int kz0 = P.dim == 3 ? 1 : 0, kz1 = P.dim == 3 ? g.n[2] - 2 : 0;
    int j0 = P.periodic_y ? 0 : 1, j1 = P.periodic_y ? g.n[1] - 1 : g.n[1] - 2;
    for (int k = kz0; k <= kz1; ++k)
      for (int j = j0; j <= j1; ++j)
        for (int i = 1; i <= g.n[0] - 2; ++i) {
          long long p = (long long)k * g.plane + (long long)j * g.pitch + i;
          cmap[(size_t)p] = (int)cidx.size();
          cidx.push_back(p);
        }
    c->nc = (int)cidx.size();
    if (c->nc > 0) {
      CK(cudaMemcpyAsync(c->cidx, cidx.data(), sizeof(long long) * cidx.size(), cudaMemcpyHostToDevice, c->stream));
      CK(cudaMemcpyAsync(c->cmap, cmap.data(), sizeof(int) * cmap.size(), cudaMemcpyHostToDevice, c->stream));
      if (c->cg_mode) {
        CK(cudaMemsetAsync(c->cgw, 0, sizeof(double) * 4 * (size_t)c->geo[1].count, c->stream));
      } else {
        CK(cudaMemsetAsync(c->Ainv, 0, sizeof(double) * (size_t)c->nc * c->nc, c->stream));
        launch_assemble_dense<double>(lc, lev64(c, 1), lev_kind(c, 1), c->cidx, c->cmap, c->nc, c->Ainv);
        for (int k = 0; k < c->nc; ++k) launch_gj_step(lc, c->Ainv, c->gjcol, c->nc, k);
      }
    }
    CK(cudaStreamSynchronize(c->stream));   // host vectors above go out of scope
  }
  // single-CTA coarse kernel: level views, programs, coarsest indices in the compact layout
  if (c->lcut) {
    std::vector<char> tab((size_t)(MAXLEV + 1) * 512, 0);
    long long gp[MAXLEV + 1], gpl[MAXLEV + 1];
    for (int l = 1; l <= c->lcut; ++l) {
      gp[l] = c->geo[l].pitch;
      gpl[l] = c->geo[l].plane;
    }
    if (c->mixed) {
      std::vector<Lev<float>> lv(MAXLEV + 1);
      for (int l = 1; l <= c->lcut; ++l) lv[l] = lev32(c, l);
      c->csk_smem = coarse_fill_levels<float>(tab.data(), c->lcut, lv.data(), gp, gpl, c->kind, line_smoother(P));
    } else {
      std::vector<Lev<double>> lv(MAXLEV + 1);
      for (int l = 1; l <= c->lcut; ++l) lv[l] = lev64(c, l);
      c->csk_smem = coarse_fill_levels<double>(tab.data(), c->lcut, lv.data(), gp, gpl, c->kind, line_smoother(P));
    }
    std::vector<int4> all;
    for (int pid = 0; pid < 9; ++pid) {
      ProgBuilder pb(c);
      if (pid == PROG_FMG) {
        if (c->lcut < 2) continue;
        pb.fmg(c->lcut);
      } else if (pid < 4) {
        if (c->lcut != L) continue;
        pb.fine(L, pid / 2, pid % 2);
      } else {
        if (c->lcut == L) continue;
        pb.sub(c->lcut, (pid - 4) / 2, (pid - 4) % 2);
      }
      c->prog_off[pid] = (int)all.size();
      c->prog_len[pid] = (int)pb.ops.size();
      all.insert(all.end(), pb.ops.begin(), pb.ops.end());
    }
    c->prog_used = (int)all.size();
    if (all.size() > 32768) {
      c->err = "coarse program too long";
      return MG_EINVAL;
    }
    const LevGeom &g1 = c->geo[1];
    std::vector<long long> cs;
    int kz0 = P.dim == 3 ? 1 : 0, kz1 = P.dim == 3 ? g1.n[2] - 2 : 0;
    int j0 = P.periodic_y ? 0 : 1, j1 = P.periodic_y ? g1.n[1] - 1 : g1.n[1] - 2;
    for (int k = kz0; k <= kz1; ++k)
      for (int j = j0; j <= j1; ++j)
        for (int i = 1; i <= g1.n[0] - 2; ++i) cs.push_back(((long long)k * g1.n[1] + j) * g1.n[0] + i);
    CK(cudaMemcpyAsync(c->slev, tab.data(), tab.size(), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->prog, all.data(), sizeof(int4) * all.size(), cudaMemcpyHostToDevice, c->stream));
    if (!cs.empty())
      CK(cudaMemcpyAsync(c->cidx_s, cs.data(), sizeof(long long) * cs.size(), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  CK(cudaMemsetAsync(c->scal, 0, sizeof(double) * 16, c->stream));
  mg_status st = last_launch(c);
  if (st) return st;
  CK(cudaStreamSynchronize(c->stream));
  return MG_OK;
}

// ---- single steps ---------------------------------------------------------------------
// Each runs the kernels the cycle runs, in the context's precision: FP64 contexts on the FP64
// level arrays, MG_MIXED contexts on the FP32 ones (inputs rounded to FP32 on the way in,
// results widened to FP64 on the way out).
template <typename T>
static void pack_lvl(mg_ctx *c, const Launch &lc, int l, const double *src, T *dst) {
  Lev<T> L = LevOf<T>::get(c, l);
  if (c->swap) launch_pack_swapped<T>(lc, L, src, dst, 1);
  else launch_pack<T>(lc, L, src, dst, 1);
}
template <typename T>
static void unpack_lvl(mg_ctx *c, const Launch &lc, int l, const T *src, double *dst) {
  Lev<T> L = LevOf<T>::get(c, l);
  if (c->swap) launch_unpack_swapped<T>(lc, L, src, dst, 1.0);
  else launch_unpack<T>(lc, L, src, dst, 1.0);
}

// the end of a step: wait, then report a launch error or a bounded wait that gave up
static mg_status step_end(mg_ctx *c) {
  CK(cudaStreamSynchronize(c->stream));
  mg_status st = last_launch(c);
  if (st) return st;
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, c->st + 2, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (flag) {
    CK(cudaMemsetAsync(c->st + 2, 0, sizeof(int), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->err = "a bounded device wait gave up";
    return MG_ETIMEOUT;
  }
  return MG_OK;
}

template <typename T>
static mg_status step_smooth_t(mg_ctx *c, int level, const double *u, const double *g, double *out, int sweeps,
                               int order) {
  Launch lc{c->stream, &c->launches};
  LevData<T> &D = LevOf<T>::data(c, level);
  pack_lvl<T>(c, lc, level, u, D.u[0]);
  pack_lvl<T>(c, lc, level, g, D.g);
  c->cur[level] = 0;
  Sched S{c, lc, false};
  smooth<T>(S, level, D.g, sweeps, order ? 1 : 0, false);
  unpack_lvl<T>(c, lc, level, D.u[c->cur[level]], out);
  c->cur[level] = 0;
  return step_end(c);
}

template <typename T>
static mg_status step_defect_t(mg_ctx *c, int level, const double *u, const double *g, double *r) {
  Launch lc{c->stream, &c->launches};
  LevData<T> &D = LevOf<T>::data(c, level);
  pack_lvl<T>(c, lc, level, u, D.u[0]);
  pack_lvl<T>(c, lc, level, g, D.g);
  launch_defect<T>(lc, LevOf<T>::get(c, level), lev_kind(c, level), D.u[0], D.g, D.r);
  unpack_lvl<T>(c, lc, level, D.r, r);
  return step_end(c);
}

template <typename T>
static mg_status step_restrict_t(mg_ctx *c, int level, const double *r, double *gc) {
  Launch lc{c->stream, &c->launches};
  LevData<T> &D = LevOf<T>::data(c, level), &Dc = LevOf<T>::data(c, level - 1);
  pack_lvl<T>(c, lc, level, r, D.r);
  launch_restrict<T>(lc, LevOf<T>::get(c, level), LevOf<T>::get(c, level - 1), D.r, Dc.g);
  unpack_lvl<T>(c, lc, level - 1, Dc.g, gc);
  return step_end(c);
}

template <typename T>
static mg_status step_prolong_t(mg_ctx *c, int level, const double *ec, const double *u, double *u_out, double w) {
  Launch lc{c->stream, &c->launches};
  LevData<T> &D = LevOf<T>::data(c, level), &Dc = LevOf<T>::data(c, level - 1);
  pack_lvl<T>(c, lc, level - 1, ec, Dc.u[0]);
  pack_lvl<T>(c, lc, level, u, D.u[0]);
  launch_prolong_add<T>(lc, LevOf<T>::get(c, level), LevOf<T>::get(c, level - 1), Dc.u[0], D.u[0], (T)w);
  unpack_lvl<T>(c, lc, level, D.u[0], u_out);
  return step_end(c);
}

template <typename T>
static mg_status step_descend_t(mg_ctx *c, int level, const double *u, const double *g, double *u_out,
                                double *gc, int transposed) {
  Launch lc{c->stream, &c->launches};
  LevData<T> &D = LevOf<T>::data(c, level), &Dc = LevOf<T>::data(c, level - 1);
  if (u) pack_lvl<T>(c, lc, level, u, D.u[0]);
  else CK(cudaMemsetAsync(D.u[0], 0, sizeof(T) * (size_t)c->geo[level].count, c->stream));
  pack_lvl<T>(c, lc, level, g, D.g);
  c->cur[level] = 0;
  Sched S{c, lc, false};
  descend<T>(S, level, D.g, transposed ? 1 : 0, u == nullptr);
  unpack_lvl<T>(c, lc, level, D.u[c->cur[level]], u_out);
  unpack_lvl<T>(c, lc, level - 1, Dc.g, gc);
  c->cur[level] = 0;
  return step_end(c);
}

template <typename T>
static mg_status step_ascend_t(mg_ctx *c, int level, const double *ec, const double *u, const double *g,
                               double *u_out, int transposed) {
  Launch lc{c->stream, &c->launches};
  LevData<T> &D = LevOf<T>::data(c, level), &Dc = LevOf<T>::data(c, level - 1);
  pack_lvl<T>(c, lc, level - 1, ec, Dc.u[0]);
  pack_lvl<T>(c, lc, level, u, D.u[0]);
  pack_lvl<T>(c, lc, level, g, D.g);
  c->cur[level] = 0;
  c->cur[level - 1] = 0;
  Sched S{c, lc, false};
  ascend<T>(S, level, D.g, transposed ? 1 : 0);
  unpack_lvl<T>(c, lc, level, D.u[c->cur[level]], u_out);
  c->cur[level] = 0;
  return step_end(c);
}

template <typename T>
static mg_status step_coarse_t(mg_ctx *c, const double *g, double *u) {
  Launch lc{c->stream, &c->launches};
  LevData<T> &D = LevOf<T>::data(c, 1);
  pack_lvl<T>(c, lc, 1, g, D.g);
  CK(cudaMemsetAsync(D.u[0], 0, sizeof(T) * (size_t)c->geo[1].count, c->stream));
  coarse_solve_into<T>(c, lc, D.g, D.u[0]);
  unpack_lvl<T>(c, lc, 1, D.u[0], u);
  return step_end(c);
}

template <typename T>
static mg_status step_cycle_t(mg_ctx *c, const double *x, const double *b, double *x_out, int transposed) {
  int L = c->L;
  Launch lc{c->stream, &c->launches};
  LevData<T> &D = LevOf<T>::data(c, L);
  pack_lvl<T>(c, lc, L, b, D.g);
  pack_lvl<T>(c, lc, L, x, D.u[0]);
  Sched S{c, lc, false};
  c->cur[L] = 0;
  cycle<T>(S, L, D.g, 0, transposed ? 1 : 0, false);
  unpack_lvl<T>(c, lc, L, D.u[c->cur[L]], x_out);
  c->cur[L] = 0;
  return step_end(c);
}

// ---------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------
extern "C" {

size_t mg_workspace_bytes(const mg_params *p, const mg_coeffs *k) {
  if (check_params(p, k) != MG_OK) return 0;
  mg_ctx *c = new (std::nothrow) mg_ctx();
  if (!c) return 0;
  c->P = *p;
  c->K = *k;
  c->L = p->levels;
  c->kind = k->kind;
  c->galerkin = (p->flags & MG_FLAG_GALERKIN) != 0;
  c->ff = p->precision == MG_MIXED && p->dim == 2 && (k->kind == MG_COEF_CONST || k->kind == MG_COEF_SEPARABLE) &&
          !(p->flags & MG_FLAG_FP64_DEFECT);
  c->mixed = p->precision == MG_MIXED;
  apply_swap(c);
  size_t s = layout(c, nullptr);
  delete c;
  return s;
}

mg_status mg_setup(const mg_params *p, const mg_coeffs *k, void *workspace, size_t ws_bytes, mg_ctx **out) {
  if (!out) return MG_EINVAL;
  *out = nullptr;
  mg_status st = check_params(p, k);
  if (st) return st;
  if (!workspace || ((uintptr_t)workspace & 255)) return MG_EINVAL;
  mg_ctx *c = new (std::nothrow) mg_ctx();
  if (!c) return MG_ENOMEM;
  c->P = *p;
  if (c->P.inner_cycles < 1) c->P.inner_cycles = 1;
  c->K = *k;
  c->L = p->levels;
  c->kind = k->kind;
  c->galerkin = (p->flags & MG_FLAG_GALERKIN) != 0;
  c->ff = p->precision == MG_MIXED && p->dim == 2 && (k->kind == MG_COEF_CONST || k->kind == MG_COEF_SEPARABLE) &&
          !(p->flags & MG_FLAG_FP64_DEFECT);
  c->mixed = p->precision == MG_MIXED;
  c->stream = (cudaStream_t)p->stream;
  apply_swap(c);
  size_t need = layout(c, nullptr);
  if (ws_bytes < need) {
    delete c;
    return MG_EINVAL;
  }
  layout(c, (char *)workspace);
  if (cudaGetDevice(&c->dev) != cudaSuccess || cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->cap2, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMallocHost(&c->h_relres, sizeof(double) * 8) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return MG_ECUDA;
  }
  if (p->flags & MG_FLAG_TIMING) {
    c->ev.resize(6144);
    c->ev_bytes.assign(6144, 0.0);
    for (auto &e : c->ev) cudaEventCreate(&e);
  }
  if (p->flags & MG_FLAG_TRACE) {
    c->tr_ev.resize(2 * kTraceMarks);
    c->tr_label.assign(2 * kTraceMarks, nullptr);
    c->tr_lev.assign(2 * kTraceMarks, 0);
    for (auto &e : c->tr_ev) cudaEventCreate(&e);
  }
  st = setup_levels(c);
  if (st) {
    *out = c;   // keep the error text available through mg_last_error
    return st;
  }
  *out = c;
  return MG_OK;
}

void mg_destroy(mg_ctx *c) {
  if (!c) return;
  for (int t = 0; t < 2; ++t)
    if (c->gexec[t]) cudaGraphExecDestroy(c->gexec[t]);
  for (int t = 0; t < 2; ++t)
    if (c->lexec[t]) cudaGraphExecDestroy(c->lexec[t]);
  for (auto &e : c->ev) cudaEventDestroy(e);
  for (auto &e : c->tr_ev) cudaEventDestroy(e);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->cap2) cudaStreamDestroy(c->cap2);
  if (c->h_relres) cudaFreeHost(c->h_relres);
  delete c;
}

const char *mg_status_str(mg_status s) {
  switch (s) {
    case MG_OK: return "ok";
    case MG_EINVAL: return "invalid argument";
    case MG_ENOMEM: return "out of host memory";
    case MG_ECUDA: return "CUDA error";
    case MG_ENOCONV: return "maximum number of cycles reached";
    case MG_EDIVERGED: return "residual norm not finite";
    case MG_ETIMEOUT: return "device wait timed out";
    case MG_EBOUNDS: return "index out of bounds";
  }
  return "unknown status";
}

const char *mg_last_error(const mg_ctx *c) { return c ? c->err.c_str() : "no context"; }

mg_status mg_trace_report(mg_ctx *c, char *buf, size_t cap, size_t *len) {
  if (!c || !(c->P.flags & MG_FLAG_TRACE)) return MG_EINVAL;
  std::vector<std::pair<double, std::string>> rows;
  for (const auto &kv : c->tr_sum) {
    char line[160];
    std::snprintf(line, sizeof(line), "%-32s %3d %9lld %12.4f\n", kv.first.first.c_str(), kv.first.second,
                  kv.second.first, kv.second.second);
    rows.push_back({kv.second.second, line});
  }
  std::sort(rows.begin(), rows.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
  std::string out = "kernel                           level  launches     total_ms   (" +
                    std::to_string(c->tr_steps) + " schedules, " + std::to_string(c->tr_n[0]) + "/" +
                    std::to_string(c->tr_n[1]) + " marks, " + std::to_string(c->tr_unread) + " unreadable)\n";
  for (const auto &r : rows) out += r.second;
  if (len) *len = out.size() + 1;
  if (buf && cap) {   // a call with a buffer consumes the trace; one without only sizes it
    const size_t n = std::min(cap - 1, out.size());
    std::memcpy(buf, out.data(), n);
    buf[n] = '\0';
    c->tr_sum.clear();
    c->tr_steps = c->tr_unread = 0;
  }
  return MG_OK;
}

int mg_debug_build(void) {
#ifdef MG_DEBUG
  return 1;
#else
  return 0;
#endif
}

long long mg_launch_count(const mg_ctx *c) { return c ? c->launches : 0; }

mg_status mg_level_dims(const mg_ctx *c, int level, int n[3]) {
  if (!c || level < 1 || level > c->L || !n) return MG_EINVAL;
  for (int d = 0; d < 3; ++d) n[d] = c->geo[level].n[d];
  if (c->swap) {   // caller-facing axes
    int t = n[0];
    n[0] = n[1];
    n[1] = t;
  }
  return MG_OK;
}

// read back the timing events recorded during the last cycle
static void harvest_events(mg_ctx *c, int base, int n) {
  for (int t = base; t + 1 < base + n; t += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev[t], c->ev[t + 1]) == cudaSuccess) {
      c->t_sum_ms += ms;
      c->t_sum_bytes += c->ev_bytes[t];
      c->t_count++;
    }
  }
  cudaGetLastError();
}

// Copy a caller vector (device or host, compact) into a padded finest-level FP64 buffer,
// Dirichlet entries set to zero.
static mg_status load_vec(mg_ctx *c, const Launch &lc, const Lev<double> &F, const double *src, double *dst,
                          bool host) {
  if (!host) {
    pack_in(c, lc, F, src, dst, 1);
    return MG_OK;
  }
  size_t rows = (size_t)F.n1 * (F.dim == 3 ? F.n2 : 1);
  if (c->swap) {   // stage the caller layout on the device, then transpose into place
    double *stage = c->d64[c->L].r;
    CK(cudaMemcpyAsync(stage, src, sizeof(double) * F.n0 * rows, cudaMemcpyHostToDevice, lc.s));
    pack_in(c, lc, F, stage, dst, 1);
    return MG_OK;
  }
  CK(cudaMemcpy2DAsync(dst, sizeof(double) * F.pitch, src, sizeof(double) * F.n0, sizeof(double) * F.n0, rows,
                       cudaMemcpyHostToDevice, lc.s));
  launch_zero_boundary<double>(lc, F, dst);
  return MG_OK;
}
static mg_status store_vec(mg_ctx *c, const Launch &lc, const Lev<double> &F, const double *src, double *dst,
                           bool host) {
  if (!host) {
    unpack_out(c, lc, F, src, dst, 1.0);
    return MG_OK;
  }
  size_t rows = (size_t)F.n1 * (F.dim == 3 ? F.n2 : 1);
  if (c->swap) {
    double *stage = c->d64[c->L].r;
    unpack_out(c, lc, F, src, stage, 1.0);
    CK(cudaMemcpyAsync(dst, stage, sizeof(double) * F.n0 * rows, cudaMemcpyDeviceToHost, lc.s));
    return MG_OK;
  }
  CK(cudaMemcpy2DAsync(dst, sizeof(double) * F.n0, src, sizeof(double) * F.pitch, sizeof(double) * F.n0, rows,
                       cudaMemcpyDeviceToHost, lc.s));
  return MG_OK;
}

// Shared driver of mg_solve / mg_solve_host / mg_solve_adjoint.
static mg_status run_solve(mg_ctx *c, const double *b, double *x, double tol, mg_report *rep, int transposed,
                           bool host = false) {
  NvtxRange nr(transposed ? "adjoint solve" : "solve");
  auto t0 = std::chrono::steady_clock::now();
  int L = c->L;
  Launch lc{c->stream, &c->launches};
  bool use_graph = !(c->P.flags & MG_FLAG_NO_GRAPH);
  bool timing = (c->P.flags & (MG_FLAG_TIMING | MG_FLAG_TRACE)) != 0;   // host loop, per-step graph
  bool launched = false;
  Lev<double> F64 = lev64(c, L);
  mg_status lst;
  if (use_graph && !timing) {
    // the whole solve on the device: copy in, one graph launch, copy out, one synchronisation
    mg_status st = build_loop_graph(c, transposed);
    if (st) return st;
    if ((lst = load_vec(c, lc, F64, b, c->mixed ? c->b64 : c->d64[L].g, host))) return lst;
    if ((lst = load_vec(c, lc, F64, x, c->mixed ? c->x64 : c->d64[L].u[0], host))) return lst;
    c->h_relres[3] = tol;
    CK(cudaMemcpyAsync(c->scal + 4, c->h_relres + 3, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (c->P.flags & MG_FLAG_TEST_WAIT_TIMEOUT) CK(cudaMemsetAsync(c->st + 5, 1, sizeof(int), c->stream));
    if (c->P.flags & MG_FLAG_TEST_BOUNDS) launch_bounds_probe(lc, F64);
    CK(cudaMemsetAsync(c->st + 6, 0, sizeof(int) * 2, c->stream));   // float-float defects first; iterate in x64
    double *xin = c->mixed ? c->x64 : c->d64[L].u[0];
    std::vector<double> hbuf((size_t)c->P.max_cycles + 2), hall;
    int sth[3] = {0, 0, 0};
    int cycles = 0;
    // A loop that stopped on the float-float defect as converged whose FP64 residual is still
    // above tol (status 8: the error estimate was short) continues from its iterate with FP64
    // outer defects.
    for (int round = 0; round < 4; ++round) {
      if (round) CK(cudaMemsetAsync(c->st + 6, 1, sizeof(int), c->stream));
      CK(cudaGraphLaunch(c->lexec[transposed], c->stream));
      CK(cudaMemcpyAsync(sth, c->st, sizeof(int) * 3, cudaMemcpyDeviceToHost, c->stream));
      CK(cudaMemcpyAsync(c->h_relres, c->scal, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      CK(cudaMemcpyAsync(hbuf.data(), c->hist, sizeof(double) * hbuf.size(), cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
      if ((st = last_launch(c))) return st;
      c->launches += c->loop_init_kernels[transposed] + (long long)sth[0] * c->loop_body_kernels[transposed];
      for (int t = hall.empty() ? 0 : 1; t <= sth[0]; ++t) hall.push_back(hbuf[t]);
      cycles += sth[0];
      if (sth[1] != 8 || cycles >= c->P.max_cycles) break;
    }
    if (sth[1] == 8) sth[1] = 4;
    hbuf = hall;
    if (c->h_relres[0] == 0.0) {   // b = 0: x = 0
      CK(cudaMemsetAsync(xin, 0, sizeof(double) * (size_t)c->geo[L].count, c->stream));
    }
    if ((lst = store_vec(c, lc, F64, xin, x, host))) return lst;
    CK(cudaStreamSynchronize(c->stream));
    if ((st = last_launch(c))) return st;
    mg_status result = sth[1] == 4 ? MG_ENOCONV : sth[1] == 5 ? MG_EDIVERGED : MG_OK;
    if (sth[2] || sth[1] == 6) {   // a bounded device wait gave up: clear the flag, report it
      CK(cudaMemsetAsync(c->st + 2, 0, sizeof(int), c->stream));
      CK(cudaStreamSynchronize(c->stream));
      result = MG_ETIMEOUT;
    }
    if (rep) {
      rep->cycles = cycles;
      rep->relres = hbuf[cycles];
      rep->rate = (cycles > 0 && hbuf[0] > 0.0) ? std::pow(hbuf[cycles] / hbuf[0], 1.0 / cycles) : 0.0;
      rep->status = result;
      if (rep->history)
        for (int t = 0; t <= cycles && t < rep->history_cap; ++t) rep->history[t] = hbuf[t];
      rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return result;
  }
  bool ff_start = false;   // the start vector's defect in float-float (mixed solves)
  if (c->mixed) {
    if ((lst = load_vec(c, lc, F64, b, c->b64, host))) return lst;
    if ((lst = load_vec(c, lc, F64, x, c->x64, host))) return lst;
    if (c->P.flags & MG_FLAG_FMG_START) {
      Sched S{c, lc, false};
      emit_fmg_start(S);
    }
    launch_norm_parts<double>(lc, F64, c->b64, c->partials, norm_parts_count(), c->scal + 0);
    CK(cudaMemsetAsync(c->st + 6, 0, sizeof(int) * 2, c->stream));   // float-float defects first; iterate in x64
    ff_start = start_defect(c, lc);
  } else {
    if ((lst = load_vec(c, lc, F64, b, c->d64[L].g, host))) return lst;
    if ((lst = load_vec(c, lc, F64, x, c->d64[L].u[0], host))) return lst;
    if (c->P.flags & MG_FLAG_FMG_START) {
      Sched S{c, lc, false};
      emit_fmg_start(S);
    }
    launch_norm_parts<double>(lc, F64, c->d64[L].g, c->partials, norm_parts_count(), c->scal + 0);
    launch_defect_norm<double>(lc, F64, c->kind, c->d64[L].u[0], c->d64[L].g, c->partials, norm_parts_count(),
                               c->scal + 1);
  }
  launch_relres(lc, c->scal + 1, c->scal + 0, nullptr, 0, c->scal + 2);
  if (c->P.flags & MG_FLAG_TEST_WAIT_TIMEOUT) CK(cudaMemsetAsync(c->st + 5, 1, sizeof(int), c->stream));
  if (c->P.flags & MG_FLAG_TEST_BOUNDS) launch_bounds_probe(lc, F64);
  if (!c->mixed) CK(cudaMemsetAsync(c->st + 6, 0, sizeof(int) * 2, c->stream));
  bool ff64 = false;   // float-float defects until the loop moves to FP64
  if (use_graph) {
    mg_status st = build_graph(c, transposed);
    if (st) return st;
  }
  std::vector<double> hist;
  mg_status result = MG_OK;
  double bsq = 0.0;
  int it = 0;
  for (;; ++it) {
    CK(cudaMemcpyAsync(c->h_relres, c->scal, sizeof(double) * 6, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (timing && launched) {
      if (use_graph) harvest_events(c, 2048 * (1 + transposed), c->ev_graph_n[transposed]);
      else harvest_events(c, 0, c->ev_used);
      c->ev_used = 0;
      trace_harvest(c, transposed);
    }
    mg_status st = last_launch(c);
    if (st) return st;
    bsq = c->h_relres[0];
    double rr = c->h_relres[2];
    if (bsq == 0.0) {
      rr = 0.0;
      hist.push_back(rr);
      result = MG_OK;
      break;
    }
    // the float-float defect's residual (of the start vector, or after a refinement step) is a
    // stopping signal only: below tol by the defect's error estimate the FP64 residual is
    // computed, decides and is reported; with an estimate of half of tol or more, within
    // kFFSwitch times the estimate of tol, or after a step that cut the residual by less than
    // half, the loop moves to FP64 outer defects (as the device loop does)
    bool exact = true;
    if (c->mixed && c->ff && !ff64 && (it > 0 || ff_start) && std::isfinite(rr)) {
      const double err = kFFErr * std::sqrt(c->h_relres[5] / bsq);
      exact = rr + err <= tol;
      bool to64 =
          !exact && (err >= 0.5 * tol || rr <= tol + kFFSwitch * err || (it >= 2 && rr > 0.5 * hist.back()));
      if (exact) {
        launch_x_settle(lc, c->x64, c->x64b, (long long)c->geo[L].count, c->st + 7);
        launch_defect64_to32(lc, F64, c->kind, c->x64, c->b64, c->d32[L].g, c->partials, norm_parts_count(),
                             c->scal + 1);
        launch_relres(lc, c->scal + 1, c->scal + 0, nullptr, 0, c->scal + 2);
        CK(cudaMemcpyAsync(c->h_relres, c->scal, sizeof(double) * 3, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        rr = c->h_relres[2];
        to64 = !(rr <= tol);
      }
      if (to64) {
        ff64 = true;
        CK(cudaMemsetAsync(c->st + 6, 1, sizeof(int), c->stream));
      }
    }
    hist.push_back(rr);
    if (!std::isfinite(rr)) { result = MG_EDIVERGED; break; }
    if (exact && rr <= tol) { result = MG_OK; break; }
    if (it >= c->P.max_cycles) { result = MG_ENOCONV; break; }
    if (use_graph) {
      CK(cudaGraphLaunch(c->gexec[transposed], c->stream));
      c->launches += c->graph_kernels[transposed];
    } else {
      c->ev_used = 0;
      Sched S{c, lc, timing, 0, &c->ev_used};
      trace_begin(c, S.lc, transposed, false);
      if (c->mixed) emit_mixed_step(S, transposed);
      else emit_fp64_cycle(S, transposed);
      trace_end(c, transposed);
    }
    launched = true;
  }
  // write back the solution (after fused updates, the iterate back into x64 first)
  if (c->mixed && c->ff) launch_x_settle(lc, c->x64, c->x64b, (long long)c->geo[L].count, c->st + 7);
  if (bsq == 0.0) {
    if (c->mixed) CK(cudaMemsetAsync(c->x64, 0, sizeof(double) * (size_t)c->geo[L].count, c->stream));
    else CK(cudaMemsetAsync(c->d64[L].u[0], 0, sizeof(double) * (size_t)c->geo[L].count, c->stream));
  }
  if ((lst = store_vec(c, lc, F64, c->mixed ? c->x64 : c->d64[L].u[0], x, host))) return lst;
  int wait_flag = 0;
  CK(cudaMemcpyAsync(&wait_flag, c->st + 2, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  mg_status st = last_launch(c);
  if (st) return st;
  if (wait_flag) {   // a bounded device wait gave up: clear the flag, report it
    CK(cudaMemsetAsync(c->st + 2, 0, sizeof(int), c->stream));
    CK(cudaStreamSynchronize(c->stream));
    result = MG_ETIMEOUT;
  }
  if (rep) {
    rep->cycles = it;
    rep->relres = hist.back();
    rep->rate = (it > 0 && hist[0] > 0.0) ? std::pow(hist.back() / hist[0], 1.0 / it) : 0.0;
    rep->status = result;
    if (rep->history)
      for (int t = 0; t < (int)hist.size() && t < rep->history_cap; ++t) rep->history[t] = hist[t];
    rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return result;
}

mg_status mg_solve(mg_ctx *c, const double *b, double *x, double tol, mg_report *rep) {
  if (!c || !b || !x || !(tol >= 0.0)) return MG_EINVAL;
  return run_solve(c, b, x, tol, rep, 0);
}

mg_status mg_solve_host(mg_ctx *c, const double *b_host, double *x_host, double tol, mg_report *rep) {
  if (!c || !b_host || !x_host || !(tol >= 0.0)) return MG_EINVAL;
  return run_solve(c, b_host, x_host, tol, rep, 0, true);
}

mg_status mg_solve_adjoint(mg_ctx *c, const double *g, double *lambda, double tol, mg_report *rep) {
  if (!c || !g || !lambda || !(tol >= 0.0)) return MG_EINVAL;
  return run_solve(c, g, lambda, tol, rep, 1);
}

// ---------------------------------------------------------------------------------------
// batched solves: one graph, one independent branch per instance
// ---------------------------------------------------------------------------------------
struct mg_batch {
  std::vector<mg_ctx *> cs;
  std::vector<const double *> b;
  std::vector<double *> x;
  cudaGraphExec_t exec = nullptr;
  double *host = nullptr;        // pinned: [0] tolerance, then one report row per instance
  int stride = 0;                // doubles per report row: loop state (2), ||b||^2 (1), history
  std::vector<long long> loop_init, loop_body, extra;   // kernel counts per instance
  // persistent form: one cooperative launch over the instances marked in pers (all of them, or in
  // the automatic form those with small grids; the rest run as the graph's branches)
  bool persistent = false;
  std::vector<char> pers;
  std::vector<mg_status> pstat;   // status of each persistent instance in the last solve
  int npers = 0;
  bool has_graph = false;
  int grid = 0, nteams = 0;
  BatchTeam *d_teams = nullptr;   // device tables (in the first context's workspace)
  BatchInst *d_insts = nullptr;
  int *d_order = nullptr;
  unsigned *d_bar = nullptr;
  int epoch = 0;                  // solves launched: a finished instance's report row carries it
};

static void batch_free(mg_batch *bt) {
  if (!bt) return;
  if (bt->exec) cudaGraphExecDestroy(bt->exec);
  if (bt->host) cudaFreeHost(bt->host);
  delete bt;
}

// ---- the persistent batched solve --------------------------------------------------------
// Can this context's solve run inside the persistent batch kernel?  2-D, y not periodic,
// constant or separable coefficients, the mixed form with one FP32 cycle per refinement step,
// point Jacobi / red-black Gauss-Seidel or x-line smoothers (y-lines of the constant kind are
// x-lines after the axis swap), rediscretised coarse operators, the dense coarsest solve, the
// fixed correction weight and the caller's start vector.
static bool batch_persistent_ok(const mg_ctx *c) {
  const mg_params &P = c->P;
  if (P.dim != 2 || P.periodic_y || !c->mixed || c->galerkin || c->cg_mode) return false;
  if (c->kind != K_CONST && c->kind != K_SEP) return false;
  if (P.smoother != MG_JACOBI && P.smoother != MG_RBGS && P.smoother != MG_LINE_X && P.smoother != MG_ZEBRA_X)
    return false;
  if (P.flags & (MG_FLAG_FMG_START | MG_FLAG_ADAPTIVE_CORR)) return false;
  if (P.inner_cycles != 1) return false;
  return true;
}

// Step program of one instance (see batch_prog.h); levels with at most kSoloNodes nodes run on
// the team's first CTA alone.
struct BatchProg {
  const mg_ctx *c;
  std::vector<int4> ops;
  int cur[MAXLEV + 1];
  long long solo_nodes;
  explicit BatchProg(const mg_ctx *cc, long long solo) : c(cc), solo_nodes(solo) {
    for (int l = 0; l <= MAXLEV; ++l) cur[l] = 0;
  }
  bool small(int l) const { return (long long)c->geo[l].n[0] * c->geo[l].n[1] <= solo_nodes; }
  void op(int code, int l, int a, int b) {
    const bool solo = l >= 1 && small(l);
    ops.push_back(make_int4(code | (solo ? BP_SOLO : 0), l, a, b));
  }
  void smooth(int l, int sweeps, int order, bool zero) {
    if (sweeps <= 0) return;
    if (zero) op(BP_ZERO, l, cur[l], 0);
    for (int s = 0; s < sweeps; ++s) {
      switch (c->P.smoother) {
        case MG_JACOBI:
          op(BP_JAC, l, 0, cur[l] | (1 - cur[l]) << 4);
          cur[l] = 1 - cur[l];
          break;
        case MG_RBGS:
          op(BP_RB, l, order, cur[l]);
          op(BP_RB, l, 1 - order, cur[l]);
          break;
        case MG_ZEBRA_X:
          op(BP_XLINE, l, 1 | order << 1, cur[l] | cur[l] << 4);
          op(BP_XLINE, l, 1 | (1 - order) << 1, cur[l] | cur[l] << 4);
          break;
        default:   // MG_LINE_X
          op(BP_XLINE, l, 0, cur[l] | (1 - cur[l]) << 4);
          cur[l] = 1 - cur[l];
          break;
      }
    }
  }
  // the F-cycle (type 0) or V-cycle (1) at level l, as cycle() runs it
  void cycle(int l, int type, bool zero) {
    if (l == 1) {
      op(BP_COARSE, 1, cur[1], 0);
      return;
    }
    smooth(l, c->P.nu1, 0, zero);
    op(BP_DEFECT, l, cur[l], 0);
    op(BP_RESTRICT, l, 0, 0);
    cur[l - 1] = 0;
    if (type == 0) {
      cycle(l - 1, 0, true);
      if (l - 1 > 1) cycle(l - 1, 1, false);
    } else {
      cycle(l - 1, 1, true);
    }
    op(BP_PROLONG, l, cur[l], cur[l - 1]);
    smooth(l, c->P.nu2, 0, false);
  }
  void build() {
    const int L = c->L;
    ops.push_back(make_int4(BP_PACK, 0, 0, 0));
    ops.push_back(make_int4(BP_NORM_B, 0, 0, 0));
    ops.push_back(make_int4(BP_DEFECT64, 0, 0, 0));
    const int check0 = (int)ops.size();
    ops.push_back(make_int4(BP_CHECK, 0, 1, 0));   // w: the unpack step, filled in below
    const int loop = (int)ops.size();
    cur[L] = 0;
    cycle(L, 0, true);
    ops.push_back(make_int4(BP_UPDATE, 0, cur[L], 0));
    ops.push_back(make_int4(BP_DEFECT64, 0, 0, 0));
    const int check1 = (int)ops.size();
    ops.push_back(make_int4(BP_CHECK, loop, 0, 0));
    const int unpack = (int)ops.size();
    ops.push_back(make_int4(BP_UNPACK, 0, 0, 0));
    ops.push_back(make_int4(BP_END, 0, 0, 0));
    ops[check0].w = unpack;
    ops[check1].w = unpack;
  }
};

static const long long kBatchSoloNodes = 17000;   // grids up to 129^2 on one CTA
// MG_BATCH_AUTO: instances whose finest grid holds at most this many nodes (padded; 257^2 grids)
// go to the persistent kernel, larger ones to the graph (measured: the persistent kernel solves
// 145 instances of 65^2..257^2 in 40 ms against the graph's 49 ms, but 60 of 1025^2 in 171 ms
// against 68 ms, each such instance getting a few CTAs instead of the whole GPU)
static const long long kBatchAutoMaxNodes = 100000;

// Lay out the persistent form of a batch: programs and level tables in each instance's
// workspace (after its coarse programs), the instance, team, order and barrier tables in the
// first instance's.  Returns false (nothing launched, nothing changed on the device) when an
// instance does not qualify or the tables do not fit.
static bool batch_build_persistent(mg_batch *bt, const double *tol_dev, const std::vector<int> &sel) {
  const int count = (int)sel.size();
  if (count < 1) return false;
  for (int i : sel)
    if (!batch_persistent_ok(bt->cs[i])) return false;
  mg_ctx *c0 = bt->cs[sel[0]];
  int sms = 0, coop = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c0->dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c0->dev) != cudaSuccess || !coop) {
    cudaGetLastError();
    return false;
  }
  const int per_sm = batch_ctas_per_sm();
  if (per_sm < 1) return false;
  const int G = sms * per_sm;
  // team sizes in proportion to the finest grid's nodes, at least one CTA each
  std::vector<long long> nodes(count);
  for (int i = 0; i < count; ++i) nodes[i] = (long long)bt->cs[sel[i]]->geo[bt->cs[sel[i]]->L].count;
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return nodes[a] > nodes[b]; });
  std::vector<BatchTeam> teams;
  if (count <= G) {
    // largest alpha with sum_i max(1, min(32, floor(alpha n_i))) <= G
    auto total = [&](double a) {
      long long t = 0;
      for (int i = 0; i < count; ++i) t += std::max<long long>(1, std::min<long long>(32, (long long)(a * nodes[i])));
      return t;
    };
    double lo = 0.0, hi = 1.0;
    while (total(hi) <= G && hi < 1e9) hi *= 2;
    for (int it = 0; it < 60; ++it) {
      const double mid = 0.5 * (lo + hi);
      (total(mid) <= G ? lo : hi) = mid;
    }
    int cta = 0;
    for (int q = 0; q < count; ++q) {
      const int i = order[q];
      const int sz = (int)std::max<long long>(1, std::min<long long>(32, (long long)(lo * nodes[i])));
      teams.push_back(BatchTeam{cta, sz, q, 1, nullptr, nullptr});
      cta += sz;
    }
  } else {
    // more instances than resident CTAs: single-CTA teams, instances dealt largest first to
    // the least-loaded team
    std::vector<long long> load(G, 0);
    std::vector<std::vector<int>> lists(G);
    for (int q = 0; q < count; ++q) {
      const int t = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      lists[t].push_back(order[q]);
      load[t] += nodes[order[q]];
    }
    std::vector<int> ord2;
    for (int t = 0; t < G; ++t) {
      teams.push_back(BatchTeam{t, 1, (int)ord2.size(), (int)lists[t].size(), nullptr, nullptr});
      ord2.insert(ord2.end(), lists[t].begin(), lists[t].end());
    }
    order = ord2;
  }
  int grid = 0;
  for (const BatchTeam &t : teams) grid += t.size;
  // host rows of the reports: the kernel writes them through the mapped pinned buffer
  double *hdev = nullptr;
  if (cudaHostGetDevicePointer((void **)&hdev, bt->host, 0) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  // per-instance programs and level tables
  std::vector<BatchInst> insts(count);
  struct Up { void *dst; std::vector<char> bytes; };
  std::vector<Up> uploads;
  for (int i = 0; i < count; ++i) {
    mg_ctx *c = bt->cs[sel[i]];
    BatchProg pb(c, kBatchSoloNodes);
    pb.build();
    std::vector<BatchLev> lv(c->L);
    for (int l = 1; l <= c->L; ++l) {
      BatchLev &v = lv[l - 1];
      v.L = lev32(c, l);
      v.u[0] = c->d32[l].u[0];
      v.u[1] = c->d32[l].u[1];
      v.g = c->d32[l].g;
      v.r = c->d32[l].r;
    }
    const size_t off = ((size_t)c->prog_used + 15) / 16 * 16;   // int4 units
    const size_t lev_i4 = (sizeof(BatchLev) * lv.size() + 15) / 16;
    if (off + lev_i4 + pb.ops.size() > 32768) return false;
    BatchLev *dlev = reinterpret_cast<BatchLev *>(c->prog + off);
    int4 *dprog = c->prog + off + lev_i4;
    uploads.push_back(Up{dlev, std::vector<char>((char *)lv.data(), (char *)lv.data() + sizeof(BatchLev) * lv.size())});
    uploads.push_back(Up{dprog, std::vector<char>((char *)pb.ops.data(), (char *)(pb.ops.data() + pb.ops.size()))});
    BatchInst &I = insts[i];
    memset(&I, 0, sizeof(I));
    I.L = c->L;
    I.lev = dlev;
    I.prog = dprog;
    I.plen = (int)pb.ops.size();
    I.F64 = lev64(c, c->L);
    I.kind = c->kind;
    I.x64 = c->x64;
    I.b64 = c->b64;
    I.bcall = bt->b[sel[i]];
    I.xcall = bt->x[sel[i]];
    I.swap = c->swap ? 1 : 0;
    I.n0c = c->swap ? c->geo[c->L].n[1] : c->geo[c->L].n[0];
    I.n1c = c->swap ? c->geo[c->L].n[0] : c->geo[c->L].n[1];
    I.Ainv = c->Ainv;
    I.cidx = c->cidx;
    I.nc = c->nc;
    I.scal = c->scal;
    I.hrow = hdev + 1 + (size_t)sel[i] * bt->stride;   // the instance's report row
    I.st = c->st;
    I.tol = tol_dev;
    I.maxit = c->P.max_cycles;
    I.omega = (float)c->P.omega;
    I.omega_corr = (float)c->P.omega_corr;
    I.fail_arrival = (c->P.flags & MG_FLAG_TEST_WAIT_TIMEOUT) ? 1 : 0;
  }
  // batch-wide tables after the first instance's own
  size_t off0 = 0;
  {
    mg_ctx *c = c0;
    const size_t off = ((size_t)c->prog_used + 15) / 16 * 16;
    BatchProg pb(c, kBatchSoloNodes);
    pb.build();
    off0 = off + (sizeof(BatchLev) * c->L + 15) / 16 + pb.ops.size();
    off0 = (off0 + 15) / 16 * 16;
  }
  const size_t nt = teams.size();
  const size_t need = (sizeof(BatchInst) * count + 15) / 16 + (sizeof(BatchTeam) * nt + 15) / 16 +
                      (sizeof(int) * count + 15) / 16 + (sizeof(unsigned) * nt + 15) / 16 +
                      (sizeof(double) * 2 * (size_t)grid + 15) / 16;
  if (off0 + need > 32768) return false;
  char *base = reinterpret_cast<char *>(c0->prog + off0);
  BatchInst *d_insts = reinterpret_cast<BatchInst *>(base);
  base += (sizeof(BatchInst) * count + 15) / 16 * 16;
  BatchTeam *d_teams = reinterpret_cast<BatchTeam *>(base);
  base += (sizeof(BatchTeam) * nt + 15) / 16 * 16;
  int *d_order = reinterpret_cast<int *>(base);
  base += (sizeof(int) * count + 15) / 16 * 16;
  unsigned *d_bar = reinterpret_cast<unsigned *>(base);
  base += (sizeof(unsigned) * nt + 15) / 16 * 16;
  double *d_part = reinterpret_cast<double *>(base);
  for (size_t t = 0; t < nt; ++t) {
    teams[t].bar = d_bar + t;
    teams[t].part = d_part + 2 * (size_t)teams[t].cta0;
  }
  uploads.push_back(Up{d_insts, std::vector<char>((char *)insts.data(), (char *)(insts.data() + count))});
  uploads.push_back(Up{d_teams, std::vector<char>((char *)teams.data(), (char *)(teams.data() + nt))});
  uploads.push_back(Up{d_order, std::vector<char>((char *)order.data(), (char *)(order.data() + count))});
  for (const Up &u : uploads)
    if (cudaMemcpyAsync(u.dst, u.bytes.data(), u.bytes.size(), cudaMemcpyHostToDevice, c0->stream) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
  if (cudaStreamSynchronize(c0->stream) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  bt->persistent = true;
  bt->pers.assign(bt->cs.size(), 0);
  bt->pstat.assign(bt->cs.size(), MG_OK);
  for (int i : sel) bt->pers[i] = 1;
  bt->npers = count;
  bt->grid = grid;
  bt->nteams = (int)nt;
  bt->d_teams = d_teams;
  bt->d_insts = d_insts;
  bt->d_order = d_order;
  bt->d_bar = d_bar;
  return true;
}

static mg_status batch_create(mg_ctx *const *cs, int count, const double *const *b, double *const *x, int mode,
                              mg_batch **out) {
  if (!out) return MG_EINVAL;
  *out = nullptr;
  if (!cs || !b || !x || count < 1) return MG_EINVAL;
  int maxc = 0;
  for (int i = 0; i < count; ++i) {
    if (!cs[i] || !b[i] || !x[i]) return MG_EINVAL;
    if (cs[i]->P.flags & (MG_FLAG_NO_GRAPH | MG_FLAG_TIMING)) return MG_EINVAL;
    if (cs[i]->dev != cs[0]->dev) return MG_EINVAL;
    maxc = std::max(maxc, cs[i]->P.max_cycles);
  }
  {
    std::vector<mg_ctx *> sorted(cs, cs + count);
    std::sort(sorted.begin(), sorted.end());
    if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return MG_EINVAL;
  }
  mg_batch *bt = new (std::nothrow) mg_batch();
  if (!bt) return MG_ENOMEM;
  bt->cs.assign(cs, cs + count);
  bt->b.assign(b, b + count);
  bt->x.assign(x, x + count);
  bt->stride = 3 + maxc + 2;
  bt->loop_init.assign(count, 0);
  bt->loop_body.assign(count, 0);
  bt->extra.assign(count, 0);
  mg_ctx *c0 = cs[0];
  if (cudaMallocHost(&bt->host, sizeof(double) * (1 + (size_t)count * bt->stride)) != cudaSuccess) {
    cudaGetLastError();
    batch_free(bt);
    return MG_ECUDA;
  }
  std::memset(bt->host, 0, sizeof(double) * (1 + (size_t)count * bt->stride));
  bt->pers.assign(count, 0);
  if (mode != MG_BATCH_GRAPH) {
    // persistent: every instance (MG_BATCH_PERSISTENT), or the qualifying ones with small finest
    // grids (MG_BATCH_AUTO; larger ones solve faster as graph branches over the whole GPU)
    std::vector<int> sel;
    for (int i = 0; i < count; ++i)
      if (mode == MG_BATCH_PERSISTENT ||
          (batch_persistent_ok(cs[i]) && (long long)cs[i]->geo[cs[i]->L].count <= kBatchAutoMaxNodes))
        sel.push_back(i);
    double *hdev = nullptr;
    bool ok = !sel.empty() && cudaHostGetDevicePointer((void **)&hdev, bt->host, 0) == cudaSuccess;
    if (!ok) cudaGetLastError();
    ok = ok && batch_build_persistent(bt, hdev, sel);
    if (mode == MG_BATCH_PERSISTENT && !ok) {
      c0->err = "the persistent batched solve does not cover these instances";
      batch_free(bt);
      return MG_EINVAL;
    }
    if (ok && bt->npers == count) {
      *out = bt;
      return MG_OK;
    }
  }
  bt->has_graph = true;
  // capture: fork one branch per instance from the root stream, join them at the end
  cudaStream_t root = nullptr;
  std::vector<cudaEvent_t> evs(count + 1, nullptr);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&root, cudaStreamNonBlocking);
  for (int i = 0; i <= count && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&evs[i], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(root, cudaStreamCaptureModeThreadLocal);
  bool capturing = e == cudaSuccess;
  if (e == cudaSuccess) e = cudaEventRecord(evs[count], root);
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    if (bt->pers[i]) continue;   // solved by the persistent kernel
    mg_ctx *c = cs[i];
    cudaStream_t s = c->cap;
    Launch lc{s, &c->launches};
    Lev<double> F64 = lev64(c, c->L);
    double *row = bt->host + 1 + (size_t)i * bt->stride;
    long long k0 = c->launches;
    e = cudaStreamWaitEvent(s, evs[count], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->scal + 4, bt->host, sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->st + 6, 0, sizeof(int) * 2, s);   // float-float defects first
    if (e == cudaSuccess) {
      load_vec(c, lc, F64, b[i], c->mixed ? c->b64 : c->d64[c->L].g, false);
      load_vec(c, lc, F64, x[i], c->mixed ? c->x64 : c->d64[c->L].u[0], false);
      e = capture_loop(c, s, 0, &bt->loop_init[i], &bt->loop_body[i]);
    }
    if (e == cudaSuccess) {
      store_vec(c, lc, F64, c->mixed ? c->x64 : c->d64[c->L].u[0], x[i], false);
      e = cudaMemcpyAsync(row, c->st, sizeof(int) * 3, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(row + 2, c->scal, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(row + 3, c->hist, sizeof(double) * (c->P.max_cycles + 2), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(evs[i], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(root, evs[i], 0);
    bt->extra[i] = c->launches - k0;
    c->launches = k0;
  }
  if (capturing) {
    cudaError_t e2 = cudaStreamEndCapture(root, &graph);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) make_programmatic(c0, graph);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&bt->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  for (auto ev : evs)
    if (ev) cudaEventDestroy(ev);
  if (root) cudaStreamDestroy(root);
  if (e != cudaSuccess) {
    c0->err = std::string("batched graph: ") + cudaGetErrorString(e);
    cudaGetLastError();
    bt->exec = nullptr;
    batch_free(bt);
    return MG_ECUDA;
  }
  *out = bt;
  return MG_OK;
}

mg_status mg_batch_create(mg_ctx *const *cs, int count, const double *const *b, double *const *x, mg_batch **out) {
  return batch_create(cs, count, b, x, MG_BATCH_AUTO, out);
}

mg_status mg_batch_create_ex(mg_ctx *const *cs, int count, const double *const *b, double *const *x, int mode,
                             mg_batch **out) {
  if (mode != MG_BATCH_AUTO && mode != MG_BATCH_GRAPH && mode != MG_BATCH_PERSISTENT) return MG_EINVAL;
  return batch_create(cs, count, b, x, mode, out);
}

mg_status mg_batch_info(const mg_batch *bt, int *persistent, int *ctas, int *teams) {
  if (!bt) return MG_EINVAL;
  if (persistent) *persistent = bt->persistent ? bt->npers : 0;
  if (ctas) *ctas = bt->grid;
  if (teams) *teams = bt->nteams;
  return MG_OK;
}

// The persistent form: one cooperative launch; every finished instance's report row carries
// this launch's epoch, a row without it belongs to an instance whose team gave up a wait.
static mg_status batch_solve_persistent(mg_batch *bt, double tol, mg_report *reps) {
  auto t0 = std::chrono::steady_clock::now();
  mg_ctx *c = bt->cs[0];
  const int count = (int)bt->cs.size();
  bt->host[0] = tol;
  const int epoch = ++bt->epoch;
  CK(cudaMemsetAsync(bt->d_bar, 0, sizeof(unsigned) * (size_t)bt->nteams, c->stream));
  CK(launch_batch(c->stream, bt->grid, bt->d_teams, bt->nteams, bt->d_insts, bt->d_order, epoch, &c->launches));
  CK(cudaStreamSynchronize(c->stream));
  mg_status result = MG_OK;
  for (int i = 0; i < count; ++i) {
    if (!bt->pers[i]) continue;
    mg_ctx *ci = bt->cs[i];
    const double *row = bt->host + 1 + (size_t)i * bt->stride;
    int st4[4];
    std::memcpy(st4, row, sizeof(st4));
    const bool done = st4[3] == epoch;
    const int cycles = done ? st4[0] : 0;
    mg_status si = st4[1] == 4 ? MG_ENOCONV : st4[1] == 5 ? MG_EDIVERGED : MG_OK;
    if (!done) {   // a bounded wait gave up in this instance's team: clear the flag, report it
      CK(cudaMemsetAsync(ci->st + 2, 0, sizeof(int), c->stream));
      CK(cudaStreamSynchronize(c->stream));
      si = MG_ETIMEOUT;
    }
    if (si != MG_OK && result == MG_OK) result = si;
    bt->pstat[i] = si;
    if (reps) {
      mg_report &r = reps[i];
      const double *hist = row + 3;
      r.cycles = cycles;
      r.relres = done ? hist[cycles] : 0.0;
      r.rate = (done && cycles > 0 && hist[0] > 0.0) ? std::pow(hist[cycles] / hist[0], 1.0 / cycles) : 0.0;
      r.status = si;
      if (r.history)
        for (int t = 0; t <= cycles && t < r.history_cap; ++t) r.history[t] = done ? hist[t] : 0.0;
      r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
  }
  return result;
}

mg_status mg_batch_solve(mg_batch *bt, double tol, mg_report *reps) {
  if (!bt || !(tol >= 0.0)) return MG_EINVAL;
  if (bt->persistent && !bt->has_graph) return batch_solve_persistent(bt, tol, reps);
  mg_status pres = MG_OK;
  if (bt->persistent) {   // the small instances first, in one cooperative launch; then the graph
    pres = batch_solve_persistent(bt, tol, reps);
    if (pres != MG_OK && pres != MG_ENOCONV && pres != MG_EDIVERGED && pres != MG_ETIMEOUT) return pres;
  }
  auto t0 = std::chrono::steady_clock::now();
  mg_ctx *c = bt->cs[0];
  const int count = (int)bt->cs.size();
  bt->host[0] = tol;
  CK(cudaGraphLaunch(bt->exec, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  mg_status result = MG_OK;
  bool fixups = false;
  for (int i = 0; i < count; ++i) {
    if (bt->persistent && bt->pers[i]) {   // reported by the persistent launch above
      if (bt->pstat[i] != MG_OK && result == MG_OK) result = bt->pstat[i];
      continue;
    }
    mg_ctx *ci = bt->cs[i];
    const double *row = bt->host + 1 + (size_t)i * bt->stride;
    int st3[3];
    std::memcpy(st3, row, sizeof(st3));
    const int cycles = st3[0];
    const double bsq = row[2];
    const double *hist = row + 3;
    ci->launches += bt->extra[i] + bt->loop_init[i] + (long long)cycles * bt->loop_body[i];
    mg_status si = (st3[1] == 4 || st3[1] == 8) ? MG_ENOCONV : st3[1] == 5 ? MG_EDIVERGED : MG_OK;
    if (st3[2] || st3[1] == 6) {   // a bounded device wait gave up: clear the flag, report it
      CK(cudaMemsetAsync(ci->st + 2, 0, sizeof(int), c->stream));
      fixups = true;
      si = MG_ETIMEOUT;
    }
    if (bsq == 0.0) {   // b = 0: x = 0
      const int *n = ci->P.n;
      size_t nodes = (size_t)n[0] * n[1] * (ci->P.dim == 3 ? n[2] : 1);
      CK(cudaMemsetAsync(bt->x[i], 0, sizeof(double) * nodes, c->stream));
      fixups = true;
    }
    if (si != MG_OK && result == MG_OK) result = si;
    if (reps) {
      mg_report &r = reps[i];
      r.cycles = cycles;
      r.relres = hist[cycles];
      r.rate = (cycles > 0 && hist[0] > 0.0) ? std::pow(hist[cycles] / hist[0], 1.0 / cycles) : 0.0;
      r.status = si;
      if (r.history)
        for (int t = 0; t <= cycles && t < r.history_cap; ++t) r.history[t] = hist[t];
      r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
  }
  if (fixups) CK(cudaStreamSynchronize(c->stream));
  return result;
}

void mg_batch_destroy(mg_batch *bt) { batch_free(bt); }

mg_status mg_solve_batched(mg_ctx *const *cs, int count, const double *const *b, double *const *x, double tol,
                           mg_report *reps) {
  if (!(tol >= 0.0)) return MG_EINVAL;
  mg_batch *bt = nullptr;
  mg_status st = mg_batch_create(cs, count, b, x, &bt);
  if (st) return st;
  st = mg_batch_solve(bt, tol, reps);
  mg_batch_destroy(bt);
  return st;
}

mg_status mg_grad_coeff(mg_ctx *c, const double *u, const double *lambda, double *dk) {
  if (!c || !u || !lambda || !dk) return MG_EINVAL;
  if (c->kind != K_CELL) return MG_EINVAL;
  int L = c->L;
  Launch lc{c->stream, &c->launches};
  Lev<double> F = lev64(c, L);
  double *ub = c->mixed ? c->d64[L].u[0] : c->d64[L].u[1];
  double *lb = c->d64[L].r;
  pack_in(c, lc,F, u, ub, 1);
  pack_in(c, lc,F, lambda, lb, 1);
  launch_grad_k(lc, F, ub, lb, c->grad_tmp);
  if (c->swap) launch_cell_unpack_swapped(lc, F, c->grad_tmp, dk);
  else launch_cell_unpack(lc, F, c->grad_tmp, dk);
  CK(cudaStreamSynchronize(c->stream));
  return last_launch(c);
}

mg_status mg_residual_norm(mg_ctx *c, int level, const double *u, const double *b, double *out) {
  if (!c || !u || !b || !out || level < 1 || level > c->L) return MG_EINVAL;
  if (c->mixed && level != c->L) return MG_EINVAL;
  Launch lc{c->stream, &c->launches};
  Lev<double> Lv = lev64(c, level);
  LevData<double> &D = c->d64[level];
  pack_in(c, lc, Lv, u, D.u[0], 1);
  pack_in(c, lc, Lv, b, D.g, 1);
  launch_defect_norm<double>(lc, Lv, lev_kind(c, level), D.u[0], D.g, c->partials, norm_parts_count(), c->scal + 3);
  launch_sqrt(lc, c->scal + 3, out);
  CK(cudaStreamSynchronize(c->stream));
  return last_launch(c);
}

mg_status mg_apply(mg_ctx *c, int level, const double *u, double *Au) {
  if (!c || !u || !Au || level < 1 || level > c->L) return MG_EINVAL;
  if (c->mixed && level != c->L) return MG_EINVAL;
  Launch lc{c->stream, &c->launches};
  Lev<double> Lv = lev64(c, level);
  LevData<double> &D = c->d64[level];
  double *ub = c->mixed ? D.u[0] : D.u[1];
  pack_in(c, lc,Lv, u, ub, 1);
  CK(cudaMemsetAsync(D.g, 0, sizeof(double) * (size_t)c->geo[level].count, c->stream));
  launch_defect<double>(lc, Lv, lev_kind(c, level), ub, D.g, D.r);   // r = 0 - A u
  unpack_out(c, lc,Lv, D.r, Au, -1.0);
  CK(cudaStreamSynchronize(c->stream));
  return last_launch(c);
}

mg_status mg_step_smooth(mg_ctx *c, int level, const double *u, const double *g, double *out, int sweeps, int order) {
  if (!c || level < 1 || level > c->L || !u || !g || !out || sweeps < 0) return MG_EINVAL;
  return c->mixed ? step_smooth_t<float>(c, level, u, g, out, sweeps, order)
                  : step_smooth_t<double>(c, level, u, g, out, sweeps, order);
}

mg_status mg_step_defect(mg_ctx *c, int level, const double *u, const double *g, double *r) {
  if (!c || level < 1 || level > c->L || !u || !g || !r) return MG_EINVAL;
  return c->mixed ? step_defect_t<float>(c, level, u, g, r) : step_defect_t<double>(c, level, u, g, r);
}

mg_status mg_step_restrict(mg_ctx *c, int level, const double *r, double *gc) {
  if (!c || level < 2 || level > c->L || !r || !gc) return MG_EINVAL;
  return c->mixed ? step_restrict_t<float>(c, level, r, gc) : step_restrict_t<double>(c, level, r, gc);
}

mg_status mg_step_prolong(mg_ctx *c, int level, const double *ec, const double *u, double *u_out, double w) {
  if (!c || level < 2 || level > c->L || !ec || !u || !u_out) return MG_EINVAL;
  return c->mixed ? step_prolong_t<float>(c, level, ec, u, u_out, w)
                  : step_prolong_t<double>(c, level, ec, u, u_out, w);
}

mg_status mg_step_descend(mg_ctx *c, int level, const double *u, const double *g, double *u_out, double *gc,
                          int transposed) {
  if (!c || level < 2 || level > c->L || !g || !u_out || !gc) return MG_EINVAL;
  return c->mixed ? step_descend_t<float>(c, level, u, g, u_out, gc, transposed)
                  : step_descend_t<double>(c, level, u, g, u_out, gc, transposed);
}

mg_status mg_step_ascend(mg_ctx *c, int level, const double *ec, const double *u, const double *g, double *u_out,
                         int transposed) {
  if (!c || level < 2 || level > c->L || !ec || !u || !g || !u_out) return MG_EINVAL;
  return c->mixed ? step_ascend_t<float>(c, level, ec, u, g, u_out, transposed)
                  : step_ascend_t<double>(c, level, ec, u, g, u_out, transposed);
}

mg_status mg_step_coarse(mg_ctx *c, const double *g, double *u) {
  if (!c || !g || !u) return MG_EINVAL;
  return c->mixed ? step_coarse_t<float>(c, g, u) : step_coarse_t<double>(c, g, u);
}

mg_status mg_step_cycle(mg_ctx *c, const double *x, const double *b, double *x_out, int transposed) {
  if (!c || !x || !b || !x_out) return MG_EINVAL;
  return c->mixed ? step_cycle_t<float>(c, x, b, x_out, transposed)
                  : step_cycle_t<double>(c, x, b, x_out, transposed);
}

mg_status mg_step_outer_defect(mg_ctx *c, const double *x, const double *b, double *r, double *sq) {
  if (!c || !x || !b || !r || !c->mixed) return MG_EINVAL;
  const int L = c->L;
  Launch lc{c->stream, &c->launches};
  Lev<double> F64 = lev64(c, L);
  pack_in(c, lc, F64, x, c->x64, 1);
  pack_in(c, lc, F64, b, c->b64, 1);
  if (!(c->ff && launch_defect_ff(lc, F64, c->kind, c->x64, nullptr, c->b64, c->d32[L].g, c->partials,
                                  norm_parts_count(), c->scal + 1, c->scal + 5, nullptr)))
    launch_defect64_to32(lc, F64, c->kind, c->x64, c->b64, c->d32[L].g, c->partials, norm_parts_count(), c->scal + 1);
  unpack_lvl<float>(c, lc, L, c->d32[L].g, r);
  if (sq) CK(cudaMemcpyAsync(sq, c->scal + 1, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return step_end(c);
}

mg_status mg_kernel_timing(mg_ctx *c, double *mean_ms, int *launches, double *bytes_per_launch) {
  if (!c) return MG_EINVAL;
  if (mean_ms) *mean_ms = c->t_count ? c->t_sum_ms / c->t_count : 0.0;
  if (launches) *launches = (int)c->t_count;
  // mean algorithmic bytes of the timed launches (each recorded with its sweep's kind)
  if (bytes_per_launch) *bytes_per_launch = c->t_count ? c->t_sum_bytes / c->t_count : 0.0;
  c->t_sum_ms = 0.0;
  c->t_sum_bytes = 0.0;
  c->t_count = 0;
  return MG_OK;
}

}  // extern "C"
