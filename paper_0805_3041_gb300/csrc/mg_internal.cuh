// mg_internal.cuh -- device-side level view, stencil helpers and kernel launchers.
//
// Data layout in HBM (every level, both precisions): node (i, j, k) of level l
// lives at  base + k * plane + j * pitch + i,  pitch = round_up(n0, 128)
// elements, plane = pitch * n1, each array 256-byte aligned.  Dirichlet nodes
// are stored and hold 0; kernels only ever write unknowns.  A periodic y
// direction has n1 distinct rows and wraps.  Cell coefficients (per-cell k of
// -div(k grad u)) use the node layout of their level, cell (i, j, k) spanning
// nodes [i, i+1] x [j, j+1] x [k, k+1].
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mg {

// First statement of every kernel of the library: when the kernel is the downstream end of a
// programmatic dependency in a CUDA graph (its launch may begin while the upstream kernel drains),
// it waits here until the upstream kernel has completed and its writes are visible.  For an
// ordinary launch it returns at once.
#define MG_PDL_WAIT() asm volatile("griddepcontrol.wait;" ::: "memory")

// K_NINE: a Galerkin coarse level (2-D): a 9-point stencil per node, stored by symmetry as
// its diagonal D (dg), the weights w = -A(p, q) of the couplings to the +x (ex), +y (ey),
// +x+y (ez) and -x+y (enw) neighbours, and 1/D (ndinv); the other four couplings of a node
// are those of its neighbours.
enum Kind { K_CONST = 0, K_SEP = 1, K_CELL = 2, K_EDGE = 3, K_NINE = 4 };

// Everything a kernel needs to know about one level.  Passed by value.
template <typename T>
struct Lev {
  int dim, n0, n1, n2, per;
  long long pitch, plane;
  // constant coefficients: edge weights, diagonal, its inverse
  T cx, cy, cz, d, dinv;
  // separable coefficients: per x-index arrays of length n0 (sx has n0-1 used entries)
  const T *sx, *sy, *sz, *sdinv;
  // cell coefficients: k per cell, 1/D per node, weight factors 1/(2h^2) (2-D) or 1/(4h^2) (3-D)
  const T *k, *ndinv;
  T ax, ay, az;
  // edge coefficients: per node, the weights of the edges to the +x, +y, +z neighbours (1/D in ndinv)
  const T *ex, *ey, *ez;
  // Galerkin levels (K_NINE): diagonal, and the -x+y coupling (ez holds the +x+y one)
  const T *dg, *enw;
  // the context's bounds word (device; used by the -DMG_DEBUG build's checks only)
  unsigned *oob;

  __host__ __device__ int ylo() const { return per ? 0 : 1; }
  __host__ __device__ int yrows() const { return per ? n1 : n1 - 2; }
  __host__ __device__ int zrows() const { return dim == 3 ? n2 - 2 : 1; }
  __host__ __device__ long long unk_rows() const { return (long long)yrows() * zrows(); }
  __host__ __device__ int xunk() const { return n0 - 2; }
};

// Device-side bounds checks of the debug build (-DMG_DEBUG).  MG_CK(L, p) is true when node
// index p lies inside a node array of level L (plane * n2 elements); otherwise the first failing
// check records its site, (file id << 16) | line, in the context's bounds word and the caller
// skips the access; the host then returns MG_EBOUNDS (no trap, no fault).  MG_CKN(L, p, n) checks
// an index into an array of n elements.  In the normal build both are the constant true.
#ifndef MG_FILE_ID
#define MG_FILE_ID 0
#endif
#ifdef MG_DEBUG
template <typename T>
__device__ __forceinline__ bool mg_ck_n(const Lev<T> &L, long long p, long long n, unsigned site) {
  if (p >= 0 && p < n) return true;
  if (L.oob) atomicCAS(L.oob, 0u, site);
  return false;
}
#define MG_SITE (((unsigned)MG_FILE_ID << 16) | (unsigned)__LINE__)
#define MG_CKN(L, p, n) mg::mg_ck_n((L), (long long)(p), (long long)(n), MG_SITE)
#define MG_CK(L, p) MG_CKN((L), (p), (L).plane * ((L).dim == 3 ? (L).n2 : 1))
#else
#define MG_CKN(L, p, n) true
#define MG_CK(L, p) true
#endif

// Offsets of the y neighbours of row j (periodic wrap).
template <typename T, typename IT>
__device__ __forceinline__ void yoffs(const Lev<T> &L, int j, IT &dm, IT &dp) {
  dm = -(IT)L.pitch;
  dp = (IT)L.pitch;
  if (L.per) {
    if (j == 0) dm = (IT)(L.n1 - 1) * (IT)L.pitch;
    if (j == L.n1 - 1) dp = -(IT)(L.n1 - 1) * (IT)L.pitch;
  }
}

// Row index r in [0, unk_rows) -> (j, k) of an unknown row.
template <typename T>
__device__ __forceinline__ void row_jk(const Lev<T> &L, long long r, int &j, int &k) {
  // row counts fit in 32 bits; 2-D needs no division, 3-D a 32-bit one (a 64-bit integer
  // division is a long software sequence on the GPU)
  const int rr = (int)r;
  if (L.dim == 2) {
    j = L.ylo() + rr;
    k = 0;
  } else {
    const int yr = L.yrows(), q = rr / yr;
    j = L.ylo() + (rr - q * yr);
    k = 1 + q;
  }
}

// Edge weights around node p = (i, j, k): W, E (x), S, N (y), B, F (z), and 1/D.
template <typename T, int DIM, int KIND>
struct Weights {
  T wW, wE, wS, wN, wB, wF, dinv;
  T wSW, wSE, wNW, wNE, dd;   // K_NINE only: corner couplings and the diagonal
  template <typename IT>
  __device__ __forceinline__ void load(const Lev<T> &L, int i, IT p, IT dm) {
    if (KIND == K_NINE) {
      // 2-D Galerkin level: the node's own +x, +y, +x+y, -x+y couplings, the rest from the
      // neighbours that own them
      const IT pt = (IT)L.pitch;
      wE = L.ex[p];
      wW = L.ex[p - 1];
      wN = L.ey[p];
      wS = L.ey[p - pt];
      wNE = L.ez[p];
      wSW = L.ez[p - pt - 1];
      wNW = L.enw[p];
      wSE = L.enw[p - pt + 1];
      wB = wF = T(0);
      dd = L.dg[p];
      dinv = L.ndinv[p];
    } else if (KIND == K_CONST) {
      wW = wE = L.cx;
      wS = wN = L.cy;
      wB = wF = L.cz;
      dinv = L.dinv;
    } else if (KIND == K_SEP) {
      wW = L.sx[i - 1];
      wE = L.sx[i];
      wS = wN = L.sy[i];
      wB = wF = L.sz[i];
      dinv = L.sdinv[i];
    } else if (KIND == K_EDGE) {
      wW = L.ex[p - 1];
      wE = L.ex[p];
      wS = L.ey[p + dm];   // the +y edge of the node below (periodic: of the last row)
      wN = L.ey[p];
      if (DIM == 3) {
        wB = L.ez[p - (IT)L.plane];
        wF = L.ez[p];
      } else {
        wB = wF = T(0);
      }
      dinv = L.ndinv[p];
    } else {
      // cells around node p: SW = (i-1, j-1), SE = (i, j-1), NW = (i-1, j), NE = (i, j)
      const T *k = L.k;
      if (DIM == 2) {
        T sw = k[p + dm - 1], se = k[p + dm], nw = k[p - 1], ne = k[p];
        wW = L.ax * (sw + nw);
        wE = L.ax * (se + ne);
        wS = L.ay * (sw + se);
        wN = L.ay * (nw + ne);
        wB = wF = T(0);
      } else {
        IT pl = (IT)L.plane;
        T sw0 = k[p - pl + dm - 1], se0 = k[p - pl + dm], nw0 = k[p - pl - 1], ne0 = k[p - pl];
        T sw1 = k[p + dm - 1], se1 = k[p + dm], nw1 = k[p - 1], ne1 = k[p];
        wW = L.ax * ((sw0 + nw0) + (sw1 + nw1));
        wE = L.ax * ((se0 + ne0) + (se1 + ne1));
        wS = L.ay * ((sw0 + se0) + (sw1 + se1));
        wN = L.ay * ((nw0 + ne0) + (nw1 + ne1));
        wB = L.az * ((sw0 + se0) + (nw0 + ne0));
        wF = L.az * ((sw1 + se1) + (nw1 + ne1));
      }
      dinv = L.ndinv[p];
    }
  }
};

// r_p = g_p - (A u)_p  =  g_p - D u_p + sum_q w_pq u_q, written as an FMA chain.  IT is the
// index type: 64-bit for global arrays, 32-bit for shared-memory ones.
template <typename T, int DIM, int KIND, typename IT>
__device__ __forceinline__ T residual_at(const Lev<T> &L, const Weights<T, DIM, KIND> &w, const T *__restrict__ u,
                                         IT p, IT dm, IT dp, T gp) {
#ifdef MG_DEBUG
  if (sizeof(IT) == 8) {   // global arrays (shared-memory copies are indexed by the coarse kernel)
    const long long n = L.plane * (L.dim == 3 ? L.n2 : 1);
    const unsigned site = (15u << 16) | (unsigned)__LINE__;   // 15: this header
    bool ok = mg_ck_n(L, p - 1, n, site) && mg_ck_n(L, p + 1, n, site) && mg_ck_n(L, p + dm, n, site) &&
              mg_ck_n(L, p + dp, n, site);
    if (KIND == K_NINE) ok = ok && mg_ck_n(L, p + dm - 1, n, site) && mg_ck_n(L, p + dp + 1, n, site);
    if (DIM == 3) ok = ok && mg_ck_n(L, p - (long long)L.plane, n, site) && mg_ck_n(L, p + (long long)L.plane, n, site);
    if (!ok) return gp;
  }
#endif
  T up = u[p];
  T s;
  if (KIND == K_NINE) {
    s = fma(-w.dd, up, gp);
    s = fma(w.wW, u[p - 1], s);
    s = fma(w.wE, u[p + 1], s);
    s = fma(w.wS, u[p + dm], s);
    s = fma(w.wN, u[p + dp], s);
    s = fma(w.wSW, u[p + dm - 1], s);
    s = fma(w.wSE, u[p + dm + 1], s);
    s = fma(w.wNW, u[p + dp - 1], s);
    s = fma(w.wNE, u[p + dp + 1], s);
    return s;
  }
  if (KIND == K_CONST) {
    s = fma(-L.d, up, gp);
  } else {
    T D = (w.wW + w.wE) + (w.wS + w.wN);
    if (DIM == 3) D += w.wB + w.wF;
    s = fma(-D, up, gp);
  }
  s = fma(w.wW, u[p - 1], s);
  s = fma(w.wE, u[p + 1], s);
  s = fma(w.wS, u[p + dm], s);
  s = fma(w.wN, u[p + dp], s);
  if (DIM == 3) {
    s = fma(w.wB, u[p - (IT)L.plane], s);
    s = fma(w.wF, u[p + (IT)L.plane], s);
  }
  return s;
}

// y-line across a periodic direction (every row an unknown): a cyclic tridiagonal system, solved
// by Sherman-Morrison.  With gamma = -D_0, A = T + u v^T where T drops the two corner couplings
// (beta = -w_S of row 0, alpha = -w_N of row n1-1) and carries D_0 - gamma and
// D_{n1-1} - alpha beta / gamma on its diagonal, u = (gamma, 0, .., 0, alpha),
// v = (1, 0, .., 0, beta / gamma); x = y - (v.y / (1 + v.z)) z with T y = r and T z = u.
// The two Thomas solves share the elimination; zps holds the second one's right-hand side.
// Used by the one-thread-per-line kernel and the single-CTA coarse kernel (cps, dps, zps:
// three arrays of the level's layout, which may be the output array for dps).
template <typename T, int DIM, int KIND>
__device__ __forceinline__ void cyclic_yline(const Lev<T> &L, long long base, int i, const T *u, const T *g, T *out,
                                             T omega, T *cps, T *dps, T *zps) {
  const int m = L.n1;
  const long long stride = L.pitch;
#ifdef MG_DEBUG
  {   // the line's first and last nodes (every access of the three passes lies between them)
    const long long n = L.plane * (L.dim == 3 ? L.n2 : 1);
    const unsigned site = (15u << 16) | (unsigned)__LINE__;
    if (!mg_ck_n(L, base, n, site) || !mg_ck_n(L, base + (m - 1) * stride, n, site)) return;
  }
#endif
  T beta = T(0), gamma = T(1), cprev = T(0), yprev = T(0), zprev = T(0);
  for (int s = 0; s < m; ++s) {
    long long p = base + s * stride;
    long long dm, dp;
    yoffs(L, s, dm, dp);
    Weights<T, DIM, KIND> w;
    w.load(L, i, p, dm);
    T r = residual_at<T, DIM, KIND>(L, w, u, p, dm, dp, g[p]);
    T D = (w.wW + w.wE) + (w.wS + w.wN);
    if (DIM == 3) D += w.wB + w.wF;
    if (KIND == K_CONST) D = L.d;
    T lo = s > 0 ? -w.wS : T(0);
    T up = s < m - 1 ? -w.wN : T(0);
    T uz = T(0);
    if (s == 0) {
      beta = -w.wS;
      gamma = -D;
      D = D - gamma;
      uz = gamma;
    }
    if (s == m - 1) {
      const T alpha = -w.wN;
      D = D - alpha * beta / gamma;
      uz = alpha;
    }
    T den = D - lo * cprev;
    T cp = up / den;
    T yv = (r - lo * yprev) / den;
    T zv = (uz - lo * zprev) / den;
    cps[p] = cp;
    dps[p] = yv;
    zps[p] = zv;
    cprev = cp;
    yprev = yv;
    zprev = zv;
  }
  T y = T(0), z = T(0), y0 = T(0), z0 = T(0), ylast = T(0), zlast = T(0);
  for (int s = m - 1; s >= 0; --s) {
    long long p = base + s * stride;
    y = dps[p] - cps[p] * y;
    z = zps[p] - cps[p] * z;
    dps[p] = y;
    zps[p] = z;
    if (s == m - 1) { ylast = y; zlast = z; }
    if (s == 0) { y0 = y; z0 = z; }
  }
  const T fac = (y0 + beta / gamma * ylast) / (T(1) + z0 + beta / gamma * zlast);
  for (int s = 0; s < m; ++s) {
    long long p = base + s * stride;
    const T x = dps[p] - fac * zps[p];
    out[p] = fma(omega, x, u[p]);
  }
}

// ---------------------------------------------------------------------------------------
// launchers (defined in the kernel translation units)
// ---------------------------------------------------------------------------------------

// Per-kernel trace of a solve (MG_FLAG_TRACE): an event recorded on the launch stream after every
// kernel, with the launcher's name and the level being processed.  The time between two
// consecutive marks is the later kernel's time on the GPU timeline (launch latency included).
struct Tracer {
  cudaEvent_t *ev = nullptr;
  const char **label = nullptr;
  int *lev = nullptr;
  int cap = 0, n = 0;
  int level = 0;   // level the schedule is working on (set by the host-side cycle)
  bool capture = false;   // marks become event-record nodes of a graph being captured
  void mark(cudaStream_t s, const char *what) {
    if (n >= cap) return;
    if (capture) cudaEventRecordWithFlags(ev[n], s, cudaEventRecordExternal);
    else cudaEventRecord(ev[n], s);
    label[n] = what;
    lev[n++] = level;
  }
};

struct Launch {
  cudaStream_t s;
  long long *counter;   // incremented once per kernel launch
  Tracer *tr = nullptr; // MG_FLAG_TRACE: marks after every launch
  void done(const char *what) const {
    ++*counter;
    if (tr) tr->mark(s, what);
  }
};

template <typename T>
void launch_jacobi(const Launch &lc, const Lev<T> &L, int kind, const T *u, const T *g, T *out, T omega);
template <typename T>
void launch_jacobi_zero(const Lev<T> &L, int kind, const Launch &lc, const T *g, T *out, T omega);
template <typename T>
void launch_rb_half(const Launch &lc, const Lev<T> &L, int kind, T *u, const T *g, T omega, int colour);
// Gauss-Seidel on a 2-D Galerkin level: the nodes of colour (i mod 2, j mod 2) = (ci, cj), in place
template <typename T>
void launch_gs9_colour(const Launch &lc, const Lev<T> &L, T *u, const T *g, T omega, int ci, int cj);
template <typename T>
void launch_defect(const Launch &lc, const Lev<T> &L, int kind, const T *u, const T *g, T *r);
// sum of squares over the unknowns -> *out_sq (deterministic: per-block partials, fixed-order finish)
template <typename T>
void launch_defect_norm(const Launch &lc, const Lev<T> &L, int kind, const T *u, const T *g, double *partials,
                        int nparts, double *out_sq);
template <typename T>
void launch_norm_parts(const Launch &lc, const Lev<T> &L, const T *v, double *partials, int nparts, double *out_sq);
template <typename T>
void launch_restrict(const Launch &lc, const Lev<T> &F, const Lev<T> &C, const T *rf, T *gc);
template <typename T>
void launch_prolong_add(const Launch &lc, const Lev<T> &F, const Lev<T> &C, const T *ec, T *uf, T w);
// line smoother (dir 0: x lines, 1: y lines); zebra = 1 updates the lines of one colour in
// place (out == u), zebra = 0 is line Jacobi (out != u).  s1, s2: scratch arrays of the level;
// s3: a third one for y-lines across a periodic y (cyclic systems), else unused.
template <typename T>
void launch_line(const Launch &lc, const Lev<T> &L, int kind, int dir, int zebra, int colour, const T *u,
                 const T *g, T *out, T omega, T *s1, T *s2,
                 T *s3);

int norm_parts_count();
// a reduction over rows of this many unknowns fits in nparts block partial sums
bool norm_shape_ok(long long xunknowns, int nparts);
void launch_norm_finish(const Launch &lc, const double *partials, int nparts, double *out_sq);

// coarsest grid: u = A^{-1} g with a dense inverse (FP64), I/O in T
template <typename T>
void launch_coarse_apply(const Launch &lc, const double *Ainv, const long long *cidx, int nc, const T *g, T *u);
template <typename T>
void launch_assemble_dense(const Launch &lc, const Lev<T> &L, int kind, const long long *cidx, const int *cmap,
                           int nc, double *A);
void launch_gj_step(const Launch &lc, double *A, double *col, int n, int kstep);

// fused 2-D kernels (kernels_fast.cu): a whole red-black sweep out of place (mode 0: plain,
// 1: from a zero iterate, 2: u + omega_corr P ec applied while staging u), and the defect
// fused with full-weighting restriction
template <typename T>
void launch_rb2d(const Launch &lc, const Lev<T> &L, int kind, const T *u, const T *g, T *out, T omega, int first,
                 int mode, const Lev<T> *C, const T *ec, T omega_corr);
// two complete sweeps in one pass (temporal blocking, small grids); mode applies to the first
template <typename T>
void launch_rb2d_2(const Launch &lc, const Lev<T> &L, int kind, const T *u, const T *g, T *out, T omega, int first,
                   int mode, const Lev<T> *C, const T *ec, T omega_corr);
// two sweeps, then the defect and its full-weighting restriction into the coarse g, in one pass
// (small grids; mode 0 or 1)
template <typename T>
void launch_rb2d_2_dr(const Launch &lc, const Lev<T> &L, const Lev<T> &C, int kind, const T *u, const T *g, T *out,
                      T omega, int first, int mode, T *gc);
template <typename T>
void launch_defect_restrict2d(const Launch &lc, const Lev<T> &F, const Lev<T> &C, int kind, const T *u, const T *g,
                              T *gc);
// column-marching form of launch_rb2d (kernels_march.cu) for constant / separable
// coefficients; returns false (nothing launched) where it does not apply
template <typename T>
bool launch_rb2d_march(const Launch &lc, const Lev<T> &L, int kind, const T *u, const T *g, T *out, T omega,
                       int first, int mode, const Lev<T> *C, const T *ec, T omega_corr);

// the same sweep in FP32 with rows streamed by TMA bulk copies into a shared-memory ring
// (kernels_tma.cu); rc = rows per warp (0: default).  A wait that gives up sets *err.
// Returns false (nothing launched) where it does not apply.
bool launch_rb2d_tma(const Launch &lc, const Lev<float> &L, int kind, const float *u, const float *g, float *out,
                     float omega, int first, int mode, const Lev<float> *C, const float *ec, float omega_corr,
                     int *err, int rc,
                     int *inject = nullptr);
size_t rb2d_tma_smem(int mode);
// the fused defect + full-weighting restriction (2-D, FP32, constant or separable
// coefficients) streamed the same way; rc = coarse rows per CTA (0: from the occupancy)
bool launch_defect_restrict_tma(const Launch &lc, const Lev<float> &L, const Lev<float> &C, int kind,
                                const float *u, const float *g, float *gc, int *err, int rc);

// single-CTA coarse cycle (kernels_coarse.cu): levs = device table of shared-memory level
// views (filled by coarse_fill_levels), prog = program of CoarseOp steps
template <typename T>
void launch_coarse_cycle(const Launch &lc, int dim, int kind, const void *levs, const int4 *prog, int nops, int lcut,
                         const T *g_in, const T *u_in, T *u_out, const double *Ainv, const long long *cidx_smem,
                         int nc, T omega, T omega_corr, size_t smem_bytes,
                         bool full);
template <typename T>
size_t coarse_slev_size();
template <typename T>
size_t coarse_fill_levels(void *out, int lcut, const Lev<T> *glev, const long long *gpitch, const long long *gplane,
                          int kind, bool zscratch);

// setup
void launch_coarsen_sep(const Launch &lc, const double *fsx, const double *fsy, const double *fsz, int nf0,
                        double *csx, double *csy, double *csz, int nc0);
void launch_sep_dinv(const Launch &lc, const double *sx, const double *sy, const double *sz, int n0, int dim,
                     double *dinv);
void launch_coarsen_cell(const Launch &lc, const Lev<double> &F, const Lev<double> &C, const double *kf, double *kc);
void launch_cell_dinv(const Launch &lc, const Lev<double> &L, double *dinv);
// coarsest grid by FP64 conjugate gradients (one cooperative launch): u = A^{-1} g on level L to
// ||r|| <= rtol ||g||, at most max_it iterations.  work: 4 FP64 node arrays of L, zero off the
// unknowns; part: 2 x (blocks) doubles of scratch; iters[0] = the iterations done
template <typename T>
void launch_coarse_cg(const Launch &lc, const Lev<double> &L, int kind, const T *g, T *u, double *work, double *part,
                      int max_it, double rtol, int *iters);
// edge coefficients: coarse weights from the fine ones (harmonic mean along, x1/4), and 1/D
void launch_coarsen_edge(const Launch &lc, const Lev<double> &F, const Lev<double> &C, const double *fx,
                         const double *fy, const double *fz, double *cx, double *cy, double *cz);
void launch_edge_dinv(const Launch &lc, const Lev<double> &L, double *dinv);
// Galerkin coarse operator R A P of fine level F (kind fkind, 2-D, y not periodic) on coarse level C:
// diagonal, +x / +y / +x+y / -x+y weights (w = -A) and 1/D per coarse node
void launch_rap(const Launch &lc, const Lev<double> &F, int fkind, const Lev<double> &C, double *dg, double *ex,
                double *ey, double *ene, double *enw, double *dinv);
void launch_to_float(const Launch &lc, const double *src, float *dst, long long n);
void launch_cell_pack(const Launch &lc, const Lev<double> &L, const double *src_compact, double *dst);
void launch_cell_unpack(const Launch &lc, const Lev<double> &L, const double *src, double *dst_compact);

// copies between compact user arrays and the padded layout
template <typename T>
void launch_pack(const Launch &lc, const Lev<T> &L, const double *src, T *dst, int zero_boundary);
template <typename T>
void launch_unpack(const Launch &lc, const Lev<T> &L, const T *src, double *dst, double scale);
template <typename T>
void launch_zero_level(const Launch &lc, const Lev<T> &L, T *dst);
template <typename T>
void launch_zero_boundary(const Launch &lc, const Lev<T> &L, T *dst);
// axis-swapped copies: caller node (i, j, k) <-> internal node (j, i, k)
template <typename T>
void launch_pack_swapped(const Launch &lc, const Lev<T> &L, const double *src, T *dst, int zero_boundary);
template <typename T>
void launch_unpack_swapped(const Launch &lc, const Lev<T> &L, const T *src, double *dst, double scale);
void launch_cell_pack_swapped(const Launch &lc, const Lev<double> &L, const double *src_compact, double *dst);
void launch_cell_unpack_swapped(const Launch &lc, const Lev<double> &L, const double *src, double *dst_compact);
// x-line smoother, one CTA per line; returns false (nothing launched) for lines longer than it holds
template <typename T>
bool launch_xline(const Launch &lc, const Lev<T> &L, int kind, int zebra, int colour, const T *u, const T *g, T *out,
                  T omega);

// mixed precision
void launch_defect64_to32(const Launch &lc, const Lev<double> &L, int kind, const double *x, const double *b,
                          float *r32, double *partials, int nparts, double *out_sq);
void launch_ir_update(const Launch &lc, const Lev<double> &L, double *x, const float *c);
// the same outer defect in float-float arithmetic on the FP32 and integer pipes (2-D, constant or
// separable coefficients; false, and nothing launched, otherwise).  out_t: the sum of squares of
// |b| + |A||x| over the unknowns, the scale of the float-float error (0 in FP64 mode); use64:
// device flag (null: never set) that makes the kernel evaluate the defect in FP64 instead
// c32 != null: the refinement update is fused in -- the iterate is double-buffered (xa, xb; *par
// selects the current one), the defect is that of x + c, which is written into the other buffer,
// and *par flips; c32 == null: the defect of xa (xb and par unused)
bool launch_defect_ff(const Launch &lc, const Lev<double> &L, int kind, double *xa, double *xb, const double *b,
                      float *r32, double *partials, int nparts, double *out_sq, double *out_t, const int *use64,
                      const float *c32 = nullptr, int *par = nullptr);
// the iterate back into xa after fused updates (a copy when *par is set), then *par = 0
void launch_x_settle(const Launch &lc, double *xa, const double *xb, long long n, int *par);
// after a loop stopped on the float-float defect: its FP64 relative residual into hist[st[0]], status 8
// when it stopped as converged but the FP64 residual is above tol
void launch_final_check(const Launch &lc, const double *sq, const double *bsq, double *hist, int *st,
                        const double *tol);
// adaptive correction weight: omega = (g - A u, pe) / (A pe, pe) over the unknowns of L
// (pe = P e, zero off the unknowns), written to *omega; partials: nparts doubles of scratch;
// count: a device counter that is zero between launches (the kernel re-arms it)
template <typename T>
void launch_corr_weight(const Launch &lc, const Lev<T> &L, int kind, const T *u, const T *g, const T *pe,
                        double *partials, int nparts, unsigned *count, double *omega);
// out = P ec on every node of F (zero off the unknowns of F)
template <typename T>
void launch_interp(const Launch &lc, const Lev<T> &F, const Lev<T> &C, const T *ec, T *out);
// e[0..n) *= *omega
template <typename T>
void launch_scale_by(const Launch &lc, T *e, long long n, const double *omega);

// gradient with respect to the cell field
void launch_grad_k(const Launch &lc, const Lev<double> &L, const double *u, const double *lam, double *dk);

// finish kernel: relres = sqrt(sq) / bnorm, history, status word
void launch_relres(const Launch &lc, const double *sq, const double *bsq, double *hist, int it, double *relres_out);
// dst[0] = sqrt(src[0])
void launch_sqrt(const Launch &lc, const double *src, double *dst);
// test hook of the -DMG_DEBUG build: a bounds check one past the level's last node (no access)
void launch_bounds_probe(const Launch &lc, const Lev<double> &L);
// end of a cycle of a device-side solve loop: history, cycle count, status, WHILE condition.
// After a float-float defect (tsq: its sum of squares of |b| + |A||x|; null otherwise) the loop
// stops only when the residual is below tol by the estimated error E = ff_err * sqrt(tsq), and
// sets st[6] (FP64 defects from the next step on) when E >= tol / 2, when the residual is within
// ff_switch * E of tol, or when it fell by less than half in the step
void launch_step_end(const Launch &lc, cudaGraphConditionalHandle h, const double *sq, const double *bsq,
                     double *hist, int *st, const double *tol, int maxit, int init, const double *tsq = nullptr,
                     double ff_err = 0.0, double ff_switch = 0.0);

}  // namespace mg
