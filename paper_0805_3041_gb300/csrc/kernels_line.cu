// kernels_line.cu -- line smoothers: C = tridiagonal part of A along x or y lines
// (Wallis 2008, section "The choice of C": "Tri diagonal C"; TRIx / TRIy, and
// the line Gauss-Seidel GSTRI of the preconditioner memory table), applied as
// x <- x + omega C^{-1}(b - A x).  Line Jacobi updates every line from the old
// iterate (out of place); the zebra form updates the lines of one colour in
// place (colour = parity of the orthogonal index sum), which only reads lines
// of the other colour.
//
// y-lines, by length (m unknowns a line; rows are read coalesced, adjacent
// threads owning adjacent columns):
// - 4 <= m <= 2048: k_yline_reg, segments in registers, the reduced system by
//   parallel cyclic reduction in shared memory;
// - m > 2048: k_yline_part, segments through three scratch arrays;
// - m < 4 (and x-lines the dedicated x-line kernels do not take): k_line, one
//   thread per line, Thomas with two scratch arrays of the level's layout.
#define MG_FILE_ID 3   // bounds-check sites (-DMG_DEBUG)
#include "mg_internal.cuh"

namespace mg {

template <typename T, int DIM, int KIND>
__global__ void k_line(Lev<T> L, int dir, int zebra, int colour, const T *u, const T *__restrict__ g, T *out, T omega,
                       T *__restrict__ cps, T *__restrict__ dps, T *__restrict__ zps) {
  MG_PDL_WAIT();
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int m;
  long long base, stride;
  int a_fixed, b_fixed;   // the two orthogonal indices of the line
  if (dir == 0) {
    long long nr = L.unk_rows();
    if (t >= nr) return;
    int j, k;
    row_jk(L, t, j, k);
    if (zebra && ((j + k) & 1) != colour) return;
    m = L.n0 - 2;
    base = (long long)k * L.plane + (long long)j * L.pitch + 1;
    stride = 1;
    a_fixed = j;
    b_fixed = k;
  } else {
    int nx = L.n0 - 2;
    long long nl = (long long)nx * L.zrows();
    if (t >= nl) return;
    int i = 1 + (int)(t % nx), k = (DIM == 3 ? 1 : 0) + (int)(t / nx);
    if (zebra && ((i + k) & 1) != colour) return;
    if (L.per) {   // every row is an unknown: the cyclic system
      cyclic_yline<T, DIM, KIND>(L, (long long)k * L.plane + i, i, u, g, out, omega, cps, dps, zps);
      return;
    }
    m = L.n1 - 2;
    base = (long long)k * L.plane + L.pitch + i;
    stride = L.pitch;
    a_fixed = i;
    b_fixed = k;
  }
  (void)b_fixed;
  // forward elimination
  T cprev = T(0), dprev = T(0);
  for (int s = 0; s < m; ++s) {
    long long p = base + s * stride;
    int i = dir == 0 ? 1 + s : a_fixed;
    int j = dir == 0 ? a_fixed : 1 + s;
    long long dm, dp;
    yoffs(L, j, dm, dp);
    if (!MG_CK(L, p) || !MG_CK(L, p + dm)) return;   // debug build: the line leaves the array
    Weights<T, DIM, KIND> w;
    w.load(L, i, p, dm);
    T r = residual_at<T, DIM, KIND>(L, w, u, p, dm, dp, g[p]);
    T D = (w.wW + w.wE) + (w.wS + w.wN);
    if (DIM == 3) D += w.wB + w.wF;
    if (KIND == K_CONST) D = L.d;
    T lo = (s > 0) ? -(dir == 0 ? w.wW : w.wS) : T(0);
    T up = (s < m - 1) ? -(dir == 0 ? w.wE : w.wN) : T(0);
    T den = D - lo * cprev;
    T cp = up / den;
    T dpv = (r - lo * dprev) / den;
    cps[p] = cp;
    dps[p] = dpv;
    cprev = cp;
    dprev = dpv;
  }
  // back substitution and update
  T x = T(0);
  for (int s = m - 1; s >= 0; --s) {
    long long p = base + s * stride;
    if (!MG_CK(L, p)) return;   // debug build
    x = dps[p] - cps[p] * x;
    out[p] = fma(omega, x, u[p]);
  }
}

// Node of row s (0-based unknown index) of the y-line through column i of plane offset pl.
template <typename T>
__device__ __forceinline__ long long yline_node(const Lev<T> &L, long long pl, int i, bool per, int s) {
  return pl + (long long)(per ? s : s + 1) * L.pitch + i;
}

// Row s of the y-line through column i (m unknowns): a x_{s-1} + b x_s + c x_{s+1} = d, with d
// the defect at the node and the couplings across a periodic y wrapping round.
template <typename T, int DIM, int KIND>
__device__ __forceinline__ void yline_row(const Lev<T> &L, long long pl, int i, bool per, int m, int s, const T *u,
                                          const T *__restrict__ g, T &a, T &b, T &c, T &d) {
  const int j = per ? s : s + 1;
  const long long p = yline_node(L, pl, i, per, s);
  long long dm, dp;
  yoffs(L, j, dm, dp);
  if (!MG_CK(L, p) || !MG_CK(L, p + dm)) {   // debug build: a neutral row instead of the access
    a = c = d = T(0);
    b = T(1);
    return;
  }
  Weights<T, DIM, KIND> w;
  w.load(L, i, p, dm);
  d = residual_at<T, DIM, KIND>(L, w, u, p, dm, dp, g[p]);
  T D = (w.wW + w.wE) + (w.wS + w.wN);
  if (DIM == 3) D += w.wB + w.wF;
  b = KIND == K_CONST ? L.d : D;
  a = (per || s > 0) ? -w.wS : T(0);
  c = (per || s < m - 1) ? -w.wN : T(0);
}

// y-lines by the partition method.  A CTA takes 32 adjacent lines (one column each: rows are
// read coalesced) and YSEG segments of each line, one thread per segment.  A thread eliminates
// its segment down to two equations in the segment's end unknowns (forward elimination keeping
// the first unknown, then backward elimination keeping both ends), with the interior rows'
// coefficients in three scratch arrays; one thread per line then solves the 2 * YSEG reduced
// equations (cyclic when y is periodic: Sherman-Morrison as in cyclic_yline), and every thread
// recovers its interior unknowns.  Lines need >= 2 * YSEG unknowns.
// YC = 32 columns x YSEG = 16 segments; used for lines longer than k_yline_reg takes.
template <typename T, int DIM, int KIND, int YC, int YSEG>
__global__ void __launch_bounds__(YC * YSEG) k_yline_part(Lev<T> L, int zebra, int colour, const T *u,
                                                          const T *__restrict__ g, T *out, T omega,
                                                          T *__restrict__ sap, T *__restrict__ scp,
                                                          T *__restrict__ sdp) {
  MG_PDL_WAIT();
  constexpr int NE = 2 * YSEG;
  __shared__ T ra[NE][YC + 1], rb[NE][YC + 1], rc[NE][YC + 1], rd[NE][YC + 1], rz[NE][YC + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int k = DIM == 3 ? 1 + (int)blockIdx.y : 0;
  const int nx = L.n0 - 2;
  int i;
  if (zebra) {
    const int par = (((1 + k) & 1) == colour) ? 0 : 1;   // first column of this colour: 1 + par
    i = 1 + par + 2 * ((int)blockIdx.x * YC + tx);
  } else {
    i = 1 + (int)blockIdx.x * YC + tx;
  }
  const bool act = i <= nx;
  const bool per = L.per != 0;
  const int m = per ? L.n1 : L.n1 - 2;
  const int base_n = m / YSEG, extra = m % YSEG;
  const int n = base_n + (ty < extra ? 1 : 0);
  const int s0 = ty * base_n + (ty < extra ? ty : extra);
  const long long plane = (long long)k * L.plane;
  auto rowp = [&](int s) -> long long { return yline_node(L, plane, i, per, s); };
  auto coef = [&](int s, T &a, T &b, T &c, T &d) { yline_row<T, DIM, KIND>(L, plane, i, per, m, s, u, g, a, b, c, d); };
  T ta = T(0), tb = T(1), tc = T(0), td = T(0), ba = T(0), bb = T(1), bc = T(0), bd = T(0);
  if (act) {
    T a0, b0, c0, d0;
    coef(s0, a0, b0, c0, d0);
    T app = T(0), cpp = T(0), dpp = T(0);
    for (int q = 1; q < n; ++q) {
      T a, b, c, d;
      coef(s0 + q, a, b, c, d);
      T ap, cp, dv;
      if (q == 1) {
        const T r = T(1) / b;
        ap = a * r;
        cp = c * r;
        dv = d * r;
      } else {
        const T r = T(1) / (b - a * cpp);
        ap = -r * a * app;
        cp = r * c;
        dv = r * (d - a * dpp);
      }
      const long long p = rowp(s0 + q);
      if (!MG_CK(L, p)) continue;   // debug build
      sap[p] = ap;
      scp[p] = cp;
      sdp[p] = dv;
      app = ap;
      cpp = cp;
      dpp = dv;
    }
    ba = app;   // bottom: ap x_first + x_last + cp x_next = dp
    bc = cpp;
    bd = dpp;
    // backward elimination keeping both ends: x_q = dp_q - ap_q x_first - cp_q x_last (1 <= q <= n-2)
    T an = app, cn = cpp, dn = dpp;   // row q+1, starting at q+1 = n-1
    for (int q = n - 2; q >= 1; --q) {
      const long long p = rowp(s0 + q);
      if (!MG_CK(L, p)) continue;   // debug build
      T aq = sap[p], cq = scp[p], dq = sdp[p];
      if (q <= n - 3) {
        dq = dq - cq * dn;
        aq = aq - cq * an;
        cq = -cq * cn;
        sap[p] = aq;
        scp[p] = cq;
        sdp[p] = dq;
      }
      an = aq;
      cn = cq;
      dn = dq;
    }
    ta = a0;
    if (n == 2) {
      tb = b0;
      tc = c0;
      td = d0;
    } else {   // row 1 of the segment, eliminated: x_1 = dn - an x_first - cn x_last
      tb = b0 - c0 * an;
      tc = -c0 * cn;
      td = d0 - c0 * dn;
    }
  }
  ra[2 * ty][tx] = ta; rb[2 * ty][tx] = tb; rc[2 * ty][tx] = tc; rd[2 * ty][tx] = td;
  ra[2 * ty + 1][tx] = ba; rb[2 * ty + 1][tx] = bb; rc[2 * ty + 1][tx] = bc; rd[2 * ty + 1][tx] = bd;
  __syncthreads();
  if (ty == 0 && act) {   // the reduced line system of this column: NE equations
    T alpha = T(0), beta = T(0), gamma = T(1);
    if (per) {   // corners: equation 0 couples to the last unknown, the last to unknown 0
      beta = ra[0][tx];
      alpha = rc[NE - 1][tx];
      gamma = -rb[0][tx];
      rb[0][tx] -= gamma;
      rb[NE - 1][tx] -= alpha * beta / gamma;
      ra[0][tx] = T(0);
      rc[NE - 1][tx] = T(0);
    }
    // Thomas on the (modified) tridiagonal system; z: right-hand side (gamma, 0, .., 0, alpha)
    T cprev = T(0), dprev = T(0), zprev = T(0);
    for (int e = 0; e < NE; ++e) {
      const T a = ra[e][tx];
      const T den = rb[e][tx] - a * cprev;
      const T cp = rc[e][tx] / den;
      const T dv = (rd[e][tx] - a * dprev) / den;
      const T uz = per ? (e == 0 ? gamma : (e == NE - 1 ? alpha : T(0))) : T(0);
      const T zv = (uz - a * zprev) / den;
      rc[e][tx] = cp;
      rd[e][tx] = dv;
      rz[e][tx] = zv;
      cprev = cp;
      dprev = dv;
      zprev = zv;
    }
    T y = T(0), z = T(0);
    for (int e = NE - 1; e >= 0; --e) {
      y = rd[e][tx] - rc[e][tx] * y;
      z = rz[e][tx] - rc[e][tx] * z;
      rd[e][tx] = y;
      rz[e][tx] = z;
    }
    if (per) {
      const T fac = (rd[0][tx] + beta / gamma * rd[NE - 1][tx]) / (T(1) + rz[0][tx] + beta / gamma * rz[NE - 1][tx]);
      for (int e = 0; e < NE; ++e) rd[e][tx] -= fac * rz[e][tx];
    }
  }
  __syncthreads();
  if (!act) return;
  const T x0 = rd[2 * ty][tx], xl = rd[2 * ty + 1][tx];
  for (int q = 0; q < n; ++q) {
    const long long p = rowp(s0 + q);
    if (!MG_CK(L, p)) continue;   // debug build
    const T x = q == 0 ? x0 : (q == n - 1 ? xl : sdp[p] - sap[p] * x0 - scp[p] * xl);
    out[p] = fma(omega, x, u[p]);
  }
}

// y-lines with every segment held in registers.  A CTA of blockDim = (YC, YSEG) threads takes YC
// lines (adjacent columns of one colour) and cuts each into YSEG segments of at most NR rows.
// A thread loads its segment's rows at once, eliminates them in registers to two equations in
// the segment's end unknowns (as k_yline_part does), and the 2 * YSEG reduced equations of a line
// are solved by parallel cyclic reduction in shared memory, two equations per thread.  The
// reduction runs with wrap-around indices: that is the periodic line system itself, and with
// its two corner couplings zero it is the Dirichlet one, so one code path serves both (2 * YSEG
// is a power of two).  Equations are kept scaled to a unit diagonal.  After log2(2 * YSEG)
// steps every equation couples only to its own unknown.  The interior unknowns then follow from
// the end values.  No scratch arrays; every row is read once and written once.
constexpr int kYlineThreads = 512;
constexpr int kYlineSegMax = 256;
constexpr int kYlineShared = 2 * kYlineThreads + 2 * kYlineSegMax;   // >= 2 YSEG (YC + 1)

template <typename T, int DIM, int KIND, int NR>
__global__ void __launch_bounds__(kYlineThreads, sizeof(T) == 4 ? 2 : 1)
    k_yline_reg(Lev<T> L, int zebra, int colour, const T *u, const T *__restrict__ g, T *out, T omega) {
  MG_PDL_WAIT();
  __shared__ T sa[kYlineShared], sc[kYlineShared], sd[kYlineShared];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int YC = (int)blockDim.x, YSEG = (int)blockDim.y, NE = 2 * YSEG, ld = YC + 1;
  const int k = DIM == 3 ? 1 + (int)blockIdx.y : 0;
  int i;
  if (zebra) {
    const int par = (((1 + k) & 1) == colour) ? 0 : 1;   // first column of this colour: 1 + par
    i = 1 + par + 2 * ((int)blockIdx.x * YC + tx);
  } else {
    i = 1 + (int)blockIdx.x * YC + tx;
  }
  const bool act = i <= L.n0 - 2;
  const bool per = L.per != 0;
  const int m = per ? L.n1 : L.n1 - 2;
  const int base_n = m / YSEG, extra = m % YSEG;
  const int n = base_n + (ty < extra ? 1 : 0);   // 2 <= n <= NR
  const int s0 = ty * base_n + (ty < extra ? ty : extra);
  const long long plane = (long long)k * L.plane;
  T ra[NR], rb[NR], rc[NR], rd[NR];
  // the two reduced equations of the segment, scaled to a unit diagonal: a x_{e-1} + x_e + c x_{e+1} = d
  T a0 = T(0), c0 = T(0), d0 = T(0), a1 = T(0), c1 = T(0), d1 = T(0);
  if (act) {
#pragma unroll
    for (int q = 0; q < NR; ++q)
      if (q < n) yline_row<T, DIM, KIND>(L, plane, i, per, m, s0 + q, u, g, ra[q], rb[q], rc[q], rd[q]);
    // forward elimination keeping the first unknown: ap x_first + x_q + cp x_{q+1} = dp (q >= 1)
    T app = T(0), cpp = T(0), dpp = T(0);
#pragma unroll
    for (int q = 1; q < NR; ++q) {
      if (q < n) {
        T ap, cp, dv;
        if (q == 1) {
          const T r = T(1) / rb[1];
          ap = ra[1] * r;
          cp = rc[1] * r;
          dv = rd[1] * r;
        } else {
          const T r = T(1) / (rb[q] - ra[q] * cpp);
          ap = -r * ra[q] * app;
          cp = r * rc[q];
          dv = r * (rd[q] - ra[q] * dpp);
        }
        ra[q] = ap;
        rc[q] = cp;
        rd[q] = dv;
        app = ap;
        cpp = cp;
        dpp = dv;
      }
    }
    a1 = app;   // bottom: x_first, x_last and the next segment's first unknown
    c1 = cpp;
    d1 = dpp;
    // backward elimination keeping both ends: x_q + ap x_first + cp x_last = dp (1 <= q <= n-2)
    T an = app, cn = cpp, dn = dpp;
#pragma unroll
    for (int q = NR - 2; q >= 1; --q) {
      if (q <= n - 2) {
        if (q <= n - 3) {
          rd[q] -= rc[q] * dn;
          ra[q] -= rc[q] * an;
          rc[q] = -rc[q] * cn;
        }
        an = ra[q];
        cn = rc[q];
        dn = rd[q];
      }
    }
    // top: the previous segment's last unknown, x_first and x_last (row 1 eliminated)
    T tb = rb[0], tc = rc[0], td = rd[0];
    if (n > 2) {
      tb = rb[0] - rc[0] * an;
      tc = -rc[0] * cn;
      td = rd[0] - rc[0] * dn;
    }
    const T r = T(1) / tb;
    a0 = ra[0] * r;
    c0 = tc * r;
    d0 = td * r;
  }
  const int e0 = 2 * ty;
  sa[e0 * ld + tx] = a0; sc[e0 * ld + tx] = c0; sd[e0 * ld + tx] = d0;
  sa[(e0 + 1) * ld + tx] = a1; sc[(e0 + 1) * ld + tx] = c1; sd[(e0 + 1) * ld + tx] = d1;
  if (act) {   // the centre values for the update, loaded while the reduced system is solved
#pragma unroll
    for (int q = 0; q < NR; ++q)
      if (q < n && MG_CK(L, yline_node(L, plane, i, per, s0 + q))) rb[q] = u[yline_node(L, plane, i, per, s0 + q)];
  }
  // parallel cyclic reduction: equation e takes in e - s and e + s, then couples to e -+ 2s
  for (int s = 1; s < NE; s <<= 1) {
    __syncthreads();
    const int m0 = ((e0 - s) & (NE - 1)) * ld + tx, p0 = ((e0 + s) & (NE - 1)) * ld + tx;
    const int m1 = ((e0 + 1 - s) & (NE - 1)) * ld + tx, p1 = ((e0 + 1 + s) & (NE - 1)) * ld + tx;
    const T r0 = T(1) / (T(1) - a0 * sc[m0] - c0 * sa[p0]);
    const T r1 = T(1) / (T(1) - a1 * sc[m1] - c1 * sa[p1]);
    const T na0 = -r0 * a0 * sa[m0], nc0 = -r0 * c0 * sc[p0], nd0 = r0 * (d0 - a0 * sd[m0] - c0 * sd[p0]);
    const T na1 = -r1 * a1 * sa[m1], nc1 = -r1 * c1 * sc[p1], nd1 = r1 * (d1 - a1 * sd[m1] - c1 * sd[p1]);
    __syncthreads();
    a0 = na0; c0 = nc0; d0 = nd0;
    a1 = na1; c1 = nc1; d1 = nd1;
    sa[e0 * ld + tx] = a0; sc[e0 * ld + tx] = c0; sd[e0 * ld + tx] = d0;
    sa[(e0 + 1) * ld + tx] = a1; sc[(e0 + 1) * ld + tx] = c1; sd[(e0 + 1) * ld + tx] = d1;
  }
  if (!act) return;
  // both couplings now point at the equation's own unknown
  const T x0 = d0 / (T(1) + a0 + c0), xl = d1 / (T(1) + a1 + c1);
#pragma unroll
  for (int q = 0; q < NR; ++q) {
    if (q < n && MG_CK(L, yline_node(L, plane, i, per, s0 + q))) {
      const T x = q == 0 ? x0 : (q == n - 1 ? xl : rd[q] - ra[q] * x0 - rc[q] * xl);
      out[yline_node(L, plane, i, per, s0 + q)] = fma(omega, x, rb[q]);
    }
  }
}

// Segments per line for k_yline_reg with at most nr rows a segment: the fewest segments (a power
// of two) that keep every segment within nr rows, provided each keeps at least two rows; 0 when the
// line needs more than kYlineSegMax segments.  The launch then packs 512 / segments lines a CTA.
static inline int yline_segments(int m, int nr) {
  int seg = 1;
  while (seg * nr < m) seg *= 2;
  return (seg <= kYlineSegMax && 2 * seg <= m) ? seg : 0;
}

template <typename T>
void launch_line(const Launch &lc, const Lev<T> &L, int kind, int dir, int zebra, int colour, const T *u,
                 const T *g, T *out, T omega, T *s1, T *s2, T *s3) {
  const int mrows = L.per ? L.n1 : L.n1 - 2;
  constexpr int NR = 8;
  const int seg = dir == 1 && mrows >= 4 ? yline_segments(mrows, NR) : 0;
  if (seg) {
    const int nx = L.n0 - 2;
    const int cols = zebra ? (nx + 1) / 2 : nx;
    int yc = 1;
    while (yc * seg < kYlineThreads && yc < cols) yc *= 2;
    dim3 gr((unsigned)((cols + yc - 1) / yc), (unsigned)L.zrows()), bl((unsigned)yc, (unsigned)seg);
#define YR(D, K) k_yline_reg<T, D, K, NR><<<gr, bl, 0, lc.s>>>(L, zebra, colour, u, g, out, omega)
    if (L.dim == 2) {
      if (kind == K_CONST) YR(2, K_CONST); else if (kind == K_SEP) YR(2, K_SEP); else if (kind == K_CELL) YR(2, K_CELL); else YR(2, K_EDGE);
    } else {
      if (kind == K_CONST) YR(3, K_CONST); else if (kind == K_SEP) YR(3, K_SEP); else if (kind == K_CELL) YR(3, K_CELL); else YR(3, K_EDGE);
    }
#undef YR
    lc.done(__func__);
    return;
  }
  if (dir == 1 && s3 && mrows >= 32) {
    const int nx = L.n0 - 2;
    const int cols = zebra ? (nx + 1) / 2 : nx;
    dim3 gr((unsigned)((cols + 31) / 32), (unsigned)L.zrows()), bl(32, 16);
#define YP(D, K) k_yline_part<T, D, K, 32, 16><<<gr, bl, 0, lc.s>>>(L, zebra, colour, u, g, out, omega, s3, s1, s2)
    if (L.dim == 2) {
      if (kind == K_CONST) YP(2, K_CONST); else if (kind == K_SEP) YP(2, K_SEP); else if (kind == K_CELL) YP(2, K_CELL); else YP(2, K_EDGE);
    } else {
      if (kind == K_CONST) YP(3, K_CONST); else if (kind == K_SEP) YP(3, K_SEP); else if (kind == K_CELL) YP(3, K_CELL); else YP(3, K_EDGE);
    }
#undef YP
    lc.done(__func__);
    return;
  }
  long long nlines = dir == 0 ? L.unk_rows() : (long long)(L.n0 - 2) * L.zrows();
  int th = 64;
  unsigned bl = (unsigned)((nlines + th - 1) / th);
  if (L.dim == 2) {
    if (kind == K_CONST) k_line<T, 2, K_CONST><<<bl, th, 0, lc.s>>>(L, dir, zebra, colour, u, g, out, omega, s1, s2, s3);
    else if (kind == K_SEP) k_line<T, 2, K_SEP><<<bl, th, 0, lc.s>>>(L, dir, zebra, colour, u, g, out, omega, s1, s2, s3);
    else if (kind == K_CELL) k_line<T, 2, K_CELL><<<bl, th, 0, lc.s>>>(L, dir, zebra, colour, u, g, out, omega, s1, s2, s3);
    else k_line<T, 2, K_EDGE><<<bl, th, 0, lc.s>>>(L, dir, zebra, colour, u, g, out, omega, s1, s2, s3);
  } else {
    if (kind == K_CONST) k_line<T, 3, K_CONST><<<bl, th, 0, lc.s>>>(L, dir, zebra, colour, u, g, out, omega, s1, s2, s3);
    else if (kind == K_SEP) k_line<T, 3, K_SEP><<<bl, th, 0, lc.s>>>(L, dir, zebra, colour, u, g, out, omega, s1, s2, s3);
    else if (kind == K_CELL) k_line<T, 3, K_CELL><<<bl, th, 0, lc.s>>>(L, dir, zebra, colour, u, g, out, omega, s1, s2, s3);
    else k_line<T, 3, K_EDGE><<<bl, th, 0, lc.s>>>(L, dir, zebra, colour, u, g, out, omega, s1, s2, s3);
  }
  lc.done(__func__);
}

template void launch_line<double>(const Launch &, const Lev<double> &, int, int, int, int, const double *,
                                  const double *, double *, double, double *, double *, double *);
template void launch_line<float>(const Launch &, const Lev<float> &, int, int, int, int, const float *, const float *,
                                 float *, float, float *, float *, float *);

}  // namespace mg
