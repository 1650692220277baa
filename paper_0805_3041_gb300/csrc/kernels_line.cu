// kernels_line.cu -- line smoothers: C = tridiagonal part of A along x or y lines
// (Wallis 2008, section "The choice of C": "Tri diagonal C"; TRIx / TRIy, and
// the line Gauss-Seidel GSTRI of the preconditioner memory table), applied as
// x <- x + omega C^{-1}(b - A x).  Line Jacobi updates every line from the old
// iterate (out of place); the zebra form updates the lines of one colour in
// place (colour = parity of the orthogonal index sum), which only reads lines
// of the other colour.
//
// One thread per line: defect at the line's nodes, Thomas forward elimination
// (modified coefficients kept in two scratch arrays of the level's layout),
// back substitution.  y-lines are read fully coalesced (adjacent threads own
// adjacent columns).
#include "mg_internal.cuh"

namespace mg {

// y-line across a periodic direction (every row an unknown): a cyclic tridiagonal system, solved
// by Sherman-Morrison.  With gamma = -D_0, A = T + u v^T where T drops the two corner couplings
// (beta = -w_S of row 0, alpha = -w_N of row n1-1) and carries D_0 - gamma and
// D_{n1-1} - alpha beta / gamma on its diagonal, u = (gamma, 0, .., 0, alpha),
// v = (1, 0, .., 0, beta / gamma); x = y - (v.y / (1 + v.z)) z with T y = r and T z = u.
// The two Thomas solves share the elimination; zps holds the second one's right-hand side.
template <typename T, int DIM, int KIND>
__device__ __forceinline__ void cyclic_yline(const Lev<T> &L, long long base, int i, const T *u, const T *g, T *out,
                                             T omega, T *cps, T *dps, T *zps) {
  const int m = L.n1;
  const long long stride = L.pitch;
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

template <typename T, int DIM, int KIND>
__global__ void k_line(Lev<T> L, int dir, int zebra, int colour, const T *u, const T *__restrict__ g, T *out, T omega,
                       T *__restrict__ cps, T *__restrict__ dps, T *__restrict__ zps) {
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
    x = dps[p] - cps[p] * x;
    out[p] = fma(omega, x, u[p]);
  }
}

template <typename T>
void launch_line(const Launch &lc, const Lev<T> &L, int kind, int dir, int zebra, int colour, const T *u,
                 const T *g, T *out, T omega, T *s1, T *s2, T *s3) {
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
  ++*lc.counter;
}

template void launch_line<double>(const Launch &, const Lev<double> &, int, int, int, int, const double *,
                                  const double *, double *, double, double *, double *, double *);
template void launch_line<float>(const Launch &, const Lev<float> &, int, int, int, int, const float *, const float *,
                                 float *, float, float *, float *, float *);

}  // namespace mg
