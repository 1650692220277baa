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

template <typename T, int DIM, int KIND>
__global__ void k_line(Lev<T> L, int dir, int zebra, int colour, const T *u, const T *__restrict__ g, T *out, T omega,
                       T *__restrict__ cps, T *__restrict__ dps) {
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
                 const T *g, T *out, T omega, T *s1, T *s2) {
  long long nlines = dir == 0 ? L.unk_rows() : (long long)(L.n0 - 2) * L.zrows();
  int th = 64;
  unsigned bl = (unsigned)((nlines + th - 1) / th);
  if (L.dim == 2) {
    if (kind == K_CONST) k_line<T, 2, K_CONST><<<bl, th, 0, lc.s>>>(L, dir, zebra, colour, u, g, out, omega, s1, s2);
    else if (kind == K_SEP) k_line<T, 2, K_SEP><<<bl, th, 0, lc.s>>>(L, dir, zebra, colour, u, g, out, omega, s1, s2);
    else if (kind == K_CELL) k_line<T, 2, K_CELL><<<bl, th, 0, lc.s>>>(L, dir, zebra, colour, u, g, out, omega, s1, s2);
    else k_line<T, 2, K_EDGE><<<bl, th, 0, lc.s>>>(L, dir, zebra, colour, u, g, out, omega, s1, s2);
  } else {
    if (kind == K_CONST) k_line<T, 3, K_CONST><<<bl, th, 0, lc.s>>>(L, dir, zebra, colour, u, g, out, omega, s1, s2);
    else if (kind == K_SEP) k_line<T, 3, K_SEP><<<bl, th, 0, lc.s>>>(L, dir, zebra, colour, u, g, out, omega, s1, s2);
    else if (kind == K_CELL) k_line<T, 3, K_CELL><<<bl, th, 0, lc.s>>>(L, dir, zebra, colour, u, g, out, omega, s1, s2);
    else k_line<T, 3, K_EDGE><<<bl, th, 0, lc.s>>>(L, dir, zebra, colour, u, g, out, omega, s1, s2);
  }
  ++*lc.counter;
}

template void launch_line<double>(const Launch &, const Lev<double> &, int, int, int, int, const double *,
                                  const double *, double *, double, double *, double *);
template void launch_line<float>(const Launch &, const Lev<float> &, int, int, int, int, const float *, const float *,
                                 float *, float, float *, float *);

}  // namespace mg
