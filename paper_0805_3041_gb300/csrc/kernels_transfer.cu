// kernels_transfer.cu -- grid transfers (full-weighting restriction, bilinear /
// trilinear prolongation with correction), the coarsest-grid solve
// u = A_1^{-1} g with a dense inverse built on the device by Gauss-Jordan
// elimination, set-up kernels (coefficient coarsening, diagonal inverses), and
// layout conversions between the caller's compact arrays and the padded levels.
//
// Wallis (2008), section "The Multigrid Technique": g_{l-1} = R d_l,
// u + omega_l P u_{l-1}, and A_1^{-1} g on the coarsest grid.
#define MG_FILE_ID 2   // bounds-check sites (-DMG_DEBUG)
#include "mg_internal.cuh"

namespace mg {

static constexpr int BX = 32, BY = 8;

static inline dim3 grid2(long long xthreads, long long rows, int R) {
  long long gy = (rows + (long long)BY * R - 1) / ((long long)BY * R);
  return dim3((unsigned)((xthreads + BX - 1) / BX), (unsigned)gy, 1);
}
static inline int rpt(long long rows) { return rows >= 2048 ? 4 : 1; }

// ---------------------------------------------------------------------------------------
// full weighting: g_c(I) = sum_a prod_d w(a_d) r_f(2I + a), w = [1/4, 1/2, 1/4]
// ---------------------------------------------------------------------------------------
template <typename T, int DIM>
__global__ void __launch_bounds__(BX *BY) k_restrict(Lev<T> F, Lev<T> C, const T *__restrict__ rf, T *__restrict__ gc,
                                                     int R) {
  MG_PDL_WAIT();
  int I = 1 + blockIdx.x * BX + threadIdx.x;
  if (I > C.n0 - 2) return;
  long long r0 = ((long long)blockIdx.y * BY + threadIdx.y) * R;
  long long nr = C.unk_rows();
  for (int q = 0; q < R; ++q) {
    long long r = r0 + q;
    if (r >= nr) return;
    int J, K;
    row_jk(C, r, J, K);
    long long dm, dp;
    yoffs(F, 2 * J, dm, dp);
    long long pf = (long long)(2 * K) * F.plane + (long long)(2 * J) * F.pitch + 2 * I;
    const long long pc = (long long)K * C.plane + (long long)J * C.pitch + I;
    {
      const long long zl = DIM == 3 ? F.plane : 0;   // the 3 x 3 (x 3) fine stencil's corners
      if (!MG_CK(C, pc) || !MG_CK(F, pf - zl + dm - 1) || !MG_CK(F, pf - zl + dp + 1) || !MG_CK(F, pf + zl + dm - 1) ||
          !MG_CK(F, pf + zl + dp + 1))
        continue;
    }
    auto row3 = [&](long long c) -> T { return (rf[c - 1] + rf[c + 1]) + T(2) * rf[c]; };
    auto plane3 = [&](long long c) -> T { return (row3(c + dm) + row3(c + dp)) + T(2) * row3(c); };
    T s;
    if (DIM == 2) {
      s = plane3(pf) * T(0.0625);
    } else {
      s = ((plane3(pf - F.plane) + plane3(pf + F.plane)) + T(2) * plane3(pf)) * T(0.015625);
    }
    gc[pc] = s;
  }
}

// ---------------------------------------------------------------------------------------
// u_f += w * P e_c (bilinear / trilinear; coarse Dirichlet nodes hold 0)
// ---------------------------------------------------------------------------------------
template <typename T, int DIM>
__global__ void __launch_bounds__(BX *BY) k_prolong_add(Lev<T> F, Lev<T> C, const T *__restrict__ ec,
                                                        T *__restrict__ uf, T w, int R) {
  MG_PDL_WAIT();
  int i = 1 + blockIdx.x * BX + threadIdx.x;
  if (i > F.n0 - 2) return;
  long long r0 = ((long long)blockIdx.y * BY + threadIdx.y) * R;
  long long nr = F.unk_rows();
  int I0 = i >> 1, I1 = (i + 1) >> 1;
  for (int q = 0; q < R; ++q) {
    long long r = r0 + q;
    if (r >= nr) return;
    int j, k;
    row_jk(F, r, j, k);
    int J0 = j >> 1, J1 = (j + 1) >> 1;
    if (J1 >= C.n1) J1 -= C.n1;   // periodic wrap (only reachable when y is periodic)
    long long a0 = (long long)J0 * C.pitch, a1 = (long long)J1 * C.pitch;
    long long p = (long long)k * F.plane + (long long)j * F.pitch + i;
    {
      const long long zhi = DIM == 3 ? (long long)((k + 1) >> 1) * C.plane : 0;
      const long long zlo = DIM == 3 ? (long long)(k >> 1) * C.plane : 0;
      if (!MG_CK(F, p) || !MG_CK(C, zlo + a0 + I0) || !MG_CK(C, zhi + a1 + I1) || !MG_CK(C, zlo + a1 + I0) ||
          !MG_CK(C, zhi + a0 + I1))
        continue;
    }
    T s;
    if (DIM == 2) {
      s = ((ec[a0 + I0] + ec[a0 + I1]) + (ec[a1 + I0] + ec[a1 + I1])) * T(0.25);
    } else {
      long long z0 = (long long)(k >> 1) * C.plane, z1 = (long long)((k + 1) >> 1) * C.plane;
      T s0 = (ec[z0 + a0 + I0] + ec[z0 + a0 + I1]) + (ec[z0 + a1 + I0] + ec[z0 + a1 + I1]);
      T s1 = (ec[z1 + a0 + I0] + ec[z1 + a0 + I1]) + (ec[z1 + a1 + I0] + ec[z1 + a1 + I1]);
      s = (s0 + s1) * T(0.125);
    }
    uf[p] = fma(w, s, uf[p]);
  }
}

// out = P ec on every node of F: the interpolation at the unknowns, zero on the Dirichlet
// nodes (the whole node array is written, so no clearing pass is needed)
template <typename T, int DIM>
__global__ void __launch_bounds__(BX *BY) k_interp(Lev<T> F, Lev<T> C, const T *__restrict__ ec,
                                                   T *__restrict__ out, int R) {
  MG_PDL_WAIT();
  int i = blockIdx.x * BX + threadIdx.x;
  if (i >= F.n0) return;
  long long r0 = ((long long)blockIdx.y * BY + threadIdx.y) * R;
  const int nrows = F.n1 * (DIM == 3 ? F.n2 : 1);
  const bool xin = i >= 1 && i <= F.n0 - 2;
  const int I0 = i >> 1, I1 = (i + 1) >> 1;
  for (int q = 0; q < R; ++q) {
    long long r = r0 + q;
    if (r >= nrows) return;
    const int j = DIM == 3 ? (int)r % F.n1 : (int)r, k = DIM == 3 ? (int)r / F.n1 : 0;
    const bool unk = xin && (F.per || (j >= 1 && j <= F.n1 - 2)) && (DIM == 2 || (k >= 1 && k <= F.n2 - 2));
    T s = T(0);
    const long long po = (long long)k * F.plane + (long long)j * F.pitch + i;
    if (!MG_CK(F, po)) continue;
    if (unk) {
      int J0 = j >> 1, J1 = (j + 1) >> 1;
      if (J1 >= C.n1) J1 -= C.n1;   // periodic wrap
      long long a0 = (long long)J0 * C.pitch, a1 = (long long)J1 * C.pitch;
      const long long zhi = DIM == 3 ? (long long)((k + 1) >> 1) * C.plane : 0;
      const long long zlo = DIM == 3 ? (long long)(k >> 1) * C.plane : 0;
      if (!MG_CK(C, zlo + a0 + I0) || !MG_CK(C, zhi + a1 + I1) || !MG_CK(C, zlo + a1 + I0) || !MG_CK(C, zhi + a0 + I1))
        continue;
      if (DIM == 2) {
        s = ((ec[a0 + I0] + ec[a0 + I1]) + (ec[a1 + I0] + ec[a1 + I1])) * T(0.25);
      } else {
        long long z0 = (long long)(k >> 1) * C.plane, z1 = (long long)((k + 1) >> 1) * C.plane;
        T s0 = (ec[z0 + a0 + I0] + ec[z0 + a0 + I1]) + (ec[z0 + a1 + I0] + ec[z0 + a1 + I1]);
        T s1 = (ec[z1 + a0 + I0] + ec[z1 + a0 + I1]) + (ec[z1 + a1 + I0] + ec[z1 + a1 + I1]);
        s = (s0 + s1) * T(0.125);
      }
    }
    out[po] = s;
  }
}

template <typename T>
void launch_interp(const Launch &lc, const Lev<T> &F, const Lev<T> &C, const T *ec, T *out) {
  long long rows = (long long)F.n1 * (F.dim == 3 ? F.n2 : 1);
  int R = rpt(rows);
  dim3 gr = grid2(F.n0, rows, R), bl(BX, BY);
  if (F.dim == 2) k_interp<T, 2><<<gr, bl, 0, lc.s>>>(F, C, ec, out, R);
  else k_interp<T, 3><<<gr, bl, 0, lc.s>>>(F, C, ec, out, R);
  lc.done(__func__);
}

template <typename T>
void launch_restrict(const Launch &lc, const Lev<T> &F, const Lev<T> &C, const T *rf, T *gc) {
  long long rows = C.unk_rows();
  int R = rpt(rows);
  dim3 gr = grid2(C.xunk(), rows, R), bl(BX, BY);
  if (F.dim == 2) k_restrict<T, 2><<<gr, bl, 0, lc.s>>>(F, C, rf, gc, R);
  else k_restrict<T, 3><<<gr, bl, 0, lc.s>>>(F, C, rf, gc, R);
  lc.done(__func__);
}

template <typename T>
void launch_prolong_add(const Launch &lc, const Lev<T> &F, const Lev<T> &C, const T *ec, T *uf, T w) {
  long long rows = F.unk_rows();
  int R = rpt(rows);
  dim3 gr = grid2(F.xunk(), rows, R), bl(BX, BY);
  if (F.dim == 2) k_prolong_add<T, 2><<<gr, bl, 0, lc.s>>>(F, C, ec, uf, w, R);
  else k_prolong_add<T, 3><<<gr, bl, 0, lc.s>>>(F, C, ec, uf, w, R);
  lc.done(__func__);
}

// ---------------------------------------------------------------------------------------
// coarsest grid
// ---------------------------------------------------------------------------------------

// u[cidx[r]] = sum_c Ainv[r][c] g[cidx[c]], FP64 arithmetic, one warp per row
template <typename T>
__global__ void k_coarse_apply(const double *__restrict__ Ainv, const long long *__restrict__ cidx, int nc,
                               const T *__restrict__ g, T *__restrict__ u) {
  MG_PDL_WAIT();
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nc) return;
  const double *row = Ainv + (long long)warp * nc;
  double s = 0.0;
  for (int c = lane; c < nc; c += 32) s = fma(row[c], (double)g[cidx[c]], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) u[cidx[warp]] = (T)s;
}

template <typename T>
void launch_coarse_apply(const Launch &lc, const double *Ainv, const long long *cidx, int nc, const T *g, T *u) {
  int threads = 256, blocks = (nc * 32 + threads - 1) / threads;
  k_coarse_apply<T><<<blocks, threads, 0, lc.s>>>(Ainv, cidx, nc, g, u);
  lc.done(__func__);
}

// Dense matrix of the coarsest operator: row r of unknown p = cidx[r] holds D_p on the
// diagonal and -w_e for every edge to another unknown (Dirichlet neighbours drop out).
template <typename T, int DIM, int KIND>
__global__ void k_assemble_dense(Lev<T> L, const long long *__restrict__ cidx, const int *__restrict__ cmap, int nc,
                                 double *__restrict__ A) {
  MG_PDL_WAIT();
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nc) return;
  long long p = cidx[r];
  int k = (int)(p / L.plane);
  int j = (int)((p - (long long)k * L.plane) / L.pitch);
  int i = (int)(p - (long long)k * L.plane - (long long)j * L.pitch);
  long long dm, dp;
  yoffs(L, j, dm, dp);
  Weights<T, DIM, KIND> w;
  w.load(L, i, p, dm);
  double *row = A + (long long)r * nc;
  if (KIND == K_NINE) {   // 2-D Galerkin level: the 9-point stencil
    row[r] += (double)w.dd;
    const long long nb9[8] = {p - 1, p + 1, p + dm, p + dp, p + dm - 1, p + dm + 1, p + dp - 1, p + dp + 1};
    const double w9[8] = {(double)w.wW, (double)w.wE, (double)w.wS, (double)w.wN,
                          (double)w.wSW, (double)w.wSE, (double)w.wNW, (double)w.wNE};
    for (int e = 0; e < 8; ++e) {
      int c = cmap[nb9[e]];
      if (c >= 0) row[c] -= w9[e];
    }
    return;
  }
  double D = (double)w.wW + (double)w.wE + (double)w.wS + (double)w.wN;
  if (DIM == 3) D += (double)w.wB + (double)w.wF;
  row[r] += D;
  long long nb[6] = {p - 1, p + 1, p + dm, p + dp, p - L.plane, p + L.plane};
  double ww[6] = {(double)w.wW, (double)w.wE, (double)w.wS, (double)w.wN, (double)w.wB, (double)w.wF};
  for (int e = 0; e < 2 * DIM; ++e) {
    int c = cmap[nb[e]];
    if (c >= 0) row[c] -= ww[e];
  }
}

template <typename T>
void launch_assemble_dense(const Launch &lc, const Lev<T> &L, int kind, const long long *cidx, const int *cmap,
                           int nc, double *A) {
  int th = 128, bl = (nc + th - 1) / th;
  if (L.dim == 2) {
    if (kind == K_NINE) k_assemble_dense<T, 2, K_NINE><<<bl, th, 0, lc.s>>>(L, cidx, cmap, nc, A);
    else if (kind == K_CONST) k_assemble_dense<T, 2, K_CONST><<<bl, th, 0, lc.s>>>(L, cidx, cmap, nc, A);
    else if (kind == K_SEP) k_assemble_dense<T, 2, K_SEP><<<bl, th, 0, lc.s>>>(L, cidx, cmap, nc, A);
    else if (kind == K_CELL) k_assemble_dense<T, 2, K_CELL><<<bl, th, 0, lc.s>>>(L, cidx, cmap, nc, A);
    else k_assemble_dense<T, 2, K_EDGE><<<bl, th, 0, lc.s>>>(L, cidx, cmap, nc, A);
  } else {
    if (kind == K_CONST) k_assemble_dense<T, 3, K_CONST><<<bl, th, 0, lc.s>>>(L, cidx, cmap, nc, A);
    else if (kind == K_SEP) k_assemble_dense<T, 3, K_SEP><<<bl, th, 0, lc.s>>>(L, cidx, cmap, nc, A);
    else if (kind == K_CELL) k_assemble_dense<T, 3, K_CELL><<<bl, th, 0, lc.s>>>(L, cidx, cmap, nc, A);
    else k_assemble_dense<T, 3, K_EDGE><<<bl, th, 0, lc.s>>>(L, cidx, cmap, nc, A);
  }
  lc.done(__func__);
}

// In-place Gauss-Jordan inversion of an SPD matrix (no pivoting needed), step k:
//   (a) save column k, divide row k by the pivot, set A[k][k] = 1/pivot;
//   (b) A[i][j] -= col[i] * A[k][j] for i != k, with A[i][k] := -col[i] / pivot.
__global__ void k_gj_a(double *A, double *col, int n, int k) {
  MG_PDL_WAIT();
  for (int i = threadIdx.x; i < n; i += blockDim.x) col[i] = A[(long long)i * n + k];
  __syncthreads();
  double piv = col[k];
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    A[(long long)k * n + j] = (j == k ? 1.0 : A[(long long)k * n + j]) / piv;
}
__global__ void k_gj_b(double *A, const double *__restrict__ col, int n, int k) {
  MG_PDL_WAIT();
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  int i = (int)(t / n), j = (int)(t % n);
  if (i == k) return;
  double a = (j == k) ? 0.0 : A[t];
  A[t] = a - col[i] * A[(long long)k * n + j];
}
void launch_gj_step(const Launch &lc, double *A, double *col, int n, int kstep) {
  k_gj_a<<<1, 256, 0, lc.s>>>(A, col, n, kstep);
  long long tot = (long long)n * n;
  k_gj_b<<<(unsigned)((tot + 255) / 256), 256, 0, lc.s>>>(A, col, n, kstep);
  lc.done("k_gj_a");
  lc.done("k_gj_b");
}

// ---------------------------------------------------------------------------------------
// set-up: coefficient coarsening and diagonal inverses (FP64)
// ---------------------------------------------------------------------------------------

// separable weights: W_x(I) = 1/4 H(w_x(2I), w_x(2I+1)), W_y(I) = 1/4 w_y(2I), W_z(I) = 1/4 w_z(2I)
__global__ void k_coarsen_sep(const double *fsx, const double *fsy, const double *fsz, int nf0, double *csx,
                              double *csy, double *csz, int nc0) {
  MG_PDL_WAIT();
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc0) return;
  if (I < nc0 - 1) {
    double a = fsx[2 * I], b = fsx[2 * I + 1];
    csx[I] = 0.25 * (2.0 * a * b / (a + b));
  } else {
    csx[I] = 0.0;
  }
  csy[I] = 0.25 * fsy[2 * I];
  csz[I] = 0.25 * fsz[2 * I];
}
void launch_coarsen_sep(const Launch &lc, const double *fsx, const double *fsy, const double *fsz, int nf0,
                        double *csx, double *csy, double *csz, int nc0) {
  k_coarsen_sep<<<(nc0 + 127) / 128, 128, 0, lc.s>>>(fsx, fsy, fsz, nf0, csx, csy, csz, nc0);
  lc.done(__func__);
}

__global__ void k_sep_dinv(const double *sx, const double *sy, const double *sz, int n0, int dim, double *dinv) {
  MG_PDL_WAIT();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n0) return;
  if (i < 1 || i > n0 - 2) { dinv[i] = 0.0; return; }
  double D = sx[i - 1] + sx[i] + sy[i] + sy[i];
  if (dim == 3) D += sz[i] + sz[i];
  dinv[i] = 1.0 / D;
}
void launch_sep_dinv(const Launch &lc, const double *sx, const double *sy, const double *sz, int n0, int dim,
                     double *dinv) {
  k_sep_dinv<<<(n0 + 127) / 128, 128, 0, lc.s>>>(sx, sy, sz, n0, dim, dinv);
  lc.done(__func__);
}

// coarse cell coefficient = mean of the 2^d child cells
__global__ void k_coarsen_cell(Lev<double> F, Lev<double> C, const double *__restrict__ kf, double *__restrict__ kc) {
  MG_PDL_WAIT();
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  int J = blockIdx.y, K = blockIdx.z;
  int ncx = C.n0 - 1, ncy = C.per ? C.n1 : C.n1 - 1;
  if (I >= ncx || J >= ncy) return;
  int nz = C.dim == 3 ? 2 : 1;
  if (!MG_CK(C, (long long)K * C.plane + (long long)J * C.pitch + I) ||
      !MG_CK(F, (long long)(2 * K + nz - 1) * F.plane + (long long)(2 * J + 1) * F.pitch + 2 * I + 1))
    return;
  double s = 0.0;
  for (int z = 0; z < nz; ++z)
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a)
        s += kf[(long long)(2 * K + (C.dim == 3 ? z : 0)) * F.plane + (long long)(2 * J + b) * F.pitch + 2 * I + a];
  kc[(long long)K * C.plane + (long long)J * C.pitch + I] = s * (C.dim == 3 ? 0.125 : 0.25);
}
void launch_coarsen_cell(const Launch &lc, const Lev<double> &F, const Lev<double> &C, const double *kf, double *kc) {
  int ncx = C.n0 - 1, ncy = C.per ? C.n1 : C.n1 - 1, ncz = C.dim == 3 ? C.n2 - 1 : 1;
  dim3 gr((ncx + 127) / 128, ncy, ncz);
  k_coarsen_cell<<<gr, 128, 0, lc.s>>>(F, C, kf, kc);
  lc.done(__func__);
}

template <int DIM>
__global__ void k_cell_dinv(Lev<double> L, double *__restrict__ dinv) {
  MG_PDL_WAIT();
  int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
  if (i > L.n0 - 2) return;
  long long r = blockIdx.y + (long long)blockIdx.z * gridDim.y;
  if (r >= L.unk_rows()) return;
  int j, k;
  row_jk(L, r, j, k);
  long long p = (long long)k * L.plane + (long long)j * L.pitch + i, dm, dp;
  yoffs(L, j, dm, dp);
  const double *kk = L.k;
  double D;
  if (DIM == 2) {
    double sw = kk[p + dm - 1], se = kk[p + dm], nw = kk[p - 1], ne = kk[p];
    D = L.ax * (sw + nw) + L.ax * (se + ne) + L.ay * (sw + se) + L.ay * (nw + ne);
  } else {
    long long pl = L.plane;
    double sw0 = kk[p - pl + dm - 1], se0 = kk[p - pl + dm], nw0 = kk[p - pl - 1], ne0 = kk[p - pl];
    double sw1 = kk[p + dm - 1], se1 = kk[p + dm], nw1 = kk[p - 1], ne1 = kk[p];
    D = L.ax * ((sw0 + nw0) + (sw1 + nw1)) + L.ax * ((se0 + ne0) + (se1 + ne1)) +
        L.ay * ((sw0 + se0) + (sw1 + se1)) + L.ay * ((nw0 + ne0) + (nw1 + ne1)) +
        L.az * ((sw0 + se0) + (nw0 + ne0)) + L.az * ((sw1 + se1) + (nw1 + ne1));
  }
  dinv[p] = 1.0 / D;
}
void launch_cell_dinv(const Launch &lc, const Lev<double> &L, double *dinv) {
  long long rows = L.unk_rows();
  unsigned gy = (unsigned)(rows < 65535 ? rows : 65535), gz = (unsigned)((rows + gy - 1) / gy);
  dim3 gr((L.xunk() + 127) / 128, gy, gz);
  if (L.dim == 2) k_cell_dinv<2><<<gr, 128, 0, lc.s>>>(L, dinv);
  else k_cell_dinv<3><<<gr, 128, 0, lc.s>>>(L, dinv);
  lc.done(__func__);
}

// ---------------------------------------------------------------------------------------
// Galerkin coarse operator A_c = R A P (2-D, y not periodic): R full weighting, P = 4 R^T
// bilinear interpolation, both over the unknowns.  For coarse unknown P and offset (al, be):
//   A_c(P, P + (al, be)) = sum_p R(P, p) sum_q A(p, q) P(q, P + (al, be)),
// p over the fine unknowns within one node of 2P (weights w(pa) w(pb), w(0) = 1/2, w(+-1) = 1/4),
// q over the stencil of p, P(q, Q) = (2 w(dx)) (2 w(dy)) with (dx, dy) = q - 2Q within one node.
// One thread per coarse node writes D, the +x, +y, +x+y, -x+y weights (w = -A) and 1/D;
// nodes that are not unknowns, and couplings to them, get 0.

// A(p, p + (a, b)) of fine level F at unknown p = (i, j); 0 if p + (a, b) is not an unknown
template <int KIND>
__device__ __forceinline__ double stencil_entry(const Lev<double> &F, int i, int j, int a, int b) {
  const int qi = i + a, qj = j + b;
  if (qi < 1 || qi > F.n0 - 2 || qj < 1 || qj > F.n1 - 2) return 0.0;
  const long long p = (long long)j * F.pitch + i, dm = -F.pitch;
  Weights<double, 2, KIND> w;
  w.load(F, i, p, dm);
  if (KIND == K_NINE) {
    if (a == 0 && b == 0) return w.dd;
    if (b == 0) return a > 0 ? -w.wE : -w.wW;
    if (a == 0) return b > 0 ? -w.wN : -w.wS;
    if (b > 0) return a > 0 ? -w.wNE : -w.wNW;
    return a > 0 ? -w.wSE : -w.wSW;
  }
  if (a == 0 && b == 0) return KIND == K_CONST ? F.d : (w.wW + w.wE) + (w.wS + w.wN);
  if (b == 0) return a > 0 ? -w.wE : -w.wW;
  if (a == 0) return b > 0 ? -w.wN : -w.wS;
  return 0.0;
}

__device__ __forceinline__ double fw1(int a) { return a == 0 ? 0.5 : 0.25; }

template <int KIND>
__global__ void k_rap(Lev<double> F, Lev<double> C, double *__restrict__ dg, double *__restrict__ ex,
                      double *__restrict__ ey, double *__restrict__ ene, double *__restrict__ enw,
                      double *__restrict__ dinv) {
  MG_PDL_WAIT();
  const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y;
  if (I >= C.n0 || J >= C.n1) return;
  const long long pc = (long long)J * C.pitch + I;
  const bool unk = I >= 1 && I <= C.n0 - 2 && J >= 1 && J <= C.n1 - 2;
  double a9[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  if (unk) {
    for (int be = -1; be <= 1; ++be)
      for (int al = -1; al <= 1; ++al) {
        const int QI = I + al, QJ = J + be;
        if (QI < 1 || QI > C.n0 - 2 || QJ < 1 || QJ > C.n1 - 2) continue;
        double s = 0.0;
        for (int pb = -1; pb <= 1; ++pb)
          for (int pa = -1; pa <= 1; ++pa) {
            const int pi = 2 * I + pa, pj = 2 * J + pb;
            if (pi < 1 || pi > F.n0 - 2 || pj < 1 || pj > F.n1 - 2) continue;
            double t = 0.0;
            for (int qb = -1; qb <= 1; ++qb)
              for (int qa = -1; qa <= 1; ++qa) {
                const int dx = pi + qa - 2 * QI, dy = pj + qb - 2 * QJ;
                if (dx < -1 || dx > 1 || dy < -1 || dy > 1) continue;
                t += stencil_entry<KIND>(F, pi, pj, qa, qb) * (2.0 * fw1(dx)) * (2.0 * fw1(dy));
              }
            s += fw1(pa) * fw1(pb) * t;
          }
        a9[be + 1][al + 1] = s;
      }
  }
  dg[pc] = a9[1][1];
  ex[pc] = -a9[1][2];
  ey[pc] = -a9[2][1];
  ene[pc] = -a9[2][2];
  enw[pc] = -a9[2][0];
  dinv[pc] = unk ? 1.0 / a9[1][1] : 0.0;
}

void launch_rap(const Launch &lc, const Lev<double> &F, int fkind, const Lev<double> &C, double *dg, double *ex,
                double *ey, double *ene, double *enw, double *dinv) {
  dim3 gr((C.n0 + 127) / 128, C.n1, 1);
  if (fkind == K_CONST) k_rap<K_CONST><<<gr, 128, 0, lc.s>>>(F, C, dg, ex, ey, ene, enw, dinv);
  else if (fkind == K_SEP) k_rap<K_SEP><<<gr, 128, 0, lc.s>>>(F, C, dg, ex, ey, ene, enw, dinv);
  else if (fkind == K_CELL) k_rap<K_CELL><<<gr, 128, 0, lc.s>>>(F, C, dg, ex, ey, ene, enw, dinv);
  else if (fkind == K_EDGE) k_rap<K_EDGE><<<gr, 128, 0, lc.s>>>(F, C, dg, ex, ey, ene, enw, dinv);
  else k_rap<K_NINE><<<gr, 128, 0, lc.s>>>(F, C, dg, ex, ey, ene, enw, dinv);
  lc.done(__func__);
}

// edge coefficients: coarse weights edge by edge, and 1/D
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double harm0(double a, double b) { return a + b > 0.0 ? 2.0 * a * b / (a + b) : 0.0; }

// The coarse edge from node (I, J, K) to its +x (+y, +z) neighbour spans the two fine edges
// from (2I, 2J, 2K) in that direction: their harmonic mean (series) times 1/4; the fine line
// through the coarse node is taken across (injection).  Edges absent on the coarse grid are 0.
__global__ void k_coarsen_edge(Lev<double> F, Lev<double> C, const double *__restrict__ fx,
                               const double *__restrict__ fy, const double *__restrict__ fz, double *__restrict__ cx,
                               double *__restrict__ cy, double *__restrict__ cz) {
  MG_PDL_WAIT();
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  int J = blockIdx.y, K = blockIdx.z;
  if (I >= C.n0) return;
  long long pc = (long long)K * C.plane + (long long)J * C.pitch + I;
  long long pf = (long long)(C.dim == 3 ? 2 * K : 0) * F.plane + (long long)(2 * J) * F.pitch + 2 * I;
  cx[pc] = I < C.n0 - 1 ? 0.25 * harm0(fx[pf], fx[pf + 1]) : 0.0;
  cy[pc] = (C.per || J < C.n1 - 1) ? 0.25 * harm0(fy[pf], fy[pf + F.pitch]) : 0.0;
  if (C.dim == 3) cz[pc] = K < C.n2 - 1 ? 0.25 * harm0(fz[pf], fz[pf + F.plane]) : 0.0;
}
void launch_coarsen_edge(const Launch &lc, const Lev<double> &F, const Lev<double> &C, const double *fx,
                         const double *fy, const double *fz, double *cx, double *cy, double *cz) {
  dim3 gr((C.n0 + 127) / 128, C.n1, C.dim == 3 ? C.n2 : 1);
  k_coarsen_edge<<<gr, 128, 0, lc.s>>>(F, C, fx, fy, fz, cx, cy, cz);
  lc.done(__func__);
}

// 1/D at the unknowns, D = the sum of the weights of the edges at the node
template <int DIM>
__global__ void k_edge_dinv(Lev<double> L, double *__restrict__ dinv) {
  MG_PDL_WAIT();
  int i = 1 + blockIdx.x * blockDim.x + threadIdx.x;
  if (i > L.n0 - 2) return;
  long long r = blockIdx.y + (long long)blockIdx.z * gridDim.y;
  if (r >= L.unk_rows()) return;
  int j, k;
  row_jk(L, r, j, k);
  long long p = (long long)k * L.plane + (long long)j * L.pitch + i, dm, dp;
  yoffs(L, j, dm, dp);
  Weights<double, DIM, K_EDGE> w;
  w.load(L, i, p, dm);
  double D = (w.wW + w.wE) + (w.wS + w.wN);
  if (DIM == 3) D += w.wB + w.wF;
  dinv[p] = 1.0 / D;
}
void launch_edge_dinv(const Launch &lc, const Lev<double> &L, double *dinv) {
  long long rows = L.unk_rows();
  unsigned gy = (unsigned)(rows < 65535 ? rows : 65535), gz = (unsigned)((rows + gy - 1) / gy);
  dim3 gr((L.xunk() + 127) / 128, gy, gz);
  if (L.dim == 2) k_edge_dinv<2><<<gr, 128, 0, lc.s>>>(L, dinv);
  else k_edge_dinv<3><<<gr, 128, 0, lc.s>>>(L, dinv);
  lc.done(__func__);
}

__global__ void k_to_float(const double *__restrict__ s, float *__restrict__ d, long long n) {
  MG_PDL_WAIT();
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long st = (long long)gridDim.x * blockDim.x;
  for (; t < n; t += st) d[t] = (float)s[t];
}
void launch_to_float(const Launch &lc, const double *src, float *dst, long long n) {
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_to_float<<<(unsigned)blocks, 256, 0, lc.s>>>(src, dst, n);
  lc.done(__func__);
}

// ---------------------------------------------------------------------------------------
// layout conversions (compact caller arrays <-> padded level arrays)
// ---------------------------------------------------------------------------------------
// A block of 128 threads copies PACK_ELEMS * 128 consecutive nodes of one row, each thread
// PACK_ELEMS of them 128 apart: every load of a thread is issued before its stores.
constexpr int PACK_ELEMS = 4;
template <typename T>
__global__ void k_pack(Lev<T> L, const double *__restrict__ src, T *__restrict__ dst, int zero_boundary) {
  MG_PDL_WAIT();
  const int i0 = blockIdx.x * (PACK_ELEMS * 128) + threadIdx.x;
  const int j = blockIdx.y, k = blockIdx.z;
  const long long s0 = ((long long)k * L.n1 + j) * L.n0, d0 = (long long)k * L.plane + (long long)j * L.pitch;
  const bool brow = (!L.per && (j == 0 || j == L.n1 - 1)) || (L.dim == 3 && (k == 0 || k == L.n2 - 1));
  double v[PACK_ELEMS];
#pragma unroll
  for (int q = 0; q < PACK_ELEMS; ++q) {
    const int i = i0 + 128 * q;
    v[q] = i < L.n0 ? src[s0 + i] : 0.0;
  }
#pragma unroll
  for (int q = 0; q < PACK_ELEMS; ++q) {
    const int i = i0 + 128 * q;
    if (i >= L.n0 || !MG_CK(L, d0 + i)) continue;
    const bool bnd = brow || i == 0 || i == L.n0 - 1;
    dst[d0 + i] = (zero_boundary && bnd) ? T(0) : (T)v[q];
  }
}
template <typename T>
__global__ void k_unpack(Lev<T> L, const T *__restrict__ src, double *__restrict__ dst, double scale) {
  MG_PDL_WAIT();
  const int i0 = blockIdx.x * (PACK_ELEMS * 128) + threadIdx.x;
  const int j = blockIdx.y, k = blockIdx.z;
  const long long s0 = (long long)k * L.plane + (long long)j * L.pitch, d0 = ((long long)k * L.n1 + j) * L.n0;
  T v[PACK_ELEMS];
#pragma unroll
  for (int q = 0; q < PACK_ELEMS; ++q) {
    const int i = i0 + 128 * q;
    v[q] = (i < L.n0 && MG_CK(L, s0 + i)) ? src[s0 + i] : T(0);
  }
#pragma unroll
  for (int q = 0; q < PACK_ELEMS; ++q) {
    const int i = i0 + 128 * q;
    if (i < L.n0 && MG_CK(L, s0 + i)) dst[d0 + i] = scale * (double)v[q];
  }
}
template <typename T>
__global__ void k_zero_boundary(Lev<T> L, T *__restrict__ dst) {
  MG_PDL_WAIT();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y, k = blockIdx.z;
  if (i >= L.n0) return;
  bool bnd = (i == 0 || i == L.n0 - 1) || (!L.per && (j == 0 || j == L.n1 - 1)) ||
             (L.dim == 3 && (k == 0 || k == L.n2 - 1));
  const long long d = (long long)k * L.plane + (long long)j * L.pitch + i;
  if (bnd && MG_CK(L, d)) dst[d] = T(0);
}
template <typename T>
void launch_zero_boundary(const Launch &lc, const Lev<T> &L, T *dst) {
  dim3 gr((L.n0 + 127) / 128, L.n1, L.dim == 3 ? L.n2 : 1);
  k_zero_boundary<T><<<gr, 128, 0, lc.s>>>(L, dst);
  lc.done(__func__);
}
template <typename T>
__global__ void k_zero_level(Lev<T> L, T *__restrict__ dst) {
  MG_PDL_WAIT();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.pitch) return;
  const long long d = (long long)blockIdx.z * L.plane + (long long)blockIdx.y * L.pitch + i;
  if (MG_CK(L, d)) dst[d] = T(0);
}

template <typename T>
void launch_pack(const Launch &lc, const Lev<T> &L, const double *src, T *dst, int zero_boundary) {
  dim3 gr((L.n0 + PACK_ELEMS * 128 - 1) / (PACK_ELEMS * 128), L.n1, L.dim == 3 ? L.n2 : 1);
  k_pack<T><<<gr, 128, 0, lc.s>>>(L, src, dst, zero_boundary);
  lc.done(__func__);
}
template <typename T>
void launch_unpack(const Launch &lc, const Lev<T> &L, const T *src, double *dst, double scale) {
  dim3 gr((L.n0 + PACK_ELEMS * 128 - 1) / (PACK_ELEMS * 128), L.n1, L.dim == 3 ? L.n2 : 1);
  k_unpack<T><<<gr, 128, 0, lc.s>>>(L, src, dst, scale);
  lc.done(__func__);
}
template <typename T>
void launch_zero_level(const Launch &lc, const Lev<T> &L, T *dst) {
  dim3 gr((unsigned)((L.pitch + 127) / 128), L.n1, L.dim == 3 ? L.n2 : 1);
  k_zero_level<T><<<gr, 128, 0, lc.s>>>(L, dst);
  lc.done(__func__);
}

// Axis-swapped copies (y-line smoothers run as x-line smoothers on the transposed
// problem): internal node (i', j', k) <-> caller node (i = j', j = i', k).  32 x 32 tiles
// through shared memory keep both sides coalesced.  rows_i, cols_i: internal extent of the
// copied array (nodes: n1 x n0; cells: ncy x ncx), pitch_i / plane_i its padded layout;
// the caller array is compact (cols_i x rows_i per plane).
template <typename T, typename U>
__global__ void k_transpose_copy(const U *__restrict__ src, T *__restrict__ dst, int rows_i, int cols_i,
                                 long long pitch_i, long long plane_i, int to_internal, double scale) {
  MG_PDL_WAIT();
  __shared__ double tile[32][33];
  int k = blockIdx.z;
  int bx = blockIdx.x * 32, by = blockIdx.y * 32;   // internal column / row origin
  long long cplane = (long long)rows_i * cols_i;
  if (to_internal) {
    // read caller rows: caller row index = internal column i', caller column = internal row j'
    for (int r = threadIdx.y; r < 32; r += 8) {
      int ic = bx + r, jr = by + threadIdx.x;       // internal (col ic, row jr)
      if (ic < cols_i && jr < rows_i) tile[r][threadIdx.x] = (double)src[k * cplane + (long long)ic * rows_i + jr];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
      int jr = by + r, ic = bx + threadIdx.x;
      if (ic < cols_i && jr < rows_i) dst[k * plane_i + (long long)jr * pitch_i + ic] = (T)(scale * tile[threadIdx.x][r]);
    }
  } else {
    for (int r = threadIdx.y; r < 32; r += 8) {
      int jr = by + r, ic = bx + threadIdx.x;
      if (ic < cols_i && jr < rows_i) tile[r][threadIdx.x] = (double)src[k * plane_i + (long long)jr * pitch_i + ic];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
      int ic = bx + r, jr = by + threadIdx.x;
      if (ic < cols_i && jr < rows_i) dst[k * cplane + (long long)ic * rows_i + jr] = (T)(scale * tile[threadIdx.x][r]);
    }
  }
}

template <typename T>
void launch_pack_swapped(const Launch &lc, const Lev<T> &L, const double *src, T *dst, int zero_boundary) {
  dim3 gr((L.n0 + 31) / 32, (L.n1 + 31) / 32, L.dim == 3 ? L.n2 : 1), bl(32, 8);
  k_transpose_copy<T, double><<<gr, bl, 0, lc.s>>>(src, dst, L.n1, L.n0, L.pitch, L.plane, 1, 1.0);
  lc.done(__func__);
  if (zero_boundary) launch_zero_boundary<T>(lc, L, dst);
}
template <typename T>
void launch_unpack_swapped(const Launch &lc, const Lev<T> &L, const T *src, double *dst, double scale) {
  dim3 gr((L.n0 + 31) / 32, (L.n1 + 31) / 32, L.dim == 3 ? L.n2 : 1), bl(32, 8);
  k_transpose_copy<double, T><<<gr, bl, 0, lc.s>>>(src, dst, L.n1, L.n0, L.pitch, L.plane, 0, scale);
  lc.done(__func__);
}
void launch_cell_pack_swapped(const Launch &lc, const Lev<double> &L, const double *src_compact, double *dst) {
  int ncx = L.n0 - 1, ncy = L.per ? L.n1 : L.n1 - 1, ncz = L.dim == 3 ? L.n2 - 1 : 1;
  dim3 gr((ncx + 31) / 32, (ncy + 31) / 32, ncz), bl(32, 8);
  k_transpose_copy<double, double><<<gr, bl, 0, lc.s>>>(src_compact, dst, ncy, ncx, L.pitch, L.plane, 1, 1.0);
  lc.done(__func__);
}
void launch_cell_unpack_swapped(const Launch &lc, const Lev<double> &L, const double *src, double *dst_compact) {
  int ncx = L.n0 - 1, ncy = L.per ? L.n1 : L.n1 - 1, ncz = L.dim == 3 ? L.n2 - 1 : 1;
  dim3 gr((ncx + 31) / 32, (ncy + 31) / 32, ncz), bl(32, 8);
  k_transpose_copy<double, double><<<gr, bl, 0, lc.s>>>(src, dst_compact, ncy, ncx, L.pitch, L.plane, 0, 1.0);
  lc.done(__func__);
}
template void launch_pack_swapped<double>(const Launch &, const Lev<double> &, const double *, double *, int);
template void launch_pack_swapped<float>(const Launch &, const Lev<float> &, const double *, float *, int);
template void launch_unpack_swapped<double>(const Launch &, const Lev<double> &, const double *, double *, double);
template void launch_unpack_swapped<float>(const Launch &, const Lev<float> &, const float *, double *, double);

// cell arrays: compact (ncz, ncy, n0-1) <-> node layout of the level
__global__ void k_cell_pack(Lev<double> L, const double *__restrict__ src, double *__restrict__ dst, int dir) {
  MG_PDL_WAIT();
  int ncx = L.n0 - 1, ncy = L.per ? L.n1 : L.n1 - 1;
  int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
  if (i >= ncx || j >= ncy) return;
  long long c = ((long long)k * ncy + j) * ncx + i;
  long long d = (long long)k * L.plane + (long long)j * L.pitch + i;
  if (!MG_CK(L, d)) return;
  if (dir == 0) dst[d] = src[c];
  else dst[c] = src[d];
}
void launch_cell_pack(const Launch &lc, const Lev<double> &L, const double *src_compact, double *dst) {
  int ncy = L.per ? L.n1 : L.n1 - 1, ncz = L.dim == 3 ? L.n2 - 1 : 1;
  dim3 gr((L.n0 - 1 + 127) / 128, ncy, ncz);
  k_cell_pack<<<gr, 128, 0, lc.s>>>(L, src_compact, dst, 0);
  lc.done(__func__);
}
void launch_cell_unpack(const Launch &lc, const Lev<double> &L, const double *src, double *dst_compact) {
  int ncy = L.per ? L.n1 : L.n1 - 1, ncz = L.dim == 3 ? L.n2 - 1 : 1;
  dim3 gr((L.n0 - 1 + 127) / 128, ncy, ncz);
  k_cell_pack<<<gr, 128, 0, lc.s>>>(L, src, dst_compact, 1);
  lc.done(__func__);
}

#define INST(T)                                                                                              \
  template void launch_restrict<T>(const Launch &, const Lev<T> &, const Lev<T> &, const T *, T *);          \
  template void launch_prolong_add<T>(const Launch &, const Lev<T> &, const Lev<T> &, const T *, T *, T);    \
  template void launch_interp<T>(const Launch &, const Lev<T> &, const Lev<T> &, const T *, T *);           \
  template void launch_coarse_apply<T>(const Launch &, const double *, const long long *, int, const T *, T *); \
  template void launch_pack<T>(const Launch &, const Lev<T> &, const double *, T *, int);                    \
  template void launch_unpack<T>(const Launch &, const Lev<T> &, const T *, double *, double);                       \
  template void launch_zero_level<T>(const Launch &, const Lev<T> &, T *);                                   \
  template void launch_zero_boundary<T>(const Launch &, const Lev<T> &, T *);
INST(double)
INST(float)
template void launch_assemble_dense<double>(const Launch &, const Lev<double> &, int, const long long *, const int *,
                                            int, double *);

}  // namespace mg
