// kernels_xline.cu -- line smoothers along x (contiguous rows), one CTA per line.
//
// C = tridiagonal part of A along the line (Wallis 2008, section "The choice of
// C": "Tri diagonal C"); x <- x + omega C^{-1}(b - A x), equivalently
// x_line = (1 - omega) x + omega C^{-1}(b + off-line couplings).  Lines along y
// are run through the same kernel on an axis-swapped copy of the problem (the
// paper's "virtually transposed" TRIy / GSTRIy).
//
// Per line of m unknowns (one CTA, NT threads):
//  1. the right-hand side b + sum of off-line couplings is formed coalesced and
//     staged in shared memory (skewed to avoid bank conflicts);
//  2. partition method: thread t owns a segment of <= SMAX consecutive unknowns
//     and eliminates it down to two equations in the segment's first and last
//     unknowns (forward elimination keeping the first unknown, then backward
//     elimination keeping the first and last), held in registers;
//  3. the 2 x (threads) reduced tridiagonal system is solved by parallel cyclic
//     reduction in shared memory;
//  4. every thread recovers its interior unknowns from the two solved ends and
//     the result is written back coalesced.
// Reads the off-line neighbours and b once, writes the line once.
#define MG_FILE_ID 6   // bounds-check sites (-DMG_DEBUG)
#include "mg_internal.cuh"

namespace mg {

namespace {
constexpr int NT = 256;     // threads per line
constexpr int SMAX = 16;    // unknowns per thread: lines up to NT * SMAX = 4096 unknowns
constexpr int XL_SZ = NT * SMAX + NT * SMAX / 16 + 8;   // skewed line buffer length
__device__ __forceinline__ int skew(int i) { return i + (i >> 4); }
}  // namespace

// zebra: only lines with (j + k) % 2 == colour are processed (in place, out == u)
template <typename T, int DIM, int KIND>
__global__ void __launch_bounds__(NT) k_xline(Lev<T> L, const T *u, const T *__restrict__ g, T *out, T omega,
                                              int zebra, int colour) {
  MG_PDL_WAIT();
  extern __shared__ __align__(16) unsigned char xl_raw[];
  T *sd = reinterpret_cast<T *>(xl_raw);                     // rhs, later the solution
  T *sa = sd + XL_SZ, *sb = sa + XL_SZ, *sc = sb + XL_SZ;    // coefficients (variable kinds)
  T *rbase = KIND == K_CONST ? sd + XL_SZ : sd + 4 * XL_SZ;  // reduced system, double buffered
  T(*ra)[2 * NT] = reinterpret_cast<T(*)[2 * NT]>(rbase);
  T(*rb)[2 * NT] = reinterpret_cast<T(*)[2 * NT]>(rbase + 4 * NT);
  T(*rc)[2 * NT] = reinterpret_cast<T(*)[2 * NT]>(rbase + 8 * NT);
  T(*rd)[2 * NT] = reinterpret_cast<T(*)[2 * NT]>(rbase + 12 * NT);
  const int tid = threadIdx.x;
  int j, k;
  row_jk(L, (long long)blockIdx.x, j, k);
  if (zebra && ((j + k) & 1) != colour) return;
  const int m = L.n0 - 2;
  const long long row = (long long)k * L.plane + (long long)j * L.pitch;
  long long dm, dp;
  yoffs(L, j, dm, dp);
  {   // debug build: the line and its neighbour lines lie inside the arrays (uniform per CTA)
    const long long zp = DIM == 3 ? L.plane : 0;
    if (!MG_CK(L, row + 1 + (dm < dp ? dm : dp) - zp) || !MG_CK(L, row + m + (dm < dp ? dp : dm) + zp)) return;
  }
  // 1. right-hand side of the line system and its coefficients
  for (int q = tid; q < m; q += NT) {
    int i = q + 1;
    long long p = row + i;
    Weights<T, DIM, KIND> w;
    w.load(L, i, p, dm);
    T d = g[p];
    d = fma(w.wS, u[p + dm], d);
    d = fma(w.wN, u[p + dp], d);
    if (DIM == 3) {
      d = fma(w.wB, u[p - L.plane], d);
      d = fma(w.wF, u[p + L.plane], d);
    }
    sd[skew(q)] = d;
    if (KIND != K_CONST) {
      T D = (w.wW + w.wE) + (w.wS + w.wN);
      if (DIM == 3) D += w.wB + w.wF;
      sa[skew(q)] = q > 0 ? -w.wW : T(0);
      sb[skew(q)] = D;
      sc[skew(q)] = q < m - 1 ? -w.wE : T(0);
    }
  }
  __syncthreads();
  // 2. segment of this thread: balanced split of m over nt active threads (>= 2 unknowns each)
  int nt = m / 2 < NT ? (m / 2 > 0 ? m / 2 : 1) : NT;
  int per = m / nt, extra = m % nt;
  int n = 0, s0 = 0;
  if (tid < nt) {
    n = per + (tid < extra ? 1 : 0);
    s0 = tid * per + (tid < extra ? tid : extra);
  }
  auto A = [&](int q) -> T { return KIND == K_CONST ? (q > 0 ? -L.cx : T(0)) : sa[skew(q)]; };
  auto B = [&](int q) -> T { return KIND == K_CONST ? L.d : sb[skew(q)]; };
  auto Cc = [&](int q) -> T { return KIND == K_CONST ? (q < m - 1 ? -L.cx : T(0)) : sc[skew(q)]; };
  T ap[SMAX], cp[SMAX], dpv[SMAX];
  T top_a = T(0), top_b = T(1), top_c = T(0), top_d = T(0);
  T bot_a = T(0), bot_b = T(1), bot_c = T(0), bot_d = T(0);
  if (n == 1) {
    // single unknown: its own equation is both reduced equations (first == last)
    top_a = A(s0); top_b = B(s0); top_c = Cc(s0); top_d = sd[skew(s0)];
  } else if (n >= 2) {
    // forward elimination keeping the first unknown x0: x_q + ap_q x0 + cp_q x_{q+1} = dp_q (q >= 1)
#pragma unroll
    for (int q = 1; q < SMAX; ++q) {
      if (q < n) {
        int gq = s0 + q;
        T a = A(gq), b = B(gq), c = Cc(gq), d = sd[skew(gq)];
        if (q == 1) {
          T r = T(1) / b;
          ap[1] = a * r;
          cp[1] = c * r;
          dpv[1] = d * r;
        } else {
          T r = T(1) / (b - a * cp[q - 1]);
          ap[q] = -r * a * ap[q - 1];
          cp[q] = r * c;
          dpv[q] = r * (d - a * dpv[q - 1]);
        }
        // bottom reduced equation ap x0 + x_{n-1} + cp x_n = dp: the values of the last
        // active row q = n-1 (kept as running scalars: no dynamic register indexing)
        bot_a = ap[q];
        bot_c = cp[q];
        bot_d = dpv[q];
      }
    }
    // backward elimination keeping x0 and x_{n-1}: x_q = dp_q - ap_q x0 - cp_q x_{n-1}  (1 <= q <= n-2)
#pragma unroll
    for (int q = SMAX - 2; q >= 1; --q) {
      if (q <= n - 3) {
        dpv[q] = dpv[q] - cp[q] * dpv[q + 1];
        ap[q] = ap[q] - cp[q] * ap[q + 1];
        cp[q] = -cp[q] * cp[q + 1];
      }
    }
    // top reduced equation from row 0: a0 x_{-1} + b0 x0 + c0 x1 = d0 with x1 eliminated (n >= 3)
    T a0 = A(s0), b0 = B(s0), c0 = Cc(s0), d0 = sd[skew(s0)];
    if (n == 2) {
      top_a = a0; top_b = b0; top_c = c0; top_d = d0;
    } else {
      top_a = a0;
      top_b = b0 - c0 * ap[1];
      top_c = -c0 * cp[1];
      top_d = d0 - c0 * dpv[1];
    }
  }
  // 3. reduced system (2 equations per active thread; n == 1 threads contribute an identity row)
  int N = 2 * nt;
  int Np = 1;
  while (Np < N) Np <<= 1;
  for (int e = tid; e < Np; e += NT) {
    if (e >= N) { ra[0][e] = T(0); rb[0][e] = T(1); rc[0][e] = T(0); rd[0][e] = T(0); }
  }
  if (tid < nt) {
    ra[0][2 * tid] = top_a; rb[0][2 * tid] = top_b; rc[0][2 * tid] = top_c; rd[0][2 * tid] = top_d;
    if (n == 1) {   // a one-unknown line: x_last - x_first = 0
      ra[0][2 * tid + 1] = T(-1); rb[0][2 * tid + 1] = T(1); rc[0][2 * tid + 1] = T(0); rd[0][2 * tid + 1] = T(0);
    } else {
      ra[0][2 * tid + 1] = bot_a; rb[0][2 * tid + 1] = T(1); rc[0][2 * tid + 1] = bot_c; rd[0][2 * tid + 1] = bot_d;
    }
  }
  __syncthreads();
  int cur = 0;
  for (int s = 1; s < Np; s <<= 1) {
    for (int e = tid; e < Np; e += NT) {
      T a = ra[cur][e], b = rb[cur][e], c = rc[cur][e], d = rd[cur][e];
      T na = T(0), nc = T(0);
      if (e - s >= 0) {
        T al = -a / rb[cur][e - s];
        na = al * ra[cur][e - s];
        b = fma(al, rc[cur][e - s], b);
        d = fma(al, rd[cur][e - s], d);
      }
      if (e + s < Np) {
        T ga = -c / rb[cur][e + s];
        nc = ga * rc[cur][e + s];
        b = fma(ga, ra[cur][e + s], b);
        d = fma(ga, rd[cur][e + s], d);
      }
      ra[1 - cur][e] = na; rb[1 - cur][e] = b; rc[1 - cur][e] = nc; rd[1 - cur][e] = d;
    }
    __syncthreads();
    cur = 1 - cur;
  }
  // 4. interior unknowns, damped update, write back
  if (tid < nt) {
    T x0 = rd[cur][2 * tid] / rb[cur][2 * tid];
    T xl = rd[cur][2 * tid + 1] / rb[cur][2 * tid + 1];
    sd[skew(s0)] = x0;
    if (n >= 2) sd[skew(s0 + n - 1)] = xl;
#pragma unroll
    for (int q = 1; q < SMAX - 1; ++q)
      if (q <= n - 2) sd[skew(s0 + q)] = dpv[q] - ap[q] * x0 - cp[q] * xl;
  }
  __syncthreads();
  for (int q = tid; q < m; q += NT) {
    long long p = row + q + 1;
    T x = sd[skew(q)];
    out[p] = (omega == T(1)) ? x : fma(omega, x - u[p], u[p]);
  }
}

// Short lines (up to 32 * WSMAX unknowns): one warp per line, WL lines per CTA.  The same
// partition method with lane t owning a segment of <= WSMAX unknowns; the 2 x 32 reduced
// system is solved by parallel cyclic reduction across the warp with shuffles (no block
// barriers).  The line's right-hand side and coefficients are staged coalesced in a
// per-warp shared-memory buffer, and the solution leaves through it.
namespace {
constexpr int WL = 4;        // lines (warps) per CTA
constexpr int WSMAX = 16;    // unknowns per lane
constexpr int WBUF = 32 * WSMAX + 32 * WSMAX / 16 + 8;
}  // namespace

template <typename T, int DIM, int KIND>
__global__ void __launch_bounds__(32 * WL) k_xline_warp(Lev<T> L, const T *u, const T *__restrict__ g, T *out,
                                                         T omega, int zebra, int colour) {
  MG_PDL_WAIT();
  extern __shared__ __align__(16) unsigned char xw_raw[];
  constexpr int NB = KIND == K_CONST ? 1 : 4;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T *sd = reinterpret_cast<T *>(xw_raw) + (size_t)warp * NB * WBUF;
  T *sa = sd + WBUF, *sb = sa + WBUF, *sc = sb + WBUF;
  const long long line = (long long)blockIdx.x * WL + warp;
  if (line >= L.unk_rows()) return;   // the whole warp
  int j, k;
  row_jk(L, line, j, k);
  if (zebra && ((j + k) & 1) != colour) return;   // the whole warp
  const int m = L.n0 - 2;
  const long long row = (long long)k * L.plane + (long long)j * L.pitch;
  long long dm, dp;
  yoffs(L, j, dm, dp);
  {   // debug build: the line and its neighbour lines lie inside the arrays (uniform per warp)
    const long long zp = DIM == 3 ? L.plane : 0;
    if (!MG_CK(L, row + 1 + (dm < dp ? dm : dp) - zp) || !MG_CK(L, row + m + (dm < dp ? dp : dm) + zp)) return;
  }
  // 1. right-hand side (g + off-line couplings) and the line's coefficients, coalesced
  for (int q = lane; q < m; q += 32) {
    int i = q + 1;
    long long p = row + i;
    Weights<T, DIM, KIND> w;
    w.load(L, i, p, dm);
    T d = g[p];
    d = fma(w.wS, u[p + dm], d);
    d = fma(w.wN, u[p + dp], d);
    if (DIM == 3) {
      d = fma(w.wB, u[p - L.plane], d);
      d = fma(w.wF, u[p + L.plane], d);
    }
    sd[skew(q)] = d;
    if (KIND != K_CONST) {
      T D = (w.wW + w.wE) + (w.wS + w.wN);
      if (DIM == 3) D += w.wB + w.wF;
      sa[skew(q)] = q > 0 ? -w.wW : T(0);
      sb[skew(q)] = D;
      sc[skew(q)] = q < m - 1 ? -w.wE : T(0);
    }
  }
  __syncwarp();
  // 2. this lane's segment: m split over min(32, m / 2) lanes, >= 2 unknowns each (the reduced
  // form of a one-unknown segment below is exact only for a line of one unknown)
  const int nt = m / 2 < 32 ? (m / 2 > 0 ? m / 2 : 1) : 32;
  int n = 0, s0 = 0;
  if (lane < nt) {
    const int per = m / nt, extra = m % nt;
    n = per + (lane < extra ? 1 : 0);
    s0 = lane * per + (lane < extra ? lane : extra);
  }
  auto A = [&](int q) -> T { return KIND == K_CONST ? (q > 0 ? -L.cx : T(0)) : sa[skew(q)]; };
  auto B = [&](int q) -> T { return KIND == K_CONST ? L.d : sb[skew(q)]; };
  auto Cc = [&](int q) -> T { return KIND == K_CONST ? (q < m - 1 ? -L.cx : T(0)) : sc[skew(q)]; };
  T ap[WSMAX], cp[WSMAX], dpv[WSMAX];
  // top and bottom reduced equations of the segment (identity rows for a lane without unknowns)
  T ta = T(0), tb = T(1), tc = T(0), td = T(0);
  T ba = T(0), bb = T(1), bc = T(0), bd = T(0);
  if (n == 1) {   // m == 1: the line's one equation (no couplings), and x_last - x_first = 0
    ta = A(s0); tb = B(s0); tc = Cc(s0); td = sd[skew(s0)];
    ba = T(-1);
  } else if (n >= 2) {
#pragma unroll
    for (int q = 1; q < WSMAX; ++q) {
      if (q < n) {
        int gq = s0 + q;
        T a = A(gq), b = B(gq), c = Cc(gq), d = sd[skew(gq)];
        if (q == 1) {
          T r = T(1) / b;
          ap[1] = a * r;
          cp[1] = c * r;
          dpv[1] = d * r;
        } else {
          T r = T(1) / (b - a * cp[q - 1]);
          ap[q] = -r * a * ap[q - 1];
          cp[q] = r * c;
          dpv[q] = r * (d - a * dpv[q - 1]);
        }
        ba = ap[q];
        bc = cp[q];
        bd = dpv[q];
      }
    }
#pragma unroll
    for (int q = WSMAX - 2; q >= 1; --q) {
      if (q <= n - 3) {
        dpv[q] = dpv[q] - cp[q] * dpv[q + 1];
        ap[q] = ap[q] - cp[q] * ap[q + 1];
        cp[q] = -cp[q] * cp[q + 1];
      }
    }
    T a0 = A(s0), b0 = B(s0), c0 = Cc(s0), d0 = sd[skew(s0)];
    ta = a0;
    if (n == 2) {
      tb = b0; tc = c0; td = d0;
    } else {
      tb = b0 - c0 * ap[1];
      tc = -c0 * cp[1];
      td = d0 - c0 * dpv[1];
    }
  }
  // 3. parallel cyclic reduction of the 64 equations (top of lane t: 2t, bottom: 2t + 1)
  const unsigned full = 0xffffffffu;
  auto reduce = [&](T &a, T &b, T &c, T &d, bool hl, T la, T lb, T lc, T ld, bool hr, T ra, T rb, T rc, T rd) {
    T na = T(0), nc = T(0);
    if (hl) {
      T al = -a / lb;
      na = al * la;
      b = fma(al, lc, b);
      d = fma(al, ld, d);
    }
    if (hr) {
      T ga = -c / rb;
      nc = ga * rc;
      b = fma(ga, ra, b);
      d = fma(ga, rd, d);
    }
    a = na;
    c = nc;
  };
  {   // stride 1: the top's neighbours are the previous lane's bottom and this lane's bottom
    T pa = __shfl_up_sync(full, ba, 1), pb = __shfl_up_sync(full, bb, 1);
    T pc = __shfl_up_sync(full, bc, 1), pd = __shfl_up_sync(full, bd, 1);
    T xa = __shfl_down_sync(full, ta, 1), xb = __shfl_down_sync(full, tb, 1);
    T xc = __shfl_down_sync(full, tc, 1), xd = __shfl_down_sync(full, td, 1);
    T ta0 = ta, tb0 = tb, tc0 = tc, td0 = td;
    reduce(ta, tb, tc, td, lane > 0, pa, pb, pc, pd, true, ba, bb, bc, bd);
    reduce(ba, bb, bc, bd, true, ta0, tb0, tc0, td0, lane < 31, xa, xb, xc, xd);
  }
#pragma unroll
  for (int h = 1; h < 32; h <<= 1) {   // stride 2h: lanes h apart, top with top, bottom with bottom
    T pta = __shfl_up_sync(full, ta, h), ptb = __shfl_up_sync(full, tb, h);
    T ptc = __shfl_up_sync(full, tc, h), ptd = __shfl_up_sync(full, td, h);
    T nta = __shfl_down_sync(full, ta, h), ntb = __shfl_down_sync(full, tb, h);
    T ntc = __shfl_down_sync(full, tc, h), ntd = __shfl_down_sync(full, td, h);
    T pba = __shfl_up_sync(full, ba, h), pbb = __shfl_up_sync(full, bb, h);
    T pbc = __shfl_up_sync(full, bc, h), pbd = __shfl_up_sync(full, bd, h);
    T nba = __shfl_down_sync(full, ba, h), nbb = __shfl_down_sync(full, bb, h);
    T nbc = __shfl_down_sync(full, bc, h), nbd = __shfl_down_sync(full, bd, h);
    const bool hl = lane >= h, hr = lane + h < 32;
    reduce(ta, tb, tc, td, hl, pta, ptb, ptc, ptd, hr, nta, ntb, ntc, ntd);
    reduce(ba, bb, bc, bd, hl, pba, pbb, pbc, pbd, hr, nba, nbb, nbc, nbd);
  }
  // 4. interior unknowns, damped update, write back
  __syncwarp();
  if (n >= 1) {
    T x0 = td / tb, xl = bd / bb;
    sd[skew(s0)] = x0;
    if (n >= 2) sd[skew(s0 + n - 1)] = xl;
#pragma unroll
    for (int q = 1; q < WSMAX - 1; ++q)
      if (q <= n - 2) sd[skew(s0 + q)] = dpv[q] - ap[q] * x0 - cp[q] * xl;
  }
  __syncwarp();
  for (int q = lane; q < m; q += 32) {
    long long p = row + q + 1;
    T x = sd[skew(q)];
    out[p] = (omega == T(1)) ? x : fma(omega, x - u[p], u[p]);
  }
}

template <typename T>
bool launch_xline(const Launch &lc, const Lev<T> &L, int kind, int zebra, int colour, const T *u, const T *g, T *out,
                  T omega) {
  int m = L.n0 - 2;
  if (m < 1 || m > NT * SMAX) return false;
  unsigned nl = (unsigned)L.unk_rows();
  if (m <= 32 * WSMAX) {
    size_t smemw = sizeof(T) * (kind == K_CONST ? 1 : 4) * (size_t)WBUF * WL;
    unsigned blocks = (nl + WL - 1) / WL;
#define XW(D, K)                                                                                         \
  do {                                                                                                   \
    cudaFuncSetAttribute(k_xline_warp<T, D, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smemw); \
    k_xline_warp<T, D, K><<<blocks, 32 * WL, smemw, lc.s>>>(L, u, g, out, omega, zebra, colour);          \
  } while (0)
    if (L.dim == 2) {
      if (kind == K_CONST) XW(2, K_CONST); else if (kind == K_SEP) XW(2, K_SEP); else if (kind == K_CELL) XW(2, K_CELL); else XW(2, K_EDGE);
    } else {
      if (kind == K_CONST) XW(3, K_CONST); else if (kind == K_SEP) XW(3, K_SEP); else if (kind == K_CELL) XW(3, K_CELL); else XW(3, K_EDGE);
    }
#undef XW
    lc.done(__func__);
    return true;
  }
  size_t smem = sizeof(T) * ((kind == K_CONST ? 1 : 4) * (size_t)XL_SZ + 16 * NT);
#define XL(D, K)                                                                                   \
  do {                                                                                             \
    cudaFuncSetAttribute(k_xline<T, D, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    k_xline<T, D, K><<<nl, NT, smem, lc.s>>>(L, u, g, out, omega, zebra, colour);                  \
  } while (0)
  if (L.dim == 2) {
    if (kind == K_CONST) XL(2, K_CONST); else if (kind == K_SEP) XL(2, K_SEP); else if (kind == K_CELL) XL(2, K_CELL); else XL(2, K_EDGE);
  } else {
    if (kind == K_CONST) XL(3, K_CONST); else if (kind == K_SEP) XL(3, K_SEP); else if (kind == K_CELL) XL(3, K_CELL); else XL(3, K_EDGE);
  }
#undef XL
  lc.done(__func__);
  return true;
}

template bool launch_xline<double>(const Launch &, const Lev<double> &, int, int, int, const double *, const double *,
                                   double *, double);
template bool launch_xline<float>(const Launch &, const Lev<float> &, int, int, int, const float *, const float *,
                                  float *, float);

}  // namespace mg
