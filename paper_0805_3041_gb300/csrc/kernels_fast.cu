// kernels_fast.cu -- fused 2-D kernels of the hot path.
//
//  * k_rb2d: one complete red-black Gauss-Seidel sweep (C = D + L in red-black
//    order, Wallis 2008, section "The choice of C") in a single pass, out of
//    place.  A 64 x 16 output tile is staged in shared memory with a halo of 2
//    for u and 1 for g; the first colour is relaxed on the tile plus a one-node
//    ring, the second colour on the tile, and the tile is written back.  Reads u
//    and g once and writes u once (12 B / unknown in FP32, 24 in FP64), against
//    twice that for two half-sweeps.  Optional fusions in the load stage: a zero
//    iterate (first pre-smoothing sweep after restriction: u is not read) and
//    the coarse-grid correction u + omega_l P e (first post-smoothing sweep:
//    the prolongation never makes its own pass over u).
//  * k_defect_restrict2d: d = g - A u on a fine tile and g_c = R d (full
//    weighting) of the 32 x 8 coarse nodes it covers, without writing d.
#include "mg_internal.cuh"

namespace mg {

namespace {
constexpr int TX = 64, TY = 16, HX = TX + 4, HY = TY + 4;   // RB tile and its halo-2 extent
constexpr int CX = 32, CY = 8;                              // coarse tile of the defect/restriction

template <typename T>
__device__ __forceinline__ T load_or_zero(const T *__restrict__ a, const Lev<T> &L, int i, int j) {
  if (i < 0 || i >= L.n0) return T(0);
  if (L.per) {
    j = (j % L.n1 + L.n1) % L.n1;
  } else if (j < 0 || j >= L.n1) {
    return T(0);
  }
  return a[(long long)j * L.pitch + i];
}

// node (i, j) of the staged region is an unknown (a periodic row outside [0, n1) is the
// wrapped copy of a real row and is relaxed like it)
template <typename T>
__device__ __forceinline__ bool unknown2d(const Lev<T> &L, int i, int j) {
  return i >= 1 && i <= L.n0 - 2 && (L.per ? true : (j >= 1 && j <= L.n1 - 2));
}
// node (i, j) is an unknown owned by this tile (real rows only)
template <typename T>
__device__ __forceinline__ bool owned2d(const Lev<T> &L, int i, int j) {
  return i >= 1 && i <= L.n0 - 2 && (L.per ? (j >= 0 && j < L.n1) : (j >= 1 && j <= L.n1 - 2));
}

// wrapped row offset of node row j (j may be -1 or n1 for a periodic grid)
template <typename T>
__device__ __forceinline__ long long row_of(const Lev<T> &L, int j) {
  if (L.per) j = (j % L.n1 + L.n1) % L.n1;
  return (long long)j * L.pitch;
}

// relax node (i, j) whose stencil values sit in shared memory at (r, c) of s (row stride SX)
template <typename T, int KIND, int SX>
__device__ __forceinline__ T relax_smem(const Lev<T> &L, const T (*s)[SX], int r, int c, T gp, int i, int j,
                                        T omega) {
  long long p = row_of(L, j) + i;
  long long dm = row_of(L, j - 1) - row_of(L, j);
  Weights<T, 2, KIND> w;
  w.load(L, i, p, dm);
  T uc = s[r][c];
  T sum;
  if (KIND == K_CONST) {
    sum = fma(-L.d, uc, gp);
  } else {
    T D = (w.wW + w.wE) + (w.wS + w.wN);
    sum = fma(-D, uc, gp);
  }
  sum = fma(w.wW, s[r][c - 1], sum);
  sum = fma(w.wE, s[r][c + 1], sum);
  sum = fma(w.wS, s[r - 1][c], sum);
  sum = fma(w.wN, s[r + 1][c], sum);
  return fma(omega * w.dinv, sum, uc);
}
}  // namespace

// MODE 0: plain sweep; 1: from a zero iterate; 2: u := u + omega_corr P ec before the sweep
template <typename T, int KIND, int MODE>
__global__ void __launch_bounds__(256) k_rb2d(Lev<T> L, const T *__restrict__ u, const T *__restrict__ g,
                                              T *__restrict__ out, T omega, int first, Lev<T> C,
                                              const T *__restrict__ ec, T omega_corr) {
  __shared__ T su[HY][HX + 1];
  __shared__ T sg[TY + 2][TX + 3];
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  // stage u (halo 2) and g (halo 1)
  for (int e = tid; e < HY * HX; e += 256) {
    int r = e / HX, cc = e % HX;
    int i = i0 - 2 + cc, j = j0 - 2 + r;
    T v = T(0);
    if (MODE != 1) v = load_or_zero(u, L, i, j);
    if (MODE == 2 && unknown2d(L, i, j)) {
      int jw = L.per ? (j % L.n1 + L.n1) % L.n1 : j;
      int I0 = i >> 1, I1 = (i + 1) >> 1, J0 = jw >> 1, J1 = (jw + 1) >> 1;
      if (J1 >= C.n1) J1 -= C.n1;
      long long a0 = (long long)J0 * C.pitch, a1 = (long long)J1 * C.pitch;
      T s = ((ec[a0 + I0] + ec[a0 + I1]) + (ec[a1 + I0] + ec[a1 + I1])) * T(0.25);
      v = fma(omega_corr, s, v);
    }
    su[r][cc] = v;
  }
  for (int e = tid; e < (TY + 2) * (TX + 2); e += 256) {
    int r = e / (TX + 2), cc = e % (TX + 2);
    sg[r][cc] = load_or_zero(g, L, i0 - 1 + cc, j0 - 1 + r);
  }
  __syncthreads();
  // first colour on the tile plus a one-node ring (33 nodes of that colour per extended row)
  for (int e = tid; e < (TY + 2) * 33; e += 256) {
    int rr = e / 33, q = e % 33;
    int j = j0 - 1 + rr;
    int i = i0 - 1 + 2 * q + ((first + i0 + 1 + j) & 1);
    if (i > i0 + TX || !unknown2d(L, i, j)) continue;
    int r = rr + 1, cc = i - i0 + 2;
    su[r][cc] = relax_smem<T, KIND, HX + 1>(L, su, r, cc, sg[rr][i - i0 + 1], i, j, omega);
  }
  __syncthreads();
  // second colour on the tile
  for (int e = tid; e < TY * 32; e += 256) {
    int rr = e / 32, q = e % 32;
    int j = j0 + rr;
    int i = i0 + 2 * q + ((1 - first + i0 + j) & 1);
    if (!owned2d(L, i, j)) continue;
    int r = rr + 2, cc = i - i0 + 2;
    su[r][cc] = relax_smem<T, KIND, HX + 1>(L, su, r, cc, sg[rr + 1][i - i0 + 1], i, j, omega);
  }
  __syncthreads();
  // write the tile's unknowns
  for (int e = tid; e < TY * TX; e += 256) {
    int rr = e / TX, cc = e % TX;
    int i = i0 + cc, j = j0 + rr;
    if (owned2d(L, i, j)) out[(long long)j * L.pitch + i] = su[rr + 2][cc + 2];
  }
}

template <typename T, int KIND>
__global__ void __launch_bounds__(256) k_defect_restrict2d(Lev<T> F, Lev<T> C, const T *__restrict__ u,
                                                           const T *__restrict__ g, T *__restrict__ gc) {
  constexpr int RX = 2 * CX + 1, RY = 2 * CY + 1;   // fine defect region
  __shared__ T su[RY + 2][RX + 3];
  __shared__ T sr[RY][RX + 1];
  const int tid = threadIdx.x;
  const int I0 = blockIdx.x * CX, J0 = blockIdx.y * CY;
  const int fi0 = 2 * I0 - 1, fj0 = 2 * J0 - 1;     // fine origin of the defect region
  for (int e = tid; e < (RY + 2) * (RX + 2); e += 256) {
    int r = e / (RX + 2), cc = e % (RX + 2);
    su[r][cc] = load_or_zero(u, F, fi0 - 1 + cc, fj0 - 1 + r);
  }
  __syncthreads();
  for (int e = tid; e < RY * RX; e += 256) {
    int r = e / RX, cc = e % RX;
    int i = fi0 + cc, j = fj0 + r;
    T d = T(0);
    if (unknown2d(F, i, j)) {
      long long p = row_of(F, j) + i;
      long long dm = row_of(F, j - 1) - row_of(F, j);
      Weights<T, 2, KIND> w;
      w.load(F, i, p, dm);
      T uc = su[r + 1][cc + 1];
      T s;
      if (KIND == K_CONST) {
        s = fma(-F.d, uc, g[p]);
      } else {
        T D = (w.wW + w.wE) + (w.wS + w.wN);
        s = fma(-D, uc, g[p]);
      }
      s = fma(w.wW, su[r + 1][cc], s);
      s = fma(w.wE, su[r + 1][cc + 2], s);
      s = fma(w.wS, su[r][cc + 1], s);
      s = fma(w.wN, su[r + 2][cc + 1], s);
      d = s;
    }
    sr[r][cc] = d;
  }
  __syncthreads();
  int I = I0 + (tid & 31), J = J0 + (tid >> 5);
  if (I >= 1 && I <= C.n0 - 2 && (C.per ? J < C.n1 : (J >= 1 && J <= C.n1 - 2))) {
    int r = 2 * (J - J0) + 1, cc = 2 * (I - I0) + 1;   // centre of the stencil in sr
    auto row3 = [&](int rr) -> T { return (sr[rr][cc - 1] + sr[rr][cc + 1]) + T(2) * sr[rr][cc]; };
    T s = ((row3(r - 1) + row3(r + 1)) + T(2) * row3(r)) * T(0.0625);
    gc[(long long)J * C.pitch + I] = s;
  }
}

template <typename T>
void launch_rb2d(const Launch &lc, const Lev<T> &L, int kind, const T *u, const T *g, T *out, T omega, int first,
                 int mode, const Lev<T> *C, const T *ec, T omega_corr) {
  dim3 gr((L.n0 + TX - 1) / TX, (L.n1 + TY - 1) / TY);
  Lev<T> Cv = C ? *C : L;
#define RB_L(K, M) k_rb2d<T, K, M><<<gr, 256, 0, lc.s>>>(L, u, g, out, omega, first, Cv, ec, omega_corr)
  if (kind == K_CONST) {
    if (mode == 0) RB_L(K_CONST, 0); else if (mode == 1) RB_L(K_CONST, 1); else RB_L(K_CONST, 2);
  } else if (kind == K_SEP) {
    if (mode == 0) RB_L(K_SEP, 0); else if (mode == 1) RB_L(K_SEP, 1); else RB_L(K_SEP, 2);
  } else {
    if (mode == 0) RB_L(K_CELL, 0); else if (mode == 1) RB_L(K_CELL, 1); else RB_L(K_CELL, 2);
  }
#undef RB_L
  ++*lc.counter;
}

template <typename T>
void launch_defect_restrict2d(const Launch &lc, const Lev<T> &F, const Lev<T> &C, int kind, const T *u, const T *g,
                              T *gc) {
  dim3 gr((C.n0 + CX - 1) / CX, (C.n1 + CY - 1) / CY);
  if (kind == K_CONST) k_defect_restrict2d<T, K_CONST><<<gr, 256, 0, lc.s>>>(F, C, u, g, gc);
  else if (kind == K_SEP) k_defect_restrict2d<T, K_SEP><<<gr, 256, 0, lc.s>>>(F, C, u, g, gc);
  else k_defect_restrict2d<T, K_CELL><<<gr, 256, 0, lc.s>>>(F, C, u, g, gc);
  ++*lc.counter;
}

template void launch_rb2d<double>(const Launch &, const Lev<double> &, int, const double *, const double *, double *,
                                  double, int, int, const Lev<double> *, const double *, double);
template void launch_rb2d<float>(const Launch &, const Lev<float> &, int, const float *, const float *, float *, float,
                                 int, int, const Lev<float> *, const float *, float);
template void launch_defect_restrict2d<double>(const Launch &, const Lev<double> &, const Lev<double> &, int,
                                               const double *, const double *, double *);
template void launch_defect_restrict2d<float>(const Launch &, const Lev<float> &, const Lev<float> &, int,
                                              const float *, const float *, float *);

}  // namespace mg
