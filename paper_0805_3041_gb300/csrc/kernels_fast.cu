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
//
// All loops are row-per-warp (8 warps, lanes along x): no integer division per
// element, one bounds / periodic-wrap decision per row, 128-byte aligned
// main-body accesses with the halo columns loaded by a few lanes.
#define MG_FILE_ID 5   // bounds-check sites (-DMG_DEBUG)
#include "mg_internal.cuh"

namespace mg {

namespace {
constexpr int TX = 64, TY = 16;   // RB output tile
// Tile widths of the multi-sweep kernels: the widest half-sweep region (tile + 2 (2 NS - 1)
// columns; + 2 (2 NS + 1) with the fused defect) is 64 columns, 32 nodes of one colour a row,
// so every row of every half-sweep is one pass of a full warp.  Even, so that a tile's first
// column has the parity of its index and coarse node I sits at fine column 2I.
template <int NS>
constexpr int kTxNs = 64 - 2 * (2 * NS - 1);
template <int NS>
constexpr int kTxNsDr = 64 - 2 * (2 * NS + 1);
constexpr int SX = TX + 5;        // smem row stride of the u tile (halo 2 + pad)
constexpr int CX = 32;            // coarse tile of the defect/restriction: CX x CY_OF(T)
template <typename T>
struct CYOf { static constexpr int v = sizeof(T) == 8 ? 8 : 16; };   // FP64 within 48 KB static smem

// row pointer of node row j, or nullptr for a row outside a Dirichlet grid; periodic rows wrap
template <typename T>
__device__ __forceinline__ const T *row_ptr(const T *a, const Lev<T> &L, int j) {
  if (L.per) {
    j = j < 0 ? j + L.n1 : (j >= L.n1 ? j - L.n1 : j);
    if (j < 0 || j >= L.n1) j = ((j % L.n1) + L.n1) % L.n1;   // tiny periodic grids
  } else if (j < 0 || j >= L.n1) {
    return nullptr;
  }
  if (!MG_CKN(L, j, L.n1)) return nullptr;
  return a + (long long)j * L.pitch;
}
template <typename T>
__device__ __forceinline__ int wrap_row(const Lev<T> &L, int j) {
  if (!L.per) return j;
  j = j < 0 ? j + L.n1 : (j >= L.n1 ? j - L.n1 : j);
  if (j < 0 || j >= L.n1) j = ((j % L.n1) + L.n1) % L.n1;
  return j;
}
template <typename T>
__device__ __forceinline__ bool unk_row(const Lev<T> &L, int j) {
  return L.per ? true : (j >= 1 && j <= L.n1 - 2);   // periodic rows outside [0, n1) are wrapped copies
}
template <typename T>
__device__ __forceinline__ bool owned_row(const Lev<T> &L, int j) {
  return L.per ? (j >= 0 && j < L.n1) : (j >= 1 && j <= L.n1 - 2);
}

// relax node (i, j) (smem position r, c of a tile with row stride S) with its weights
template <typename T, int KIND, int S>
__device__ __forceinline__ T relax_at(const Lev<T> &L, const T *s, int r, int c, T gp, int i, long long p,
                                      long long dm, T omega) {
  T uc = s[r * S + c];
  if (!MG_CK(L, p) || !MG_CK(L, p + dm)) return uc;   // the weights' reads (cell / edge kinds)
  Weights<T, 2, KIND> w;
  w.load(L, i, p, dm);
  T sum;
  if (KIND == K_CONST) {
    sum = fma(-L.d, uc, gp);
  } else {
    T D = (w.wW + w.wE) + (w.wS + w.wN);
    sum = fma(-D, uc, gp);
  }
  sum = fma(w.wW, s[r * S + c - 1], sum);
  sum = fma(w.wE, s[r * S + c + 1], sum);
  sum = fma(w.wS, s[(r - 1) * S + c], sum);
  sum = fma(w.wN, s[(r + 1) * S + c], sum);
  return fma(omega * w.dinv, sum, uc);
}

// Stage rows [j0 - H, j0 - H + RW) x columns [i0 - H, i0 - H + W) of u and g into shared memory
// (row stride S): every thread first issues all of its loads, then its shared-memory stores, so
// the tile costs one round trip to L2 instead of one per element.  Rows outside a Dirichlet grid
// and columns outside [0, n0) read 0; periodic rows wrap.  MODE 1: u is zero (not read); MODE 2:
// u + omega_corr P ec at the unknowns (the coarse-grid correction folded into the staging).
template <typename T, int KIND, int MODE, int RW, int W, int S>
__device__ __forceinline__ void stage_tile(const Lev<T> &L, const T *__restrict__ u, const T *__restrict__ g, int i0,
                                           int j0, int H, T *su, T *sg, const Lev<T> &C, const T *__restrict__ ec,
                                           T omega_corr) {
  constexpr int N = RW * W, PER = (N + 255) / 256;
  T vu[PER], vg[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int t = (int)threadIdx.x + 256 * q;
    vu[q] = T(0);
    vg[q] = T(0);
    if (t < N) {
      const int r = t / W, c = t - r * W;
      const int j = j0 - H + r, i = i0 - H + c;
      const bool inx = i >= 0 && i < L.n0;
      const T *rp = (MODE == 1) ? nullptr : row_ptr(u, L, j);
      const T *gp = row_ptr(g, L, j);
      if (rp && inx) vu[q] = rp[i];
      if (gp && inx) vg[q] = gp[i];
      if (MODE == 2 && unk_row(L, j) && i >= 1 && i <= L.n0 - 2) {
        const int jw = wrap_row(L, j);
        int J0 = jw >> 1, J1 = (jw + 1) >> 1;
        if (J1 >= C.n1) J1 -= C.n1;
        if (MG_CKN(C, J0, C.n1) && MG_CKN(C, J1, C.n1) && MG_CKN(C, (i + 1) >> 1, C.n0)) {
          const T *e0 = ec + (long long)J0 * C.pitch, *e1 = ec + (long long)J1 * C.pitch;
          const int I0 = i >> 1, I1 = (i + 1) >> 1;
          const T sc = ((e0[I0] + e0[I1]) + (e1[I0] + e1[I1])) * T(0.25);
          vu[q] = fma(omega_corr, sc, vu[q]);
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int t = (int)threadIdx.x + 256 * q;
    if (t < N) {
      const int r = t / W, c = t - r * W;
      su[r * S + c] = vu[q];
      sg[r * S + c] = vg[q];
    }
  }
}
}  // namespace

// MODE 0: plain sweep; 1: from a zero iterate; 2: u := u + omega_corr P ec before the sweep
template <typename T, int KIND, int MODE>
__global__ void __launch_bounds__(256) k_rb2d(Lev<T> L, const T *__restrict__ u, const T *__restrict__ g,
                                              T *__restrict__ out, T omega, int first, Lev<T> C,
                                              const T *__restrict__ ec, T omega_corr) {
  MG_PDL_WAIT();
  __shared__ T su[(TY + 4) * SX];        // u rows j0-2 .. j0+TY+1, columns i0-2 .. i0+TX+1 at c = 0 .. TX+3
  __shared__ T sg[(TY + 2) * SX];        // g rows j0-1 .. j0+TY, columns i0-1 .. i0+TX at c = 1 .. TX+2
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const bool xin = (i0 >= 2) && (i0 + TX + 2 <= L.n0);   // every staged column exists
  // ---- stage u (with the optional fused correction) ----
  for (int r = warp; r < TY + 4; r += 8) {
    int j = j0 - 2 + r;
    const T *rp = (MODE == 1) ? nullptr : row_ptr(u, L, j);
    bool corr = (MODE == 2) && unk_row(L, j);
    int jw = wrap_row(L, j);
    int J0 = jw >> 1, J1 = (jw + 1) >> 1;
    if (J1 >= C.n1) J1 -= C.n1;
    const T *e0 = ec + (long long)J0 * C.pitch, *e1 = ec + (long long)J1 * C.pitch;
    for (int c = lane; c < TX + 4; c += 32) {
      int i = i0 - 2 + c;
      bool inx = xin || (i >= 0 && i < L.n0);
      T v = (rp && inx) ? rp[i] : T(0);
      if (MODE == 2 && corr && i >= 1 && i <= L.n0 - 2 && MG_CKN(C, J0, C.n1) && MG_CKN(C, J1, C.n1) &&
          MG_CKN(C, (i + 1) >> 1, C.n0)) {
        int I0 = i >> 1, I1 = (i + 1) >> 1;
        T s = ((e0[I0] + e0[I1]) + (e1[I0] + e1[I1])) * T(0.25);
        v = fma(omega_corr, s, v);
      }
      su[r * SX + c] = v;
    }
  }
  // ---- stage g ----
  for (int r = warp; r < TY + 2; r += 8) {
    const T *rp = row_ptr(g, L, j0 - 1 + r);
    for (int c = lane; c < TX + 2; c += 32) {
      int i = i0 - 1 + c;
      bool inx = xin || (i >= 0 && i < L.n0);
      sg[r * SX + c + 1] = (rp && inx) ? rp[i] : T(0);
    }
  }
  __syncthreads();
  // ---- first colour on rows j0-1 .. j0+TY, columns i0-1 .. i0+TX ----
  for (int rr = warp; rr < TY + 2; rr += 8) {
    int j = j0 - 1 + rr;
    if (!unk_row(L, j)) continue;
    int jw = wrap_row(L, j);
    long long rowoff = (long long)jw * L.pitch;
    long long dm = (long long)wrap_row(L, jw - 1) * L.pitch - rowoff;
    int par = (first + i0 + 1 + j) & 1;   // i = i0 - 1 + 2q + par has colour `first`
    for (int q = lane; q < TX / 2 + 1; q += 32) {
      int i = i0 - 1 + 2 * q + par;
      if (i < 1 || i > L.n0 - 2 || i > i0 + TX) continue;
      int r = rr + 1, c = i - i0 + 2;
      su[r * SX + c] = relax_at<T, KIND, SX>(L, su, r, c, sg[rr * SX + c], i, rowoff + i, dm, omega);
    }
  }
  __syncthreads();
  // ---- second colour on the tile ----
  for (int rr = warp; rr < TY; rr += 8) {
    int j = j0 + rr;
    if (!owned_row(L, j)) continue;
    long long rowoff = (long long)j * L.pitch;
    long long dm = (long long)wrap_row(L, j - 1) * L.pitch - rowoff;
    int i = i0 + 2 * lane + ((1 - first + i0 + j) & 1);
    if (i < 1 || i > L.n0 - 2) continue;
    int r = rr + 2, c = i - i0 + 2;
    su[r * SX + c] = relax_at<T, KIND, SX>(L, su, r, c, sg[(rr + 1) * SX + c], i, rowoff + i, dm, omega);
  }
  __syncthreads();
  // ---- write the tile's unknowns ----
  for (int rr = warp; rr < TY; rr += 8) {
    int j = j0 + rr;
    if (!owned_row(L, j)) continue;
    T *op = out + (long long)j * L.pitch;
    for (int c = lane; c < TX; c += 32) {
      int i = i0 + c;
      if (i >= 1 && i <= L.n0 - 2 && MG_CK(L, (long long)j * L.pitch + i)) op[i] = su[(rr + 2) * SX + c + 2];
    }
  }
}

// NS complete sweeps in one pass (temporal blocking, for small latency-bound grids): u is
// staged with a halo of 2 NS and g with 2 NS - 1; half-sweep h (colours alternating from
// `first`) relaxes the tile plus a ring of width 2 NS - 1 - h, so every node of the tile
// ends with exactly the values NS successive sweeps give.  MODE applies to the first sweep
// (1: zero iterate, 2: coarse-grid correction folded in), as in k_rb2d.
template <typename T, int KIND, int MODE, int NS, int THY>
__global__ void __launch_bounds__(256) k_rb2d_ns(Lev<T> L, const T *__restrict__ u, const T *__restrict__ g,
                                                 T *__restrict__ out, T omega, int first, Lev<T> C,
                                                 const T *__restrict__ ec, T omega_corr) {
  MG_PDL_WAIT();
  constexpr int TXN = kTxNs<NS>;            // tile width
  constexpr int H = 2 * NS;                 // halo of the u tile
  constexpr int RW = THY + 2 * H;            // staged rows j0-H .. j0+THY+H-1
  constexpr int SXN = TXN + 2 * H + 1;       // smem row stride
  __shared__ T su[RW * SXN];
  __shared__ T sg[RW * SXN];                // same indexing as su (outer ring unused)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = blockIdx.x * TXN, j0 = blockIdx.y * THY;
  // ---- stage u (with the optional fused correction) and g ----
  stage_tile<T, KIND, MODE, RW, TXN + 2 * H, SXN>(L, u, g, i0, j0, H, su, sg, C, ec, omega_corr);
  __syncthreads();
  // ---- 2 NS half-sweeps on shrinking regions ----
#pragma unroll 1
  for (int h = 0; h < 2 * NS; ++h) {
    const int col = (h & 1) ? 1 - first : first, w = 2 * NS - 1 - h;
    for (int rr = warp; rr < THY + 2 * w; rr += 8) {
      int j = j0 - w + rr;
      if (!unk_row(L, j)) continue;
      int jw = wrap_row(L, j);
      long long rowoff = (long long)jw * L.pitch;
      long long dm = (long long)wrap_row(L, jw - 1) * L.pitch - rowoff;
      int ib = i0 - w;                               // first column of the region
      int par = (col + ib + j) & 1;                  // i = ib + 2q + par has colour col
      int r = j - (j0 - H);
      for (int q = lane; 2 * q + par < TXN + 2 * w; q += 32) {
        int i = ib + 2 * q + par;
        if (i < 1 || i > L.n0 - 2) continue;
        int c = i - (i0 - H);
        su[r * SXN + c] = relax_at<T, KIND, SXN>(L, su, r, c, sg[r * SXN + c], i, rowoff + i, dm, omega);
      }
    }
    __syncthreads();
  }
  // ---- write the tile's unknowns ----
  for (int rr = warp; rr < THY; rr += 8) {
    int j = j0 + rr;
    if (!owned_row(L, j)) continue;
    T *op = out + (long long)j * L.pitch;
    for (int c = lane; c < TXN; c += 32) {
      int i = i0 + c;
      if (i >= 1 && i <= L.n0 - 2 && MG_CK(L, (long long)j * L.pitch + i)) op[i] = su[(rr + H) * SXN + c + H];
    }
  }
}

// NS sweeps, then the defect and its full-weighting restriction, in one pass (small grids:
// the pre-smoothing of a level visit and the restriction that follows it).  The sweeps
// run as in k_rb2d_ns on regions 2 nodes wider (halo 2 NS + 2), so the smoothed u is exact
// on the tile plus a ring of 2; the defect is formed on the tile plus a ring of 1 and
// restricted to the tile's 32 x 8 coarse nodes (coarse node I sits at fine 2I).  Writes
// the tile of u and the coarse g; the fine defect is never stored.
template <typename T, int KIND, int MODE, int NS, int THY>
__global__ void __launch_bounds__(256) k_rb2d_ns_dr(Lev<T> L, Lev<T> C, const T *__restrict__ u,
                                                    const T *__restrict__ g, T *__restrict__ out, T omega, int first,
                                                    T *__restrict__ gc) {
  MG_PDL_WAIT();
  constexpr int TXN = kTxNsDr<NS>;          // tile width
  constexpr int H = 2 * NS + 2;             // halo of the u tile
  constexpr int RW = THY + 2 * H;            // staged rows j0-H .. j0+THY+H-1
  constexpr int SXN = TXN + 2 * H + 1;       // smem row stride
  constexpr int DS = TXN + 3;                // stride of the defect tile (rows j0-1 .. j0+THY)
  __shared__ T su[RW * SXN];
  __shared__ T sg[RW * SXN];
  __shared__ T sr[(THY + 2) * DS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i0 = blockIdx.x * TXN, j0 = blockIdx.y * THY;
  stage_tile<T, KIND, MODE == 1 ? 1 : 0, RW, TXN + 2 * H, SXN>(L, u, g, i0, j0, H, su, sg, L, u, T(0));
  __syncthreads();
#pragma unroll 1
  for (int h = 0; h < 2 * NS; ++h) {
    const int col = (h & 1) ? 1 - first : first, w = 2 * NS + 1 - h;
    for (int rr = warp; rr < THY + 2 * w; rr += 8) {
      int j = j0 - w + rr;
      if (!unk_row(L, j)) continue;
      int jw = wrap_row(L, j);
      long long rowoff = (long long)jw * L.pitch;
      long long dm = (long long)wrap_row(L, jw - 1) * L.pitch - rowoff;
      int ib = i0 - w;
      int par = (col + ib + j) & 1;
      int r = j - (j0 - H);
      for (int q = lane; 2 * q + par < TXN + 2 * w; q += 32) {
        int i = ib + 2 * q + par;
        if (i < 1 || i > L.n0 - 2) continue;
        int c = i - (i0 - H);
        su[r * SXN + c] = relax_at<T, KIND, SXN>(L, su, r, c, sg[r * SXN + c], i, rowoff + i, dm, omega);
      }
    }
    __syncthreads();
  }
  // ---- defect on rows j0-1 .. j0+THY, columns i0-1 .. i0+TXN ----
  for (int rr = warp; rr < THY + 2; rr += 8) {
    int j = j0 - 1 + rr;
    bool rowok = unk_row(L, j);
    int jw = wrap_row(L, j);
    long long rowoff = (long long)jw * L.pitch;
    long long dm = (long long)wrap_row(L, jw - 1) * L.pitch - rowoff;
    int r = j - (j0 - H);
    for (int cc = lane; cc < TXN + 2; cc += 32) {
      int i = i0 - 1 + cc;
      T d = T(0);
      if (rowok && i >= 1 && i <= L.n0 - 2 && MG_CK(L, rowoff + i) && MG_CK(L, rowoff + i + dm)) {
        long long p = rowoff + i;
        Weights<T, 2, KIND> wt;
        wt.load(L, i, p, dm);
        const T *sp = su + r * SXN + (i - (i0 - H));
        T uc = sp[0];
        T sum;
        if (KIND == K_CONST) {
          sum = fma(-L.d, uc, sg[r * SXN + (i - (i0 - H))]);
        } else {
          T D = (wt.wW + wt.wE) + (wt.wS + wt.wN);
          sum = fma(-D, uc, sg[r * SXN + (i - (i0 - H))]);
        }
        sum = fma(wt.wW, sp[-1], sum);
        sum = fma(wt.wE, sp[1], sum);
        sum = fma(wt.wS, sp[-SXN], sum);
        sum = fma(wt.wN, sp[SXN], sum);
        d = sum;
      }
      sr[rr * DS + cc] = d;
    }
  }
  __syncthreads();
  // ---- the tile of u, and the coarse g ----
  for (int rr = warp; rr < THY; rr += 8) {
    int j = j0 + rr;
    if (!owned_row(L, j)) continue;
    T *op = out + (long long)j * L.pitch;
    for (int c = lane; c < TXN; c += 32) {
      int i = i0 + c;
      if (i >= 1 && i <= L.n0 - 2 && MG_CK(L, (long long)j * L.pitch + i)) op[i] = su[(rr + H) * SXN + c + H];
    }
  }
  // the tile's THY / 2 coarse rows (TXN / 2 coarse columns), one a warp at a time
  for (int cy = warp; cy < THY / 2; cy += 8) {
    const int I = (i0 >> 1) + lane, J = (j0 >> 1) + cy;
    if (lane < TXN / 2 && I >= 1 && I <= C.n0 - 2 && (C.per ? J < C.n1 : (J >= 1 && J <= C.n1 - 2)) &&
        MG_CK(C, (long long)J * C.pitch + I)) {
      const T *sp = sr + (2 * cy + 1) * DS + (2 * lane + 1);   // fine (2I, 2J) in sr
      auto row3 = [&](const T *q) -> T { return (q[-1] + q[1]) + T(2) * q[0]; };
      gc[(long long)J * C.pitch + I] = ((row3(sp - DS) + row3(sp + DS)) + T(2) * row3(sp)) * T(0.0625);
    }
  }
}

template <typename T, int KIND>
__global__ void __launch_bounds__(256) k_defect_restrict2d(Lev<T> F, Lev<T> C, const T *__restrict__ u,
                                                           const T *__restrict__ g, T *__restrict__ gc) {
  MG_PDL_WAIT();
  constexpr int CY = CYOf<T>::v;
  constexpr int RX = 2 * CX + 1, RY = 2 * CY + 1;   // fine defect region
  constexpr int US = RX + 3;                        // smem stride
  __shared__ T su[(RY + 2) * US];
  __shared__ T sgf[RY * US];
  __shared__ T sr[RY * US];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int I0 = blockIdx.x * CX, J0 = blockIdx.y * CY;
  const int fi0 = 2 * I0 - 1, fj0 = 2 * J0 - 1;     // fine origin of the defect region
  // u (with a ring of 1) and g in one round of loads
  for (int r = warp; r < RY + 2; r += 8) {
    const T *rp = row_ptr(u, F, fj0 - 1 + r);
    const T *gp = (r >= 1 && r <= RY) ? row_ptr(g, F, fj0 - 1 + r) : nullptr;
    for (int c = lane; c < RX + 2; c += 32) {
      int i = fi0 - 1 + c;
      bool inx = i >= 0 && i < F.n0;
      su[r * US + c] = (rp && inx) ? rp[i] : T(0);
      if (r >= 1 && r <= RY && c >= 1 && c <= RX) sgf[(r - 1) * US + (c - 1)] = (gp && inx) ? gp[i] : T(0);
    }
  }
  __syncthreads();
  for (int r = warp; r < RY; r += 8) {
    int j = fj0 + r;
    bool rowok = unk_row(F, j);
    int jw = wrap_row(F, j);
    long long rowoff = (long long)jw * F.pitch;
    long long dm = (long long)wrap_row(F, jw - 1) * F.pitch - rowoff;
    for (int c = lane; c < RX; c += 32) {
      int i = fi0 + c;
      T d = T(0);
      if (rowok && i >= 1 && i <= F.n0 - 2 && MG_CK(F, rowoff + i) && MG_CK(F, rowoff + i + dm)) {
        long long p = rowoff + i;
        Weights<T, 2, KIND> w;
        w.load(F, i, p, dm);
        const T *s = su + (r + 1) * US + (c + 1);
        T uc = s[0];
        T sum;
        if (KIND == K_CONST) {
          sum = fma(-F.d, uc, sgf[r * US + c]);
        } else {
          T D = (w.wW + w.wE) + (w.wS + w.wN);
          sum = fma(-D, uc, sgf[r * US + c]);
        }
        sum = fma(w.wW, s[-1], sum);
        sum = fma(w.wE, s[1], sum);
        sum = fma(w.wS, s[-US], sum);
        sum = fma(w.wN, s[US], sum);
        d = sum;
      }
      sr[r * US + c] = d;
    }
  }
  __syncthreads();
  for (int cy = warp; cy < CY; cy += 8) {
    int I = I0 + lane, J = J0 + cy;
    if (I >= 1 && I <= C.n0 - 2 && (C.per ? J < C.n1 : (J >= 1 && J <= C.n1 - 2)) &&
        MG_CK(C, (long long)J * C.pitch + I)) {
      const T *s = sr + (2 * cy + 1) * US + (2 * lane + 1);   // centre of the stencil in sr
      auto row3 = [&](const T *q) -> T { return (q[-1] + q[1]) + T(2) * q[0]; };
      T v = ((row3(s - US) + row3(s + US)) + T(2) * row3(s)) * T(0.0625);
      gc[(long long)J * C.pitch + I] = v;
    }
  }
}

template <typename T>
void launch_rb2d(const Launch &lc, const Lev<T> &L, int kind, const T *u, const T *g, T *out, T omega, int first,
                 int mode, const Lev<T> *C, const T *ec, T omega_corr) {
  dim3 gr((L.n0 + TX - 1) / TX, (L.n1 + TY - 1) / TY);
  Lev<T> Cv = C ? *C : L;
  const T *e = ec ? ec : u;
#define RB_L(K, M) k_rb2d<T, K, M><<<gr, 256, 0, lc.s>>>(L, u, g, out, omega, first, Cv, e, omega_corr)
  if (kind == K_CONST) {
    if (mode == 0) RB_L(K_CONST, 0); else if (mode == 1) RB_L(K_CONST, 1); else RB_L(K_CONST, 2);
  } else if (kind == K_SEP) {
    if (mode == 0) RB_L(K_SEP, 0); else if (mode == 1) RB_L(K_SEP, 1); else RB_L(K_SEP, 2);
  } else {
    if (kind == K_CELL) {
      if (mode == 0) RB_L(K_CELL, 0); else if (mode == 1) RB_L(K_CELL, 1); else RB_L(K_CELL, 2);
    } else {
      if (mode == 0) RB_L(K_EDGE, 0); else if (mode == 1) RB_L(K_EDGE, 1); else RB_L(K_EDGE, 2);
    }
  }
#undef RB_L
  lc.done(__func__);
}

// Tile height of the two-sweep tile kernels: on small grids each CTA's chain of staging, four
// half-sweeps and stores is the launch's time, and a shorter tile shortens it: 4 rows up to 257^2,
// 8 up to 513^2; above, where the launch is bound by instructions, a taller tile recomputes less
// of its halo: 32 rows in FP32, 16 in FP64 (within 48 KB of static shared memory)
template <typename T>
constexpr int kTileRowsBig = sizeof(T) == 8 ? 16 : 32;
template <typename T>
static inline int tile_rows(const Lev<T> &L) {
  const long long nn = (long long)L.n0 * L.n1;
  return nn <= 66049 ? 4 : nn <= 263169 ? 8 : kTileRowsBig<T>;
}

template <typename T>
void launch_rb2d_2(const Launch &lc, const Lev<T> &L, int kind, const T *u, const T *g, T *out, T omega, int first,
                   int mode, const Lev<T> *C, const T *ec, T omega_corr) {
  const int th = tile_rows(L);
  dim3 gr((L.n0 + kTxNs<2> - 1) / kTxNs<2>, (L.n1 + th - 1) / th);
  Lev<T> Cv = C ? *C : L;
  const T *e = ec ? ec : u;
#define RB2_L(K, M)                                                                                      \
  do {                                                                                                   \
    if (th == 4) k_rb2d_ns<T, K, M, 2, 4><<<gr, 256, 0, lc.s>>>(L, u, g, out, omega, first, Cv, e, omega_corr);  \
    else if (th == 8) k_rb2d_ns<T, K, M, 2, 8><<<gr, 256, 0, lc.s>>>(L, u, g, out, omega, first, Cv, e, omega_corr); \
    else k_rb2d_ns<T, K, M, 2, kTileRowsBig<T>><<<gr, 256, 0, lc.s>>>(L, u, g, out, omega, first, Cv, e, omega_corr); \
  } while (0)
  if (kind == K_CONST) {
    if (mode == 0) RB2_L(K_CONST, 0); else if (mode == 1) RB2_L(K_CONST, 1); else RB2_L(K_CONST, 2);
  } else if (kind == K_SEP) {
    if (mode == 0) RB2_L(K_SEP, 0); else if (mode == 1) RB2_L(K_SEP, 1); else RB2_L(K_SEP, 2);
  } else {
    if (kind == K_CELL) {
      if (mode == 0) RB2_L(K_CELL, 0); else if (mode == 1) RB2_L(K_CELL, 1); else RB2_L(K_CELL, 2);
    } else {
      if (mode == 0) RB2_L(K_EDGE, 0); else if (mode == 1) RB2_L(K_EDGE, 1); else RB2_L(K_EDGE, 2);
    }
  }
#undef RB2_L
  lc.done(__func__);
}

template <typename T>
void launch_rb2d_2_dr(const Launch &lc, const Lev<T> &L, const Lev<T> &C, int kind, const T *u, const T *g, T *out,
                      T omega, int first, int mode, T *gc) {
  const int th = tile_rows(L);
  dim3 gr((L.n0 + kTxNsDr<2> - 1) / kTxNsDr<2>, (L.n1 + th - 1) / th);
#define RB2D_L(K, M)                                                                                   \
  do {                                                                                                 \
    if (th == 4) k_rb2d_ns_dr<T, K, M, 2, 4><<<gr, 256, 0, lc.s>>>(L, C, u, g, out, omega, first, gc);     \
    else if (th == 8) k_rb2d_ns_dr<T, K, M, 2, 8><<<gr, 256, 0, lc.s>>>(L, C, u, g, out, omega, first, gc); \
    else k_rb2d_ns_dr<T, K, M, 2, kTileRowsBig<T>><<<gr, 256, 0, lc.s>>>(L, C, u, g, out, omega, first, gc);  \
  } while (0)
  if (kind == K_CONST) {
    if (mode == 1) RB2D_L(K_CONST, 1); else RB2D_L(K_CONST, 0);
  } else if (kind == K_SEP) {
    if (mode == 1) RB2D_L(K_SEP, 1); else RB2D_L(K_SEP, 0);
  } else {
    if (kind == K_CELL) {
      if (mode == 1) RB2D_L(K_CELL, 1); else RB2D_L(K_CELL, 0);
    } else {
      if (mode == 1) RB2D_L(K_EDGE, 1); else RB2D_L(K_EDGE, 0);
    }
  }
#undef RB2D_L
  lc.done(__func__);
}

template <typename T>
void launch_defect_restrict2d(const Launch &lc, const Lev<T> &F, const Lev<T> &C, int kind, const T *u, const T *g,
                              T *gc) {
  dim3 gr((C.n0 + CX - 1) / CX, (C.n1 + CYOf<T>::v - 1) / CYOf<T>::v);
  if (kind == K_CONST) k_defect_restrict2d<T, K_CONST><<<gr, 256, 0, lc.s>>>(F, C, u, g, gc);
  else if (kind == K_SEP) k_defect_restrict2d<T, K_SEP><<<gr, 256, 0, lc.s>>>(F, C, u, g, gc);
  else if (kind == K_CELL) k_defect_restrict2d<T, K_CELL><<<gr, 256, 0, lc.s>>>(F, C, u, g, gc);
  else k_defect_restrict2d<T, K_EDGE><<<gr, 256, 0, lc.s>>>(F, C, u, g, gc);
  lc.done(__func__);
}

template void launch_rb2d<double>(const Launch &, const Lev<double> &, int, const double *, const double *, double *,
                                  double, int, int, const Lev<double> *, const double *, double);
template void launch_rb2d<float>(const Launch &, const Lev<float> &, int, const float *, const float *, float *, float,
                                 int, int, const Lev<float> *, const float *, float);
template void launch_rb2d_2<double>(const Launch &, const Lev<double> &, int, const double *, const double *, double *,
                                    double, int, int, const Lev<double> *, const double *, double);
template void launch_rb2d_2<float>(const Launch &, const Lev<float> &, int, const float *, const float *, float *,
                                   float, int, int, const Lev<float> *, const float *, float);
template void launch_rb2d_2_dr<double>(const Launch &, const Lev<double> &, const Lev<double> &, int, const double *,
                                       const double *, double *, double, int, int, double *);
template void launch_rb2d_2_dr<float>(const Launch &, const Lev<float> &, const Lev<float> &, int, const float *,
                                      const float *, float *, float, int, int, float *);
template void launch_defect_restrict2d<double>(const Launch &, const Lev<double> &, const Lev<double> &, int,
                                               const double *, const double *, double *);
template void launch_defect_restrict2d<float>(const Launch &, const Lev<float> &, const Lev<float> &, int,
                                              const float *, const float *, float *);

}  // namespace mg
