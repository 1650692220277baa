// kernels_march.cu -- column-marching fused red-black sweep (2-D, constant or separable
// coefficients), the HBM-rate form of one Gauss-Seidel sweep in red-black order
// (Wallis 2008, section "The choice of C": C = D + L).
//
// One warp streams a strip of 32 x NV columns (NV = 4 floats / 2 doubles per thread,
// one 16-byte vector) down a chunk of RC rows.  Per row it loads, one row ahead of use:
// the old iterate and g of the thread's columns; the strip-edge lanes also load the
// outside column's u, the u beyond it and its g.  For output row r the window holds
// the old rows r .. r+2 and the half-updated rows H_{r-1}, H_r, H_{r+1} (first colour
// relaxed, second colour old); H_{r+1} is formed when row r+2 is in registers, then
// the second colour of row r is relaxed from H and the row is stored.  x-neighbours
// come from warp shuffles; the edge lanes recompute the outside first-colour value
// from their prefetched scalars.  Each node is read once and written once:
// 12 B / unknown in FP32, 24 B in FP64.
#define MG_FILE_ID 7   // bounds-check sites (-DMG_DEBUG)
#include "mg_internal.cuh"

namespace mg {

namespace {
template <typename T> struct Vec;
template <> struct Vec<float> { using V = float4; static constexpr int N = 4; };
template <> struct Vec<double> { using V = double2; static constexpr int N = 2; };

// one row of the window: thread columns, their g, and the edge-lane scalars
template <typename T>
struct RowW {
  T u[Vec<T>::N], g[Vec<T>::N];
  T out;    // u of the outside column (i0-1 for lane 0, i0+NV for lane 31; neighbour lanes: shuffled)
  T out2;   // u one column further out (edge lanes only)
  T gout;   // g of the outside column (edge lanes only)
};

template <typename T>
__device__ __forceinline__ void vload(T (&r)[Vec<T>::N], const T *p) {
  typename Vec<T>::V x = *reinterpret_cast<const typename Vec<T>::V *>(p);
  if constexpr (Vec<T>::N == 4) {
    r[0] = x.x; r[1] = x.y; r[2] = x.z; r[3] = x.w;
  } else {
    r[0] = x.x; r[1] = x.y;
  }
}
template <typename T>
__device__ __forceinline__ void vstore(T *p, const T (&r)[Vec<T>::N]) {
  typename Vec<T>::V x;
  if constexpr (Vec<T>::N == 4) {
    x.x = r[0]; x.y = r[1]; x.z = r[2]; x.w = r[3];
  } else {
    x.x = r[0]; x.y = r[1];
  }
  *reinterpret_cast<typename Vec<T>::V *>(p) = x;
}
}  // namespace

template <typename T, int KIND, int MODE>
__global__ void __launch_bounds__(128) k_rb2d_march(Lev<T> L, const T *__restrict__ u, const T *__restrict__ g,
                                                    T *__restrict__ out, T omega, int first, Lev<T> C,
                                                    const T *__restrict__ ec, T omega_corr, int RC) {
  MG_PDL_WAIT();
  constexpr int NV = Vec<T>::N;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int wg = blockIdx.x * 4 + (threadIdx.x >> 5);
  const int nstrips = (int)(L.pitch / (32 * NV));
  const int strip = wg % nstrips, chunk = wg / nstrips;
  const int ylo = L.per ? 0 : 1, yhi = L.per ? L.n1 - 1 : L.n1 - 2;   // unknown rows
  const int j0 = ylo + chunk * RC;
  if (j0 > yhi) return;   // uniform per warp
  const int j1 = min(j0 + RC, yhi + 1);
  const int i0 = strip * 32 * NV + lane * NV;   // first column of this thread
  const bool edge = lane == 0 || lane == 31;
  const int io = lane == 0 ? i0 - 1 : i0 + NV;  // outside column of an edge lane
  const int io2 = lane == 0 ? i0 - 2 : i0 + NV + 1;

  // ---- coefficients: per column (separable) or scalars (constant) ----
  bool act[NV];
  T sW[NV], sE[NV], sY[NV], sD[NV], sO[NV];
#pragma unroll
  for (int e = 0; e < NV; ++e) {
    int i = i0 + e;
    act[e] = i >= 1 && i <= L.n0 - 2;
    if (KIND == K_SEP) {
      int ic = act[e] ? i : 1;
      sW[e] = L.sx[ic - 1]; sE[e] = L.sx[ic]; sY[e] = L.sy[ic];
      sD[e] = (sW[e] + sE[e]) + (sY[e] + sY[e]);
      sO[e] = omega * L.sdinv[ic];
    }
  }
  const T cW = L.cx, cY = L.cy, cD = L.d, cO = omega * L.dinv;
#define CW(e) (KIND == K_CONST ? cW : sW[e])
#define CE(e) (KIND == K_CONST ? cW : sE[e])
#define CY(e) (KIND == K_CONST ? cY : sY[e])
#define CD(e) (KIND == K_CONST ? cD : sD[e])
#define CO(e) (KIND == K_CONST ? cO : sO[e])
  // coefficients of the outside column (edge lanes)
  const bool oact = io >= 1 && io <= L.n0 - 2;
  T oW = cW, oE = cW, oY = cY, oD = cD, oO = cO;
  if (KIND == K_SEP && edge) {
    int ic = oact ? io : 1;
    oW = L.sx[ic - 1]; oE = L.sx[ic]; oY = L.sy[ic];
    oD = (oW + oE) + (oY + oY);
    oO = omega * L.sdinv[ic];
  }

  auto wrap = [&](int j) -> int {
    if (!L.per) return j;
    j = j < 0 ? j + L.n1 : (j >= L.n1 ? j - L.n1 : j);
    if (j < 0 || j >= L.n1) j = ((j % L.n1) + L.n1) % L.n1;
    return j;
  };
  auto row_ok = [&](int j) { return L.per || (j >= 0 && j < L.n1); };
  auto unk_row = [&](int j) { return L.per || (j >= 1 && j <= L.n1 - 2); };
  // coarse-grid correction omega_corr P ec at (i, j)
  auto corr = [&](int i, int jw) -> T {
    int J0 = jw >> 1, J1 = (jw + 1) >> 1;
    if (J1 >= C.n1) J1 -= C.n1;
    const T *e0 = ec + (long long)J0 * C.pitch, *e1 = ec + (long long)J1 * C.pitch;
    int I0 = i >> 1, I1 = (i + 1) >> 1;
    return omega_corr * (((e0[I0] + e0[I1]) + (e1[I0] + e1[I1])) * T(0.25));
  };

  // ---- load one row of the window ----
  auto load_row = [&](RowW<T> &R, int j) {
    bool ok = row_ok(j);
    int jw = wrap(j);
    if (ok && (!MG_CKN(L, jw, L.n1) || !MG_CKN(L, i0 + NV - 1, L.pitch))) ok = false;   // debug build
    const T *up = u + (long long)jw * L.pitch, *gp = g + (long long)jw * L.pitch;
    if (ok) {
      if (MODE != 1) vload<T>(R.u, up + i0);
      vload<T>(R.g, gp + i0);
    }
#pragma unroll
    for (int e = 0; e < NV; ++e) {
      if (!ok) R.g[e] = T(0);
      if (MODE == 1 || !ok) R.u[e] = T(0);
    }
    R.out = T(0);
    R.out2 = T(0);
    R.gout = T(0);
    if (edge && ok) {
      if (MODE != 1) {
        if (io >= 0 && io < L.pitch) R.out = up[io];
        if (io2 >= 0 && io2 < L.pitch) R.out2 = up[io2];
      }
      if (io >= 0 && io < L.pitch) R.gout = gp[io];
    }
    if (MODE == 2 && unk_row(j) && MG_CKN(C, (jw + 1) >> 1 >= C.n1 ? 0 : (jw + 1) >> 1, C.n1) &&
        MG_CKN(C, jw >> 1, C.n1)) {
      // coarse values of the thread's columns: coarse columns c0 .. c0 + NV/2 of rows J0, J1
      int J0 = jw >> 1, J1 = (jw + 1) >> 1;
      if (J1 >= C.n1) J1 -= C.n1;
      const T *e0 = ec + (long long)J0 * C.pitch, *e1 = ec + (long long)J1 * C.pitch;
      const int c0 = i0 >> 1;
      T s[NV / 2 + 1];
#pragma unroll
      for (int q = 0; q <= NV / 2; ++q) s[q] = (c0 + q < C.n0) ? e0[c0 + q] + e1[c0 + q] : T(0);
#pragma unroll
      for (int e = 0; e < NV; ++e)
        if (act[e]) R.u[e] += omega_corr * ((s[e >> 1] + s[(e + 1) >> 1]) * T(0.25));
      if (edge) {
        if (oact) R.out += corr(io, jw);
        if (io2 >= 1 && io2 <= L.n0 - 2) R.out2 += corr(io2, jw);
      }
    }
  };
  auto is_first = [&](int i, int j) { return ((i + j) & 1) == first; };

  // Relax the elements of one colour of a row (o = c elsewhere): in each pair (2k, 2k+1) of
  // the thread's columns exactly one node has that colour, the one with index parity p, so
  // operands are selected instead of relaxing both and discarding one.
  auto relax_sel = [&](T (&o)[NV], const T (&c)[NV], T left, T right, const T (&n)[NV], const T (&s)[NV],
                       const T (&gg)[NV], int p, bool rowok) {
#pragma unroll
    for (int k = 0; k < NV / 2; ++k) {
      const int a = 2 * k, b = 2 * k + 1;
      T cc = p ? c[b] : c[a];
      T wv = p ? c[a] : (a > 0 ? c[a - 1] : left);
      T ev = p ? (b + 1 < NV ? c[b + 1] : right) : c[b];
      T nn = p ? n[b] : n[a], ss = p ? s[b] : s[a], gv = p ? gg[b] : gg[a];
      T r = fma(-(p ? CD(b) : CD(a)), cc, gv);
      r = fma(p ? CW(b) : CW(a), wv, r);
      r = fma(p ? CE(b) : CE(a), ev, r);
      T y = p ? CY(b) : CY(a);
      r = fma(y, nn, r);
      r = fma(y, ss, r);
      T nv = fma(p ? CO(b) : CO(a), r, cc);
      bool on = rowok && (p ? act[b] : act[a]);
      o[a] = (!p && on) ? nv : c[a];
      o[b] = (p && on) ? nv : c[b];
    }
  };

  // ---- first colour relaxed on row j (Rm, R, Rp = rows j-1, j, j+1) -> H (+ outside value ho) ----
  auto half_row = [&](T (&H)[NV], T &ho, const RowW<T> &Rm, const RowW<T> &R, const RowW<T> &Rp, int j) {
    T left = __shfl_up_sync(FULL, R.u[NV - 1], 1), right = __shfl_down_sync(FULL, R.u[0], 1);
    if (lane == 0) left = R.out;
    if (lane == 31) right = R.out;
    bool rowu = unk_row(j);
    // first-colour columns of row j have index parity (first + j) % 2 (i0 is even)
    relax_sel(H, R.u, left, right, Rm.u, Rp.u, R.g, (first + j) & 1, rowu);
    ho = R.out;
    if (edge && rowu && oact && is_first(io, j)) {
      T w_ = lane == 0 ? R.out2 : R.u[NV - 1], e_ = lane == 0 ? R.u[0] : R.out2;
      T s = fma(-oD, R.out, R.gout);
      s = fma(oW, w_, s);
      s = fma(oE, e_, s);
      s = fma(oY, Rm.out, s);
      s = fma(oY, Rp.out, s);
      ho = fma(oO, s, R.out);
    }
  };

  // ---- prologue ----
  RowW<T> W0, W1, W2, W3;   // rows j, j+1, j+2 (in use), j+3 (in flight)
  T Hm[NV], Hc[NV], Hp[NV], hom, hoc, hop;
  {
    RowW<T> Wa;   // row j0-2
    load_row(Wa, j0 - 2);
    RowW<T> Wb;   // row j0-1
    load_row(Wb, j0 - 1);
    load_row(W0, j0);
    load_row(W1, j0 + 1);
    load_row(W2, j0 + 2);
    half_row(Hm, hom, Wa, Wb, W0, j0 - 1);
    half_row(Hc, hoc, Wb, W0, W1, j0);
  }
  // One output row.  The window rotates by renaming: the loop below is unrolled over the
  // 12 rotations of (4 row slots, 3 half-row slots), so no registers are copied.
  auto step = [&](RowW<T> &w0, RowW<T> &w1, RowW<T> &w2, RowW<T> &w3, T (&hm)[NV], T &hom_, T (&hc)[NV], T &hoc_,
                  T (&hp)[NV], T &hop_, int j) {
    (void)hom_;
    load_row(w3, j + 3);                    // prefetch, consumed by the next row
    half_row(hp, hop_, w0, w1, w2, j + 1);
    T hl = __shfl_up_sync(FULL, hc[NV - 1], 1), hr = __shfl_down_sync(FULL, hc[0], 1);
    if (lane == 0) hl = hoc_;
    if (lane == 31) hr = hoc_;
    // second colour on row j; its own values are still the old ones in hc
    T O[NV];
    relax_sel(O, hc, hl, hr, hm, hp, w0.g, 1 - ((first + j) & 1), true);
    if (MG_CK(L, (long long)j * L.pitch + i0 + NV - 1))
      vstore<T>(out + (long long)j * L.pitch + i0, O);   // rows j0 .. j1-1 are real unknown rows
  };
  for (int j = j0; j < j1; j += 12) {
    step(W0, W1, W2, W3, Hm, hom, Hc, hoc, Hp, hop, j);
    if (j + 1 >= j1) break;
    step(W1, W2, W3, W0, Hc, hoc, Hp, hop, Hm, hom, j + 1);
    if (j + 2 >= j1) break;
    step(W2, W3, W0, W1, Hp, hop, Hm, hom, Hc, hoc, j + 2);
    if (j + 3 >= j1) break;
    step(W3, W0, W1, W2, Hm, hom, Hc, hoc, Hp, hop, j + 3);
    if (j + 4 >= j1) break;
    step(W0, W1, W2, W3, Hc, hoc, Hp, hop, Hm, hom, j + 4);
    if (j + 5 >= j1) break;
    step(W1, W2, W3, W0, Hp, hop, Hm, hom, Hc, hoc, j + 5);
    if (j + 6 >= j1) break;
    step(W2, W3, W0, W1, Hm, hom, Hc, hoc, Hp, hop, j + 6);
    if (j + 7 >= j1) break;
    step(W3, W0, W1, W2, Hc, hoc, Hp, hop, Hm, hom, j + 7);
    if (j + 8 >= j1) break;
    step(W0, W1, W2, W3, Hp, hop, Hm, hom, Hc, hoc, j + 8);
    if (j + 9 >= j1) break;
    step(W1, W2, W3, W0, Hm, hom, Hc, hoc, Hp, hop, j + 9);
    if (j + 10 >= j1) break;
    step(W2, W3, W0, W1, Hc, hoc, Hp, hop, Hm, hom, j + 10);
    if (j + 11 >= j1) break;
    step(W3, W0, W1, W2, Hp, hop, Hm, hom, Hc, hoc, j + 11);
  }
#undef CW
#undef CE
#undef CY
#undef CD
#undef CO
}

template <typename T>
bool launch_rb2d_march(const Launch &lc, const Lev<T> &L, int kind, const T *u, const T *g, T *out, T omega,
                       int first, int mode, const Lev<T> *C, const T *ec, T omega_corr) {
  constexpr int NV = Vec<T>::N;
  if (L.dim != 2 || kind == K_CELL || kind == K_EDGE || L.pitch % (32 * NV) != 0) return false;
  int rows = L.per ? L.n1 : L.n1 - 2;
  int RC = 32;
  int nstrips = (int)(L.pitch / (32 * NV));
  int nchunks = (rows + RC - 1) / RC;
  long long warps = (long long)nstrips * nchunks;
  unsigned blocks = (unsigned)((warps + 3) / 4);
  Lev<T> Cv = C ? *C : L;
  const T *e = ec ? ec : u;
#define MARCH(K, M) k_rb2d_march<T, K, M><<<blocks, 128, 0, lc.s>>>(L, u, g, out, omega, first, Cv, e, omega_corr, RC)
  if (kind == K_CONST) {
    if (mode == 0) MARCH(K_CONST, 0); else if (mode == 1) MARCH(K_CONST, 1); else MARCH(K_CONST, 2);
  } else {
    if (mode == 0) MARCH(K_SEP, 0); else if (mode == 1) MARCH(K_SEP, 1); else MARCH(K_SEP, 2);
  }
#undef MARCH
  lc.done(__func__);
  return true;
}

template bool launch_rb2d_march<double>(const Launch &, const Lev<double> &, int, const double *, const double *,
                                        double *, double, int, int, const Lev<double> *, const double *, double);
template bool launch_rb2d_march<float>(const Launch &, const Lev<float> &, int, const float *, const float *, float *,
                                       float, int, int, const Lev<float> *, const float *, float);

}  // namespace mg
