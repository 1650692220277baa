// kernels_coarse.cu -- the coarse end of the cycle in one CTA.
//
// Every grid at or below a cut-off level lc lives in shared memory (compact
// layout, pitch = n0).  One CTA executes the whole recursive part of the cycle
// below the finer grid that calls it -- pre-smoothing, defect, full-weighting
// restriction, the coarsest solve A_1^{-1} g, bilinear/trilinear correction,
// post-smoothing (Wallis 2008, section "The Multigrid Technique") -- as a
// program of steps built on the host, with one __syncthreads() between steps.
// This turns the ~L^2/2 coarse level visits of an F-cycle, each a handful of
// latency-bound kernels, into a single launch per visit of level lc + 1.
#define MG_FILE_ID 4   // bounds-check sites (-DMG_DEBUG)
#include "mg_internal.cuh"
#include "coarse_prog.h"

namespace mg {

template <typename T>
struct SLev {
  Lev<T> L;              // smem view: pitch = n0, k / ndinv / ex.. point into shared memory
  int off_u0, off_u1, off_g, off_r, off_k, off_dinv;   // element offsets into the smem pool
  int off_ex, off_ey, off_ez;                          // edge weights (-1: not held)
  int off_z;                                           // line-step scratch (-1: not held)
  long long gpitch, gplane;                            // padded global layout of this level
  const T *gk, *gdinv;                                 // global cell data (loaded at start)
  const T *gex, *gey, *gez;                            // global edge weights (loaded at start)
};

template <typename T>
__device__ __forceinline__ T *sarr(T *pool, int off) { return off >= 0 ? pool + off : nullptr; }

// loop over the unknowns of a level (node index p, coordinates i, j, k): working warp wid_
// of nw_ takes rows wid_, wid_ + nw_, ..., its lanes the x positions of the row (no
// divisions per node)
#define FOR_UNK(Lv, ...)                                                                    \
  {                                                                                         \
    int nx_ = (Lv).n0 - 2, ny_ = (Lv).yrows();                                              \
    int rows_ = ny_ * (Lv).zrows();                                                         \
    for (int r_ = wid_; r_ < rows_; r_ += nw_) {                                            \
      int j = (Lv).ylo() + (DIM == 3 ? r_ % ny_ : r_);                                      \
      int k = DIM == 3 ? 1 + r_ / ny_ : 0;                                                  \
      int rowp_ = k * (int)(Lv).plane + j * (int)(Lv).pitch;                                \
      for (int i = 1 + (int)(threadIdx.x & 31); i <= nx_; i += 32) {                        \
        int p = rowp_ + i;                                                                  \
        __VA_ARGS__                                                                         \
      }                                                                                     \
    }                                                                                       \
  }
// the same over the unknowns of one colour ((i + j + k) % 2 == colour)
#define FOR_COLOUR(Lv, colour, ...)                                                         \
  {                                                                                         \
    int nx_ = (Lv).n0 - 2, ny_ = (Lv).yrows();                                              \
    int rows_ = ny_ * (Lv).zrows();                                                         \
    for (int r_ = wid_; r_ < rows_; r_ += nw_) {                                            \
      int j = (Lv).ylo() + (DIM == 3 ? r_ % ny_ : r_);                                      \
      int k = DIM == 3 ? 1 + r_ / ny_ : 0;                                                  \
      int rowp_ = k * (int)(Lv).plane + j * (int)(Lv).pitch;                                \
      int par_ = ((colour) + j + k + 1) & 1;                                                \
      for (int i = 1 + par_ + 2 * (int)(threadIdx.x & 31); i <= nx_; i += 64) {             \
        int p = rowp_ + i;                                                                  \
        __VA_ARGS__                                                                         \
      }                                                                                     \
    }                                                                                       \
  }

static constexpr int CSK_STAGED_OPS = 1024;   // program steps staged in shared memory
// threads of the one CTA: 512 in FP32 (up to 128 registers each), 256 in FP64, where a coarse
// cycle measured 5-10 % faster with fewer, busier threads (65^2: 173 against 183 us a cycle)
template <typename T>
constexpr int csk_threads() {
  return sizeof(T) == 8 ? 256 : 512;
}

// bilinear / trilinear interpolation of the coarse array ec at fine node (i, j, k)
template <typename T, int DIM>
__device__ __forceinline__ T interp_at(const Lev<T> &C, const T *ec, int i, int j, int k) {
  int I0 = i >> 1, I1 = (i + 1) >> 1;
  int J0 = j >> 1, J1 = (j + 1) >> 1;
  if (J1 >= C.n1) J1 -= C.n1;
  int a0 = J0 * (int)C.pitch, a1 = J1 * (int)C.pitch;
  if (DIM == 2) return ((ec[a0 + I0] + ec[a0 + I1]) + (ec[a1 + I0] + ec[a1 + I1])) * T(0.25);
  int z0 = (k >> 1) * (int)C.plane, z1 = ((k + 1) >> 1) * (int)C.plane;
  T s0 = (ec[z0 + a0 + I0] + ec[z0 + a0 + I1]) + (ec[z0 + a1 + I0] + ec[z0 + a1 + I1]);
  T s1 = (ec[z1 + a0 + I0] + ec[z1 + a0 + I1]) + (ec[z1 + a1 + I0] + ec[z1 + a1 + I1]);
  return (s0 + s1) * T(0.125);
}

// Equations a thread holds in one line pass by cyclic reduction: lines x rows <= K * threads.  FP32
// levels of the coarse kernel reach 5000 nodes (the 3-D cut, and the larger of the two cuts the
// autotuner tries in 2-D), FP64 ones 1200 (and twice the registers a value).
template <typename T>
__host__ __device__ constexpr int line_pcr_k() { return sizeof(T) == 4 ? 8 : 4; }

// One line pass (TRI along x or y; the zebra form takes the lines of one colour) on a level held
// in shared memory, with every line solved at once by parallel cyclic reduction.  Row e of a line
// is a x_{e-1} + x_e + c x_{e+1} = d after scaling by its diagonal: sa, sc and sd hold a, c and d
// at the row's node.  At stride s each row takes in rows e - s and e + s and then couples to e -+ 2s.
// A Dirichlet line ends after the stride passes m - 1, with no coupling left.  A periodic line
// (m a power of two) wraps its indices and ends with both couplings on the row itself.
// Thread t holds the equations q = t + u * nthr (u < K), q = row * NL + line over all NL
// lines of the level (lines of the other colour idle).  The scaled values are held in registers
// between the read and the write of a step.  x = d / (1 + a + c), dst = src + omega x.
// dst may be sd (line Jacobi writes its scratch array); in the zebra form it is src.
template <typename T, int DIM, int KIND>
__device__ __forceinline__ void lines_pcr(const Lev<T> &L, int dir, int zebra, int colour, const T *src,
                                          const T *__restrict__ g, T *dst, T omega, T *sa, T *sc, T *sd, int tid,
                                          int nthr) {
  constexpr int kLinePcrK = line_pcr_k<T>();
  const bool cyc = dir == 1 && L.per;
  const int nx = L.n0 - 2;
  const int m = dir == 0 ? nx : L.yrows();
  const int NL = dir == 0 ? (int)L.unk_rows() : nx * L.zrows();
  const int stride = dir == 0 ? 1 : (int)L.pitch;
  int pn[kLinePcrK], rw[kLinePcrK];   // node and row of each held equation (pn < 0: none)
#pragma unroll
  for (int u = 0; u < kLinePcrK; ++u) {
    const int q = tid + u * nthr;
    pn[u] = -1;
    rw[u] = 0;
    if (q >= NL * m) continue;
    const int line = q % NL, row = q / NL;
    int i, j, k;
    if (dir == 0) {
      row_jk(L, line, j, k);
      i = 1 + row;
      if (zebra && ((j + k) & 1) != colour) continue;
    } else {
      i = 1 + line % nx;
      k = DIM == 3 ? 1 + line / nx : 0;
      j = L.ylo() + row;
      if (zebra && ((i + k) & 1) != colour) continue;
    }
    const int p = k * (int)L.plane + j * (int)L.pitch + i;
    int dm, dp;
    yoffs(L, j, dm, dp);
    Weights<T, DIM, KIND> w;
    w.load(L, i, p, dm);
    const T d = residual_at<T, DIM, KIND>(L, w, src, p, dm, dp, g[p]);
    T D = (w.wW + w.wE) + (w.wS + w.wN);
    if (DIM == 3) D += w.wB + w.wF;
    if (KIND == K_CONST) D = L.d;
    const T lo = dir == 0 ? w.wW : w.wS, hi = dir == 0 ? w.wE : w.wN;
    const T rD = T(1) / D;
    sa[p] = (cyc || row > 0) ? -lo * rD : T(0);
    sc[p] = (cyc || row < m - 1) ? -hi * rD : T(0);
    sd[p] = d * rD;
    pn[u] = p;
    rw[u] = row;
  }
  for (int s = 1; s < m; s <<= 1) {
    __syncthreads();
    T na[kLinePcrK], nc[kLinePcrK], nd[kLinePcrK];
#pragma unroll
    for (int u = 0; u < kLinePcrK; ++u) {
      if (pn[u] < 0) continue;
      const int p = pn[u];
      const T a = sa[p], c = sc[p], d = sd[p];
      T am = T(0), cm = T(0), dmv = T(0), ap = T(0), cp = T(0), dpv = T(0);
      // a row with no neighbour at distance s (Dirichlet) has a zero coupling there
      if (rw[u] >= s || cyc) {
        const int q = rw[u] >= s ? p - s * stride : p + (m - s) * stride;
        am = sa[q];
        cm = sc[q];
        dmv = sd[q];
      }
      if (rw[u] + s < m || cyc) {
        const int q = rw[u] + s < m ? p + s * stride : p - (m - s) * stride;
        ap = sa[q];
        cp = sc[q];
        dpv = sd[q];
      }
      const T rr = T(1) / (T(1) - a * cm - c * ap);
      na[u] = -rr * a * am;
      nc[u] = -rr * c * cp;
      nd[u] = rr * (d - a * dmv - c * dpv);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kLinePcrK; ++u) {
      if (pn[u] < 0) continue;
      sa[pn[u]] = na[u];
      sc[pn[u]] = nc[u];
      sd[pn[u]] = nd[u];
    }
  }
#pragma unroll
  for (int u = 0; u < kLinePcrK; ++u) {
    if (pn[u] < 0) continue;
    const int p = pn[u];
    const T x = sd[p] / (T(1) + sa[p] + sc[p]);
    dst[p] = fma(omega, x, src[p]);
  }
}

// FULL = false leaves out the line-smoother and adaptive-weight steps (programs of the point
// smoothers with a fixed weight never hold them): a smaller kernel spends less of each step
// fetching instructions.
// The kernel always runs as one block on one SM: the bound of one resident block lets the compiler
// give each thread the registers it needs (at its default choice the FP64 forms spilled to local
// memory).
template <typename T, int DIM, int KIND, bool FULL>
__global__ void __launch_bounds__(csk_threads<T>(), 1) k_coarse_cycle(const SLev<T> *__restrict__ levs, const int4 *__restrict__ prog,
                                                       int nops, int lc, const T *__restrict__ g_in,
                                                       const T *__restrict__ u_in, T *__restrict__ u_out,
                                                       const double *__restrict__ Ainv,
                                                       const long long *__restrict__ cidx_smem, int nc, T omega,
                                                       T omega_corr) {
  MG_PDL_WAIT();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *pool = reinterpret_cast<T *>(smem_raw);
  // stage the level table and the program in shared memory (each step reads them)
  __shared__ SLev<T> s_levs[17];
  __shared__ int4 s_prog[CSK_STAGED_OPS];
  __shared__ double s_red[2][32];   // warp totals of the adaptive-weight inner products
  {
    const int *src = reinterpret_cast<const int *>(levs);
    int *dst = reinterpret_cast<int *>(s_levs);
    int nwords = (int)((lc + 1) * sizeof(SLev<T>) / sizeof(int));
    for (int t = threadIdx.x; t < nwords; t += blockDim.x) dst[t] = src[t];
    int nst = nops < CSK_STAGED_OPS ? nops : CSK_STAGED_OPS;
    for (int t = threadIdx.x; t < nst; t += blockDim.x) s_prog[t] = prog[t];
    __syncthreads();
    if (KIND == K_CELL && threadIdx.x == 0) {   // cell data of every level lives in the pool
      for (int l = 1; l <= lc; ++l) {
        s_levs[l].L.k = pool + s_levs[l].off_k;
        s_levs[l].L.ndinv = pool + s_levs[l].off_dinv;
      }
    }
    if (KIND == K_EDGE && threadIdx.x == 0) {   // so do the edge weights
      for (int l = 1; l <= lc; ++l) {
        s_levs[l].L.ex = pool + s_levs[l].off_ex;
        s_levs[l].L.ey = pool + s_levs[l].off_ey;
        s_levs[l].L.ez = DIM == 3 ? pool + s_levs[l].off_ez : nullptr;
        s_levs[l].L.ndinv = pool + s_levs[l].off_dinv;
      }
    }
    __syncthreads();
    levs = s_levs;
  }
  // zero all level arrays, load cell data
  for (int l = 1; l <= lc; ++l) {
    const SLev<T> &S = levs[l];
    int cnt = (int)(S.L.plane * S.L.n2);
    T *u0 = pool + S.off_u0, *u1 = pool + S.off_u1, *g = pool + S.off_g, *r = pool + S.off_r;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      u0[t] = T(0);
      u1[t] = T(0);
      g[t] = T(0);
      r[t] = T(0);
    }
    if (KIND == K_CELL) {
      T *kk = pool + S.off_k, *dv = pool + S.off_dinv;
      for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        int i = t % S.L.n0, rr = t / S.L.n0, j = rr % S.L.n1, k = rr / S.L.n1;
        long long gp = (long long)k * S.gplane + (long long)j * S.gpitch + i;
        if (!MG_CKN(S.L, gp, S.gplane * S.L.n2)) continue;   // debug build
        kk[t] = S.gk[gp];
        dv[t] = S.gdinv[gp];
      }
    }
    if (KIND == K_EDGE) {
      T *wx = pool + S.off_ex, *wy = pool + S.off_ey, *dv = pool + S.off_dinv;
      for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
        int i = t % S.L.n0, rr = t / S.L.n0, j = rr % S.L.n1, k = rr / S.L.n1;
        long long gp = (long long)k * S.gplane + (long long)j * S.gpitch + i;
        if (!MG_CKN(S.L, gp, S.gplane * S.L.n2)) continue;   // debug build
        wx[t] = S.gex[gp];
        wy[t] = S.gey[gp];
        if (DIM == 3) pool[S.off_ez + t] = S.gez[gp];
        dv[t] = S.gdinv[gp];
      }
    }
  }
  __syncthreads();
  const int wid_ = (int)(threadIdx.x >> 5), nw_ = (int)(blockDim.x >> 5);
  const int tid_ = (int)threadIdx.x, nthr_ = (int)blockDim.x;
  for (int op = 0; op < nops; ++op) {
    int4 o = op < CSK_STAGED_OPS ? s_prog[op] : prog[op];
    const SLev<T> &S = levs[o.y];
    // a register copy of the level view: the steps store through pool pointers, which the
    // compiler cannot prove distinct from the level table, so fields read in place would be
    // reloaded after every store
    const Lev<T> L = S.L;
    T *const ub0 = pool + S.off_u0, *const ub1 = pool + S.off_u1;
    auto ub = [&](int b) -> T * { return b ? ub1 : ub0; };   // no runtime-indexed array (local memory)
    T *g = pool + S.off_g, *r = pool + S.off_r;
    // unknowns of this level from a global array: every thread issues a batch of loads before
    // its shared-memory stores (one load at a time is latency-bound)
    auto load_unk = [&](T *dst, const T *__restrict__ src) {
      const int nx = L.n0 - 2, ny = L.yrows(), tot = nx * ny * L.zrows();
      constexpr int B = 8;
      for (int t0 = tid_; t0 < tot; t0 += B * nthr_) {
        T v[B];
        int pp[B];
#pragma unroll
        for (int q = 0; q < B; ++q) {
          const int t = t0 + q * nthr_;
          pp[q] = -1;
          if (t < tot) {
            const int i = 1 + t % nx, rr = t / nx;
            const int j = L.ylo() + (DIM == 3 ? rr % ny : rr), k = DIM == 3 ? 1 + rr / ny : 0;
            pp[q] = k * (int)L.plane + j * (int)L.pitch + i;
            const long long gq = (long long)k * S.gplane + (long long)j * S.gpitch + i;
            if (!MG_CKN(L, gq, S.gplane * L.n2)) {   // debug build
              pp[q] = -1;
              continue;
            }
            v[q] = src[gq];
          }
        }
#pragma unroll
        for (int q = 0; q < B; ++q)
          if (pp[q] >= 0) dst[pp[q]] = v[q];
      }
    };
    int rb_desc = -1;            // red-black sweeps run after the switch (RB_HALF, or fused after PROLONG)
    T *rb_u = nullptr;
    const T *rs_src = nullptr;   // restriction run after the switch (RESTRICT, or fused after DEFECT)
    bool sync_first = false;     // a barrier before the deferred part (it reads what the step wrote)
    switch (o.x) {
      case CP_LOAD_G:
        load_unk(g, g_in);
        break;
      case CP_LOAD_U:
        load_unk(ub(o.z), u_in);
        break;
      case CP_STORE_U:
        FOR_UNK(L, {
          const long long gq = (long long)k * S.gplane + (long long)j * S.gpitch + i;
          if (MG_CKN(L, gq, S.gplane * L.n2)) u_out[gq] = ub(o.z)[p];
        });
        break;
      case CP_ZERO_U:
        FOR_UNK(L, { ub(o.z)[p] = T(0); });
        break;
      case CP_JACOBI: {   // z = src, w = dst; src < 0: zero iterate
        const T *src = o.z >= 0 ? ub(o.z) : nullptr;
        T *dst = ub(o.w);
        FOR_UNK(L, {
          int dm, dp;
          yoffs(L, j, dm, dp);
          Weights<T, DIM, KIND> w;
          w.load(L, i, p, dm);
          if (src) dst[p] = fma(omega * w.dinv, residual_at<T, DIM, KIND>(L, w, src, p, dm, dp, g[p]), src[p]);
          else dst[p] = omega * w.dinv * g[p];
        });
        break;
      }
      case CP_RB_HALF:   // z = sweep descriptor, w = buffer (the sweeps run after the switch)
        rb_desc = o.z;
        rb_u = ub(o.w);
        break;
      case CP_LINE: {   // z = dir | zebra << 1 | colour << 2, w = src | dst << 4 | scratch << 8
        if (!FULL) break;
        int dir = o.z & 1, zebra = (o.z >> 1) & 1, colour = (o.z >> 2) & 1;
        T *src = ub(o.w & 15), *dst = ub((o.w >> 4) & 15);
        T *cps = r, *dps = ub((o.w >> 8) & 15);
        int nlines = dir == 0 ? (int)L.unk_rows() : (L.n0 - 2) * L.zrows();
        {   // every line at once by cyclic reduction where the level fits (r, z and the scratch array).
          // In one SM its (lines x rows x log rows) work is issue-bound, a Thomas line a chain of rows:
          // it pays where the chain is long (FP64 divisions, or the cyclic solve's extra passes) and
          // few lines are active.  Measured on 65x65, 65x64 and 17x16x17 levels: FP32 Dirichlet
          // lines and many short lines are faster with Thomas.
          const int mrow = dir == 0 ? L.n0 - 2 : L.yrows();
          const bool cyc = dir == 1 && L.per, pow2 = (mrow & (mrow - 1)) == 0;
          const int active = zebra ? (nlines + 1) / 2 : nlines;
          if (S.off_z >= 0 && (sizeof(T) == 8 || cyc) && active <= mrow && nlines * mrow <= line_pcr_k<T>() * nthr_ &&
              (!cyc || pow2)) {
            lines_pcr<T, DIM, KIND>(L, dir, zebra, colour, src, g, dst, omega, cps, pool + S.off_z, dps, tid_, nthr_);
            break;
          }
        }
        for (int t = tid_; t < nlines; t += nthr_) {
          int m, a_fixed, kk;
          int base, stride;
          if (dir == 0) {
            int jj, k2;
            row_jk(L, t, jj, k2);
            if (zebra && ((jj + k2) & 1) != colour) continue;
            m = L.n0 - 2;
            base = k2 * (int)L.plane + jj * (int)L.pitch + 1;
            stride = 1;
            a_fixed = jj;
            kk = k2;
          } else {
            int nx = L.n0 - 2;
            int ii = 1 + t % nx, k2 = (DIM == 3 ? 1 : 0) + t / nx;
            if (zebra && ((ii + k2) & 1) != colour) continue;
            if (L.per) {   // every row an unknown: the cyclic system (third scratch array z)
              cyclic_yline<T, DIM, KIND>(L, (long long)k2 * L.plane + ii, ii, src, g, dst, omega, cps, dps,
                                         pool + S.off_z);
              continue;
            }
            m = L.n1 - 2;
            base = k2 * (int)L.plane + (int)L.pitch + ii;
            stride = (int)L.pitch;
            a_fixed = ii;
            kk = k2;
          }
          (void)kk;
          T cprev = T(0), dprev = T(0);
          for (int s = 0; s < m; ++s) {
            int p = base + s * stride;
            int i = dir == 0 ? 1 + s : a_fixed;
            int j = dir == 0 ? a_fixed : 1 + s;
            int dm, dp;
            yoffs(L, j, dm, dp);
            Weights<T, DIM, KIND> w;
            w.load(L, i, p, dm);
            T res = residual_at<T, DIM, KIND>(L, w, src, p, dm, dp, g[p]);
            T D = (w.wW + w.wE) + (w.wS + w.wN);
            if (DIM == 3) D += w.wB + w.wF;
            if (KIND == K_CONST) D = L.d;
            T lo = (s > 0) ? -(dir == 0 ? w.wW : w.wS) : T(0);
            T up = (s < m - 1) ? -(dir == 0 ? w.wE : w.wN) : T(0);
            T den = D - lo * cprev;
            T cp = up / den;
            T dpv = (res - lo * dprev) / den;
            cps[p] = cp;
            dps[p] = dpv;
            cprev = cp;
            dprev = dpv;
          }
          T x = T(0);
          for (int s = m - 1; s >= 0; --s) {
            int p = base + s * stride;
            x = dps[p] - cps[p] * x;
            dst[p] = fma(omega, x, src[p]);
          }
        }
        break;
      }
      case CP_DEFECT: {   // z = buffer; w = 1: the restriction of r follows in the same step
        const T *u = ub(o.z);
        FOR_UNK(L, {
          int dm, dp;
          yoffs(L, j, dm, dp);
          Weights<T, DIM, KIND> w;
          w.load(L, i, p, dm);
          r[p] = residual_at<T, DIM, KIND>(L, w, u, p, dm, dp, g[p]);
        });
        if (o.w) {
          rs_src = r;
          sync_first = true;
        }
        break;
      }
      case CP_RESTRICT:   // level y -> y-1: r of level y, or g when z = 1 (runs after the switch)
        rs_src = o.z ? g : r;
        break;
      case CP_PROLONG:     // level y (fine), z = fine buffer, w = coarse buffer | (sweeps + 1) << 1
      case CP_INTERP: {
        const SLev<T> &Cs = levs[o.y - 1];
        Lev<T> C = Cs.L;
        const T *ec = ((o.w & 1) ? pool + Cs.off_u1 : pool + Cs.off_u0);
        T *uf = ub(o.z);
        const bool interp = o.x == CP_INTERP;
        FOR_UNK(L, {
          T s = interp_at<T, DIM>(C, ec, i, j, k);
          uf[p] = interp ? s : fma(omega_corr, s, uf[p]);
        });
        if (o.w >> 1) {   // the post-smoothing red-black sweeps follow in the same step
          rb_desc = (o.w >> 1) - 1;
          rb_u = uf;
          sync_first = true;
        }
        break;
      }
      case CP_ADAPT: {   // z = fine buffer, w = coarse buffer: u_y[z] += omega P e with its own weight
        if (!FULL) break;
        const SLev<T> &Cs = levs[o.y - 1];
        Lev<T> C = Cs.L;
        const T *ec = o.w ? pool + Cs.off_u1 : pool + Cs.off_u0;
        T *u = ub(o.z);
        FOR_UNK(L, { r[p] = interp_at<T, DIM>(C, ec, i, j, k); });   // P e (r is zero off the unknowns)
        __syncthreads();
        T a0 = T(0), a1 = T(0);   // per-thread sums in the level's precision
        FOR_UNK(L, {
          int dm, dp;
          yoffs(L, j, dm, dp);
          Weights<T, DIM, KIND> w;
          w.load(L, i, p, dm);
          T d = residual_at<T, DIM, KIND>(L, w, u, p, dm, dp, g[p]);
          T ape = -residual_at<T, DIM, KIND>(L, w, r, p, dm, dp, T(0));
          a0 = fma(d, r[p], a0);
          a1 = fma(ape, r[p], a1);
        });
        for (int o2 = 16; o2 > 0; o2 >>= 1) {
          a0 += __shfl_down_sync(0xffffffffu, a0, o2);
          a1 += __shfl_down_sync(0xffffffffu, a1, o2);
        }
        if ((threadIdx.x & 31) == 0) {
          s_red[0][wid_] = (double)a0;
          s_red[1][wid_] = (double)a1;
        }
        __syncthreads();
        double num = 0.0, den = 0.0;   // every thread sums the warp totals in the same order
        for (int q = 0; q < nw_; ++q) {
          num += s_red[0][q];
          den += s_red[1][q];
        }
        const T wgt = (T)(den > 0.0 ? num / den : 1.0);
        FOR_UNK(L, { u[p] = fma(wgt, r[p], u[p]); });
        break;
      }
      case CP_COARSE: {   // level 1: u[z] = A^{-1} g, one warp per row of the dense inverse
        T *u = ub(o.z);
        const int lane = threadIdx.x & 31;
        for (int row = wid_; row < nc; row += nw_) {
          const double *arow = Ainv + (long long)row * nc;
          double s = 0.0;
          for (int c = lane; c < nc; c += 32) s = fma(arow[c], (double)g[cidx_smem[c]], s);
          for (int o2 = 16; o2 > 0; o2 >>= 1) s += __shfl_down_sync(0xffffffffu, s, o2);
          if (lane == 0) u[cidx_smem[row]] = (T)s;
        }
        break;
      }
    }
    if (rs_src) {   // full weighting of rs_src into g of level y-1
      if (sync_first) __syncthreads();
      const SLev<T> &Cs = levs[o.y - 1];
      Lev<T> C = Cs.L;
      T *gc = pool + Cs.off_g;
      const T *rs = rs_src;
      FOR_UNK(C, {
        int I = i, J = j, K = k;
        int dm, dp;
        yoffs(L, 2 * J, dm, dp);
        int pf = (2 * K) * (int)L.plane + (2 * J) * (int)L.pitch + 2 * I;
        auto row3 = [&](int c) -> T { return (rs[c - 1] + rs[c + 1]) + T(2) * rs[c]; };
        auto plane3 = [&](int c) -> T { return (row3(c + dm) + row3(c + dp)) + T(2) * row3(c); };
        T s;
        if (DIM == 2) s = plane3(pf) * T(0.0625);
        else s = ((plane3(pf - (int)L.plane) + plane3(pf + (int)L.plane)) + T(2) * plane3(pf)) * T(0.015625);
        gc[p] = s;
      });
    }
    if (rb_desc >= 0) {   // red-black half sweeps on rb_u, in place, one barrier between them
      if (sync_first) __syncthreads();
      T *u = rb_u;
      const int nh = 1 + (rb_desc >> 2);
      for (int h = 0; h < nh; ++h) {
        const int colour = (rb_desc + h) & 1;
        if (h == 0 && (rb_desc & 2)) {   // from a zero iterate: sets every unknown (its residual is g)
          FOR_UNK(L, {
            T v = T(0);
            if (((i + j + k) & 1) == colour) {
              int dm, dp;
              yoffs(L, j, dm, dp);
              Weights<T, DIM, KIND> w;
              w.load(L, i, p, dm);
              v = fma(omega * w.dinv, g[p], T(0));
            }
            u[p] = v;
          });
        } else {
          FOR_COLOUR(L, colour, {
            int dm, dp;
            yoffs(L, j, dm, dp);
            Weights<T, DIM, KIND> w;
            w.load(L, i, p, dm);
            u[p] = fma(omega * w.dinv, residual_at<T, DIM, KIND>(L, w, u, p, dm, dp, g[p]), u[p]);
          });
        }
        if (h + 1 < nh) __syncthreads();
      }
    }
    __syncthreads();
  }
}

template <typename T>
void launch_coarse_cycle(const Launch &lc, int dim, int kind, const void *levs, const int4 *prog, int nops, int lcut,
                         const T *g_in, const T *u_in, T *u_out, const double *Ainv, const long long *cidx_smem,
                         int nc, T omega, T omega_corr, size_t smem_bytes, bool full) {
#define CC_LAUNCH(D, K)                                                                                      \
  do {                                                                                                       \
    auto fn = full ? k_coarse_cycle<T, D, K, true> : k_coarse_cycle<T, D, K, false>;                        \
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);                  \
    fn<<<1, csk_threads<T>(), smem_bytes, lc.s>>>((const SLev<T> *)levs, prog, nops, lcut, g_in, u_in, u_out, Ainv,       \
                                      cidx_smem, nc, omega, omega_corr);                                     \
  } while (0)
  if (dim == 2) {
    if (kind == K_CONST) CC_LAUNCH(2, K_CONST);
    else if (kind == K_SEP) CC_LAUNCH(2, K_SEP);
    else if (kind == K_CELL) CC_LAUNCH(2, K_CELL);
    else CC_LAUNCH(2, K_EDGE);
  } else {
    if (kind == K_CONST) CC_LAUNCH(3, K_CONST);
    else if (kind == K_SEP) CC_LAUNCH(3, K_SEP);
    else if (kind == K_CELL) CC_LAUNCH(3, K_CELL);
    else CC_LAUNCH(3, K_EDGE);
  }
#undef CC_LAUNCH
  lc.done(__func__);
}

template <typename T>
size_t coarse_slev_size() {
  return sizeof(SLev<T>);
}

// Fill the level descriptors (host): smem offsets in elements of T, returns the pool size in bytes.
template <typename T>
size_t coarse_fill_levels(void *out, int lcut, const Lev<T> *glev, const long long *gpitch, const long long *gplane,
                          int kind, bool zscratch) {
  static_assert(sizeof(SLev<T>) <= 512, "level table slot");
  SLev<T> *S = (SLev<T> *)out;
  int off = 0;
  auto take = [&](long long cnt) {
    int o = off;
    off += (int)((cnt + 3) / 4 * 4);
    return o;
  };
  for (int l = 1; l <= lcut; ++l) {
    SLev<T> &s = S[l];
    s.L = glev[l];
    s.L.pitch = s.L.n0;
    s.L.plane = (long long)s.L.n0 * s.L.n1;
    long long cnt = s.L.plane * s.L.n2;
    s.gpitch = gpitch[l];
    s.gplane = gplane[l];
    s.gk = glev[l].k;
    s.gdinv = glev[l].ndinv;
    s.gex = glev[l].ex;
    s.gey = glev[l].ey;
    s.gez = glev[l].ez;
    s.off_u0 = take(cnt);
    s.off_u1 = take(cnt);
    s.off_g = take(cnt);
    s.off_r = take(cnt);
    s.off_k = s.off_dinv = s.off_ex = s.off_ey = s.off_ez = -1;
    s.off_z = zscratch ? take(cnt) : -1;
    if (kind == K_CELL) {
      s.off_k = take(cnt);
      s.off_dinv = take(cnt);
    } else if (kind == K_EDGE) {
      s.off_ex = take(cnt);
      s.off_ey = take(cnt);
      if (s.L.dim == 3) s.off_ez = take(cnt);
      s.off_dinv = take(cnt);
    }
    s.L.k = nullptr;
    s.L.ndinv = nullptr;
    s.L.ex = s.L.ey = s.L.ez = nullptr;
  }
  return (size_t)off * sizeof(T);
}

template void launch_coarse_cycle<double>(const Launch &, int, int, const void *, const int4 *, int, int, const double *,
                                          const double *, double *, const double *, const long long *, int, double,
                                          double, size_t, bool);
template void launch_coarse_cycle<float>(const Launch &, int, int, const void *, const int4 *, int, int, const float *,
                                         const float *, float *, const double *, const long long *, int, float, float,
                                         size_t, bool);
template size_t coarse_slev_size<double>();
template size_t coarse_slev_size<float>();
template size_t coarse_fill_levels<double>(void *, int, const Lev<double> *, const long long *, const long long *, int,
                                           bool);
template size_t coarse_fill_levels<float>(void *, int, const Lev<float> *, const long long *, const long long *, int,
                                          bool);

}  // namespace mg
