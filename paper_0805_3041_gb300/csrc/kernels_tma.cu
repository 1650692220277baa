// kernels_tma.cu -- one red-black Gauss-Seidel sweep (2-D, FP32, constant or separable
// coefficients; Wallis 2008, section "The choice of C": C = D + L in red-black order)
// with the rows of u and g streamed through shared memory by TMA bulk copies.
//
// A CTA owns a band of RC rows of a 512-column group and marches down it.  Four compute
// warps each own a strip of 128 columns (4 per lane); a fifth, producer warp keeps a ring
// of RING row slots filled ahead of them with cp.async.bulk copies of the group's row
// segments -- u and g over columns [s0 - 4, s0 + 516) and, for the sweep that folds in the
// coarse-grid correction u + omega_l P e, the coarse rows of e it interpolates from.  Each
// slot has a "full" mbarrier (the copies' bytes) and an "empty" one (one arrival per
// compute warp done with the row); the producer refills a slot as soon as it is empty, so
// the copies queued ahead cover HBM latency without the compute warps ever waiting on one
// another, and one 2 KB copy per array and row keeps HBM reads close to a contiguous
// stream.  Each row goes from its slot into registers once.  For output row j a warp
// holds the old rows j, j+1, j+2 and the half-relaxed rows H_{j-1}, H_j, H_{j+1} (first
// colour relaxed, second colour old): H_{j+1} is formed when row j+2 arrives, then the
// second colour of row j is relaxed from the H rows and the row is stored.  The window
// rotates by renaming over a three-step unrolled loop.  x-neighbours come from warp
// shuffles; the strip-edge lanes relax the outside first-colour node themselves from the
// columns beside the strip.  Each node is read once and written once: 12 B per unknown.
//
// Every wait on an mbarrier is bounded (by the SM cycle counter).  A compute warp whose
// wait gives up sets *err and stops; the producer then gives up waiting for its slots,
// waits (bounded again) for the copies still in flight and stops too; the solver reports
// MG_ETIMEOUT.
#include <stdint.h>

#include <algorithm>

#define MG_FILE_ID 8   // bounds-check sites (-DMG_DEBUG)
#include "mg_internal.cuh"

namespace mg {

namespace {
constexpr int NW = 4;                  // warps per CTA = strips per column group
constexpr int RING = 8;                // row slots (power of two)
constexpr int RING_LOG = 3;
constexpr int SEGW = 128 * NW + 8;     // floats per fine row segment: 4 + 512 + 4
constexpr int CSEGW = 64 * NW + 8;     // floats per coarse row segment: 4 + 256 + 4
// A ring slot of the sweep holds the row's g segment, after its u segment unless the iterate
// starts at zero (mode 1, u is not read), then in mode 2 one coarse row of e: slot j holds
// coarse row (j + 1) >> 1, so that fine row j interpolates from its own slot's coarse row and,
// for odd j, the previous slot's -- each coarse row is copied twice, not three times.  The
// first streamed row's previous coarse row has a segment of its own after the ring.
__host__ __device__ constexpr int slot_floats(int mode) {
  return (mode == 1 ? SEGW : 2 * SEGW) + (mode == 2 ? CSEGW : 0);
}
__host__ __device__ constexpr int pre_floats(int mode) { return mode == 2 ? CSEGW : 0; }
__host__ __device__ constexpr int g_offset(int mode) { return mode == 1 ? 0 : SEGW; }
// waits are bounded by the SM's cycle counter (a register read; 2^30 cycles is about 0.5 s)
constexpr long long WAIT_CYCLES = 1ll << 30;    // give up a wait after this many cycles
constexpr long long DRAIN_CYCLES = 1ll << 28;   // and drain each copy for at most this many

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// true once the phase of the given parity has completed; false after limit cycles
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (clock64() - t0 > limit) return false;
  }
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

struct Coef {
  float W[4], E[4], Y[4], D[4], O[4];
  bool act[4];
};
struct URow {      // one old row in registers
  float u[4];
  float out, out2;  // edge lanes: u of the outside column and of the one beyond it
};
struct HRow {      // one half-relaxed row
  float h[4];
  float ho;         // edge lanes: value of the outside column
};

// Relax the nodes of one colour in the thread's four columns: in each pair (2k, 2k+1)
// exactly one node has that colour, the one with index parity P.  o = c elsewhere.
template <int P>
__device__ __forceinline__ void relax_colour(float (&o)[4], const float (&c)[4], float left, float right,
                                             const float (&n)[4], const float (&s)[4], const float (&gg)[4],
                                             const Coef &K, bool rowok) {
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int a = 2 * k, b = a + 1, x = P ? b : a;
    const float wv = P ? c[a] : (a > 0 ? c[a - 1] : left);
    const float ev = P ? (b + 1 < 4 ? c[b + 1] : right) : c[b];
    float r = fmaf(-K.D[x], c[x], gg[x]);
    r = fmaf(K.W[x], wv, r);
    r = fmaf(K.E[x], ev, r);
    r = fmaf(K.Y[x], n[x], r);
    r = fmaf(K.Y[x], s[x], r);
    const float nv = fmaf(K.O[x], r, c[x]);
    o[a] = c[a];
    o[b] = c[b];
    if (rowok && K.act[x]) o[x] = nv;
  }
}
}  // namespace

// The sweep over one band of rows [j0, j1) of one column group.  IN: every streamed row
// j0-2 .. j1+1 is an unknown row of the grid (no wrap, no boundary rows), so the row tests
// fold away.  The level descriptors come by value: a reference to a kernel parameter would
// turn each field read in the row loop into a load through the L1 path.
template <int KIND, int MODE, bool IN>
__device__ __forceinline__ void band_sweep(const Lev<float> L, const float *__restrict__ u,
                                           const float *__restrict__ g, float *__restrict__ out, float omega,
                                           int first, const Lev<float> C, const float *__restrict__ ec,
                                           float omega_corr, int j0, int j1, int s0, float *ring, float *pre,
                                           uint64_t *full, uint64_t *empty, int *err, int *inject) {
  constexpr int SLOT = slot_floats(MODE);   // floats per ring slot
  constexpr int GOFF = g_offset(MODE), EOFF = 2 * SEGW;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sw = s0 + 128 * warp;             // first column of the warp's strip
  const int i0 = sw + 4 * lane;               // first column of the thread
  const int c0 = 4 + 128 * warp + 4 * lane;   // its position in a row segment
  const bool edge = lane == 0 || lane == 31;
  const int io = lane == 0 ? sw - 1 : sw + 128;    // outside column of an edge lane
  const int io2 = lane == 0 ? sw - 2 : sw + 129;   // and the one beyond it
  const int co = lane == 0 ? c0 - 1 : c0 + 4, co2 = lane == 0 ? c0 - 2 : c0 + 5;

  // ---- coefficients of the thread's columns and of the outside column ----
  Coef K;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int i = i0 + e;
    K.act[e] = i >= 1 && i <= L.n0 - 2;
    if (KIND == K_CONST) {
      K.W[e] = L.cx; K.E[e] = L.cx; K.Y[e] = L.cy; K.D[e] = L.d; K.O[e] = omega * L.dinv;
    } else {
      const int ic = K.act[e] ? i : 1;
      K.W[e] = L.sx[ic - 1]; K.E[e] = L.sx[ic]; K.Y[e] = L.sy[ic];
      K.D[e] = (K.W[e] + K.E[e]) + (K.Y[e] + K.Y[e]);
      K.O[e] = omega * L.sdinv[ic];
    }
  }
  const bool oact = edge && io >= 1 && io <= L.n0 - 2;
  float oW = L.cx, oE = L.cx, oY = L.cy, oD = L.d, oO = omega * L.dinv;
  if (KIND == K_SEP && edge) {
    const int ic = oact ? io : 1;
    oW = L.sx[ic - 1]; oE = L.sx[ic]; oY = L.sy[ic];
    oD = (oW + oE) + (oY + oY);
    oO = omega * L.sdinv[ic];
  }

  // ---- the part of the group's row segment that exists in memory, and where it lands ----
  const int cs = max(0, s0 - 4), ce = min((int)L.pitch, s0 + 128 * NW + 4);
  const int doff = cs - (s0 - 4);
  const uint32_t seg_bytes = (uint32_t)(ce - cs) * 4u;
  const int cbase = (s0 >> 1) - 4;   // coarse column at coarse-segment position 0
  const int ccs = max(0, cbase), cce = min((int)C.pitch, cbase + CSEGW);
  const int cdoff = ccs - cbase;
  const uint32_t cseg_bytes = MODE == 2 ? (uint32_t)(cce - ccs) * 4u : 0u;

  auto valid = [&](int j) { return IN || L.per || (j >= 0 && j < L.n1); };
  auto unk = [&](int j) { return IN || L.per || (j >= 1 && j <= L.n1 - 2); };
  auto wrap = [&](int j) -> int {
    if (IN || !L.per) return j;
    j = j < 0 ? j + L.n1 : (j >= L.n1 ? j - L.n1 : j);
    if (j < 0 || j >= L.n1) j = ((j % L.n1) + L.n1) % L.n1;
    return j;
  };

  const int jfirst = j0 - 2, jlast = j1 + 1;   // rows the CTA streams
  auto slot_of = [&](int j) -> const float * { return ring + ((j - jfirst) & (RING - 1)) * SLOT; };
  // full[s]: one arrival (the issuing thread) plus the bytes of the row's copies per phase;
  // rows outside the grid (at most one at each end of the stream) are never copied, so
  // the phase of row j's slot counts the copied rows before it in that slot.
  const int jv0 = valid(jfirst) ? jfirst : (valid(jfirst + 1) ? jfirst + 1 : jfirst + 2);
  auto full_parity = [&](int j) -> uint32_t { return (uint32_t)(((j - jv0) >> RING_LOG) & 1); };
  // empty[s]: one arrival per active warp when it is done with a row, for every streamed row
  auto empty_parity = [&](int j) -> uint32_t { return (uint32_t)(((j - jfirst) >> RING_LOG) & 1); };

  // ---- issuing thread: copies of row j into its slot ----
  auto issue = [&](int j) {
    if (!valid(j)) return;
    const int k = j - jfirst;
    float *slot = ring + (k & (RING - 1)) * SLOT;
    uint64_t *bar = &full[k & (RING - 1)];
    const int jw = wrap(j);
    // mode 2: every streamed row carries coarse row (jw + 1) >> 1; the first also jw >> 1
    int Jc = (jw + 1) >> 1;
    if (Jc >= C.n1) Jc -= C.n1;
    const bool pre_row = MODE == 2 && j == jfirst;
    // debug build: the copies' rows and spans lie inside u, g and ec; else nothing is issued and
    // the compute warps' bounded waits run out
    if (!MG_CKN(L, jw, L.n1) || !MG_CKN(L, ce - 1, L.pitch) ||
        (MODE == 2 && (!MG_CKN(C, Jc, C.n1) || !MG_CKN(C, jw >> 1, C.n1) || !MG_CKN(C, cce - 1, C.pitch))))
      return;
    const uint32_t bytes = (MODE == 1 ? 1u : 2u) * seg_bytes + (MODE == 2 ? (pre_row ? 2u : 1u) * cseg_bytes : 0u);
    mbar_expect_tx(bar, bytes);
    const long long ro = (long long)jw * L.pitch;
    if (MODE != 1) tma_load_1d(slot + doff, u + ro + cs, seg_bytes, bar);
    tma_load_1d(slot + GOFF + doff, g + ro + cs, seg_bytes, bar);
    if (MODE == 2) {
      tma_load_1d(slot + EOFF + cdoff, ec + (long long)Jc * C.pitch + ccs, cseg_bytes, bar);
      if (pre_row) tma_load_1d(pre + cdoff, ec + (long long)(jw >> 1) * C.pitch + ccs, cseg_bytes, bar);
    }
  };
  // ---- producer warp (lane 0): every streamed row in order, each into its slot once all
  // compute warps have released the row eight before it; then it waits until they have
  // released the last rows, so that no copy is in flight when the CTA ends ----
  if (warp == NW) {
    if (lane != 0) return;
    // test hook (MG_FLAG_TEST_WAIT_TIMEOUT): once per solve, one producer leaves its first valid
    // row uncopied, so that the compute warps' bounded waits run out and the timeout path is taken
    bool skip_pending = inject && blockIdx.x == 0 && atomicExch(inject, 0) != 0;
    int r = jfirst;   // rows jfirst .. r-1 have been issued
    bool ok = true;
    for (; r <= jlast; ++r) {
      if (r - RING >= jfirst &&
          !mbar_wait(&empty[(r - jfirst) & (RING - 1)], empty_parity(r - RING), WAIT_CYCLES)) {
        ok = false;
        break;
      }
      if (skip_pending && valid(r)) skip_pending = false;   // this row's copy never comes
      else issue(r);
    }
    for (int q = max(jfirst, jlast - RING + 1); q <= jlast && ok; ++q)
      ok = mbar_wait(&empty[(q - jfirst) & (RING - 1)], empty_parity(q), WAIT_CYCLES);
    if (!ok) {
      atomicExch(err, 1);
      // each slot holds at most one copy that no compute warp has released: those of the
      // last RING rows issued
      for (int q = max(jfirst, r - RING); q < r; ++q)
        if (valid(q)) mbar_wait(&full[(q - jfirst) & (RING - 1)], full_parity(q), DRAIN_CYCLES);
    }
    return;
  }

  // every lane waits for row j (bounded); the warp agrees on the outcome
  auto arrive_row = [&](int j) -> bool {
    bool ok = true;
    if (valid(j)) ok = mbar_wait(&full[(j - jfirst) & (RING - 1)], full_parity(j), WAIT_CYCLES);
    return __all_sync(FULL, ok);
  };
  // the warp is done with row j: release its slot
  auto release = [&](int j) {
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[(j - jfirst) & (RING - 1)]);
  };

  // read row j from its slot into registers (with omega_l P e added in MODE 2)
  auto load_row = [&](URow &R, int j) {
#pragma unroll
    for (int e = 0; e < 4; ++e) R.u[e] = 0.f;
    R.out = 0.f;
    R.out2 = 0.f;
    if (!valid(j)) return;
    const float *slot = slot_of(j);
    if (MODE != 1) {
      const float4 v = *reinterpret_cast<const float4 *>(slot + c0);
      R.u[0] = v.x; R.u[1] = v.y; R.u[2] = v.z; R.u[3] = v.w;
      if (edge) {
        R.out = slot[co];
        R.out2 = slot[co2];
      }
    }
    if (MODE == 2 && unk(j)) {
      // omega_l P e at the thread's columns: i >> 1 and (i + 1) >> 1 sit at coarse-segment
      // positions 4 + 64 warp + 2 lane + {0, 1, 2}
      const int jw = wrap(j);
      // coarse rows jw >> 1 (e0) and (jw + 1) >> 1 (e1): this slot's, and for odd jw the previous
      // row's slot (the segment after the ring for the first streamed row)
      const float *e1 = slot + EOFF;
      const float *e0 = (jw & 1) ? (j == jfirst ? pre : slot_of(j - 1) + EOFF) : e1;
      const int q = 4 + 64 * warp + 2 * lane;
      const float2 a0 = *reinterpret_cast<const float2 *>(e0 + q), a1 = *reinterpret_cast<const float2 *>(e1 + q);
      const float sq[3] = {a0.x + a1.x, a0.y + a1.y, e0[q + 2] + e1[q + 2]};
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (K.act[e]) R.u[e] += omega_corr * ((sq[e >> 1] + sq[(e + 1) >> 1]) * 0.25f);
      if (edge) {
        // the outside columns, in the same form the neighbouring strip gives its own columns: lane 0's
        // sw - 1 and sw - 2 take coarse positions q - 1 and q, lane 31's sw + 128 and sw + 129 take
        // q + 2 and q + 3 (s = e0 + e1 at each)
        const int qx = lane == 0 ? q - 1 : q + 3;
        const float sx = e0[qx] + e1[qx];
        const float c_out = lane == 0 ? sx + sq[0] : sq[2] + sq[2];
        const float c_out2 = lane == 0 ? sx + sx : sq[2] + sx;
        if (oact) R.out += omega_corr * (c_out * 0.25f);
        if (io2 >= 1 && io2 <= L.n0 - 2) R.out2 += omega_corr * (c_out2 * 0.25f);
      }
    }
  };

  // first colour of row j relaxed from the old rows j-1, j, j+1 (row j lies in the grid)
  auto half_row = [&](HRow &H, const URow &Rm, const URow &R, const URow &Rp, int j) {
    const float *slot = slot_of(j);
    const float4 g4 = *reinterpret_cast<const float4 *>(slot + GOFF + c0);
    const float gg[4] = {g4.x, g4.y, g4.z, g4.w};
    if (MODE == 1) {
      // zero iterate: the residual of a first-colour node is g, its new value omega/D g
      // (the same rounding as the general chain with zero operands); the rest stays 0
      const bool rowu = unk(j);
      const int p = (first + j) & 1;
#pragma unroll
      for (int e = 0; e < 4; ++e) H.h[e] = (rowu && K.act[e] && (e & 1) == p) ? fmaf(K.O[e], gg[e], 0.f) : 0.f;
      H.ho = (oact && rowu && (((io + j) & 1) == first)) ? fmaf(oO, slot[GOFF + co], 0.f) : 0.f;
      return;
    }
    float left = __shfl_up_sync(FULL, R.u[3], 1), right = __shfl_down_sync(FULL, R.u[0], 1);
    if (lane == 0) left = R.out;
    if (lane == 31) right = R.out;
    const bool rowu = unk(j);
    if ((first + j) & 1) relax_colour<1>(H.h, R.u, left, right, Rm.u, Rp.u, gg, K, rowu);
    else relax_colour<0>(H.h, R.u, left, right, Rm.u, Rp.u, gg, K, rowu);
    H.ho = R.out;
    if (oact && rowu && (((io + j) & 1) == first)) {
      const float gout = slot[GOFF + co];
      const float w_ = lane == 0 ? R.out2 : R.u[3], e_ = lane == 0 ? R.u[0] : R.out2;
      float s = fmaf(-oD, R.out, gout);
      s = fmaf(oW, w_, s);
      s = fmaf(oE, e_, s);
      s = fmaf(oY, Rm.out, s);
      s = fmaf(oY, Rp.out, s);
      H.ho = fmaf(oO, s, R.out);
    }
  };
  // second colour of row j from the half-relaxed rows j-1, j, j+1; store the row
  auto out_row = [&](const HRow &Hm, const HRow &Hc, const HRow &Hp, int j) {
    const float4 g4 = *reinterpret_cast<const float4 *>(slot_of(j) + GOFF + c0);
    const float gg[4] = {g4.x, g4.y, g4.z, g4.w};
    float hl = __shfl_up_sync(FULL, Hc.h[3], 1), hr = __shfl_down_sync(FULL, Hc.h[0], 1);
    if (lane == 0) hl = Hc.ho;
    if (lane == 31) hr = Hc.ho;
    float o[4];
    if ((first + j) & 1) relax_colour<0>(o, Hc.h, hl, hr, Hm.h, Hp.h, gg, K, true);
    else relax_colour<1>(o, Hc.h, hl, hr, Hm.h, Hp.h, gg, K, true);
    if (MG_CK(L, (long long)j * L.pitch + i0 + 3))
      *reinterpret_cast<float4 *>(out + (long long)j * L.pitch + i0) = make_float4(o[0], o[1], o[2], o[3]);
  };

  bool ok = true;
  // output row j: U0 = u(j), U1 = u(j+1) held, U2 <- u(j+2); H0 = H_{j-1}, H1 = H_j, H2 <- H_{j+1}
  auto step = [&](URow &U0, URow &U1, URow &U2, HRow &H0, HRow &H1, HRow &H2, int j) -> bool {
    if (!arrive_row(j + 2)) return false;
    load_row(U2, j + 2);
    half_row(H2, U0, U1, U2, j + 1);
    out_row(H0, H1, H2, j);
    release(j);
    return true;
  };

  URow A, B, Cr;
  HRow X, Y, Z;
  ok = arrive_row(j0 - 2) && arrive_row(j0 - 1) && arrive_row(j0) && arrive_row(j0 + 1);
  if (ok) {
    load_row(Cr, j0 - 2);
    load_row(A, j0 - 1);
    load_row(B, j0);
    half_row(X, Cr, A, B, j0 - 1);
    load_row(Cr, j0 + 1);
    half_row(Y, A, B, Cr, j0);
    release(j0 - 2);
    release(j0 - 1);
    // here A = u(j0-1), B = u(j0), Cr = u(j0+1), X = H_{j0-1}, Y = H_{j0}
    for (int j = j0; j < j1; j += 3) {
      if (!(ok = step(B, Cr, A, X, Y, Z, j))) break;
      if (j + 1 >= j1) break;
      if (!(ok = step(Cr, A, B, Y, Z, X, j + 1))) break;
      if (j + 2 >= j1) break;
      if (!(ok = step(A, B, Cr, Z, X, Y, j + 2))) break;
    }
  }
  if (ok) {
    release(j1);       // the last two streamed rows, so that the producer sees every row released
    release(j1 + 1);
  } else if (lane == 0) {
    atomicExch(err, 1);
  }
}

template <int KIND, int MODE>
__global__ void __launch_bounds__(32 * (NW + 1)) k_rb2d_tma(Lev<float> L, const float *__restrict__ u,
                                                      const float *__restrict__ g, float *__restrict__ out,
                                                      float omega, int first, Lev<float> C,
                                                      const float *__restrict__ ec, float omega_corr, int RC,
                                                      int ngroups, int *err, int *inject) {
  MG_PDL_WAIT();
  constexpr int SLOT = slot_floats(MODE), PRE = pre_floats(MODE);
  extern __shared__ __align__(128) unsigned char tma_smem[];
  float *ring = reinterpret_cast<float *>(tma_smem);
  float *pre = ring + RING * SLOT;
  uint64_t *full = reinterpret_cast<uint64_t *>(pre + PRE);
  uint64_t *empty = full + RING;

  const int grp = blockIdx.x % ngroups, band = blockIdx.x / ngroups;
  const int ylo = L.per ? 0 : 1, yhi = L.per ? L.n1 - 1 : L.n1 - 2;   // unknown rows
  const int j0 = ylo + band * RC;
  if (j0 > yhi) return;   // the whole CTA
  const int j1 = min(j0 + RC, yhi + 1);
  const int s0 = grp * 128 * NW;   // first column of the group
  // the last group of a row may have idle warps (strips beyond the pitch)
  const int nact = min(NW, (int)(L.pitch - s0) / 128);

  // Segment positions that no copy writes (outside the array: the grid's left and right
  // margins) stay zero.
  for (int t = threadIdx.x; t < RING * SLOT + PRE; t += 32 * (NW + 1)) ring[t] = 0.f;
  if (threadIdx.x == 0) {
    for (int s = 0; s < RING; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], nact);
    }
    fence_mbar_init();
  }
  fence_proxy_async();
  __syncthreads();
  const int warp = threadIdx.x >> 5;   // warps 0 .. NW-1 compute, warp NW issues the copies
  if (warp < NW && warp >= nact) return;

  const bool interior = L.per ? (j0 - 2 >= 0 && j1 + 1 <= L.n1 - 1) : (j0 - 2 >= 1 && j1 + 1 <= L.n1 - 2);
  if (interior)
    band_sweep<KIND, MODE, true>(L, u, g, out, omega, first, C, ec, omega_corr, j0, j1, s0, ring, pre, full, empty,
                                 err, inject);
  else
    band_sweep<KIND, MODE, false>(L, u, g, out, omega, first, C, ec, omega_corr, j0, j1, s0, ring, pre, full, empty,
                                  err, inject);
}

// ---------------------------------------------------------------------------------------
// The defect d = g - A u of a fine level and its full-weighting restriction g_c = R d
// (Wallis 2008, section "The Multigrid Technique"), streamed the same way: a CTA owns a band
// of coarse rows [J0, J1) of a 256-coarse-column group (512 fine columns); the producer warp
// streams fine rows 2 J0 - 2 .. 2 J1 of u and g through the ring; each compute warp keeps
// three u rows in registers, forms the defect of the middle row (4 columns per lane, x
// neighbours by shuffles, the strip-edge lane also forms the defect one column to the left),
// folds it into the row sums (d_{i-1} + d_{i+1}) + 2 d_i at its two coarse columns, and
// writes coarse row J when the defect of fine row 2J + 1 is done.  The fine defect is never
// stored: 8 B read per fine unknown and 1 B written (FP32).  Same arithmetic, in the same
// order, as the tile kernel k_defect_restrict2d.
template <int KIND, bool IN>
__device__ __forceinline__ void band_dr(const Lev<float> L, const Lev<float> C, const float *__restrict__ u,
                                        const float *__restrict__ g, float *__restrict__ gc, int J0, int J1, int s0,
                                        float *ring, uint64_t *full, uint64_t *empty, int *err) {
  constexpr int SLOT = 2 * SEGW;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sw = s0 + 128 * warp;
  const int i0 = sw + 4 * lane;
  const int c0 = 4 + 128 * warp + 4 * lane;
  const bool edge = lane == 0 || lane == 31;
  const int io = lane == 0 ? sw - 1 : sw + 128;
  const int co = lane == 0 ? c0 - 1 : c0 + 4, co2 = lane == 0 ? c0 - 2 : c0 + 5;

  Coef K;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int i = i0 + e;
    K.act[e] = i >= 1 && i <= L.n0 - 2;
    if (KIND == K_CONST) {
      K.W[e] = L.cx; K.E[e] = L.cx; K.Y[e] = L.cy; K.D[e] = L.d; K.O[e] = 0.f;
    } else {
      const int ic = K.act[e] ? i : 1;
      K.W[e] = L.sx[ic - 1]; K.E[e] = L.sx[ic]; K.Y[e] = L.sy[ic];
      K.D[e] = (K.W[e] + K.E[e]) + (K.Y[e] + K.Y[e]);
      K.O[e] = 0.f;
    }
  }
  // the extra defect of lane 0 at column sw - 1
  const bool oact = lane == 0 && io >= 1 && io <= L.n0 - 2;
  float oW = L.cx, oE = L.cx, oY = L.cy, oD = L.d;
  if (KIND == K_SEP && lane == 0) {
    const int ic = oact ? io : 1;
    oW = L.sx[ic - 1]; oE = L.sx[ic]; oY = L.sy[ic];
    oD = (oW + oE) + (oY + oY);
  }

  const int cs = max(0, s0 - 4), ce = min((int)L.pitch, s0 + 128 * NW + 4);
  const int doff = cs - (s0 - 4);
  const uint32_t seg_bytes = (uint32_t)(ce - cs) * 4u;

  auto valid = [&](int j) { return IN || L.per || (j >= 0 && j < L.n1); };
  auto unk = [&](int j) { return IN || L.per || (j >= 1 && j <= L.n1 - 2); };
  auto wrap = [&](int j) -> int {
    if (IN || !L.per) return j;
    j = j < 0 ? j + L.n1 : (j >= L.n1 ? j - L.n1 : j);
    if (j < 0 || j >= L.n1) j = ((j % L.n1) + L.n1) % L.n1;
    return j;
  };
  const int jfirst = 2 * J0 - 2, jlast = 2 * J1;   // fine rows streamed
  auto slot_of = [&](int j) -> const float * { return ring + ((j - jfirst) & (RING - 1)) * SLOT; };
  const int jv0 = valid(jfirst) ? jfirst : (valid(jfirst + 1) ? jfirst + 1 : jfirst + 2);
  auto full_parity = [&](int j) -> uint32_t { return (uint32_t)(((j - jv0) >> RING_LOG) & 1); };
  auto empty_parity = [&](int j) -> uint32_t { return (uint32_t)(((j - jfirst) >> RING_LOG) & 1); };

  auto issue = [&](int j) {
    if (!valid(j)) return;
    const int k = j - jfirst;
    float *slot = ring + (k & (RING - 1)) * SLOT;
    uint64_t *bar = &full[k & (RING - 1)];
    const long long ro = (long long)wrap(j) * L.pitch;
    if (!MG_CKN(L, wrap(j), L.n1) || !MG_CKN(L, ce - 1, L.pitch)) return;   // debug build, as in the sweep
    mbar_expect_tx(bar, 2u * seg_bytes);
    tma_load_1d(slot + doff, u + ro + cs, seg_bytes, bar);
    tma_load_1d(slot + SEGW + doff, g + ro + cs, seg_bytes, bar);
  };
  if (warp == NW) {   // producer (lane 0): as in band_sweep
    if (lane != 0) return;
    int r = jfirst;
    bool ok = true;
    for (; r <= jlast; ++r) {
      if (r - RING >= jfirst &&
          !mbar_wait(&empty[(r - jfirst) & (RING - 1)], empty_parity(r - RING), WAIT_CYCLES)) {
        ok = false;
        break;
      }
      issue(r);
    }
    for (int q = max(jfirst, jlast - RING + 1); q <= jlast && ok; ++q)
      ok = mbar_wait(&empty[(q - jfirst) & (RING - 1)], empty_parity(q), WAIT_CYCLES);
    if (!ok) {
      atomicExch(err, 1);
      for (int q = max(jfirst, r - RING); q < r; ++q)
        if (valid(q)) mbar_wait(&full[(q - jfirst) & (RING - 1)], full_parity(q), DRAIN_CYCLES);
    }
    return;
  }
  auto arrive_row = [&](int j) -> bool {
    bool ok = true;
    if (valid(j)) ok = mbar_wait(&full[(j - jfirst) & (RING - 1)], full_parity(j), WAIT_CYCLES);
    return __all_sync(FULL, ok);
  };
  auto release = [&](int j) {
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[(j - jfirst) & (RING - 1)]);
  };
  auto load_row = [&](URow &R, int j) {
#pragma unroll
    for (int e = 0; e < 4; ++e) R.u[e] = 0.f;
    R.out = 0.f;
    R.out2 = 0.f;
    if (!valid(j)) return;
    const float *slot = slot_of(j);
    const float4 v = *reinterpret_cast<const float4 *>(slot + c0);
    R.u[0] = v.x; R.u[1] = v.y; R.u[2] = v.z; R.u[3] = v.w;
    if (edge) {
      R.out = slot[co];
      R.out2 = slot[co2];
    }
  };
  // row sums (d_{i-1} + d_{i+1}) + 2 d_i of the defect of fine row j at the lane's coarse columns
  // (fine 4L and 4L + 2 of the strip)
  auto defect_row3 = [&](const URow &Rm, const URow &R, const URow &Rp, int j, float &ra, float &rb) {
    const bool rowu = unk(j);
    const float4 g4 = *reinterpret_cast<const float4 *>(slot_of(j) + SEGW + c0);
    const float gg[4] = {g4.x, g4.y, g4.z, g4.w};
    float left = __shfl_up_sync(FULL, R.u[3], 1), right = __shfl_down_sync(FULL, R.u[0], 1);
    if (lane == 0) left = R.out;
    if (lane == 31) right = R.out;
    float d[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float wv = e > 0 ? R.u[e - 1] : left, ev = e < 3 ? R.u[e + 1] : right;
      float s = fmaf(-K.D[e], R.u[e], gg[e]);
      s = fmaf(K.W[e], wv, s);
      s = fmaf(K.E[e], ev, s);
      s = fmaf(K.Y[e], Rm.u[e], s);
      s = fmaf(K.Y[e], Rp.u[e], s);
      d[e] = (rowu && K.act[e]) ? s : 0.f;
    }
    // defect at column 4L - 1: the left lane's d[3]; lane 0 forms its own
    float dl = __shfl_up_sync(FULL, d[3], 1);
    if (lane == 0) {
      dl = 0.f;
      if (oact && rowu) {
        const float gl = slot_of(j)[SEGW + co];
        float s = fmaf(-oD, R.out, gl);
        s = fmaf(oW, R.out2, s);
        s = fmaf(oE, R.u[0], s);
        s = fmaf(oY, Rm.out, s);
        s = fmaf(oY, Rp.out, s);
        dl = s;
      }
    }
    ra = (dl + d[1]) + 2.f * d[0];
    rb = (d[1] + d[3]) + 2.f * d[2];
  };
  auto store_coarse = [&](int J, float va, float vb) {
    const bool Jok = C.per ? (J >= 0 && J < C.n1) : (J >= 1 && J <= C.n1 - 2);
    if (!Jok) return;
    const int I = (sw >> 1) + 2 * lane;
    float *rowp = gc + (long long)J * C.pitch;
    if (!MG_CK(C, (long long)J * C.pitch + I + 1)) return;
    if (I >= 1 && I <= C.n0 - 2) rowp[I] = va;
    if (I + 1 >= 1 && I + 1 <= C.n0 - 2) rowp[I + 1] = vb;
  };

  URow A, B, Cr;
  float pa = 0.f, pb = 0.f, ea = 0.f, eb = 0.f;   // row sums of fine rows 2J - 1 (odd) and 2J (even)
  bool ok = arrive_row(jfirst) && arrive_row(jfirst + 1);
  if (ok) {
    load_row(A, jfirst);
    load_row(B, jfirst + 1);
  }
  // fine row jf arrives -> defect of row jf - 1 (rows A = jf-2, B = jf-1, Cr = jf)
  auto step = [&](URow &Um, URow &Uc, URow &Up, int jf) -> bool {
    if (!arrive_row(jf)) return false;
    load_row(Up, jf);
    const int jd = jf - 1;   // row of the defect
    float ra, rb;
    defect_row3(Um, Uc, Up, jd, ra, rb);
    const int rel = jd - (2 * J0 - 1);   // 0, 1, 2, ... : rows 2J0-1, 2J0, 2J0+1, ...
    if (rel == 0) {
      pa = ra;
      pb = rb;
    } else if (rel & 1) {
      ea = ra;
      eb = rb;
    } else {   // jd = 2J + 1 with J = J0 + rel / 2 - 1
      const int J = J0 + rel / 2 - 1;
      store_coarse(J, ((pa + ra) + 2.f * ea) * 0.0625f, ((pb + rb) + 2.f * eb) * 0.0625f);
      pa = ra;
      pb = rb;
    }
    release(jf - 2);
    return true;
  };
  if (ok) {
    for (int jf = jfirst + 2; jf <= jlast; jf += 3) {
      if (!(ok = step(A, B, Cr, jf))) break;
      if (jf + 1 > jlast) break;
      if (!(ok = step(B, Cr, A, jf + 1))) break;
      if (jf + 2 > jlast) break;
      if (!(ok = step(Cr, A, B, jf + 2))) break;
    }
  }
  if (ok) {
    release(jlast - 1);
    release(jlast);
  } else if (lane == 0) {
    atomicExch(err, 1);
  }
}

template <int KIND>
__global__ void __launch_bounds__(32 * (NW + 1)) k_defect_restrict_tma(Lev<float> L, Lev<float> C,
                                                                       const float *__restrict__ u,
                                                                       const float *__restrict__ g,
                                                                       float *__restrict__ gc, int RCc, int ngroups,
                                                                       int *err) {
  MG_PDL_WAIT();
  constexpr int SLOT = 2 * SEGW;
  extern __shared__ __align__(128) unsigned char tma_smem[];
  float *ring = reinterpret_cast<float *>(tma_smem);
  uint64_t *full = reinterpret_cast<uint64_t *>(ring + RING * SLOT);
  uint64_t *empty = full + RING;
  const int grp = blockIdx.x % ngroups, band = blockIdx.x / ngroups;
  const int Jlo = C.per ? 0 : 1, Jhi = C.per ? C.n1 - 1 : C.n1 - 2;   // coarse unknown rows
  const int J0 = Jlo + band * RCc;
  if (J0 > Jhi) return;
  const int J1 = min(J0 + RCc, Jhi + 1);
  const int s0 = grp * 128 * NW;
  const int nact = min(NW, (int)(L.pitch - s0) / 128);
  for (int t = threadIdx.x; t < RING * SLOT; t += 32 * (NW + 1)) ring[t] = 0.f;
  if (threadIdx.x == 0) {
    for (int s = 0; s < RING; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], nact);
    }
    fence_mbar_init();
  }
  fence_proxy_async();
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  if (warp < NW && warp >= nact) return;
  const bool interior = L.per ? (2 * J0 - 2 >= 0 && 2 * J1 <= L.n1 - 1) : (2 * J0 - 2 >= 1 && 2 * J1 <= L.n1 - 2);
  if (interior) band_dr<KIND, true>(L, C, u, g, gc, J0, J1, s0, ring, full, empty, err);
  else band_dr<KIND, false>(L, C, u, g, gc, J0, J1, s0, ring, full, empty, err);
}

bool launch_defect_restrict_tma(const Launch &lc, const Lev<float> &L, const Lev<float> &C, int kind,
                                const float *u, const float *g, float *gc, int *err, int rc) {
  if (L.dim != 2 || kind == K_CELL || kind == K_EDGE || L.pitch % 128 != 0 || L.n0 < 5 || !err) return false;
  if (((uintptr_t)u | (uintptr_t)g) & 15) return false;
  const int crows = C.per ? C.n1 : C.n1 - 2;
  if (crows <= 0) return false;
  const int nstrips = (int)(L.pitch / 128);
  const int ngroups = (nstrips + NW - 1) / NW;
  const size_t smem = rb2d_tma_smem(0);
  const int ki = kind == K_CONST ? 0 : 1;
  int dev = 0;
  cudaGetDevice(&dev);
  static thread_local int occ_dev = -1, occ[2] = {0, 0}, sms = 0;
  if (occ_dev != dev) {
    occ_dev = dev;
    occ[0] = occ[1] = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  if (occ[ki] <= 0) {
    if (kind == K_CONST) {
      cudaFuncSetAttribute(k_defect_restrict_tma<K_CONST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[ki], k_defect_restrict_tma<K_CONST>, 32 * (NW + 1), smem);
    } else {
      cudaFuncSetAttribute(k_defect_restrict_tma<K_SEP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[ki], k_defect_restrict_tma<K_SEP>, 32 * (NW + 1), smem);
    }
    if (occ[ki] <= 0) occ[ki] = 1;
  }
  int RCc = rc;
  if (RCc <= 0) {
    const long long slots = (long long)std::max(sms, 1) * occ[ki];
    const long long nb = std::max<long long>(1, slots / ngroups);
    RCc = (int)std::max<long long>(4, (crows + nb - 1) / nb);
  }
  const int nbands = (crows + RCc - 1) / RCc;
  const unsigned blocks = (unsigned)((long long)ngroups * nbands);
  if (kind == K_CONST)
    k_defect_restrict_tma<K_CONST><<<blocks, 32 * (NW + 1), smem, lc.s>>>(L, C, u, g, gc, RCc, ngroups, err);
  else
    k_defect_restrict_tma<K_SEP><<<blocks, 32 * (NW + 1), smem, lc.s>>>(L, C, u, g, gc, RCc, ngroups, err);
  lc.done(__func__);
  return true;
}

size_t rb2d_tma_smem(int mode) {
  const int slot = slot_floats(mode);
  return ((size_t)RING * slot + pre_floats(mode)) * sizeof(float) + 2 * RING * sizeof(uint64_t);
}

namespace {
// resident CTAs per SM of one kernel instance and the SM count, queried once per device
struct TmaOcc {
  int dev = -1, sms = 0, occ[2][3] = {{0, 0, 0}, {0, 0, 0}};
};
thread_local TmaOcc tma_occ;
}  // namespace

bool launch_rb2d_tma(const Launch &lc, const Lev<float> &L, int kind, const float *u, const float *g, float *out,
                     float omega, int first, int mode, const Lev<float> *C, const float *ec, float omega_corr,
                     int *err, int rc, int *inject) {
  if (L.dim != 2 || kind == K_CELL || kind == K_EDGE || L.pitch % 128 != 0 || L.n0 < 3 || !err) return false;
  if (mode == 2 && (!C || !ec || C->pitch % 128 != 0)) return false;
  // every copy starts on a 16-byte boundary: 16-byte aligned arrays, pitches of 128 floats
  if (((uintptr_t)u | (uintptr_t)g | (uintptr_t)out | (uintptr_t)(ec ? ec : u)) & 15) return false;
  const int rows = L.per ? L.n1 : L.n1 - 2;
  if (rows <= 0) return false;
  const int nstrips = (int)(L.pitch / 128);
  const int ngroups = (nstrips + NW - 1) / NW;
  const size_t smem = rb2d_tma_smem(mode);
  const int ki = kind == K_CONST ? 0 : 1;

  int dev = 0;
  cudaGetDevice(&dev);
  if (tma_occ.dev != dev) {
    tma_occ = TmaOcc();
    tma_occ.dev = dev;
    cudaDeviceGetAttribute(&tma_occ.sms, cudaDevAttrMultiProcessorCount, dev);
  }
#define TMA_K(K, M) k_rb2d_tma<K, M>
#define TMA_OCC(K, M)                                                                                          \
  do {                                                                                                         \
    cudaFuncSetAttribute(TMA_K(K, M), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);                 \
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&tma_occ.occ[ki][mode], TMA_K(K, M), 32 * (NW + 1), smem);         \
  } while (0)
  if (tma_occ.occ[ki][mode] <= 0) {
    if (kind == K_CONST) {
      if (mode == 0) TMA_OCC(K_CONST, 0); else if (mode == 1) TMA_OCC(K_CONST, 1); else TMA_OCC(K_CONST, 2);
    } else {
      if (mode == 0) TMA_OCC(K_SEP, 0); else if (mode == 1) TMA_OCC(K_SEP, 1); else TMA_OCC(K_SEP, 2);
    }
    if (tma_occ.occ[ki][mode] <= 0) tma_occ.occ[ki][mode] = 1;
  }
#undef TMA_OCC
  // rows per CTA: as many bands as fill every SM's resident CTA slots once (8 rows at least)
  int RC = rc;
  if (RC <= 0) {
    const long long slots = (long long)std::max(tma_occ.sms, 1) * tma_occ.occ[ki][mode];
    const long long nb = std::max<long long>(1, slots / ngroups);
    RC = (int)std::max<long long>(8, (rows + nb - 1) / nb);
  }
  const int nbands = (rows + RC - 1) / RC;
  const unsigned blocks = (unsigned)((long long)ngroups * nbands);
  const Lev<float> Cv = C ? *C : L;
  const float *e = ec ? ec : u;
#define TMA_L(K, M)                                                                                          \
  TMA_K(K, M)<<<blocks, 32 * (NW + 1), smem, lc.s>>>(L, u, g, out, omega, first, Cv, e, omega_corr, RC, ngroups, err, \
                                                       inject)
  if (kind == K_CONST) {
    if (mode == 0) TMA_L(K_CONST, 0); else if (mode == 1) TMA_L(K_CONST, 1); else TMA_L(K_CONST, 2);
  } else {
    if (mode == 0) TMA_L(K_SEP, 0); else if (mode == 1) TMA_L(K_SEP, 1); else TMA_L(K_SEP, 2);
  }
#undef TMA_L
#undef TMA_K
  lc.done(__func__);
  return true;
}

}  // namespace mg
