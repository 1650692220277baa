// kernels_batch.cu -- many independent solves in one persistent, cooperative launch.
//
// Each instance is owned by a team of CTAs; the team runs the instance's step program: the
// copy of b and x into the instance's workspace, ||b||, the FP64 defect, then the refinement
// loop -- one FP32 F-cycle (Wallis 2008, section "The Multigrid Technique", algorithm
// MG(l, u, g), with the smoothers of section "The choice of C"), the FP64 update, the FP64
// defect and the convergence test -- and the copy of x out.  A team barrier (a counter in
// global memory, bounded wait) separates steps; steps on small grids run on the team's first
// CTA alone with block barriers.  Every step is a team-strided loop over the level's nodes;
// x-lines are solved one line per thread by the Thomas algorithm.  Supported: 2-D, y not
// periodic, constant or separable coefficients, point Jacobi / red-black Gauss-Seidel and
// x-line Jacobi / zebra smoothers (y-lines of the constant kind arrive as x-lines of the
// axis-swapped problem), FP32 cycles with FP64 refinement.
//
// A wait that runs out (about a second) sets the instance's wait flag and the team stops;
// the host reports MG_ETIMEOUT for it and for the instances the team had not reached.
#define MG_FILE_ID 11   // bounds-check sites (-DMG_DEBUG)
#include "batch_prog.h"
#include "coarse_prog.h"

namespace mg {

namespace {
constexpr int BT = kBatchThreads;
constexpr long long kBarWait = 1ll << 31;   // cycles a team barrier waits before it gives up (~1 s)

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

struct TeamState {
  int rank, size;
  unsigned gen;      // team barriers passed
  unsigned *bar;
  double *part;
  int red;           // reductions done (selects the half of part in use)
  int *err;          // the current instance's wait flag
  bool fail_arrival; // test hook armed for the current instance
};

// All CTAs of the team: every write before the barrier is visible after it.  Returns false
// when the wait gave up (or another CTA of the team gave up, or the test hook fired).
__device__ bool team_sync(TeamState &t) {
  __syncthreads();
  if (t.size == 1) return true;
  __shared__ int s_ok;
  t.gen += 1;
  if (threadIdx.x == 0) {
    int ok = 1;
    if (t.fail_arrival && t.rank == t.size - 1) {
      ok = 0;   // this CTA leaves without arriving: the others' bounded waits run out
    } else {
      __threadfence();
      atomicAdd(t.bar, 1u);
      const unsigned target = t.gen * (unsigned)t.size;
      const long long t0 = clock64();
      while (ld_acquire_u32(t.bar) < target) {
        if (*(volatile int *)t.err) { ok = 0; break; }
        if (clock64() - t0 > kBarWait) {
          atomicExch(t.err, 1);
          ok = 0;
          break;
        }
        __nanosleep(128);
      }
      __threadfence();
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ double block_sum_d(double v) {
  __shared__ double red[BT / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < BT / 32; ++w) s += red[w];
  __syncthreads();
  return s;   // valid in thread 0
}

// the team's total of one value per CTA (thread 0's), the same in every CTA (fixed order)
__device__ bool team_sum(TeamState &t, double v, double &out) {
  __shared__ double s_tot;
  if (t.size == 1) {
    if (threadIdx.x == 0) s_tot = v;
    __syncthreads();
    out = s_tot;
    return true;
  }
  double *buf = t.part + (t.red & 1) * t.size;
  t.red += 1;
  if (threadIdx.x == 0) buf[t.rank] = v;
  if (!team_sync(t)) return false;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < t.size; ++q) s += *(volatile double *)&buf[q];
    s_tot = s;
  }
  __syncthreads();
  out = s_tot;
  return true;
}

// ---- stencil pieces (2-D, y not periodic; plain pointers: data changes between steps) ----
template <typename T, int KIND>
struct W5 {
  T w, e, s, n, d, dinv;
  __device__ __forceinline__ void load(const Lev<T> &L, int i) {
    if (KIND == K_CONST) {
      w = e = L.cx;
      s = n = L.cy;
      d = L.d;
      dinv = L.dinv;
    } else {
      w = L.sx[i - 1];
      e = L.sx[i];
      s = n = L.sy[i];
      d = (w + e) + (s + n);
      dinv = L.sdinv[i];
    }
  }
};

template <typename T, int KIND>
__device__ __forceinline__ T resid5(const Lev<T> &L, const W5<T, KIND> &c, const T *u, long long p, T gp) {
  const long long pt = L.pitch;
  if (!MG_CK(L, p - pt) || !MG_CK(L, p + pt)) return gp;   // debug build (p -+ 1 lie between)
  T s = fma(-c.d, u[p], gp);
  s = fma(c.w, u[p - 1], s);
  s = fma(c.e, u[p + 1], s);
  s = fma(c.s, u[p - pt], s);
  s = fma(c.n, u[p + pt], s);
  return s;
}

// ---- steps (gt: this thread's index in the workers, nt: their number) ----
template <int KIND>
__device__ void st_rb(const BatchLev &V, float *u, int colour, float omega, int gt, int nt) {
  const Lev<float> &L = V.L;
  const int nx = L.n0 - 2, ny = L.n1 - 2, hx = (nx + 1) / 2;
  const long long total = (long long)hx * ny;
  for (long long t = gt; t < total; t += nt) {
    const int jr = (int)(t / hx), ti = (int)(t - (long long)jr * hx);
    const int j = 1 + jr, i = 1 + 2 * ti + ((colour + j + 1) & 1);
    if (i > nx) continue;
    const long long p = (long long)j * L.pitch + i;
    if (!MG_CK(L, p)) continue;   // debug build
    W5<float, KIND> c;
    c.load(L, i);
    u[p] = fmaf(omega * c.dinv, resid5<float, KIND>(L, c, u, p, V.g[p]), u[p]);
  }
}

template <int KIND>
__device__ void st_jac(const BatchLev &V, const float *u, float *out, float omega, int gt, int nt) {
  const Lev<float> &L = V.L;
  const int nx = L.n0 - 2, ny = L.n1 - 2;
  const long long total = (long long)nx * ny;
  for (long long t = gt; t < total; t += nt) {
    const int jr = (int)(t / nx), i = 1 + (int)(t - (long long)jr * nx), j = 1 + jr;
    const long long p = (long long)j * L.pitch + i;
    if (!MG_CK(L, p)) continue;   // debug build
    W5<float, KIND> c;
    c.load(L, i);
    out[p] = fmaf(omega * c.dinv, resid5<float, KIND>(L, c, u, p, V.g[p]), u[p]);
  }
}

template <int KIND>
__device__ void st_defect(const BatchLev &V, const float *u, int gt, int nt) {
  const Lev<float> &L = V.L;
  const int nx = L.n0 - 2, ny = L.n1 - 2;
  const long long total = (long long)nx * ny;
  for (long long t = gt; t < total; t += nt) {
    const int jr = (int)(t / nx), i = 1 + (int)(t - (long long)jr * nx), j = 1 + jr;
    const long long p = (long long)j * L.pitch + i;
    if (!MG_CK(L, p)) continue;   // debug build
    W5<float, KIND> c;
    c.load(L, i);
    V.r[p] = resid5<float, KIND>(L, c, u, p, V.g[p]);
  }
}

// x-lines (one thread a line, Thomas): the line system is the tridiagonal part of A along the
// line, its right-hand side g plus the couplings to the rows above and below.  s1 and s2 hold
// the eliminated right-hand side and upper diagonal; zebra lines (colour (j & 1)) update u in
// place, line Jacobi writes out.
template <int KIND>
__device__ void st_xline(const BatchLev &V, const float *u, float *out, float *s1, float *s2, int zebra, int colour,
                         float omega, int gt, int nt) {
  const Lev<float> &L = V.L;
  const int nx = L.n0 - 2, ny = L.n1 - 2;
  for (int jr = gt; jr < ny; jr += nt) {
    const int j = 1 + jr;
    if (zebra && (j & 1) != colour) continue;
    const long long row = (long long)j * L.pitch;
    if (!MG_CK(L, row + 1 - L.pitch) || !MG_CK(L, row + nx + L.pitch)) continue;   // debug build
    float cprev = 0.f, dprev = 0.f;
    for (int i = 1; i <= nx; ++i) {
      const long long p = row + i;
      W5<float, KIND> c;
      c.load(L, i);
      const float a = i > 1 ? -c.w : 0.f, cu = i < nx ? -c.e : 0.f;
      float d = V.g[p];
      d = fmaf(c.s, u[p - L.pitch], d);
      d = fmaf(c.n, u[p + L.pitch], d);
      const float den = c.d - a * cprev;
      const float cp = cu / den, dp = (d - a * dprev) / den;
      s2[p] = cp;
      s1[p] = dp;
      cprev = cp;
      dprev = dp;
    }
    float x = 0.f;
    for (int i = nx; i >= 1; --i) {
      const long long p = row + i;
      x = s1[p] - s2[p] * x;
      const float uo = u[p];
      out[p] = omega == 1.f ? x : fmaf(omega, x - uo, uo);
    }
  }
}

__device__ void st_restrict(const BatchLev &F, const BatchLev &C, int gt, int nt) {
  const int nx = C.L.n0 - 2, ny = C.L.n1 - 2;
  const long long total = (long long)nx * ny;
  for (long long t = gt; t < total; t += nt) {
    const int jr = (int)(t / nx), I = 1 + (int)(t - (long long)jr * nx), J = 1 + jr;
    const long long pf = (long long)(2 * J) * F.L.pitch + 2 * I, pt = F.L.pitch;
    if (!MG_CK(F.L, pf - pt - 1) || !MG_CK(F.L, pf + pt + 1) || !MG_CK(C.L, (long long)J * C.L.pitch + I)) continue;
    const float *r = F.r;
    const float rowm = (r[pf - pt - 1] + r[pf - pt + 1]) + 2.f * r[pf - pt];
    const float row0 = (r[pf - 1] + r[pf + 1]) + 2.f * r[pf];
    const float rowp = (r[pf + pt - 1] + r[pf + pt + 1]) + 2.f * r[pf + pt];
    C.g[(long long)J * C.L.pitch + I] = ((rowm + rowp) + 2.f * row0) * 0.0625f;
  }
}

__device__ void st_prolong(const BatchLev &F, const BatchLev &C, float *u, const float *e, float w, int gt, int nt) {
  const int nx = F.L.n0 - 2, ny = F.L.n1 - 2;
  const long long total = (long long)nx * ny;
  for (long long t = gt; t < total; t += nt) {
    const int jr = (int)(t / nx), i = 1 + (int)(t - (long long)jr * nx), j = 1 + jr;
    const int I0 = i >> 1, I1 = (i + 1) >> 1, J0 = j >> 1, J1 = (j + 1) >> 1;
    const long long a0 = (long long)J0 * C.L.pitch, a1 = (long long)J1 * C.L.pitch;
    const long long p = (long long)j * F.L.pitch + i;
    if (!MG_CK(F.L, p) || !MG_CK(C.L, a0 + I0) || !MG_CK(C.L, a1 + I1)) continue;   // debug build
    const float corr = ((e[a0 + I0] + e[a0 + I1]) + (e[a1 + I0] + e[a1 + I1])) * 0.25f;
    u[p] = fmaf(w, corr, u[p]);
  }
}

__device__ void st_fill(float *a, long long n, float v, int gt, int nt) {
  for (long long t = gt; t < n; t += nt) a[t] = v;
}
__device__ void st_copy(const float *a, float *b, long long n, int gt, int nt) {
  for (long long t = gt; t < n; t += nt) b[t] = a[t];
}

// u_1 = A_1^{-1} g_1 over the coarsest unknowns (FP64 inverse, FP64 sums)
__device__ void st_coarse(const BatchInst &I, const BatchLev &V, float *u, int gt, int nt) {
  for (int r = gt; r < I.nc; r += nt) {
    const double *row = I.Ainv + (long long)r * I.nc;
    double s = 0.0;
    for (int c = 0; c < I.nc; ++c) s = fma(row[c], (double)V.g[I.cidx[c]], s);
    u[I.cidx[r]] = (float)s;
  }
}

// FP64 defect of the finest level into g_L (FP32), and the sum of its squares (thread 0's value)
template <int KIND>
__device__ double st_defect64(const BatchInst &I, const BatchLev &V, int gt, int nt) {
  const Lev<double> &L = I.F64;
  const int nx = L.n0 - 2, ny = L.n1 - 2;
  const long long total = (long long)nx * ny;
  float acc = 0.f;
  for (long long t = gt; t < total; t += nt) {
    const int jr = (int)(t / nx), i = 1 + (int)(t - (long long)jr * nx), j = 1 + jr;
    const long long p = (long long)j * L.pitch + i;
    if (!MG_CK(L, p)) continue;   // debug build
    W5<double, KIND> c;
    c.load(L, i);
    const float s = (float)resid5<double, KIND>(L, c, I.x64, p, I.b64[p]);
    V.g[p] = s;
    acc = fmaf(s, s, acc);
  }
  return block_sum_d((double)acc);
}

__device__ double st_norm_b(const BatchInst &I, int gt, int nt) {
  const Lev<double> &L = I.F64;
  const int nx = L.n0 - 2, ny = L.n1 - 2;
  const long long total = (long long)nx * ny;
  double acc = 0.0;
  for (long long t = gt; t < total; t += nt) {
    const int jr = (int)(t / nx), i = 1 + (int)(t - (long long)jr * nx), j = 1 + jr;
    if (!MG_CK(L, (long long)j * L.pitch + i)) continue;   // debug build
    const double v = I.b64[(long long)j * L.pitch + i];
    acc = fma(v, v, acc);
  }
  return block_sum_d(acc);
}

__device__ void st_update(const BatchInst &I, const float *c, int gt, int nt) {
  const Lev<double> &L = I.F64;
  const int nx = L.n0 - 2, ny = L.n1 - 2;
  const long long total = (long long)nx * ny;
  for (long long t = gt; t < total; t += nt) {
    const int jr = (int)(t / nx), i = 1 + (int)(t - (long long)jr * nx), j = 1 + jr;
    const long long p = (long long)j * L.pitch + i;
    if (!MG_CK(L, p)) continue;   // debug build
    I.x64[p] += (double)c[p];
  }
}

// caller (compact) <-> internal (padded; transposed when the axes are swapped)
__device__ __forceinline__ long long caller_index(const BatchInst &I, int i, int j) {
  return I.swap ? (long long)i * I.n0c + j : (long long)j * I.n0c + i;
}
__device__ void st_pack(const BatchInst &I, int gt, int nt) {
  const Lev<double> &L = I.F64;
  const long long total = (long long)L.n0 * L.n1;
  for (long long t = gt; t < total; t += nt) {
    const int j = (int)(t / L.n0), i = (int)(t - (long long)j * L.n0);
    const bool unk = i >= 1 && i <= L.n0 - 2 && j >= 1 && j <= L.n1 - 2;
    const long long q = caller_index(I, i, j), p = (long long)j * L.pitch + i;
    if (!MG_CK(L, p)) continue;   // debug build
    I.x64[p] = unk ? I.xcall[q] : 0.0;
    I.b64[p] = unk ? I.bcall[q] : 0.0;
  }
}
__device__ void st_unpack(const BatchInst &I, bool zero, int gt, int nt) {
  const Lev<double> &L = I.F64;
  const long long total = (long long)L.n0 * L.n1;
  for (long long t = gt; t < total; t += nt) {
    const int j = (int)(t / L.n0), i = (int)(t - (long long)j * L.n0);
    if (!MG_CK(L, (long long)j * L.pitch + i)) continue;   // debug build
    I.xcall[caller_index(I, i, j)] = zero ? 0.0 : I.x64[(long long)j * L.pitch + i];
  }
}

// Run one instance's program.  Returns false if the team has to stop (a wait gave up).
template <int KIND>
__device__ bool run_instance(const BatchInst &I, TeamState &t, int epoch) {
  const int4 *prog = I.prog;
  const int plen = I.plen;
  const int gt_team = t.rank * BT + threadIdx.x, nt_team = t.size * BT;
  __shared__ double s_bsq, s_sq;
  __shared__ int s_it;
  if (threadIdx.x == 0) {
    s_it = 0;
    s_bsq = 0.0;
    s_sq = 0.0;
  }
  __syncthreads();
  int pc = 0;
  while (pc < plen) {
    const int4 op = prog[pc];
    const int code = op.x & 0xff;
    const bool solo = (op.x & BP_SOLO) && t.size > 1;
    if (solo && t.rank != 0) {
      // skip the run of solo steps; meet the first CTA at the barrier after it
      while (pc < plen && (prog[pc].x & BP_SOLO)) ++pc;
      if (!team_sync(t)) return false;
      continue;
    }
    const int gt = solo ? (int)threadIdx.x : gt_team, nt = solo ? BT : nt_team;
    const int l = op.y;
    int next = pc + 1;
    bool ok = true;
    switch (code) {
      case BP_PACK: st_pack(I, gt, nt); break;
      case BP_NORM_B: {
        double v = st_norm_b(I, gt, nt), tot;
        ok = team_sum(t, v, tot);
        if (threadIdx.x == 0) s_bsq = tot;
        break;
      }
      case BP_DEFECT64: {
        double v = st_defect64<KIND>(I, I.lev[I.L - 1], gt, nt), tot;
        ok = team_sum(t, v, tot);
        if (threadIdx.x == 0) s_sq = tot;
        break;
      }
      case BP_CHECK: {
        __syncthreads();
        const double b = s_bsq;
        const double rel = b == 0.0 ? 0.0 : sqrt(s_sq) / sqrt(b);
        const int it = op.z ? 0 : s_it + 1;
        int go = 1, status = 0;
        if (!(rel == rel) || rel > 1.7976931348623157e308) {
          go = 0;
          status = 5;
        } else if (rel <= *I.tol || b == 0.0) {
          go = 0;
        } else if (it >= I.maxit) {
          go = 0;
          status = 4;
        }
        __syncthreads();
        if (threadIdx.x == 0) s_it = it;
        if (t.rank == 0 && threadIdx.x == 0) {
          int *hi = reinterpret_cast<int *>(I.hrow);
          I.hrow[3 + it] = rel;
          hi[0] = it;
          hi[1] = status;
          I.scal[0] = b;
          I.scal[1] = s_sq;
        }
        next = go ? (op.z ? pc + 1 : op.y) : op.w;
        break;
      }
      case BP_ZERO: {
        const BatchLev &V = I.lev[l - 1];
        st_fill(V.u[op.z], V.L.pitch * (long long)V.L.n1, 0.f, gt, nt);
        break;
      }
      case BP_RB: {
        const BatchLev &V = I.lev[l - 1];
        st_rb<KIND>(V, V.u[op.w], op.z, I.omega, gt, nt);
        break;
      }
      case BP_JAC: {
        const BatchLev &V = I.lev[l - 1];
        st_jac<KIND>(V, V.u[op.w & 15], V.u[op.w >> 4], I.omega, gt, nt);
        break;
      }
      case BP_XLINE: {
        const BatchLev &V = I.lev[l - 1];
        const int src = op.w & 15, dst = op.w >> 4, zebra = op.z & 1, colour = op.z >> 1;
        // scratch: r and the buffer that is neither read nor written (zebra: the other u;
        // line Jacobi: the eliminated right-hand side goes to r, the upper diagonal to dst
        // before the back substitution overwrites it)
        float *s1 = V.r, *s2 = zebra ? V.u[1 - src] : V.u[dst];
        if (!zebra) {
          s1 = V.u[dst];
          s2 = V.r;
        }
        st_xline<KIND>(V, V.u[src], V.u[dst], s1, s2, zebra, colour, I.omega, gt, nt);
        break;
      }
      case BP_DEFECT: {
        const BatchLev &V = I.lev[l - 1];
        st_defect<KIND>(V, V.u[op.z], gt, nt);
        break;
      }
      case BP_RESTRICT: st_restrict(I.lev[l - 1], I.lev[l - 2], gt, nt); break;
      case BP_PROLONG: {
        const BatchLev &F = I.lev[l - 1], &C = I.lev[l - 2];
        st_prolong(F, C, F.u[op.z], C.u[op.w], I.omega_corr, gt, nt);
        break;
      }
      case BP_COARSE: {
        const BatchLev &V = I.lev[0];
        st_coarse(I, V, V.u[op.z], gt, nt);
        break;
      }
      case BP_COPY: {
        const BatchLev &V = I.lev[l - 1];
        st_copy(V.u[op.z], V.u[op.w], V.L.pitch * (long long)V.L.n1, gt, nt);
        break;
      }
      case BP_UPDATE: st_update(I, I.lev[I.L - 1].u[op.z], gt, nt); break;
      case BP_JUMP: next = op.y; break;
      case BP_UNPACK: {
        __syncthreads();
        st_unpack(I, s_bsq == 0.0, gt, nt);
        if (t.rank == 0 && threadIdx.x == 0) {
          int *hi = reinterpret_cast<int *>(I.hrow);
          I.hrow[2] = s_bsq;
          hi[2] = 0;
          __threadfence_system();
          hi[3] = epoch;
        }
        break;
      }
      case BP_END:
      default: next = plen; break;
    }
    if (!ok) return false;
    if (next >= plen) break;
    // barrier before the next step: block-wide between two solo steps, else team-wide
    const bool next_solo = (prog[next].x & BP_SOLO) && t.size > 1;
    if (solo && next_solo) __syncthreads();
    else if (!team_sync(t)) return false;
    pc = next;
  }
  __syncthreads();
  return true;
}

__global__ void __launch_bounds__(BT) k_batch(const BatchTeam *teams, int nteams, const BatchInst *insts,
                                              const int *order, int epoch) {
  MG_PDL_WAIT();
  // this CTA's team
  int lo = 0, hi = nteams - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (teams[mid].cta0 <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const BatchTeam tm = teams[lo];
  if ((int)blockIdx.x >= tm.cta0 + tm.size) return;   // spare CTA (none in a well-formed launch)
  TeamState t;
  t.rank = blockIdx.x - tm.cta0;
  t.size = tm.size;
  t.gen = 0;
  t.bar = tm.bar;
  t.part = tm.part;
  t.red = 0;
  for (int q = 0; q < tm.count; ++q) {
    const BatchInst &I = insts[order[tm.first + q]];
    t.err = I.st + 2;
    t.fail_arrival = I.fail_arrival != 0;
    const bool ok = I.kind == K_CONST ? run_instance<K_CONST>(I, t, epoch) : run_instance<K_SEP>(I, t, epoch);
    if (!ok) return;   // the team stops; instances it did not reach keep an older epoch
  }
}
}  // namespace

int batch_ctas_per_sm() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch, BT, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_batch(cudaStream_t s, int grid, const BatchTeam *teams, int nteams, const BatchInst *insts,
                         const int *order, int epoch, long long *counter) {
  int ep = epoch;
  void *args[] = {(void *)&teams, (void *)&nteams, (void *)&insts, (void *)&order, (void *)&ep};
  cudaError_t e = cudaLaunchCooperativeKernel((const void *)k_batch, dim3(grid), dim3(BT), args, 0, s);
  if (e == cudaSuccess) ++*counter;
  return e;
}

}  // namespace mg
