// kernels_ff.cu -- the outer defect of the mixed-precision refinement in float-float arithmetic.
//
// The refinement loop (row a11: r = b - A x in FP64 drives an FP32 F-cycle) needs the defect of
// the FP64 iterate to far more than FP32 accuracy: near convergence its 5-point sums cancel
// terms some 1e7 times larger than the result.  In FP64 that is five FMAs per unknown on a
// GPU whose FP64 pipe runs at ~1/50 of its FP32 rate, which bounds the kernel well below the
// memory rate.  Here every FP64 operand is split into a pair of floats (hi + lo, 47 significant
// bits) by integer operations on its bit pattern, and the stencil is evaluated with error-free
// FP32 transformations (TwoSum; a product and its exact rounding error by FMA), so the kernel
// runs on the FP32 and integer pipes.  The defect leaves rounded to FP32 (the FP32 cycle's
// right-hand side), with the sum of its squares for the stopping test.
//
// Accuracy: the pair keeps |d - (hi + lo)| <= 2^-46 |d| of each operand; the stencil terms are
// then summed almost exactly, so the defect's error at a node is a few 2^-46 times its largest
// terms, |b| + |A||x|, instead of FP64's 2^-53.  How much of that shows in ||r|| depends on the
// problem: on the 4097^2 isotropic benchmark near convergence the error is ~1e-12 ||b||
// (0.04 of 2^-46 ||(|b| + |A||x|)||); on strongly anisotropic lines (eps = 1e3) it is 0.19 of
// that norm, 7e-11 ||b||, too large for a 1e-10 stopping test.  The kernel therefore also
// returns the sum of squares of |b| + |A||x| (from the leading parts), the solver estimates
// the error as a fraction of its root, stops on this defect only when the residual is below
// the tolerance by that margin, and switches the loop to FP64 defects (use64, which this
// kernel reads) once the residual is within the margin of the tolerance.  The relative
// residual reported is that of a final FP64 defect.
//
// One warp covers 32 columns and marches down a band of rows, holding the split rows j-1, j,
// j+1 in registers and the loads of the next rows in flight; x-neighbours come by shuffles (the
// strip's edge lanes split the column beside the strip themselves).  2-D, constant or separable
// coefficients.
#define MG_FILE_ID 12   // bounds-check sites (-DMG_DEBUG)
#include "mg_internal.cuh"

namespace mg {

namespace {
constexpr int FX = 32, FY = 8;   // block: 8 warps, each one strip of 32 columns

struct FF {
  float h, l;
};

// d = h + l with h its leading 24 significant bits (truncated) and l the next 23 (truncated),
// from the bit pattern alone.  |d| below 2^-80 splits with l = 0 (an absolute error below
// 2^-103), below 2^-126 to h = l = 0: far below every other term of the stencil.
__device__ __forceinline__ FF split(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const unsigned sign = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7ffu);
  const int ef = e - 896;   // float biased exponent of h: e - 1023 + 127
  FF r;
  if (ef < 1) {
    r.h = 0.f;
    r.l = 0.f;
    return r;
  }
  const unsigned m23 = ((hw & 0xfffffu) << 3) | (lw >> 29);
  r.h = __uint_as_float(sign | ((unsigned)ef << 23) | m23);
  // next 23 mantissa bits as an integer m: lo = m * 2^(e - 1023 - 46); 2^23 + m has the float
  // bit pattern 0x4b000000 | m, so that float minus 2^23 is m exactly
  const unsigned m = (lw >> 6) & 0x7fffffu;
  const int es = e - 942;   // biased exponent of 2^(e - 1069)
  const float fm = __uint_as_float(0x4b000000u | m) - 8388608.0f;
  const float v = es >= 1 ? fm * __uint_as_float((unsigned)es << 23) : 0.f;
  r.l = __uint_as_float(__float_as_uint(v) | sign);
  return r;
}

// s + t = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &t) {
  s = a + b;
  const float bb = s - a;
  t = (a - (s - bb)) + (b - bb);
}

// (hi, lo) with hi + lo ~ c * x: the product of the leading parts exactly (FMA), plus the
// cross terms; c's and x's low parts product is below 2^-92 of the result and is dropped
__device__ __forceinline__ void prod(const FF &c, const FF &x, float &p, float &e) {
  p = c.h * x.h;
  e = fmaf(c.h, x.h, -p);
  e = fmaf(c.h, x.l, e);
  e = fmaf(c.l, x.h, e);
}

// a + b for two pairs (the sum of the leading parts exactly, the low parts added)
__device__ __forceinline__ FF add(const FF &a, const FF &b) {
  float s, t;
  two_sum(a.h, b.h, s, t);
  FF r;
  r.h = s;
  r.l = t + (a.l + b.l);
  return r;
}

// block sums of two values; thread 0 gets both
__device__ __forceinline__ void block_sum2_ff(float &v, float &w) {
  __shared__ float red[2][FX * FY / 32];
  for (int o = 16; o > 0; o >>= 1) {
    v += __shfl_down_sync(0xffffffffu, v, o);
    w += __shfl_down_sync(0xffffffffu, w, o);
  }
  const int t = threadIdx.y * FX + threadIdx.x;
  if ((t & 31) == 0) {
    red[0][t >> 5] = v;
    red[1][t >> 5] = w;
  }
  __syncthreads();
  if (t == 0) {
    v = w = 0.f;
    for (int k = 0; k < FX * FY / 32; ++k) {
      v += red[0][k];
      w += red[1][k];
    }
  }
}

// r32 = (float)(b - A x) at the unknowns of rows [band * R, band * R + R), one partial sum of
// r32^2 per block, and one of (|b| + |A||x|)^2 per block (partials + half).  With *use64 set
// the same marching evaluates the defect in FP64, in the FP64 defect kernel's order, and the
// second sum is 0.
// Fused refinement update (c32 != null): the iterate is double-buffered, *par selecting the
// current buffer (xa or xb).  The kernel reads the current one only, forms x + (double) c at
// every node it touches (the FP64 update of the refinement step, rounded as a separate update
// would round it), takes the defect of that, and writes it into the other buffer at its own
// nodes; the buffer it reads is never written during the launch, so neighbouring blocks need no
// ordering.  The finish kernel then flips *par.  c32 == null: the defect of xa, nothing written.
template <int KIND>
__global__ void __launch_bounds__(FX *FY) k_defect_ff(Lev<double> L, const double *__restrict__ xa,
                                                      double *__restrict__ xb, const double *__restrict__ b,
                                                      float *__restrict__ r32, double *__restrict__ partials,
                                                      int half, int R, const int *__restrict__ use64,
                                                      const float *__restrict__ c32, const int *__restrict__ par) {
  MG_PDL_WAIT();
  const bool f64 = use64 != nullptr && *use64 != 0;
  const bool upd = c32 != nullptr;
  const bool odd = upd && *par != 0;
  const double *__restrict__ x = odd ? xb : xa;   // the current iterate (read only)
  double *__restrict__ xout = odd ? const_cast<double *>(xa) : xb;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x;
  const int i = 1 + (blockIdx.x * FY + threadIdx.y) * FX + lane;   // this thread's column
  const int nx = L.n0 - 2;
  const int rows = L.per ? L.n1 : L.n1 - 2, ylo = L.per ? 0 : 1;
  const int r0 = blockIdx.y * R, r1 = min(rows, r0 + R);
  const bool act = i <= nx;
  const int ic = act ? i : 1;
  const bool edge = lane == 0 || lane == 31;
  const int io = lane == 0 ? i - 1 : i + 1;   // the column beside the strip (edge lanes)
  const bool oin = io >= 1 && io <= nx;        // an unknown column (else it reads as 0)
  // coefficients of the column (FP64, split once)
  FF cW, cE, cY, cD;
  if (KIND == K_CONST) {
    cW = cE = split(L.cx);
    cY = split(L.cy);
    cD = split(L.d);
  } else {
    const double w = L.sx[ic - 1], e = L.sx[ic], y = L.sy[ic];
    cW = split(w);
    cE = split(e);
    cY = split(y);
    cD = split((w + e) + (y + y));
  }
  auto row_of = [&](int r) -> long long {   // node offset of unknown row r (wrapped when periodic)
    int j = ylo + r;
    if (L.per) j = j < 0 ? j + L.n1 : (j >= L.n1 ? j - L.n1 : j);
    return (long long)j * L.pitch;
  };
  // x at node q, updated by the correction when the update is fused
  auto xat = [&](long long q) -> double { return upd ? x[q] + (double)c32[q] : x[q]; };
  auto raw = [&](int r) -> double {   // x at (i, row r); rows outside the unknowns (Dirichlet) read 0
    if (!act || (!L.per && (r < 0 || r >= rows))) return 0.0;
    const long long q = row_of(r) + i;
    return MG_CK(L, q) ? xat(q) : 0.0;   // (the check: debug build only)
  };
  auto bval = [&](int r) -> double {   // b at (i, row r) of an unknown row
    const long long q = row_of(r) + i;
    return MG_CK(L, q) ? b[q] : 0.0;
  };
  float acc = 0.f, acc2 = 0.f;
  if (f64 && r0 < r1) {
    double wW, wE, wY, dD;
    if (KIND == K_CONST) {
      wW = wE = L.cx;
      wY = L.cy;
      dD = L.d;
    } else {
      wW = L.sx[ic - 1];
      wE = L.sx[ic];
      wY = L.sy[ic];
      dD = (wW + wE) + (wY + wY);
    }
    double xm = raw(r0 - 1), xc = raw(r0), xnext = raw(r0 + 1);
    double bcur = act ? bval(r0) : 0.0;
    for (int r = r0; r < r1; ++r) {
      const double xafter = raw(r + 2);
      const double bnext = (act && r + 1 < r1) ? bval(r + 1) : 0.0;
      const double xp = xnext;
      const long long p = row_of(r) + i;
      double xw = __shfl_up_sync(FULL, xc, 1), xe = __shfl_down_sync(FULL, xc, 1);
      if (edge) {
        const double xo = (oin && MG_CK(L, p - i + io)) ? xat(p - i + io) : 0.0;
        if (lane == 0) xw = xo;
        else xe = xo;
      }
      if (act) {
        double s = fma(-dD, xc, bcur);
        s = fma(wW, xw, s);
        s = fma(wE, xe, s);
        s = fma(wY, xm, s);
        s = fma(wY, xp, s);
        const float res = (float)s;
        if (MG_CK(L, p)) {
          r32[p] = res;
          if (upd) xout[p] = xc;
        }
        acc = fmaf(res, res, acc);
      }
      xm = xc;
      xc = xp;
      xnext = xafter;
      bcur = bnext;
    }
  } else if (r0 < r1) {
    const float aW = fabsf(cW.h), aE = fabsf(cE.h), aY = fabsf(cY.h), aD = fabsf(cD.h);
    double xcd = raw(r0);   // row r's x in FP64 (written to the other buffer when the update is fused)
    FF xm = split(raw(r0 - 1)), xc = split(xcd), xp;
    // one row of lookahead: the loads of row r + 2 (x) and r + 1 (b) are in flight while row r
    // is computed
    double xnext = raw(r0 + 1);
    double bcur = act ? bval(r0) : 0.0;
    for (int r = r0; r < r1; ++r) {
      const double xafter = raw(r + 2);
      const double bnext = (act && r + 1 < r1) ? bval(r + 1) : 0.0;
      xp = split(xnext);
      const long long p = row_of(r) + i;
      // x-neighbours: the adjacent lanes' values, the edge lanes' from the column beside
      FF xw, xe;
      xw.h = __shfl_up_sync(FULL, xc.h, 1);
      xw.l = __shfl_up_sync(FULL, xc.l, 1);
      xe.h = __shfl_down_sync(FULL, xc.h, 1);
      xe.l = __shfl_down_sync(FULL, xc.l, 1);
      if (edge) {
        FF xo;
        xo.h = 0.f;
        xo.l = 0.f;
        if (oin && MG_CK(L, p - i + io)) xo = split(xat(p - i + io));
        if (lane == 0) xw = xo;
        else xe = xo;
      }
      if (act) {
        const FF bb = split(bcur);
        float p1, e1, p2, e2, p3, e3;
        prod(cD, xc, p1, e1);
        const FF sy = add(xm, xp);
        prod(cY, sy, p3, e3);
        // b - D x_p + W x_w + E x_e + Y (x_s + x_n): the leading parts by TwoSum, the rest added
        float s, t1, t2, t3;
        two_sum(bb.h, -p1, s, t1);
        float lo;
        if (KIND == K_CONST) {
          const FF sx = add(xw, xe);
          prod(cW, sx, p2, e2);
          two_sum(s, p2, s, t2);
          two_sum(s, p3, s, t3);
          lo = ((bb.l - e1) + (e2 + e3)) + ((t1 + t2) + t3);
        } else {
          float p4, e4, t4;
          prod(cW, xw, p2, e2);
          prod(cE, xe, p4, e4);
          two_sum(s, p2, s, t2);
          two_sum(s, p3, s, t3);
          two_sum(s, p4, s, t4);
          lo = (((bb.l - e1) + (e2 + e3)) + e4) + ((t1 + t2) + (t3 + t4));
        }
        const float res = s + lo;
        if (MG_CK(L, p)) {
          r32[p] = res;
          if (upd) xout[p] = xcd;
        }
        acc = fmaf(res, res, acc);
        // |b| + |A||x| from the leading parts: the scale of this node's float-float error
        const float tt = fmaf(aD, fabsf(xc.h),
                              fmaf(aW, fabsf(xw.h), fmaf(aE, fabsf(xe.h), fmaf(aY, fabsf(xm.h) + fabsf(xp.h),
                                                                                fabsf(bb.h)))));
        acc2 = fmaf(tt, tt, acc2);
      }
      xm = xc;
      xc = xp;
      xcd = xnext;
      xnext = xafter;
      bcur = bnext;
    }
  }
  block_sum2_ff(acc, acc2);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    const int q = blockIdx.y * gridDim.x + blockIdx.x;
    partials[q] = (double)acc;
    partials[half + q] = (double)acc2;
  }
}

// block 0: out_sq = sum of partials[0, n); block 1: out_t = sum of partials[half, half + n)
// (fixed order, as the norm finish)
__global__ void __launch_bounds__(1024) k_ff_finish(const double *__restrict__ partials, int n, int half,
                                                    double *out_sq, double *out_t, int *par) {
  MG_PDL_WAIT();
  if (par && blockIdx.x == 0 && threadIdx.x == 0) par[0] ^= 1;   // the fused update's buffer swap
  const double *src = partials + (blockIdx.x ? half : 0);
  double acc = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) acc += src[t];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) (blockIdx.x ? out_t : out_sq)[0] = s;
  }
}
}  // namespace

bool launch_defect_ff(const Launch &lc, const Lev<double> &L, int kind, double *xa, double *xb, const double *b,
                      float *r32, double *partials, int nparts, double *out_sq, double *out_t, const int *use64,
                      const float *c32, int *par) {
  if (L.dim != 2 || (kind != K_CONST && kind != K_SEP)) return false;
  if (c32 && (!xb || !par)) return false;
  const int nx = L.n0 - 2, rows = L.per ? L.n1 : L.n1 - 2;
  if (nx < 1 || rows < 1) return false;
  const int half = nparts / 2;   // the two sums' partials side by side
  const int gx = (nx + FX * FY - 1) / (FX * FY);
  if (gx > half) return false;
  // rows per block: 32, more when the blocks would outnumber the partial sums or gridDim.y
  long long R = 32;
  const long long gy_max = std::min<long long>(65535, half / gx);
  if ((rows + R - 1) / R > gy_max) R = (rows + gy_max - 1) / gy_max;
  const dim3 gr((unsigned)gx, (unsigned)((rows + R - 1) / R)), bl(FX, FY);
  if (kind == K_CONST)
    k_defect_ff<K_CONST><<<gr, bl, 0, lc.s>>>(L, xa, xb, b, r32, partials, half, (int)R, use64, c32, par);
  else
    k_defect_ff<K_SEP><<<gr, bl, 0, lc.s>>>(L, xa, xb, b, r32, partials, half, (int)R, use64, c32, par);
  lc.done(__func__);
  k_ff_finish<<<2, 1024, 0, lc.s>>>(partials, (int)(gr.x * gr.y), half, out_sq, out_t, c32 ? par : nullptr);
  lc.done(__func__);
  return true;
}

// After a loop of fused updates: bring the iterate into xa (copy from xb when *par is set).
__global__ void k_x_settle(double *__restrict__ xa, const double *__restrict__ xb, long long n,
                           const int *__restrict__ par) {
  MG_PDL_WAIT();
  if (*par == 0) return;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    xa[t] = xb[t];
}
void launch_x_settle(const Launch &lc, double *xa, const double *xb, long long n, int *par) {
  k_x_settle<<<1216, 256, 0, lc.s>>>(xa, xb, n, par);
  lc.done(__func__);
  cudaMemsetAsync(par, 0, sizeof(int), lc.s);
}

}  // namespace mg
