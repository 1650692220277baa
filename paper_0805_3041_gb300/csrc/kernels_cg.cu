// kernels_cg.cu -- the coarsest-grid solve by conjugate gradients, for coarsest grids too large
// for a dense inverse.
//
// The coarsest solve of the cycle is exact (Wallis 2008, section "The Multigrid Technique": the
// coarsest level returns A_1^{-1} g).  Up to 4096 unknowns it applies a dense inverse; above
// that, FP64 conjugate gradients run to a relative residual of 1e-14 (A_1 is symmetric positive
// definite).  The whole iteration is one cooperative launch: the blocks meet at the grid
// barrier after each reduction, and every block forms the same fixed-order sum of the block
// partials, so all blocks take identical decisions and the result does not depend on timing.
#include <cooperative_groups.h>

#define MG_FILE_ID 10   // bounds-check sites (-DMG_DEBUG)
#include "mg_internal.cuh"

namespace mg {

namespace cgx = cooperative_groups;

namespace {
constexpr int CG_THREADS = 256;

// sum over the block (fixed shuffle pattern, fixed shared-memory tree); every thread gets it
__device__ __forceinline__ double cg_block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();   // red is reused by consecutive calls
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double s = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}
}  // namespace

// u = A^{-1} g on level L (unknowns; g and u in the level's precision T, iteration in FP64).
// x, r, p, ap: FP64 node arrays of the level, zero off the unknowns.  part: 2 * gridDim.x doubles.
// Stops when ||r||^2 <= rtol2 ||g||^2 or after max_it iterations; iters[0] = iterations done.
template <typename T, int DIM, int KIND>
__global__ void __launch_bounds__(CG_THREADS) k_coarse_cg(Lev<double> L, const T *__restrict__ g, T *__restrict__ u,
                                                           double *__restrict__ x, double *__restrict__ r,
                                                           double *__restrict__ p, double *__restrict__ ap,
                                                           double *__restrict__ part, int max_it, double rtol2,
                                                           int *__restrict__ iters) {
  MG_PDL_WAIT();
  cgx::grid_group grid = cgx::this_grid();
  __shared__ double red[33];
  const int nx = L.n0 - 2;
  const long long nunk = L.unk_rows() * nx;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x, nt = (long long)gridDim.x * blockDim.x;
  const int nb = (int)gridDim.x;
  auto node = [&](long long t, int &i, int &j, int &k) -> long long {
    const long long rr = t / nx;
    i = 1 + (int)(t - rr * nx);
    row_jk(L, rr, j, k);
    return (long long)k * L.plane + (long long)j * L.pitch + i;
  };
  // the same fixed-order total in every block: block sums -> grid barrier -> warp 0 of each
  // block adds the partials in a fixed lane order
  auto allsum = [&](double v, int buf) -> double {
    double bs = cg_block_sum(v, red);
    if (threadIdx.x == 0) part[buf * nb + blockIdx.x] = bs;
    grid.sync();
    double s = 0.0;
    if (threadIdx.x < 32) {
      for (int q = (int)threadIdx.x; q < nb; q += 32) s += part[buf * nb + q];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (threadIdx.x == 0) red[32] = s;
    }
    __syncthreads();
    s = red[32];
    __syncthreads();
    return s;
  };
  double loc = 0.0;
  for (long long t = t0; t < nunk; t += nt) {
    int i, j, k;
    const long long q = node(t, i, j, k);
    if (!MG_CK(L, q)) continue;   // debug build
    const double v = (double)g[q];
    x[q] = 0.0;
    r[q] = v;
    p[q] = v;
    loc = fma(v, v, loc);
  }
  double rr = allsum(loc, 1);
  const double stop = rtol2 * rr;
  int it = 0;
  for (; it < max_it && rr > stop; ++it) {
    grid.sync();   // p complete before the product
    loc = 0.0;
    for (long long t = t0; t < nunk; t += nt) {
      int i, j, k;
      const long long q = node(t, i, j, k);
      if (!MG_CK(L, q)) continue;   // debug build
      long long dm, dp;
      yoffs(L, j, dm, dp);
      Weights<double, DIM, KIND> w;
      w.load(L, i, q, dm);
      const double a = -residual_at<double, DIM, KIND>(L, w, p, q, dm, dp, 0.0);   // (A p)_q
      ap[q] = a;
      loc = fma(p[q], a, loc);
    }
    const double pap = allsum(loc, 0);
    if (!(pap > 0.0)) break;   // exact solution reached (p = 0) or a non-positive curvature
    const double alpha = rr / pap;
    loc = 0.0;
    for (long long t = t0; t < nunk; t += nt) {
      int i, j, k;
      const long long q = node(t, i, j, k);
      if (!MG_CK(L, q)) continue;   // debug build
      x[q] = fma(alpha, p[q], x[q]);
      const double rv = fma(-alpha, ap[q], r[q]);
      r[q] = rv;
      loc = fma(rv, rv, loc);
    }
    const double rn = allsum(loc, 1);
    const double beta = rn / rr;
    rr = rn;
    for (long long t = t0; t < nunk; t += nt) {
      int i, j, k;
      const long long q = node(t, i, j, k);
      if (!MG_CK(L, q)) continue;   // debug build
      p[q] = fma(beta, p[q], r[q]);
    }
  }
  for (long long t = t0; t < nunk; t += nt) {
    int i, j, k;
    const long long q = node(t, i, j, k);
    if (!MG_CK(L, q)) continue;   // debug build
    u[q] = (T)x[q];
  }
  if (t0 == 0) iters[0] = it;
}

template <typename T>
void launch_coarse_cg(const Launch &lc, const Lev<double> &L, int kind, const T *g, T *u, double *work, double *part,
                      int max_it, double rtol, int *iters) {
  const long long count = L.plane * (L.dim == 3 ? L.n2 : 1);
  double *x = work, *r = work + count, *p = work + 2 * count, *ap = work + 3 * count;
  double rtol2 = rtol * rtol;
  void *args[] = {(void *)&L, (void *)&g, (void *)&u, (void *)&x, (void *)&r, (void *)&p, (void *)&ap,
                  (void *)&part, (void *)&max_it, (void *)&rtol2, (void *)&iters};
  const long long nunk = L.unk_rows() * (L.n0 - 2);
  auto go = [&](auto fn) {
    // every block must be resident at once (cooperative launch): at most the occupancy limit
    static thread_local int occ = -1, sms = 0;
    if (occ < 0) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, CG_THREADS, 0);
    }
    long long want = (nunk + CG_THREADS - 1) / CG_THREADS;
    long long cap = (long long)(occ > 0 ? occ : 1) * (sms > 0 ? sms : 1);
    unsigned blocks = (unsigned)(want < cap ? (want > 0 ? want : 1) : cap);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(CG_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = lc.s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelExC(&cfg, (const void *)fn, args);
  };
  if (L.dim == 2) {
    if (kind == K_CONST) go(k_coarse_cg<T, 2, K_CONST>);
    else if (kind == K_SEP) go(k_coarse_cg<T, 2, K_SEP>);
    else if (kind == K_CELL) go(k_coarse_cg<T, 2, K_CELL>);
    else go(k_coarse_cg<T, 2, K_EDGE>);
  } else {
    if (kind == K_CONST) go(k_coarse_cg<T, 3, K_CONST>);
    else if (kind == K_SEP) go(k_coarse_cg<T, 3, K_SEP>);
    else if (kind == K_CELL) go(k_coarse_cg<T, 3, K_CELL>);
    else go(k_coarse_cg<T, 3, K_EDGE>);
  }
  lc.done(__func__);
}

template void launch_coarse_cg<double>(const Launch &, const Lev<double> &, int, const double *, double *, double *,
                                       double *, int, double, int *);
template void launch_coarse_cg<float>(const Launch &, const Lev<double> &, int, const float *, float *, double *,
                                      double *, int, double, int *);

}  // namespace mg
