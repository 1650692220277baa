// kernels_point.cu -- point-wise stencil kernels: damped Jacobi, red-black
// Gauss-Seidel half-sweeps, defect, defect norms, the mixed-precision defect and
// refinement update, and the cell-coefficient gradient.
//
// Smoothers are preconditioned Richardson steps x <- x + omega C^{-1}(b - A x)
// (Wallis 2008, section "Smoothers"); C = D for Jacobi and C = D + L in
// red-black order for Gauss-Seidel (section "The choice of C").
//
// Launch shape: blocks of 32 x 8 threads.  threadIdx.x runs along x (coalesced
// rows), each thread handles R consecutive unknown rows (j, k).  Every thread
// writes only unknown nodes of its own rows.
#define MG_FILE_ID 1   // bounds-check sites (-DMG_DEBUG)
#include "mg_internal.cuh"

namespace mg {

static constexpr int BX = 32, BY = 8;

static inline int rows_per_thread(long long rows) { return rows >= 2048 ? 4 : 1; }

static inline dim3 grid_for(long long xthreads, long long rows, int R) {
  long long gy = (rows + (long long)BY * R - 1) / ((long long)BY * R);
  return dim3((unsigned)((xthreads + BX - 1) / BX), (unsigned)gy, 1);
}

// ---------------------------------------------------------------------------------------
// damped Jacobi, out of place: out = u + omega D^{-1} (g - A u)
// ---------------------------------------------------------------------------------------
template <typename T, int DIM, int KIND>
__global__ void __launch_bounds__(BX *BY) k_jacobi(Lev<T> L, const T *__restrict__ u, const T *__restrict__ g,
                                                   T *__restrict__ out, T omega, int R) {
  MG_PDL_WAIT();
  int i = 1 + blockIdx.x * BX + threadIdx.x;
  if (i > L.n0 - 2) return;
  long long r0 = ((long long)blockIdx.y * BY + threadIdx.y) * R;
  long long nr = L.unk_rows();
  for (int q = 0; q < R; ++q) {
    long long r = r0 + q;
    if (r >= nr) return;
    int j, k;
    row_jk(L, r, j, k);
    long long p = (long long)k * L.plane + (long long)j * L.pitch + i, dm, dp;
    yoffs(L, j, dm, dp);
    if (!MG_CK(L, p)) continue;
    Weights<T, DIM, KIND> w;
    w.load(L, i, p, dm);
    T s = residual_at<T, DIM, KIND>(L, w, u, p, dm, dp, g[p]);
    out[p] = fma(omega * w.dinv, s, u[p]);
  }
}

// first sweep from a zero iterate: out = omega D^{-1} g
template <typename T, int DIM, int KIND>
__global__ void __launch_bounds__(BX *BY) k_jacobi_zero(Lev<T> L, const T *__restrict__ g, T *__restrict__ out,
                                                        T omega, int R) {
  MG_PDL_WAIT();
  int i = 1 + blockIdx.x * BX + threadIdx.x;
  if (i > L.n0 - 2) return;
  long long r0 = ((long long)blockIdx.y * BY + threadIdx.y) * R;
  long long nr = L.unk_rows();
  for (int q = 0; q < R; ++q) {
    long long r = r0 + q;
    if (r >= nr) return;
    int j, k;
    row_jk(L, r, j, k);
    long long p = (long long)k * L.plane + (long long)j * L.pitch + i, dm, dp;
    yoffs(L, j, dm, dp);
    if (!MG_CK(L, p)) continue;
    Weights<T, DIM, KIND> w;
    w.load(L, i, p, dm);
    out[p] = omega * w.dinv * g[p];
  }
}

// ---------------------------------------------------------------------------------------
// red-black Gauss-Seidel half-sweep, in place on the nodes with (i+j+k) % 2 == colour.
// Only nodes of the other colour are read as neighbours, so the update is race free.
// Thread t of a row handles node i = 1 + 2t + ((colour + j + k + 1) & 1).
// ---------------------------------------------------------------------------------------
template <typename T, int DIM, int KIND>
__global__ void __launch_bounds__(BX *BY) k_rb_half(Lev<T> L, T *u, const T *__restrict__ g, T omega, int colour,
                                                    int R) {
  MG_PDL_WAIT();
  int t = blockIdx.x * BX + threadIdx.x;
  long long r0 = ((long long)blockIdx.y * BY + threadIdx.y) * R;
  long long nr = L.unk_rows();
  for (int q = 0; q < R; ++q) {
    long long r = r0 + q;
    if (r >= nr) return;
    int j, k;
    row_jk(L, r, j, k);
    int i = 1 + 2 * t + ((colour + j + k + 1) & 1);
    if (i > L.n0 - 2) continue;
    long long p = (long long)k * L.plane + (long long)j * L.pitch + i, dm, dp;
    yoffs(L, j, dm, dp);
    if (!MG_CK(L, p)) continue;
    Weights<T, DIM, KIND> w;
    w.load(L, i, p, dm);
    T s = residual_at<T, DIM, KIND>(L, w, u, p, dm, dp, g[p]);
    u[p] = fma(omega * w.dinv, s, u[p]);
  }
}

// ---------------------------------------------------------------------------------------
// Gauss-Seidel on a 2-D Galerkin level (9-point stencil), in place on the nodes of one of the
// four colours (i mod 2, j mod 2) = (ci, cj): nodes of one colour are two apart in both
// directions and share no stencil, so the update is race free.  Thread t of colour row q
// handles node i = 2 + 2t - ci... written below as i = (ci ? 1 : 2) + 2t, row j = (cj ? 1 : 2) + 2q.
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(BX *BY) k_gs9_colour(Lev<T> L, T *u, const T *__restrict__ g, T omega, int ci,
                                                       int cj, int R) {
  MG_PDL_WAIT();
  const int t = blockIdx.x * BX + threadIdx.x;
  const int i = (ci ? 1 : 2) + 2 * t;
  if (i > L.n0 - 2) return;
  const int jlo = cj ? 1 : 2;
  const int nr = (L.n1 - 2 - jlo) / 2 + 1;   // rows j = jlo, jlo + 2, ... <= n1 - 2
  const int q0 = (blockIdx.y * BY + threadIdx.y) * R;
  for (int q = q0; q < q0 + R && q < nr; ++q) {
    const int j = jlo + 2 * q;
    long long p = (long long)j * L.pitch + i, dm, dp;
    yoffs(L, j, dm, dp);
    if (!MG_CK(L, p)) continue;
    Weights<T, 2, K_NINE> w;
    w.load(L, i, p, dm);
    T s = residual_at<T, 2, K_NINE>(L, w, u, p, dm, dp, g[p]);
    u[p] = fma(omega * w.dinv, s, u[p]);
  }
}

// ---------------------------------------------------------------------------------------
// defect r = g - A u
// ---------------------------------------------------------------------------------------
template <typename T, int DIM, int KIND>
__global__ void __launch_bounds__(BX *BY) k_defect(Lev<T> L, const T *__restrict__ u, const T *__restrict__ g,
                                                   T *__restrict__ r_out, int R) {
  MG_PDL_WAIT();
  int i = 1 + blockIdx.x * BX + threadIdx.x;
  if (i > L.n0 - 2) return;
  long long r0 = ((long long)blockIdx.y * BY + threadIdx.y) * R;
  long long nr = L.unk_rows();
  for (int q = 0; q < R; ++q) {
    long long r = r0 + q;
    if (r >= nr) return;
    int j, k;
    row_jk(L, r, j, k);
    long long p = (long long)k * L.plane + (long long)j * L.pitch + i, dm, dp;
    yoffs(L, j, dm, dp);
    if (!MG_CK(L, p)) continue;
    Weights<T, DIM, KIND> w;
    w.load(L, i, p, dm);
    r_out[p] = residual_at<T, DIM, KIND>(L, w, u, p, dm, dp, g[p]);
  }
}

// deterministic block sum of a double (fixed shuffle pattern, fixed smem tree)
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31, wid = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  int nw = (blockDim.x * blockDim.y + 31) >> 5;
  double s = 0.0;
  if (wid == 0) {
    s = lane < nw ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;
}

// the same in FP32 (for FP32 squares: keeps the FP64 pipe free in FP64-bound kernels)
__device__ __forceinline__ float block_sum_f(float v) {
  __shared__ float redf[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31, wid = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
  if (lane == 0) redf[wid] = v;
  __syncthreads();
  int nw = (blockDim.x * blockDim.y + 31) >> 5;
  float s = 0.f;
  if (wid == 0) {
    s = lane < nw ? redf[lane] : 0.f;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;
}

// sum of squares of the defect over the unknowns, one partial per block
template <typename T, int DIM, int KIND>
__global__ void __launch_bounds__(BX *BY) k_defect_norm(Lev<T> L, const T *__restrict__ u, const T *__restrict__ g,
                                                        double *__restrict__ partials, int R) {
  MG_PDL_WAIT();
  int i = 1 + blockIdx.x * BX + threadIdx.x;
  long long r0 = ((long long)blockIdx.y * BY + threadIdx.y) * R;
  long long nr = L.unk_rows();
  double acc = 0.0;
  if (i <= L.n0 - 2) {
    for (int q = 0; q < R; ++q) {
      long long r = r0 + q;
      if (r >= nr) break;
      int j, k;
      row_jk(L, r, j, k);
      long long p = (long long)k * L.plane + (long long)j * L.pitch + i, dm, dp;
      yoffs(L, j, dm, dp);
      if (!MG_CK(L, p)) continue;
      Weights<T, DIM, KIND> w;
      w.load(L, i, p, dm);
      double s = (double)residual_at<T, DIM, KIND>(L, w, u, p, dm, dp, g[p]);
      acc = fma(s, s, acc);
    }
  }
  double bs = block_sum(acc);
  if (threadIdx.x == 0 && threadIdx.y == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = bs;
}

template <typename T>
__global__ void __launch_bounds__(BX *BY) k_norm_parts(Lev<T> L, const T *__restrict__ v, double *__restrict__ partials,
                                                       int R) {
  MG_PDL_WAIT();
  int i = 1 + blockIdx.x * BX + threadIdx.x;
  long long r0 = ((long long)blockIdx.y * BY + threadIdx.y) * R;
  long long nr = L.unk_rows();
  double acc = 0.0;
  if (i <= L.n0 - 2) {
    for (int q = 0; q < R; ++q) {
      long long r = r0 + q;
      if (r >= nr) break;
      int j, k;
      row_jk(L, r, j, k);
      const long long p = (long long)k * L.plane + (long long)j * L.pitch + i;
      if (!MG_CK(L, p)) continue;
      double s = (double)v[p];
      acc = fma(s, s, acc);
    }
  }
  double bs = block_sum(acc);
  if (threadIdx.x == 0 && threadIdx.y == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = bs;
}

// single block: out[0] = sum of partials in a fixed order
__global__ void __launch_bounds__(1024) k_norm_finish(const double *__restrict__ partials, int n, double *out) {
  MG_PDL_WAIT();
  double acc = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) acc += partials[t];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) out[0] = s;
  }
}

// ---------------------------------------------------------------------------------------
// adaptive correction weight (Wallis 2008, section "Multigrid": omega_l chosen to minimise
// the energy norm of the error): omega = (d, P e) / (A P e, P e) with d = g - A u
// ---------------------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T block_sum_t(T v);
template <>
__device__ __forceinline__ double block_sum_t<double>(double v) { return block_sum(v); }
template <>
__device__ __forceinline__ float block_sum_t<float>(float v) { return block_sum_f(v); }

// Sums of d . Pe and (A Pe) . Pe over the unknowns (pe holds P e, zero off the unknowns),
// accumulated per thread in the level's precision (FP64 throughput is the limit in FP32
// levels otherwise), one FP64 partial pair per block.  The last block to finish sums the
// partials in a fixed order, writes omega = sum1 / sum2 (1 when P e = 0) and re-arms the
// counter.
template <typename T, int DIM, int KIND>
__global__ void __launch_bounds__(BX *BY) k_corr_dots(Lev<T> L, const T *__restrict__ u, const T *__restrict__ g,
                                                      const T *__restrict__ pe, double *__restrict__ partials,
                                                      unsigned *__restrict__ count, double *__restrict__ omega, int R) {
  MG_PDL_WAIT();
  int i = 1 + blockIdx.x * BX + threadIdx.x;
  long long r0 = ((long long)blockIdx.y * BY + threadIdx.y) * R;
  long long nr = L.unk_rows();
  T a0 = T(0), a1 = T(0);
  if (i <= L.n0 - 2) {
    for (int q = 0; q < R; ++q) {
      long long r = r0 + q;
      if (r >= nr) break;
      int j, k;
      row_jk(L, r, j, k);
      long long p = (long long)k * L.plane + (long long)j * L.pitch + i, dm, dp;
      yoffs(L, j, dm, dp);
      if (!MG_CK(L, p)) continue;
      Weights<T, DIM, KIND> w;
      w.load(L, i, p, dm);
      T d = residual_at<T, DIM, KIND>(L, w, u, p, dm, dp, g[p]);
      T ape = -residual_at<T, DIM, KIND>(L, w, pe, p, dm, dp, T(0));
      T v = pe[p];
      a0 = fma(d, v, a0);
      a1 = fma(ape, v, a1);
    }
  }
  const int nb = (int)(gridDim.x * gridDim.y), b = blockIdx.y * gridDim.x + blockIdx.x;
  const bool t0 = threadIdx.x == 0 && threadIdx.y == 0;
  double s0 = (double)block_sum_t<T>(a0);
  __syncthreads();   // block_sum's shared slots are reused
  double s1 = (double)block_sum_t<T>(a1);
  __shared__ bool last;
  if (t0) {
    partials[b] = s0;
    partials[nb + b] = s1;
    __threadfence();
    last = atomicAdd(count, 1u) == (unsigned)nb - 1u;
  }
  __syncthreads();
  if (!last) return;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  double n0 = 0.0, n1 = 0.0;
  for (int t = tid; t < nb; t += nt) {
    n0 += __ldcg(partials + t);
    n1 += __ldcg(partials + nb + t);
  }
  n0 = block_sum(n0);
  __syncthreads();
  n1 = block_sum(n1);
  if (t0) {
    omega[0] = n1 > 0.0 ? n0 / n1 : 1.0;
    count[0] = 0u;
  }
}

// e *= omega over a whole node array
template <typename T>
__global__ void k_scale_by(T *__restrict__ e, long long n, const double *__restrict__ w) {
  MG_PDL_WAIT();
  const T f = (T)w[0];
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    e[t] *= f;
}

// relres = sqrt(sq) / sqrt(bsq), recorded in the device history
__global__ void k_relres(const double *sq, const double *bsq, double *hist, int it, double *out) {
  MG_PDL_WAIT();
  double rel = sqrt(sq[0]) / sqrt(bsq[0]);
  out[0] = rel;
  if (hist) hist[it] = rel;
}

// ---------------------------------------------------------------------------------------
// mixed precision: r32 = (float)(b - A x) with the defect in FP64, plus norm partials;
// refinement update x += (double)c
// ---------------------------------------------------------------------------------------
// The defect is FP64-pipe bound on this GPU (5 DFMA per unknown for the 5-point stencil):
// the R rows of a thread are a compile-time count (RT > 0) where it can be, so their FMA
// chains interleave, and the norm is summed on the FP32 pipe -- squares of the FP32 result,
// block sums of ~10^3 terms in FP32 (relative error ~1e-6), one FP64 partial per block
// summed in FP64 -- since it only drives the stopping test.
template <int DIM, int KIND, int RT>
__global__ void __launch_bounds__(BX *BY) k_defect64_to32(Lev<double> L, const double *__restrict__ x,
                                                          const double *__restrict__ b, float *__restrict__ r32,
                                                          long long pitch32, long long plane32,
                                                          double *__restrict__ partials, int Rrt) {
  MG_PDL_WAIT();
  const int R = RT > 0 ? RT : Rrt;
  int i = 1 + blockIdx.x * BX + threadIdx.x;
  long long r0 = ((long long)blockIdx.y * BY + threadIdx.y) * R;
  long long nr = L.unk_rows();
  float acc = 0.f;
  if (i <= L.n0 - 2) {
#pragma unroll
    for (int q = 0; q < R; ++q) {
      long long r = r0 + q;
      if (r < nr) {
        int j, k;
        row_jk(L, r, j, k);
        long long p = (long long)k * L.plane + (long long)j * L.pitch + i, dm, dp;
        yoffs(L, j, dm, dp);
        if (!MG_CK(L, p)) continue;
        Weights<double, DIM, KIND> w;
        w.load(L, i, p, dm);
        double s = residual_at<double, DIM, KIND>(L, w, x, p, dm, dp, b[p]);
        float s32 = (float)s;
        const long long p32 = (long long)k * plane32 + (long long)j * pitch32 + i;
        if (!MG_CKN(L, p32, plane32 * (L.dim == 3 ? L.n2 : 1))) continue;
        r32[p32] = s32;
        acc = fmaf(s32, s32, acc);
      }
    }
  }
  double bs = (double)block_sum_f(acc);
  if (threadIdx.x == 0 && threadIdx.y == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = bs;
}

template <int RT>
__global__ void __launch_bounds__(BX *BY) k_ir_update(Lev<double> L, double *__restrict__ x, const float *__restrict__ c,
                                                      long long pitch32, long long plane32, int Rrt) {
  MG_PDL_WAIT();
  const int R = RT > 0 ? RT : Rrt;
  int i = 1 + blockIdx.x * BX + threadIdx.x;
  if (i > L.n0 - 2) return;
  long long r0 = ((long long)blockIdx.y * BY + threadIdx.y) * R;
  long long nr = L.unk_rows();
#pragma unroll
  for (int q = 0; q < R; ++q) {
    long long r = r0 + q;
    if (r < nr) {
      int j, k;
      row_jk(L, r, j, k);
      long long p = (long long)k * L.plane + (long long)j * L.pitch + i;
      const long long p32 = (long long)k * plane32 + (long long)j * pitch32 + i;
      if (!MG_CK(L, p) || !MG_CKN(L, p32, plane32 * (L.dim == 3 ? L.n2 : 1))) continue;
      x[p] += (double)c[p32];
    }
  }
}

// ---------------------------------------------------------------------------------------
// dL/dk for the cell field: dk_c = -sum_{edges e of cell c} (dw_e/dk_c)(u_p-u_q)(l_p-l_q)
// (2-D: 4 edges with dw/dk = 1/(2h^2); 3-D: 12 edges with dw/dk = 1/(4h^2))
// ---------------------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(BX *BY) k_grad_k(Lev<double> L, const double *__restrict__ u,
                                                   const double *__restrict__ lam, double *__restrict__ dk, int R) {
  MG_PDL_WAIT();
  int i = blockIdx.x * BX + threadIdx.x;   // cell x index 0 .. n0-2
  if (i > L.n0 - 2) return;
  int ncy = L.per ? L.n1 : L.n1 - 1, ncz = DIM == 3 ? L.n2 - 1 : 1;
  long long nrows = (long long)ncy * ncz;
  long long r0 = ((long long)blockIdx.y * BY + threadIdx.y) * R;
  for (int q = 0; q < R; ++q) {
    long long r = r0 + q;
    if (r >= nrows) return;
    int j = (int)(r % ncy), k = (int)(r / ncy);
    long long p = (long long)k * L.plane + (long long)j * L.pitch + i;
    long long up = (L.per && j == L.n1 - 1) ? -(long long)(L.n1 - 1) * L.pitch : L.pitch;
    // the cell's far corner (and, for the periodic wrap, the row it wraps to)
    if (!MG_CK(L, p) || !MG_CK(L, p + up + 1 + (DIM == 3 ? L.plane : 0))) continue;
    if (DIM == 2) {
      double u00 = u[p], u10 = u[p + 1], u01 = u[p + up], u11 = u[p + up + 1];
      double l00 = lam[p], l10 = lam[p + 1], l01 = lam[p + up], l11 = lam[p + up + 1];
      double sx = (u00 - u10) * (l00 - l10) + (u01 - u11) * (l01 - l11);
      double sy = (u00 - u01) * (l00 - l01) + (u10 - u11) * (l10 - l11);
      dk[p] = -(L.ax * sx + L.ay * sy);
    } else {
      double sx = 0.0, sy = 0.0, sz = 0.0;
      for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b) {
          long long q0 = p + c * L.plane + b * up;   // x-edges at (j+b, k+c)
          sx += (u[q0] - u[q0 + 1]) * (lam[q0] - lam[q0 + 1]);
          long long q1 = p + c * L.plane + b;        // y-edges at (i+b, k+c)
          sy += (u[q1] - u[q1 + up]) * (lam[q1] - lam[q1 + up]);
          long long q2 = p + c * up + b;             // z-edges at (i+b, j+c)
          sz += (u[q2] - u[q2 + L.plane]) * (lam[q2] - lam[q2 + L.plane]);
        }
      dk[p] = -(L.ax * sx + L.ay * sy + L.az * sz);
    }
  }
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------
#define DISPATCH_DK(DIMV, KINDV, KERNEL, ...)                                  \
  do {                                                                         \
    if ((DIMV) == 2) {                                                         \
      if ((KINDV) == K_CONST) KERNEL<T, 2, K_CONST> __VA_ARGS__;               \
      else if ((KINDV) == K_SEP) KERNEL<T, 2, K_SEP> __VA_ARGS__;              \
      else if ((KINDV) == K_CELL) KERNEL<T, 2, K_CELL> __VA_ARGS__;            \
      else KERNEL<T, 2, K_EDGE> __VA_ARGS__;                                   \
    } else {                                                                   \
      if ((KINDV) == K_CONST) KERNEL<T, 3, K_CONST> __VA_ARGS__;               \
      else if ((KINDV) == K_SEP) KERNEL<T, 3, K_SEP> __VA_ARGS__;              \
      else if ((KINDV) == K_CELL) KERNEL<T, 3, K_CELL> __VA_ARGS__;            \
      else KERNEL<T, 3, K_EDGE> __VA_ARGS__;                                   \
    }                                                                          \
  } while (0)

// the same, with the 2-D Galerkin (9-point) levels: for the kernels that run on every kind of level
#define DISPATCH_DK9(DIMV, KINDV, KERNEL, ...)                                 \
  do {                                                                         \
    if ((DIMV) == 2 && (KINDV) == K_NINE) KERNEL<T, 2, K_NINE> __VA_ARGS__;    \
    else DISPATCH_DK(DIMV, KINDV, KERNEL, __VA_ARGS__);                        \
  } while (0)

template <typename T>
void launch_jacobi(const Launch &lc, const Lev<T> &L, int kind, const T *u, const T *g, T *out, T omega) {
  long long rows = L.unk_rows();
  int R = rows_per_thread(rows);
  dim3 gr = grid_for(L.xunk(), rows, R), bl(BX, BY);
  DISPATCH_DK9(L.dim, kind, k_jacobi, <<<gr, bl, 0, lc.s>>>(L, u, g, out, omega, R));
  lc.done(__func__);
}

template <typename T>
void launch_jacobi_zero(const Lev<T> &L, int kind, const Launch &lc, const T *g, T *out, T omega) {
  long long rows = L.unk_rows();
  int R = rows_per_thread(rows);
  dim3 gr = grid_for(L.xunk(), rows, R), bl(BX, BY);
  DISPATCH_DK9(L.dim, kind, k_jacobi_zero, <<<gr, bl, 0, lc.s>>>(L, g, out, omega, R));
  lc.done(__func__);
}

template <typename T>
void launch_rb_half(const Launch &lc, const Lev<T> &L, int kind, T *u, const T *g, T omega, int colour) {
  long long rows = L.unk_rows();
  int R = rows_per_thread(rows);
  dim3 gr = grid_for((L.xunk() + 1) / 2, rows, R), bl(BX, BY);
  DISPATCH_DK(L.dim, kind, k_rb_half, <<<gr, bl, 0, lc.s>>>(L, u, g, omega, colour, R));
  lc.done(__func__);
}

template <typename T>
void launch_gs9_colour(const Launch &lc, const Lev<T> &L, T *u, const T *g, T omega, int ci, int cj) {
  const int jlo = cj ? 1 : 2;
  const long long rows = L.n1 - 2 >= jlo ? (L.n1 - 2 - jlo) / 2 + 1 : 0;
  const long long xs = L.n0 - 2 >= (ci ? 1 : 2) ? (L.n0 - 2 - (ci ? 1 : 2)) / 2 + 1 : 0;
  if (rows <= 0 || xs <= 0) return;
  int R = rows_per_thread(rows);
  dim3 gr = grid_for(xs, rows, R), bl(BX, BY);
  k_gs9_colour<T><<<gr, bl, 0, lc.s>>>(L, u, g, omega, ci, cj, R);
  lc.done(__func__);
}

template <typename T>
void launch_defect(const Launch &lc, const Lev<T> &L, int kind, const T *u, const T *g, T *r) {
  long long rows = L.unk_rows();
  int R = rows_per_thread(rows);
  dim3 gr = grid_for(L.xunk(), rows, R), bl(BX, BY);
  DISPATCH_DK9(L.dim, kind, k_defect, <<<gr, bl, 0, lc.s>>>(L, u, g, r, R));
  lc.done(__func__);
}

// Rows per thread of a reduction over `rows` unknown rows of `xthreads` unknowns each, such that
// its blocks (one partial sum each) number at most nparts and gridDim.y stays within 65535.
// -1 when no R fits: the rows are wider than BX * nparts unknowns (norm_shape_ok is false).
static inline int norm_R(long long rows, long long xthreads, int nparts) {
  const long long gx = (xthreads + BX - 1) / BX;
  if (gx < 1 || gx > nparts) return -1;
  long long gy_max = nparts / gx;
  if (gy_max > 65535) gy_max = 65535;
  const long long per = (long long)BY * gy_max;               // rows covered per unit of R
  long long R = (rows + per - 1) / per;
  const long long R0 = rows_per_thread(rows);
  if (R < R0) R = R0;
  return (int)R;   // rows < 2^35 (set-up's node limit) and per >= 8: R < 2^32 / 2
}

bool norm_shape_ok(long long xunknowns, int nparts) { return (xunknowns + BX - 1) / BX <= nparts; }

int norm_parts_count() { return 65536; }

template <typename T>
void launch_defect_norm(const Launch &lc, const Lev<T> &L, int kind, const T *u, const T *g, double *partials,
                        int nparts, double *out_sq) {
  long long rows = L.unk_rows();
  int R = norm_R(rows, L.xunk(), nparts);
  dim3 gr = grid_for(L.xunk(), rows, R), bl(BX, BY);
  DISPATCH_DK9(L.dim, kind, k_defect_norm, <<<gr, bl, 0, lc.s>>>(L, u, g, partials, R));
  lc.done(__func__);
  launch_norm_finish(lc, partials, (int)(gr.x * gr.y), out_sq);
}

template <typename T>
void launch_norm_parts(const Launch &lc, const Lev<T> &L, const T *v, double *partials, int nparts, double *out_sq) {
  long long rows = L.unk_rows();
  int R = norm_R(rows, L.xunk(), nparts);
  dim3 gr = grid_for(L.xunk(), rows, R), bl(BX, BY);
  k_norm_parts<T><<<gr, bl, 0, lc.s>>>(L, v, partials, R);
  lc.done(__func__);
  launch_norm_finish(lc, partials, (int)(gr.x * gr.y), out_sq);
}

template <typename T>
void launch_corr_weight(const Launch &lc, const Lev<T> &L, int kind, const T *u, const T *g, const T *pe,
                        double *partials, int nparts, unsigned *count, double *omega) {
  long long rows = L.unk_rows();
  int R = norm_R(rows, L.xunk(), nparts / 2 < 4096 ? nparts / 2 : 4096);
  dim3 gr = grid_for(L.xunk(), rows, R), bl(BX, BY);
  DISPATCH_DK(L.dim, kind, k_corr_dots, <<<gr, bl, 0, lc.s>>>(L, u, g, pe, partials, count, omega, R));
  lc.done(__func__);
}

template <typename T>
void launch_scale_by(const Launch &lc, T *e, long long n, const double *omega) {
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_scale_by<T><<<(unsigned)blocks, 256, 0, lc.s>>>(e, n, omega);
  lc.done(__func__);
}

void launch_norm_finish(const Launch &lc, const double *partials, int nparts, double *out_sq) {
  k_norm_finish<<<1, 1024, 0, lc.s>>>(partials, nparts, out_sq);
  lc.done(__func__);
}

// End of a cycle inside a device-side solve loop (a CUDA-graph WHILE node): record the
// relative residual, count the cycle and set the loop condition.  st[0] = cycles done,
// st[1] = status (0 running / converged, 4 no convergence, 5 non-finite, 6 a bounded
// device wait gave up), st[2] = set by a kernel whose wait gave up, st[6] = the loop's outer
// defect runs in FP64 (set here, see below).  init = 1 for the check before the first cycle.
// ||b|| = 0 stops at once (x = 0); a non-finite ||b|| gives a non-finite relative residual.
// tsq (float-float outer defect, st[6] clear): the defect's error is estimated as
// E = ff_err * sqrt(tsq) / ||b|| relative to ||b||; the loop stops when the residual plus E is
// within tol, and sets st[6] (FP64 defects from the next step on) when E is half of tol or more
// (the float-float residual could never decide), when the residual is within ff_switch * E of
// tol, or when it fell by less than half in the step: near the defect's error the FP32 cycle
// is driven by that error, whose smooth part it amplifies, and the loop stalls.
__global__ void k_step_end(cudaGraphConditionalHandle h, const double *sq, const double *bsq, double *hist, int *st,
                           const double *tol, int maxit, int init, const double *tsq, double ff_err,
                           double ff_switch) {
  MG_PDL_WAIT();
  double b = bsq[0];
  double rel = b == 0.0 ? 0.0 : sqrt(sq[0]) / sqrt(b);
  int it = init ? 0 : st[0] + 1;
  st[0] = it;
  if (hist) hist[it] = rel;
  int go = 1, status = 0;
  const double err = (tsq && !st[6] && b != 0.0) ? ff_err * sqrt(tsq[0]) / sqrt(b) : 0.0;
  if (st[2]) {
    go = 0;
    status = 6;
  } else if (!(rel == rel) || rel > 1.7976931348623157e308) {
    go = 0;
    status = 5;
  } else if (rel + err <= tol[0] || b == 0.0) {
    go = 0;
  } else {
    if (err > 0.0 && (err >= 0.5 * tol[0] || rel <= tol[0] + ff_switch * err ||
                      (it >= 2 && hist && rel > 0.5 * hist[it - 1])))
      st[6] = 1;
    if (it >= maxit) {
      go = 0;
      status = 4;
    }
  }
  st[1] = status;
  cudaGraphSetConditional(h, go ? 1u : 0u);
}
void launch_step_end(const Launch &lc, cudaGraphConditionalHandle h, const double *sq, const double *bsq,
                     double *hist, int *st, const double *tol, int maxit, int init, const double *tsq,
                     double ff_err, double ff_switch) {
  k_step_end<<<1, 1, 0, lc.s>>>(h, sq, bsq, hist, st, tol, maxit, init, tsq, ff_err, ff_switch);
  lc.done(__func__);
}

// After a loop that stopped on the float-float defect: the FP64 relative residual replaces
// the last entry of the history; a loop that stopped as converged but is not (beyond tol in
// FP64) gets status 8, which the host resolves by continuing the iteration.
__global__ void k_final_check(const double *sq, const double *bsq, double *hist, int *st, const double *tol) {
  MG_PDL_WAIT();
  const double b = bsq[0];
  const double rel = b == 0.0 ? 0.0 : sqrt(sq[0]) / sqrt(b);
  if (hist) hist[st[0]] = rel;
  if (st[1] == 0 && b != 0.0 && !(rel <= tol[0])) st[1] = 8;
}
void launch_final_check(const Launch &lc, const double *sq, const double *bsq, double *hist, int *st,
                        const double *tol) {
  k_final_check<<<1, 1, 0, lc.s>>>(sq, bsq, hist, st, tol);
  lc.done(__func__);
}

// Test hook of the -DMG_DEBUG build (MG_FLAG_TEST_BOUNDS): one bounds check of the index one past
// the level's last node, which fails and is recorded; nothing is read or written there.
__global__ void k_bounds_probe(Lev<double> L) {
  MG_PDL_WAIT();
  if (!MG_CK(L, L.plane * (L.dim == 3 ? L.n2 : 1))) return;
}
void launch_bounds_probe(const Launch &lc, const Lev<double> &L) {
  k_bounds_probe<<<1, 1, 0, lc.s>>>(L);
  lc.done(__func__);
}

__global__ void k_sqrt(const double *src, double *dst) {
  MG_PDL_WAIT();
  dst[0] = sqrt(src[0]);
}
void launch_sqrt(const Launch &lc, const double *src, double *dst) {
  k_sqrt<<<1, 1, 0, lc.s>>>(src, dst);
  lc.done(__func__);
}

void launch_relres(const Launch &lc, const double *sq, const double *bsq, double *hist, int it, double *relres_out) {
  k_relres<<<1, 1, 0, lc.s>>>(sq, bsq, hist, it, relres_out);
  lc.done(__func__);
}

void launch_defect64_to32(const Launch &lc, const Lev<double> &L, int kind, const double *x, const double *b,
                          float *r32, double *partials, int nparts, double *out_sq) {
  long long rows = L.unk_rows();
  int R = norm_R(rows, L.xunk(), nparts);
  dim3 gr = grid_for(L.xunk(), rows, R), bl(BX, BY);
  long long p32 = L.pitch, pl32 = L.plane;   // the FP32 finest level uses the same element pitch
#define D64_R(D, K)                                                                                          \
  do {                                                                                                       \
    if (R == 4) k_defect64_to32<D, K, 4><<<gr, bl, 0, lc.s>>>(L, x, b, r32, p32, pl32, partials, R);         \
    else if (R == 1) k_defect64_to32<D, K, 1><<<gr, bl, 0, lc.s>>>(L, x, b, r32, p32, pl32, partials, R);    \
    else k_defect64_to32<D, K, 0><<<gr, bl, 0, lc.s>>>(L, x, b, r32, p32, pl32, partials, R);                \
  } while (0)
  if (L.dim == 2) {
    if (kind == K_CONST) D64_R(2, K_CONST);
    else if (kind == K_SEP) D64_R(2, K_SEP);
    else if (kind == K_CELL) D64_R(2, K_CELL);
    else D64_R(2, K_EDGE);
  } else {
    if (kind == K_CONST) D64_R(3, K_CONST);
    else if (kind == K_SEP) D64_R(3, K_SEP);
    else if (kind == K_CELL) D64_R(3, K_CELL);
    else D64_R(3, K_EDGE);
  }
#undef D64_R
  lc.done(__func__);
  launch_norm_finish(lc, partials, (int)(gr.x * gr.y), out_sq);
}

void launch_ir_update(const Launch &lc, const Lev<double> &L, double *x, const float *c) {
  long long rows = L.unk_rows();
  int R = rows_per_thread(rows);
  dim3 gr = grid_for(L.xunk(), rows, R), bl(BX, BY);
  if (R == 4) k_ir_update<4><<<gr, bl, 0, lc.s>>>(L, x, c, L.pitch, L.plane, R);
  else k_ir_update<0><<<gr, bl, 0, lc.s>>>(L, x, c, L.pitch, L.plane, R);
  lc.done(__func__);
}

void launch_grad_k(const Launch &lc, const Lev<double> &L, const double *u, const double *lam, double *dk) {
  int ncy = L.per ? L.n1 : L.n1 - 1, ncz = L.dim == 3 ? L.n2 - 1 : 1;
  long long rows = (long long)ncy * ncz;
  int R = rows_per_thread(rows);
  dim3 gr = grid_for(L.n0 - 1, rows, R), bl(BX, BY);
  if (L.dim == 2) k_grad_k<2><<<gr, bl, 0, lc.s>>>(L, u, lam, dk, R);
  else k_grad_k<3><<<gr, bl, 0, lc.s>>>(L, u, lam, dk, R);
  lc.done(__func__);
}

#define INST(T)                                                                                              \
  template void launch_jacobi<T>(const Launch &, const Lev<T> &, int, const T *, const T *, T *, T);         \
  template void launch_jacobi_zero<T>(const Lev<T> &, int, const Launch &, const T *, T *, T);              \
  template void launch_rb_half<T>(const Launch &, const Lev<T> &, int, T *, const T *, T, int);             \
  template void launch_gs9_colour<T>(const Launch &, const Lev<T> &, T *, const T *, T, int, int);          \
  template void launch_defect<T>(const Launch &, const Lev<T> &, int, const T *, const T *, T *);           \
  template void launch_defect_norm<T>(const Launch &, const Lev<T> &, int, const T *, const T *, double *, int, \
                                      double *);                                                              \
  template void launch_norm_parts<T>(const Launch &, const Lev<T> &, const T *, double *, int, double *);      \
  template void launch_corr_weight<T>(const Launch &, const Lev<T> &, int, const T *, const T *, const T *,    \
                                      double *, int, unsigned *, double *);                                   \
  template void launch_scale_by<T>(const Launch &, T *, long long, const double *);
INST(double)
INST(float)

}  // namespace mg
