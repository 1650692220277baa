// noalloc.cu -- residual norm that needs no workspace at all.
//
// mg_residual_norm (mg_capi.cu) keeps its per-block partial sums in the caller's
// workspace, which a caller has to allocate before it can create a context.  Some
// callers cannot allocate device memory at the point where they want a residual:
// code whose device memory is owned entirely by another allocator or a fixed
// budget, or code running while its stream is being captured, where a cudaMalloc
// is not allowed.  mg_residual_norm_noalloc gives them the same defect-norm
// kernels with the partial sums in a file-scope __device__ array instead: nothing
// is allocated by the call, the caller only passes its inputs and output.
#include <cstring>
#include <mutex>

#include "../../include/mg.h"
#define MG_FILE_ID 9   // bounds-check sites (-DMG_DEBUG)
#include "mg_internal.cuh"

using namespace mg;

namespace {
// Partial sums of the block reduction plus the finished sum.  Every loaded copy of
// the library holds this array on every GPU it touches until the process exits.
constexpr int kNoallocParts = 65536;
static __device__ __align__(256) double g_noalloc_scratch[kNoallocParts + 32];

// Device address of g_noalloc_scratch per device.  In host code the symbol is only a
// host-side stand-in, so the real address is queried once per device, with that
// device current, and handed to the kernels.
constexpr int kMaxDevices = 256;
double *g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

mg_status scratch_for_current_device(double **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return MG_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    double *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      cudaGetLastError();
      return MG_ECUDA;
    }
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return MG_OK;
}
}  // namespace

extern "C" mg_status mg_residual_norm_noalloc(const mg_params *p, const mg_coeffs *k, const double *u,
                                             const double *b, double *out) {
  if (!p || !k || !u || !b || !out) return MG_EINVAL;
  if (p->dim != 2 && p->dim != 3) return MG_EINVAL;
  if (k->kind != MG_COEF_CONST && k->kind != MG_COEF_SEPARABLE) return MG_EINVAL;
  if (k->kind == MG_COEF_SEPARABLE && (!k->sx || !k->sy || (p->dim == 3 && !k->sz))) return MG_EINVAL;
  int n0 = p->n[0], n1 = p->n[1], n2 = p->dim == 3 ? p->n[2] : 1;
  if (n0 < 3 || n1 < (p->periodic_y ? 2 : 3) || (p->dim == 3 && n2 < 3)) return MG_EINVAL;
  if (p->periodic_y && (n1 % 2)) return MG_EINVAL;
  if ((long long)n0 * n1 * n2 > MG_NOALLOC_MAX_NODES) return MG_EINVAL;
  // one partial sum per block of 32 x-unknowns (at least) must fit in the array
  if (!norm_shape_ok(n0 - 2, kNoallocParts)) return MG_EINVAL;
  double *scratch = nullptr;
  mg_status st = scratch_for_current_device(&scratch);
  if (st) return st;

  // the caller's compact arrays are read in place: pitch = n0
  Lev<double> L;
  memset(&L, 0, sizeof(L));
  L.dim = p->dim;
  L.n0 = n0;
  L.n1 = n1;
  L.n2 = n2;
  L.per = p->periodic_y ? 1 : 0;
  L.pitch = n0;
  L.plane = (long long)n0 * n1;
  if (k->kind == MG_COEF_CONST) {
    L.cx = k->c[0];
    L.cy = k->c[1];
    L.cz = p->dim == 3 ? k->c[2] : 0.0;
    L.d = 2.0 * (L.cx + L.cy + L.cz);
    L.dinv = 1.0 / L.d;
  } else {
    L.sx = k->sx;
    L.sy = k->sy;
    L.sz = p->dim == 3 ? k->sz : k->sy;
    L.sdinv = k->sy;   // the defect does not use 1/D; any array of length n0 keeps the load in bounds
  }
  long long launches = 0;
  Launch lc{(cudaStream_t)p->stream, &launches};
  // every partial the finish step reads is written by this call's reduction, and the
  // finished sum is overwritten: nothing in the shared array has to be cleared
  launch_defect_norm<double>(lc, L, k->kind, u, b, scratch, kNoallocParts, scratch + kNoallocParts);
  launch_sqrt(lc, scratch + kNoallocParts, out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MG_OK : MG_ECUDA;
}
