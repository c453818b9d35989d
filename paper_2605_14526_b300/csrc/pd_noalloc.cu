// pd_solve_noalloc: x = A^-1 b through the same two sparse products as
// pd_solve, for callers that must not allocate device memory while they run.
//
// Such callers exist: code running under a CUDA-graph stream capture or inside
// a real-time control loop, hosts embedding the library in a process whose
// device memory is owned by another allocator (a framework's caching pool or a
// fixed arena that the library must not grow), and callers that cannot take
// the implicit synchronisation of cudaMalloc/cudaFree. pd_solve needs two
// [n_f][3] work vectors; they come from the context, which the caller may not
// be able to size for this purpose. Here they live in one file-scope device
// array of fixed size, which every GPU that loads the library holds until the
// process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/pd_b300.h"
#include "pd_internal.h"
#include "pd_launch.h"
#include "pd_noalloc.h"

namespace {

// Largest number of free (unpinned) vertices pd_solve_noalloc accepts.
constexpr int kNoAllocMaxFree = PD_NOALLOC_MAX_FREE;

// [0, 3*kNoAllocMaxFree): right-hand side in elimination order;
// [3*kNoAllocMaxFree, 6*kNoAllocMaxFree): the accumulator of S b.
// 2 * 3 * 65536 doubles = 3 MiB.
static __device__ __align__(256) double g_solve_scratch[2 * 3 * kNoAllocMaxFree];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_solve_scratch on the current device (looked up once per
// device: in host code the symbol's name is only a host-side stand-in).
cudaError_t scratch_on(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_solve_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int pd_solve_noalloc(pd_ctx* ctx, const double* b, double* x, void* stream) {
  if (!ctx) return PD_ERR_ARG;
  const pdk::Dev* d = nullptr;
  int device = 0, factored = 0;
  pd_internal_state(ctx, &d, &device, &factored);
  if (!d) {
    pd_internal_set_error(ctx, "pd_solve_noalloc is single-instance only");
    return PD_ERR_ARG;
  }
  if (d->tmode) {
    pd_internal_set_error(ctx, "pd_solve_noalloc applies the inverse factor S; this context factored for solve "
                               "mode T (use pd_solve, or solve_mode = PD_SOLVE_S)");
    return PD_ERR_ARG;
  }
  if (d->n_f > kNoAllocMaxFree) {
    pd_internal_set_error(ctx, "pd_solve_noalloc: the mesh has more free vertices than the fixed scratch holds "
                               "(limit PD_NOALLOC_MAX_FREE = 65536); use pd_solve");
    return PD_ERR_TOO_LARGE;
  }
  if (!factored) {
    pd_internal_set_error(ctx, "pd_factor must run before pd_solve_noalloc");
    return PD_ERR_NOT_FACTORED;
  }
  if (!b || !x) {
    pd_internal_set_error(ctx, "b and x are required");
    return PD_ERR_ARG;
  }
  cudaError_t e = cudaSetDevice(device);
  double* scratch = nullptr;
  if (e == cudaSuccess) e = scratch_on(device, &scratch);
  if (e != cudaSuccess) {
    pd_internal_set_error(ctx, cudaGetErrorString(e));
    return PD_ERR_CUDA;
  }
  float2* xs = reinterpret_cast<float2*>(scratch);   // double-float pairs, 8 bytes like a double
  pdk::launch_solve(*d, static_cast<cudaStream_t>(stream), b, xs, xs + 3 * (size_t)kNoAllocMaxFree, d->s_part_na,
                    d->s_cnt_na, x);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    pd_internal_set_error(ctx, cudaGetErrorString(e));
    return PD_ERR_CUDA;
  }
  return PD_OK;
}
