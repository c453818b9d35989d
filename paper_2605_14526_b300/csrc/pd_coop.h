// Cooperative launch of the persistent kernels through cudaLaunchKernelEx
// with the cooperative attribute, which (unlike cudaLaunchCooperativeKernel)
// can be captured into a CUDA graph.
#pragma once
#include <cuda_runtime.h>

#include <utility>

#include "pd_internal.h"

namespace pdk {

template <typename... K, typename... A>
inline cudaError_t coop_launch(void (*fn)(K...), int grid, int block, size_t smem, cudaStream_t s, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fn, std::forward<A>(args)...);
}

}  // namespace pdk
