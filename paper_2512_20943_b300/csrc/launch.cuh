// Programmatic stream serialisation for chains of short kernels (sm_103a).
//
// A kernel launched through launch_serialised may begin while the previous
// kernel on the stream finishes; its first act must be wait_prior_grid()
// (griddepcontrol.wait), which returns once that kernel has completed and its
// memory is visible.  Only the launch latency overlaps; the order of effects
// is that of an ordinary launch.  wait_prior_grid() is a no-op in a kernel that
// was launched ordinarily.
#pragma once
#include <cuda_runtime.h>

#include <utility>

namespace airgs {

__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
static cudaError_t launch_serialised(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                     Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace airgs
