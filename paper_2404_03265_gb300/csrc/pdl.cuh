// Programmatic dependent launch (PTX griddepcontrol) for chains of dependent
// kernels on one stream, also under stream capture into CUDA graphs.
//
// A kernel launched with launch_ex(true, ...) may be scheduled before the
// kernel launched before it on the stream has finished, as soon as every block
// of that kernel has called pdl_trigger() (or exited).  It must call pdl_wait()
// before it reads what that kernel wrote or writes what that kernel reads:
// pdl_wait() returns once that kernel has completed and its writes are visible.
// For a kernel launched without the dependency both calls do nothing.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace pff {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// Launch of kernel `fn` on stream s, programmatically dependent on the launch
// before it in the stream when pdl is set.
template <typename... KArgs, typename... Args>
cudaError_t launch_ex(bool pdl, void (*fn)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                      Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, fn, std::forward<Args>(args)...);
}

}  // namespace pff
