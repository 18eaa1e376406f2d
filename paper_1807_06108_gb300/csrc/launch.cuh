// launch.cuh -- the high-priority (and optionally programmatic-dependent)
// kernel launch shared by the translation units that launch rollouts.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace mj {

// The greatest stream priority of the device (launch attribute), so that a
// rollout's blocks are scheduled ahead of a concurrent noise pass.
inline int high_priority() {
  static int prio = [] {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return 0;
    return greatest;
  }();
  return prio;
}

template <class... Params, class... Args>
void launch_hi(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
               Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributePriority;
  attr[0].val.priority = high_priority();
  // a programmatic dependent of the previous kernel in the stream: it may be
  // scheduled once that kernel's blocks have all started, and waits in
  // griddep_wait() for its completion before touching what it wrote
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 2 : 1;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace mj
