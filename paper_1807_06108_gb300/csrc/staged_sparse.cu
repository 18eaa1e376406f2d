// staged_sparse.cu -- the staged rollout with sparse state-jump records
// (jump masks; the producer warp gathers the records of the jumping steps).
#include "staged_launch.cuh"

namespace mj {

cudaError_t prepare_staged_sparse() {
  cudaError_t e = allow_staged_smem_jm<kJumpDefaultSparse>();
  if (e == cudaSuccess) e = allow_staged_smem_jm<kJumpRowsSparse>();
  return e;
}

void launch_staged_sparse(const StagedLaunch& L, bool velocity_rows) {
  if (velocity_rows) launch_staged_jm<kJumpDefaultSparse>(L);
  else launch_staged_jm<kJumpRowsSparse>(L);
}

}  // namespace mj
