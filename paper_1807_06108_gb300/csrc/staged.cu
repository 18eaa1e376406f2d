// staged.cu -- the staged rollout without jumps in its step data (control-
// channel jumps are folded into delta_eff) and with dense state-jump records.
#include "staged_launch.cuh"

namespace mj {

cudaError_t prepare_staged_dense() {
  cudaError_t e = allow_staged_smem_jm<kJumpNone>();
  if (e == cudaSuccess) e = allow_staged_smem_jm<kJumpDefault>();
  if (e == cudaSuccess) e = allow_staged_smem_jm<kJumpRows>();
  return e;
}

void launch_staged_dense(const StagedLaunch& L, int jump_mode) {
  if (jump_mode == kJumpNone) launch_staged_jm<kJumpNone>(L);
  else if (jump_mode == kJumpDefault) launch_staged_jm<kJumpDefault>(L);
  else launch_staged_jm<kJumpRows>(L);
}

}  // namespace mj
