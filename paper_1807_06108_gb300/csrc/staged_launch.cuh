// staged_launch.cuh -- instantiation and launch of rollout_staged_kernel for
// one jump-record form, included by staged.cu (dense records, no jumps) and
// staged_sparse.cu (sparse records), which compile side by side.
#pragma once

#include "internal.h"
#include "kernels.cuh"
#include "launch.cuh"

namespace mj {

template <int SYS, bool BF16, int JM, bool PART>
cudaError_t allow_staged_smem() {
  cudaError_t e = cudaFuncSetAttribute(rollout_staged_kernel<SYS, BF16, 4, JM, PART>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kStagedSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(rollout_staged_kernel<SYS, BF16, 8, JM, PART>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kStagedSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(rollout_staged_kernel<SYS, BF16, 16, JM, PART>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kStagedSmemMax);
  return e;
}

// every plant, noise dtype and record source of jump mode JM
template <int JM>
cudaError_t allow_staged_smem_jm() {
  cudaError_t e = allow_staged_smem<0, false, JM, false>();
  if (e == cudaSuccess) e = allow_staged_smem<0, true, JM, false>();
  if (e == cudaSuccess) e = allow_staged_smem<1, false, JM, false>();
  if (e == cudaSuccess) e = allow_staged_smem<1, true, JM, false>();
  if (e == cudaSuccess) e = allow_staged_smem<0, false, JM, true>();
  if (e == cudaSuccess) e = allow_staged_smem<0, true, JM, true>();
  if (e == cudaSuccess) e = allow_staged_smem<1, false, JM, true>();
  if (e == cudaSuccess) e = allow_staged_smem<1, true, JM, true>();
  return e;
}

template <int SYS, bool BF16, int JM, bool PART>
void launch_staged_s(const StagedLaunch& L) {
  const DevProblem& P = *L.P;
  const IterBuffers& b = *L.b;
  const int nt = L.tile->block;
  // the masks only for the sparse forms
  const uint32_t* jmask = JM == kJumpDefaultSparse || JM == kJumpRowsSparse ? b.jmask : nullptr;
  if (L.tile->chunk == 4)
    launch_hi(rollout_staged_kernel<SYS, BF16, 4, JM, PART>, dim3(L.blocks), dim3(nt + 32), L.smem, L.s, L.pdl,
              P, b.x0, b.U, b.noise, jmask, b.jrec, b.s_part, b.rho_key, b.status, b.rec);
  else if (L.tile->chunk == 16)
    launch_hi(rollout_staged_kernel<SYS, BF16, 16, JM, PART>, dim3(L.blocks), dim3(nt + 32), L.smem, L.s,
              L.pdl, P, b.x0, b.U, b.noise, jmask, b.jrec, b.s_part, b.rho_key, b.status, b.rec);
  else
    launch_hi(rollout_staged_kernel<SYS, BF16, 8, JM, PART>, dim3(L.blocks), dim3(nt + 32), L.smem, L.s, L.pdl,
              P, b.x0, b.U, b.noise, jmask, b.jrec, b.s_part, b.rho_key, b.status, b.rec);
}

template <int JM>
void launch_staged_jm(const StagedLaunch& L) {
  const DevProblem& P = *L.P;
  switch (P.system * 4 + (P.noise_bf16 ? 2 : 0) + (L.part ? 1 : 0)) {
    case 0: launch_staged_s<0, false, JM, false>(L); break;
    case 1: launch_staged_s<0, false, JM, true>(L); break;
    case 2: launch_staged_s<0, true, JM, false>(L); break;
    case 3: launch_staged_s<0, true, JM, true>(L); break;
    case 4: launch_staged_s<1, false, JM, false>(L); break;
    case 5: launch_staged_s<1, false, JM, true>(L); break;
    case 6: launch_staged_s<1, true, JM, false>(L); break;
    default: launch_staged_s<1, true, JM, true>(L); break;
  }
}

}  // namespace mj
