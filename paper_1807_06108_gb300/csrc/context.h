// context.h -- the single-problem context behind the C ABI (shared by api.cu
// and step.cu).  Not part of the public ABI.
#pragma once

#include <cstdio>
#include <map>
#include <vector>

#include "internal.h"

struct mppi_jump_ctx {
  mppi_jump_config cfg;
  mj::DevProblem P;
  mj::UpdateGeom geom;
  mj::RolloutTile tile;
  cudaStream_t stream = nullptr;  // every call enqueues here
  cudaStream_t aux = nullptr;     // second branch of the captured step (noise prefetch)
  cudaStream_t aux2 = nullptr;    // third branch (marks passes of sparse jump records)
  bool own_stream = false;
  int device = 0;
  // one device allocation carved into the buffers below
  void* arena = nullptr;
  size_t arena_bytes = 0;
  float* x0 = nullptr;          // [n]
  float* U = nullptr;           // [T][m]
  void* noise[2] = {};          // two sets of [T][Kpad][m] delta_eff (f32 or bf16)
  uint32_t* jmask[2] = {};      // [Kpad/32][mask_cols(T)] jump masks (state jumps)
  float4* jrec[2] = {};         // [T][Kpad] jump records (state jumps)
  float* s_part = nullptr;      // [Kpad]
  float* rec = nullptr;         // [ceil(Kpad/32)][2 + T*m] partial records of the rollout blocks
  float* partial = nullptr;     // [max_chunks][T][m]
  int max_chunks = 0;
  float* zpart = nullptr;       // [groups][max_chunks]
  float* gpart = nullptr;       // [groups][m] edge values, [groups] control costs
  float* scal = nullptr;        // cconst, diag[4] (rho~, Z, F, rho)
  int* status = nullptr;        // device status word
  uint32_t* it = nullptr;       // iteration counter
  uint32_t* rho_key = nullptr;  // running cost minimum
  unsigned* done = nullptr;     // update completion ticket, then [groups] group tickets
  float* u0 = nullptr;          // [m]
  // pinned host staging for the synchronous step
  float* h_x0 = nullptr;
  float* h_u0 = nullptr;
  int* h_status = nullptr;
  uint8_t* dbg_counts = nullptr;
  float* dbg_J = nullptr;
  int last_set = 0;  // buffer set holding the last iteration's noise
  std::map<int, cudaGraphExec_t> graphs;
  std::vector<cudaEvent_t> links;  // fork/join events used while capturing
  // phase timing: events recorded inside the captured step
  bool timing = false;
  std::vector<cudaEvent_t> events;  // 3 per iteration: before rollout, after, after update
  int timed_iters = 0;              // iterations covered by the last timed step
  char err[256] = {0};
};

namespace mj {

mppi_status cuda_fail(mppi_jump_ctx* ctx, cudaError_t e, const char* what);
IterBuffers ctx_buffers(mppi_jump_ctx* ctx, float* costs, int set);
void drop_graphs(mppi_jump_ctx* ctx);

}  // namespace mj

#define CK(call, what)                                          \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return mj::cuda_fail(ctx, e_, what); \
  } while (0)
