// internal.h -- host-side helpers shared by the translation units of
// libmppi_jump.so (configuration checks, device-problem packing, launch
// geometry).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/mppi_jump.h"
#include "device.cuh"

namespace mj {

// Set a message into buf (size >= 256) and return st.
mppi_status fail(char* buf, mppi_status st, const char* fmt, ...);

// Validate cfg; on success fill the packed device problem (thresholds,
// reciprocals, Philox key).  msg receives a reason on failure.
mppi_status pack_problem(const mppi_jump_config* cfg, DevProblem* P, char* msg);

inline int state_dim(int system) { return system == MPPI_CARTPOLE ? 4 : 12; }
inline int control_dim(int system) { return system == MPPI_CARTPOLE ? 1 : 4; }
inline int pad_k(int K) { return (K + 31) / 32 * 32; }
inline size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Launch geometry of the split-K update for one problem.
struct UpdateGeom {
  int vpt;     // 16-byte vectors per thread
  int chunks;  // blocks along K
  int rows;    // steps per block
  int groups;  // blocks along T
};
UpdateGeom update_geometry(int Kpad, int T, int m, bool bf16, int num_sms);

// Per-process kernel attributes (dynamic shared memory limits); call on the
// current device before the first launch or stream capture.
cudaError_t prepare_kernels();

// Enqueue the kernels of one iteration for a single problem.  it_ptr and the
// other pointers are device pointers; shift != 0 performs the MPC shift and
// writes u0 (if not NULL) after the update.
struct IterBuffers {
  const float* x0;
  float* U;
  void* noise;
  float* s_part;
  float* w;
  float* partial;
  float* cconst;
  float* diag;
  int* status;
  uint32_t* it;
  float* costs;        // may be NULL
  uint8_t* dbg_counts; // may be NULL
  float* dbg_J;        // may be NULL
};
cudaError_t launch_rollout(const DevProblem& P, const IterBuffers& b, cudaStream_t s);
cudaError_t launch_weights_update(const DevProblem& P, const IterBuffers& b, const UpdateGeom& g,
                                  int shift, float* u0, cudaStream_t s);

}  // namespace mj
