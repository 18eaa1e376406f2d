// internal.h -- host-side helpers shared by the translation units of
// libmppi_jump.so (configuration checks, device-problem packing, launch
// geometry, kernel launches).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/mppi_jump.h"
#include "device.cuh"

#ifndef MPPI_NO_NVTX
#include <nvtx3/nvToolsExt.h>
#endif

namespace mj {

// NVTX range around a host call (shown by profilers on the CPU timeline; a
// no-op unless a profiler is attached; compiled out with MPPI_NO_NVTX).
struct NvtxRange {
#ifndef MPPI_NO_NVTX
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
#else
  explicit NvtxRange(const char*) {}
#endif
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Set a message into buf (size >= 256) and return st.
mppi_status fail(char* buf, mppi_status st, const char* fmt, ...);

// Validate cfg; on success fill the packed device problem (thresholds,
// reciprocals, Philox key).  msg receives a reason on failure.
mppi_status pack_problem(const mppi_jump_config* cfg, DevProblem* P, char* msg);

// SMs of the current device.
int num_sms_of_current();

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

// Per-process kernel attributes; call on the current device before the first
// launch or stream capture.
cudaError_t prepare_kernels();

// Rollout launch shape: variant 1 = fused (one kernel draws and rolls out),
// 2 = split (noise_kernel over K*T/4 threads, then rollout_split_kernel),
// 3 = staged (the split form with bulk copies into shared memory), 4 =
// staged, each block also forming its partial record for the update;
// block = threads per block of the rollout kernel; chunk = steps per unrolled
// chunk of the split rollout (its load-ahead depth: 2, 4 or 8).
struct RolloutTile {
  int variant;
  int block;
  int chunk;
};
RolloutTile default_tile(const DevProblem& P, int num_sms);
bool valid_tile(const RolloutTile& t);

// Device buffers of one problem (one noise set; the MPC step alternates two).
struct IterBuffers {
  const float* x0;
  float* U;
  void* noise;         // [T][Kpad][m] delta_eff, float32 or bfloat16
  uint32_t* jmask;     // [Kpad/32][mask_cols(T)] jump masks (sparse records): bit l of
                       // word [w][j] set when rollout 32w+l jumps at step j
  float4* jrec;        // [T][Kpad] jump records J (state jumps; dense: every step, zero
                       // without a jump; sparse: valid where the mask bit is set)
  float* s_part;       // [Kpad] k-dependent cost part
  float* partial;      // [chunks][T][m] (max_chunks chunks)
  int max_chunks;      // chunks the partial and zpart buffers hold
  float* rec;          // [ceil(Kpad/32)][2 + T*m] partial records of the rollout blocks
  float* zpart;        // [groups][chunks]
  float* gpart;        // [groups][m] shifted edge values, then [groups] control costs
  uint32_t* rho_key;   // running minimum of the costs (order key)
  uint32_t* rho_key_next;  // the running minimum of the next iteration
  unsigned* done;      // completion ticket of the update, then [groups] group tickets
  float* cconst;       // k-independent cost term
  float* diag;         // rho, Z, F
  int* status;
  uint32_t* it;        // iteration counter at the start of the step
  float* costs;        // may be NULL
  uint8_t* dbg_counts; // may be NULL
  float* dbg_J;        // may be NULL
  uint32_t* arm_key;   // NULL, or a running minimum the noise pass re-arms (empty)
};

// Split variant, part 1: noise of iteration *it + it_off into b.noise etc.
// With s_marks (and ev) the marks pass of sparse jump records, when the
// problem has one, runs on s_marks after an event hop, at the highest
// priority; without, everything runs on s.
cudaError_t launch_noise(const DevProblem& P, const IterBuffers& b, uint32_t it_off, cudaStream_t s,
                         cudaStream_t s_marks = nullptr, cudaEvent_t ev = nullptr);
// Whether the problem's noise pass is followed by marks_kernel (sparse
// state-jump records).
bool has_marks_pass(const DevProblem& P);

// State-channel jump records: dense (the noise pass draws the marks and
// writes every step's record) while the rollout blocks of 128 fit on the SMs
// at once, sparse beyond (jump masks, marks_kernel, gathered records).
bool marks_in_noise(const DevProblem& P);
// The jump masks of sparse records, or NULL (dense records, control-channel
// jumps).
uint32_t* sparse_mask(const DevProblem& P, const IterBuffers& b);

// One launch of the staged rollout (staged.cu, staged_sparse.cu): the dense
// and sparse jump-record forms are instantiated in two translation units.
constexpr int kStagedSmemMax = 160 * 1024;
struct StagedLaunch {
  const DevProblem* P;
  const IterBuffers* b;
  const RolloutTile* tile;
  int blocks;
  size_t smem;
  bool pdl;
  cudaStream_t s;
  bool part;
};
void launch_staged_dense(const StagedLaunch& L, int jump_mode);  // kJumpNone, kJumpDefault, kJumpRows
void launch_staged_sparse(const StagedLaunch& L, bool velocity_rows);
cudaError_t prepare_staged_dense();  // the kernels' shared-memory limits
cudaError_t prepare_staged_sparse();
// Split variant, part 2: the sequential rollout of iteration *it + it_off
// over the stored noise.  pdl: launch as a programmatic dependent of the
// previous kernel in the stream, which must then not be the noise pass that
// wrote b.noise (the staged rollout starts copying step data before it waits
// for that kernel).
cudaError_t launch_rollout_seq(const DevProblem& P, const IterBuffers& b, const RolloutTile& tile,
                               uint32_t it_off, bool pdl, cudaStream_t s);
// Whole rollout (either variant) of iteration *it + it_off.  arm_min resets
// the running cost minimum first (the update re-arms it after every
// iteration, so only a rollout that follows no update needs it).
cudaError_t launch_rollout(const DevProblem& P, const IterBuffers& b, const RolloutTile& tile,
                           uint32_t it_off, bool arm_min, cudaStream_t s);
// Where the update's partial sums come from: NULL, or rec == NULL, streams
// the stored perturbations; otherwise nb partial records (rho_b, Z_b, N_b)
// (of the rollout blocks of a tile-4 rollout, or of rollout shards) are
// rescaled and summed, rho taken from the records (rho_from_rec) or from the
// running minimum.  export_out != NULL writes the combined record
// (rho, Z, N[T][m]) there instead of updating U.
struct UpdateSource {
  const float* rec;
  int nb;
  int rho_from_rec;
  float* export_out;
};
// Records a chunk of the record-source update sums (m = 1 or 4).
int records_per_chunk(int m);
// Weights + update of iteration r of an MPC step (step size alpha *
// alpha_decay^r); shift != 0 performs the MPC shift and writes u0 (if not
// NULL); the counter advances by it_advance.  An ordinary launch (it
// starts once the preceding kernel has completed).
cudaError_t launch_update(const DevProblem& P, const IterBuffers& b, const UpdateGeom& g, int r,
                          int shift, uint32_t it_advance, float* u0, cudaStream_t s,
                          const UpdateSource* src = nullptr);
// costs[k] = S~_k (the full augmented cost) when b.costs is not NULL.
cudaError_t launch_costs(const DevProblem& P, const IterBuffers& b, cudaStream_t s);
// w_k = exp((rho - S~_k)/lambda) / Z (rho = diag[3], Z = diag[1]) for the
// weights getter.
cudaError_t launch_weights(const float* s_part, const float* diag, float inv_lam, int K, float* w,
                           cudaStream_t s);

}  // namespace mj
