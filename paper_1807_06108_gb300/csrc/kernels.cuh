// kernels.cuh -- the kernels of one MPPI iteration on jump diffusions:
//   rollout_kernel         fused sampling + rollout + augmented cost (A1+A2)
//   noise_kernel           split form, part 1: sampling over K x T/4 threads (A1)
//   rollout_split_kernel   split form, part 2: sequential rollout + cost (A2),
//                          step data through a register ring
//   rollout_staged_kernel  split form, part 2 (the default): step data moved
//                          into shared memory by a producer warp's bulk copies
//   update_kernel          free-energy weights, split-K weighted sum, combine,
//                          U update, counter and MPC shift (A3+A4+A5)
// Every rollout form publishes min_k S~_k through one atomic per warp.  The
// random stream of an iteration is selected by *it_ptr + it_off, so the noise
// of a later iteration can be drawn while the current one is still rolled out.
// Included by the translation units that launch them.
#pragma once

#include "device.cuh"

namespace mj {

constexpr int kRolloutThreads = 128;
constexpr int kNoiseThreads = 128;       // noise-pass block, small problems
constexpr int kNoiseThreadsLarge = 256;  // and with sparse jump records
constexpr int kUpdateThreads = 256;
constexpr int kStatusNonFinite = 5;
constexpr int kStatusBounds = 7;  // MPPI_EBOUNDS

// Debug build (MPPI_CHECK_BOUNDS): every kernel first checks that its launch
// geometry and dynamic shared memory match the problem it was given; a
// failed check writes MPPI_EBOUNDS into the status word and the whole block
// returns before touching memory (no trap, no assert).  The conditions are
// the same for every block of a launch, so no block is left waiting at a
// barrier.  Compiled out otherwise.
#ifdef MPPI_CHECK_BOUNDS
__device__ __forceinline__ void bounds_failed(int* status) {
  if (status) atomicExch(status, kStatusBounds);
}
#define MJ_CHECK(cond, status)    \
  do {                            \
    if (!(cond)) {                \
      bounds_failed(status);      \
      return;                     \
    }                             \
  } while (0)
#else
#define MJ_CHECK(cond, status) \
  do {                         \
  } while (0)
#endif

__device__ __forceinline__ uint32_t dynamic_smem_bytes() {
  uint32_t r;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
  return r;
}
constexpr uint32_t kKeyEmpty = 0xffffffffu;  // larger than every cost key
constexpr uint32_t kKeyInf = 0xff800000u;    // order key of +inf

// ---------------------------------------------------------------------------
// Order-preserving map between float32 and uint32 (an atomic minimum over
// costs of either sign): larger key <=> larger float.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t order_key(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_to_float(uint32_t key) {
  return __uint_as_float((key & 0x80000000u) ? (key & 0x7fffffffu) : ~key);
}

// Warp minimum of the rollout costs folded into a global atomic minimum (one
// atomic per warp).  Every lane of the warp must call it.
__device__ __forceinline__ void publish_min_cost(float sk, uint32_t* rho_key) {
  const uint32_t w = __reduce_min_sync(0xffffffffu, order_key(sk));
  if ((threadIdx.x & 31) == 0) atomicMin(rho_key, w);
}

// Compensated sum over the warp (every lane gets the result).
__device__ __forceinline__ void warp_sum2(float& s, float& c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
    const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
    two_sum_merge(s, c, s2, c2);
  }
}

// Programmatic dependent launch: a kernel launched as the programmatic
// dependent of the previous kernel in its stream may start while that kernel
// still runs; griddep_wait() returns once the previous kernel has completed
// and its memory is visible (at once when there is no such dependency), and
// griddep_launch_dependents() lets the next kernel start launching.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Mark of the nj-th jump of step j (stream 2+nj of the Philox counter) added
// to J.  The rounding is explicit (one fused multiply-add per Normal
// component, one rounded add per Laplace component), so every kernel that
// draws marks accumulates them bit for bit alike.
__device__ __forceinline__ void add_mark(const DevProblem& P, uint32_t k, uint32_t j, uint32_t it,
                                         int nj, float J[4]) {
  const uint4 wm = philox4x32_10(k, j, it, 2u + (uint32_t)nj, P.key0, P.key1);
  if (P.mark_law == 0) {
    float z[4];
    normals4(wm, z);
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (c < P.q) J[c] = fmaf(P.mark_scale[c], z[c], J[c]);
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (c < P.q) J[c] = __fadd_rn(J[c], laplace_mark(P.mark_scale[c], word_of(wm, c)));
  }
}

// Summed marks of the N jumps of one step, in jump order.
__device__ __forceinline__ void draw_marks(const DevProblem& P, uint32_t k, uint32_t j, uint32_t it,
                                           int N, float J[4]) {
  for (int nj = 0; nj < N; ++nj) add_mark(P, k, j, it, nj, J);
}

template <int M, bool BF16>
__device__ __forceinline__ void store_noise(void* __restrict__ noise, size_t row, const float* de,
                                            bool active) {
  if constexpr (BF16) {
    if constexpr (M == 4) {
      const __nv_bfloat162 lo = __floats2bfloat162_rn(active ? de[0] : 0.0f, active ? de[1] : 0.0f);
      const __nv_bfloat162 hi = __floats2bfloat162_rn(active ? de[2] : 0.0f, active ? de[3] : 0.0f);
      uint2 pk;
      pk.x = *reinterpret_cast<const uint32_t*>(&lo);
      pk.y = *reinterpret_cast<const uint32_t*>(&hi);
      reinterpret_cast<uint2*>(noise)[row] = pk;
    } else {
      reinterpret_cast<__nv_bfloat16*>(noise)[row] = __float2bfloat16_rn(active ? de[0] : 0.0f);
    }
  } else {
    if constexpr (M == 4) {
      reinterpret_cast<float4*>(noise)[row] = active ? make_float4(de[0], de[1], de[2], de[3])
                                                     : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    } else {
      reinterpret_cast<float*>(noise)[row] = active ? de[0] : 0.0f;
    }
  }
}

template <int M, bool BF16>
__device__ __forceinline__ void load_noise(const void* __restrict__ noise, size_t row, float* de) {
  if constexpr (BF16) {
    if constexpr (M == 4) {
      const uint2 pk = reinterpret_cast<const uint2*>(noise)[row];
      de[0] = __uint_as_float(pk.x << 16);
      de[1] = __uint_as_float(pk.x & 0xffff0000u);
      de[2] = __uint_as_float(pk.y << 16);
      de[3] = __uint_as_float(pk.y & 0xffff0000u);
    } else {
      const unsigned short h = reinterpret_cast<const unsigned short*>(noise)[row];
      de[0] = __uint_as_float((uint32_t)h << 16);
    }
  } else {
    if constexpr (M == 4) {
      const float4 v = reinterpret_cast<const float4*>(noise)[row];
      de[0] = v.x;
      de[1] = v.y;
      de[2] = v.z;
      de[3] = v.w;
    } else {
      de[0] = reinterpret_cast<const float*>(noise)[row];
    }
  }
}

// One step of cost and dynamics shared by the rollout forms: the
// k-dependent part of the augmented running cost of Eq. 34-35 in control
// units (the term lambda/2 u^T Sigma^-1 u is the same for every rollout and
// cancels in the weights; it is summed once per iteration by
// control_cost_sum) and the Euler step of Algorithm 1 with the control-affine
// drift of Eq. 4.  A state-channel jump of the step follows (state_jump).
template <int SYS>
__device__ __forceinline__ void cost_and_step(const DevProblem& P, float* x, const float* u,
                                              const float* de, float& s, float& sc) {
  using PL = Plant<SYS>;
  constexpr int n = PL::n, m = PL::m;
  float uSd = 0.0f, dSd = 0.0f;
#pragma unroll
  for (int i = 0; i < m; ++i) {
    const float ad = P.inv_sigma2[i] * de[i];
    uSd += u[i] * ad;
    dSd += de[i] * ad;
  }
  const float qx = PL::state_cost(P.pl, x);
  two_sum_acc(s, sc, qx * P.dt + P.lam * (uSd + P.is_coef * dSd));
  float v[m], xd[n];
#pragma unroll
  for (int i = 0; i < m; ++i) v[i] = u[i] + de[i];
  PL::xdot(P.pl, x, v, xd);
#pragma unroll
  for (int i = 0; i < n; ++i) x[i] += xd[i] * P.dt;
}

// The state-channel jump of a step (Eq. 2, Algorithm 1), after its Euler
// step: x[H rows] += s_J J, s_J = sqrt(dt) or 1.  It is applied on every
// step (J is zero for a step without a jump, which leaves x unchanged, as in
// the oracle), so the step loop has no branch.  state_jump_default serves
// the plant's velocity rows, (xdot, thetadot) or (vx, vy, vz); state_jump_rows
// any rows; state_jump picks one at run time.
template <int SYS>
__device__ __forceinline__ void state_jump_default(const DevProblem& P, float* x, const float J[4]) {
  if constexpr (SYS == 0) {
    x[1] += P.s_jump * J[0];
    x[3] += P.s_jump * J[1];
  } else {
    x[3] += P.s_jump * J[0];
    x[4] += P.s_jump * J[1];
    x[5] += P.s_jump * J[2];
  }
}

template <int SYS>
__device__ __forceinline__ void state_jump_rows(const DevProblem& P, float* x, const float J[4]) {
  constexpr int n = Plant<SYS>::n;
#pragma unroll
  for (int r = 0; r < n; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (c < P.q && P.jump_rows[c] == r) x[r] += P.s_jump * J[c];
}

template <int SYS>
__device__ __forceinline__ void state_jump(const DevProblem& P, float* x, const float J[4]) {
  if (P.jump_default) state_jump_default<SYS>(P, x, J);
  else state_jump_rows<SYS>(P, x, J);
}

// Final cost of a rollout: terminal cost, non-finite -> +inf, and the warp's
// contribution to the running minimum.
template <int SYS>
__device__ __forceinline__ float finish_rollout(const DevProblem& P, int k, bool active, const float* x,
                                                float s, float sc, float* __restrict__ s_part,
                                                uint32_t* __restrict__ rho_key) {
  two_sum_acc(s, sc, Plant<SYS>::terminal_cost(P.pl, x));
  float sk = s + sc;
  if (!isfinite(sk) || !active) sk = INFINITY;
  s_part[k] = sk;
  publish_min_cost(sk, rho_key);  // Kpad is a multiple of 32: whole warps
  return sk;
}


// ---------------------------------------------------------------------------
// Fused rollout: one thread per rollout k, the plant state in registers.  Per
// step j: the Gaussian perturbation (stream 0), the jump count (stream 1, one
// Philox block per four steps) and, when the count is positive, the marks
// (streams 2+n); delta_eff is rounded to bfloat16 first when the noise is
// stored in that type, so the rollout uses exactly the stored value; then
// cost_and_step.  delta_eff is stored step-major, noise[(j*Kpad + k)*m + i],
// so each warp store is contiguous.  Rollouts K..Kpad-1 (padding) store zero
// noise and an infinite cost.
// ---------------------------------------------------------------------------
template <int SYS, bool BF16, bool DBG, bool COHERENT, int CH>
__device__ __forceinline__ void fused_rollout_thread(
    const DevProblem& P, const float* __restrict__ x0, const float* __restrict__ U, uint32_t it, int k,
    float* __restrict__ s_part, void* __restrict__ noise, uint32_t* __restrict__ rho_key,
    uint8_t* __restrict__ dbg_counts, float* __restrict__ dbg_J);

// CH: steps per unrolled chunk (4, 8 or 16): the chunk's count blocks (one
// per four steps) are drawn together at its start and its steps are
// unrolled, so the random numbers of later steps can be computed while the
// dynamics of earlier ones wait on their dependencies.  Every CH gives the
// same values.
template <int SYS, bool BF16, bool DBG, int CH>
__global__ void __launch_bounds__(kRolloutThreads)
rollout_kernel(const DevProblem P, const float* __restrict__ x0, const float* __restrict__ U,
               const uint32_t* __restrict__ it_ptr, uint32_t it_off, float* __restrict__ s_part,
               void* __restrict__ noise,
               uint32_t* __restrict__ rho_key, uint8_t* __restrict__ dbg_counts,
               float* __restrict__ dbg_J, int* __restrict__ status) {
  MJ_CHECK(blockDim.x % 32 == 0 && blockDim.x <= kRolloutThreads && P.Kpad % 32 == 0 && P.K <= P.Kpad,
           status);
  griddep_launch_dependents();
  griddep_wait();  // U and the running minimum come from the previous update
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P.Kpad) return;
  fused_rollout_thread<SYS, BF16, DBG, false, CH>(P, x0, U, __ldg(it_ptr) + it_off, k, s_part, noise,
                                                  rho_key, dbg_counts, dbg_J);
}

// The body of the fused rollout for rollout k < Kpad of a problem; every lane
// of the warp must run it (k >= Kpad lanes are not allowed: Kpad is a
// multiple of 32).  COHERENT reads x0 and U through L2, for callers in which
// another block of the same launch may have written them.
template <int SYS, bool BF16, bool DBG, bool COHERENT, int CH>
__device__ __forceinline__ void fused_rollout_thread(
    const DevProblem& P, const float* __restrict__ x0, const float* __restrict__ U, uint32_t it, int k,
    float* __restrict__ s_part, void* __restrict__ noise, uint32_t* __restrict__ rho_key,
    uint8_t* __restrict__ dbg_counts, float* __restrict__ dbg_J) {
  static_assert(CH == 4 || CH == 8 || CH == 16, "steps per chunk");
  constexpr int n = Plant<SYS>::n, m = Plant<SYS>::m;
  constexpr int NB = CH / 4;  // count blocks of a chunk
  const bool active = k < P.K;
  const uint32_t uk = P.k_base + (uint32_t)k;  // the rollout's index in the Philox counter
  float x[n];
#pragma unroll
  for (int i = 0; i < n; ++i) x[i] = COHERENT ? __ldcg(x0 + i) : __ldg(x0 + i);
  float s = 0.0f, sc = 0.0f;
  for (int j0 = 0; j0 < P.T; j0 += CH) {
    uint4 wcount[NB];
    float zc[NB][4];
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      const uint32_t b = (uint32_t)((j0 >> 2) + c);
      wcount[c] = philox4x32_10(uk, b, it, 1u, P.key0, P.key1);
      if constexpr (m == 1) normals4(philox4x32_10(uk, b, it, 0u, P.key0, P.key1), zc[c]);
    }
#pragma unroll
    for (int jj = 0; jj < CH; ++jj) {
      const int j = j0 + jj;
      if (j >= P.T) break;
      float de[m];
      if constexpr (m == 1) {
        de[0] = __fmul_rn(P.sqc_sigma[0], zc[jj >> 2][jj & 3]);
      } else {
        float z[4];
        normals4(philox4x32_10(uk, (uint32_t)j, it, 0u, P.key0, P.key1), z);
#pragma unroll
        for (int i = 0; i < m; ++i) de[i] = __fmul_rn(P.sqc_sigma[i], z[i]);
      }
      const int N = jump_count(P, word_of(wcount[jj >> 2], jj & 3));
      float J[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      if (N > 0) {
        draw_marks(P, uk, (uint32_t)j, it, N, J);
        if (P.jump_channel == 1) {
#pragma unroll
          for (int i = 0; i < m; ++i) de[i] = __fadd_rn(de[i], J[i]);
        }
      }
      if constexpr (BF16) {
#pragma unroll
        for (int i = 0; i < m; ++i) de[i] = __bfloat162float(__float2bfloat16_rn(de[i]));
      }
      float u[m];
#pragma unroll
      for (int i = 0; i < m; ++i) u[i] = COHERENT ? __ldcg(U + j * m + i) : __ldg(U + j * m + i);
      cost_and_step<SYS>(P, x, u, de, s, sc);
      if (P.jump_channel == 0) state_jump<SYS>(P, x, J);  // J = 0 without a jump
      store_noise<m, BF16>(noise, (size_t)j * P.Kpad + k, de, active);
      if (DBG && active) {
        const size_t rk = (size_t)j * P.K + k;
        if (dbg_counts) dbg_counts[rk] = (uint8_t)N;
        if (dbg_J)
          for (int c = 0; c < P.q; ++c) dbg_J[rk * P.q + c] = J[c];
      }
    }
  }
  finish_rollout<SYS>(P, k, active, x, s, sc, s_part, rho_key);
}

// ---------------------------------------------------------------------------
// Split form, part 1.  noise_kernel: thread (k, b), k = blockIdx.x * 128 +
// threadIdx.x and b = blockIdx.y, draws steps 4b .. 4b+3 of rollout k (the
// four steps that share one jump-count Philox block), so the sampling runs
// over K * T/4 threads instead of K.  It stores delta_eff (the bfloat16
// rounding applied); consecutive threads take consecutive k, so every store
// is contiguous.  MARKS: the thread also draws the marks of its jumps -- for
// control-channel jumps, which are folded into delta_eff, for the debug copy
// of J, and (with jrec_marks) for dense state-channel jump records, which it
// writes for every step (J, or zero without a jump).  Sparse state-channel
// records (jmask != NULL): the pass stores the jump masks, a warp's ballot of
// "count > 0" per step, bit l of jmask[w][j] for rollout 32w + l (padding
// rollouts 0), lane 0 writing the four steps' words at once; marks_kernel
// then writes the records where a bit is set, and a record is read only
// there, so none is ever cleared.  The pass touches nothing the rollout or
// update of another iteration reads, so it can run concurrently with them on
// a second buffer set.  arm_key (may be NULL): the running minimum to re-arm.
// ---------------------------------------------------------------------------
template <int M, bool BF16, bool DBG, bool MARKS>
__global__ void __launch_bounds__(kNoiseThreadsLarge)
noise_kernel(const DevProblem P, const uint32_t* __restrict__ it_ptr, uint32_t it_off,
             void* __restrict__ noise, uint32_t* __restrict__ jmask, float4* __restrict__ jrec,
             int jrec_marks, uint8_t* __restrict__ dbg_counts, float* __restrict__ dbg_J,
             int* __restrict__ status, uint32_t* __restrict__ arm_key) {
  static_assert(MARKS || !DBG, "the debug copy of J needs the marks");
  // the first noise pass of an MPC step re-arms the running minimum of the
  // step's first rollout (which launches after this pass)
  if (arm_key && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *arm_key = kKeyEmpty;
  MJ_CHECK((blockDim.x == kNoiseThreads || blockDim.x == kNoiseThreadsLarge) && 4 * (int)blockIdx.y < P.T && P.Kpad % 32 == 0 && P.K <= P.Kpad &&
               P.m == M,
           status);
  const int k = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
  if (k >= P.Kpad) return;
  const bool active = k < P.K;
  const uint32_t it = __ldg(it_ptr) + it_off;
  const uint32_t uk = P.k_base + (uint32_t)k;  // the rollout's index in the Philox counter
  const int ns = min(4, P.T - 4 * b);  // steps of this thread
  const uint4 wcount = philox4x32_10_rk(uk, (uint32_t)b, it, 1u, P.rk);
  int N[4];
#pragma unroll
  for (int jj = 0; jj < 4; ++jj) N[jj] = jj < ns ? jump_count(P, word_of(wcount, jj)) : 0;
  float J[4][4];
#pragma unroll
  for (int jj = 0; jj < 4; ++jj)
#pragma unroll
    for (int c = 0; c < 4; ++c) J[jj][c] = 0.0f;
  if constexpr (MARKS) {
    // Marks, one loop trip per jump in (step, jump) order: a warp runs the
    // mark code as often as its busiest lane has jumps in its four steps, and
    // the code exists once.  Each step's marks are summed in jump order, as
    // in draw_marks.
    const int c0 = N[0], c1 = c0 + N[1], c2 = c1 + N[2], total = c2 + N[3];
#pragma unroll 1
    for (int i = 0; i < total; ++i) {
      const int jj = i < c0 ? 0 : (i < c1 ? 1 : (i < c2 ? 2 : 3));
      const int first = jj == 0 ? 0 : (jj == 1 ? c0 : (jj == 2 ? c1 : c2));
      // the step's running sum, through add_mark as in draw_marks
      float Jt[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) Jt[c] = jj == 0 ? J[0][c] : (jj == 1 ? J[1][c] : (jj == 2 ? J[2][c] : J[3][c]));
      add_mark(P, uk, (uint32_t)(4 * b + jj), it, i - first, Jt);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q == jj)
#pragma unroll
          for (int c = 0; c < 4; ++c) J[q][c] = Jt[c];
    }
  }
  if ((!MARKS || DBG) && jmask) {  // sparse records are drawn by marks_kernel
    // the warp's 32 rollouts: one mask word per step (zero past T)
    uint4 mw;
    mw.x = __ballot_sync(0xffffffffu, active && N[0] > 0);
    mw.y = __ballot_sync(0xffffffffu, active && N[1] > 0);
    mw.z = __ballot_sync(0xffffffffu, active && N[2] > 0);
    mw.w = __ballot_sync(0xffffffffu, active && N[3] > 0);
    if ((threadIdx.x & 31) == 0)
      reinterpret_cast<uint4*>(jmask + (size_t)(k >> 5) * mask_cols(P.T))[b] = mw;
  }
  // The four steps' perturbations first, as independent dependency chains
  // (the four Philox blocks of the steps interleave); a thread of the last
  // step block with fewer than four steps draws the missing ones and drops
  // them.
  float de[4][M];
  if constexpr (M == 1) {
    float zc[4];
    normals4(philox4x32_10_rk(uk, (uint32_t)b, it, 0u, P.rk), zc);
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) de[jj][0] = __fmul_rn(P.sqc_sigma[0], zc[jj]);
  } else {
    uint4 w[4];
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) w[jj] = philox4x32_10_rk(uk, (uint32_t)(4 * b + jj), it, 0u, P.rk);
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      float z[4];
      normals4(w[jj], z);
#pragma unroll
      for (int i = 0; i < M; ++i) de[jj][i] = __fmul_rn(P.sqc_sigma[i], z[i]);
    }
  }
#pragma unroll
  for (int jj = 0; jj < 4; ++jj) {
    const int j = 4 * b + jj;
    if (jj >= ns) break;
    const size_t row = (size_t)j * P.Kpad + k;
    if (MARKS && P.jump_channel == 1 && N[jj] > 0) {
#pragma unroll
      for (int i = 0; i < M; ++i) de[jj][i] = __fadd_rn(de[jj][i], J[jj][i]);
    }
    store_noise<M, BF16>(noise, row, de[jj], active);  // rounds to bfloat16 (RNE) when BF16
    if (MARKS && jrec && jrec_marks)  // dense records: J, or zero without a jump
      jrec[row] = active ? make_float4(J[jj][0], J[jj][1], J[jj][2], J[jj][3]) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (DBG && active) {
      const size_t rk = (size_t)j * P.K + k;
      if (dbg_counts) dbg_counts[rk] = (uint8_t)N[jj];
      if (dbg_J)
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (c < P.q) dbg_J[rk * P.q + c] = J[jj][c];
    }
  }
}

// ---------------------------------------------------------------------------
// Split form, part 1b (state-channel jumps).  marks_kernel: the marks of every
// (step, rollout) whose jump mask bit is set, with the lanes of a warp busy on
// jumps rather than on steps.  A warp covers one 32-rollout row of the masks
// over 32 steps (lane i loads the word of step 32c + i), lists the set bits in
// shared memory (a ballot prefix sum: deterministic positions) and handles one
// jump per lane: the step's count again from its Philox block (stream 1, as
// in the noise pass), its summed marks (draw_marks, streams 2+n, as every
// other form draws them) into the step's jump record.  At the large
// workload's jump probability (2.5 % per step) a warp lists about 26 jumps:
// one pass of its lanes.  Grid (ceil(Kpad / (32 * kMarkWarps)),
// ceil(T / 32)), 32 * kMarkWarps threads.
// ---------------------------------------------------------------------------
constexpr int kMarkWarps = 4;
constexpr int kMarkThreads = 32 * kMarkWarps;

static __global__ void __launch_bounds__(kMarkThreads)
marks_kernel(const DevProblem P, const uint32_t* __restrict__ it_ptr, uint32_t it_off,
             const uint32_t* __restrict__ jmask, float4* __restrict__ jrec, int* __restrict__ status) {
  __shared__ uint16_t list[kMarkWarps][1024];
  MJ_CHECK(blockDim.x == kMarkThreads && 32 * (int)blockIdx.y < P.T && P.Kpad % 32 == 0, status);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int row = blockIdx.x * kMarkWarps + w;  // the warp's 32 rollouts: 32 row .. 32 row + 31
  const int j = 32 * (int)blockIdx.y + lane;    // this lane's step
  if (row >= P.Kpad / 32) return;               // the same for every lane of the warp
  const uint32_t word = j < P.T ? jmask[(size_t)row * mask_cols(P.T) + j] : 0u;
  const int ne = __popc(word);  // 0 .. 32
  uint32_t bal[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) bal[q] = __ballot_sync(0xffffffffu, (ne >> q) & 1);
  const uint32_t lt = (1u << lane) - 1u;
  int total = 0, pos = 0;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    total += __popc(bal[q]) << q;
    pos += __popc(bal[q] & lt) << q;
  }
  if (total == 0) return;  // the same for every lane of the warp
  for (uint32_t mw = word; mw; mw &= mw - 1u)  // this lane's jumps, in rollout order
    list[w][pos++] = (uint16_t)((lane << 5) | (__ffs(mw) - 1));
  __syncwarp();
  const uint32_t it = __ldg(it_ptr) + it_off;
  for (int e = lane; e < total; e += 32) {
    const uint32_t ev = list[w][e];
    const int js = 32 * (int)blockIdx.y + (int)(ev >> 5), k = 32 * row + (int)(ev & 31u);
    const uint32_t uk = P.k_base + (uint32_t)k;
    const int c = jump_count(P, word_of(philox4x32_10_rk(uk, (uint32_t)(js >> 2), it, 1u, P.rk), js & 3));
    float J[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    draw_marks(P, uk, (uint32_t)js, it, c, J);
    jrec[(size_t)js * P.Kpad + k] = make_float4(J[0], J[1], J[2], J[3]);
  }
}

// ---------------------------------------------------------------------------
// Split form, part 2.  rollout_split_kernel: one thread per rollout runs the
// sequential dynamics from the stored step data.  A register ring of kAhead
// slots keeps the loads of step j + kAhead in flight while step j is
// computed (the loop is unrolled by kAhead so every slot index is static);
// kAhead is the tile's "steps per unrolled chunk".  State-channel jumps add the
// step's jump record (dense records: zero without a jump; sparse: loaded only
// where the warp's mask word of the step, one broadcast load, has the lane's
// bit, zero elsewhere).
// ---------------------------------------------------------------------------
template <int SYS, bool BF16, int kAhead>
__global__ void __launch_bounds__(kRolloutThreads)
rollout_split_kernel(const DevProblem P, const float* __restrict__ x0, const float* __restrict__ U,
                     const void* __restrict__ noise, const uint32_t* __restrict__ jmask,
                     const float4* __restrict__ jrec, float* __restrict__ s_part, uint32_t* __restrict__ rho_key,
                     int* __restrict__ status) {
  constexpr int n = Plant<SYS>::n, m = Plant<SYS>::m;
  MJ_CHECK(blockDim.x % 32 == 0 && blockDim.x <= kRolloutThreads && P.Kpad % 32 == 0 && P.m == m, status);
  griddep_launch_dependents();
  griddep_wait();  // U and the running minimum come from the previous update
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P.Kpad) return;  // whole warps: Kpad is a multiple of 32
  const bool active = k < P.K;
  const int T = active ? P.T : 0;  // padding lanes skip the loop
  const bool sj = P.jump_channel == 0;
  const uint32_t* mrow = sj && jmask ? jmask + (size_t)(k >> 5) * mask_cols(P.T) : nullptr;
  const uint32_t lane_bit = 1u << (k & 31);
  float x[n];
#pragma unroll
  for (int i = 0; i < n; ++i) x[i] = __ldg(x0 + i);
  float s = 0.0f, sc = 0.0f;

  float rd[kAhead][m], ru[kAhead][m];
  float4 rj[kAhead];
  auto fetch = [&](int step, float* d, float* u, float4& jr) {
    const size_t row = (size_t)step * P.Kpad + k;
    load_noise<m, BF16>(noise, row, d);
    if constexpr (m == 4) {  // U rows are 16-byte aligned
      const float4 u4 = __ldg(reinterpret_cast<const float4*>(U) + step);
      u[0] = u4.x;
      u[1] = u4.y;
      u[2] = u4.z;
      u[3] = u4.w;
    } else {
#pragma unroll
      for (int i = 0; i < m; ++i) u[i] = __ldg(U + step * m + i);
    }
    jr = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (sj && (!mrow || (__ldg(mrow + step) & lane_bit))) jr = __ldg(jrec + row);
  };
#pragma unroll
  for (int sl = 0; sl < kAhead; ++sl)
    if (sl < T) fetch(sl, rd[sl], ru[sl], rj[sl]);

  for (int j0 = 0; j0 < T; j0 += kAhead) {
#pragma unroll
    for (int jj = 0; jj < kAhead; ++jj) {
      const int j = j0 + jj;
      if (j >= T) break;
      float de[m], u[m];
#pragma unroll
      for (int i = 0; i < m; ++i) {
        de[i] = rd[jj][i];
        u[i] = ru[jj][i];
      }
      const float J[4] = {rj[jj].x, rj[jj].y, rj[jj].z, rj[jj].w};
      if (j + kAhead < T) fetch(j + kAhead, rd[jj], ru[jj], rj[jj]);
      cost_and_step<SYS>(P, x, u, de, s, sc);
      if (sj) state_jump<SYS>(P, x, J);  // a zero record without a jump
    }
  }
  finish_rollout<SYS>(P, k, active, x, s, sc, s_part, rho_key);
}

// ---------------------------------------------------------------------------
// Bulk copies into shared memory with mbarrier completion (sm_90+ PTX).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Orders this thread's earlier shared-memory accesses before later
// async-proxy (bulk copy) accesses to the same memory.
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// One 16-byte copy global -> shared (dst, src 16-byte aligned), completed
// asynchronously; cp_async_arrive makes an mbarrier track this thread's
// earlier copies (one pending arrival, released when they have landed).
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for phase `parity` of *bar to complete; false after limit_ns of wall
// time (or 2^24 polls), so a copy that never lands cannot hang the kernel.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = timer_ns();
  for (uint32_t it = 1; it < (1u << 24); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 31) == 0 && timer_ns() - t0 > limit_ns) return false;
  }
  return false;
}

constexpr uint64_t kCopyWaitNs = 1000000000ull;  // 1 s
constexpr int kStatusTimeout = 4;               // MPPI_ETIMEOUT

// ---------------------------------------------------------------------------
// Split form, part 2, staged.  rollout_staged_kernel: the same per-rollout
// sequential dynamics as rollout_split_kernel, but the step data of the
// block's rollouts (delta_eff rows, the control rows and, for state-channel
// jumps, the jump records) is moved into shared memory, S steps per stage,
// two stage buffers.  The block is nt compute threads (one per rollout) plus
// one producer warp.
//
// Each stage buffer has a "landed" mbarrier (its copies are complete) and an
// "empty" one (every compute warp is done with it).  The producer's lane 0
// issues the bulk copies of stage s + 2 into a buffer once its compute warps
// have released it from stage s.  State-channel jump records come in one of
// two forms.  Dense (jmask == NULL, the records of every step written, zero
// without a jump): lane 0 bulk-copies the record rows with the rest.  Sparse
// (jmask != NULL, records valid only where the mask bit is set; the large
// problems, where a jump is 2.5 % of the steps and dense rows would double
// the bytes the rollout reads): each producer lane takes mask words (32
// rollouts x one step, loaded a stage ahead), zeroes the slots whose bit was
// set when the buffer was last filled, issues one 16-byte cp.async per set
// bit into the rollout's slot and makes "landed" track its copies; lane 0's
// second arrival on "landed" follows them.  Either way every slot holds the
// step's record or zero.  The sparse gather of stage 0 is issued before the
// wait on the previous kernel.  A compute warp waits for "landed", runs its S
// steps from shared memory, releases the buffer and moves on; no compute
// thread issues a copy or waits for another, and the dependency chain of the
// dynamics never waits on a global load.  For block b the rows are
// contiguous: step j covers elements [j*Kpad + b*nt, j*Kpad + b*nt + nk) of
// every step-major array (nk = the block's rollouts, a multiple of 32, so
// every copy is 16-byte aligned and a multiple of 16 bytes).  The
// control-row copy is rounded up to 16 bytes and may read up to 12 bytes past
// U's end (U must sit in an allocation padded to 16 bytes).  A compute thread
// adds s_J * J from its jump-record slot on every step (zero for a step
// without a jump), so the step loop has no branch.  Every wait is
// bounded.  Launch with nt + 32 threads and staged_smem_total() bytes of
// dynamic shared memory.
// ---------------------------------------------------------------------------
constexpr int kStagedMaxThreads = kRolloutThreads + 32;

// How a staged rollout applies jumps (a template argument, so that the step
// loop carries only what the problem needs):
//   kJumpNone    jumps act on the controls (folded into delta_eff);
//   kJumpDefault state jumps on the plant's velocity rows;
//   kJumpRows    state jumps on any other rows;
// and for state jumps whether their records are dense (the two above) or
// sparse (kJumpDefaultSparse, kJumpRowsSparse: gathered by jump mask).
constexpr int kJumpNone = 0, kJumpDefault = 1, kJumpRows = 2, kJumpDefaultSparse = 3, kJumpRowsSparse = 4;

// Shared-memory layout of the staged rollout (bytes), shared with the host:
// two stage buffers, four mbarriers and the partial record's scratch (PART).
__host__ __device__ constexpr uint32_t staged_stage_bytes(int nt, int m, int sb, int S, bool jumps) {
  return (uint32_t)S * ((uint32_t)nt * m * sb + (jumps ? (uint32_t)nt * 16u : 0u)) +
         (((uint32_t)S * m * 4u + 15u) & ~15u);
}
__host__ __device__ constexpr uint32_t staged_tail_offset(int nt, int m, int sb, int S, bool jumps) {
  return 2u * staged_stage_bytes(nt, m, sb, S, jumps) + 4u * 8u;
}
constexpr uint32_t kTailFloats = kRolloutThreads + 16;
__host__ __device__ constexpr uint32_t staged_smem_total(int nt, int m, int sb, int S, bool jumps, bool part) {
  return staged_tail_offset(nt, m, sb, S, jumps) + (part ? 4u * kTailFloats : 0u);
}

// PART: after its rollouts the block forms its partial record (Eq. 36-37
// restricted to its rollouts) rec[b] = (rho_b, Z_b, N_b[T][m]):
// rho_b = min S~_k, e_k = exp(-(S~_k - rho_b)/lambda), Z_b = sum e_k and
// N_b[j][i] = sum_k e_k delta_eff[j][k][i], re-reading its perturbation rows
// through the same two stage buffers (the producer copies them again, each
// compute warp reduces whole rows: per-lane products, compensated shuffle
// sums).  The update then only rescales and sums the records
// (update_kernel with the record source), with no second pass over the
// perturbations.
template <int SYS, bool BF16, int S, int JM, bool PART>
__global__ void __launch_bounds__(kStagedMaxThreads, PART ? 4 : 0)
rollout_staged_kernel(const DevProblem P, const float* __restrict__ x0, const float* __restrict__ U,
                      const void* __restrict__ noise, const uint32_t* __restrict__ jmask,
                      const float4* __restrict__ jrec, float* __restrict__ s_part, uint32_t* __restrict__ rho_key,
                      int* __restrict__ status, float* __restrict__ rec) {
  constexpr int n = Plant<SYS>::n, m = Plant<SYS>::m;
  constexpr bool kJ = JM != kJumpNone;
  constexpr bool kSparse = JM == kJumpDefaultSparse || JM == kJumpRowsSparse;
  constexpr bool kVelocityRows = JM == kJumpDefault || JM == kJumpDefaultSparse;
  static_assert(S == 4 || S == 8 || S == 16, "a stage's mask words: at most 2 per producer lane");
  constexpr uint32_t SB = BF16 ? 2u : 4u;
  extern __shared__ __align__(128) unsigned char stage_smem[];
  const int nt = blockDim.x - 32, tid = threadIdx.x;  // compute threads, then the producer warp
  const int k0 = blockIdx.x * nt;
  const int nk = min(nt, P.Kpad - k0);
  const int T = P.T;
  const uint32_t d_stride = (uint32_t)nt * m * SB;         // delta_eff of one step
  const uint32_t j_stride = kJ ? (uint32_t)nt * 16u : 0u;  // jump records of one step
  const uint32_t t_off = S * d_stride;                     // jump records
  const uint32_t u_off = S * (d_stride + j_stride);        // control rows
  const uint32_t stage_bytes = staged_stage_bytes(nt, m, (int)SB, S, kJ);
  uint64_t* landed = reinterpret_cast<uint64_t*>(stage_smem + 2 * stage_bytes);
  uint64_t* empty = landed + 2;
  float* tail = reinterpret_cast<float*>(stage_smem + staged_tail_offset(nt, m, (int)SB, S, kJ));
  int* abort_flag = reinterpret_cast<int*>(tail + kRolloutThreads + 8);
  const int n_stages = (T + S - 1) / S;
  const int compute_warps = nt / 32;
  const uint32_t d_bytes = (uint32_t)nk * m * SB;
  MJ_CHECK(nt >= 32 && nt <= kRolloutThreads && nt % 32 == 0 && k0 < P.Kpad && P.Kpad % 32 == 0 && T >= 1 &&
               P.m == m && (P.noise_bf16 != 0) == BF16 &&
               dynamic_smem_bytes() >= staged_smem_total(nt, m, (int)SB, S, kJ, PART),
           status);

  griddep_launch_dependents();
  if constexpr (kSparse) {
    // every jump-record slot of both buffers starts at zero
    for (uint32_t i = tid; i < 2u * S * nt; i += blockDim.x)
      reinterpret_cast<float4*>(stage_smem + (i / (S * nt)) * stage_bytes + t_off)[i % (S * nt)] =
          make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  }
  if (tid == nt) {
    // landed: lane 0's arrival with the byte count and, sparse, its arrival
    // after the lanes' record copies were issued
    mbar_init(landed, kSparse ? 2 : 1);
    mbar_init(landed + 1, kSparse ? 2 : 1);
    mbar_init(empty, (uint32_t)compute_warps);
    mbar_init(empty + 1, (uint32_t)compute_warps);
    mbar_init_fence();
    fence_async_smem();
    if (PART) *abort_flag = 0;
  }
  __syncthreads();

  // lane 0 of the producer: the perturbation rows of stage g (stage g >=
  // n_stages is pass g - n_stages over the rows, for the partial record) into
  // buffer g & 1
  auto issue_delta = [&](int g, int j0, int ns) {
    unsigned char* base = stage_smem + (g & 1) * stage_bytes;
    for (int jj = 0; jj < ns; ++jj) {
      const size_t row = (size_t)(j0 + jj) * P.Kpad + k0;
      bulk_load(base + jj * d_stride, static_cast<const unsigned char*>(noise) + row * m * SB, d_bytes,
                landed + (g & 1));
    }
  };
  int issued = 0;  // stages whose copies the producer issued
  bool ok = true;

  if (tid >= nt && !kSparse) {
    // ---- producer warp, dense records: lane 0 issues every stage's copies
    if (!PART && tid != nt) return;
    if (tid == nt) {
      const uint32_t j_bytes = kJ ? (uint32_t)nk * 16u : 0u;
      for (int st = 0; st < n_stages && ok; ++st) {
        const int buf = st & 1;
        if (st >= 2) {
          // every compute warp released the buffer (use st/2 - 1 of it)
          ok = mbar_wait_bounded(empty + buf, (uint32_t)((st >> 1) - 1) & 1u, kCopyWaitNs);
          if (!ok) break;
          fence_async_smem();
        }
        const int j0 = st * S;
        const int ns = min(S, T - j0);
        unsigned char* base = stage_smem + buf * stage_bytes;
        const uint32_t u_bytes = ((uint32_t)ns * m * 4 + 15) & ~15u;
        mbar_expect_tx(landed + buf, (uint32_t)ns * (d_bytes + j_bytes) + u_bytes);
        issue_delta(st, j0, ns);
        if (kJ)
          for (int jj = 0; jj < ns; ++jj)
            bulk_load(base + t_off + jj * j_stride, jrec + (size_t)(j0 + jj) * P.Kpad + k0, j_bytes,
                      landed + buf);
        // the step data was drawn before the previous kernel; the controls
        // come from the previous update
        if (st == 0) griddep_wait();
        bulk_load(base + u_off, U + (size_t)j0 * m, u_bytes, landed + buf);
        ++issued;
      }
      if (!ok) {
        atomicExch(status, kStatusTimeout);
        if (PART) *abort_flag = 1;
      }
      if (!PART) {
        // leave only when the copies of the last two stages have landed (bounded)
        for (int ls = max(0, issued - 2); ls < issued; ++ls)
          mbar_wait_bounded(landed + (ls & 1), (uint32_t)(ls >> 1) & 1u, kCopyWaitNs);
        return;
      }
    }
    issued = __shfl_sync(0xffffffffu, issued, 0);
  } else if (kSparse && tid >= nt) {
    // ---- producer warp, sparse records: lane 0 issues every stage's bulk
    // copies, every lane gathers records
    const int lane = tid - nt;
    const int mrows = nk >> 5;  // mask rows (32 rollouts each) of this block
    // the lane's mask words of a stage: pair p = lane + 32 r is row p / S, step p % S
    auto load_masks = [&](int st, uint32_t& w0, uint32_t& w1) {
      const int j0 = st * S, ns = min(S, T - j0);
      const uint32_t* mb = jmask + (size_t)(k0 >> 5) * mask_cols(T) + j0;
      const int p0 = lane, p1 = lane + 32;
      w0 = (p0 / S < mrows && p0 % S < ns) ? __ldg(mb + (size_t)(p0 / S) * mask_cols(T) + p0 % S) : 0u;
      w1 = (p1 / S < mrows && p1 % S < ns) ? __ldg(mb + (size_t)(p1 / S) * mask_cols(T) + p1 % S) : 0u;
    };
    uint32_t cur0 = 0, cur1 = 0;              // masks of the stage being issued
    uint32_t oa0 = 0, oa1 = 0, ob0 = 0, ob1 = 0;  // masks last gathered into buffer 0 / 1
    // sparse: the record slots of pair p, zero where only the old mask is
    // set, a copy where the new one is
    auto gather = [&](int p, int j0, unsigned char* base, uint32_t nw, uint32_t ow) {
      unsigned char* slot = base + t_off + (p % S) * j_stride + (p / S) * 32 * 16;
      for (uint32_t z = ow & ~nw; z; z &= z - 1u)
        *reinterpret_cast<float4*>(slot + (__ffs(z) - 1) * 16) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      const float4* src = jrec + (size_t)(j0 + p % S) * P.Kpad + k0 + (p / S) * 32;
      for (uint32_t z = nw; z; z &= z - 1u) cp_async16(slot + (__ffs(z) - 1) * 16, src + (__ffs(z) - 1));
    };
    for (int st = 0; st < n_stages && ok; ++st) {
      const int buf = st & 1;
      if (st >= 2) {
        // every compute warp released the buffer (use st/2 - 1 of it)
        if (lane == 0) ok = mbar_wait_bounded(empty + buf, (uint32_t)((st >> 1) - 1) & 1u, kCopyWaitNs);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        __syncwarp();  // the lanes' slot writes come after the compute warps' reads
        if (lane == 0) fence_async_smem();
      }
      const int j0 = st * S;
      const int ns = min(S, T - j0);
      unsigned char* base = stage_smem + buf * stage_bytes;
      const uint32_t u_bytes = ((uint32_t)ns * m * 4 + 15) & ~15u;
      if (lane == 0) {
        mbar_expect_tx(landed + buf, (uint32_t)ns * d_bytes + u_bytes);
        issue_delta(st, j0, ns);
      }
      if constexpr (kSparse) {
        if (st == 0) load_masks(0, cur0, cur1);
        gather(lane, j0, base, cur0, buf ? ob0 : oa0);
        gather(lane + 32, j0, base, cur1, buf ? ob1 : oa1);
        if (buf) {
          ob0 = cur0;
          ob1 = cur1;
        } else {
          oa0 = cur0;
          oa1 = cur1;
        }
        cp_async_arrive(landed + buf);
        __syncwarp();
        if (lane == 0) mbar_arrive(landed + buf);
        if (st + 1 < n_stages) load_masks(st + 1, cur0, cur1);
      }
      if (lane == 0) {
        // the step data was drawn before the previous kernel; the controls
        // come from the previous update
        if (st == 0) griddep_wait();
        bulk_load(base + u_off, U + (size_t)j0 * m, u_bytes, landed + buf);
      }
      ++issued;
    }
    cp_async_wait_all();
    if (!ok && lane == 0) {
      atomicExch(status, kStatusTimeout);
      if (PART) *abort_flag = 1;
    }
    if (!PART) {
      // leave only when the copies of the last two stages have landed (bounded)
      if (lane == 0)
        for (int ls = max(0, issued - 2); ls < issued; ++ls)
          mbar_wait_bounded(landed + (ls & 1), (uint32_t)(ls >> 1) & 1u, kCopyWaitNs);
      return;
    }
  } else {
    // ---- compute threads: one rollout each
    const int k = k0 + tid;
    const bool mine = tid < nk;  // a rollout slot of this block (whole warps)
    const bool active = k < P.K;
    float x[n];
#pragma unroll
    for (int i = 0; i < n; ++i) x[i] = __ldg(x0 + i);
    float s = 0.0f, sc = 0.0f;
    for (int st = 0; st < n_stages; ++st) {
      const int buf = st & 1;
      if (!mbar_wait_bounded(landed + buf, (uint32_t)(st >> 1) & 1u, kCopyWaitNs)) {
        atomicExch(status, kStatusTimeout);
        if (!PART) return;
        ok = false;
        break;
      }
      if (mine && active) {
        const unsigned char* base = stage_smem + buf * stage_bytes;
        const int j0 = st * S;
        const int ns = min(S, T - j0);
        // step data of step jj of this stage, from shared memory
        auto fetch = [&](int jj, float* de, float* u) {
          load_noise<m, BF16>(base + jj * d_stride, tid, de);
          if constexpr (m == 4) {
            const float4 u4 = reinterpret_cast<const float4*>(base + u_off)[jj];
            u[0] = u4.x;
            u[1] = u4.y;
            u[2] = u4.z;
            u[3] = u4.w;
          } else {
            u[0] = reinterpret_cast<const float*>(base + u_off)[jj];
          }
        };
        // Each step reads its data from shared memory at its start.  Long
        // stages (one block per SM, one warp per scheduler) unroll four steps,
        // which lets the compiler issue the reads of later steps early; short
        // ones (several blocks per SM, issue-bound) do not unroll, and the small
        // loop body stays in the instruction cache.  Measured on GB300 against
        // a one-step register prefetch with two-fold unrolling: MPC step 0.3217
        // -> 0.3187 ms at K = 4096, 1.3056 -> 1.2826 ms at K = 65536.
        constexpr int kUnroll = S >= 16 ? 4 : 1;
#pragma unroll kUnroll
        for (int jj = 0; jj < ns; ++jj) {
          float de[m], u[m];
          fetch(jj, de, u);
          cost_and_step<SYS>(P, x, u, de, s, sc);
          if constexpr (kJ) {
            const float4 jr = reinterpret_cast<const float4*>(base + t_off + jj * j_stride)[tid];
            const float J[4] = {jr.x, jr.y, jr.z, jr.w};  // zero for a step without a jump
            if constexpr (kVelocityRows) state_jump_default<SYS>(P, x, J);
            else state_jump_rows<SYS>(P, x, J);
          }
        }
      }
      // this warp is done with the buffer
      __syncwarp();
      if ((tid & 31) == 0) mbar_arrive(empty + buf);
    }
    griddep_wait();  // the running minimum was re-armed by the previous update
    if constexpr (!PART) {
      if (mine) finish_rollout<SYS>(P, k, active, x, s, sc, s_part, rho_key);
      return;
    } else {
      float sk = INFINITY;
      if (mine && ok) sk = finish_rollout<SYS>(P, k, active, x, s, sc, s_part, rho_key);
      tail[tid] = sk;
      if (!ok) *abort_flag = 1;
    }
  }

  if constexpr (PART) {
    // ---- the block's partial record
    float* e_sh = tail;                        // [nt]: S~_k, then e_k
    float* zw = tail + kRolloutThreads;        // [8]: compensated Z of each compute warp
    float* rho_sh = tail + kRolloutThreads + 9;
    const size_t R = 2 + (size_t)T * m;
    float* rb = rec + (size_t)blockIdx.x * R;
    __syncthreads();
    const bool go = *abort_flag == 0;
    if (go) {
      if (tid < 32) {
        float r = INFINITY;
        for (int t = tid; t < nt; t += 32) r = fminf(r, e_sh[t]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r = fminf(r, __shfl_xor_sync(0xffffffffu, r, o));
        if (tid == 0) *rho_sh = r;
      }
      __syncthreads();
      const float rho_b = *rho_sh;
      const bool any = rho_b < INFINITY;
      if (tid < nt) {
        const float sk = e_sh[tid];
        const float e = (any && sk < INFINITY) ? expf((rho_b - sk) * P.inv_lam) : 0.0f;
        e_sh[tid] = e;
        float zs = e, zc = 0.0f;
        warp_sum2(zs, zc);
        if ((tid & 31) == 0) {
          zw[2 * (tid >> 5)] = zs;
          zw[2 * (tid >> 5) + 1] = zc;
        }
      }
      __syncthreads();
      if (tid == 0) {
        float zs = 0.0f, zc = 0.0f;
        for (int w = 0; w < compute_warps; ++w) two_sum_merge(zs, zc, zw[2 * w], zw[2 * w + 1]);
        rb[0] = rho_b;
        rb[1] = any ? zs + zc : 0.0f;
      }
      if (!any) {
        for (int idx = tid; idx < T * m; idx += nt + 32) rb[2 + idx] = 0.0f;
      } else if (tid >= nt) {
        // producer: the perturbation rows again, stage by stage
        if (tid == nt) {
          fence_async_smem();
          for (int ts = 0; ts < n_stages; ++ts) {
            const int g = n_stages + ts;
            if (ts >= 2 && !mbar_wait_bounded(empty + (g & 1), (uint32_t)((g >> 1) - 1) & 1u, kCopyWaitNs)) {
              atomicExch(status, kStatusTimeout);
              break;
            }
            if (ts >= 2) fence_async_smem();
            const int j0 = ts * S, ns = min(S, T - j0);
            mbar_expect_tx(landed + (g & 1), (uint32_t)ns * d_bytes);
            if (kSparse) mbar_arrive(landed + (g & 1));  // no records in this pass
            issue_delta(g, j0, ns);
            issued = g + 1;
          }
        }
        issued = __shfl_sync(0xffffffffu, issued, 0);
      } else {
        // compute warps: whole rows, lane l takes rollouts l, l + 32, ...
        const int wid = tid >> 5, lane = tid & 31;
        for (int ts = 0; ts < n_stages; ++ts) {
          const int g = n_stages + ts;
          if (!mbar_wait_bounded(landed + (g & 1), (uint32_t)(g >> 1) & 1u, kCopyWaitNs)) {
            atomicExch(status, kStatusTimeout);
            break;
          }
          const unsigned char* base = stage_smem + (g & 1) * stage_bytes;
          const int j0 = ts * S, ns = min(S, T - j0);
          for (int jj = wid; jj < ns; jj += compute_warps) {
            float acc[m];
#pragma unroll
            for (int i = 0; i < m; ++i) acc[i] = 0.0f;
            for (int t = lane; t < nk; t += 32) {
              float d[m];
              load_noise<m, BF16>(base + jj * d_stride, t, d);
              const float e = e_sh[t];
#pragma unroll
              for (int i = 0; i < m; ++i) acc[i] = fmaf(e, d[i], acc[i]);
            }
#pragma unroll
            for (int i = 0; i < m; ++i) {
              float c = 0.0f;
              warp_sum2(acc[i], c);
              if (lane == 0) rb[2 + (size_t)(j0 + jj) * m + i] = acc[i] + c;
            }
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(empty + (g & 1));
        }
      }
    }
  }
  if (PART && tid == nt) {
    // leave only when the copies of the last two issued stages have landed (bounded)
    for (int ls = max(0, issued - 2); ls < issued; ++ls)
      mbar_wait_bounded(landed + (ls & 1), (uint32_t)(ls >> 1) & 1u, kCopyWaitNs);
  }
}

// ---------------------------------------------------------------------------
// Block reductions (NT threads per block)
// ---------------------------------------------------------------------------

// Shared scratch of the update bodies for NT threads: per-warp partial sums
// and the weights of one chunk of rollouts (ECAP floats).
template <int NT, int ECAP, bool REC = false>
struct UpdateShared {
  float sh_s[NT / 32], sh_c[NT / 32];
  unsigned ticket;
  float rho;
  __align__(16) float e[ECAP];
  float red[REC ? NT : 1];  // partial sums of the record source
};

// Rollouts per chunk of the weighted sum: NT * VPT 16-byte vectors of a row.
template <bool BF16, int M, int VPT, int NT>
__host__ __device__ constexpr int chunk_rollouts() {
  return NT * VPT * ((BF16 ? 8 : 4) / M);
}

// Compensated sum over the block; every thread gets the result.
template <int NT>
__device__ __forceinline__ float block_sum2(float s, float c, float* sh_s, float* sh_c) {
  constexpr int W = NT / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  warp_sum2(s, c);
  __syncthreads();
  if (lane == 0) {
    sh_s[wid] = s;
    sh_c[wid] = c;
  }
  __syncthreads();
  float a = lane < W ? sh_s[lane] : 0.0f;
  float b = lane < W ? sh_c[lane] : 0.0f;
  warp_sum2(a, b);
  return a + b;
}

// C = sum_j lambda/2 u_j^T Sigma^-1 u_j, the rollout-independent part of S~
// (Eq. 35), summed with compensation by the whole block (every thread gets C).
// U is read through L2 (it may have been written by another block of the
// same launch).
template <int M, int NT>
__device__ __forceinline__ float control_cost_sum(const float* __restrict__ U, int T, float lam,
                                                  const float* inv_sigma2, float* sh_s, float* sh_c) {
  float s = 0.0f, c = 0.0f;
  for (int idx = threadIdx.x; idx < T * M; idx += NT) {
    const float u = __ldcg(U + idx);
    two_sum_acc(s, c, 0.5f * lam * (u * inv_sigma2[idx % M] * u));
  }
  return block_sum2<NT>(s, c, sh_s, sh_c);
}

// costs[k] = C + (S~_k - C), the full augmented cost of Eq. 34, for the
// rollout_cost output (each block recomputes C from U).
template <int M>
__global__ void __launch_bounds__(kUpdateThreads)
costs_kernel(const float* __restrict__ U, int T, float lam, float4 inv_sigma2,
             const float* __restrict__ s_part, int K, float* __restrict__ costs) {
  __shared__ float sh_s[kUpdateThreads / 32], sh_c[kUpdateThreads / 32];
  const float is2[4] = {inv_sigma2.x, inv_sigma2.y, inv_sigma2.z, inv_sigma2.w};
  const float C = control_cost_sum<M, kUpdateThreads>(U, T, lam, is2, sh_s, sh_c);
  const int k = blockIdx.x * kUpdateThreads + threadIdx.x;
  if (k < K) costs[k] = C + s_part[k];
}

// ---------------------------------------------------------------------------
// Weights and update (Eq. 36-37, 49), split over K.
//
// With rho = min_k S~_k (published by the rollout) the unnormalised weights
// e_k = exp((rho - S~_k)/lambda) are formed in registers.  The partial body
// of chunk c (NT * VPT 16-byte vectors of each step-major noise row) and
// steps j_begin .. j_end-1 writes
//   N_c[j][i] = sum_{k in c} e_k delta_eff[j][k][i]
// to partial[(c*T + j)*M + i]; the block that owns the first steps of a
// chunk also writes Z_c = sum_{k in c} e_k and the e_k themselves.  The
// combine body sums the chunks in chunk order: Z = sum_c Z_c,
// dU = sum_c N_c / Z, U += alpha dU; it then emits u0 and shifts the sequence
// when asked, writes the free-energy diagnostics, advances the iteration
// counter and re-arms the running minimum.  This is Eq. 37 with the
// normalisation applied once at the end.  Each lane accumulates its share of
// a row (up to 64 products at K = 65536) in plain float32 fused
// multiply-adds; the lanes' sums, the chunk partials, Z and the group sums
// are merged with compensated (TwoSum) additions.  Every order is fixed, so
// the result does not depend on scheduling.  Data that other blocks of the
// same launch wrote is read through L2 (ld.global.cg).
// ---------------------------------------------------------------------------
struct UpdateArgs {
  const void* noise;
  const float* s_part;
  // partial records [nb][2 + T*M] = (rho_b, Z_b, N_b[T][M]) of rollout blocks
  // or rollout shards, summed bps records per chunk (record source only)
  const float* rec;
  int nb, bps;
  int rho_from_rec;   // rho = min over the records' rho_b (else the running minimum)
  float* export_out;  // non-NULL: write the combined record (rho, Z, N) instead of updating U
  int K, Kpad, T, rows;
  float inv_lam, lam, alpha;
  float inv_sigma2[4];
  int chunks, groups;
  float* partial;  // [chunks][T][M]
  float* zpart;    // [groups][chunks] (one launch) or [chunks]
  unsigned* gdone;  // [groups] completion tickets of the step groups
  float* edge;     // [groups][M] shifted first-row values of each group
  float* cpart;    // [groups] control cost of each group's rows
  float* e_out;    // [Kpad] or NULL
  float* U;        // [T][M]
  float* u0_out;   // [M] or NULL
  float* diag;     // rho, Z, F
  int* status;
  unsigned* done;
  uint32_t* rho_key;       // running minimum of this iteration's costs
  uint32_t* rho_key_next;  // the next iteration's, re-armed here (or NULL)
  uint32_t* it;
  uint32_t it_advance;
  int shift;
  int need_final;  // run the final body even when every cost is finite
  float u_init[4];
};

// Loads of a partial body that do not depend on rho, issued early so that
// their latency overlaps other work: the first batch of 16-byte vectors of
// the warp's first row, and the chunk's first costs S~_k.
template <bool BF16, int M, int VPT, int NT>
struct UpdatePrefetch {
  // 16-byte loads per lane in flight: with one vector per thread a warp's
  // whole row of the chunk (256 vectors) is one batch, loaded up front
  static constexpr int kB = VPT == 1 ? 8 : 4;
  static constexpr int kWT = chunk_rollouts<BF16, M, VPT, NT>() / NT;  // costs per thread
  static constexpr int kWB = kWT < 8 ? kWT : 8;                        // of them, loaded up front
  uint4 q[kB];
  float s[kWB];
};

template <bool BF16, int M, int VPT, int NT, class PF>
__device__ __forceinline__ void update_prefetch_noise(const UpdateArgs& a, int chunk, int j_begin,
                                                      int j_end, PF& pf) {
  constexpr int E = BF16 ? 8 : 4;
  constexpr int CV = NT * VPT;
  const int lane = threadIdx.x & 31, j_first = j_begin + (threadIdx.x >> 5);
  const int nvec = a.Kpad * M / E;
  const int v0 = chunk * CV;
  const int nvc = min(CV, nvec - v0);
  if (j_first < j_end) {
    const uint4* row = reinterpret_cast<const uint4*>(a.noise) + (size_t)j_first * nvec + v0;
#pragma unroll
    for (int h = 0; h < PF::kB; ++h) {
      const int v = lane + 32 * h;
      pf.q[h] = v < nvc ? __ldcs(row + v) : make_uint4(0u, 0u, 0u, 0u);
    }
  }
}

template <bool BF16, int M, int VPT, int NT, class PF>
__device__ __forceinline__ void update_prefetch_costs(const UpdateArgs& a, int chunk, PF& pf) {
  constexpr int RPV = (BF16 ? 8 : 4) / M;
  constexpr int CV = NT * VPT;
  const int v0 = chunk * CV;
  const int nr = min(CV, a.Kpad * M / (BF16 ? 8 : 4) - v0) * RPV;  // rollouts of the chunk
#pragma unroll
  for (int t = 0; t < PF::kWB; ++t) {
    const int r = threadIdx.x + t * NT;
    pf.s[t] = r < nr ? __ldcg(a.s_part + v0 * RPV + r) : 0.0f;
  }
}

template <bool BF16, int M, int VPT, int NT, class PF, class SH>
__device__ __forceinline__ void update_partial_body(const UpdateArgs& a, float rho, int chunk,
                                                    int j_begin, int j_end, bool write_e, float* zdst,
                                                    PF& pf, SH& sh) {
  constexpr int E = BF16 ? 8 : 4;  // elements per 16-byte vector
  constexpr int RPV = E / M;       // rollouts per vector
  constexpr int W = NT / 32;
  constexpr int CV = NT * VPT;     // vectors per chunk
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nvec = a.Kpad * M / E;
  const int v0 = chunk * CV;
  const int nvc = min(CV, nvec - v0);  // vectors of this chunk
  constexpr int B = PF::kB;            // 16-byte loads in flight per lane
  const uint4* nv = reinterpret_cast<const uint4*>(a.noise);
  const int j_first = j_begin + wid;  // its first batch is in pf.q
  uint4* q = pf.q;
  // the chunk's weights, once, into shared memory (all loads of a thread
  // are independent, so they are in flight together)
  float zs = 0.0f, zc = 0.0f;
  const int nr = nvc * RPV;
#pragma unroll
  for (int t = 0; t < PF::kWT; ++t) {
    const int r = tid + t * NT;
    float sv;
    if (t < PF::kWB) sv = pf.s[t < PF::kWB ? t : 0];
    else sv = r < nr ? __ldcg(a.s_part + v0 * RPV + r) : 0.0f;
    if (r < nr) {
      const float e = expf((rho - sv) * a.inv_lam);
      sh.e[r] = e;
      if (write_e && a.e_out) a.e_out[v0 * RPV + r] = e;
      two_sum_acc(zs, zc, e);
    }
  }
  if (zdst) {
    const float z = block_sum2<NT>(zs, zc, sh.sh_s, sh.sh_c);  // its barriers publish sh.e
    if (tid == 0) *zdst = z;
  } else {
    __syncthreads();
  }
  // every warp reduces whole rows of the chunk: no block barrier per row, and
  // each lane keeps B independent 16-byte loads in flight
  for (int j = j_first; j < j_end; j += W) {
    const uint4* row = nv + (size_t)j * nvec + v0;
    float acc[M];
#pragma unroll
    for (int i = 0; i < M; ++i) acc[i] = 0.0f;
    for (int base = 0; base < nvc; base += 32 * B) {
      if (j != j_first || base != 0) {
#pragma unroll
        for (int h = 0; h < B; ++h) {
          const int v = base + lane + 32 * h;
          q[h] = v < nvc ? __ldcs(row + v) : make_uint4(0u, 0u, 0u, 0u);
        }
      }
#pragma unroll
      for (int h = 0; h < B; ++h) {
        const int v = base + lane + 32 * h;
        if (v >= nvc) continue;
        float val[E];
        if constexpr (BF16) {
          const uint32_t wd[4] = {q[h].x, q[h].y, q[h].z, q[h].w};
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            val[2 * t] = __uint_as_float(wd[t] << 16);
            val[2 * t + 1] = __uint_as_float(wd[t] & 0xffff0000u);
          }
        } else {
          val[0] = __uint_as_float(q[h].x);
          val[1] = __uint_as_float(q[h].y);
          val[2] = __uint_as_float(q[h].z);
          val[3] = __uint_as_float(q[h].w);
        }
        float ew[RPV];
        if constexpr (RPV == 1) {
          ew[0] = sh.e[v];
        } else if constexpr (RPV == 2) {
          const float2 t = reinterpret_cast<const float2*>(sh.e)[v];
          ew[0] = t.x;
          ew[1] = t.y;
        } else {
#pragma unroll
          for (int t = 0; t < RPV / 4; ++t) {
            const float4 w4 = reinterpret_cast<const float4*>(sh.e)[v * (RPV / 4) + t];
            ew[4 * t] = w4.x;
            ew[4 * t + 1] = w4.y;
            ew[4 * t + 2] = w4.z;
            ew[4 * t + 3] = w4.w;
          }
        }
#pragma unroll
        for (int q2 = 0; q2 < E; ++q2) acc[q2 % M] = fmaf(ew[q2 / M], val[q2], acc[q2 % M]);
      }
    }
#pragma unroll
    for (int i = 0; i < M; ++i) {
      float c = 0.0f;
      warp_sum2(acc[i], c);
      if (lane == 0) a.partial[((size_t)chunk * a.T + j) * M + i] = acc[i] + c;
    }
  }
}

// Partial body over partial records (Eq. 37 split over rollout blocks or
// shards): record b holds rho_b = min S~ over its rollouts, Z_b =
// sum exp(-(S~_k - rho_b)/lambda) and N_b[j][i] = sum e_k delta_eff[j][k][i]
// with the same e_k.  With s_b = exp(-(rho_b - rho)/lambda) the shift-
// invariant rescaling gives Z_c = sum_b s_b Z_b and N_c = sum_b s_b N_b over
// the chunk's records b in [c*bps, c*bps + bps), written like the streaming
// partial body's output, so the group combine and final body are shared.
template <int M, int NT, class SH>
__device__ __forceinline__ void update_partial_records(const UpdateArgs& a, float rho, int chunk,
                                                       int j_begin, int j_end, float* zdst, SH& sh) {
  constexpr int GM = (NT / 32) * M;  // outputs of a full step group
  constexpr int PS = NT / GM;        // partial sums per output
  const int tid = threadIdx.x;
  const size_t R = 2 + (size_t)a.T * M;  // record stride
  const int b0 = chunk * a.bps, b1 = min(a.nb, b0 + a.bps);
  const int nbc = b1 - b0;
  float zs = 0.0f, zc = 0.0f;
  for (int i = tid; i < nbc; i += NT) {
    const float rb = __ldcg(a.rec + (size_t)(b0 + i) * R);
    const float zb = __ldcg(a.rec + (size_t)(b0 + i) * R + 1);
    const float sc = rb < INFINITY ? expf((rho - rb) * a.inv_lam) : 0.0f;  // rho <= rb
    sh.e[i] = sc;
    two_sum_acc(zs, zc, sc * zb);
  }
  if (zdst) {
    const float z = block_sum2<NT>(zs, zc, sh.sh_s, sh.sh_c);  // its barriers publish sh.e
    if (tid == 0) *zdst = z;
  } else {
    __syncthreads();
  }
  const int o = tid % GM, p = tid / GM;
  const int G = (j_end - j_begin) * M;
  float sv = 0.0f, cv = 0.0f;
  if (o < G)
    for (int i = p; i < nbc; i += PS)
      two_sum_acc(sv, cv, sh.e[i] * __ldcg(a.rec + (size_t)(b0 + i) * R + 2 + (size_t)j_begin * M + o));
  sh.red[tid] = sv + cv;
  __syncthreads();
  if (tid < G) {
    float ts = 0.0f, tc = 0.0f;
#pragma unroll
    for (int q = 0; q < PS; ++q) two_sum_acc(ts, tc, sh.red[q * GM + tid]);
    a.partial[((size_t)chunk * a.T + j_begin) * M + tid] = ts + tc;
  }
}

template <int M, int NT, class SH>
__device__ __forceinline__ void update_combine_body(const UpdateArgs& a, bool ok, float rho,
                                                    int chunks, SH& sh) {
  const int tid = threadIdx.x;
  const int TM = a.T * M;
  float Z = 0.0f, C = 0.0f;
  if (ok) {
    // the rollout-independent cost of the controls that were rolled out
    C = control_cost_sum<M, NT>(a.U, a.T, a.lam, a.inv_sigma2, sh.sh_s, sh.sh_c);
    float zs = 0.0f, zc = 0.0f;
    for (int c = tid; c < chunks; c += NT) two_sum_acc(zs, zc, __ldcg(a.zpart + c));
    Z = block_sum2<NT>(zs, zc, sh.sh_s, sh.sh_c);
    const float inv_Z = 1.0f / Z;
    // One block-wide slice at a time: every thread reads its old U entry and
    // forms the updated value; with the MPC shift, the value is written one
    // step earlier (entry idx - M; the first step's value is u0) after a
    // barrier, so no thread overwrites an entry another thread has yet to
    // read, and no entry written here is read back.
    for (int base = 0; base < TM; base += NT) {
      const int idx = base + tid;
      float v = 0.0f;
      if (idx < TM) {
        float s = 0.0f, c = 0.0f;
        int ch = 0;
        for (; ch + 4 <= chunks; ch += 4) {  // four loads in flight
          float p[4];
#pragma unroll
          for (int h = 0; h < 4; ++h) p[h] = __ldcg(a.partial + (size_t)(ch + h) * TM + idx);
#pragma unroll
          for (int h = 0; h < 4; ++h) two_sum_acc(s, c, p[h]);
        }
        for (; ch < chunks; ++ch) two_sum_acc(s, c, __ldcg(a.partial + (size_t)ch * TM + idx));
        v = __ldcg(a.U + idx) + a.alpha * ((s + c) * inv_Z);
      }
      if (a.shift) {
        __syncthreads();
        if (idx < TM) {
          if (idx >= M) a.U[idx - M] = v;
          else if (a.u0_out) a.u0_out[idx] = v;
          if (idx >= TM - M) a.U[idx] = a.u_init[idx - (TM - M)];
        }
        __syncthreads();
      } else if (idx < TM) {
        a.U[idx] = v;
      }
    }
  } else {
    if (a.shift && a.u0_out && tid < M) a.u0_out[tid] = __ldcg(a.U + tid);
  }
  if (tid == 0) {
    if (ok) {
      const float rf = rho + C;
      a.diag[0] = rf;
      a.diag[1] = Z;
      a.diag[2] = rf * a.inv_lam - logf(Z / (float)a.K);
    } else {
      *a.status = kStatusNonFinite;
    }
    *a.it = *a.it + a.it_advance;
    *a.rho_key = kKeyEmpty;
  }
}

// Combine of step group g in the one-launch update, run by the last block of
// the group to finish its partial sums: for the group's rows (one per warp
// of a block, rows * M <= 32 outputs) N = sum_c partial[c], then
// U_j <- U_j + alpha N_j / Z (Eq. 37 with the normalisation of Eq. 36), and
// with the MPC shift the value of row j goes to row j - 1; the group's first
// row goes to u0 (group 0) or to edge[g], written into the last row of group
// g - 1 by the final block.  Also the control cost of the group's old rows.
// Every block of a group computed the same z_c, so every group (and the final
// block) obtains the same Z.
template <int M, int NT, class SH>
__device__ __forceinline__ void update_group_combine(const UpdateArgs& a, int g, SH& sh) {
  constexpr int G = (NT / 32) * M;  // outputs of a group
  constexpr int P = NT / G;         // partial sums per output
  static_assert(G <= 32, "a group's outputs are handled by one warp");
  const int tid = threadIdx.x;
  const int TM = a.T * M;
  const int o = tid % G, p = tid / G;
  const int idx = g * a.rows * M + o;
  float s = 0.0f, c = 0.0f;
  if (idx < TM) {
#pragma unroll 4
    for (int ch = p; ch < a.chunks; ch += P) two_sum_acc(s, c, __ldcg(a.partial + (size_t)ch * TM + idx));
  }
  float zs = 0.0f, zc = 0.0f;
  for (int ch = tid; ch < a.chunks; ch += NT) two_sum_acc(zs, zc, __ldcg(a.zpart + (size_t)g * a.chunks + ch));
  sh.e[tid] = s + c;
  const float Z = block_sum2<NT>(zs, zc, sh.sh_s, sh.sh_c);  // its barriers publish sh.e
  if (tid < G) {  // warp 0
    float ns = 0.0f, nc = 0.0f;
#pragma unroll 4
    for (int q = 0; q < P; ++q) two_sum_acc(ns, nc, sh.e[q * G + tid]);
    float v = 0.0f, cs = 0.0f;
    if (idx < TM) {
      const float uo = __ldcg(a.U + idx);
      v = uo + a.alpha * ((ns + nc) * (1.0f / Z));
      cs = 0.5f * a.lam * (uo * a.inv_sigma2[tid % M] * uo);
    }
    __syncwarp(G == 32 ? 0xffffffffu : ((1u << G) - 1u));
    // every read of the group's old rows is done before any write below
    if (idx < TM && a.export_out) {
      a.export_out[2 + idx] = ns + nc;  // the combined N, not divided by Z
    } else if (idx < TM) {
      if (a.shift) {
        if (tid >= M) a.U[idx - M] = v;
        else if (g == 0) {
          if (a.u0_out) a.u0_out[tid] = v;
        } else {
          a.edge[g * M + tid] = v;
        }
        if (idx >= TM - M) a.U[idx] = a.u_init[idx - (TM - M)];
      } else {
        a.U[idx] = v;
      }
    }
    sh.e[tid] = cs;
  }
  __syncthreads();
  if (tid == 0) {
    float s2 = 0.0f, c2 = 0.0f;
    for (int q = 0; q < G; ++q) two_sum_acc(s2, c2, sh.e[q]);
    a.cpart[g] = s2 + c2;
  }
}

// Final block of the one-launch update: the control cost C over all groups,
// the shifted edge rows, the diagnostics (rho~ = rho + C, Z, free energy
// F = rho~/lambda - ln(Z/K) of Eq. 36), the counter advance and re-arming of
// the running minimum.
template <int M, int NT, class SH>
__device__ __forceinline__ void update_final_body(const UpdateArgs& a, bool ok, float rho, SH& sh) {
  const int tid = threadIdx.x;
  float C = 0.0f, Z = 0.0f;
  if (ok) {
    float cs = 0.0f, cc = 0.0f;
    for (int g = tid; g < a.groups; g += NT) two_sum_acc(cs, cc, __ldcg(a.cpart + g));
    C = block_sum2<NT>(cs, cc, sh.sh_s, sh.sh_c);
    float zs = 0.0f, zc = 0.0f;
    for (int ch = tid; ch < a.chunks; ch += NT) two_sum_acc(zs, zc, __ldcg(a.zpart + ch));
    Z = block_sum2<NT>(zs, zc, sh.sh_s, sh.sh_c);
    if (a.shift && !a.export_out)
      for (int q = tid; q < (a.groups - 1) * M; q += NT) {
        const int g = 1 + q / M, i = q % M;
        a.U[(size_t)(g * a.rows - 1) * M + i] = __ldcg(a.edge + g * M + i);
      }
  } else if (a.export_out) {
    for (int idx = tid; idx < a.T * M; idx += NT) a.export_out[2 + idx] = 0.0f;
  } else if (a.shift && a.u0_out && tid < M) {
    a.u0_out[tid] = __ldcg(a.U + tid);
  }
  if (tid == 0) {
    if (ok) {
      const float rf = rho + C;
      a.diag[0] = rf;
      a.diag[1] = Z;
      a.diag[2] = rf * a.inv_lam - logf(Z / (float)a.K);
      a.diag[3] = rho;
    } else if (!a.export_out) {
      *a.status = kStatusNonFinite;  // an exported shard may have no finite cost
    }
    if (a.export_out) {
      a.export_out[0] = ok ? rho : INFINITY;
      a.export_out[1] = ok ? Z : 0.0f;
    }
    *a.it = *a.it + a.it_advance;
    *a.rho_key = kKeyEmpty;
  }
}

// One launch: block (c, g) runs the partial body for chunk c and the rows of
// step group g, then takes its group's completion ticket (one atomic per
// block, no waiting); the last block of a group combines the group's rows and
// takes the launch's ticket, and the last group runs the final body.  The
// tickets are re-armed by their last holders.  An intermediate iteration of
// an MPC step (no shift, no counter advance, every cost finite) needs no
// final body: its diagnostics are overwritten by the next iteration.
// SRC = 0: the partial body streams the stored perturbations (chunks of
// rollouts); SRC = 1: it rescales and sums partial records (chunks of
// records).
template <bool BF16, int M, int VPT, int SRC>
__global__ void __launch_bounds__(kUpdateThreads, VPT == 1 ? 4 : 6) update_kernel(const UpdateArgs a) {
  constexpr int kECap = chunk_rollouts<BF16, M, VPT, kUpdateThreads>();
  __shared__ UpdateShared<kUpdateThreads, kECap, SRC == 1> sh;
  MJ_CHECK(blockDim.x == kUpdateThreads && (int)gridDim.x == a.chunks && (int)gridDim.y == a.groups &&
               a.rows == kUpdateThreads / 32 && a.rows * M <= 32 && a.Kpad % 32 == 0 &&
               (SRC == 0 ? (int)blockIdx.x * kUpdateThreads * VPT < a.Kpad * M / (BF16 ? 8 : 4)
                         : (a.bps <= kECap && (int)blockIdx.x * a.bps < a.nb)),
           a.status);
  griddep_launch_dependents();
  const int g = blockIdx.y;
  const int j_begin = g * a.rows;
  const int j_end = min(a.T, j_begin + a.rows);
  // The update is launched as an ordinary dependent of the rollout, so the
  // wait returns at once; it keeps the kernel correct as a programmatic
  // dependent too (nothing before it may write global memory).  The rollout
  // of the next iteration is launched as a programmatic dependent of this
  // kernel and waits for its completion before it writes anything.
  griddep_wait();
  // the next iteration's running minimum: its last reader (the previous
  // update) has finished, and its next writer (the next rollout) writes it
  // only after this kernel has completed
  if (a.rho_key_next && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0)
    *a.rho_key_next = kKeyEmpty;
  float rho;
  bool ok;
  if constexpr (SRC == 0) {
    UpdatePrefetch<BF16, M, VPT, kUpdateThreads> pf;
    update_prefetch_noise<BF16, M, VPT, kUpdateThreads>(a, blockIdx.x, j_begin, j_end, pf);
    update_prefetch_costs<BF16, M, VPT, kUpdateThreads>(a, blockIdx.x, pf);
    const uint32_t key = __ldcg(a.rho_key);
    ok = key < kKeyInf;  // at least one finite cost
    rho = ok ? key_to_float(key) : 0.0f;
    if (ok) {
      update_partial_body<BF16, M, VPT, kUpdateThreads>(
          a, rho, blockIdx.x, j_begin, j_end, g == 0, a.zpart + (size_t)g * a.chunks + blockIdx.x, pf, sh);
    }
  } else {
    if (a.rho_from_rec) {
      float r = INFINITY;
      const size_t R = 2 + (size_t)a.T * M;
      for (int b = threadIdx.x; b < a.nb; b += kUpdateThreads) r = fminf(r, __ldcg(a.rec + (size_t)b * R));
      r = fminf(r, __shfl_xor_sync(0xffffffffu, r, 16));
      r = fminf(r, __shfl_xor_sync(0xffffffffu, r, 8));
      r = fminf(r, __shfl_xor_sync(0xffffffffu, r, 4));
      r = fminf(r, __shfl_xor_sync(0xffffffffu, r, 2));
      r = fminf(r, __shfl_xor_sync(0xffffffffu, r, 1));
      if ((threadIdx.x & 31) == 0) sh.red[threadIdx.x >> 5] = r;
      __syncthreads();
      if (threadIdx.x == 0) {
        float m = INFINITY;
        for (int w = 0; w < kUpdateThreads / 32; ++w) m = fminf(m, sh.red[w]);
        sh.rho = m;
      }
      __syncthreads();
      rho = sh.rho;
      ok = rho < INFINITY;
    } else {
      const uint32_t key = __ldcg(a.rho_key);
      ok = key < kKeyInf;
      rho = ok ? key_to_float(key) : 0.0f;
    }
    if (ok) {
      update_partial_records<M, kUpdateThreads>(a, rho, blockIdx.x, j_begin, j_end,
                                                a.zpart + (size_t)g * a.chunks + blockIdx.x, sh);
    }
  }
  // the barrier orders the block's stores before thread 0's fence and
  // ticket; each winner fences again before reading what the others wrote
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    sh.ticket = atomicAdd(a.gdone + g, 1u);
  }
  __syncthreads();
  if (sh.ticket != gridDim.x - 1) return;
  __threadfence();
  if (ok) update_group_combine<M, kUpdateThreads>(a, g, sh);
  if (ok && !a.need_final) {  // an intermediate iteration: U is final here
    if (threadIdx.x == 0) a.gdone[g] = 0u;
    return;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a.gdone[g] = 0u;
    __threadfence();
    sh.ticket = atomicAdd(a.done, 1u);
  }
  __syncthreads();
  if (sh.ticket != gridDim.y - 1) return;
  __threadfence();
  update_final_body<M, kUpdateThreads>(a, ok, rho, sh);
  if (threadIdx.x == 0) *a.done = 0u;
}

// Small problems (the perturbations of one iteration within kSmallMaxBytes,
// Kpad <= kSmallMaxK, T*M <= kSmallMaxTM): the whole update (Eq. 35-37) in
// one block of kSmallThreads threads, with no tickets and no partial sums in
// global memory, so its latency is one pass over the perturbations rather
// than a chain of barriers, atomics and second reads.  The block forms
// e_k = exp(-(S~_k - rho)/lambda) for every rollout in shared memory with
// their compensated sum Z, then each warp reduces whole rows j of delta_eff
// (N_j[i] = sum_k e_k delta_eff[j][k][i], per-lane products, compensated
// shuffle sums), and after a barrier every thread updates its entries of U
// (U_j <- U_j + alpha N_j / Z; with the MPC shift, row j's value goes to row
// j - 1, the first to u0, the last row to u_init).  Diagnostics, the status
// word, the counter advance and the re-arming of the running minima as in
// the one-launch update.  The plain source only (no records, no export).
constexpr int kSmallThreads = 1024;
constexpr int kSmallMaxK = 8192;
constexpr int kSmallMaxTM = 2048;
constexpr size_t kSmallMaxBytes = 256u * 1024u;

template <bool BF16, int M>
__global__ void __launch_bounds__(kSmallThreads, 1) update_small_kernel(const UpdateArgs a) {
  constexpr int NT = kSmallThreads;
  constexpr int E = BF16 ? 8 : 4;  // elements per 16-byte vector
  constexpr int RPV = E / M;       // rollouts per vector
  constexpr int B = 4;             // 16-byte loads per lane in flight
  __shared__ __align__(16) float e[kSmallMaxK];
  __shared__ float nsum[kSmallMaxTM];
  __shared__ float sh_s[NT / 32], sh_c[NT / 32];
  MJ_CHECK(blockDim.x == NT && gridDim.x == 1 && gridDim.y == 1 && a.Kpad <= kSmallMaxK &&
               a.T * M <= kSmallMaxTM && a.Kpad % 32 == 0 && !a.export_out && !a.rec,
           a.status);
  griddep_launch_dependents();
  griddep_wait();
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int TM = a.T * M;
  if (a.rho_key_next && tid == 0) *a.rho_key_next = kKeyEmpty;
  const uint32_t key = __ldcg(a.rho_key);
  const bool ok = key < kKeyInf;  // at least one finite cost
  const float rho = ok ? key_to_float(key) : 0.0f;
  // the rollout-independent cost of the controls that were rolled out
  const float C = control_cost_sum<M, NT>(a.U, a.T, a.lam, a.inv_sigma2, sh_s, sh_c);
  float Z = 0.0f;
  if (ok) {
    float zs = 0.0f, zc = 0.0f;
    for (int k = tid; k < a.Kpad; k += NT) {
      const float ev = expf((rho - __ldcg(a.s_part + k)) * a.inv_lam);
      e[k] = ev;
      two_sum_acc(zs, zc, ev);
    }
    Z = block_sum2<NT>(zs, zc, sh_s, sh_c);  // its barriers publish e
    const int nvec = a.Kpad * M / E;
    const uint4* nv = reinterpret_cast<const uint4*>(a.noise);
    for (int j = wid; j < a.T; j += NT / 32) {
      const uint4* row = nv + (size_t)j * nvec;
      float acc[M];
#pragma unroll
      for (int i = 0; i < M; ++i) acc[i] = 0.0f;
      for (int base = 0; base < nvec; base += 32 * B) {
        uint4 q[B];
#pragma unroll
        for (int h = 0; h < B; ++h) {
          const int v = base + lane + 32 * h;
          q[h] = v < nvec ? __ldcs(row + v) : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int h = 0; h < B; ++h) {
          const int v = base + lane + 32 * h;
          if (v >= nvec) continue;
          float val[E];
          if constexpr (BF16) {
            const uint32_t wd[4] = {q[h].x, q[h].y, q[h].z, q[h].w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              val[2 * t] = __uint_as_float(wd[t] << 16);
              val[2 * t + 1] = __uint_as_float(wd[t] & 0xffff0000u);
            }
          } else {
            val[0] = __uint_as_float(q[h].x);
            val[1] = __uint_as_float(q[h].y);
            val[2] = __uint_as_float(q[h].z);
            val[3] = __uint_as_float(q[h].w);
          }
          float ew[RPV];  // the weights of the vector's rollouts
          if constexpr (RPV == 1) {
            ew[0] = e[v];
          } else if constexpr (RPV == 2) {
            const float2 t2 = reinterpret_cast<const float2*>(e)[v];
            ew[0] = t2.x;
            ew[1] = t2.y;
          } else {
#pragma unroll
            for (int t = 0; t < RPV / 4; ++t) {
              const float4 t4 = reinterpret_cast<const float4*>(e)[v * (RPV / 4) + t];
              ew[4 * t] = t4.x;
              ew[4 * t + 1] = t4.y;
              ew[4 * t + 2] = t4.z;
              ew[4 * t + 3] = t4.w;
            }
          }
#pragma unroll
          for (int q2 = 0; q2 < E; ++q2) acc[q2 % M] = fmaf(ew[q2 / M], val[q2], acc[q2 % M]);
        }
      }
#pragma unroll
      for (int i = 0; i < M; ++i) {
        float c = 0.0f;
        warp_sum2(acc[i], c);
        if (lane == 0) nsum[j * M + i] = acc[i] + c;
      }
    }
    __syncthreads();
    // every new value before any write: with the shift a row's value goes
    // to the row before it
    const float inv_Z = 1.0f / Z;
    float v0 = 0.0f, v1 = 0.0f;
    if (tid < TM) v0 = __ldcg(a.U + tid) + a.alpha * (nsum[tid] * inv_Z);
    if (tid + NT < TM) v1 = __ldcg(a.U + tid + NT) + a.alpha * (nsum[tid + NT] * inv_Z);
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int idx = tid + h * NT;
      const float v = h ? v1 : v0;
      if (idx >= TM) continue;
      if (a.shift) {
        if (idx >= M) a.U[idx - M] = v;
        else if (a.u0_out) a.u0_out[idx] = v;
        if (idx >= TM - M) a.U[idx] = a.u_init[idx - (TM - M)];
      } else {
        a.U[idx] = v;
      }
    }
  } else if (a.shift && a.u0_out && tid < M) {
    a.u0_out[tid] = __ldcg(a.U + tid);
  }
  if (tid == 0) {
    if (ok) {
      const float rf = rho + C;
      a.diag[0] = rf;
      a.diag[1] = Z;
      a.diag[2] = rf * a.inv_lam - logf(Z / (float)a.K);
      a.diag[3] = rho;
    } else {
      *a.status = kStatusNonFinite;
    }
    *a.it = *a.it + a.it_advance;
    *a.rho_key = kKeyEmpty;
  }
}

// w_k = exp((rho - S~_k)/lambda) / Z for the weights getter (the e_k of the
// update, normalised), from the costs and the diagnostics (Z, raw rho).
static __global__ void weights_kernel(const float* __restrict__ s_part, const float* __restrict__ diag,
                                      float inv_lam, int K, float* __restrict__ w) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < K) w[k] = expf((diag[3] - s_part[k]) * inv_lam) / diag[1];
}

}  // namespace mj
