// iteration.cu -- configuration packing and the launches of one MPPI
// iteration (rollout, softmin, split-K update, combine) for a single problem.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <utility>

#include "internal.h"
#include "kernels.cuh"
#include "launch.cuh"

namespace mj {

mppi_status fail(char* buf, mppi_status st, const char* fmt, ...) {
  if (buf) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 256, fmt, ap);
    va_end(ap);
  }
  return st;
}

static bool finite_pos(float v) { return std::isfinite(v) && v > 0.0f; }

mppi_status pack_problem(const mppi_jump_config* cfg, DevProblem* P, char* msg) {
  if (!cfg || !P) return fail(msg, MPPI_EINVAL, "null configuration");
  if (cfg->system != MPPI_CARTPOLE && cfg->system != MPPI_QUADROTOR)
    return fail(msg, MPPI_EINVAL, "unknown system %d", cfg->system);
  const int n = state_dim(cfg->system), m = control_dim(cfg->system);
  if (cfg->K < 1 || cfg->K > (1 << 24)) return fail(msg, MPPI_EINVAL, "K=%d out of [1, 2^24]", cfg->K);
  if (cfg->T < 1 || cfg->T > 4096) return fail(msg, MPPI_EINVAL, "T=%d out of [1, 4096]", cfg->T);
  if (!finite_pos(cfg->dt)) return fail(msg, MPPI_EINVAL, "dt must be finite and > 0");
  if (!finite_pos(cfg->lambda)) return fail(msg, MPPI_EINVAL, "lambda must be finite and > 0");
  if (!finite_pos(cfg->c)) return fail(msg, MPPI_EINVAL, "c must be finite and > 0");
  if (!std::isfinite(cfg->alpha)) return fail(msg, MPPI_EINVAL, "alpha must be finite");
  if (!(cfg->alpha_decay >= 0.0f && cfg->alpha_decay <= 1.0f))
    return fail(msg, MPPI_EINVAL, "alpha_decay must be in [0, 1]");
  for (int i = 0; i < m; ++i)
    if (!finite_pos(cfg->sigma[i])) return fail(msg, MPPI_EINVAL, "sigma[%d] must be finite and > 0", i);
  if (cfg->count_law != MPPI_COUNT_POISSON && cfg->count_law != MPPI_COUNT_BERNOULLI)
    return fail(msg, MPPI_EINVAL, "unknown count law %d", cfg->count_law);
  if (cfg->mark_law != MPPI_MARK_NORMAL && cfg->mark_law != MPPI_MARK_LAPLACE)
    return fail(msg, MPPI_EINVAL, "unknown mark law %d", cfg->mark_law);
  if (cfg->jump_channel != MPPI_JUMP_STATE && cfg->jump_channel != MPPI_JUMP_CONTROL)
    return fail(msg, MPPI_EINVAL, "unknown jump channel %d", cfg->jump_channel);
  if (cfg->noise_dtype != MPPI_NOISE_F32 && cfg->noise_dtype != MPPI_NOISE_BF16)
    return fail(msg, MPPI_EINVAL, "unknown noise dtype %d", cfg->noise_dtype);
  if (cfg->q < 0 || cfg->q > 4) return fail(msg, MPPI_EINVAL, "q=%d out of [0, 4]", cfg->q);
  if (cfg->jump_channel == MPPI_JUMP_CONTROL && cfg->q != m)
    return fail(msg, MPPI_EINVAL, "control-channel jumps need q == m (%d)", m);
  if (cfg->jump_channel == MPPI_JUMP_STATE)
    for (int c = 0; c < cfg->q; ++c)
      if (cfg->jump_rows[c] < 0 || cfg->jump_rows[c] >= n)
        return fail(msg, MPPI_EINVAL, "jump_rows[%d]=%d out of [0, %d)", c, cfg->jump_rows[c], n);
  for (int c = 0; c < cfg->q; ++c)
    if (!(std::isfinite(cfg->mark_scale[c]) && cfg->mark_scale[c] >= 0.0f))
      return fail(msg, MPPI_EINVAL, "mark_scale[%d] must be finite and >= 0", c);
  for (int i = 0; i < m; ++i)
    if (!std::isfinite(cfg->u_init[i])) return fail(msg, MPPI_EINVAL, "u_init must be finite");

  std::memset(P, 0, sizeof(*P));
  int32_t nmax = 0;
  mppi_status st = mppi_jump_count_table(cfg->jump_rate, cfg->dt, cfg->count_law, P->thr, &nmax);
  if (st != MPPI_OK)
    return fail(msg, st, "jump rate %g with dt %g gives no valid count table", (double)cfg->jump_rate,
                (double)cfg->dt);
  P->system = cfg->system;
  P->K = cfg->K;
  P->Kpad = pad_k(cfg->K);
  P->T = cfg->T;
  P->n = n;
  P->m = m;
  P->q = cfg->q;
  P->count_law = cfg->count_law;
  P->mark_law = cfg->mark_law;
  P->jump_channel = cfg->jump_channel;
  P->nmax = nmax;
  P->noise_bf16 = cfg->noise_dtype == MPPI_NOISE_BF16;
  // the plant's velocity rows get a specialised jump update
  P->jump_default = 0;
  if (cfg->jump_channel == MPPI_JUMP_STATE) {
    if (cfg->system == MPPI_CARTPOLE)
      P->jump_default = cfg->q == 2 && cfg->jump_rows[0] == 1 && cfg->jump_rows[1] == 3;
    else
      P->jump_default = cfg->q == 3 && cfg->jump_rows[0] == 3 && cfg->jump_rows[1] == 4 &&
                        cfg->jump_rows[2] == 5;
  }
  for (int c = 0; c < 4; ++c) P->jump_rows[c] = c < cfg->q ? cfg->jump_rows[c] : -1;
  P->key0 = (uint32_t)(cfg->seed & 0xffffffffull);
  P->key1 = (uint32_t)(cfg->seed >> 32);
  for (int r = 0; r < 10; ++r) {
    P->rk[2 * r] = P->key0 + (uint32_t)r * 0x9E3779B9u;
    P->rk[2 * r + 1] = P->key1 + (uint32_t)r * 0xBB67AE85u;
  }
  P->dt = cfg->dt;
  P->lam = cfg->lambda;
  P->inv_lam = (float)(1.0 / (double)cfg->lambda);
  P->is_coef = (float)(0.5 * (1.0 - 1.0 / (double)cfg->c));
  P->alpha = cfg->alpha;
  P->alpha_decay = cfg->alpha_decay == 0.0f ? 1.0f : cfg->alpha_decay;
  P->s_jump = cfg->jump_sqrt_dt ? (float)std::sqrt((double)cfg->dt) : 1.0f;
  const double sqc = std::sqrt((double)cfg->c);
  for (int i = 0; i < 4; ++i) {
    const bool on = i < m;
    P->sqc_sigma[i] = on ? (float)(sqc * (double)cfg->sigma[i]) : 0.0f;
    P->inv_sigma2[i] = on ? (float)(1.0 / ((double)cfg->sigma[i] * (double)cfg->sigma[i])) : 0.0f;
    P->u_init[i] = on ? cfg->u_init[i] : 0.0f;
    P->mark_scale[i] = i < cfg->q ? cfg->mark_scale[i] : 0.0f;
  }
  DevPlant& pl = P->pl;
  if (cfg->system == MPPI_CARTPOLE) {
    const mppi_cartpole_params& c = cfg->cartpole;
    if (!finite_pos(c.mc) || !(std::isfinite(c.mp) && c.mp >= 0.0f) || !finite_pos(c.l) ||
        !std::isfinite(c.g))
      return fail(msg, MPPI_EINVAL, "cart-pole constants must be finite (mc, l > 0, mp >= 0)");
    pl.mc = c.mc;
    pl.mp = c.mp;
    pl.l = c.l;
    pl.g = c.g;
    pl.inv_l = (float)(1.0 / (double)c.l);
    pl.mcp_g = (float)(((double)c.mc + (double)c.mp) * (double)c.g);
    for (int i = 0; i < 4; ++i) {
      pl.goal[i] = c.goal[i];
      pl.Q[i] = c.Q[i];
      pl.Qf[i] = c.Qf[i];
    }
  } else {
    const mppi_quadrotor_params& q = cfg->quadrotor;
    if (!finite_pos(q.mass) || !finite_pos(q.J[0]) || !finite_pos(q.J[1]) || !finite_pos(q.J[2]) ||
        !std::isfinite(q.arm) || !std::isfinite(q.kappa) || !std::isfinite(q.g) ||
        !(std::isfinite(q.obs_r) && q.obs_r >= 0.0f) || !std::isfinite(q.obs_cost))
      return fail(msg, MPPI_EINVAL, "quadrotor constants must be finite (mass, J > 0)");
    pl.inv_mass = (float)(1.0 / (double)q.mass);
    for (int i = 0; i < 3; ++i) {
      pl.J[i] = q.J[i];
      pl.invJ[i] = (float)(1.0 / (double)q.J[i]);
      pl.pgoal[i] = q.goal[i];
      pl.obs[i] = q.obs[i];
    }
    pl.arm = q.arm;
    pl.kappa = q.kappa;
    pl.qg = q.g;
    pl.wp = q.wp;
    pl.wv = q.wv;
    pl.weta = q.weta;
    pl.wom = q.wom;
    pl.obs_r2 = (float)((double)q.obs_r * (double)q.obs_r);
    pl.obs_cost = q.obs_cost;
  }
  return MPPI_OK;
}

// How the staged rollout applies the problem's state jumps (kJumpNone,
// kJumpDefault or kJumpRows; the sparse forms are chosen at launch).
static int jump_mode(const DevProblem& P) {
  if (P.jump_channel != MPPI_JUMP_STATE) return kJumpNone;
  return P.jump_default ? kJumpDefault : kJumpRows;
}

// Dynamic shared memory of the staged rollout: two stages of S steps of the
// block's delta_eff rows, jump-record slots (state jumps) and control rows,
// the four mbarriers and (block records) the record scratch.
static size_t staged_smem_bytes(const DevProblem& P, int block, int S, bool part) {
  return staged_smem_total(block, P.m, P.noise_bf16 ? 2 : 4, S, jump_mode(P) != kJumpNone, part);
}

cudaError_t prepare_kernels() {
  cudaError_t e = prepare_staged_dense();
  if (e == cudaSuccess) e = prepare_staged_sparse();
  return e;
}

UpdateGeom update_geometry(int Kpad, int T, int m, bool bf16, int num_sms) {
  UpdateGeom g;
  const int E = bf16 ? 8 : 4;
  const int nvec = Kpad * m / E;
  constexpr int W = kUpdateThreads / 32;  // warps of a block, one row each at a time
  const int row_sets = (T + W - 1) / W;
  // the longest chunks that still give every SM several blocks: at small K
  // each block is short, and latency (not bandwidth) sets the duration
  const int target = 4 * (num_sms > 0 ? num_sms : 152);
  g.vpt = 1;
  for (int v = 4; v >= 1; v /= 2) {
    const int chunks = (nvec + kUpdateThreads * v - 1) / (kUpdateThreads * v);
    if ((long long)chunks * row_sets >= target) {
      g.vpt = v;
      break;
    }
  }
  g.chunks = (nvec + kUpdateThreads * g.vpt - 1) / (kUpdateThreads * g.vpt);
  g.rows = W;
  g.groups = row_sets;
  return g;
}

// The rollout and the update are the sequential critical path of an MPC step;
// the noise pass of the next iteration only fills idle issue slots beside
// them.  They launch at the device's highest priority, so that the block
// scheduler places their blocks first when the two compete for SMs.  The
// rollout launches as a programmatic dependent of the update before it,
// which hides its launch latency and lets its copies of the step data start
// early (it calls griddep_wait() before it touches anything the update
// writes); the update launches as an ordinary dependent of the rollout
// (launch_hi, launch.cuh).

// Measured on GB300: the staged form (a producer warp moves the step data
// into shared memory with bulk copies) is the fastest rollout at every size;
// while the rollout blocks fit on the SMs about once, 16-step stages (one
// block per SM, see launch_staged), beyond that 8-step stages so that
// several blocks share an SM.  While blocks of 96 fit on the SMs at once,
// blocks of 96: three compute warps and the producer warp put one warp on
// each scheduler, where with 128 one compute warp shares its scheduler with
// the producer and holds the block back (quadrotor K = 4096: 0.2181 against
// 0.2225 ms per MPC step, three runs each; cart-pole K = 1000: 0.0303
// against 0.0306 ms).
RolloutTile default_tile(const DevProblem& P, int num_sms) {
  const int sms = num_sms > 0 ? num_sms : 152;
  const int blocks = (P.Kpad + 127) / 128;
  RolloutTile t;
  t.variant = 3;
  t.block = 128;
  t.chunk = blocks >= 2 * sms ? 8 : 16;
  if ((P.Kpad + 95) / 96 <= sms) t.block = 96;
  return t;
}

bool valid_tile(const RolloutTile& t) {
  if (t.block < 32 || t.block > kRolloutThreads || t.block % 32 != 0) return false;
  // fused and staged forms: steps per unrolled chunk or per stage; split
  // form: how many steps ahead its loads run
  if (t.variant == 1 || t.variant == 3 || t.variant == 4) return t.chunk == 4 || t.chunk == 8 || t.chunk == 16;
  return t.variant == 2 && (t.chunk == 2 || t.chunk == 4 || t.chunk == 8);
}

// Where the marks of state-channel jumps are drawn, and in which record form.
// While the rollout blocks fit on the SMs at once (the rollout is
// latency-bound and the noise pass runs beside it on the other SMs), the
// noise pass draws them in its own threads and writes dense records (J or
// zero for every step), which the rollout copies as whole rows: one launch
// fewer before the first rollout of a step and no per-record copies in the
// rollout's latency chain (measured on GB300: cart-pole K = 1000, T = 50 at
// 0.0360 ms per MPC step against 0.0409 ms with marks_kernel).  Beyond that
// the per-thread mark loop, run by a warp as often as its busiest lane has
// jumps, is a fifth of an issue-bound pass; there the noise pass writes jump
// masks, marks_kernel draws the marks with the warp's lanes on jumps and
// writes sparse records, and the rollout gathers only those (the dense rows
// would double the bytes it reads).
bool marks_in_noise(const DevProblem& P) {
  return P.jump_channel == MPPI_JUMP_STATE && (P.Kpad + kRolloutThreads - 1) / kRolloutThreads <= num_sms_of_current();
}

// The jump masks of sparse records, or NULL (dense records, control-channel
// jumps).
uint32_t* sparse_mask(const DevProblem& P, const IterBuffers& b) {
  return P.jump_channel == MPPI_JUMP_STATE && !marks_in_noise(P) ? b.jmask : nullptr;
}

bool has_marks_pass(const DevProblem& P) {
  return P.jump_channel == MPPI_JUMP_STATE && P.nmax > 0 && !marks_in_noise(P);
}

template <int M, bool BF16, bool DBG, bool MARKS>
static void launch_noise_t(const DevProblem& P, const IterBuffers& b, uint32_t it_off, cudaStream_t s) {
  // With sparse records the pass runs beside the rollout and update of the
  // previous iteration, in blocks of 256 threads: one retiring block leaves
  // room for a rollout block (160 threads, 48 registers each).  Measured on
  // GB300, large quadrotor, marks passes on their own branch: 0.935 ms per
  // MPC step with 256-thread blocks, 0.949 with 512; 128-thread blocks gave
  // 0.933 in a build that also had a third buffer set (each against about
  // 0.964 for the build before, on its own box), so the size is not what
  // decides the time.
  const int nt = has_marks_pass(P) ? kNoiseThreadsLarge : kNoiseThreads;
  const dim3 grid((P.Kpad + nt - 1) / nt, (P.T + 3) / 4);
  const bool sj = P.jump_channel == MPPI_JUMP_STATE;
  noise_kernel<M, BF16, DBG, MARKS><<<grid, nt, 0, s>>>(
      P, b.it, it_off, b.noise, sparse_mask(P, b), sj ? b.jrec : nullptr, marks_in_noise(P) ? 1 : 0,
      b.dbg_counts, b.dbg_J, b.status, b.arm_key);
}

template <int M, bool BF16>
static void launch_noise_m(const DevProblem& P, const IterBuffers& b, uint32_t it_off, bool dbg,
                           cudaStream_t s) {
  // the marks are drawn here for control-channel jumps (folded into
  // delta_eff), for the debug copy of J and for state-channel records of
  // small problems
  if (dbg) launch_noise_t<M, BF16, true, true>(P, b, it_off, s);
  else if (P.jump_channel == MPPI_JUMP_CONTROL || marks_in_noise(P))
    launch_noise_t<M, BF16, false, true>(P, b, it_off, s);
  else launch_noise_t<M, BF16, false, false>(P, b, it_off, s);
}

cudaError_t launch_noise(const DevProblem& P, const IterBuffers& b, uint32_t it_off, cudaStream_t s,
                         cudaStream_t s_marks, cudaEvent_t ev) {
  const bool dbg = b.dbg_counts != nullptr || b.dbg_J != nullptr;
  switch ((P.m == 4 ? 2 : 0) + (P.noise_bf16 ? 1 : 0)) {
    case 0: launch_noise_m<1, false>(P, b, it_off, dbg, s); break;
    case 1: launch_noise_m<1, true>(P, b, it_off, dbg, s); break;
    case 2: launch_noise_m<4, false>(P, b, it_off, dbg, s); break;
    default: launch_noise_m<4, true>(P, b, it_off, dbg, s); break;
  }
  // state-channel jumps of large problems: their marks into the jump records
  if (has_marks_pass(P)) {
    const int rows = P.Kpad / 32;
    const dim3 grid((rows + kMarkWarps - 1) / kMarkWarps, (P.T + 31) / 32);
    if (s_marks) {
      cudaError_t e = cudaEventRecord(ev, s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s_marks, ev, 0);
      if (e != cudaSuccess) return e;
      launch_hi(marks_kernel, grid, dim3(kMarkThreads), 0, s_marks, false, P, (const uint32_t*)b.it, it_off,
                (const uint32_t*)b.jmask, b.jrec, b.status);
    } else {
      marks_kernel<<<grid, kMarkThreads, 0, s>>>(P, b.it, it_off, b.jmask, b.jrec, b.status);
    }
  }
  return cudaGetLastError();
}

template <int SYS, bool BF16>
static void launch_seq_t(const DevProblem& P, const IterBuffers& b, const RolloutTile& tile,
                         uint32_t it_off, bool pdl, cudaStream_t s) {
  const int blocks = (P.Kpad + tile.block - 1) / tile.block;
  if (tile.chunk == 2)
    launch_hi(rollout_split_kernel<SYS, BF16, 2>, dim3(blocks), dim3(tile.block), 0, s, pdl,
        P, b.x0, b.U, b.noise, sparse_mask(P, b), b.jrec, b.s_part, b.rho_key, b.status);
  else if (tile.chunk == 8)
    launch_hi(rollout_split_kernel<SYS, BF16, 8>, dim3(blocks), dim3(tile.block), 0, s, pdl,
        P, b.x0, b.U, b.noise, sparse_mask(P, b), b.jrec, b.s_part, b.rho_key, b.status);
  else
    launch_hi(rollout_split_kernel<SYS, BF16, 4>, dim3(blocks), dim3(tile.block), 0, s, pdl,
        P, b.x0, b.U, b.noise, sparse_mask(P, b), b.jrec, b.s_part, b.rho_key, b.status);
}

static cudaError_t launch_staged(const DevProblem& P, const IterBuffers& b, const RolloutTile& tile, bool pdl,
                                 cudaStream_t s) {
  const int blocks = (P.Kpad + tile.block - 1) / tile.block;
  const bool part = tile.variant == 4;
  if (part && !b.rec) return cudaErrorInvalidValue;
  size_t smem = staged_smem_bytes(P, tile.block, tile.chunk, part);
  if (smem > (size_t)kStagedSmemMax) return cudaErrorInvalidValue;
  // While the blocks fit on the SMs at once, each reserves kStagedSmemMax of
  // shared memory (one block per SM).  Measured on GB300: with less (66 KB
  // for control-channel jumps, which need no jump records) blocks of the
  // concurrent noise pass shared the rollout's SMs, and the MPC step of the
  // K = 4096 quadrotor with control-channel jumps took 0.427 ms against
  // 0.280 ms with the reservation (0.344 ms with 100 KB).
  if (blocks <= num_sms_of_current()) smem = (size_t)kStagedSmemMax;
  const StagedLaunch L = {&P, &b, &tile, blocks, smem, pdl, s, part};
  const int jm = jump_mode(P);
  if (jm != kJumpNone && sparse_mask(P, b)) launch_staged_sparse(L, jm == kJumpDefault);
  else launch_staged_dense(L, jm);
  return cudaSuccess;
}

cudaError_t launch_rollout_seq(const DevProblem& P, const IterBuffers& b, const RolloutTile& tile,
                               uint32_t it_off, bool pdl, cudaStream_t s) {
  if (!valid_tile(tile) || tile.variant == 1) return cudaErrorInvalidValue;
  if (tile.variant >= 3) {
    const cudaError_t e = launch_staged(P, b, tile, pdl, s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
  }
  switch (P.system * 2 + (P.noise_bf16 ? 1 : 0)) {
    case 0: launch_seq_t<0, false>(P, b, tile, it_off, pdl, s); break;
    case 1: launch_seq_t<0, true>(P, b, tile, it_off, pdl, s); break;
    case 2: launch_seq_t<1, false>(P, b, tile, it_off, pdl, s); break;
    default: launch_seq_t<1, true>(P, b, tile, it_off, pdl, s); break;
  }
  return cudaGetLastError();
}

template <int SYS, bool BF16, bool DBG>
static void launch_fused_t(const DevProblem& P, const IterBuffers& b, const RolloutTile& tile,
                           uint32_t it_off, cudaStream_t s) {
  const int blocks = (P.Kpad + tile.block - 1) / tile.block;
  if (tile.chunk == 16)
    launch_hi(rollout_kernel<SYS, BF16, DBG, 16>, dim3(blocks), dim3(tile.block), 0, s, true, P, b.x0, b.U,
              b.it, it_off, b.s_part, b.noise, b.rho_key, b.dbg_counts, b.dbg_J, b.status);
  else if (tile.chunk == 8)
    launch_hi(rollout_kernel<SYS, BF16, DBG, 8>, dim3(blocks), dim3(tile.block), 0, s, true, P, b.x0, b.U,
              b.it, it_off, b.s_part, b.noise, b.rho_key, b.dbg_counts, b.dbg_J, b.status);
  else
    launch_hi(rollout_kernel<SYS, BF16, DBG, 4>, dim3(blocks), dim3(tile.block), 0, s, true, P, b.x0, b.U,
              b.it, it_off, b.s_part, b.noise, b.rho_key, b.dbg_counts, b.dbg_J, b.status);
}

cudaError_t launch_rollout(const DevProblem& P, const IterBuffers& b, const RolloutTile& tile,
                           uint32_t it_off, bool arm_min, cudaStream_t s) {
  if (!valid_tile(tile)) return cudaErrorInvalidValue;
  if (arm_min) {
    cudaError_t e = cudaMemsetAsync(b.rho_key, 0xff, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
  }
  if (tile.variant >= 2) {
    cudaError_t e = launch_noise(P, b, it_off, s);
    if (e != cudaSuccess) return e;
    // the rollout reads what the noise pass just wrote: an ordinary launch
    return launch_rollout_seq(P, b, tile, it_off, false, s);
  }
  const bool dbg = b.dbg_counts != nullptr || b.dbg_J != nullptr;
  switch (P.system * 4 + (P.noise_bf16 ? 2 : 0) + (dbg ? 1 : 0)) {
    case 0: launch_fused_t<0, false, false>(P, b, tile, it_off, s); break;
    case 1: launch_fused_t<0, false, true>(P, b, tile, it_off, s); break;
    case 2: launch_fused_t<0, true, false>(P, b, tile, it_off, s); break;
    case 3: launch_fused_t<0, true, true>(P, b, tile, it_off, s); break;
    case 4: launch_fused_t<1, false, false>(P, b, tile, it_off, s); break;
    case 5: launch_fused_t<1, false, true>(P, b, tile, it_off, s); break;
    case 6: launch_fused_t<1, true, false>(P, b, tile, it_off, s); break;
    default: launch_fused_t<1, true, true>(P, b, tile, it_off, s); break;
  }
  return cudaGetLastError();
}

template <bool BF16, int M, int VPT, int SRC>
static void launch_update_t(const UpdateArgs& a, dim3 grid, cudaStream_t s) {
  // Measured on GB300: as a programmatic dependent of the rollout, the
  // update's blocks were resident early and waited on SMs that the
  // concurrent noise pass of the next iteration could have used; an ordinary
  // launch made the MPC step 2 % faster at K = 4096 and at K = 65536.
  launch_hi(update_kernel<BF16, M, VPT, SRC>, grid, dim3(kUpdateThreads), 0, s, false, a);
}

template <bool BF16, int M>
static void launch_update_m(const UpdateArgs& a, const UpdateGeom& g, bool records, cudaStream_t s) {
  const dim3 grid(a.chunks, a.groups);
  if (records) launch_update_t<BF16, M, 1, 1>(a, grid, s);
  else if (g.vpt == 4) launch_update_t<BF16, M, 4, 0>(a, grid, s);
  else if (g.vpt == 2) launch_update_t<BF16, M, 2, 0>(a, grid, s);
  else launch_update_t<BF16, M, 1, 0>(a, grid, s);
}

int records_per_chunk(int m) {
  // every thread of a record chunk sums at most eight records (a step group
  // has 8 m outputs, so 256 / (8 m) partial sums per output)
  return 8 * (kUpdateThreads / (8 * m));
}

cudaError_t launch_update(const DevProblem& P, const IterBuffers& b, const UpdateGeom& g, int r, int shift,
                          uint32_t it_advance, float* u0, cudaStream_t s, const UpdateSource* src) {
  UpdateArgs a;
  a.noise = b.noise;
  a.s_part = b.s_part;
  a.rec = nullptr;
  a.nb = 0;
  a.bps = 0;
  a.rho_from_rec = 0;
  a.export_out = nullptr;
  a.K = P.K;
  a.Kpad = P.Kpad;
  a.T = P.T;
  a.rows = g.rows;
  a.inv_lam = P.inv_lam;
  a.lam = P.lam;
  a.alpha = (float)((double)P.alpha * std::pow((double)P.alpha_decay, (double)r));
  for (int i = 0; i < 4; ++i) a.inv_sigma2[i] = P.inv_sigma2[i];
  a.chunks = g.chunks;
  a.groups = g.groups;
  const bool records = src && src->rec;
  if (src) a.export_out = src->export_out;
  if (records) {
    a.rec = src->rec;
    a.nb = src->nb;
    a.bps = records_per_chunk(P.m);
    a.rho_from_rec = src->rho_from_rec;
    a.chunks = (a.nb + a.bps - 1) / a.bps;
    if (a.nb < 1 || a.chunks > b.max_chunks) return cudaErrorInvalidValue;
  }
  a.partial = b.partial;
  a.zpart = b.zpart;
  a.gdone = b.done + 4;
  a.edge = b.gpart;
  a.cpart = b.gpart + (size_t)g.groups * P.m;
  a.e_out = nullptr;  // the weights getter recomputes e_k from the costs
  a.U = b.U;
  a.u0_out = u0;
  a.diag = b.diag;
  a.status = b.status;
  a.done = b.done;
  a.rho_key = b.rho_key;
  a.rho_key_next = b.rho_key_next;
  a.need_final = (shift || it_advance > 0 || a.export_out) ? 1 : 0;
  a.it = b.it;
  a.it_advance = it_advance;
  a.shift = a.export_out ? 0 : shift;
  for (int i = 0; i < 4; ++i) a.u_init[i] = P.u_init[i];
  const size_t delta_bytes = (size_t)P.T * P.Kpad * P.m * (P.noise_bf16 ? 2 : 4);
  if (!records && !a.export_out && P.Kpad <= kSmallMaxK && P.T * P.m <= kSmallMaxTM &&
      delta_bytes <= kSmallMaxBytes) {
    // One block does the whole update (update_small_kernel), launched as a
    // programmatic dependent of the kernel before it: the block becomes
    // resident while the rollout runs and waits in griddep_wait(), which
    // hides the launch latency, and it holds only one SM (measured on GB300:
    // cart-pole MPC step 0.0293 -> 0.0283 ms; the same for the many-block
    // update_kernel made the K = 4096 quadrotor step 2 % slower, 0.2181 ->
    // 0.2224 ms, its waiting blocks crowding out the concurrent noise pass).
    const dim3 grid(1), block(kSmallThreads);
    if (P.m == 4) {
      if (P.noise_bf16) launch_hi(update_small_kernel<true, 4>, grid, block, 0, s, true, a);
      else launch_hi(update_small_kernel<false, 4>, grid, block, 0, s, true, a);
    } else {
      if (P.noise_bf16) launch_hi(update_small_kernel<true, 1>, grid, block, 0, s, true, a);
      else launch_hi(update_small_kernel<false, 1>, grid, block, 0, s, true, a);
    }
    return cudaGetLastError();
  }
  if (P.m == 4) {
    if (P.noise_bf16) launch_update_m<true, 4>(a, g, records, s);
    else launch_update_m<false, 4>(a, g, records, s);
  } else {
    if (P.noise_bf16) launch_update_m<true, 1>(a, g, records, s);
    else launch_update_m<false, 1>(a, g, records, s);
  }
  return cudaGetLastError();
}

cudaError_t launch_costs(const DevProblem& P, const IterBuffers& b, cudaStream_t s) {
  if (!b.costs) return cudaSuccess;
  const float4 is2 = make_float4(P.inv_sigma2[0], P.inv_sigma2[1], P.inv_sigma2[2], P.inv_sigma2[3]);
  const int blocks = (P.K + kUpdateThreads - 1) / kUpdateThreads;
  if (P.m == 4)
    costs_kernel<4><<<blocks, kUpdateThreads, 0, s>>>(b.U, P.T, P.lam, is2, b.s_part, P.K, b.costs);
  else
    costs_kernel<1><<<blocks, kUpdateThreads, 0, s>>>(b.U, P.T, P.lam, is2, b.s_part, P.K, b.costs);
  return cudaGetLastError();
}

cudaError_t launch_weights(const float* s_part, const float* diag, float inv_lam, int K, float* w,
                           cudaStream_t s) {
  weights_kernel<<<(K + 255) / 256, 256, 0, s>>>(s_part, diag, inv_lam, K, w);
  return cudaGetLastError();
}

}  // namespace mj

// Poisson / Bernoulli count thresholds (see the header): the Poisson CDF is
// summed term by term in double precision, F(n) = F(n-1) + term_n with
// term_n = term_{n-1} * mu / n, and T_n = ceil(2^32 F(n-1)).
extern "C" mppi_status mppi_jump_count_table(float jump_rate, float dt, int32_t count_law,
                                             uint32_t thr_host[MPPI_MAX_JUMPS],
                                             int32_t* nmax_host) {
  if (!thr_host || !nmax_host) return MPPI_EINVAL;
  for (int i = 0; i < MPPI_MAX_JUMPS; ++i) thr_host[i] = 0u;
  *nmax_host = 0;
  const double mu = (double)jump_rate * (double)dt;
  if (!(mu >= 0.0) || !std::isfinite(mu)) return MPPI_EINVAL;
  if (count_law == MPPI_COUNT_BERNOULLI) {
    if (!(mu < 1.0)) return MPPI_EINVAL;
    const double t = std::floor(std::ldexp(mu, 32) + 0.5);
    thr_host[0] = (uint32_t)t;
    *nmax_host = thr_host[0] > 0u ? 1 : 0;
    return MPPI_OK;
  }
  if (count_law != MPPI_COUNT_POISSON) return MPPI_EINVAL;
  double term = std::exp(-mu);
  double F = term;
  int n = 1;
  for (;; ++n) {
    const double t = std::ceil(std::ldexp(F, 32));
    if (t >= 4294967296.0) break;
    if (n > MPPI_MAX_JUMPS) return MPPI_EINVAL;
    thr_host[n - 1] = (uint32_t)t;
    term = term * mu / (double)n;
    F = F + term;
  }
  *nmax_host = n - 1;
  return MPPI_OK;
}
