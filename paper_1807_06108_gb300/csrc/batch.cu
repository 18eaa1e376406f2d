// batch.cu -- the batched form: many independent, uneven MPC instances (mixed
// plants, K, T, iteration counts) solved by ONE persistent kernel per batched
// step, replayed from a CUDA graph.
//
// The host builds a static work list of items
//   R(i, r, t)  rollout tile t (NT rollouts) of instance i, iteration r
//   W(i, r, c, g) weighted-sum partial of chunk c, step group g
//   C(i, r)     combine: weights normalisation, U update, shift on the last
//               iteration, diagnostics, counter
// ordered by iteration round, longest rollouts first, so that every item
// depends only on items earlier in the list: R(i, r) on C(i, r-1), W(i, r) on
// all R(i, r), C(i, r) on all W(i, r).  Blocks of the persistent grid claim
// items in list order with one atomic; a claimed item is always held by a
// running block, so the earliest unfinished item can always proceed and the
// schedule cannot deadlock.  A block whose dependency is not yet met waits on
// the instance's completion counter with a bounded spin (2 s of wall time);
// on expiry it raises MPPI_ETIMEOUT in the batch status word and every block
// stops claiming work.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"
#include "kernels.cuh"

namespace mj {
namespace {

constexpr int kBatchVPT = 4;         // 16-byte vectors per thread in a W item
constexpr int kBatchMaxRows = 16;    // steps per W item
constexpr int kStateStride = 12;     // x0s [n][12]
constexpr int kControlStride = 4;    // u0s [n][4]

// kItemStall waits on a counter that nothing increments (the failure-path
// test hook of mppi_batch_inject_stall).
enum : uint32_t { kItemR = 0, kItemW = 1, kItemC = 2, kItemStall = 3 };

struct WorkItem {
  uint32_t type;
  uint32_t inst;
  uint32_t r;
  uint32_t a;  // R: tile; W: chunk
  uint32_t b;  // W: step group
};

// Everything the persistent kernel needs about one instance.
struct BatchInst {
  DevProblem P;
  int iters;
  int tiles;   // rollout tiles of NT rollouts
  int chunks;  // W chunks
  int groups;  // W step groups
  int rows;    // steps per W group
  float* x0;
  float* U;
  void* noise;
  float* s_part;
  float* e;
  float* partial;
  float* zpart;
  float* diag;
  uint32_t* rho_key;
  uint32_t* it;
  float* u0;
  unsigned* done_R;  // [iters]
  unsigned* done_W;  // [iters]
  unsigned* done_C;  // [iters]
};

struct BatchArgs {
  const BatchInst* inst;
  const WorkItem* items;
  int n_items;
  unsigned* next;  // work claim counter
  int* status;     // batch status word
  int* abort;      // set when a wait expires
  const unsigned* never;  // a counter that stays 0
};

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned load_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0 waits until *ctr >= target (bounded); returns false on expiry or
// when another block has aborted.
__device__ bool wait_counter(const unsigned* ctr, unsigned target, const BatchArgs& a) {
  const uint64_t t0 = global_ns();
  unsigned sleep_ns = 32;
  while (load_acquire(ctr) < target) {
    if (*(volatile int*)a.abort) return false;
    if (global_ns() - t0 > 2000000000ull) {
      atomicExch(a.status, (int)MPPI_ETIMEOUT);
      atomicExch(a.abort, 1);
      return false;
    }
    __nanosleep(sleep_ns);
    if (sleep_ns < 1024) sleep_ns <<= 1;
  }
  return true;
}

__device__ __forceinline__ UpdateArgs update_args(const BatchInst& I, int r) {
  const DevProblem& P = I.P;
  UpdateArgs u;
  u.noise = I.noise;
  u.s_part = I.s_part;
  u.rec = nullptr;  // the batched items stream the perturbations
  u.nb = 0;
  u.bps = 0;
  u.rho_from_rec = 0;
  u.export_out = nullptr;
  u.K = P.K;
  u.Kpad = P.Kpad;
  u.T = P.T;
  u.rows = I.rows;
  u.inv_lam = P.inv_lam;
  u.lam = P.lam;
  u.alpha = P.alpha * powf(P.alpha_decay, (float)r);
  for (int i = 0; i < 4; ++i) {
    u.inv_sigma2[i] = P.inv_sigma2[i];
    u.u_init[i] = P.u_init[i];
  }
  u.chunks = I.chunks;
  u.groups = I.groups;
  u.partial = I.partial;
  u.zpart = I.zpart;
  u.gdone = nullptr;  // the work list orders the combine after every W item
  u.edge = nullptr;
  u.cpart = nullptr;
  u.e_out = I.e;
  u.U = I.U;
  const bool last = r == I.iters - 1;
  u.u0_out = last ? I.u0 : nullptr;
  u.diag = I.diag;
  u.status = nullptr;  // set by the caller
  u.done = nullptr;
  u.rho_key = I.rho_key;
  u.rho_key_next = nullptr;
  u.need_final = 1;
  u.it = I.it;
  u.it_advance = last ? (uint32_t)I.iters : 0u;
  u.shift = last ? 1 : 0;
  return u;
}

template <int NT, bool BF16, int SYS, int CH>
__device__ void run_rollout_item(const BatchInst& I, int r, int tile) {
  const DevProblem& P = I.P;
  const int k = tile * NT + threadIdx.x;
  // NT and Kpad are multiples of 32, so the k < Kpad test keeps whole warps
  if (k < P.Kpad)
    fused_rollout_thread<SYS, BF16, false, true, CH>(P, I.x0, I.U, __ldcg(I.it) + (uint32_t)r, k, I.s_part,
                                                     I.noise, I.rho_key, nullptr, nullptr);
}

// NT: rollouts per rollout item (and threads per block); CH: steps per
// unrolled chunk of a rollout item (4 or 8).
template <int NT, bool BF16, int CH>
__global__ void __launch_bounds__(NT) batch_kernel(const BatchArgs a) {
  // one shared scratch, viewed per channel count
  __shared__ __align__(16) unsigned char sh_raw[
      sizeof(UpdateShared<NT, chunk_rollouts<BF16, 4, kBatchVPT, NT>()>) >
              sizeof(UpdateShared<NT, chunk_rollouts<BF16, 1, kBatchVPT, NT>()>)
          ? sizeof(UpdateShared<NT, chunk_rollouts<BF16, 4, kBatchVPT, NT>()>)
          : sizeof(UpdateShared<NT, chunk_rollouts<BF16, 1, kBatchVPT, NT>()>)];
  auto& sh4 = *reinterpret_cast<UpdateShared<NT, chunk_rollouts<BF16, 4, kBatchVPT, NT>()>*>(sh_raw);
  auto& sh1 = *reinterpret_cast<UpdateShared<NT, chunk_rollouts<BF16, 1, kBatchVPT, NT>()>*>(sh_raw);
  __shared__ int item_sh;
  __shared__ int go_sh;
  for (;;) {
    if (threadIdx.x == 0) {
      const int idx = *(volatile int*)a.abort ? a.n_items : (int)atomicAdd(a.next, 1u);
      item_sh = idx;
      bool go = idx < a.n_items;
      if (go) {
        const WorkItem w = a.items[idx];
        const BatchInst& I = a.inst[w.inst];
        if (w.type == kItemStall) {
          go = wait_counter(a.never, 1u, a);
        } else if (w.type == kItemR) {
          if (w.r > 0) go = wait_counter(I.done_C + w.r - 1, 1u, a);
        } else if (w.type == kItemW) {
          go = wait_counter(I.done_R + w.r, (unsigned)I.tiles, a);
        } else {
          go = wait_counter(I.done_W + w.r, (unsigned)(I.chunks * I.groups), a);
        }
        if (go) __threadfence();
      }
      go_sh = go ? 1 : 0;
    }
    __syncthreads();
    if (!go_sh) return;
    const WorkItem w = a.items[item_sh];
    const BatchInst& I = a.inst[w.inst];
    const int r = (int)w.r;
    unsigned* signal;
    if (w.type == kItemR) {
      if (I.P.system == 0) run_rollout_item<NT, BF16, 0, CH>(I, r, (int)w.a);
      else run_rollout_item<NT, BF16, 1, CH>(I, r, (int)w.a);
      signal = I.done_R + r;
    } else {
      UpdateArgs u = update_args(I, r);
      u.status = a.status;
      const uint32_t key = __ldcg(I.rho_key);
      const bool ok = key < kKeyInf;
      const float rho = ok ? key_to_float(key) : 0.0f;
      if (w.type == kItemW) {
        if (ok) {
          const int j_begin = (int)w.b * I.rows;
          const int j_end = min(I.P.T, j_begin + I.rows);
          float* zdst = w.b == 0 ? u.zpart + w.a : nullptr;
          if (I.P.m == 4) {
            UpdatePrefetch<BF16, 4, kBatchVPT, NT> pf;
            update_prefetch_noise<BF16, 4, kBatchVPT, NT>(u, (int)w.a, j_begin, j_end, pf);
            update_prefetch_costs<BF16, 4, kBatchVPT, NT>(u, (int)w.a, pf);
            update_partial_body<BF16, 4, kBatchVPT, NT>(u, rho, (int)w.a, j_begin, j_end, w.b == 0, zdst, pf,
                                                        sh4);
          } else {
            UpdatePrefetch<BF16, 1, kBatchVPT, NT> pf;
            update_prefetch_noise<BF16, 1, kBatchVPT, NT>(u, (int)w.a, j_begin, j_end, pf);
            update_prefetch_costs<BF16, 1, kBatchVPT, NT>(u, (int)w.a, pf);
            update_partial_body<BF16, 1, kBatchVPT, NT>(u, rho, (int)w.a, j_begin, j_end, w.b == 0, zdst, pf,
                                                        sh1);
          }
        }
        signal = I.done_W + r;
      } else {
        if (I.P.m == 4) update_combine_body<4, NT>(u, ok, rho, I.chunks, sh4);
        else update_combine_body<1, NT>(u, ok, rho, I.chunks, sh1);
        signal = I.done_C + r;
      }
    }
    // publish completion: the barrier orders the block's stores before
    // thread 0's fence and counter increment
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(signal, 1u);
    }
  }
}

}  // namespace
}  // namespace mj

using namespace mj;

struct mppi_batch {
  int n = 0;
  int block = 128;  // rollouts per block (persistent block size)
  int chunk = 4;    // steps per unrolled chunk of a rollout item
  std::vector<mppi_jump_config> cfgs;
  std::vector<int> iters;
  std::vector<BatchInst> hinst;
  std::vector<WorkItem> hitems;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* arena = nullptr;  // device: everything below
  BatchInst* d_inst = nullptr;
  WorkItem* d_items = nullptr;
  unsigned* counters = nullptr;  // next, then done_R/W/C of every instance
  size_t counters_bytes = 0;
  uint32_t* rho_keys = nullptr;  // n contiguous running minima
  int* status = nullptr;         // status, abort
  float* x0s = nullptr;          // [n][12]
  float* u0s = nullptr;          // [n][4]
  float* h_io = nullptr;         // pinned host staging
  int grid = 0;
  bool stall = false;  // test hook: prepend an item whose dependency never completes
  long long steps_per_solve = 0;
  cudaGraphExec_t graph = nullptr;
  char err[256] = {0};
};

namespace {

mppi_status bfail(mppi_batch* b, cudaError_t e, const char* what) {
  snprintf(b->err, sizeof(b->err), "%s: %s", what, cudaGetErrorString(e));
  return MPPI_ECUDA;
}

#define BCK(call, what)                                     \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return bfail(b, e_, what);       \
  } while (0)

template <int NT, bool BF16, int CH>
cudaError_t launch_batch(mppi_batch* b, cudaStream_t s) {
  BatchArgs a;
  a.inst = b->d_inst;
  a.items = b->d_items;
  a.n_items = (int)b->hitems.size();
  a.next = b->counters;
  a.status = b->status;
  a.abort = b->status + 1;
  a.never = (const unsigned*)(b->status + 2);
  batch_kernel<NT, BF16, CH><<<b->grid, NT, 0, s>>>(a);
  return cudaGetLastError();
}

template <int NT, bool BF16>
cudaError_t launch_batch_c(mppi_batch* b, cudaStream_t s) {
  return b->chunk == 8 ? launch_batch<NT, BF16, 8>(b, s) : launch_batch<NT, BF16, 4>(b, s);
}

cudaError_t launch_batch_any(mppi_batch* b, cudaStream_t s) {
  const bool bf16 = b->cfgs[0].noise_dtype == MPPI_NOISE_BF16;
  switch (b->block) {
    case 64: return bf16 ? launch_batch_c<64, true>(b, s) : launch_batch_c<64, false>(b, s);
    case 256: return bf16 ? launch_batch_c<256, true>(b, s) : launch_batch_c<256, false>(b, s);
    default: return bf16 ? launch_batch_c<128, true>(b, s) : launch_batch_c<128, false>(b, s);
  }
}

template <int NT, bool BF16>
int occupancy_of(int chunk) {
  int per_sm = 0;
  if (chunk == 8)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<NT, BF16, 8>, NT, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<NT, BF16, 4>, NT, 0);
  return per_sm;
}

int occupancy(int block, int chunk, bool bf16) {
  switch (block) {
    case 64: return bf16 ? occupancy_of<64, true>(chunk) : occupancy_of<64, false>(chunk);
    case 256: return bf16 ? occupancy_of<256, true>(chunk) : occupancy_of<256, false>(chunk);
    default: return bf16 ? occupancy_of<128, true>(chunk) : occupancy_of<128, false>(chunk);
  }
}

// Geometry and work list for the current block size; instance buffers are
// sized for the smallest block (most chunks) at creation.
void build_items(mppi_batch* b) {
  const int NT = b->block;
  b->hitems.clear();
  if (b->stall) b->hitems.push_back({kItemStall, 0, 0, 0, 0});
  int max_iters = 0;
  for (int i = 0; i < b->n; ++i) {
    BatchInst& I = b->hinst[i];
    const DevProblem& P = I.P;
    const int E = P.noise_bf16 ? 8 : 4;
    const int nvec = P.Kpad * P.m / E;
    I.tiles = (P.Kpad + NT - 1) / NT;
    I.chunks = (nvec + NT * kBatchVPT - 1) / (NT * kBatchVPT);
    I.rows = kBatchMaxRows;
    I.groups = (P.T + I.rows - 1) / I.rows;
    max_iters = std::max(max_iters, I.iters);
  }
  // instances grouped by plant (the costlier quadrotor first), each group by
  // decreasing horizon: the longest rollouts start first, and blocks that run
  // at the same time mostly execute the same plant's code, which keeps the
  // instruction cache warm
  std::vector<int> order(b->n);
  for (int i = 0; i < b->n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const DevProblem& px = b->hinst[x].P;
    const DevProblem& py = b->hinst[y].P;
    if (px.system != py.system) return px.system > py.system;
    return px.T > py.T;
  });
  for (int r = 0; r < max_iters; ++r) {
    for (int i : order)
      if (r < b->hinst[i].iters)
        for (int t = 0; t < b->hinst[i].tiles; ++t) b->hitems.push_back({kItemR, (uint32_t)i, (uint32_t)r, (uint32_t)t, 0});
    for (int i : order)
      if (r < b->hinst[i].iters)
        for (int g = 0; g < b->hinst[i].groups; ++g)
          for (int c = 0; c < b->hinst[i].chunks; ++c)
            b->hitems.push_back({kItemW, (uint32_t)i, (uint32_t)r, (uint32_t)c, (uint32_t)g});
    for (int i : order)
      if (r < b->hinst[i].iters) b->hitems.push_back({kItemC, (uint32_t)i, (uint32_t)r, 0, 0});
  }
}

mppi_status upload_plan(mppi_batch* b) {
  build_items(b);
  if (b->d_items) cudaFree(b->d_items);
  b->d_items = nullptr;
  BCK(cudaMalloc(&b->d_items, sizeof(WorkItem) * b->hitems.size()), "work list");
  BCK(cudaMemcpyAsync(b->d_items, b->hitems.data(), sizeof(WorkItem) * b->hitems.size(),
                      cudaMemcpyHostToDevice, b->stream),
      "work list");
  BCK(cudaMemcpyAsync(b->d_inst, b->hinst.data(), sizeof(BatchInst) * b->n, cudaMemcpyHostToDevice,
                      b->stream),
      "instances");
  int sms = 152, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int occ = std::max(1, occupancy(b->block, b->chunk, b->cfgs[0].noise_dtype == MPPI_NOISE_BF16));
  b->grid = sms * occ;
  BCK(cudaStreamSynchronize(b->stream), "plan upload");
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  return MPPI_OK;
}

mppi_status capture(mppi_batch* b) {
  NvtxRange nv("mppi batch capture");
  if (b->graph) return MPPI_OK;
  cudaGraph_t g = nullptr;
  BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  cudaError_t e = cudaMemsetAsync(b->counters, 0, b->counters_bytes, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->rho_keys, 0xff, sizeof(uint32_t) * b->n, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->status, 0, 3 * sizeof(int), b->stream);
  if (e == cudaSuccess) e = launch_batch_any(b, b->stream);
  cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return bfail(b, e, "batch capture");
  }
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return bfail(b, e, "batch instantiate");
  return MPPI_OK;
}

}  // namespace

extern "C" {

const char* mppi_batch_last_error(const mppi_batch* b) { return b ? b->err : "no batch"; }

mppi_status mppi_batch_destroy(mppi_batch* b) {
  if (!b) return MPPI_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->d_items) cudaFree(b->d_items);
  if (b->arena) cudaFree(b->arena);
  if (b->h_io) cudaFreeHost(b->h_io);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return MPPI_OK;
}

mppi_status mppi_batch_create(const mppi_jump_config* cfgs, const int32_t* iters, int32_t n,
                              void* stream, mppi_batch** out) {
  if (!out || !cfgs || !iters || n < 1) return MPPI_EINVAL;
  *out = nullptr;
  mppi_batch* b = new (std::nothrow) mppi_batch();
  if (!b) return MPPI_ENOMEM;
  b->n = n;
  b->cfgs.assign(cfgs, cfgs + n);
  b->iters.assign(iters, iters + n);
  b->hinst.resize(n);
  for (int i = 0; i < n; ++i) {
    BatchInst& I = b->hinst[i];
    std::memset(&I, 0, sizeof(I));
    mppi_status st = pack_problem(&cfgs[i], &I.P, b->err);
    if (st != MPPI_OK || iters[i] < 1 || cfgs[i].noise_dtype != cfgs[0].noise_dtype) {
      if (st == MPPI_OK)
        snprintf(b->err, sizeof(b->err), "instance %d: iterations must be >= 1 and every instance "
                 "must use the same noise dtype", i);
      mppi_batch_destroy(b);
      return MPPI_EINVAL;
    }
    I.iters = iters[i];
  }
  // device layout: instances, counters, running minima, status, x0s, u0s,
  // then per-instance buffers (sized for 64-thread tiles: the most chunks)
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes);
    return o;
  };
  const size_t o_inst = take(sizeof(BatchInst) * n);
  size_t n_counters = 1;
  for (int i = 0; i < n; ++i) n_counters += 3 * (size_t)iters[i];
  const size_t o_cnt = take(sizeof(unsigned) * n_counters);
  const size_t o_rho = take(sizeof(uint32_t) * n);
  const size_t o_status = take(sizeof(int) * 4);
  const size_t o_x0 = take(sizeof(float) * kStateStride * n);
  const size_t o_u0 = take(sizeof(float) * kControlStride * n);
  std::vector<size_t> o_U(n), o_noise(n), o_s(n), o_e(n), o_part(n), o_z(n), o_diag(n), o_it(n);
  for (int i = 0; i < n; ++i) {
    const DevProblem& P = b->hinst[i].P;
    const int E = P.noise_bf16 ? 8 : 4;
    const int nvec = P.Kpad * P.m / E;
    const int max_chunks = (nvec + 64 * kBatchVPT - 1) / (64 * kBatchVPT);
    o_U[i] = take(sizeof(float) * (size_t)P.T * P.m);
    o_noise[i] = take((size_t)(P.noise_bf16 ? 2 : 4) * P.T * P.Kpad * P.m);
    o_s[i] = take(sizeof(float) * P.Kpad);
    o_e[i] = take(sizeof(float) * P.Kpad);
    o_part[i] = take(sizeof(float) * (size_t)max_chunks * P.T * P.m);
    o_z[i] = take(sizeof(float) * max_chunks);
    o_diag[i] = take(sizeof(float) * 4);
    o_it[i] = take(sizeof(uint32_t) * 4);
  }
  cudaError_t e = cudaSuccess;
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    b->own_stream = e == cudaSuccess;
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->arena, off);
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_io, sizeof(float) * (kStateStride + kControlStride) * n + 64);
  if (e != cudaSuccess) {
    const bool oom = e == cudaErrorMemoryAllocation;
    snprintf(b->err, sizeof(b->err), "allocation: %s", cudaGetErrorString(e));
    mppi_batch_destroy(b);
    return oom ? MPPI_ENOMEM : MPPI_ECUDA;
  }
  char* A = (char*)b->arena;
  b->d_inst = (BatchInst*)(A + o_inst);
  b->counters = (unsigned*)(A + o_cnt);
  b->counters_bytes = sizeof(unsigned) * n_counters;
  b->rho_keys = (uint32_t*)(A + o_rho);
  b->status = (int*)(A + o_status);
  b->x0s = (float*)(A + o_x0);
  b->u0s = (float*)(A + o_u0);
  unsigned* cnt = b->counters + 1;
  for (int i = 0; i < n; ++i) {
    BatchInst& I = b->hinst[i];
    I.x0 = b->x0s + kStateStride * i;
    I.u0 = b->u0s + kControlStride * i;
    I.U = (float*)(A + o_U[i]);
    I.noise = A + o_noise[i];
    I.s_part = (float*)(A + o_s[i]);
    I.e = (float*)(A + o_e[i]);
    I.partial = (float*)(A + o_part[i]);
    I.zpart = (float*)(A + o_z[i]);
    I.diag = (float*)(A + o_diag[i]);
    I.it = (uint32_t*)(A + o_it[i]);
    I.rho_key = b->rho_keys + i;
    I.done_R = cnt;
    I.done_W = cnt + I.iters;
    I.done_C = cnt + 2 * I.iters;
    cnt += 3 * I.iters;
    b->steps_per_solve += (long long)I.P.K * I.P.T * I.iters;
  }
  mppi_status st = MPPI_OK;
  e = cudaMemsetAsync(b->arena, 0, off, b->stream);
  if (e != cudaSuccess) st = bfail(b, e, "clear");
  // U = u_init for every instance
  for (int i = 0; i < n && st == MPPI_OK; ++i) {
    const DevProblem& P = b->hinst[i].P;
    std::vector<float> hU((size_t)P.T * P.m);
    for (int j = 0; j < P.T; ++j)
      for (int c = 0; c < P.m; ++c) hU[(size_t)j * P.m + c] = cfgs[i].u_init[c];
    e = cudaMemcpyAsync(b->hinst[i].U, hU.data(), sizeof(float) * hU.size(), cudaMemcpyHostToDevice,
                        b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) st = bfail(b, e, "controls");
  }
  if (st == MPPI_OK) st = upload_plan(b);
  if (st != MPPI_OK) {
    mppi_batch_destroy(b);
    return st;
  }
  *out = b;
  return MPPI_OK;
}

mppi_status mppi_batch_info(mppi_batch* b, int64_t* steps_per_solve, int32_t* n_items,
                            int32_t* grid) {
  if (!b) return MPPI_EINVAL;
  if (steps_per_solve) *steps_per_solve = b->steps_per_solve;
  if (n_items) *n_items = (int32_t)b->hitems.size();
  if (grid) *grid = b->grid;
  return MPPI_OK;
}

mppi_status mppi_batch_set_tuning(mppi_batch* b, int32_t block) {
  if (!b) return MPPI_EINVAL;
  return mppi_batch_set_tile(b, block, b->chunk);
}

mppi_status mppi_batch_set_tile(mppi_batch* b, int32_t block, int32_t chunk) {
  if (!b || (block != 64 && block != 128 && block != 256) || (chunk != 4 && chunk != 8)) return MPPI_EINVAL;
  BCK(cudaStreamSynchronize(b->stream), "set_tile");
  b->block = block;
  b->chunk = chunk;
  return upload_plan(b);
}

mppi_status mppi_batch_get_tile(mppi_batch* b, int32_t* block_host, int32_t* chunk_host) {
  if (!b || !block_host || !chunk_host) return MPPI_EINVAL;
  *block_host = b->block;
  *chunk_host = b->chunk;
  return MPPI_OK;
}

mppi_status mppi_batch_inject_stall(mppi_batch* b, int32_t on) {
  if (!b) return MPPI_EINVAL;
  BCK(cudaStreamSynchronize(b->stream), "inject_stall");
  b->stall = on != 0;
  return upload_plan(b);
}

mppi_status mppi_batch_get_tuning(mppi_batch* b, int32_t* block) {
  if (!b || !block) return MPPI_EINVAL;
  *block = b->block;
  return MPPI_OK;
}

mppi_status mppi_batch_step_async(mppi_batch* b, const float* x0s, float* u0s) {
  NvtxRange nv("mppi batch step");
  if (!b || !x0s) return MPPI_EINVAL;
  mppi_status st = capture(b);
  if (st != MPPI_OK) return st;
  BCK(cudaMemcpyAsync(b->x0s, x0s, sizeof(float) * kStateStride * b->n, cudaMemcpyDefault, b->stream),
      "x0s copy");
  BCK(cudaGraphLaunch(b->graph, b->stream), "batch launch");
  if (u0s)
    BCK(cudaMemcpyAsync(u0s, b->u0s, sizeof(float) * kControlStride * b->n, cudaMemcpyDefault,
                        b->stream),
        "u0s copy");
  return MPPI_OK;
}

mppi_status mppi_batch_sync(mppi_batch* b) {
  if (!b) return MPPI_EINVAL;
  int* hs = (int*)(b->h_io + (kStateStride + kControlStride) * b->n);
  BCK(cudaMemcpyAsync(hs, b->status, sizeof(int), cudaMemcpyDeviceToHost, b->stream), "status");
  BCK(cudaStreamSynchronize(b->stream), "sync");
  if (hs[0] == MPPI_ETIMEOUT) {
    snprintf(b->err, sizeof(b->err), "a work-list dependency wait expired");
    return MPPI_ETIMEOUT;
  }
  if (hs[0] != 0) {
    snprintf(b->err, sizeof(b->err), "an instance had only non-finite rollout costs");
    return (mppi_status)hs[0];
  }
  return MPPI_OK;
}

mppi_status mppi_batch_step(mppi_batch* b, const float* x0s_host, float* u0s_host) {
  if (!b || !x0s_host || !u0s_host) return MPPI_EINVAL;
  float* hx = b->h_io;
  float* hu = b->h_io + kStateStride * b->n;
  std::memcpy(hx, x0s_host, sizeof(float) * kStateStride * b->n);
  mppi_status st = mppi_batch_step_async(b, hx, hu);
  if (st != MPPI_OK) return st;
  st = mppi_batch_sync(b);
  std::memcpy(u0s_host, hu, sizeof(float) * kControlStride * b->n);
  return st;
}

mppi_status mppi_batch_get_controls(mppi_batch* b, int32_t i, float* U) {
  if (!b || !U || i < 0 || i >= b->n) return MPPI_EINVAL;
  const DevProblem& P = b->hinst[i].P;
  BCK(cudaMemcpyAsync(U, b->hinst[i].U, sizeof(float) * P.T * P.m, cudaMemcpyDefault, b->stream),
      "get_controls");
  BCK(cudaStreamSynchronize(b->stream), "get_controls");
  return MPPI_OK;
}

mppi_status mppi_batch_set_controls(mppi_batch* b, int32_t i, const float* U) {
  if (!b || !U || i < 0 || i >= b->n) return MPPI_EINVAL;
  const DevProblem& P = b->hinst[i].P;
  BCK(cudaMemcpyAsync(b->hinst[i].U, U, sizeof(float) * P.T * P.m, cudaMemcpyDefault, b->stream),
      "set_controls");
  BCK(cudaStreamSynchronize(b->stream), "set_controls");
  return MPPI_OK;
}

mppi_status mppi_batch_get_iteration(mppi_batch* b, int32_t i, uint32_t* it_host) {
  if (!b || !it_host || i < 0 || i >= b->n) return MPPI_EINVAL;
  BCK(cudaMemcpyAsync(it_host, b->hinst[i].it, sizeof(uint32_t), cudaMemcpyDefault, b->stream),
      "get_iteration");
  BCK(cudaStreamSynchronize(b->stream), "get_iteration");
  return MPPI_OK;
}

mppi_status mppi_batch_autotune(mppi_batch* b, const float* x0s, int32_t reps, int32_t* best_block,
                                float* best_ms) {
  if (!b || !x0s || reps < 1) return MPPI_EINVAL;
  // save every instance's controls and counter, time each block size, restore
  std::vector<std::vector<float>> Us(b->n);
  std::vector<uint32_t> its(b->n);
  for (int i = 0; i < b->n; ++i) {
    const DevProblem& P = b->hinst[i].P;
    Us[i].resize((size_t)P.T * P.m);
    mppi_status st = mppi_batch_get_controls(b, i, Us[i].data());
    if (st == MPPI_OK) st = mppi_batch_get_iteration(b, i, &its[i]);
    if (st != MPPI_OK) return st;
  }
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0), "events");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return bfail(b, cudaErrorUnknown, "events");
  }
  const int cands[6][2] = {{128, 4}, {64, 4}, {256, 4}, {128, 8}, {64, 8}, {256, 8}};
  int best = b->block, best_chunk = b->chunk;
  float best_t = 1e30f;
  mppi_status st = MPPI_OK;
  for (const auto& c : cands) {
    st = mppi_batch_set_tile(b, c[0], c[1]);
    if (st == MPPI_OK) st = mppi_batch_step_async(b, x0s, nullptr);
    if (st == MPPI_OK && cudaEventRecord(e0, b->stream) != cudaSuccess) st = MPPI_ECUDA;
    for (int r = 0; r < reps && st == MPPI_OK; ++r) st = mppi_batch_step_async(b, x0s, nullptr);
    float ms = 0.0f;
    if (st == MPPI_OK && (cudaEventRecord(e1, b->stream) != cudaSuccess ||
                          cudaEventSynchronize(e1) != cudaSuccess ||
                          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      st = MPPI_ECUDA;
    if (st == MPPI_OK) st = mppi_batch_sync(b);
    if (st != MPPI_OK) break;
    ms /= (float)reps;
    if (ms < best_t) {
      best_t = ms;
      best = c[0];
      best_chunk = c[1];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != MPPI_OK) return st;
  st = mppi_batch_set_tile(b, best, best_chunk);
  for (int i = 0; i < b->n && st == MPPI_OK; ++i) {
    st = mppi_batch_set_controls(b, i, Us[i].data());
    if (st == MPPI_OK) {
      cudaError_t e = cudaMemcpyAsync(b->hinst[i].it, &its[i], sizeof(uint32_t), cudaMemcpyHostToDevice,
                                      b->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
      if (e != cudaSuccess) st = bfail(b, e, "restore");
    }
  }
  if (st != MPPI_OK) return st;
  if (best_block) *best_block = best;
  if (best_ms) *best_ms = best_t;
  return MPPI_OK;
}

}  // extern "C"
