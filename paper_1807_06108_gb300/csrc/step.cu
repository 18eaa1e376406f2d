// step.cu -- the compute calls of the single-problem C ABI: rollout_cost,
// update, the graph-replayed MPC step, phase timing, rollout tiles and the
// tile autotuner.
//
// The MPC step is captured once per iteration count as a CUDA graph with two
// branches: with the split or staged rollout tiles, the noise of iteration
// r+1 is drawn on the second branch (into the other buffer set) while
// iteration r is rolled out and updated on the first, so the sampling costs
// no time on the critical path; on the first branch each rollout is a
// programmatic dependent of the update before it.  Iteration r of a step uses
// the Philox stream of counter value it + r; the last update advances the
// counter by the iteration count.
#include <cstring>
#include <vector>

#include "context.h"

using namespace mj;

namespace {

// The status word of a finished step as a return code, with its message.
mppi_status status_of(mppi_jump_ctx* ctx, int st) {
  if (st == MPPI_ENONFINITE)
    snprintf(ctx->err, sizeof(ctx->err), "every rollout cost was non-finite; U left unchanged");
  else if (st == MPPI_ETIMEOUT)
    snprintf(ctx->err, sizeof(ctx->err), "a bounded device wait expired");
  else if (st == MPPI_EBOUNDS)
    snprintf(ctx->err, sizeof(ctx->err), "a kernel's launch check failed (checked build)");
  return (mppi_status)st;
}

// The update's partial source for the context's tile: the records of the
// rollout blocks (tile 4) or the stored perturbations.
UpdateSource block_records(const mppi_jump_ctx* ctx) {
  UpdateSource src = {nullptr, 0, 0, nullptr};
  if (ctx->tile.variant == 4) {
    src.rec = ctx->rec;
    src.nb = (ctx->P.Kpad + ctx->tile.block - 1) / ctx->tile.block;
  }
  return src;
}

mppi_status capture_step(mppi_jump_ctx* ctx, int iters, cudaGraphExec_t* exec) {
  NvtxRange nv("mppi step capture");
  const bool split = ctx->tile.variant >= 2;
  const size_t need_links = 3 * (size_t)iters + 2;
  while (ctx->links.size() < need_links) {
    cudaEvent_t ev;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event create");
    ctx->links.push_back(ev);
  }
  if (ctx->timing) {
    while ((int)ctx->events.size() < 3 * iters) {
      cudaEvent_t ev;
      CK(cudaEventCreate(&ev), "event create");
      ctx->events.push_back(ev);
    }
  }
  cudaEvent_t* evN = ctx->links.data();          // noise of iteration r drawn
  cudaEvent_t* evU = ctx->links.data() + iters;  // update of iteration r done
  cudaEvent_t evFork = ctx->links[2 * iters];
  cudaEvent_t* evM = ctx->links.data() + 2 * iters + 2;  // noise pass r done (marks hop)
  cudaStream_t main = ctx->stream, aux = ctx->aux;
  // Sparse jump records: each marks pass runs on a third branch at the
  // highest priority, so that the next noise pass starts on the second
  // branch as soon as the current one ends and fills the SMs beside it.
  // Measured on GB300, large quadrotor, with the per-node priorities below
  // (one box, both builds with a third noise buffer set, which the library
  // does not keep): 0.9487 ms per MPC step with the marks passes on the
  // noise branch, 0.9327 with them here.
  cudaStream_t marks = has_marks_pass(ctx->P) ? ctx->aux2 : nullptr;

  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(main, cudaStreamCaptureModeThreadLocal), "begin capture");
  // No memset nodes: the status word keeps a device-side error until a
  // synchronising call reads and clears it, and the running minimum of the
  // first iteration is re-armed by the step's first noise pass (split and
  // staged tiles; measured on GB300, the two memset nodes cost 6 us of the
  // 34 us cart-pole step) or by one memset (fused tile).
  cudaError_t e = cudaSuccess;
  if (!split) e = cudaMemsetAsync(ctx->rho_key, 0xff, sizeof(uint32_t), main);
  auto mark = [&](int idx) {
    if (ctx->timing && e == cudaSuccess)
      e = cudaEventRecordWithFlags(ctx->events[idx], main, cudaEventRecordExternal);
  };
  if (split) {
    if (e == cudaSuccess) e = cudaEventRecord(evFork, main);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(aux, evFork, 0);
    IterBuffers b0 = ctx_buffers(ctx, nullptr, 0);
    b0.arm_key = b0.rho_key;
    if (e == cudaSuccess) e = launch_noise(ctx->P, b0, 0u, aux, marks, evM[0]);
    if (e == cudaSuccess) e = cudaEventRecord(evN[0], marks ? marks : aux);
  }
  for (int r = 0; r < iters && e == cudaSuccess; ++r) {
    const IterBuffers b = ctx_buffers(ctx, nullptr, r & 1);
    const bool last = r == iters - 1;
    if (split) {
      if (r + 1 < iters) {
        // the other buffer set is free once the update of iteration r-1 is done
        if (r >= 1) e = cudaStreamWaitEvent(aux, evU[r - 1], 0);
        if (e == cudaSuccess)
          e = launch_noise(ctx->P, ctx_buffers(ctx, nullptr, (r + 1) & 1), (uint32_t)(r + 1), aux, marks,
                           evM[r + 1]);
        if (e == cudaSuccess) e = cudaEventRecord(evN[r + 1], marks ? marks : aux);
      }
      if (e == cudaSuccess) e = cudaStreamWaitEvent(main, evN[r], 0);
      mark(3 * r);
      // the noise arrives through an event (an ordinary dependency); the
      // kernel before it in this stream is the previous update
      if (e == cudaSuccess) e = launch_rollout_seq(ctx->P, b, ctx->tile, (uint32_t)r, true, main);
    } else {
      mark(3 * r);
      if (e == cudaSuccess) e = launch_rollout(ctx->P, b, ctx->tile, (uint32_t)r, false, main);
    }
    mark(3 * r + 1);
    const UpdateSource src = block_records(ctx);
    if (e == cudaSuccess)
      e = launch_update(ctx->P, b, ctx->geom, r, last ? 1 : 0, last ? (uint32_t)iters : 0u,
                        last ? ctx->u0 : nullptr, main, &src);
    mark(3 * r + 2);
    if (split && e == cudaSuccess) e = cudaEventRecord(evU[r], main);
  }
  cudaError_t e2 = cudaStreamEndCapture(main, &graph);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(ctx, e, "step capture");
  }
  cudaGraphExec_t ex = nullptr;
  // The rollout, update and marks nodes carry the highest launch priority;
  // graph replay honours per-node priorities only with this flag (without
  // it, measured on GB300, the large quadrotor's update waited about 55 us
  // per iteration behind the blocks of the concurrent noise pass).
  e = cudaGraphInstantiate(&ex, graph, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "graph instantiate");
  *exec = ex;
  return MPPI_OK;
}

mppi_status get_graph(mppi_jump_ctx* ctx, int iters, cudaGraphExec_t* exec) {
  auto it = ctx->graphs.find(iters);
  if (it != ctx->graphs.end()) {
    *exec = it->second;
    return MPPI_OK;
  }
  mppi_status st = capture_step(ctx, iters, exec);
  if (st == MPPI_OK) ctx->graphs[iters] = *exec;
  return st;
}

}  // namespace

extern "C" {

mppi_status mppi_jump_rollout_cost(mppi_jump_ctx* ctx, const float* x0, float* costs) {
  NvtxRange nv("mppi rollout_cost (A1-A2)");
  if (!ctx || !x0) return MPPI_EINVAL;
  CK(cudaMemcpyAsync(ctx->x0, x0, sizeof(float) * ctx->P.n, cudaMemcpyDefault, ctx->stream), "x0 copy");
  const IterBuffers b = ctx_buffers(ctx, costs, 0);
  CK(launch_rollout(ctx->P, b, ctx->tile, 0u, true, ctx->stream), "rollout launch");
  CK(launch_costs(ctx->P, b, ctx->stream), "costs launch");
  ctx->last_set = 0;
  return MPPI_OK;
}

mppi_status mppi_jump_update(mppi_jump_ctx* ctx) {
  NvtxRange nv("mppi update (A3-A4)");
  if (!ctx) return MPPI_EINVAL;
  const UpdateSource src = block_records(ctx);
  CK(launch_update(ctx->P, ctx_buffers(ctx, nullptr, 0), ctx->geom, 0, 0, 1u, nullptr, ctx->stream, &src),
     "update launch");
  return MPPI_OK;
}

mppi_status mppi_jump_set_rollout_offset(mppi_jump_ctx* ctx, uint32_t k_offset) {
  if (!ctx) return MPPI_EINVAL;
  if ((uint64_t)k_offset + (uint64_t)ctx->P.Kpad > 0x100000000ull)
    return fail(ctx->err, MPPI_EINVAL, "rollout offset %u + K exceeds the 32-bit rollout index", k_offset);
  CK(cudaStreamSynchronize(ctx->stream), "set_rollout_offset");
  ctx->P.k_base = k_offset;
  drop_graphs(ctx);
  return MPPI_OK;
}

mppi_status mppi_jump_rollout_partial(mppi_jump_ctx* ctx, const float* x0, float* partial) {
  NvtxRange nv("mppi rollout_partial");
  if (!ctx || !x0 || !partial) return MPPI_EINVAL;
  CK(cudaMemcpyAsync(ctx->x0, x0, sizeof(float) * ctx->P.n, cudaMemcpyDefault, ctx->stream), "x0 copy");
  const IterBuffers b = ctx_buffers(ctx, nullptr, 0);
  CK(launch_rollout(ctx->P, b, ctx->tile, 0u, true, ctx->stream), "rollout launch");
  ctx->last_set = 0;
  UpdateSource src = block_records(ctx);
  src.export_out = partial;
  CK(launch_update(ctx->P, b, ctx->geom, 0, 0, 0u, nullptr, ctx->stream, &src), "partial launch");
  return MPPI_OK;
}

mppi_status mppi_jump_apply_partials(mppi_jump_ctx* ctx, const float* partials, int32_t n_parts, int32_t r,
                                     int32_t shift, float* u0) {
  NvtxRange nv("mppi apply_partials");
  if (!ctx || !partials || n_parts < 1 || r < 0) return MPPI_EINVAL;
  if (n_parts > records_per_chunk(ctx->P.m) * ctx->max_chunks)
    return fail(ctx->err, MPPI_EINVAL, "%d partial records exceed the limit", n_parts);
  const UpdateSource src = {partials, n_parts, 1, nullptr};
  CK(launch_update(ctx->P, ctx_buffers(ctx, nullptr, 0), ctx->geom, r, shift ? 1 : 0, 1u, shift ? u0 : nullptr,
                   ctx->stream, &src),
     "apply launch");
  return MPPI_OK;
}

mppi_status mppi_jump_sync(mppi_jump_ctx* ctx) {
  if (!ctx) return MPPI_EINVAL;
  CK(cudaMemcpyAsync(ctx->h_status, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream),
     "status copy");
  CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream), "status reset");
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  return status_of(ctx, ctx->h_status[0]);
}

mppi_status mppi_jump_set_tuning(mppi_jump_ctx* ctx, const mppi_jump_tuning* tuning_host) {
  if (!ctx || !tuning_host) return MPPI_EINVAL;
  RolloutTile t;
  t.variant = tuning_host->rollout_variant;
  t.block = tuning_host->rollout_block;
  t.chunk = tuning_host->rollout_chunk;
  if (!valid_tile(t))
    return fail(ctx->err, MPPI_EINVAL, "invalid tile (variant %d, block %d, chunk %d)", t.variant,
                t.block, t.chunk);
  CK(cudaStreamSynchronize(ctx->stream), "set_tuning");
  ctx->tile = t;
  drop_graphs(ctx);
  return MPPI_OK;
}

mppi_status mppi_jump_get_tuning(mppi_jump_ctx* ctx, mppi_jump_tuning* tuning_host) {
  if (!ctx || !tuning_host) return MPPI_EINVAL;
  tuning_host->rollout_variant = ctx->tile.variant;
  tuning_host->rollout_block = ctx->tile.block;
  tuning_host->rollout_chunk = ctx->tile.chunk;
  return MPPI_OK;
}

mppi_status mppi_jump_enable_timing(mppi_jump_ctx* ctx, int32_t on) {
  if (!ctx) return MPPI_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream), "enable_timing");
  ctx->timing = on != 0;
  drop_graphs(ctx);
  ctx->timed_iters = 0;
  return MPPI_OK;
}

mppi_status mppi_jump_phase_times(mppi_jump_ctx* ctx, float out_host[2], int32_t* iters_host) {
  if (!ctx || !out_host) return MPPI_EINVAL;
  out_host[0] = out_host[1] = 0.0f;
  if (iters_host) *iters_host = 0;
  if (!ctx->timing || ctx->timed_iters == 0) return MPPI_OK;
  CK(cudaStreamSynchronize(ctx->stream), "phase_times");
  for (int r = 0; r < ctx->timed_iters; ++r) {
    float a = 0.0f, b = 0.0f;
    CK(cudaEventElapsedTime(&a, ctx->events[3 * r], ctx->events[3 * r + 1]), "elapsed");
    CK(cudaEventElapsedTime(&b, ctx->events[3 * r + 1], ctx->events[3 * r + 2]), "elapsed");
    out_host[0] += a;
    out_host[1] += b;
  }
  if (iters_host) *iters_host = ctx->timed_iters;
  return MPPI_OK;
}

mppi_status mppi_jump_step_async(mppi_jump_ctx* ctx, const float* x0, int32_t iters, float* u0) {
  NvtxRange nv("mppi step_async (graph replay)");
  if (!ctx || !x0 || iters < 1) return MPPI_EINVAL;
  cudaGraphExec_t ex;
  mppi_status st = get_graph(ctx, iters, &ex);
  if (st != MPPI_OK) return st;
  if (ctx->timing) ctx->timed_iters = iters;
  CK(cudaMemcpyAsync(ctx->x0, x0, sizeof(float) * ctx->P.n, cudaMemcpyDefault, ctx->stream), "x0 copy");
  CK(cudaGraphLaunch(ex, ctx->stream), "graph launch");
  ctx->last_set = ctx->tile.variant >= 2 ? (iters - 1) & 1 : 0;
  if (u0)
    CK(cudaMemcpyAsync(u0, ctx->u0, sizeof(float) * ctx->P.m, cudaMemcpyDefault, ctx->stream), "u0 copy");
  return MPPI_OK;
}

mppi_status mppi_jump_step(mppi_jump_ctx* ctx, const float* x0_host, int32_t iters, float* u0_host) {
  NvtxRange nv("mppi step (graph replay, host x0/u0)");
  if (!ctx || !x0_host || !u0_host || iters < 1) return MPPI_EINVAL;
  cudaGraphExec_t ex;
  mppi_status st = get_graph(ctx, iters, &ex);
  if (st != MPPI_OK) return st;
  if (ctx->timing) ctx->timed_iters = iters;
  std::memcpy(ctx->h_x0, x0_host, sizeof(float) * ctx->P.n);
  CK(cudaMemcpyAsync(ctx->x0, ctx->h_x0, sizeof(float) * ctx->P.n, cudaMemcpyHostToDevice, ctx->stream),
     "x0 copy");
  CK(cudaGraphLaunch(ex, ctx->stream), "graph launch");
  ctx->last_set = ctx->tile.variant >= 2 ? (iters - 1) & 1 : 0;
  CK(cudaMemcpyAsync(ctx->h_u0, ctx->u0, sizeof(float) * ctx->P.m, cudaMemcpyDeviceToHost, ctx->stream),
     "u0 copy");
  CK(cudaMemcpyAsync(ctx->h_status, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream),
     "status copy");
  CK(cudaStreamSynchronize(ctx->stream), "step sync");
  std::memcpy(u0_host, ctx->h_u0, sizeof(float) * ctx->P.m);
  // read: clear it for the next step (only after an error)
  if (ctx->h_status[0] != 0) CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream), "status reset");
  return status_of(ctx, ctx->h_status[0]);
}

mppi_status mppi_jump_autotune(mppi_jump_ctx* ctx, const float* x0, int32_t iters, int32_t reps,
                               mppi_jump_tuning* best_host, float* best_ms_host) {
  NvtxRange nv("mppi autotune");
  if (!ctx || !x0 || iters < 1 || reps < 1) return MPPI_EINVAL;
  const size_t TM = (size_t)ctx->P.T * ctx->P.m;
  std::vector<float> U_save(TM);
  uint32_t it_save = 0;
  mppi_status st = mppi_jump_get_iteration(ctx, &it_save);
  if (st != MPPI_OK) return st;
  CK(cudaMemcpyAsync(U_save.data(), ctx->U, TM * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream),
     "autotune save");
  CK(cudaStreamSynchronize(ctx->stream), "autotune save");
  const bool timing_save = ctx->timing;
  ctx->timing = false;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0), "autotune events");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(ctx->err, MPPI_ECUDA, "autotune events");
  }
  const RolloutTile cands[] = {{2, 128, 4}, {2, 64, 4},  {2, 32, 4},  {2, 128, 2}, {2, 64, 2},
                               {2, 32, 2},  {2, 128, 8}, {2, 64, 8},  {2, 32, 8},  {3, 128, 4},
                               {3, 128, 8}, {3, 64, 8},  {3, 32, 8},  {3, 128, 16}, {3, 64, 16},
                               {4, 128, 8}, {4, 64, 8},  {4, 128, 16}, {4, 64, 16},
                               {1, 128, 4}, {1, 64, 4},  {1, 32, 4}};
  RolloutTile best = ctx->tile;
  float best_ms = 1e30f;
  for (const RolloutTile& t : cands) {
    mppi_jump_tuning tt = {t.variant, t.block, t.chunk};
    st = mppi_jump_set_tuning(ctx, &tt);
    if (st == MPPI_OK) st = mppi_jump_step_async(ctx, x0, iters, nullptr);
    if (st == MPPI_OK && cudaEventRecord(e0, ctx->stream) != cudaSuccess) st = MPPI_ECUDA;
    for (int r = 0; r < reps && st == MPPI_OK; ++r) st = mppi_jump_step_async(ctx, x0, iters, nullptr);
    float ms = 0.0f;
    if (st == MPPI_OK && (cudaEventRecord(e1, ctx->stream) != cudaSuccess ||
                          cudaEventSynchronize(e1) != cudaSuccess ||
                          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      st = MPPI_ECUDA;
    if (st != MPPI_OK) break;
    ms /= (float)reps;
    if (ms < best_ms) {
      best_ms = ms;
      best = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->timing = timing_save;
  if (st != MPPI_OK) return st;
  mppi_jump_tuning bt = {best.variant, best.block, best.chunk};
  st = mppi_jump_set_tuning(ctx, &bt);
  if (st != MPPI_OK) return st;
  CK(cudaMemcpyAsync(ctx->U, U_save.data(), TM * sizeof(float), cudaMemcpyHostToDevice, ctx->stream),
     "autotune restore");
  CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream), "autotune restore");
  st = mppi_jump_set_iteration(ctx, it_save);
  if (st != MPPI_OK) return st;
  if (best_host) *best_host = bt;
  if (best_ms_host) *best_ms_host = best_ms;
  return MPPI_OK;
}

}  // extern "C"
