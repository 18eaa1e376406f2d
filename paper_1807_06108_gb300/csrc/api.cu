// api.cu -- the single-problem C ABI of libmppi_jump.so (see mppi_jump.h):
// context lifetime, the rollout_cost / update / step calls, the CUDA graph
// that replays an MPC step, debug copies and checkpointing.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "internal.h"

using namespace mj;

struct mppi_jump_ctx {
  mppi_jump_config cfg;
  DevProblem P;
  UpdateGeom geom;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  // one device allocation carved into the buffers below
  void* arena = nullptr;
  size_t arena_bytes = 0;
  float* x0 = nullptr;       // [n]
  float* U = nullptr;        // [T][m]
  void* noise = nullptr;     // [T][Kpad][m] f32 or bf16
  float* s_part = nullptr;   // [Kpad]
  float* w = nullptr;        // [Kpad]
  float* partial = nullptr;  // [chunks][T][m]
  float* scal = nullptr;     // cconst, diag[3]
  int* status = nullptr;     // device status word
  uint32_t* it = nullptr;    // iteration counter
  float* u0 = nullptr;       // [m]
  // pinned host staging for the synchronous step
  float* h_x0 = nullptr;
  float* h_u0 = nullptr;
  int* h_status = nullptr;
  uint8_t* dbg_counts = nullptr;
  float* dbg_J = nullptr;
  std::map<int, cudaGraphExec_t> graphs;
  // phase timing: events recorded inside the captured step
  bool timing = false;
  std::vector<cudaEvent_t> events;  // 3 per iteration: before rollout, after, after update
  int timed_iters = 0;              // iterations covered by the last timed step
  char err[256] = {0};
};

namespace {

struct Layout {
  size_t x0, U, noise, s_part, w, partial, scal, status, it, u0, total;
};

Layout layout_of(const DevProblem& P, const UpdateGeom& g) {
  Layout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += align256(bytes);
    return o;
  };
  const size_t sb = P.noise_bf16 ? 2 : 4;
  L.x0 = take(sizeof(float) * 16);
  L.U = take(sizeof(float) * (size_t)P.T * P.m);
  L.noise = take(sb * (size_t)P.T * P.Kpad * P.m);
  L.s_part = take(sizeof(float) * P.Kpad);
  L.w = take(sizeof(float) * P.Kpad);
  L.partial = take(sizeof(float) * (size_t)g.chunks * P.T * P.m);
  L.scal = take(sizeof(float) * 8);
  L.status = take(sizeof(int) * 4);
  L.it = take(sizeof(uint32_t) * 4);
  L.u0 = take(sizeof(float) * 4);
  L.total = off;
  return L;
}

int num_sms_of_current() {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

mppi_status cuda_fail(mppi_jump_ctx* ctx, cudaError_t e, const char* what) {
  snprintf(ctx->err, sizeof(ctx->err), "%s: %s", what, cudaGetErrorString(e));
  return MPPI_ECUDA;
}

#define CK(call, what)                          \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
  } while (0)

IterBuffers buffers(mppi_jump_ctx* ctx, float* costs) {
  IterBuffers b;
  b.x0 = ctx->x0;
  b.U = ctx->U;
  b.noise = ctx->noise;
  b.s_part = ctx->s_part;
  b.w = ctx->w;
  b.partial = ctx->partial;
  b.cconst = ctx->scal;
  b.diag = ctx->scal + 1;
  b.status = ctx->status;
  b.it = ctx->it;
  b.costs = costs;
  b.dbg_counts = ctx->dbg_counts;
  b.dbg_J = ctx->dbg_J;
  return b;
}

void fill_u_init(const mppi_jump_config& cfg, float* host, int T, int m) {
  for (int j = 0; j < T; ++j)
    for (int i = 0; i < m; ++i) host[(size_t)j * m + i] = cfg.u_init[i];
}

}  // namespace

extern "C" {

const char* mppi_jump_status_string(mppi_status st) {
  switch (st) {
    case MPPI_OK: return "ok";
    case MPPI_EINVAL: return "invalid argument";
    case MPPI_ENOMEM: return "out of memory";
    case MPPI_ECUDA: return "CUDA error";
    case MPPI_ETIMEOUT: return "device wait timed out";
    case MPPI_ENONFINITE: return "all rollout costs non-finite";
    case MPPI_EBUSY: return "busy";
  }
  return "unknown status";
}

const char* mppi_jump_last_error(const mppi_jump_ctx* ctx) {
  return ctx ? ctx->err : "no context";
}

mppi_status mppi_jump_default_config(int32_t system, mppi_jump_config* out) {
  if (!out || (system != MPPI_CARTPOLE && system != MPPI_QUADROTOR)) return MPPI_EINVAL;
  std::memset(out, 0, sizeof(*out));
  out->system = system;
  out->lambda = 1.0f;
  out->c = 1.0f;
  out->alpha = 1.0f;
  out->count_law = MPPI_COUNT_POISSON;
  out->mark_law = MPPI_MARK_NORMAL;
  out->jump_channel = MPPI_JUMP_STATE;
  out->noise_dtype = MPPI_NOISE_F32;
  out->seed = 0;
  mppi_cartpole_params& c = out->cartpole;
  c.mc = 1.0f;
  c.mp = 0.1f;
  c.l = 0.5f;
  c.g = 9.81f;
  const float goal[4] = {0.0f, 0.0f, 3.14159265358979f, 0.0f};
  const float Q[4] = {1.0f, 0.1f, 10.0f, 0.1f};
  for (int i = 0; i < 4; ++i) {
    c.goal[i] = goal[i];
    c.Q[i] = Q[i];
    c.Qf[i] = Q[i];
  }
  mppi_quadrotor_params& q = out->quadrotor;
  q.mass = 1.0f;
  q.J[0] = 0.01f;
  q.J[1] = 0.01f;
  q.J[2] = 0.02f;
  q.arm = 0.2f;
  q.kappa = 0.02f;
  q.g = 9.81f;
  q.goal[0] = 4.0f;
  q.goal[1] = 0.0f;
  q.goal[2] = 1.0f;
  q.wp = 10.0f;
  q.wv = 1.0f;
  q.weta = 1.0f;
  q.wom = 0.1f;
  q.obs[0] = 2.0f;
  q.obs[1] = 0.0f;
  q.obs[2] = 1.0f;
  q.obs_r = 0.5f;
  q.obs_cost = 1.0e4f;
  if (system == MPPI_CARTPOLE) {
    out->K = 1000;
    out->T = 50;
    out->dt = 0.02f;
    out->sigma[0] = 1.0f;
    out->jump_rate = 1.0f;
    out->q = 2;
    out->jump_rows[0] = 1;
    out->jump_rows[1] = 3;
    out->mark_scale[0] = out->mark_scale[1] = 0.5f;
    out->u_init[0] = 0.0f;
  } else {
    out->K = 4096;
    out->T = 100;
    out->dt = 0.01f;
    for (int i = 0; i < 4; ++i) {
      out->sigma[i] = 0.2f;
      out->u_init[i] = q.mass * q.g / 4.0f;
    }
    out->jump_rate = 2.0f;
    out->q = 3;
    out->jump_rows[0] = 3;
    out->jump_rows[1] = 4;
    out->jump_rows[2] = 5;
    out->mark_scale[0] = out->mark_scale[1] = out->mark_scale[2] = 1.0f;
  }
  return MPPI_OK;
}

mppi_status mppi_jump_validate(const mppi_jump_config* cfg) {
  DevProblem P;
  return pack_problem(cfg, &P, nullptr);
}

size_t mppi_jump_config_bytes(void) { return sizeof(mppi_jump_config); }

mppi_status mppi_jump_workspace_bytes(const mppi_jump_config* cfg, size_t* bytes_host) {
  if (!bytes_host) return MPPI_EINVAL;
  DevProblem P;
  mppi_status st = pack_problem(cfg, &P, nullptr);
  if (st != MPPI_OK) return st;
  const UpdateGeom g = update_geometry(P.Kpad, P.T, P.m, P.noise_bf16 != 0, num_sms_of_current());
  *bytes_host = layout_of(P, g).total;
  return MPPI_OK;
}

mppi_status mppi_jump_init(const mppi_jump_config* cfg, void* stream, mppi_jump_ctx** out) {
  if (!out) return MPPI_EINVAL;
  *out = nullptr;
  mppi_jump_ctx* ctx = new (std::nothrow) mppi_jump_ctx();
  if (!ctx) return MPPI_ENOMEM;
  mppi_status st = pack_problem(cfg, &ctx->P, ctx->err);
  if (st != MPPI_OK) {
    delete ctx;
    return st;
  }
  ctx->cfg = *cfg;
  ctx->cfg.reserved = 0;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = prepare_kernels();
  if (e == cudaSuccess) {
    ctx->geom = update_geometry(ctx->P.Kpad, ctx->P.T, ctx->P.m, ctx->P.noise_bf16 != 0,
                                num_sms_of_current());
    const Layout L = layout_of(ctx->P, ctx->geom);
    ctx->arena_bytes = L.total;
    if (stream) {
      ctx->stream = (cudaStream_t)stream;
    } else {
      e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
      ctx->own_stream = e == cudaSuccess;
    }
    if (e == cudaSuccess) e = cudaMalloc(&ctx->arena, L.total);
    if (e == cudaSuccess) {
      char* a = (char*)ctx->arena;
      ctx->x0 = (float*)(a + L.x0);
      ctx->U = (float*)(a + L.U);
      ctx->noise = a + L.noise;
      ctx->s_part = (float*)(a + L.s_part);
      ctx->w = (float*)(a + L.w);
      ctx->partial = (float*)(a + L.partial);
      ctx->scal = (float*)(a + L.scal);
      ctx->status = (int*)(a + L.status);
      ctx->it = (uint32_t*)(a + L.it);
      ctx->u0 = (float*)(a + L.u0);
      e = cudaMallocHost(&ctx->h_x0, sizeof(float) * 64);
    }
    if (e == cudaSuccess) {
      ctx->h_u0 = ctx->h_x0 + 16;
      ctx->h_status = (int*)(ctx->h_x0 + 32);
      e = cudaMemsetAsync(ctx->arena, 0, L.total, ctx->stream);
    }
    if (e == cudaSuccess) {
      const size_t TM = (size_t)ctx->P.T * ctx->P.m;
      float* hU = (float*)std::malloc(sizeof(float) * TM);
      if (!hU) {
        e = cudaErrorMemoryAllocation;
      } else {
        fill_u_init(*cfg, hU, ctx->P.T, ctx->P.m);
        e = cudaMemcpyAsync(ctx->U, hU, sizeof(float) * TM, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        std::free(hU);
      }
    }
  }
  if (e != cudaSuccess) {
    const bool oom = e == cudaErrorMemoryAllocation;
    mppi_jump_destroy(ctx);
    return oom ? MPPI_ENOMEM : MPPI_ECUDA;
  }
  *out = ctx;
  return MPPI_OK;
}

mppi_status mppi_jump_destroy(mppi_jump_ctx* ctx) {
  if (!ctx) return MPPI_OK;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
  for (cudaEvent_t ev : ctx->events) cudaEventDestroy(ev);
  if (ctx->arena) cudaFree(ctx->arena);
  if (ctx->h_x0) cudaFreeHost(ctx->h_x0);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return MPPI_OK;
}

mppi_status mppi_jump_set_controls(mppi_jump_ctx* ctx, const float* U) {
  if (!ctx || !U) return MPPI_EINVAL;
  CK(cudaMemcpyAsync(ctx->U, U, sizeof(float) * ctx->P.T * ctx->P.m, cudaMemcpyDefault, ctx->stream),
     "set_controls");
  return MPPI_OK;
}

mppi_status mppi_jump_get_controls(mppi_jump_ctx* ctx, float* U) {
  if (!ctx || !U) return MPPI_EINVAL;
  CK(cudaMemcpyAsync(U, ctx->U, sizeof(float) * ctx->P.T * ctx->P.m, cudaMemcpyDefault, ctx->stream),
     "get_controls");
  return MPPI_OK;
}

mppi_status mppi_jump_set_iteration(mppi_jump_ctx* ctx, uint32_t it) {
  if (!ctx) return MPPI_EINVAL;
  ctx->h_status[4] = (int)it;
  CK(cudaMemcpyAsync(ctx->it, &ctx->h_status[4], sizeof(uint32_t), cudaMemcpyHostToDevice, ctx->stream),
     "set_iteration");
  CK(cudaStreamSynchronize(ctx->stream), "set_iteration");
  return MPPI_OK;
}

mppi_status mppi_jump_get_iteration(mppi_jump_ctx* ctx, uint32_t* it_host) {
  if (!ctx || !it_host) return MPPI_EINVAL;
  CK(cudaMemcpyAsync(&ctx->h_status[4], ctx->it, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream),
     "get_iteration");
  CK(cudaStreamSynchronize(ctx->stream), "get_iteration");
  *it_host = (uint32_t)ctx->h_status[4];
  return MPPI_OK;
}

mppi_status mppi_jump_rollout_cost(mppi_jump_ctx* ctx, const float* x0, float* costs) {
  if (!ctx || !x0) return MPPI_EINVAL;
  CK(cudaMemcpyAsync(ctx->x0, x0, sizeof(float) * ctx->P.n, cudaMemcpyDefault, ctx->stream), "x0 copy");
  CK(launch_rollout(ctx->P, buffers(ctx, costs), ctx->stream), "rollout launch");
  return MPPI_OK;
}

mppi_status mppi_jump_update(mppi_jump_ctx* ctx) {
  if (!ctx) return MPPI_EINVAL;
  CK(launch_weights_update(ctx->P, buffers(ctx, nullptr), ctx->geom, 0, nullptr, ctx->stream),
     "update launch");
  return MPPI_OK;
}

mppi_status mppi_jump_sync(mppi_jump_ctx* ctx) {
  if (!ctx) return MPPI_EINVAL;
  CK(cudaMemcpyAsync(ctx->h_status, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream),
     "status copy");
  CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream), "status reset");
  CK(cudaStreamSynchronize(ctx->stream), "sync");
  if (ctx->h_status[0] != 0) {
    snprintf(ctx->err, sizeof(ctx->err), "every rollout cost was non-finite; U left unchanged");
    return (mppi_status)ctx->h_status[0];
  }
  return MPPI_OK;
}

static mppi_status get_graph(mppi_jump_ctx* ctx, int iters, cudaGraphExec_t* exec) {
  auto it = ctx->graphs.find(iters);
  if (it != ctx->graphs.end()) {
    *exec = it->second;
    return MPPI_OK;
  }
  // The captured sequence reads x0 from ctx->x0 and writes u0 to ctx->u0.
  if (ctx->timing) {
    while ((int)ctx->events.size() < 3 * iters) {
      cudaEvent_t ev;
      CK(cudaEventCreate(&ev), "event create");
      ctx->events.push_back(ev);
    }
  }
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  cudaError_t e = cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream);
  const IterBuffers b = buffers(ctx, nullptr);
  auto mark = [&](int idx) {
    if (ctx->timing && e == cudaSuccess)
      e = cudaEventRecordWithFlags(ctx->events[idx], ctx->stream, cudaEventRecordExternal);
  };
  for (int r = 0; r < iters && e == cudaSuccess; ++r) {
    mark(3 * r);
    e = launch_rollout(ctx->P, b, ctx->stream);
    mark(3 * r + 1);
    if (e == cudaSuccess)
      e = launch_weights_update(ctx->P, b, ctx->geom, r == iters - 1, ctx->u0, ctx->stream);
    mark(3 * r + 2);
  }
  cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &graph);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(ctx, e, "step capture");
  }
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "graph instantiate");
  ctx->graphs[iters] = ex;
  *exec = ex;
  return MPPI_OK;
}

mppi_status mppi_jump_enable_timing(mppi_jump_ctx* ctx, int32_t on) {
  if (!ctx) return MPPI_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream), "enable_timing");
  ctx->timing = on != 0;
  for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
  ctx->graphs.clear();
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
  if (!ctx || !x0 || iters < 1) return MPPI_EINVAL;
  cudaGraphExec_t ex;
  mppi_status st = get_graph(ctx, iters, &ex);
  if (st != MPPI_OK) return st;
  if (ctx->timing) ctx->timed_iters = iters;
  CK(cudaMemcpyAsync(ctx->x0, x0, sizeof(float) * ctx->P.n, cudaMemcpyDefault, ctx->stream), "x0 copy");
  CK(cudaGraphLaunch(ex, ctx->stream), "graph launch");
  if (u0)
    CK(cudaMemcpyAsync(u0, ctx->u0, sizeof(float) * ctx->P.m, cudaMemcpyDefault, ctx->stream), "u0 copy");
  return MPPI_OK;
}

mppi_status mppi_jump_step(mppi_jump_ctx* ctx, const float* x0_host, int32_t iters, float* u0_host) {
  if (!ctx || !x0_host || !u0_host || iters < 1) return MPPI_EINVAL;
  cudaGraphExec_t ex;
  mppi_status st = get_graph(ctx, iters, &ex);
  if (st != MPPI_OK) return st;
  if (ctx->timing) ctx->timed_iters = iters;
  std::memcpy(ctx->h_x0, x0_host, sizeof(float) * ctx->P.n);
  CK(cudaMemcpyAsync(ctx->x0, ctx->h_x0, sizeof(float) * ctx->P.n, cudaMemcpyHostToDevice, ctx->stream),
     "x0 copy");
  CK(cudaGraphLaunch(ex, ctx->stream), "graph launch");
  CK(cudaMemcpyAsync(ctx->h_u0, ctx->u0, sizeof(float) * ctx->P.m, cudaMemcpyDeviceToHost, ctx->stream),
     "u0 copy");
  CK(cudaMemcpyAsync(ctx->h_status, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream),
     "status copy");
  CK(cudaStreamSynchronize(ctx->stream), "step sync");
  std::memcpy(u0_host, ctx->h_u0, sizeof(float) * ctx->P.m);
  if (ctx->h_status[0] != 0) {
    snprintf(ctx->err, sizeof(ctx->err), "every rollout cost was non-finite; U left unchanged");
    return (mppi_status)ctx->h_status[0];
  }
  return MPPI_OK;
}

mppi_status mppi_jump_set_debug(mppi_jump_ctx* ctx, uint8_t* counts, float* jumps) {
  if (!ctx) return MPPI_EINVAL;
  ctx->dbg_counts = counts;
  ctx->dbg_J = jumps;
  for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
  ctx->graphs.clear();
  return MPPI_OK;
}

mppi_status mppi_jump_get_noise(mppi_jump_ctx* ctx, void* noise) {
  if (!ctx || !noise) return MPPI_EINVAL;
  const size_t sb = ctx->P.noise_bf16 ? 2 : 4;
  const size_t row_dst = sb * ctx->P.K * ctx->P.m, row_src = sb * ctx->P.Kpad * ctx->P.m;
  CK(cudaMemcpy2DAsync(noise, row_dst, ctx->noise, row_src, row_dst, ctx->P.T, cudaMemcpyDefault,
                       ctx->stream),
     "get_noise");
  return MPPI_OK;
}

mppi_status mppi_jump_get_weights(mppi_jump_ctx* ctx, float* weights) {
  if (!ctx || !weights) return MPPI_EINVAL;
  CK(cudaMemcpyAsync(weights, ctx->w, sizeof(float) * ctx->P.K, cudaMemcpyDefault, ctx->stream),
     "get_weights");
  return MPPI_OK;
}

mppi_status mppi_jump_get_free_energy(mppi_jump_ctx* ctx, float out_host[3]) {
  if (!ctx || !out_host) return MPPI_EINVAL;
  CK(cudaMemcpyAsync(ctx->h_u0, ctx->scal + 1, sizeof(float) * 3, cudaMemcpyDeviceToHost, ctx->stream),
     "get_free_energy");
  CK(cudaStreamSynchronize(ctx->stream), "get_free_energy");
  for (int i = 0; i < 3; ++i) out_host[i] = ctx->h_u0[i];
  return MPPI_OK;
}

// Checkpoint layout: magic, ABI version, config, counter, U [T][m].
static const uint32_t kCkptMagic = 0x4d50504au;  // "MPPJ"

mppi_status mppi_jump_get_state(mppi_jump_ctx* ctx, void* buf_host, size_t* size_host) {
  if (!ctx || !size_host) return MPPI_EINVAL;
  const size_t TM = (size_t)ctx->P.T * ctx->P.m;
  const size_t need = 2 * sizeof(uint32_t) + sizeof(mppi_jump_config) + sizeof(uint32_t) + TM * sizeof(float);
  if (!buf_host) {
    *size_host = need;
    return MPPI_OK;
  }
  if (*size_host < need) {
    *size_host = need;
    snprintf(ctx->err, sizeof(ctx->err), "checkpoint buffer too small (%zu bytes needed)", need);
    return MPPI_EINVAL;
  }
  char* p = (char*)buf_host;
  const uint32_t hdr[2] = {kCkptMagic, MPPI_JUMP_ABI_VERSION};
  std::memcpy(p, hdr, sizeof(hdr));
  p += sizeof(hdr);
  std::memcpy(p, &ctx->cfg, sizeof(ctx->cfg));
  p += sizeof(ctx->cfg);
  uint32_t it = 0;
  mppi_status st = mppi_jump_get_iteration(ctx, &it);
  if (st != MPPI_OK) return st;
  std::memcpy(p, &it, sizeof(it));
  p += sizeof(it);
  CK(cudaMemcpyAsync(p, ctx->U, TM * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream), "get_state");
  CK(cudaStreamSynchronize(ctx->stream), "get_state");
  *size_host = need;
  return MPPI_OK;
}

mppi_status mppi_jump_set_state(mppi_jump_ctx* ctx, const void* buf_host, size_t size) {
  if (!ctx || !buf_host) return MPPI_EINVAL;
  const size_t TM = (size_t)ctx->P.T * ctx->P.m;
  const size_t need = 2 * sizeof(uint32_t) + sizeof(mppi_jump_config) + sizeof(uint32_t) + TM * sizeof(float);
  if (size != need) return fail(ctx->err, MPPI_EINVAL, "checkpoint size %zu, expected %zu", size, need);
  const char* p = (const char*)buf_host;
  uint32_t hdr[2];
  std::memcpy(hdr, p, sizeof(hdr));
  if (hdr[0] != kCkptMagic || hdr[1] != MPPI_JUMP_ABI_VERSION)
    return fail(ctx->err, MPPI_EINVAL, "not a checkpoint of this library version");
  p += sizeof(hdr);
  mppi_jump_config cfg;
  std::memcpy(&cfg, p, sizeof(cfg));
  cfg.reserved = 0;
  if (std::memcmp(&cfg, &ctx->cfg, sizeof(cfg)) != 0)
    return fail(ctx->err, MPPI_EINVAL, "checkpoint was taken with another configuration");
  p += sizeof(cfg);
  uint32_t it;
  std::memcpy(&it, p, sizeof(it));
  p += sizeof(it);
  CK(cudaMemcpyAsync(ctx->U, p, TM * sizeof(float), cudaMemcpyHostToDevice, ctx->stream), "set_state");
  CK(cudaStreamSynchronize(ctx->stream), "set_state");
  return mppi_jump_set_iteration(ctx, it);
}

}  // extern "C"
