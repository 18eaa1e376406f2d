// api.cu -- the single-problem C ABI of libmppi_jump.so (see mppi_jump.h):
// configuration, context lifetime, controls and counter, debug copies and
// checkpointing.  The rollout / update / step calls are in step.cu.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>

#include "context.h"

using namespace mj;

namespace mj {

mppi_status cuda_fail(mppi_jump_ctx* ctx, cudaError_t e, const char* what) {
  snprintf(ctx->err, sizeof(ctx->err), "%s: %s", what, cudaGetErrorString(e));
  return MPPI_ECUDA;
}

int num_sms_of_current() {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

IterBuffers ctx_buffers(mppi_jump_ctx* ctx, float* costs, int set) {
  IterBuffers b;
  b.x0 = ctx->x0;
  b.U = ctx->U;
  b.noise = ctx->noise[set];
  b.jmask = ctx->jmask[set];
  b.jrec = ctx->jrec[set];
  b.s_part = ctx->s_part;
  b.rec = ctx->rec;
  b.max_chunks = ctx->max_chunks;
  b.partial = ctx->partial;
  b.zpart = ctx->zpart;
  b.gpart = ctx->gpart;
  b.rho_key = ctx->rho_key + (set & 1);
  b.rho_key_next = ctx->rho_key + ((set + 1) & 1);
  b.done = ctx->done;
  b.cconst = ctx->scal;
  b.diag = ctx->scal + 1;
  b.status = ctx->status;
  b.it = ctx->it;
  b.costs = costs;
  b.dbg_counts = ctx->dbg_counts;
  b.dbg_J = ctx->dbg_J;
  b.arm_key = nullptr;
  return b;
}

void drop_graphs(mppi_jump_ctx* ctx) {
  for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
  ctx->graphs.clear();
}

}  // namespace mj

namespace {

struct Layout {
  size_t x0, U, noise[2], jmask[2], jrec[2], s_part, rec, partial, zpart, gpart, scal, status, it,
      rho_key, done, u0, total;
  int max_chunks;
};

// Partial records the update may combine at once (rollout shards).
constexpr int kMaxParts = 4096;

Layout layout_of(const DevProblem& P, const UpdateGeom& g) {
  Layout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += align256(bytes);
    return o;
  };
  const size_t sb = P.noise_bf16 ? 2 : 4;
  const size_t TK = (size_t)P.T * P.Kpad;
  L.x0 = take(sizeof(float) * 16);
  L.U = take(sizeof(float) * (size_t)P.T * P.m);
  for (int s = 0; s < 2; ++s) {
    L.noise[s] = take(sb * TK * P.m);
    const bool sj = P.jump_channel == MPPI_JUMP_STATE;
    L.jmask[s] = take(sj ? sizeof(uint32_t) * (size_t)(P.Kpad / 32) * mask_cols(P.T) : 0);
    L.jrec[s] = take(sj ? sizeof(float4) * TK : 0);
  }
  L.s_part = take(sizeof(float) * P.Kpad);
  // partial records of the rollout blocks (tile 4; the smallest block is 32)
  const size_t max_blocks = ((size_t)P.Kpad + 31) / 32;
  L.rec = take(sizeof(float) * max_blocks * (2 + (size_t)P.T * P.m));
  // chunk partials of the update: rollout chunks, or chunks of records
  const int bps = records_per_chunk(P.m);
  L.max_chunks = g.chunks;
  L.max_chunks = std::max(L.max_chunks, (int)((max_blocks + bps - 1) / bps));
  L.max_chunks = std::max(L.max_chunks, (kMaxParts + bps - 1) / bps);
  L.partial = take(sizeof(float) * (size_t)L.max_chunks * P.T * P.m);
  L.zpart = take(sizeof(float) * (size_t)g.groups * L.max_chunks);
  L.gpart = take(sizeof(float) * (size_t)g.groups * (P.m + 1));
  L.scal = take(sizeof(float) * 8);
  L.status = take(sizeof(int) * 4);
  L.it = take(sizeof(uint32_t) * 4);
  L.rho_key = take(sizeof(uint32_t) * 4);
  L.done = take(sizeof(unsigned) * (4 + (size_t)g.groups));
  L.u0 = take(sizeof(float) * 4);
  L.total = off;
  return L;
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
    case MPPI_EBOUNDS: return "kernel launch check failed";
  }
  return "unknown status";
}

const char* mppi_jump_last_error(const mppi_jump_ctx* ctx) { return ctx ? ctx->err : "no context"; }

mppi_status mppi_jump_default_config(int32_t system, mppi_jump_config* out) {
  if (!out || (system != MPPI_CARTPOLE && system != MPPI_QUADROTOR)) return MPPI_EINVAL;
  std::memset(out, 0, sizeof(*out));
  out->system = system;
  out->lambda = 1.0f;
  out->c = 1.0f;
  out->alpha = 1.0f;
  out->alpha_decay = 1.0f;
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
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = prepare_kernels();
  if (e == cudaSuccess) {
    const int sms = num_sms_of_current();
    ctx->geom = update_geometry(ctx->P.Kpad, ctx->P.T, ctx->P.m, ctx->P.noise_bf16 != 0, sms);
    ctx->tile = default_tile(ctx->P, sms);
    const Layout L = layout_of(ctx->P, ctx->geom);
    ctx->arena_bytes = L.total;
    if (stream) {
      ctx->stream = (cudaStream_t)stream;
    } else {
      e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
      ctx->own_stream = e == cudaSuccess;
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->aux2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->arena, L.total);
    if (e == cudaSuccess) {
      char* a = (char*)ctx->arena;
      ctx->x0 = (float*)(a + L.x0);
      ctx->U = (float*)(a + L.U);
      for (int s = 0; s < 2; ++s) {
        ctx->noise[s] = a + L.noise[s];
        const bool sj = ctx->P.jump_channel == MPPI_JUMP_STATE;
        ctx->jmask[s] = sj ? (uint32_t*)(a + L.jmask[s]) : nullptr;
        ctx->jrec[s] = sj ? (float4*)(a + L.jrec[s]) : nullptr;
      }
      ctx->s_part = (float*)(a + L.s_part);
      ctx->rec = (float*)(a + L.rec);
      ctx->max_chunks = L.max_chunks;
      ctx->partial = (float*)(a + L.partial);
      ctx->zpart = (float*)(a + L.zpart);
      ctx->gpart = (float*)(a + L.gpart);
      ctx->scal = (float*)(a + L.scal);
      ctx->status = (int*)(a + L.status);
      ctx->it = (uint32_t*)(a + L.it);
      ctx->rho_key = (uint32_t*)(a + L.rho_key);
      ctx->done = (unsigned*)(a + L.done);
      ctx->u0 = (float*)(a + L.u0);
      e = cudaMallocHost(&ctx->h_x0, sizeof(float) * 64);
    }
    if (e == cudaSuccess) {
      ctx->h_u0 = ctx->h_x0 + 16;
      ctx->h_status = (int*)(ctx->h_x0 + 32);
      e = cudaMemsetAsync(ctx->arena, 0, L.total, ctx->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(ctx->rho_key, 0xff, 2 * sizeof(uint32_t), ctx->stream);
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
  drop_graphs(ctx);
  for (cudaEvent_t ev : ctx->events) cudaEventDestroy(ev);
  for (cudaEvent_t ev : ctx->links) cudaEventDestroy(ev);
  if (ctx->arena) cudaFree(ctx->arena);
  if (ctx->h_x0) cudaFreeHost(ctx->h_x0);
  if (ctx->aux) cudaStreamDestroy(ctx->aux);
  if (ctx->aux2) cudaStreamDestroy(ctx->aux2);
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
  CK(cudaStreamSynchronize(ctx->stream), "set_iteration");
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

mppi_status mppi_jump_set_debug(mppi_jump_ctx* ctx, uint8_t* counts, float* jumps) {
  if (!ctx) return MPPI_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream), "set_debug");
  ctx->dbg_counts = counts;
  ctx->dbg_J = jumps;
  drop_graphs(ctx);
  return MPPI_OK;
}

mppi_status mppi_jump_get_noise(mppi_jump_ctx* ctx, void* noise) {
  if (!ctx || !noise) return MPPI_EINVAL;
  const size_t sb = ctx->P.noise_bf16 ? 2 : 4;
  const size_t row_dst = sb * ctx->P.K * ctx->P.m, row_src = sb * ctx->P.Kpad * ctx->P.m;
  CK(cudaMemcpy2DAsync(noise, row_dst, ctx->noise[ctx->last_set], row_src, row_dst, ctx->P.T,
                       cudaMemcpyDefault, ctx->stream),
     "get_noise");
  return MPPI_OK;
}

mppi_status mppi_jump_get_weights(mppi_jump_ctx* ctx, float* weights) {
  if (!ctx || !weights) return MPPI_EINVAL;
  CK(launch_weights(ctx->s_part, ctx->scal + 1, ctx->P.inv_lam, ctx->P.K, weights, ctx->stream),
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

static size_t ckpt_bytes(const mppi_jump_ctx* ctx) {
  return 2 * sizeof(uint32_t) + sizeof(mppi_jump_config) + sizeof(uint32_t) +
         (size_t)ctx->P.T * ctx->P.m * sizeof(float);
}

mppi_status mppi_jump_get_state(mppi_jump_ctx* ctx, void* buf_host, size_t* size_host) {
  if (!ctx || !size_host) return MPPI_EINVAL;
  const size_t TM = (size_t)ctx->P.T * ctx->P.m;
  const size_t need = ckpt_bytes(ctx);
  if (!buf_host) {
    *size_host = need;
    return MPPI_OK;
  }
  if (*size_host < need) {
    *size_host = need;
    return fail(ctx->err, MPPI_EINVAL, "checkpoint buffer too small (%zu bytes needed)", need);
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
  const size_t need = ckpt_bytes(ctx);
  if (size != need) return fail(ctx->err, MPPI_EINVAL, "checkpoint size %zu, expected %zu", size, need);
  const char* p = (const char*)buf_host;
  uint32_t hdr[2];
  std::memcpy(hdr, p, sizeof(hdr));
  if (hdr[0] != kCkptMagic || hdr[1] != MPPI_JUMP_ABI_VERSION)
    return fail(ctx->err, MPPI_EINVAL, "not a checkpoint of this library version");
  p += sizeof(hdr);
  mppi_jump_config cfg;
  std::memcpy(&cfg, p, sizeof(cfg));
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
