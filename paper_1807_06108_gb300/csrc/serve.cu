// serve.cu -- the served form: a native request loop that admits single MPC
// steps for many sessions (any mix of plants, K, T) as they arrive.
//
// Every session keeps its warm-started control sequence and Philox counter in
// its own device context (Sec. V: the un-executed controls seed the next
// solve).  A worker thread admits queued requests as soon as (a) the session
// has no request in flight (per-session order is the submission order),
// (b) one of `max_inflight` slots is free and (c) the session's device
// memory fits the budget -- resident idle sessions are checkpointed to the
// host and released, least recently used first, to make room.  Each admitted
// request runs as the session's graph-replayed MPC step on the session's own
// stream, so requests admitted while others are on the GPU execute
// concurrently with them; completion is detected with CUDA events, never by
// blocking the loop.  A session's result depends only on its own state and
// inputs (every reduction has a fixed order), so it is the same whether the
// request ran alone or in the mix.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "context.h"

using mj::control_dim;
using mj::state_dim;

namespace {

using Clock = std::chrono::steady_clock;

double now_s() {
  return std::chrono::duration<double>(Clock::now().time_since_epoch()).count();
}

struct Request {
  int session = -1;
  float x0[12] = {0};
  float u0[4] = {0};
  double t_submit = 0, t_admit = 0, t_done = 0;
  int status = MPPI_OK;
  bool done = false;
};

struct Session {
  mppi_jump_config cfg;
  int iters = 1;
  size_t bytes = 0;
  mppi_jump_ctx* ctx = nullptr;  // resident when not NULL
  std::vector<char> ckpt;        // host copy of the state while evicted
  bool busy = false;
  double last_used = 0;
  std::deque<uint64_t> queue;
};

struct Slot {
  bool busy = false;
  int session = -1;
  uint64_t ticket = 0;
  cudaEvent_t ev = nullptr;
  float* h = nullptr;  // pinned: x0 [12], u0 [4], status
};

}  // namespace

struct mppi_server {
  int device = 0;
  size_t budget = 0, used = 0;
  std::vector<Session> sessions;
  std::vector<Slot> slots;
  std::vector<Request> reqs;
  std::deque<uint64_t> arrivals;  // submitted, not yet sorted into sessions
  std::vector<double> latencies;
  int64_t evictions = 0;
  double t_first = 0, t_last = 0;
  std::mutex mu;
  std::condition_variable cv_done;
  std::atomic<bool> stop{false};
  std::thread worker;
  char err[256] = {0};
};

namespace {

// Make session i resident within the budget; false if it must wait.
bool make_resident(mppi_server* S, int i, int* status) {
  mj::NvtxRange nv("mppi serve make resident");
  Session& ses = S->sessions[i];
  if (ses.ctx) return true;
  while (S->used + ses.bytes > S->budget) {
    int victim = -1;
    for (int j = 0; j < (int)S->sessions.size(); ++j) {
      const Session& o = S->sessions[j];
      if (j != i && o.ctx && !o.busy && (victim < 0 || o.last_used < S->sessions[victim].last_used))
        victim = j;
    }
    if (victim < 0) return false;  // wait for a running session to finish
    Session& v = S->sessions[victim];
    size_t n = 0;
    mppi_jump_get_state(v.ctx, nullptr, &n);
    v.ckpt.resize(n);
    if (mppi_jump_get_state(v.ctx, v.ckpt.data(), &n) != MPPI_OK) {
      *status = MPPI_ECUDA;
      return false;
    }
    mppi_jump_destroy(v.ctx);
    v.ctx = nullptr;
    S->used -= v.bytes;
    ++S->evictions;
  }
  mppi_status st = mppi_jump_init(&ses.cfg, nullptr, &ses.ctx);
  if (st == MPPI_OK && !ses.ckpt.empty()) st = mppi_jump_set_state(ses.ctx, ses.ckpt.data(), ses.ckpt.size());
  if (st != MPPI_OK) {
    if (ses.ctx) mppi_jump_destroy(ses.ctx);
    ses.ctx = nullptr;
    *status = st;
    return false;
  }
  ses.ckpt.clear();
  S->used += ses.bytes;
  return true;
}

// Launch ticket t of session i on slot s.
mppi_status launch(mppi_server* S, Slot& slot, int i, uint64_t t) {
  mj::NvtxRange nv("mppi serve admit");
  Session& ses = S->sessions[i];
  Request& r = S->reqs[t];
  mppi_jump_ctx* ctx = ses.ctx;
  std::memcpy(slot.h, r.x0, sizeof(r.x0));
  mppi_status st = mppi_jump_step_async(ctx, slot.h, ses.iters, slot.h + 12);
  if (st != MPPI_OK) return st;
  int* hs = reinterpret_cast<int*>(slot.h + 16);
  if (cudaMemcpyAsync(hs, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
      cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream) != cudaSuccess ||
      cudaEventRecord(slot.ev, ctx->stream) != cudaSuccess)
    return MPPI_ECUDA;
  slot.busy = true;
  slot.session = i;
  slot.ticket = t;
  ses.busy = true;
  r.t_admit = now_s();
  return MPPI_OK;
}

void finish(mppi_server* S, Request& r, int status) {
  r.status = status;
  r.t_done = now_s();
  r.done = true;
  S->latencies.push_back(r.t_done - r.t_submit);
  S->t_last = r.t_done;
}

void worker_loop(mppi_server* S) {
  cudaSetDevice(S->device);
  for (;;) {
    bool progress = false;
    std::unique_lock<std::mutex> lock(S->mu);
    // 1. sort new arrivals into their sessions' queues (submission order)
    while (!S->arrivals.empty()) {
      const uint64_t t = S->arrivals.front();
      S->arrivals.pop_front();
      S->sessions[S->reqs[t].session].queue.push_back(t);
      progress = true;
    }
    // 2. completions
    for (Slot& slot : S->slots) {
      if (!slot.busy) continue;
      const cudaError_t q = cudaEventQuery(slot.ev);
      if (q == cudaErrorNotReady) continue;
      Request& r = S->reqs[slot.ticket];
      Session& ses = S->sessions[slot.session];
      std::memcpy(r.u0, slot.h + 12, sizeof(r.u0));
      const int st = q == cudaSuccess ? *reinterpret_cast<int*>(slot.h + 16) : (int)MPPI_ECUDA;
      finish(S, r, st);
      ses.busy = false;
      ses.last_used = r.t_done;
      slot.busy = false;
      progress = true;
    }
    if (progress) S->cv_done.notify_all();
    // 3. admissions, oldest waiting request first
    for (;;) {
      int best = -1;
      for (int i = 0; i < (int)S->sessions.size(); ++i) {
        const Session& ses = S->sessions[i];
        if (ses.busy || ses.queue.empty()) continue;
        if (best < 0 || ses.queue.front() < S->sessions[best].queue.front()) best = i;
      }
      if (best < 0) break;
      Slot* free_slot = nullptr;
      for (Slot& slot : S->slots)
        if (!slot.busy) {
          free_slot = &slot;
          break;
        }
      if (!free_slot) break;
      int st = MPPI_OK;
      if (!make_resident(S, best, &st)) {
        if (st != MPPI_OK) {  // cannot run at all: fail the request
          Session& ses = S->sessions[best];
          const uint64_t t = ses.queue.front();
          ses.queue.pop_front();
          finish(S, S->reqs[t], st);
          S->cv_done.notify_all();
          continue;
        }
        break;  // wait for memory
      }
      Session& ses = S->sessions[best];
      const uint64_t t = ses.queue.front();
      ses.queue.pop_front();
      const mppi_status ls = launch(S, *free_slot, best, t);
      if (ls != MPPI_OK) {
        finish(S, S->reqs[t], ls);
        S->cv_done.notify_all();
      }
      progress = true;
    }
    bool idle = true;
    for (const Slot& slot : S->slots) idle = idle && !slot.busy;
    for (const Session& ses : S->sessions) idle = idle && ses.queue.empty();
    idle = idle && S->arrivals.empty();
    if (S->stop.load() && idle) break;
    lock.unlock();
    if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(idle ? 200 : 5));
  }
}

double percentile(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = p * (double)(v.size() - 1);
  const size_t lo = (size_t)pos;
  const size_t hi = std::min(lo + 1, v.size() - 1);
  return v[lo] + (pos - (double)lo) * (v[hi] - v[lo]);
}

}  // namespace

extern "C" {

mppi_status mppi_serve_destroy(mppi_server* S) {
  if (!S) return MPPI_OK;
  S->stop.store(true);
  if (S->worker.joinable()) S->worker.join();
  for (Session& ses : S->sessions)
    if (ses.ctx) mppi_jump_destroy(ses.ctx);
  for (Slot& slot : S->slots) {
    if (slot.ev) cudaEventDestroy(slot.ev);
    if (slot.h) cudaFreeHost(slot.h);
  }
  delete S;
  return MPPI_OK;
}

mppi_status mppi_serve_create(const mppi_jump_config* cfgs_host, const int32_t* iters_host,
                              int32_t n_sessions, size_t budget_bytes, int32_t max_inflight,
                              mppi_server** out) {
  if (!out || !cfgs_host || !iters_host || n_sessions < 1 || max_inflight < 1 || budget_bytes == 0)
    return MPPI_EINVAL;
  *out = nullptr;
  mppi_server* S = new (std::nothrow) mppi_server();
  if (!S) return MPPI_ENOMEM;
  cudaGetDevice(&S->device);
  S->budget = budget_bytes;
  S->sessions.resize(n_sessions);
  for (int i = 0; i < n_sessions; ++i) {
    Session& ses = S->sessions[i];
    ses.cfg = cfgs_host[i];
    ses.iters = iters_host[i];
    mppi_status st = mppi_jump_workspace_bytes(&ses.cfg, &ses.bytes);
    if (st != MPPI_OK || ses.iters < 1 || ses.bytes > budget_bytes) {
      snprintf(S->err, sizeof(S->err), "session %d: invalid configuration, iterations or over budget", i);
      delete S;
      return st != MPPI_OK ? st : MPPI_EINVAL;
    }
  }
  S->slots.resize(max_inflight);
  for (Slot& slot : S->slots) {
    if (cudaEventCreateWithFlags(&slot.ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(&slot.h, sizeof(float) * 32) != cudaSuccess) {
      mppi_serve_destroy(S);
      return MPPI_ECUDA;
    }
  }
  S->reqs.reserve(1 << 16);
  S->worker = std::thread(worker_loop, S);
  *out = S;
  return MPPI_OK;
}

const char* mppi_serve_last_error(const mppi_server* S) { return S ? S->err : "no server"; }

mppi_status mppi_serve_submit(mppi_server* S, int32_t session, const float* x0_host, uint64_t* ticket_out) {
  if (!S || !x0_host || !ticket_out) return MPPI_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  if (session < 0 || session >= (int)S->sessions.size()) return MPPI_EINVAL;
  Request r;
  r.session = session;
  const int n = state_dim(S->sessions[session].cfg.system);
  std::memcpy(r.x0, x0_host, sizeof(float) * n);
  r.t_submit = now_s();
  if (S->reqs.empty() || S->t_first == 0) S->t_first = r.t_submit;
  const uint64_t t = S->reqs.size();
  S->reqs.push_back(r);
  S->arrivals.push_back(t);
  *ticket_out = t;
  return MPPI_OK;
}

mppi_status mppi_serve_poll(mppi_server* S, uint64_t ticket, float* u0_host, int32_t* done_host) {
  if (!S || !done_host) return MPPI_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  if (ticket >= S->reqs.size()) return MPPI_EINVAL;
  const Request& r = S->reqs[ticket];
  *done_host = r.done ? 1 : 0;
  if (!r.done) return MPPI_OK;
  if (u0_host) std::memcpy(u0_host, r.u0, sizeof(float) * control_dim(S->sessions[r.session].cfg.system));
  return (mppi_status)r.status;
}

mppi_status mppi_serve_wait(mppi_server* S, uint64_t ticket, float* u0_host, double timeout_s) {
  if (!S) return MPPI_EINVAL;
  std::unique_lock<std::mutex> lock(S->mu);
  if (ticket >= S->reqs.size()) return MPPI_EINVAL;
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                          std::chrono::duration<double>(timeout_s));
  if (!S->cv_done.wait_until(lock, deadline, [&] { return S->reqs[ticket].done; }))
    return MPPI_ETIMEOUT;
  const Request& r = S->reqs[ticket];
  if (u0_host) std::memcpy(u0_host, r.u0, sizeof(float) * control_dim(S->sessions[r.session].cfg.system));
  return (mppi_status)r.status;
}

mppi_status mppi_serve_drain(mppi_server* S, double timeout_s) {
  if (!S) return MPPI_EINVAL;
  std::unique_lock<std::mutex> lock(S->mu);
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                          std::chrono::duration<double>(timeout_s));
  const bool ok = S->cv_done.wait_until(lock, deadline, [&] {
    for (const Request& r : S->reqs)
      if (!r.done) return false;
    return true;
  });
  return ok ? MPPI_OK : MPPI_ETIMEOUT;
}

mppi_status mppi_serve_get_stats(mppi_server* S, mppi_serve_stats* out) {
  if (!S || !out) return MPPI_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = (int64_t)S->reqs.size();
  out->completed = (int64_t)S->latencies.size();
  for (const Slot& slot : S->slots) out->inflight += slot.busy ? 1 : 0;
  out->evictions = S->evictions;
  out->resident_bytes = S->used;
  double sum = 0, mx = 0;
  for (double l : S->latencies) {
    sum += l;
    mx = std::max(mx, l);
  }
  out->mean_ms = S->latencies.empty() ? 0 : 1e3 * sum / (double)S->latencies.size();
  out->max_ms = 1e3 * mx;
  out->p50_ms = 1e3 * percentile(S->latencies, 0.50);
  out->p99_ms = 1e3 * percentile(S->latencies, 0.99);
  out->span_s = S->t_last > S->t_first ? S->t_last - S->t_first : 0.0;
  return MPPI_OK;
}

mppi_status mppi_serve_reset_stats(mppi_server* S) {
  if (!S) return MPPI_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  for (const Request& r : S->reqs)
    if (!r.done) return MPPI_EBUSY;
  S->latencies.clear();
  S->reqs.clear();
  S->t_first = S->t_last = 0;
  S->evictions = 0;
  return MPPI_OK;
}

mppi_status mppi_serve_get_controls(mppi_server* S, int32_t session, float* U_host) {
  if (!S || !U_host) return MPPI_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  if (session < 0 || session >= (int)S->sessions.size()) return MPPI_EINVAL;
  Session& ses = S->sessions[session];
  if (ses.busy || !ses.queue.empty()) return MPPI_EBUSY;
  const size_t TM = (size_t)ses.cfg.T * control_dim(ses.cfg.system);
  if (ses.ctx) {
    if (mppi_jump_get_controls(ses.ctx, U_host) != MPPI_OK ||
        cudaStreamSynchronize(ses.ctx->stream) != cudaSuccess)
      return MPPI_ECUDA;
    return MPPI_OK;
  }
  if (!ses.ckpt.empty()) {  // evicted: the controls sit at the end of the checkpoint
    std::memcpy(U_host, ses.ckpt.data() + ses.ckpt.size() - TM * sizeof(float), TM * sizeof(float));
    return MPPI_OK;
  }
  for (size_t j = 0; j < (size_t)ses.cfg.T; ++j)  // never run: u_init
    for (int c = 0; c < control_dim(ses.cfg.system); ++c)
      U_host[j * control_dim(ses.cfg.system) + c] = ses.cfg.u_init[c];
  return MPPI_OK;
}

}  // extern "C"
