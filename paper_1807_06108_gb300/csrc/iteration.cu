// iteration.cu -- configuration packing and the launches of one MPPI
// iteration (rollout, softmin, split-K update, combine) for a single problem.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "internal.h"
#include "kernels.cuh"

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
  for (int c = 0; c < 4; ++c) P->jump_rows[c] = c < cfg->q ? cfg->jump_rows[c] : -1;
  P->key0 = (uint32_t)(cfg->seed & 0xffffffffull);
  P->key1 = (uint32_t)(cfg->seed >> 32);
  P->dt = cfg->dt;
  P->lam = cfg->lambda;
  P->inv_lam = (float)(1.0 / (double)cfg->lambda);
  P->is_coef = (float)(0.5 * (1.0 - 1.0 / (double)cfg->c));
  P->alpha = cfg->alpha;
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

cudaError_t prepare_kernels() {
  // the combine kernel keeps the whole sequence (up to 4096 x 4 floats) in
  // shared memory; idempotent, called before any launch or capture
  return cudaFuncSetAttribute(update_combine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              4096 * 4 * (int)sizeof(float));
}

UpdateGeom update_geometry(int Kpad, int T, int m, bool bf16, int num_sms) {
  UpdateGeom g;
  const int E = bf16 ? 8 : 4;
  const int nvec = Kpad * m / E;
  g.vpt = nvec >= 4 * kUpdateThreads ? 4 : (nvec >= 2 * kUpdateThreads ? 2 : 1);
  g.chunks = (nvec + kUpdateThreads * g.vpt - 1) / (kUpdateThreads * g.vpt);
  const int target = 2 * (num_sms > 0 ? num_sms : 152);
  int groups = (target + g.chunks - 1) / g.chunks;
  if (groups > T) groups = T;
  if (groups < 1) groups = 1;
  g.rows = (T + groups - 1) / groups;
  g.groups = (T + g.rows - 1) / g.rows;
  return g;
}

template <int SYS, bool BF16, bool DBG>
static void launch_rollout_t(const DevProblem& P, const IterBuffers& b, cudaStream_t s) {
  const int blocks = (P.Kpad + kRolloutThreads - 1) / kRolloutThreads;
  rollout_kernel<SYS, BF16, DBG><<<blocks, kRolloutThreads, 0, s>>>(
      P, b.x0, b.U, b.it, b.s_part, b.costs, b.cconst, b.noise, b.dbg_counts, b.dbg_J);
}

cudaError_t launch_rollout(const DevProblem& P, const IterBuffers& b, cudaStream_t s) {
  const bool dbg = b.dbg_counts != nullptr || b.dbg_J != nullptr;
  const int sel = P.system * 4 + (P.noise_bf16 ? 2 : 0) + (dbg ? 1 : 0);
  switch (sel) {
    case 0: launch_rollout_t<0, false, false>(P, b, s); break;
    case 1: launch_rollout_t<0, false, true>(P, b, s); break;
    case 2: launch_rollout_t<0, true, false>(P, b, s); break;
    case 3: launch_rollout_t<0, true, true>(P, b, s); break;
    case 4: launch_rollout_t<1, false, false>(P, b, s); break;
    case 5: launch_rollout_t<1, false, true>(P, b, s); break;
    case 6: launch_rollout_t<1, true, false>(P, b, s); break;
    default: launch_rollout_t<1, true, true>(P, b, s); break;
  }
  return cudaGetLastError();
}

template <bool BF16, int M, int VPT>
static void launch_partial_t(const IterBuffers& b, const UpdateGeom& g, int Kpad, int T,
                             cudaStream_t s) {
  dim3 grid(g.chunks, g.groups);
  update_partial_kernel<BF16, M, VPT><<<grid, kUpdateThreads, 0, s>>>(b.noise, b.w, Kpad, T, g.rows,
                                                                      b.partial, b.status);
}

template <bool BF16, int M>
static void launch_partial_m(const IterBuffers& b, const UpdateGeom& g, int Kpad, int T,
                             cudaStream_t s) {
  if (g.vpt == 4) launch_partial_t<BF16, M, 4>(b, g, Kpad, T, s);
  else if (g.vpt == 2) launch_partial_t<BF16, M, 2>(b, g, Kpad, T, s);
  else launch_partial_t<BF16, M, 1>(b, g, Kpad, T, s);
}

cudaError_t launch_weights_update(const DevProblem& P, const IterBuffers& b, const UpdateGeom& g,
                                  int shift, float* u0, cudaStream_t s) {
  softmin_kernel<<<1, kSoftminThreads, 0, s>>>(b.s_part, P.K, P.Kpad, P.inv_lam, b.cconst, b.w,
                                                b.diag, b.status);
  if (P.m == 4) {
    if (P.noise_bf16) launch_partial_m<true, 4>(b, g, P.Kpad, P.T, s);
    else launch_partial_m<false, 4>(b, g, P.Kpad, P.T, s);
  } else {
    if (P.noise_bf16) launch_partial_m<true, 1>(b, g, P.Kpad, P.T, s);
    else launch_partial_m<false, 1>(b, g, P.Kpad, P.T, s);
  }
  const size_t smem = (size_t)P.T * P.m * sizeof(float);
  update_combine_kernel<<<1, kCombineThreads, smem, s>>>(b.partial, g.chunks, P.T, P.m, P.alpha, b.U,
                                                         b.status, b.it, shift, P, u0);
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
