// kernels.cuh -- the four kernels of one MPPI iteration on jump diffusions:
//   rollout_kernel        sampling + rollout + augmented cost (A1+A2)
//   softmin_kernel        free-energy weights (A3)
//   update_partial_kernel split-K weighted sum of the perturbations (A4)
//   update_combine_kernel fixed-order combine, U update, counter, MPC shift (A4/A5)
// Included by the translation units that launch them.
#pragma once

#include "device.cuh"

namespace mj {

constexpr int kRolloutThreads = 128;
constexpr int kSoftminThreads = 1024;
constexpr int kUpdateThreads = 256;
constexpr int kCombineThreads = 1024;
constexpr int kStatusNonFinite = 5;

// ---------------------------------------------------------------------------
// Rollout: one thread per rollout k, the plant state in registers.  Per step
// j: the Gaussian perturbation (stream 0), the jump count (stream 1, one
// Philox block per four steps) and, when the count is positive, the marks
// (streams 2+n); delta_eff is rounded to bfloat16 first when the noise is
// stored in that type, so the rollout uses exactly the stored value; the
// augmented cost of Eq. 34-35 is accumulated with compensated summation and
// the k-independent term lambda/2 u^T Sigma^-1 u is kept apart (it cancels in
// the weights); the Euler step adds the state jump.  delta_eff is stored
// step-major, noise[(j*Kpad + k)*m + i], so each warp store is contiguous.
// Rollouts K..Kpad-1 (padding) store zero noise and an infinite cost.
// ---------------------------------------------------------------------------
template <int SYS, bool BF16, bool DBG>
__global__ void __launch_bounds__(kRolloutThreads)
rollout_kernel(const DevProblem P, const float* __restrict__ x0, const float* __restrict__ U,
               const uint32_t* __restrict__ it_ptr, float* __restrict__ s_part,
               float* __restrict__ costs, float* __restrict__ cconst, void* __restrict__ noise,
               uint8_t* __restrict__ dbg_counts, float* __restrict__ dbg_J) {
  using PL = Plant<SYS>;
  constexpr int n = PL::n, m = PL::m;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P.Kpad) return;
  const bool active = k < P.K;
  const uint32_t it = __ldg(it_ptr);
  const uint32_t uk = (uint32_t)k;

  float x[n];
#pragma unroll
  for (int i = 0; i < n; ++i) x[i] = __ldg(x0 + i);
  float s = 0.0f, sc = 0.0f, C = 0.0f, Cc = 0.0f;

  for (int j0 = 0; j0 < P.T; j0 += 4) {
    const uint4 wcount = philox4x32_10(uk, (uint32_t)(j0 >> 2), it, 1u, P.key0, P.key1);
    float zc[4];
    if constexpr (m == 1) normals4(philox4x32_10(uk, (uint32_t)(j0 >> 2), it, 0u, P.key0, P.key1), zc);
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int j = j0 + jj;
      if (j >= P.T) break;
      float de[m];
      if constexpr (m == 1) {
        de[0] = P.sqc_sigma[0] * zc[jj];
      } else {
        float z[4];
        normals4(philox4x32_10(uk, (uint32_t)j, it, 0u, P.key0, P.key1), z);
#pragma unroll
        for (int i = 0; i < m; ++i) de[i] = P.sqc_sigma[i] * z[i];
      }
      const int N = jump_count(P, word_of(wcount, jj));
      float J[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      if (N > 0) {
        for (int nj = 0; nj < N; ++nj) {
          const uint4 wm = philox4x32_10(uk, (uint32_t)j, it, 2u + (uint32_t)nj, P.key0, P.key1);
          if (P.mark_law == 0) {
            float z[4];
            normals4(wm, z);
#pragma unroll
            for (int c = 0; c < 4; ++c)
              if (c < P.q) J[c] += P.mark_scale[c] * z[c];
          } else {
#pragma unroll
            for (int c = 0; c < 4; ++c)
              if (c < P.q) J[c] += laplace_mark(P.mark_scale[c], word_of(wm, c));
          }
        }
        if (P.jump_channel == 1) {
#pragma unroll
          for (int i = 0; i < m; ++i) de[i] += J[i];
        }
      }
      if constexpr (BF16) {
#pragma unroll
        for (int i = 0; i < m; ++i) de[i] = __bfloat162float(__float2bfloat16_rn(de[i]));
      }
      // augmented running cost (Eq. 34-35 in control units)
      float u[m];
      float uSu = 0.0f, uSd = 0.0f, dSd = 0.0f;
#pragma unroll
      for (int i = 0; i < m; ++i) {
        u[i] = __ldg(U + j * m + i);
        const float a = P.inv_sigma2[i];
        uSu += u[i] * a * u[i];
        uSd += u[i] * a * de[i];
        dSd += de[i] * a * de[i];
      }
      const float qx = PL::state_cost(P.pl, x);
      two_sum_acc(s, sc, qx * P.dt + P.lam * (uSd + P.is_coef * dSd));
      two_sum_acc(C, Cc, 0.5f * P.lam * uSu);
      // Euler step (Algorithm 1) with the control-affine drift (Eq. 4)
      float v[m], xd[n];
#pragma unroll
      for (int i = 0; i < m; ++i) v[i] = u[i] + de[i];
      PL::xdot(P.pl, x, v, xd);
#pragma unroll
      for (int i = 0; i < n; ++i) x[i] += xd[i] * P.dt;
      if (N > 0 && P.jump_channel == 0) {
#pragma unroll
        for (int r = 0; r < n; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c)
            if (c < P.q && P.jump_rows[c] == r) x[r] += P.s_jump * J[c];
      }
      // store delta_eff, step-major
      const size_t row = (size_t)j * P.Kpad + k;
      if constexpr (BF16) {
        if constexpr (m == 4) {
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
        if constexpr (m == 4) {
          reinterpret_cast<float4*>(noise)[row] = active ? make_float4(de[0], de[1], de[2], de[3])
                                                         : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        } else {
          reinterpret_cast<float*>(noise)[row] = active ? de[0] : 0.0f;
        }
      }
      if (DBG && active) {
        const size_t rk = (size_t)j * P.K + k;
        if (dbg_counts) dbg_counts[rk] = (uint8_t)N;
        if (dbg_J)
          for (int c = 0; c < P.q; ++c) dbg_J[rk * P.q + c] = J[c];
      }
    }
  }
  two_sum_acc(s, sc, PL::terminal_cost(P.pl, x));
  if (active) {
    float sk = s + sc;
    if (!isfinite(sk)) sk = INFINITY;
    s_part[k] = sk;
    const float cc = C + Cc;
    if (costs) costs[k] = cc + sk;
    if (k == 0) *cconst = cc;
  } else {
    s_part[k] = INFINITY;
  }
}

// ---------------------------------------------------------------------------
// Block reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ void warp_sum2(float& s, float& c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, o);
    const float c2 = __shfl_xor_sync(0xffffffffu, c, o);
    two_sum_merge(s, c, s2, c2);
  }
}

// ---------------------------------------------------------------------------
// Softmin (Eq. 36-37 with the minimum subtracted): one block of 1024 threads.
//   rho = min s_k over finite costs; e_k = exp((rho - s_k)/lambda);
//   Z = sum e_k (compensated); w_k = e_k / Z.
// diag = {rho + C, Z, (rho + C)/lambda - ln(Z/K)} with C the k-independent
// cost term.  No finite cost: status = non-finite, weights untouched.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSoftminThreads)
softmin_kernel(const float* __restrict__ s_part, int K, int Kpad, float inv_lam,
               const float* __restrict__ cconst, float* __restrict__ w, float* __restrict__ diag,
               int* __restrict__ status) {
  __shared__ float red_s[32], red_c[32];
  __shared__ float sh_rho, sh_Z;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  float mn = INFINITY;
  for (int k = tid; k < K; k += blockDim.x) mn = fminf(mn, s_part[k]);
  mn = warp_min(mn);
  if (lane == 0) red_s[wid] = mn;
  __syncthreads();
  if (wid == 0) {
    float v = lane < (int)(blockDim.x >> 5) ? red_s[lane] : INFINITY;
    v = warp_min(v);
    if (lane == 0) sh_rho = v;
  }
  __syncthreads();
  const float rho = sh_rho;
  if (!isfinite(rho)) {
    if (tid == 0) *status = kStatusNonFinite;
    return;
  }
  float zs = 0.0f, zc = 0.0f;
  for (int k = tid; k < K; k += blockDim.x) two_sum_acc(zs, zc, expf((rho - s_part[k]) * inv_lam));
  warp_sum2(zs, zc);
  if (lane == 0) {
    red_s[wid] = zs;
    red_c[wid] = zc;
  }
  __syncthreads();
  if (wid == 0) {
    float a = lane < (int)(blockDim.x >> 5) ? red_s[lane] : 0.0f;
    float b = lane < (int)(blockDim.x >> 5) ? red_c[lane] : 0.0f;
    warp_sum2(a, b);
    if (lane == 0) sh_Z = a + b;
  }
  __syncthreads();
  const float Z = sh_Z;
  for (int k = tid; k < Kpad; k += blockDim.x)
    w[k] = k < K ? expf((rho - s_part[k]) * inv_lam) / Z : 0.0f;
  if (tid == 0) {
    const float rf = rho + *cconst;
    diag[0] = rf;
    diag[1] = Z;
    diag[2] = rf * inv_lam - logf(Z / (float)K);
  }
}

// ---------------------------------------------------------------------------
// Weighted update, split over K.  Block (c, g) owns the rollout chunk c
// (kUpdateThreads * VPT 16-byte vectors of the step-major noise rows) and the
// steps g*rows .. g*rows+rows-1.  Each thread keeps the weights of its
// rollouts in registers across steps, multiplies them into its vectors, and
// the block reduces the m channel sums with compensated shuffles; the result
// goes to partial[(c*T + j)*m + i].  Vectors beyond the row are skipped.
// ---------------------------------------------------------------------------
template <bool BF16, int M, int VPT>
__global__ void __launch_bounds__(kUpdateThreads)
update_partial_kernel(const void* __restrict__ noise, const float* __restrict__ w, int Kpad, int T,
                      int rows, float* __restrict__ partial, const int* __restrict__ status) {
  constexpr int E = BF16 ? 8 : 4;  // elements per 16-byte vector
  constexpr int RPV = E / M;       // rollouts per vector
  __shared__ float red_s[kUpdateThreads / 32][M], red_c[kUpdateThreads / 32][M];
  if (*status != 0) return;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nvec = Kpad * M / E;  // vectors per row
  const int vbase = blockIdx.x * (kUpdateThreads * VPT) + tid;
  float wr[VPT][RPV];
#pragma unroll
  for (int t = 0; t < VPT; ++t) {
    const int v = vbase + t * kUpdateThreads;
#pragma unroll
    for (int r = 0; r < RPV; ++r) wr[t][r] = v < nvec ? __ldg(w + v * RPV + r) : 0.0f;
  }
  const int j_begin = blockIdx.y * rows;
  const int j_end = min(T, j_begin + rows);
  const uint4* nv = reinterpret_cast<const uint4*>(noise);
  for (int j = j_begin; j < j_end; ++j) {
    uint4 buf[VPT];
#pragma unroll
    for (int t = 0; t < VPT; ++t) {
      const int v = vbase + t * kUpdateThreads;
      buf[t] = v < nvec ? __ldcs(nv + (size_t)j * nvec + v) : make_uint4(0u, 0u, 0u, 0u);
    }
    float acc[M];
#pragma unroll
    for (int i = 0; i < M; ++i) acc[i] = 0.0f;
#pragma unroll
    for (int t = 0; t < VPT; ++t) {
      float val[E];
      if (BF16) {
        const uint32_t wd[4] = {buf[t].x, buf[t].y, buf[t].z, buf[t].w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          val[2 * h] = __uint_as_float(wd[h] << 16);
          val[2 * h + 1] = __uint_as_float(wd[h] & 0xffff0000u);
        }
      } else {
        val[0] = __uint_as_float(buf[t].x);
        val[1] = __uint_as_float(buf[t].y);
        val[2] = __uint_as_float(buf[t].z);
        val[3] = __uint_as_float(buf[t].w);
      }
#pragma unroll
      for (int e = 0; e < E; ++e) acc[e % M] = fmaf(wr[t][e / M], val[e], acc[e % M]);
    }
    float cmp[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
      cmp[i] = 0.0f;
      warp_sum2(acc[i], cmp[i]);
    }
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < M; ++i) {
        red_s[wid][i] = acc[i];
        red_c[wid][i] = cmp[i];
      }
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
      for (int i = 0; i < M; ++i) {
        float a = lane < kUpdateThreads / 32 ? red_s[lane][i] : 0.0f;
        float b = lane < kUpdateThreads / 32 ? red_c[lane][i] : 0.0f;
        warp_sum2(a, b);
        if (lane == 0) partial[((size_t)blockIdx.x * T + j) * M + i] = a + b;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Combine the chunk partials in chunk order (compensated), U += alpha * dU,
// advance the iteration counter, and on the last iteration of an MPC step
// emit u0 = U_0 and shift (U_i <- U_{i+1}, U_{T-1} <- u_init).  One block;
// `sh` holds the updated sequence (T*m floats of dynamic shared memory).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kCombineThreads)
update_combine_kernel(const float* __restrict__ partial, int chunks, int T, int m, float alpha,
                      float* __restrict__ U, const int* __restrict__ status,
                      uint32_t* __restrict__ it_ptr, int shift, DevProblem P,
                      float* __restrict__ u0_out) {
  extern __shared__ float sh[];
  const int TM = T * m;
  const bool ok = *status == 0;
  for (int idx = threadIdx.x; idx < TM; idx += blockDim.x) {
    float v = U[idx];
    if (ok) {
      float s = 0.0f, c = 0.0f;
      for (int ch = 0; ch < chunks; ++ch) two_sum_acc(s, c, partial[(size_t)ch * TM + idx]);
      v = v + alpha * (s + c);
    }
    sh[idx] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) *it_ptr = *it_ptr + 1u;
  if (shift && ok) {
    if (u0_out)
      for (int i = threadIdx.x; i < m; i += blockDim.x) u0_out[i] = sh[i];
    for (int idx = threadIdx.x; idx < TM; idx += blockDim.x)
      U[idx] = idx + m < TM ? sh[idx + m] : P.u_init[idx - (TM - m)];
  } else {
    if (shift && u0_out)
      for (int i = threadIdx.x; i < m; i += blockDim.x) u0_out[i] = sh[i];
    if (ok)
      for (int idx = threadIdx.x; idx < TM; idx += blockDim.x) U[idx] = sh[idx];
  }
}

}  // namespace mj
