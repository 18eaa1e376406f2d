// device.cuh -- device-side building blocks of the MPPI jump-diffusion path:
// the Philox4x32-10 counter generator, uniforms and Box-Muller normals, the
// jump sampler, the two plants and their costs, and compensated summation.
// Everything here runs in registers inside the fused kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mj {

constexpr int kMaxJumps = 16;

// Plant constants, pre-processed on the host (reciprocals, squared radius).
struct DevPlant {
  // cart-pole: point-mass pole, theta = 0 hanging down
  float mc, mp, l, g, inv_l, mcp_g;  // mcp_g = (mc + mp) g
  float goal[4], Q[4], Qf[4];
  // quadrotor
  float inv_mass, J[3], invJ[3], arm, kappa, qg;
  float pgoal[3], wp, wv, weta, wom, obs[3], obs_r2, obs_cost;
};

// Everything a rollout needs, passed by value as a kernel parameter.
struct DevProblem {
  int32_t system, K, Kpad, T, n, m, q;
  int32_t count_law, mark_law, jump_channel, nmax, noise_bf16;
  int32_t jump_default;  // state jumps hit the plant's velocity rows (1, 3) / (3, 4, 5)
  int32_t jump_rows[4];
  uint32_t key0, key1;
  uint32_t rk[20];  // Philox round keys: rk[2r] = key0 + r * 0x9E3779B9, rk[2r+1] = key1 + r * 0xBB67AE85
  uint32_t k_base;  // Philox index of local rollout 0 (a rollout shard starts at k_base)
  uint32_t thr[kMaxJumps];  // jump-count thresholds (see the header)
  float dt, lam, inv_lam, is_coef, alpha, s_jump;
  float alpha_decay;  // step size alpha * alpha_decay^r at iteration r of a step
  float sqc_sigma[4];   // sqrt(c) * sigma_i
  float inv_sigma2[4];  // 1 / sigma_i^2
  float mark_scale[4];
  float u_init[4];
  DevPlant pl;
};

// Columns of a jump-mask row (one row per 32 rollouts, one 32-bit word per
// step): the steps rounded up to 16, so that every row starts on a 64-byte
// boundary and the words of steps 4b .. 4b+3 are one aligned 16-byte store.
__host__ __device__ constexpr int mask_cols(int T) { return (T + 15) & ~15; }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds, each two
// 32x32->64-bit products whose high halves are xored with the other two
// counter words and the round key; the key advances by the Weyl constants
// (golden ratio, sqrt(3) - 1) between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    // one 32x32 -> 64-bit multiply gives both halves of each product
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
    const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return make_uint4(c0, c1, c2, c3);
}

// The same generator with the ten round keys precomputed (rk as in
// DevProblem): in a kernel whose problem is a launch parameter they are
// constant-bank operands of the XORs, and no key arithmetic is left per round.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                  const uint32_t* rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
    const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
    const uint32_t n0 = hi1 ^ c1 ^ rk[2 * r];
    const uint32_t n2 = hi0 ^ c3 ^ rk[2 * r + 1];
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return make_uint4(c0, c1, c2, c3);
}

// Uniform on (0, 1): (top 23 bits + 1/2) * 2^-23, exact in float32 (one
// fused multiply-add of exact terms).
__device__ __forceinline__ float uniform01(uint32_t w) {
  return fmaf(__uint2float_rn(w >> 9), 0x1p-23f, 0x1p-24f);
}

// sin(2 pi u) and cos(2 pi u) for the uniforms above.  With x = 4u (exact),
// the nearest integer q of x (adding and subtracting 1.5 * 2^23 rounds it,
// and the low two bits of the sum's encoding are q mod 4) is the quadrant and
// f = x - q in [-1/2, 1/2] (exact) places the angle (pi/2) f within it, so
// that sin(q pi/2 + a) and cos(q pi/2 + a) come from sin a and cos a by a
// swap (q odd) and sign flips (q mod 4 in {2, 3} for sin, {1, 2} for cos).
// sin a and cos a, |a| <= pi/4, come from their Taylor series in f, to
// degree 9 and 10 (truncation below 3e-9); the coefficients are
// (pi/2)^n / n! with alternating signs.  Over all 2^23 uniforms the float32
// result is within 1.7 ulp of sin and cos (checked against a double-precision
// evaluation).
__device__ __forceinline__ void sincos_2pi(float u, float& s, float& c) {
  constexpr float kS1 = 1.57079637050628662f, kS3 = -0.645964086055755615f, kS5 = 0.0796926245093345642f,
                  kS7 = -0.00468175392597913742f, kS9 = 0.000160441180923953652f;
  constexpr float kC2 = -1.23370051383972168f, kC4 = 0.253669500350952148f, kC6 = -0.0208634808659553528f,
                  kC8 = 0.000919260259252041578f, kC10 = -2.52020417974563315e-05f;
  constexpr float kRound = 12582912.0f;  // 1.5 * 2^23
  const float x = 4.0f * u;
  const float y = __fadd_rn(x, kRound);
  const float f = __fsub_rn(x, __fsub_rn(y, kRound));
  const uint32_t q = __float_as_uint(y);
  const float f2 = f * f;
  const float sp = f * fmaf(f2, fmaf(f2, fmaf(f2, fmaf(f2, kS9, kS7), kS5), kS3), kS1);
  const float cp = fmaf(f2, fmaf(f2, fmaf(f2, fmaf(f2, fmaf(f2, kC10, kC8), kC6), kC4), kC2), 1.0f);
  const bool odd = (q & 1u) != 0u;
  const float sv = odd ? cp : sp, cv = odd ? sp : cp;
  s = __uint_as_float(__float_as_uint(sv) ^ ((q << 30) & 0x80000000u));
  c = __uint_as_float(__float_as_uint(cv) ^ (((q + 1u) << 30) & 0x80000000u));
}

// Box-Muller (1958): r = sqrt(-2 ln u_a), (r cos 2 pi u_b, r sin 2 pi u_b).
// -2 ln u_a >= 1.2e-7 for these uniforms (u_a <= 1 - 2^-24), so the square
// root is taken as x * rsqrt(x) (within 3 ulp).
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, float& z0, float& z1) {
  const float x = -2.0f * logf(uniform01(wa));
  const float r = x * rsqrtf(x);
  float s, c;
  sincos_2pi(uniform01(wb), s, c);
  z0 = r * c;
  z1 = r * s;
}

__device__ __forceinline__ void normals4(const uint4 w, float z[4]) {
  box_muller(w.x, w.y, z[0], z[1]);
  box_muller(w.z, w.w, z[2], z[3]);
}

__device__ __forceinline__ uint32_t word_of(const uint4 w, int i) {
  return i == 0 ? w.x : (i == 1 ? w.y : (i == 2 ? w.z : w.w));
}

// Jump count of one step from its 32-bit word (Poisson thresholds or the
// Bernoulli timer of the zero-one law).
__device__ __forceinline__ int jump_count(const DevProblem& P, uint32_t w) {
  if (P.count_law == 1) return (P.nmax > 0 && w < P.thr[0]) ? 1 : 0;
  int n = 0;
  while (n < P.nmax && w >= P.thr[n]) ++n;
  return n;
}

// Laplace(0, b) mark from a uniform: -b sgn(u - 1/2) ln(1 - 2|u - 1/2|).
// u - 1/2 and 1 - 2|u - 1/2| are exact for the 23-bit uniforms above.
__device__ __forceinline__ float laplace_mark(float b, uint32_t w) {
  const float h = uniform01(w) - 0.5f;
  const float mag = __fmul_rn(-b, logf(1.0f - 2.0f * fabsf(h)));  // never fused with a later add
  return h > 0.0f ? mag : -mag;
}

// ---------------------------------------------------------------------------
// Compensated summation (Knuth's branch-free TwoSum): (s, c) holds the sum and
// the accumulated rounding error.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float y) {
  const float t = __fadd_rn(s, y);
  const float bp = __fsub_rn(t, s);
  const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(y, bp));
  c = __fadd_rn(c, e);
  s = t;
}

// Merge two compensated pairs.
__device__ __forceinline__ void two_sum_merge(float& s, float& c, float s2, float c2) {
  two_sum_acc(s, c, s2);
  c = __fadd_rn(c, c2);
}

// ---------------------------------------------------------------------------
// Plants: F(x, v) = f(x) + G(x) v (Eq. 4), Euler-stepped by the caller.
// The trigonometric functions and reciprocals use the hardware approximations
// (__sincosf: absolute error about 2^-21 for |x| <= pi; __fdividef: 2 ulp):
// they sit on the sequential critical path of every step, and their error is
// far below the float32-vs-float64 parity tolerance of the costs.
// ---------------------------------------------------------------------------
template <int SYS>
struct Plant;

// Cart-pole (Lagrangian of a cart with a point-mass pole):
//   xdd  = [f + mp s (l thd^2 + g c)] / D,            D = mc + mp s^2
//   thdd = [-f c - mp l thd^2 c s - (mc + mp) g s] / (l D)
template <>
struct Plant<0> {
  static constexpr int n = 4, m = 1;
  __device__ __forceinline__ static void xdot(const DevPlant& p, const float* x, const float* v,
                                              float* xd) {
    float s, c;
    __sincosf(x[2], &s, &c);
    const float thd = x[3];
    const float D = p.mc + p.mp * s * s;
    const float thd2 = thd * thd;
    const float f = v[0];
    const float inv_D = __fdividef(1.0f, D);
    const float xdd = (f + p.mp * s * (p.l * thd2 + p.g * c)) * inv_D;
    const float thdd = (-f * c - p.mp * p.l * thd2 * c * s - p.mcp_g * s) * (inv_D * p.inv_l);
    xd[0] = x[1];
    xd[1] = xdd;
    xd[2] = thd;
    xd[3] = thdd;
  }
  __device__ __forceinline__ static float state_cost(const DevPlant& p, const float* x) {
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float e = x[i] - p.goal[i];
      s += p.Q[i] * e * e;
    }
    return s;
  }
  __device__ __forceinline__ static float terminal_cost(const DevPlant& p, const float* x) {
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float e = x[i] - p.goal[i];
      s += p.Qf[i] * e * e;
    }
    return s;
  }
};

// Quadrotor rigid body, ZYX Euler angles, "+" rotor layout:
//   p' = v,  v' = (sum f / m) R(eta) e3 - g e3,  eta' = W(eta) omega,
//   J omega' = tau - omega x J omega,
//   tau = (L (f2 - f4), L (f3 - f1), kappa (f1 - f2 + f3 - f4)).
template <>
struct Plant<1> {
  static constexpr int n = 12, m = 4;
  __device__ __forceinline__ static void xdot(const DevPlant& p, const float* x, const float* v,
                                              float* xd) {
    float sph, cph, sth, cth, sps, cps;
    __sincosf(x[6], &sph, &cph);
    __sincosf(x[7], &sth, &cth);
    __sincosf(x[8], &sps, &cps);
    const float wp = x[9], wq = x[10], wr = x[11];
    const float a = (v[0] + v[1] + v[2] + v[3]) * p.inv_mass;
    xd[0] = x[3];
    xd[1] = x[4];
    xd[2] = x[5];
    xd[3] = a * (cph * sth * cps + sph * sps);
    xd[4] = a * (cph * sth * sps - sph * cps);
    xd[5] = a * (cph * cth) - p.qg;
    // phi' = p + (sin phi q + cos phi r) tan theta, psi' = (sin phi q +
    // cos phi r) / cos theta: the common factor is formed while the
    // reciprocal of cos theta is computed, leaving two dependent operations
    // after it on the step's longest dependency chain
    const float inv_cth = __fdividef(1.0f, cth);
    const float a_qr = fmaf(sph, wq, cph * wr);
    const float b_qr = a_qr * inv_cth;
    xd[6] = fmaf(b_qr, sth, wp);
    xd[7] = cph * wq - sph * wr;
    xd[8] = b_qr;
    const float taux = p.arm * (v[1] - v[3]);
    const float tauy = p.arm * (v[2] - v[0]);
    const float tauz = p.kappa * (v[0] - v[1] + v[2] - v[3]);
    const float Jp = p.J[0] * wp, Jq = p.J[1] * wq, Jr = p.J[2] * wr;
    xd[9] = (taux - (wq * Jr - wr * Jq)) * p.invJ[0];
    xd[10] = (tauy - (wr * Jp - wp * Jr)) * p.invJ[1];
    xd[11] = (tauz - (wp * Jq - wq * Jp)) * p.invJ[2];
  }
  __device__ __forceinline__ static float quad_terms(const DevPlant& p, const float* x) {
    float ep = 0.0f, ev = 0.0f, ee = 0.0f, ew = 0.0f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float d = x[i] - p.pgoal[i];
      ep += d * d;
      ev += x[3 + i] * x[3 + i];
      ee += x[6 + i] * x[6 + i];
      ew += x[9 + i] * x[9 + i];
    }
    return p.wp * ep + p.wv * ev + p.weta * ee + p.wom * ew;
  }
  __device__ __forceinline__ static float state_cost(const DevPlant& p, const float* x) {
    float eo = 0.0f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float o = x[i] - p.obs[i];
      eo += o * o;
    }
    const float s = quad_terms(p, x);
    return eo < p.obs_r2 ? s + p.obs_cost : s;
  }
  __device__ __forceinline__ static float terminal_cost(const DevPlant& p, const float* x) {
    return quad_terms(p, x);
  }
};

}  // namespace mj
