/*
 * oracle.c -- plain FP64 CPU oracle for information-theoretic MPC on jump
 * diffusion processes (Wang, Williams & Theodorou, "Information Theoretic
 * Model Predictive Control on Jump Diffusion Processes").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference for the
 * CUDA library.  Only the test suite, the package entry point's smoke check
 * and the benchmark's CPU-baseline leg may load or call it; the product path
 * never does.  It shares no code, header, table or helper with the CUDA
 * sources: every step below is written from the paper (and, for the random
 * stream and the two plants, from the published definitions named beside
 * them), in the paper's order, in double precision, with no blocking or
 * fusion beyond what the method states.
 *
 * What it computes (one optimisation iteration of Algorithm 1):
 *   1. perturbations eps ~ N(0, c*Sigma_D) per rollout and step (Alg. 1,
 *      sampling step); here delta = eps/sqrt(dt) is drawn in control units,
 *      delta ~ N(0, c*diag(sigma^2)).
 *   2. jump counts per step: compound Poisson with E[dP] = nu*dt (Eq. 2), or
 *      the zero-one (Bernoulli) jump timer of Algorithm 1 / Sec. IV-B; marks
 *      N(0, Sigma_J) (Eq. 2) or, as an extension, Laplace(0, b).
 *   3. Euler rollout x_{j+1} = x_j + (f + G v_j) dt [+ H J_j] (Eq. 2, 4 and
 *      Algorithm 1) with the augmented cost S~ of Eq. 34-35 written in
 *      control units (R = lambda G^T Sigma^-1 G, Eq. 14; B = H = G, Sec. IV).
 *   4. weights w_m = exp(-S~_m/lambda) / sum exp(-S~/lambda)  (Eq. 36-37),
 *      evaluated with the minimum subtracted (exact by shift invariance).
 *   5. control update u_j += alpha * sum_m w_m delta_eff_{m,j}  (Eq. 37, 49).
 *   6. MPC step: repeat 1-5, emit u_0, shift, append u_init (Algorithm 1).
 *
 * Random stream (shared *definition* with the CUDA path, separate code):
 *   Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
 *   easy as 1, 2, 3", SC'11).  Key = (seed mod 2^32, seed >> 32).  Counter =
 *   (rollout k, block b, iteration it, stream s):
 *     s = 0: control normals; normal number f = j*m + i lives in block f/4,
 *            slot f%4 (Box-Muller on word pairs (0,1) and (2,3)).
 *     s = 1: jump-count words; step j uses block j/4, word j%4.
 *     s = 2+n: marks of the n-th jump at step j (block j): four normals
 *            (Normal law) or four uniforms (Laplace law), one per component.
 *   Uniform u(w) = ((w >> 9) + 1/2) * 2^-23, exact in float and double.
 *   Box-Muller (Box & Muller, 1958): r = sqrt(-2 ln u_a),
 *     z_a = r cos(2 pi u_b), z_b = r sin(2 pi u_b).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_JUMPS 16

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_ENONFINITE = 5 };

/* Problem description in double precision.  The Python wrapper fills it from
 * the same seeded problem dictionary that the CUDA binding reads. */
typedef struct {
  int32_t system; /* 0 = cartpole (n=4, m=1), 1 = quadrotor (n=12, m=4) */
  int32_t K;      /* rollouts M */
  int32_t T;      /* horizon steps N */
  double dt, lambda, c, alpha;
  double sigma[4]; /* std of the control-unit perturbation per channel */
  double nu;       /* jump rate (per second) */
  int32_t count_law;    /* 0 = Poisson, 1 = Bernoulli (zero-one law) */
  int32_t mark_law;     /* 0 = Normal, 1 = Laplace */
  double mark_scale[4]; /* Normal std or Laplace scale, per mark component */
  int32_t jump_channel; /* 0 = state rows (H selects rows), 1 = control */
  int32_t jump_sqrt_dt; /* state mode: 1 multiplies the jump by sqrt(dt) */
  int32_t noise_bf16;   /* 1: delta_eff is rounded to bfloat16 before use */
  int32_t q;            /* mark dimension */
  int32_t jump_rows[4]; /* state rows hit by the marks (state mode) */
  double u_init[4];
  uint64_t seed;
  /* cartpole */
  double cp_mc, cp_mp, cp_l, cp_g, cp_goal[4], cp_Q[4], cp_Qf[4];
  /* quadrotor */
  double qr_mass, qr_J[3], qr_arm, qr_kappa, qr_g, qr_goal[3];
  double qr_wp, qr_wv, qr_weta, qr_wom, qr_obs[3], qr_obs_r, qr_obs_cost;
  /* step sizes alpha^r = alpha * alpha_decay^r over the iterations r of one
   * MPC step (Eq. 48-49); 1 keeps alpha constant */
  double alpha_decay;
} orc_problem;

int orc_state_dim(const orc_problem* P) { return P->system == 0 ? 4 : 12; }
int orc_control_dim(const orc_problem* P) { return P->system == 0 ? 1 : 4; }

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, written from the SC'11 description: ten rounds of two      */
/* 32x32->64 multiplications whose halves are xored with the other counter   */
/* words and the round key; the key is bumped by the Weyl constants between */
/* rounds.                                                                   */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += W0;
    k1 += W1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Uniform on (0,1) from the top 23 bits: (y + 1/2) * 2^-23. */
double orc_uniform(uint32_t w) { return ((double)(w >> 9) + 0.5) * 0x1p-23; }

/* Four standard normals from one Philox block (two Box-Muller pairs). */
void orc_normals4(const uint32_t w[4], double z[4]) {
  const double two_pi = 6.283185307179586476925286766559;
  for (int p = 0; p < 2; ++p) {
    double ua = orc_uniform(w[2 * p]);
    double ub = orc_uniform(w[2 * p + 1]);
    double r = sqrt(-2.0 * log(ua));
    z[2 * p] = r * cos(two_pi * ub);
    z[2 * p + 1] = r * sin(two_pi * ub);
  }
}

static void draw_block(const orc_problem* P, uint32_t k, uint32_t b, uint32_t it,
                       uint32_t s, uint32_t out[4]) {
  uint32_t key[2] = {(uint32_t)(P->seed & 0xffffffffu), (uint32_t)(P->seed >> 32)};
  uint32_t ctr[4] = {k, b, it, s};
  orc_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* Jump-count thresholds.  Poisson (Eq. 2, E[dP] = nu dt): with mu = nu*dt  */
/* and F the Poisson CDF, T_n = ceil(2^32 F(n-1)); the count of a 32-bit    */
/* word w is #{n >= 1 : w >= T_n}, so P(count >= n) = 1 - F(n-1) up to      */
/* 2^-32.  Entries equal to 2^32 are unreachable and end the table.         */
/* Bernoulli (zero-one law, Algorithm 1 jump timer p < nu dt): one threshold */
/* T_B = round(2^32 mu) and count = [w < T_B].                              */
/* F is summed term by term: term_0 = e^-mu, term_n = term_{n-1}*mu/n.      */
/* ------------------------------------------------------------------------ */
int orc_count_table(double nu, double dt, int32_t law, uint32_t thr[ORC_MAX_JUMPS],
                    int32_t* nmax) {
  double mu = nu * dt;
  for (int i = 0; i < ORC_MAX_JUMPS; ++i) thr[i] = 0;
  *nmax = 0;
  if (!(mu >= 0.0) || !isfinite(mu)) return ORC_EINVAL;
  if (law == 1) {
    if (!(mu < 1.0)) return ORC_EINVAL;
    double t = floor(ldexp(mu, 32) + 0.5);
    thr[0] = (uint32_t)t;
    *nmax = thr[0] > 0 ? 1 : 0;
    return ORC_OK;
  }
  if (law != 0) return ORC_EINVAL;
  double term = exp(-mu);
  double F = term;
  int n;
  for (n = 1; n <= ORC_MAX_JUMPS + 1; ++n) {
    double t = ceil(ldexp(F, 32));
    if (t >= 4294967296.0) break;
    if (n > ORC_MAX_JUMPS) return ORC_EINVAL; /* tail beyond 16 jumps */
    thr[n - 1] = (uint32_t)t;
    term = term * mu / (double)n;
    F = F + term;
  }
  *nmax = n - 1;
  return ORC_OK;
}

static int count_from_word(int32_t law, const uint32_t* thr, int32_t nmax, uint32_t w) {
  if (law == 1) return (nmax > 0 && w < thr[0]) ? 1 : 0;
  int n = 0;
  while (n < nmax && w >= thr[n]) ++n;
  return n;
}

/* ------------------------------------------------------------------------ */
/* Plants (the paper names them but prints no equations; textbook forms).   */
/* Both are control affine, F(x, v) = f(x) + G(x) v (Eq. 4).                */
/* ------------------------------------------------------------------------ */

/* Cart-pole: point-mass pole of mass mp at distance l from the pivot, theta
 * measured from hanging down, frictionless; from the Lagrangian
 * L = 1/2 (mc+mp) xd^2 + mp l xd thd cos(th) + 1/2 mp l^2 thd^2 + mp g l cos(th). */
static void cartpole_xdot(const orc_problem* P, const double* x, const double* v, double* xd) {
  double mc = P->cp_mc, mp = P->cp_mp, l = P->cp_l, g = P->cp_g;
  double s = sin(x[2]), co = cos(x[2]);
  double thd = x[3];
  double D = mc + mp * s * s;
  double f = v[0];
  double xdd = (f + mp * s * (l * thd * thd + g * co)) / D;
  double thdd = (-f * co - mp * l * thd * thd * co * s - (mc + mp) * g * s) / (l * D);
  xd[0] = x[1];
  xd[1] = xdd;
  xd[2] = thd;
  xd[3] = thdd;
}

/* Quadrotor: rigid body, ZYX Euler angles eta = (phi, theta, psi), body rates
 * omega = (p, q, r), four rotor thrusts f1..f4 in a "+" layout with rotors 1,
 * 2, 3, 4 on the body +x, +y, -x, -y arms (arm length L) and rotors 1, 3
 * spinning against 2, 4 (reaction torque kappa per unit thrust):
 *   tau = (L (f2 - f4), L (f3 - f1), kappa (f1 - f2 + f3 - f4)).
 *   p'     = v
 *   v'     = (sum f / m) R(eta) e3 - g e3
 *   eta'   = W(eta) omega
 *   J w'   = tau - omega x (J omega)                                        */
static void quadrotor_xdot(const orc_problem* P, const double* x, const double* v, double* xd) {
  double m = P->qr_mass, L = P->qr_arm, kap = P->qr_kappa, g = P->qr_g;
  double Jx = P->qr_J[0], Jy = P->qr_J[1], Jz = P->qr_J[2];
  double ph = x[6], th = x[7], ps = x[8];
  double p = x[9], q = x[10], r = x[11];
  double sph = sin(ph), cph = cos(ph), sth = sin(th), cth = cos(th);
  double sps = sin(ps), cps = cos(ps);
  double thrust = v[0] + v[1] + v[2] + v[3];
  double Re3x = cph * sth * cps + sph * sps;
  double Re3y = cph * sth * sps - sph * cps;
  double Re3z = cph * cth;
  xd[0] = x[3];
  xd[1] = x[4];
  xd[2] = x[5];
  xd[3] = thrust / m * Re3x;
  xd[4] = thrust / m * Re3y;
  xd[5] = thrust / m * Re3z - g;
  double tth = sth / cth;
  xd[6] = p + sph * tth * q + cph * tth * r;
  xd[7] = cph * q - sph * r;
  xd[8] = (sph * q + cph * r) / cth;
  double taux = L * (v[1] - v[3]);
  double tauy = L * (v[2] - v[0]);
  double tauz = kap * (v[0] - v[1] + v[2] - v[3]);
  double cx = q * (Jz * r) - r * (Jy * q);
  double cy = r * (Jx * p) - p * (Jz * r);
  double cz = p * (Jy * q) - q * (Jx * p);
  xd[9] = (taux - cx) / Jx;
  xd[10] = (tauy - cy) / Jy;
  xd[11] = (tauz - cz) / Jz;
}

void orc_xdot(const orc_problem* P, const double* x, const double* v, double* xd) {
  if (P->system == 0) cartpole_xdot(P, x, v, xd);
  else quadrotor_xdot(P, x, v, xd);
}

/* State cost q(x) of Eq. 3 and terminal cost phi(x_T) of Eq. 1. */
double orc_state_cost(const orc_problem* P, const double* x) {
  if (P->system == 0) {
    double s = 0.0;
    for (int i = 0; i < 4; ++i) {
      double e = x[i] - P->cp_goal[i];
      s += P->cp_Q[i] * e * e;
    }
    return s;
  }
  double ep = 0.0, ev = 0.0, ee = 0.0, ew = 0.0, eo = 0.0;
  for (int i = 0; i < 3; ++i) {
    double d = x[i] - P->qr_goal[i];
    ep += d * d;
    ev += x[3 + i] * x[3 + i];
    ee += x[6 + i] * x[6 + i];
    ew += x[9 + i] * x[9 + i];
    double o = x[i] - P->qr_obs[i];
    eo += o * o;
  }
  double s = P->qr_wp * ep + P->qr_wv * ev + P->qr_weta * ee + P->qr_wom * ew;
  if (eo < P->qr_obs_r * P->qr_obs_r) s += P->qr_obs_cost;
  return s;
}

double orc_terminal_cost(const orc_problem* P, const double* x) {
  if (P->system == 0) {
    double s = 0.0;
    for (int i = 0; i < 4; ++i) {
      double e = x[i] - P->cp_goal[i];
      s += P->cp_Qf[i] * e * e;
    }
    return s;
  }
  double ep = 0.0, ev = 0.0, ee = 0.0, ew = 0.0;
  for (int i = 0; i < 3; ++i) {
    double d = x[i] - P->qr_goal[i];
    ep += d * d;
    ev += x[3 + i] * x[3 + i];
    ee += x[6 + i] * x[6 + i];
    ew += x[9 + i] * x[9 + i];
  }
  return P->qr_wp * ep + P->qr_wv * ev + P->qr_weta * ee + P->qr_wom * ew;
}

/* Signed squared distance margin to the obstacle sphere (quadrotor), used by
 * tests to recognise rollouts whose indicator decision sits on the boundary. */
double orc_obstacle_margin(const orc_problem* P, const double* x) {
  if (P->system != 1) return INFINITY;
  double eo = 0.0;
  for (int i = 0; i < 3; ++i) {
    double o = x[i] - P->qr_obs[i];
    eo += o * o;
  }
  return eo - P->qr_obs_r * P->qr_obs_r;
}

/* ------------------------------------------------------------------------ */
/* bfloat16 storage: a float32 value is rounded to the nearest bfloat16,     */
/* ties to even.  The decision is taken on the float32 value (the precision */
/* the stored perturbation is produced in); values whose double-precision  */
/* origin lies within 2^-20 (relative) of a rounding midpoint are flagged   */
/* as ambiguous, since a float32 computation may land on either side.       */
/* ------------------------------------------------------------------------ */
static float bf16_round(float f) {
  uint32_t b;
  memcpy(&b, &f, 4);
  if ((b & 0x7f800000u) == 0x7f800000u) {
    if (b & 0x007fffffu) b |= 0x00400000u; /* keep NaN a NaN */
    b &= 0xffff0000u;
  } else {
    uint32_t lsb = (b >> 16) & 1u;
    b += 0x7fffu + lsb;
    b &= 0xffff0000u;
  }
  memcpy(&f, &b, 4);
  return f;
}

static int bf16_ambiguous(double d) {
  float f = (float)d;
  uint32_t b;
  memcpy(&b, &f, 4);
  if ((b & 0x7f800000u) == 0x7f800000u || d == 0.0) return 0;
  uint32_t lo_b = b & 0xffff0000u;
  float lo, hi;
  memcpy(&lo, &lo_b, 4);
  uint32_t hi_b = lo_b + 0x10000u;
  memcpy(&hi, &hi_b, 4);
  double mid = 0.5 * ((double)lo + (double)hi);
  return fabs(d - mid) <= ldexp(fabs(d), -20);
}

double orc_bf16_round(double d) { return (double)bf16_round((float)d); }

/* The ambiguity test above, exported for the tests that pin it. */
int orc_bf16_ambiguous(double d) { return bf16_ambiguous(d); }

/* ------------------------------------------------------------------------ */
/* One rollout (the inner loop of Algorithm 1) for rollout index k.          */
/*   delta_{j,i} = sqrt(c) sigma_i z          (eps ~ N(0, c Sigma_D))        */
/*   N_j = jump count, J_j = sum of N_j marks (Eq. 2 / zero-one law)         */
/*   delta_eff = delta + J (control channel, Algorithm 1 / Eq. 49) or delta  */
/*   S~ += q(x_j) dt + lambda [ 1/2 u^T S^-1 u + u^T S^-1 delta_eff          */
/*                              + 1/2 (1 - 1/c) delta_eff^T S^-1 delta_eff ] */
/*        (Eq. 34-35 with R = lambda G^T Sigma^-1 G, B = G, eps = delta*sqrt(dt),*/
/*         Sigma_D = dt * diag(sigma^2); S = diag(sigma^2))                  */
/*   x_{j+1} = x_j + F(x_j, u_j + delta_eff) dt [+ s H J_j in state mode]    */
/*   S~ += phi(x_T)                                                          */
/* Optional outputs are laid out step-major: counts[j*kc + kk],              */
/* delta[(j*kc + kk)*m + i], J[(j*kc + kk)*q + c] with kk = k - k_begin.     */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint32_t thr[ORC_MAX_JUMPS];
  int32_t nmax;
} orc_table;

static double rollout_one(const orc_problem* P, const orc_table* tab, const double* x0,
                          const double* U, uint32_t it, uint32_t k, int kk, int kc,
                          uint8_t* counts, double* delta, double* Jout, uint8_t* ambig,
                          double* traj, double* min_margin) {
  const int n = orc_state_dim(P), m = orc_control_dim(P), q = P->q, T = P->T;
  const double dt = P->dt, lam = P->lambda, sqc = sqrt(P->c);
  const double s_jump = P->jump_sqrt_dt ? sqrt(dt) : 1.0;
  double x[12], xd[12], v[4], d[4], J[4], z[4];
  uint32_t w[4];
  for (int i = 0; i < n; ++i) x[i] = x0[i];
  double S = 0.0;
  double margin = INFINITY;
  int cached_block = -1;
  double zb[4] = {0, 0, 0, 0};
  for (int j = 0; j < T; ++j) {
    if (traj) for (int i = 0; i < n; ++i) traj[(size_t)j * n + i] = x[i];
    /* Gaussian perturbation, stream 0 */
    for (int i = 0; i < m; ++i) {
      int f = j * m + i;
      if (f / 4 != cached_block) {
        cached_block = f / 4;
        draw_block(P, k, (uint32_t)cached_block, it, 0u, w);
        orc_normals4(w, zb);
      }
      d[i] = sqc * P->sigma[i] * zb[f % 4];
    }
    /* jump count, stream 1 */
    draw_block(P, k, (uint32_t)(j / 4), it, 1u, w);
    int N = count_from_word(P->count_law, tab->thr, tab->nmax, w[j % 4]);
    for (int c = 0; c < q; ++c) J[c] = 0.0;
    for (int nj = 0; nj < N; ++nj) {
      draw_block(P, k, (uint32_t)j, it, 2u + (uint32_t)nj, w);
      if (P->mark_law == 0) {
        orc_normals4(w, z);
        for (int c = 0; c < q; ++c) J[c] += P->mark_scale[c] * z[c];
      } else {
        for (int c = 0; c < q; ++c) {
          double u = orc_uniform(w[c]);
          double h = u - 0.5;
          double sg = h > 0.0 ? 1.0 : -1.0;
          J[c] += -P->mark_scale[c] * sg * log(1.0 - 2.0 * fabs(h));
        }
      }
    }
    /* effective perturbation */
    double de[4];
    for (int i = 0; i < m; ++i) de[i] = d[i] + (P->jump_channel == 1 ? J[i] : 0.0);
    if (P->noise_bf16) {
      for (int i = 0; i < m; ++i) {
        if (ambig && bf16_ambiguous(de[i])) ambig[((size_t)j * kc + kk) * m + i] = 1;
        de[i] = orc_bf16_round(de[i]);
      }
    }
    /* augmented running cost, Eq. 34-35 */
    double uSu = 0.0, uSd = 0.0, dSd = 0.0;
    for (int i = 0; i < m; ++i) {
      double is2 = 1.0 / (P->sigma[i] * P->sigma[i]);
      double u = U[(size_t)j * m + i];
      uSu += u * is2 * u;
      uSd += u * is2 * de[i];
      dSd += de[i] * is2 * de[i];
    }
    S += orc_state_cost(P, x) * dt +
         lam * (0.5 * uSu + uSd + 0.5 * (1.0 - 1.0 / P->c) * dSd);
    double mg = orc_obstacle_margin(P, x);
    if (fabs(mg) < margin) margin = fabs(mg);
    /* Euler step with the jump, Algorithm 1 / Eq. 2 */
    for (int i = 0; i < m; ++i) v[i] = U[(size_t)j * m + i] + de[i];
    orc_xdot(P, x, v, xd);
    for (int i = 0; i < n; ++i) x[i] = x[i] + xd[i] * dt;
    if (P->jump_channel == 0)
      for (int c = 0; c < q; ++c) x[P->jump_rows[c]] += s_jump * J[c];
    if (counts) counts[(size_t)j * kc + kk] = (uint8_t)N;
    if (delta) for (int i = 0; i < m; ++i) delta[((size_t)j * kc + kk) * m + i] = de[i];
    if (Jout) for (int c = 0; c < q; ++c) Jout[((size_t)j * kc + kk) * q + c] = J[c];
  }
  if (traj) for (int i = 0; i < n; ++i) traj[(size_t)T * n + i] = x[i];
  S += orc_terminal_cost(P, x);
  if (!isfinite(S)) S = INFINITY;
  if (min_margin) *min_margin = margin;
  return S;
}

static int validate(const orc_problem* P, orc_table* tab) {
  if (P->system != 0 && P->system != 1) return ORC_EINVAL;
  if (P->K < 1 || P->T < 1) return ORC_EINVAL;
  if (!(P->dt > 0) || !(P->lambda > 0) || !(P->c > 0)) return ORC_EINVAL;
  int m = orc_control_dim(P);
  for (int i = 0; i < m; ++i)
    if (!(P->sigma[i] > 0)) return ORC_EINVAL;
  if (P->q < 0 || P->q > 4) return ORC_EINVAL;
  if (P->jump_channel == 1 && P->q != m) return ORC_EINVAL;
  if (P->jump_channel == 0)
    for (int c = 0; c < P->q; ++c)
      if (P->jump_rows[c] < 0 || P->jump_rows[c] >= orc_state_dim(P)) return ORC_EINVAL;
  return orc_count_table(P->nu, P->dt, P->count_law, tab->thr, &tab->nmax);
}

/* Rollouts k_begin .. k_begin+kc-1 of iteration `it`.  S_out[kk] receives S~.
 * Any of counts / delta / J / ambig / margin may be NULL; ambig must be zeroed
 * by the caller. traj (if given) holds (T+1)*n doubles per rollout. */
int orc_rollouts(const orc_problem* P, const double* x0, const double* U, uint32_t it,
                 int32_t k_begin, int32_t kc, double* S_out, uint8_t* counts, double* delta,
                 double* Jout, uint8_t* ambig, double* traj, double* margin, int32_t nthreads) {
  orc_table tab;
  int st = validate(P, &tab);
  if (st) return st;
  if (k_begin < 0 || kc < 0) return ORC_EINVAL;
  const int n = orc_state_dim(P);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
  for (int kk = 0; kk < kc; ++kk) {
    S_out[kk] = rollout_one(P, &tab, x0, U, it, (uint32_t)(k_begin + kk), kk, kc, counts,
                            delta, Jout, ambig, traj ? traj + (size_t)kk * (P->T + 1) * n : NULL,
                            margin ? margin + kk : NULL);
  }
  (void)nthreads;
  return ORC_OK;
}

/* Free-energy weights of Eq. 36-37: rho = min S~, e_k = exp(-(S~_k - rho)/lambda),
 * Z = sum e_k, w_k = e_k / Z.  Non-finite costs get weight 0; if every cost is
 * non-finite the call fails with ORC_ENONFINITE.  diag = {rho, Z, F} with the
 * Monte Carlo free energy of Eq. 5, F = rho/lambda - ln(Z/K). */
int orc_softmin(int32_t K, const double* S, double lambda, double* w, double* diag) {
  double rho = INFINITY;
  for (int k = 0; k < K; ++k)
    if (isfinite(S[k]) && S[k] < rho) rho = S[k];
  if (!isfinite(rho)) return ORC_ENONFINITE;
  double Z = 0.0;
  for (int k = 0; k < K; ++k) {
    w[k] = isfinite(S[k]) ? exp(-(S[k] - rho) / lambda) : 0.0;
    Z += w[k];
  }
  for (int k = 0; k < K; ++k) w[k] = w[k] / Z;
  if (diag) {
    diag[0] = rho;
    diag[1] = Z;
    diag[2] = rho / lambda - log(Z / (double)K);
  }
  return ORC_OK;
}

/* Weighted update of Eq. 37 / 49: U_{j,i} += alpha * sum_k w_k delta_eff_{j,k,i},
 * delta laid out [T][K][m]; the sum runs over k in increasing order. */
void orc_update(int32_t K, int32_t T, int32_t m, const double* w, const double* delta,
                double alpha, double* U) {
  for (int j = 0; j < T; ++j)
    for (int i = 0; i < m; ++i) {
      double s = 0.0;
      for (int k = 0; k < K; ++k) s += w[k] * delta[((size_t)j * K + k) * m + i];
      U[(size_t)j * m + i] += alpha * s;
    }
}

/* One optimisation iteration (Algorithm 1 without the shift): rollouts for all
 * K, weights, update of U in place.  Optional outputs: S (K), w (K), counts
 * (T*K), delta (T*K*m), diag (3), ambig (T*K*m, zeroed by the caller). */
int orc_iteration(const orc_problem* P, const double* x0, double* U, uint32_t it,
                  double* S_out, double* w_out, uint8_t* counts, double* delta_out,
                  double* diag, uint8_t* ambig, int32_t nthreads) {
  const int K = P->K, T = P->T, m = orc_control_dim(P);
  double* S = S_out ? S_out : (double*)malloc(sizeof(double) * K);
  double* w = w_out ? w_out : (double*)malloc(sizeof(double) * K);
  double* delta = delta_out ? delta_out : (double*)malloc(sizeof(double) * (size_t)T * K * m);
  int st = ORC_ENOMEM;
  if (S && w && delta) {
    st = orc_rollouts(P, x0, U, it, 0, K, S, counts, delta, NULL, ambig, NULL, NULL, nthreads);
    if (st == ORC_OK) st = orc_softmin(K, S, P->lambda, w, diag);
    if (st == ORC_OK) orc_update(K, T, m, w, delta, P->alpha, U);
  }
  if (!S_out) free(S);
  if (!w_out) free(w);
  if (!delta_out) free(delta);
  return st;
}

/* One MPC step of Algorithm 1: `iters` iterations starting at counter it0
 * from the same x0, iteration r with the step size alpha^r = alpha *
 * alpha_decay^r of the stochastic-optimisation update (Eq. 48-49), then
 * execute u_0 (returned in u0_out), shift the sequence by one step and append
 * u_init. */
int orc_step(const orc_problem* P, const double* x0, double* U, uint32_t it0, int32_t iters,
             double* u0_out, int32_t nthreads) {
  const int T = P->T, m = orc_control_dim(P);
  if (iters < 1) return ORC_EINVAL;
  orc_problem Pr = *P;
  for (int r = 0; r < iters; ++r) {
    Pr.alpha = P->alpha * pow(P->alpha_decay, (double)r);
    int st = orc_iteration(&Pr, x0, U, it0 + (uint32_t)r, NULL, NULL, NULL, NULL, NULL, NULL,
                           nthreads);
    if (st) return st;
  }
  for (int i = 0; i < m; ++i) u0_out[i] = U[i];
  for (int j = 0; j + 1 < T; ++j)
    for (int i = 0; i < m; ++i) U[(size_t)j * m + i] = U[(size_t)(j + 1) * m + i];
  for (int i = 0; i < m; ++i) U[(size_t)(T - 1) * m + i] = P->u_init[i];
  return ORC_OK;
}
