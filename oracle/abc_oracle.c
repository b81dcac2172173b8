/*
 * abc_oracle.c -- plain, slow, sequential CPU oracle for P-ABC-SMC with
 * Beta-distributed step sizes (arXiv 2106.15508).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The
 * product path (paper_2106_15508_gb300) never calls it and shares no code,
 * header, table or constant with it.
 *
 * Every function cites the passage of the paper it follows.  The paper fixes
 * the method but not its floating-point detail; the operation order below is
 * the project's numerics specification (fp32 for per-particle arithmetic,
 * explicit fmaf where the spec says fma, no contraction otherwise), written
 * from the mathematics:
 *   - Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 *     easy as 1, 2, 3", SC'11.
 *   - log/exp/expm1: Cody & Waite argument reduction (x = k ln2 + r) with the
 *     Taylor series of exp and the atanh series of log, coefficients the
 *     fp32 values nearest to 1/k! and 1/(2k+1).
 *   - log1p: Goldberg's identity log1p(x) = x log(u)/(u-1), u = 1+x.
 *   - cos(2 pi w): reduction in turns by symmetry, Taylor series of sin/cos.
 *   - Binomial: BINV inversion (Kachitvichyanukul & Schmeiser 1988) when the
 *     mean is below 10, else a rounded normal approximation.
 *   - Beta(a, b) for integer b: product of B(a+m, 1) variates.
 *
 * Parity status of every function is stated in the tests that pin it; the
 * end-to-end SAIRD posterior has no ground truth ("parity unpinned" beyond
 * oracle agreement, the invariants and recovery of the true parameters).
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared [-fopenmp]
 * (-ffp-contract=off is mandatory: it forbids the compiler from fusing a*b+c).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11): 10 rounds of two 32x32->64 multiplies, key bumped   */
/* by the Weyl constants between rounds.                                      */
/* ------------------------------------------------------------------------ */
OR_API void or_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
    uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
    uint32_t y1 = (uint32_t)p1;
    uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
    uint32_t y3 = (uint32_t)p0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void philox_ctr(const uint32_t key[2], uint32_t c0, uint32_t c1, uint32_t c2,
                       uint32_t c3, uint32_t out[4]) {
  uint32_t c[4] = {c0, c1, c2, c3};
  or_philox(c, key, out);
}

/* Stream tags: the fourth counter word. */
enum { TAG_PRIOR = 0, TAG_ANCESTOR = 1, TAG_BETA = 2, TAG_WALK = 3, TAG_SIM = 4,
       TAG_SCREEN = 5, TAG_AUDIT = 6, TAG_OBS = 7, TAG_OBS_THETA = 8, TAG_PREDICT = 11,
       TAG_PREDICT_SIM = 12 };

/* u32 -> (0,1): the top 23 bits plus one half, times 2^-23.  Every step is
 * exact in fp32 and the result lies in [2^-24, 1 - 2^-24] (with 24 bits the
 * largest value would round up to 1). */
OR_API float or_uniform(uint32_t x) {
  return ((float)(x >> 9) + 0.5f) * 0x1p-23f;
}

/* ------------------------------------------------------------------------ */
/* Transcendentals (fp32).                                                    */
/* ------------------------------------------------------------------------ */
static const float LN2_HI = 0x1.62e4p-1f;      /* 0.693145751953125, 15 significant bits */
static const float LN2_LO = 0x1.7f7d1cp-20f;   /* fp32 nearest to ln2 - LN2_HI */
static const float LOG2E  = 0x1.715476p+0f;    /* fp32 nearest to 1/ln2 */
static const float TWO_PI = 0x1.921fb6p+2f;    /* fp32 nearest to 2 pi */
static const float SQRT2F = 0x1.6a09e6p+0f;    /* fp32 nearest to sqrt 2 */
/* fp32 nearest to 1/k!, k = 0..13 */
static const float INV_FACT[14] = {
  1.0f, 1.0f, 0.5f, 0x1.555556p-3f, 0x1.555556p-5f, 0x1.111112p-7f, 0x1.6c16c2p-10f,
  0x1.a01a02p-13f, 0x1.a01a02p-16f, 0x1.71de3ap-19f, 0x1.27e4fcp-22f, 0x1.ae6456p-26f,
  0x1.1eed8ep-29f, 0x1.612462p-33f};
/* fp32 nearest to 1/(2k+1), k = 1..5 */
static const float INV_ODD[6] = {1.0f, 0x1.555556p-2f, 0x1.99999ap-3f, 0x1.24924ap-3f,
                                 0x1.c71c72p-4f, 0x1.745d18p-4f};

static inline uint32_t f2u(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static inline float u2f(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }

/* Exposes the constants so that a test can pin them to their definitions. */
OR_API int or_constants(float* out, int n) {
  float all[5 + 14 + 5] = {LN2_HI, LN2_LO, LOG2E, TWO_PI, SQRT2F};
  for (int k = 0; k < 14; ++k) all[5 + k] = INV_FACT[k];
  for (int k = 1; k <= 5; ++k) all[18 + k] = INV_ODD[k];
  int m = n < 24 ? n : 24;
  for (int i = 0; i < m; ++i) out[i] = all[i];
  return 24;
}

/* natural log: x = m 2^e, m in [sqrt(1/2), sqrt 2), log m = 2 atanh(f),
 * f = (m-1)/(m+1), series up to f^11; result e*LN2_HI + (e*LN2_LO + log m). */
OR_API float or_logf(float x) {
  if (x != x || x < 0.0f) return NAN;
  if (x == 0.0f) return -INFINITY;
  if (x == INFINITY) return INFINITY;
  int e = 0;
  if (x < 0x1p-126f) { x = x * 0x1p24f; e = -24; }
  uint32_t b = f2u(x);
  e += (int)(b >> 23) - 127;
  float m = u2f((b & 0x007FFFFFu) | 0x3F800000u);
  if (m > SQRT2F) { m = m * 0.5f; e = e + 1; }
  float f = (m - 1.0f) / (m + 1.0f);
  float f2 = f * f;
  float p = INV_ODD[5];
  p = fmaf(p, f2, INV_ODD[4]);
  p = fmaf(p, f2, INV_ODD[3]);
  p = fmaf(p, f2, INV_ODD[2]);
  p = fmaf(p, f2, INV_ODD[1]);
  float t = f2 * p;
  float r = f + f;
  float lm = fmaf(r, t, r);
  float fe = (float)e;
  float hi = fe * LN2_HI;
  float lo = fmaf(fe, LN2_LO, lm);
  return hi + lo;
}

/* 2^k as fp32 for k in [-126, 127] */
static inline float pow2i(int k) { return u2f((uint32_t)(k + 127) << 23); }

/* multiply by 2^k with at most one rounding (into the subnormal range) */
static float scale2(float p, int k) {
  if (k > 127) return (p * 0x1p127f) * pow2i(k - 127);
  if (k < -126) return (p * pow2i(k + 64)) * 0x1p-64f;
  return p * pow2i(k);
}

/* exp: k = floor(x log2e + 1/2), r = (x - k LN2_HI) - k LN2_LO, Taylor to r^8. */
OR_API float or_expf(float x) {
  if (x != x) return x;
  if (x > 88.72283935546875f) return INFINITY;
  if (x < -103.972084045410156f) return 0.0f;
  float kf = floorf(x * LOG2E + 0.5f);
  int k = (int)kf;
  float r = x - kf * LN2_HI;
  r = r - kf * LN2_LO;
  float p = INV_FACT[8];
  for (int i = 7; i >= 0; --i) p = fmaf(p, r, INV_FACT[i]);
  return scale2(p, k);
}

/* Taylor series of expm1 on |r| <= ln2/2 up to r^9: r + r^2 (1/2 + r/6 + ...) */
static float expm1_series(float r) {
  float q = INV_FACT[9];
  for (int i = 8; i >= 2; --i) q = fmaf(q, r, INV_FACT[i]);
  float t = r * r;
  return fmaf(t, q, r);
}

OR_API float or_expm1f(float x) {
  if (x != x) return x;
  if (x > 88.72283935546875f) return INFINITY;
  if (x < -17.5f) return -1.0f;
  if (fabsf(x) <= 0.3465735912322998f) return expm1_series(x);
  float kf = floorf(x * LOG2E + 0.5f);
  int k = (int)kf;
  float r = x - kf * LN2_HI;
  r = r - kf * LN2_LO;
  float em = expm1_series(r);
  if (k > 127) return INFINITY;
  float two = pow2i(k);
  return fmaf(two, em, two - 1.0f);
}

/* log1p(x), x > -1: Goldberg's identity. */
OR_API float or_log1pf(float x) {
  float u = 1.0f + x;
  if (u == 1.0f) return x;
  return (or_logf(u) / (u - 1.0f)) * x;
}

/* cos(2 pi w) for w in [0, 1]. */
OR_API float or_cos2pi(float w) {
  float v = w;
  if (v > 0.5f) v = 1.0f - v;             /* cos(2pi(1-v)) = cos(2pi v), exact */
  float sign = 1.0f;
  if (v > 0.25f) { v = 0.5f - v; sign = -1.0f; }  /* cos(pi - y) = -cos y, exact */
  float c;
  if (v <= 0.125f) {
    float x = v * TWO_PI;
    float x2 = x * x;
    /* cos x = sum (-1)^k x^2k/(2k)!, k = 0..6 */
    float p = INV_FACT[12];
    p = fmaf(p, x2, -INV_FACT[10]);
    p = fmaf(p, x2, INV_FACT[8]);
    p = fmaf(p, x2, -INV_FACT[6]);
    p = fmaf(p, x2, INV_FACT[4]);
    p = fmaf(p, x2, -INV_FACT[2]);
    c = fmaf(p, x2, 1.0f);
  } else {
    float x = (0.25f - v) * TWO_PI;          /* cos(pi/2 - y) = sin y */
    float x2 = x * x;
    /* sin x = x + x x2 Q(x2), Q = sum_{k=1..6} (-1)^k x2^(k-1)/(2k+1)! */
    float q = INV_FACT[13];
    q = fmaf(q, x2, -INV_FACT[11]);
    q = fmaf(q, x2, INV_FACT[9]);
    q = fmaf(q, x2, -INV_FACT[7]);
    q = fmaf(q, x2, INV_FACT[5]);
    q = fmaf(q, x2, -INV_FACT[3]);
    c = fmaf(x * x2, q, x);
  }
  return sign * c;
}

/* Box-Muller, cosine branch only. */
OR_API float or_normal(float w1, float w2) {
  float l = or_logf(w1);
  float t = -2.0f * l;
  float r = sqrtf(t);
  return r * or_cos2pi(w2);
}

/* ------------------------------------------------------------------------ */
/* Binomial(n, p) from two uniforms (exact-count daily transitions:        */
/* the paper's tau-leap flows, Sec. 2.2, as exact-count competing risks).    */
/* ------------------------------------------------------------------------ */
OR_API int32_t or_binomial(int32_t n, float p, float w1, float w2) {
  if (n <= 0 || !(p > 0.0f)) return 0;
  if (p >= 1.0f) return n;
  int flip = p > 0.5f;
  float q = flip ? (1.0f - p) : p;
  float nf = (float)n;
  float mu = nf * q;
  int32_t k;
  if (mu < 10.0f) {
    /* BINV: walk the pmf from 0, f(x) = f(x-1) (a/x - s) */
    float s = q / (1.0f - q);
    float a = (nf + 1.0f) * s;
    float r = or_expf(nf * or_log1pf(-q));
    float u = w1;
    int32_t cap = n < 110 ? n : 110;
    int32_t x = 0;
    for (;;) {
      if (u <= r) break;
      if (x == cap) break;
      u = u - r;
      x = x + 1;
      r = r * (a / (float)x - s);
    }
    k = x;
  } else {
    float sd = sqrtf(mu * (1.0f - q));
    float z = or_normal(w1, w2);
    float y = floorf((mu + sd * z) + 0.5f);
    if (y < 0.0f) y = 0.0f;
    if (y > nf) y = nf;
    k = (int32_t)y;
    if (k > n) k = n;
  }
  return flip ? n - k : k;
}

/* Paper's flow draw (Sec. 2.2): floor(Normal(h, sd sqrt h)), clamped to [0, cap]. */
static int32_t paper_flow(float h, int32_t cap, float w1, float w2) {
  if (cap <= 0 || !(h > 0.0f)) return 0;
  float z = or_normal(w1, w2);
  float y = floorf(h + sqrtf(h) * z);
  if (y < 0.0f) y = 0.0f;
  if (y > (float)cap) y = (float)cap;
  int32_t k = (int32_t)y;
  return k > cap ? cap : k;
}

/* ------------------------------------------------------------------------ */
/* Model description                                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t model;        /* 0 = stochastic SAIRD (Sec. 2.2), 1 = Gaussian toy      */
  int32_t sampler;      /* 0 = binomial transitions, 1 = paper floor-normal      */
  int32_t T;            /* days                                                  */
  int32_t pad0;
  int64_t P;            /* population                                            */
  int32_t A0, R0, D0;   /* observed day-0 state                                  */
  int32_t pad1;
  float theta_lo[8];    /* prior U(theta_lo, theta_hi) (Eq. 2)                   */
  float theta_hi[8];
  const int32_t* obs;   /* [3][T+1] rows A, R, D; column t = day t               */
  float x_obs[8];       /* toy model observation                                 */
  uint32_t key[2];      /* Philox key = (seed_lo, seed_hi ^ run)                  */
} or_model;

/* theta_d = lo_d + u_d (hi_d - lo_d), the paper's reparameterisation (Sec. 3.1) */
static void theta_from_u(const or_model* m, const float u[8], float th[8]) {
  for (int d = 0; d < 8; ++d) {
    float w = m->theta_hi[d] - m->theta_lo[d];
    th[d] = m->theta_lo[d] + u[d] * w;
  }
}

/* Correctly rounded double of an unsigned 128-bit integer (gcc's conversion). */
static double u128_to_double(unsigned __int128 v) { return (double)v; }

/*
 * One stochastic SAIRD trajectory (Sec. 2.2, Eq. 3-5) and its Euclidean
 * distance to the observed A, R, D series over days 1..T (Sec. 2.3).
 * theta = [alpha0, alpha, n, beta, gamma, delta, eta, kappa] (Eq. 1).
 * Philox counters: (c0, c1, 4 day + block, tag), blocks 0..2 per day.
 * traj (nullable): [T+1][6][stride] compartments S, I, A, R, D, Ru.
 */
static double simulate_saird(const or_model* m, const float th[8], uint32_t c0, uint32_t c1,
                             uint32_t tag, int32_t* traj, int64_t stride, int64_t col,
                             int32_t* out_ard) {
  float alpha0 = th[0], alpha = th[1], n = th[2], beta = th[3], gamma = th[4],
        delta = th[5], eta = th[6], kappa = th[7];
  /* initial state: Ru = 0, I0 = kappa A0, S = P - (A0 + R0 + D0 + I0) */
  int64_t A = m->A0, R = m->R0, D = m->D0;
  int64_t I = (int64_t)floorf(kappa * (float)m->A0);
  int64_t S = m->P - (A + R + D + I);
  if (S < 0) { I = m->P - (A + R + D); if (I < 0) I = 0; S = 0; }
  int64_t Ru = 0;
  float Pf = (float)m->P;
  /* per-particle constants of the competing risks out of I and A */
  float lamI = gamma + beta * eta;            /* I -> A at gamma, I -> Ru at beta eta */
  float lamA = beta + delta;                  /* A -> R at beta, A -> D at delta */
  float pI = -or_expm1f(-lamI);
  float pA = -or_expm1f(-lamA);
  float fI = lamI > 0.0f ? gamma / lamI : 0.0f;
  float fA = lamA > 0.0f ? beta / lamA : 0.0f;
  unsigned __int128 acc = 0;
  if (traj) {
    int32_t* t0 = traj + col;
    t0[0 * stride] = (int32_t)S; t0[1 * stride] = (int32_t)I; t0[2 * stride] = (int32_t)A;
    t0[3 * stride] = (int32_t)R; t0[4 * stride] = (int32_t)D; t0[5 * stride] = (int32_t)Ru;
  }
  for (int32_t day = 0; day < m->T; ++day) {
    uint32_t w[12];
    philox_ctr(m->key, c0, c1, (uint32_t)day * 4u + 0u, tag, w + 0);
    philox_ctr(m->key, c0, c1, (uint32_t)day * 4u + 1u, tag, w + 4);
    philox_ctr(m->key, c0, c1, (uint32_t)day * 4u + 2u, tag, w + 8);
    float v[10];
    for (int i = 0; i < 10; ++i) v[i] = or_uniform(w[i]);
    /* g = alpha0 + alpha / (1 + (A+R+D)^n)  (Eq. 4), x^n = exp(n log x) */
    int64_t x = A + R + D;
    float xn;
    if (x == 0) xn = n > 0.0f ? 0.0f : 1.0f;
    else xn = or_expf(n * or_logf((float)x));
    float g = alpha0 + alpha / (1.0f + xn);
    int64_t k1, k2, k3, k4, k5;
    if (m->sampler == 0) {
      /* hazard g S I / P (Eq. 5) as the per-susceptible daily probability */
      float t = g * (float)I;
      t = t / Pf;
      float pSI = -or_expm1f(-t);
      k1 = or_binomial((int32_t)S, pSI, v[0], v[1]);
      int64_t LI = or_binomial((int32_t)I, pI, v[2], v[3]);
      k2 = or_binomial((int32_t)LI, fI, v[4], v[5]);
      k5 = LI - k2;
      int64_t LA = or_binomial((int32_t)A, pA, v[6], v[7]);
      k3 = or_binomial((int32_t)LA, fA, v[8], v[9]);
      k4 = LA - k3;
    } else {
      /* the paper's floor(Normal(h, sqrt h)) in h order (Sec. 2.2) */
      float h1 = (g * (float)S) * ((float)I / Pf);
      float h2 = gamma * (float)I;
      float h3 = beta * (float)A;
      float h4 = delta * (float)A;
      float h5 = (beta * eta) * (float)I;
      k1 = paper_flow(h1, (int32_t)S, v[0], v[1]);
      k2 = paper_flow(h2, (int32_t)I, v[2], v[3]);
      k3 = paper_flow(h3, (int32_t)A, v[4], v[5]);
      k4 = paper_flow(h4, (int32_t)(A - k3), v[6], v[7]);
      k5 = paper_flow(h5, (int32_t)(I - k2), v[8], v[9]);
    }
    S -= k1;
    I += k1 - k2 - k5;
    A += k2 - k3 - k4;
    R += k3;
    D += k4;
    Ru += k5;
    if (traj) {
      int32_t* tt = traj + (int64_t)(day + 1) * 6 * stride + col;
      tt[0 * stride] = (int32_t)S; tt[1 * stride] = (int32_t)I; tt[2 * stride] = (int32_t)A;
      tt[3 * stride] = (int32_t)R; tt[4 * stride] = (int32_t)D; tt[5 * stride] = (int32_t)Ru;
    }
    if (out_ard) {
      out_ard[0 * (m->T + 1) + day + 1] = (int32_t)A;
      out_ard[1 * (m->T + 1) + day + 1] = (int32_t)R;
      out_ard[2 * (m->T + 1) + day + 1] = (int32_t)D;
    }
    if (m->obs) {
      const int32_t* o = m->obs;
      int64_t dA = A - o[0 * (m->T + 1) + day + 1];
      int64_t dR = R - o[1 * (m->T + 1) + day + 1];
      int64_t dD = D - o[2 * (m->T + 1) + day + 1];
      acc += (unsigned __int128)(uint64_t)(dA * dA);
      acc += (unsigned __int128)(uint64_t)(dR * dR);
      acc += (unsigned __int128)(uint64_t)(dD * dD);
    }
  }
  return sqrt(u128_to_double(acc));
}

/* Gaussian toy: x = theta + z, z ~ N(0, I8); distance ||x - x_obs|| (test model). */
static double simulate_toy(const or_model* m, const float th[8], uint32_t c0, uint32_t c1,
                           uint32_t tag) {
  double acc = 0.0;
  for (int b = 0; b < 4; ++b) {
    uint32_t w[4];
    philox_ctr(m->key, c0, c1, (uint32_t)b, tag, w);
    for (int h = 0; h < 2; ++h) {
      int d = 2 * b + h;
      float z = or_normal(or_uniform(w[2 * h]), or_uniform(w[2 * h + 1]));
      float x = th[d] + z;
      double e = (double)x - (double)m->x_obs[d];
      acc = acc + e * e;
    }
  }
  return sqrt(acc);
}

/*
 * Simulate n particles given in unit coordinates u ([8][n] SoA).  c0 of
 * particle i is c0_idx[i] (or i when c0_idx is NULL); skip[i] != 0 gives +inf.
 */
OR_API void or_simulate(const or_model* m, const float* u, int64_t n, const uint32_t* c0_idx,
                        uint32_t c1, uint32_t tag, const uint8_t* skip, double* dist,
                        int32_t* traj, int nthreads) {
  (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (int64_t i = 0; i < n; ++i) {
    if (skip && skip[i]) { dist[i] = INFINITY; continue; }
    float ui[8], th[8];
    for (int d = 0; d < 8; ++d) ui[d] = u[(int64_t)d * n + i];
    theta_from_u(m, ui, th);
    uint32_t c0 = c0_idx ? c0_idx[i] : (uint32_t)i;
    if (m->model == 1) dist[i] = simulate_toy(m, th, c0, c1, tag);
    else dist[i] = simulate_saird(m, th, c0, c1, tag, traj, n, i, NULL);
  }
}

/*
 * Synthetic observations (stand-in for the JHU series, Sec. 2.2): theta* from
 * the growing-epidemic sub-box [lo, hi] with the OBS_THETA stream, simulated
 * with the OBS stream; redrawn (attempt = c1) until A_T > A0, at most 64 times.
 */
OR_API int32_t or_synth_obs(or_model* m, const float lo[8], const float hi[8], int32_t* obs,
                            float* theta_star) {
  const int32_t* keep = m->obs;
  m->obs = NULL;
  int32_t attempt = 0;
  for (attempt = 0; attempt < 64; ++attempt) {
    uint32_t w[8];
    philox_ctr(m->key, 0u, (uint32_t)attempt, 0u, TAG_OBS_THETA, w);
    philox_ctr(m->key, 0u, (uint32_t)attempt, 1u, TAG_OBS_THETA, w + 4);
    float th[8];
    for (int d = 0; d < 8; ++d) {
      float v = or_uniform(w[d]);
      float span = hi[d] - lo[d];
      th[d] = lo[d] + v * span;
    }
    obs[0 * (m->T + 1)] = m->A0;
    obs[1 * (m->T + 1)] = m->R0;
    obs[2 * (m->T + 1)] = m->D0;
    simulate_saird(m, th, 0u, (uint32_t)attempt, TAG_OBS, NULL, 0, 0, obs);
    memcpy(theta_star, th, sizeof th);
    if (obs[0 * (m->T + 1) + m->T] > m->A0) break;
  }
  m->obs = keep;
  return attempt < 64 ? attempt + 1 : -64;
}

/* ------------------------------------------------------------------------ */
/* ABC-SMC steps (Sec. 2.3-2.4, 3.2)                                          */
/* ------------------------------------------------------------------------ */

/* Stage 0 (Sec. 2.4): u ~ U(0,1)^8 with the PRIOR stream, blocks 0 and 1. */
OR_API void or_prior(const or_model* m, int64_t n, float* u) {
  for (int64_t j = 0; j < n; ++j) {
    uint32_t w[8];
    philox_ctr(m->key, (uint32_t)j, 0u, 0u, TAG_PRIOR, w);
    philox_ctr(m->key, (uint32_t)j, 0u, 1u, TAG_PRIOR, w + 4);
    for (int d = 0; d < 8; ++d) u[(int64_t)d * n + j] = or_uniform(w[d]);
  }
}

static int cmp_double(const void* a, const void* b) {
  double x = *(const double*)a, y = *(const double*)b;
  return (x > y) - (x < y);
}

/* Percentile (Eq. 8): the k-th smallest distance (1-based, lower order statistic). */
OR_API double or_kth(const double* d, int64_t n, int64_t k) {
  double* c = (double*)malloc(sizeof(double) * (size_t)n);
  memcpy(c, d, sizeof(double) * (size_t)n);
  qsort(c, (size_t)n, sizeof(double), cmp_double);
  double v = c[k - 1];
  free(c);
  return v;
}

/* k = ceil(alpha N), clamped to [1, N] */
OR_API int64_t or_rank(double alpha, int64_t n) {
  int64_t k = (int64_t)ceil(alpha * (double)n);
  if (k < 1) k = 1;
  if (k > n) k = n;
  return k;
}

/*
 * Stage prior and its weights (Eq. 9-10): survivors are d_j <= eps.
 * mode 0 (paper): r_j = eps - d_j; mode 1 (importance): r_j = W_j.
 * q_j = floor(r_j * s) with s = (2^32 - 1) / max r (the largest weight gets
 * 2^32 - 1 exactly, no value exceeds it); prefix = inclusive sum of q (u64).
 * When max r is zero or not finite every survivor gets q_j = 1.  Returns
 * the total.
 */
OR_API uint64_t or_resample_prefix(const double* d, const double* W, int64_t n, double eps,
                                   int mode, uint32_t* q, uint64_t* prefix) {
  double rmax = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    double r = 0.0;
    if (d[j] <= eps) r = mode == 0 ? eps - d[j] : W[j];
    if (r > rmax) rmax = r;
  }
  uint64_t tot = 0;
  /* scale = (2^32 - 1) / max r once; the largest weight maps to 2^32 - 1
   * exactly, every other to floor(r * scale) (at most 2^32 - 1) */
  const double scale = 4294967295.0 / rmax;
  for (int64_t j = 0; j < n; ++j) {
    uint32_t qj;
    if (rmax > 0.0 && isfinite(rmax)) {
      double r = 0.0;
      if (d[j] <= eps) r = mode == 0 ? eps - d[j] : W[j];
      const double v = r == rmax ? 4294967295.0 : floor(r * scale);
      qj = (uint32_t)(v < 4294967295.0 ? v : 4294967295.0);
    } else {
      qj = d[j] <= eps ? 1u : 0u;
    }
    q[j] = qj;
    tot += qj;
    prefix[j] = tot;
  }
  return tot;
}

/* Categorical draw (Eq. 11): first k with prefix[k] > x, x = floor(U total / 2^64). */
static int64_t draw_ancestor(const uint64_t* prefix, int64_t n, uint64_t total, uint32_t w0,
                             uint32_t w1) {
  uint64_t U = ((uint64_t)w1 << 32) | (uint64_t)w0;
  uint64_t x = (uint64_t)(((unsigned __int128)U * (unsigned __int128)total) >> 64);
  /* binary search for the first k with prefix[k] > x */
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (prefix[mid] > x) hi = mid; else lo = mid + 1;
  }
  return lo;
}

/* s ~ Beta(a, b), integer b: exp(sum_{m<b} log(U_m) / (a + m)) (BETA stream). */
OR_API float or_beta(const uint32_t key[2], float a, int32_t b, uint32_t c0, uint32_t c1,
                     uint32_t attempt) {
  float acc = 0.0f;
  uint32_t w[4] = {0, 0, 0, 0};
  for (int32_t mm = 0; mm < b; ++mm) {
    if ((mm & 3) == 0)
      philox_ctr(key, c0, c1, (attempt << 8) | (uint32_t)(mm >> 2), TAG_BETA, w);
    float U = or_uniform(w[mm & 3]);
    acc = acc + or_logf(U) / (a + (float)mm);
  }
  return or_expf(acc);
}

/*
 * log of a Gamma(alpha, 1) variate, alpha > 0, by Marsaglia and Tsang's
 * squeeze-and-reject method ("A simple method for generating gamma
 * variables", ACM TOMS 26(3), 2000): with d = alpha - 1/3 and c = 1/sqrt(9d),
 * x ~ N(0,1) and v = (1 + c x)^3, the candidate d v is kept when v > 0 and
 * U < 1 - 0.0331 x^4 (squeeze) or log U < x^2/2 + d (1 - v + log v).  For
 * alpha < 1 the variate is Gamma(alpha + 1) U'^(1/alpha), taken in logs.
 * Iteration i (i < 64) reads Philox block (c0, c1, attempt << 8 | (blk0 + i),
 * BETA): words 0 and 1 give x (Box-Muller), word 2 gives U, word 3 of the
 * accepting block gives U'.  The acceptance test never reads word 3, so U' is
 * uniform and independent of the accepted candidate.  If all 64 iterations
 * reject (probability below 0.05^64) the candidate is d (v = 1).
 */
OR_API float or_gamma_log(const uint32_t key[2], float alpha, uint32_t c0, uint32_t c1,
                          uint32_t attempt, uint32_t blk0) {
  const float al = alpha < 1.0f ? alpha + 1.0f : alpha;
  const float d = al - 0x1.555556p-2f;            /* fp32 nearest to 1/3 */
  const float c = 1.0f / sqrtf(9.0f * d);
  uint32_t w[4] = {0, 0, 0, 0};
  float lg = or_logf(d);
  for (uint32_t i = 0; i < 64u; ++i) {
    philox_ctr(key, c0, c1, (attempt << 8) | (blk0 + i), TAG_BETA, w);
    const float x = or_normal(or_uniform(w[0]), or_uniform(w[1]));
    float v = 1.0f + c * x;
    if (!(v > 0.0f)) continue;
    v = (v * v) * v;
    const float U = or_uniform(w[2]);
    const float x2 = x * x;
    int keep = U < 1.0f - 0.0331f * (x2 * x2);
    if (!keep) keep = or_logf(U) < 0.5f * x2 + d * ((1.0f - v) + or_logf(v));
    if (keep) {
      lg = or_logf(d * v);
      break;
    }
  }
  if (alpha < 1.0f) lg = lg + or_logf(or_uniform(w[3])) / alpha;
  return lg;
}

/* s ~ Beta(a, b) for real a, b > 0: X / (X + Y) with X ~ Gamma(a) (blocks
 * 0..63) and Y ~ Gamma(b) (blocks 64..127), as 1 / (1 + exp(log Y - log X)). */
OR_API float or_beta_real(const uint32_t key[2], float a, float b, uint32_t c0, uint32_t c1,
                          uint32_t attempt) {
  const float lx = or_gamma_log(key, a, c0, c1, attempt, 0u);
  const float ly = or_gamma_log(key, b, c0, c1, attempt, 64u);
  return 1.0f / (1.0f + or_expf(ly - lx));
}

/*
 * Step-size Beta shapes of stage t >= 1 (Eq. 16 and the two alternatives that
 * Sec. 3.2 names).  ratio = eps_t / eps_1 rounded to fp32 (1 when eps_1 = 0).
 *   mode 0 (paper):  a = ratio, integer b = 2t while 2t <= 1024 (the
 *       product form reads one uniform per unit of b and its counter
 *       space holds 1024); from stage 513 on the same Beta(ratio, 2t) is
 *       drawn by the Gamma ratio, a and b clamped to [2^-20, 2^20];
 *   mode 1 (fixed):  a = fa, integer b = fb;
 *   mode 2 (real):   a = p1, b = p2;
 *   mode 3 (mean-variance): mean mu = p1 ratio, variance v = p2 / t;
 *       nu = mu (1 - mu) / v - 1 (= a + b), at least 1/16; a = mu nu,
 *       b = (1 - mu) nu;
 *   mode 4 (mode-concentration): mode w = p1 ratio, concentration
 *       k = p2 t; a = w (k - 2) + 1, b = (1 - w) (k - 2) + 1.
 * Modes 3 and 4 clamp a and b to [2^-20, 2^20].  out[0] = a, out[1] = b;
 * *bint = the integer b of modes 0 and 1 (product sampler), 0 for the
 * real-shape modes (Gamma-ratio sampler).
 */
OR_API void or_beta_shape(int32_t mode, float ratio, int32_t t, float fa, int32_t fb, float p1,
                          float p2, float out[2], int32_t* bint) {
  float a = 1.0f, b = 1.0f;
  int32_t bi = 0;
  if (mode == 0) {
    a = ratio;
    bi = 2 * t;
    b = (float)bi;
    if (bi > 1024) {
      bi = 0;
      if (!(a >= 0x1p-20f)) a = 0x1p-20f;
      if (a > 0x1p20f) a = 0x1p20f;
    }
  } else if (mode == 1) {
    a = fa;
    bi = fb;
    b = (float)bi;
  } else if (mode == 2) {
    a = p1;
    b = p2;
  } else {
    if (mode == 3) {
      const float mu = p1 * ratio;
      const float v = p2 / (float)t;
      float nu = (mu * (1.0f - mu)) / v - 1.0f;
      if (!(nu >= 0.0625f)) nu = 0.0625f;
      a = mu * nu;
      b = (1.0f - mu) * nu;
    } else {
      const float w = p1 * ratio;
      const float k2 = p2 * (float)t - 2.0f;
      a = w * k2 + 1.0f;
      b = (1.0f - w) * k2 + 1.0f;
    }
    if (!(a >= 0x1p-20f)) a = 0x1p-20f;
    if (!(b >= 0x1p-20f)) b = 0x1p-20f;
    if (a > 0x1p20f) a = 0x1p20f;
    if (b > 0x1p20f) b = 0x1p20f;
  }
  out[0] = a;
  out[1] = b;
  *bint = bi;
}

/*
 * BDSS perturbation (Eq. 16-17) with the categorical ancestor draw (Eq. 11)
 * and a prior-support check: for slot j of batch c1 = (t << 16) | batch,
 * attempt a = 0..max_redraw-1 draws (ancestor, s, z) afresh until
 * u' = u_anc + sqrt(s) z lies in [0,1]^8.  On exhaustion flag = 1.
 * s ~ Beta(beta_a, beta_b) by the product form when beta_b >= 1, else
 * Beta(beta_a, beta_bf) by the Gamma ratio.
 *
 * s_fixed > 0 selects the single tuned step of the MCMC baseline (Sec.
 * 2.4.1, Eq. 12): every attempt walks with variance s = s_fixed and no BETA
 * block is read.  With a uniform prior and a symmetric Gaussian walk the
 * Metropolis-Hastings ratio of Eq. 13 is 1 inside the support and 0 outside,
 * so its accept/reject step is this same support check: a proposal outside
 * [0,1]^8 is rejected and drawn again.
 */
OR_API void or_propose(const or_model* m, const float* u, int64_t n, const uint64_t* prefix,
                       uint64_t total, float beta_a, int32_t beta_b, float beta_bf, float s_fixed,
                       int64_t slots, const uint32_t* c0_idx, uint32_t c1, int32_t max_redraw,
                       float* u_out, float* s_out, int32_t* anc_out, int32_t* attempts_out,
                       uint8_t* flag_out, int nthreads) {
  (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (int64_t i = 0; i < slots; ++i) {
    uint32_t j = c0_idx ? c0_idx[i] : (uint32_t)i;
    float up[8] = {0};
    float s = 0.0f;
    int64_t anc = 0;
    int ok = 0;
    int32_t a;
    for (a = 0; a < max_redraw; ++a) {
      uint32_t w[4];
      philox_ctr(m->key, j, c1, (uint32_t)a, TAG_ANCESTOR, w);
      anc = draw_ancestor(prefix, n, total, w[0], w[1]);
      if (s_fixed > 0.0f)
        s = s_fixed;
      else
        s = beta_b > 0 ? or_beta(m->key, beta_a, beta_b, j, c1, (uint32_t)a)
                       : or_beta_real(m->key, beta_a, beta_bf, j, c1, (uint32_t)a);
      float sd = sqrtf(s);
      ok = 1;
      for (int blk = 0; blk < 4; ++blk) {
        uint32_t z4[4];
        philox_ctr(m->key, j, c1, ((uint32_t)a << 8) | (uint32_t)blk, TAG_WALK, z4);
        for (int h = 0; h < 2; ++h) {
          int d = 2 * blk + h;
          float z = or_normal(or_uniform(z4[2 * h]), or_uniform(z4[2 * h + 1]));
          float step = sd * z;
          up[d] = u[(int64_t)d * n + anc] + step;
          if (!(up[d] >= 0.0f && up[d] <= 1.0f)) ok = 0;
        }
      }
      if (ok) break;
    }
    for (int d = 0; d < 8; ++d) u_out[(int64_t)d * slots + i] = up[d];
    s_out[i] = s;
    anc_out[i] = (int32_t)anc;
    attempts_out[i] = ok ? a + 1 : max_redraw;
    flag_out[i] = ok ? 0 : 1;
  }
}

/*
 * Importance weight (auxiliary-variable form, an extension beyond the paper; not in
 * the paper): log W_j = log pi(u'_j) - log sum_k rhat_k N(u'_j; u_k, s_j I8),
 * rhat_k = q_k / total, pi uniform on the unit cube.  fp64 throughout.
 * The kernel variance is floored at 1e-30f: a row with a smaller step has
 * relative weight below (1e-30)^4 against any row with s >= 1e-6, and the
 * floor keeps 1/(2s) finite in fp32 on the device.
 */
OR_API void or_weights(const float* up, const float* s, int64_t rows, const float* u,
                       const uint32_t* q, int64_t n, uint64_t total, double* logW,
                       int nthreads) {
  (void)nthreads;
  double ltot = log((double)total);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : 1)
#endif
  for (int64_t j = 0; j < rows; ++j) {
    double sj = (double)fmaxf(s[j], 1e-30f);
    double* e = (double*)malloc(sizeof(double) * (size_t)n);
    double mx = -INFINITY;
    for (int64_t k = 0; k < n; ++k) {
      if (q[k] == 0) { e[k] = -INFINITY; continue; }
      double D = 0.0;
      for (int d = 0; d < 8; ++d) {
        double diff = (double)up[(int64_t)d * rows + j] - (double)u[(int64_t)d * n + k];
        D += diff * diff;
      }
      e[k] = (log((double)q[k]) - ltot) - D / (2.0 * sj);
      if (e[k] > mx) mx = e[k];
    }
    double sum = 0.0;
    for (int64_t k = 0; k < n; ++k)
      if (e[k] > -INFINITY) sum += exp(e[k] - mx);
    double lse = mx + log(sum);
    logW[j] = 4.0 * log(2.0 * M_PI * sj) - lse;
    free(e);
  }
}

/* W_j = exp(logW_j - max) / sum; ESS = 1 / sum W_j^2 (fp64).  A NaN log
 * weight (no valid input produces one) counts as weight 0. */
OR_API double or_normalize(const double* logW, int64_t n, double* W) {
  double mx = -INFINITY;
  for (int64_t j = 0; j < n; ++j) if (logW[j] > mx) mx = logW[j];
  if (!(mx > -INFINITY) || mx != mx) {
    for (int64_t j = 0; j < n; ++j) W[j] = 1.0 / (double)n;
    return (double)n;
  }
  double sum = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    W[j] = logW[j] == logW[j] ? exp(logW[j] - mx) : 0.0;
    sum += W[j];
  }
  double s2 = 0.0;
  for (int64_t j = 0; j < n; ++j) { W[j] = W[j] / sum; s2 += W[j] * W[j]; }
  return 1.0 / s2;
}

/* ------------------------------------------------------------------------ */
/* One SMC generation (Sec. 2.4 and 3.2).                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t N;            /* population (samples kept per stage)             */
  int32_t M;            /* proposals per batch ("parallel simulations")    */
  int32_t max_total;    /* run budget in batches (Sec. 4.1), 0: none; the   */
                        /* driver (oracle run()) applies it                 */
  double alpha;         /* survival ratio (Eq. 8), 0.5 in the paper         */
  int32_t beta_mode;    /* 0: Beta(eps_t/eps_1, 2t) (Eq. 16); 1: fixed;     */
  float beta_a;         /* 2: real shapes; 3: mean-variance; 4: mode-       */
  int32_t beta_b;       /* concentration (or_beta_shape)                    */
  float beta_p1, beta_p2;
  int32_t weight_mode;  /* 0: eps - d (Eq. 10); 1: importance weights       */
  int32_t max_batches;
  int32_t max_redraw;
  int32_t nthreads;
  float mcmc_s0;        /* beta_mode 5 (MCMC baseline): initial step s      */
  int32_t mcmc_adapt;   /* adaptation window in batches that walk with the  */
                        /* step; 0: ceil(max_total / 10) (or_mcmc_window)   */
} or_smc;

/* State of the MCMC baseline's tuned step, carried across generations. */
typedef struct {
  double s;             /* current step (variance, unit-cube coordinates)   */
  int64_t k;            /* adaptations made so far                          */
  int64_t batches;      /* batches walked with the step so far (those of    */
                        /* generations t >= 1)                              */
} or_mcmc_state;

typedef struct {
  double eps;           /* eps_t used by this generation                    */
  double eps1;          /* eps_1                                            */
  double ess;
  float beta_a;
  int32_t beta_b;       /* integer b (product sampler), 0 for real shapes   */
  float beta_bf;        /* b as fp32                                        */
  float mcmc_s;         /* MCMC baseline: step s after the generation       */
  int64_t batches, sims, exhausted, accepted_total;
  uint64_t total;       /* resampling total                                  */
  int32_t status;       /* 0 ok, 1 batch budget exhausted                   */
} or_gen_stats;

/*
 * Step adaptation of the MCMC baseline (Sec. 2.4.1, Eq. 14-15; Sec. 3.1
 * adapts once per batch of parallel simulations).  A = acc / sims is the
 * batch's empirical acceptance (Eq. 14): of the sims proposals that passed
 * the Metropolis-Hastings check and were simulated, acc reached d <= eps_t
 * (A = 0 when nothing was simulated).  Eq. 15 as printed would turn s
 * negative whenever A < A_T; it is read as the multiplicative Robbins-Monro
 * step s_new = s_old (1 + (A - A_T) / ((1 - A_T) (k + 1))) with target
 * A_T = 0.234 and gain 1 / (k + 1), k the adaptations made so far.  The
 * factor lies in [1 - A_T / ((1 - A_T) (k + 1)), 1 + 1 / (k + 1)], about
 * [0.69, 2] at k = 0, so s stays positive; it grows when more than A_T of
 * the batch is accepted.  Plain fp64 operations, each correctly rounded.
 */
OR_API double or_mcmc_adapt(double s, int64_t k, int64_t acc, int64_t sims) {
  const double A_T = 0.234;
  const double A = sims > 0 ? (double)acc / (double)sims : 0.0;
  const double gain = (1.0 - A_T) * (double)(k + 1);
  return s * (1.0 + (A - A_T) / gain);
}

/* Adaptation window in batches: mcmc_adapt, or when it is 0 a tenth of the
 * run budget (Sec. 2.4.1 and 3.1 adapt during the first 10% of the
 * simulation runs), 0 without a budget (the step stays at mcmc_s0).  The
 * window counts the batches that walk with the step, from generation 1 on:
 * generation 0 draws from the prior and has no step to tune, and counting
 * its ceil(N / M) batches would close the window before any step was taken
 * whenever N / M reaches a tenth of the budget (N = 1000 at M = 10). */
OR_API int64_t or_mcmc_window(const or_smc* c) {
  if (c->mcmc_adapt > 0) return c->mcmc_adapt;
  return ((int64_t)c->max_total + 9) / 10;
}

/* Generation 0 (Sec. 2.4): plain ABC from the prior with eps_0 = +inf. */
OR_API void or_generation0(const or_model* m, const or_smc* c, float* u, double* d, double* W) {
  or_prior(m, c->N, u);
  or_simulate(m, u, c->N, NULL, 0u, TAG_SIM, NULL, d, NULL, c->nthreads);
  for (int64_t j = 0; j < c->N; ++j) W[j] = 1.0 / (double)c->N;
}

/*
 * Generation t >= 1: eps_t from the previous population (Eq. 8), the stage
 * prior and weights (Eq. 9-10), then batches of M proposals (Eq. 11, 16, 17),
 * simulation and acceptance d' <= eps_t, appended in (batch, slot) order
 * until N are filled; then the new weights.
 *
 * beta_mode 5 is the MCMC baseline (Sec. 2.4.1, 3.1): each batch walks with
 * the run's single step s = (float) ms->s (Eq. 12), and after the batch, if
 * fewer than or_mcmc_window batches walked with the step before it, s
 * adapts to the batch's acceptance (or_mcmc_adapt).  ms (required in that
 * mode, NULL otherwise) carries s, the adaptation count and the batch count
 * across generations.
 */
OR_API int32_t or_generation(const or_model* m, const or_smc* c, int32_t t, double eps1_in,
                             const float* u, const double* d, const double* W, float* u_new,
                             double* d_new, double* W_new, float* s_new, int32_t* anc_new,
                             double* logW_new, or_gen_stats* st, or_mcmc_state* ms) {
  int64_t N = c->N, M = c->M;
  memset(st, 0, sizeof *st);
  double eps = or_kth(d, N, or_rank(c->alpha, N));
  double eps1 = t == 1 ? eps : eps1_in;
  st->eps = eps;
  st->eps1 = eps1;
  float shape[2];
  int32_t bb;
  const float ratio = eps1 > 0.0 ? (float)(eps / eps1) : 1.0f;
  or_beta_shape(c->beta_mode, ratio, t, c->beta_a, c->beta_b, c->beta_p1, c->beta_p2, shape, &bb);
  const float ba = shape[0];
  st->beta_a = ba;
  st->beta_b = bb;
  st->beta_bf = shape[1];
  const int mcmc = c->beta_mode == 5;
  if (mcmc) {
    if (!ms) return -1;
    st->beta_a = (float)ms->s;
    st->beta_b = 0;
    st->beta_bf = 0.0f;
  }
  const int64_t window = or_mcmc_window(c);
  uint32_t* q = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)N);
  uint64_t* prefix = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)N);
  uint64_t total = or_resample_prefix(d, W, N, eps, c->weight_mode, q, prefix);
  st->total = total;
  float* up = (float*)malloc(sizeof(float) * 8 * (size_t)M);
  float* sp = (float*)malloc(sizeof(float) * (size_t)M);
  int32_t* ap = (int32_t*)malloc(sizeof(int32_t) * (size_t)M);
  int32_t* att = (int32_t*)malloc(sizeof(int32_t) * (size_t)M);
  uint8_t* fl = (uint8_t*)malloc((size_t)M);
  double* dp = (double*)malloc(sizeof(double) * (size_t)M);
  int64_t filled = 0;
  int32_t b;
  for (b = 0; b < c->max_batches && filled < N; ++b) {
    uint32_t c1 = ((uint32_t)t << 16) | (uint32_t)b;
    const float s_fixed = mcmc ? (float)ms->s : 0.0f;
    or_propose(m, u, N, prefix, total, ba, bb, shape[1], s_fixed, M, NULL, c1, c->max_redraw, up,
               sp, ap, att, fl, c->nthreads);
    or_simulate(m, up, M, NULL, c1, TAG_SIM, fl, dp, NULL, c->nthreads);
    st->sims += M;
    int64_t acc_b = 0, exh_b = 0;
    for (int64_t j = 0; j < M; ++j) {
      if (fl[j]) exh_b += 1;
      int acc = !fl[j] && dp[j] <= eps;
      if (!acc) continue;
      acc_b += 1;
      st->accepted_total += 1;
      if (filled < N) {
        for (int dd = 0; dd < 8; ++dd) u_new[(int64_t)dd * N + filled] = up[(int64_t)dd * M + j];
        d_new[filled] = dp[j];
        s_new[filled] = sp[j];
        anc_new[filled] = ap[j];
        filled += 1;
      }
    }
    st->exhausted += exh_b;
    if (mcmc) {
      if (ms->batches < window) {
        ms->s = or_mcmc_adapt(ms->s, ms->k, acc_b, M - exh_b);
        ms->k += 1;
      }
      ms->batches += 1;
    }
  }
  st->batches = b;
  if (mcmc) st->mcmc_s = (float)ms->s;
  if (filled < N) {
    st->status = 1;
  } else if (c->weight_mode == 1) {
    or_weights(u_new, s_new, N, u, q, N, total, logW_new, c->nthreads);
    st->ess = or_normalize(logW_new, N, W_new);
  } else {
    for (int64_t j = 0; j < N; ++j) { W_new[j] = 1.0 / (double)N; logW_new[j] = 0.0; }
    st->ess = (double)N;
  }
  free(q); free(prefix); free(up); free(sp); free(ap); free(att); free(fl); free(dp);
  return st->status;
}

/* ------------------------------------------------------------------------ */
/* Posterior-predictive simulation (Sec. 4.2).                                */
/* ------------------------------------------------------------------------ */
static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/*
 * Sec. 4.2 predicts case data by simulating the learned parameter samples
 * from day zero over the training window plus the days ahead, and reports
 * per day the median and the central 99% range.  Here: R draws from the
 * population u [8][N] in proportion to its weights W (NULL: equal weights;
 * quantised and drawn like the stage prior, Eq. 10-11, with the PREDICT
 * stream: block (j, 0, 0, PREDICT), U = w1 2^32 + w0), each simulated for
 * `days` days with the PREDICT_SIM stream (c0 = j, c1 = 0); for every day
 * 0..days and series A, R, D the order statistic of rank k = ceil(q R),
 * clamped to [1, R] (the lower order statistic, as Eq. 8), for each level
 * q of quant[nq].  out: [days + 1][3][nq].
 */
OR_API int or_predict(const or_model* m0, const float* u, const double* W, int64_t N, int64_t R,
                      int32_t days, const double* quant, int32_t nq, int32_t* out) {
  if (N < 1 || R < 1 || days < 0 || nq < 1) return -1;
  or_model m = *m0;
  m.T = days;
  m.obs = NULL;
  double* d0 = (double*)calloc((size_t)N, sizeof(double));
  uint32_t* q = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)N);
  uint64_t* prefix = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)N);
  float* ur = (float*)malloc(sizeof(float) * 8 * (size_t)R);
  int32_t* traj = (int32_t*)malloc(sizeof(int32_t) * (size_t)(days + 1) * 6 * (size_t)R);
  int32_t* col = (int32_t*)malloc(sizeof(int32_t) * (size_t)R);
  /* weights W (importance form: every particle survives eps = 0 with d = 0),
   * or all equal (paper form with eps = d: every stage weight 0, q = 1) */
  uint64_t total = or_resample_prefix(d0, W, N, 0.0, W ? 1 : 0, q, prefix);
  for (int64_t j = 0; j < R; ++j) {
    uint32_t w[4];
    philox_ctr(m.key, (uint32_t)j, 0u, 0u, TAG_PREDICT, w);
    int64_t a = draw_ancestor(prefix, N, total, w[0], w[1]);
    for (int d = 0; d < 8; ++d) ur[(int64_t)d * R + j] = u[(int64_t)d * N + a];
  }
  for (int64_t j = 0; j < R; ++j) {
    float ui[8], th[8];
    for (int d = 0; d < 8; ++d) ui[d] = ur[(int64_t)d * R + j];
    theta_from_u(&m, ui, th);
    simulate_saird(&m, th, (uint32_t)j, 0u, TAG_PREDICT_SIM, traj, R, j, NULL);
  }
  static const int series[3] = {2, 3, 4}; /* A, R, D */
  for (int32_t t = 0; t <= days; ++t)
    for (int c = 0; c < 3; ++c) {
      memcpy(col, traj + ((int64_t)t * 6 + series[c]) * R, sizeof(int32_t) * (size_t)R);
      qsort(col, (size_t)R, sizeof(int32_t), cmp_i32);
      for (int32_t i = 0; i < nq; ++i) {
        int64_t k = (int64_t)ceil(quant[i] * (double)R);
        if (k < 1) k = 1;
        if (k > R) k = R;
        out[((int64_t)t * 3 + c) * nq + i] = col[k - 1];
      }
    }
  free(d0); free(q); free(prefix); free(ur); free(traj); free(col);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Surrogate MLP (an extension beyond the paper; not in the paper): 8 -> 256 -> 256 -> */
/* 4 with tanh-form GELU, fp64 throughout, weights given as fp64 copies of   */
/* the device's bf16 values.  Layout: W1[256][8], W2[256][256], W3[4][256]    */
/* (row = output), biases b1[256], b2[256], b3[4].                            */
/* ------------------------------------------------------------------------ */
#define OR_H 256

static double gelu(double x) {
  const double c = 0.7978845608028654;  /* sqrt(2/pi) */
  double t = tanh(c * (x + 0.044715 * x * x * x));
  return 0.5 * x * (1.0 + t);
}

static double gelu_grad(double x) {
  const double c = 0.7978845608028654;
  double t = tanh(c * (x + 0.044715 * x * x * x));
  return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * c * (1.0 + 3.0 * 0.044715 * x * x);
}

OR_API double or_gelu(double x) { return gelu(x); }

/* y[n][4] = MLP(x[n][8]) */
OR_API void or_mlp_forward(const double* W1, const double* b1, const double* W2, const double* b2,
                           const double* W3, const double* b3, const double* x, int64_t n,
                           double* y) {
  double* h1 = (double*)malloc(sizeof(double) * OR_H);
  double* h2 = (double*)malloc(sizeof(double) * OR_H);
  for (int64_t i = 0; i < n; ++i) {
    for (int o = 0; o < OR_H; ++o) {
      double z = b1[o];
      for (int k = 0; k < 8; ++k) z += W1[o * 8 + k] * x[i * 8 + k];
      h1[o] = gelu(z);
    }
    for (int o = 0; o < OR_H; ++o) {
      double z = b2[o];
      for (int k = 0; k < OR_H; ++k) z += W2[o * OR_H + k] * h1[k];
      h2[o] = gelu(z);
    }
    for (int o = 0; o < 4; ++o) {
      double z = b3[o];
      for (int k = 0; k < OR_H; ++k) z += W3[o * OR_H + k] * h2[k];
      y[i * 4 + o] = z;
    }
  }
  free(h1);
  free(h2);
}

/* loss = mean over n samples and 4 outputs of (y - t)^2; gradients of every
 * parameter (same layouts as the parameters). Returns the loss. */
OR_API double or_mlp_backward(const double* W1, const double* b1, const double* W2,
                              const double* b2, const double* W3, const double* b3,
                              const double* x, const double* t, int64_t n, double* gW1,
                              double* gb1, double* gW2, double* gb2, double* gW3, double* gb3) {
  memset(gW1, 0, sizeof(double) * OR_H * 8);
  memset(gb1, 0, sizeof(double) * OR_H);
  memset(gW2, 0, sizeof(double) * OR_H * OR_H);
  memset(gb2, 0, sizeof(double) * OR_H);
  memset(gW3, 0, sizeof(double) * 4 * OR_H);
  memset(gb3, 0, sizeof(double) * 4);
  double z1[OR_H], h1[OR_H], z2[OR_H], h2[OR_H], d2[OR_H], d1[OR_H];
  double loss = 0.0;
  const double scale = 2.0 / (4.0 * (double)n);
  for (int64_t i = 0; i < n; ++i) {
    for (int o = 0; o < OR_H; ++o) {
      double z = b1[o];
      for (int k = 0; k < 8; ++k) z += W1[o * 8 + k] * x[i * 8 + k];
      z1[o] = z;
      h1[o] = gelu(z);
    }
    for (int o = 0; o < OR_H; ++o) {
      double z = b2[o];
      for (int k = 0; k < OR_H; ++k) z += W2[o * OR_H + k] * h1[k];
      z2[o] = z;
      h2[o] = gelu(z);
    }
    double dy[4];
    for (int o = 0; o < 4; ++o) {
      double z = b3[o];
      for (int k = 0; k < OR_H; ++k) z += W3[o * OR_H + k] * h2[k];
      double e = z - t[i * 4 + o];
      loss += e * e;
      dy[o] = scale * e;
    }
    for (int o = 0; o < 4; ++o) {
      gb3[o] += dy[o];
      for (int k = 0; k < OR_H; ++k) gW3[o * OR_H + k] += dy[o] * h2[k];
    }
    for (int k = 0; k < OR_H; ++k) {
      double g = 0.0;
      for (int o = 0; o < 4; ++o) g += dy[o] * W3[o * OR_H + k];
      d2[k] = g * gelu_grad(z2[k]);
    }
    for (int o = 0; o < OR_H; ++o) {
      gb2[o] += d2[o];
      for (int k = 0; k < OR_H; ++k) gW2[o * OR_H + k] += d2[o] * h1[k];
    }
    for (int k = 0; k < OR_H; ++k) {
      double g = 0.0;
      for (int o = 0; o < OR_H; ++o) g += d2[o] * W2[o * OR_H + k];
      d1[k] = g * gelu_grad(z1[k]);
    }
    for (int o = 0; o < OR_H; ++o) {
      gb1[o] += d1[o];
      for (int k = 0; k < 8; ++k) gW1[o * 8 + k] += d1[o] * x[i * 8 + k];
    }
  }
  return loss / (4.0 * (double)n);
}

/*
 * Delayed-acceptance screen (an extension beyond the paper; not in the paper; the
 * two-stage acceptance of Christen & Fox 2005 with a surrogate first stage).
 * A proposal u' whose surrogate prediction of log1p d is y0 is simulated
 * with probability rho = min(max(sigmoid((log1p eps - y0) / tau), rho_min), 1);
 * an accepted one then has density q(u') rho(u') 1[d <= eps], so its
 * importance weight carries the factor 1/rho.  Screened-out proposals are
 * simulated anyway with probability audit_frac (never accepted) to measure
 * how often the screen rejects a proposal that d <= eps would keep.
 * Y[i][0] is the standardised prediction: y0 = ystat[0] + ystat[4] Y[i][0].
 * fp32 in this order with the oracle's own exp and log1p; the uniforms are
 * the first words of Philox blocks (i, c1, 0, SCREEN) and (i, c1, 0, AUDIT).
 * sflag: 0 simulate, 1 redraw-exhausted (flag != 0; rho 1), 2 audit only,
 * 3 screened out.
 */
OR_API void or_screen(const or_model* m, const float* Y, const float* ystat, const uint8_t* flag,
                      int64_t M, double eps, uint32_t c1, float tau, float rho_min,
                      float audit_frac, float* rho, uint8_t* sflag) {
  const float le = or_log1pf((float)eps);
  for (int64_t i = 0; i < M; ++i) {
    if (flag && flag[i]) {
      sflag[i] = 1;
      rho[i] = 1.0f;
      continue;
    }
    const float y0 = ystat[0] + ystat[4] * Y[i * 4];
    const float z = (le - y0) / tau;
    float r = 1.0f / (1.0f + or_expf(-z));
    r = fminf(fmaxf(r, rho_min), 1.0f);
    rho[i] = r;
    uint32_t w[4];
    philox_ctr(m->key, (uint32_t)i, c1, 0u, TAG_SCREEN, w);
    if (or_uniform(w[0]) < r) {
      sflag[i] = 0;
      continue;
    }
    philox_ctr(m->key, (uint32_t)i, c1, 0u, TAG_AUDIT, w);
    sflag[i] = or_uniform(w[0]) < audit_frac ? 2 : 3;
  }
}

/* Adam (Kingma & Ba 2015) on one parameter array, step count t >= 1. */
OR_API void or_adam(double* w, const double* g, double* m, double* v, int64_t n, double lr,
                    double b1, double b2, double eps, int64_t t) {
  const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    w[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
  }
}
