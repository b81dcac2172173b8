// simulate.cu -- A0 synthetic observations, A1 prior draw, A2-A3 simulator
// with the fused exact-integer distance.
//
// One thread per particle: the six compartment counts live in int32
// registers, the eight parameters in fp32 registers, the observed series in
// shared memory; every day draws three Philox blocks and five binomial
// transitions (Sec. 2.2, Eq. 3-5, as exact-count competing risks) and adds
// the day's squared error to an unsigned 128-bit accumulator (Sec. 2.3).
#include "batch.cuh"
#include "common.cuh"
#include "numerics.cuh"

namespace abc {

struct U128 {
  uint64_t hi, lo;
};

__device__ __forceinline__ void acc_sq(U128& a, int32_t x, int32_t o) {
  const int64_t d = static_cast<int64_t>(x) - static_cast<int64_t>(o);
  const uint64_t sq = static_cast<uint64_t>(d * d);
  const uint64_t lo = a.lo + sq;
  a.hi += lo < sq ? 1ull : 0ull;
  a.lo = lo;
}

// one day's three squared errors at once, for counts and observations in
// [0, 2^31): each difference fits int32, each square is below 2^62 and their
// sum below 2^64, so one 64-bit add with carry takes the day
__device__ __forceinline__ void acc_day(U128& a, int32_t x0, int32_t o0, int32_t x1, int32_t o1,
                                        int32_t x2, int32_t o2) {
  const int32_t d0 = x0 - o0, d1 = x1 - o1, d2 = x2 - o2;
  uint64_t s = static_cast<uint64_t>(static_cast<int64_t>(d0) * d0);
  s += static_cast<uint64_t>(static_cast<int64_t>(d1) * d1);
  s += static_cast<uint64_t>(static_cast<int64_t>(d2) * d2);
  const uint64_t lo = a.lo + s;
  a.hi += lo < s ? 1ull : 0ull;
  a.lo = lo;
}

// theta_d = lo_d + u_d (hi_d - lo_d)  (Sec. 3.1 reparameterisation)
__device__ __forceinline__ float theta_of(const SimParams& p, int d, float u) {
  return __fadd_rn(p.lo[d], __fmul_rn(u, __fsub_rn(p.hi[d], p.lo[d])));
}

// One SAIRD trajectory.  obs (nullable) is [3][T+1] for the distance; traj
// (nullable) is [T+1][6][stride] at column col; ard (nullable) receives the
// simulated A, R, D as [3][T+1] for days 1..T.  mask: the warp's lanes that
// run a trajectory (all of them call this together, for the same T); bq:
// the warp's queue of kBinvQueue inversion jobs in shared memory.
constexpr int kBinvQueue = 96;  // three draws per lane per batch

__device__ U128 saird_path(const SimParams& p, const float th[8], uint32_t c0, uint32_t c1,
                           uint32_t tag, const int32_t* obs, int32_t* traj, int64_t stride,
                           int64_t col, int32_t* ard, unsigned mask, BinvJob* bq,
                           int32_t* last = nullptr, bool obs_nonneg = false) {
  const float alpha0 = th[0], alpha = th[1], n = th[2], beta = th[3], gamma = th[4],
              delta = th[5], eta = th[6], kappa = th[7];
  // initial state (Sec. 2.2): Ru = 0, I0 = kappa A0, S = P - (A0 + R0 + D0 + I0)
  int32_t A = p.A0, R = p.R0, D = p.D0;
  int64_t I64 = static_cast<int64_t>(floorf(__fmul_rn(kappa, __int2float_rn(p.A0))));
  int64_t S64 = p.P - (static_cast<int64_t>(A) + R + D + I64);
  if (S64 < 0) {
    I64 = p.P - (static_cast<int64_t>(A) + R + D);
    if (I64 < 0) I64 = 0;
    S64 = 0;
  }
  int32_t S = static_cast<int32_t>(S64), I = static_cast<int32_t>(I64), Ru = 0;
  const float Pf = __ll2float_rn(p.P);
  // competing risks: I leaves at gamma + beta eta, A at beta + delta (Eq. 5)
  const float lamI = __fadd_rn(gamma, __fmul_rn(beta, eta));
  const float lamA = __fadd_rn(beta, delta);
  const float pI = -dev_expm1(-lamI);
  const float pA = -dev_expm1(-lamA);
  const float fI = lamI > 0.0f ? __fdiv_rn(gamma, lamI) : 0.0f;
  const float fA = lamA > 0.0f ? __fdiv_rn(beta, lamA) : 0.0f;
  // the four exits of I and A have fixed probabilities: their binomial
  // constants are computed once per particle (bit-identical draws)
  const BinomConst cI = binom_const(pI), cfI = binom_const(fI);
  const BinomConst cA = binom_const(pA), cfA = binom_const(fA);
  const int T = p.T;
  if (traj) {
    int32_t* t0 = traj + col;
    t0[0 * stride] = S; t0[1 * stride] = I; t0[2 * stride] = A;
    t0[3 * stride] = R; t0[4 * stride] = D; t0[5 * stride] = Ru;
  }
  U128 acc{0ull, 0ull};
  for (int day = 0; day < T; ++day) {
    const uint32_t cb = static_cast<uint32_t>(day) * 4u;
    const u32x4 b0 = philox4x32_10_rk(c0, c1, cb + 0u, tag, p.rk0, p.rk1);
    const u32x4 b1 = philox4x32_10_rk(c0, c1, cb + 1u, tag, p.rk0, p.rk1);
    const u32x4 b2 = philox4x32_10_rk(c0, c1, cb + 2u, tag, p.rk0, p.rk1);
    // g = alpha0 + alpha / (1 + (A+R+D)^n)  (Eq. 4), x^n = exp(n log x)
    const int32_t x = A + R + D;
    float xn;
    if (x == 0) xn = n > 0.0f ? 0.0f : 1.0f;
    else xn = dev_exp(__fmul_rn(n, dev_log_pos(__int2float_rn(x))));
    const float g = __fadd_rn(alpha0, __fdiv_rn(alpha, __fadd_rn(1.0f, xn)));
    int32_t k1, k2, k3, k4, k5;
    if (p.sampler == ABC_SIM_BINOMIAL) {
      const float t = __fdiv_rn(__fmul_rn(g, __int2float_rn(I)), Pf);
      const float pSI = -dev_expm1(-t);
      // the five binomial draws, in two batches of independent draws (S->I,
      // I exit, A exit; then the two splits); each batch's inversion loops
      // run together, spread over the warp
      BinvJob e{0, 0.0f, 0.0f, 0.0f};
      bool f1, fI, fA;
      int nq = 0;
      k1 = binom_front(S, pSI, unif(b0.x), unif(b0.y), f1, e);
      const int q1 = binv_push(mask, k1 < 0, e, bq, nq);
      int32_t LI = binom_front_c(I, cI, unif(b0.z), unif(b0.w), fI, e);
      const int qI = binv_push(mask, LI < 0, e, bq, nq);
      int32_t LA = binom_front_c(A, cA, unif(b1.z), unif(b1.w), fA, e);
      const int qA = binv_push(mask, LA < 0, e, bq, nq);
      if (nq) {  // warp-uniform
        binv_drain(mask, bq, nq);
        if (k1 < 0) k1 = f1 ? S - bq[q1].n : bq[q1].n;
        if (LI < 0) LI = fI ? I - bq[qI].n : bq[qI].n;
        if (LA < 0) LA = fA ? A - bq[qA].n : bq[qA].n;
        __syncwarp(mask);  // the queue is refilled below
      }
      bool f2, f3;
      nq = 0;
      k2 = binom_front_c(LI, cfI, unif(b1.x), unif(b1.y), f2, e);
      const int q2 = binv_push(mask, k2 < 0, e, bq, nq);
      k3 = binom_front_c(LA, cfA, unif(b2.x), unif(b2.y), f3, e);
      const int q3 = binv_push(mask, k3 < 0, e, bq, nq);
      if (nq) {
        binv_drain(mask, bq, nq);
        if (k2 < 0) k2 = f2 ? LI - bq[q2].n : bq[q2].n;
        if (k3 < 0) k3 = f3 ? LA - bq[q3].n : bq[q3].n;
        __syncwarp(mask);
      }
      k5 = LI - k2;
      k4 = LA - k3;
    } else {
      // the paper's floor(Normal(h, sqrt h)) flows in h order (Sec. 2.2)
      const float h1 = __fmul_rn(__fmul_rn(g, __int2float_rn(S)), __fdiv_rn(__int2float_rn(I), Pf));
      const float h2 = __fmul_rn(gamma, __int2float_rn(I));
      const float h3 = __fmul_rn(beta, __int2float_rn(A));
      const float h4 = __fmul_rn(delta, __int2float_rn(A));
      const float h5 = __fmul_rn(__fmul_rn(beta, eta), __int2float_rn(I));
      k1 = dev_paper_flow(h1, S, unif(b0.x), unif(b0.y));
      k2 = dev_paper_flow(h2, I, unif(b0.z), unif(b0.w));
      k3 = dev_paper_flow(h3, A, unif(b1.x), unif(b1.y));
      k4 = dev_paper_flow(h4, A - k3, unif(b1.z), unif(b1.w));
      k5 = dev_paper_flow(h5, I - k2, unif(b2.x), unif(b2.y));
    }
    S -= k1;
    I += k1 - k2 - k5;
    A += k2 - k3 - k4;
    R += k3;
    D += k4;
    Ru += k5;
    if (traj) {
      int32_t* tt = traj + static_cast<int64_t>(day + 1) * 6 * stride + col;
      tt[0 * stride] = S; tt[1 * stride] = I; tt[2 * stride] = A;
      tt[3 * stride] = R; tt[4 * stride] = D; tt[5 * stride] = Ru;
    }
    if (ard) {
      ard[0 * (T + 1) + day + 1] = A;
      ard[1 * (T + 1) + day + 1] = R;
      ard[2 * (T + 1) + day + 1] = D;
    }
    if (obs) {
      if (obs_nonneg) {
        acc_day(acc, A, obs[0 * (T + 1) + day + 1], R, obs[1 * (T + 1) + day + 1], D,
                obs[2 * (T + 1) + day + 1]);
      } else {
        acc_sq(acc, A, obs[0 * (T + 1) + day + 1]);
        acc_sq(acc, R, obs[1 * (T + 1) + day + 1]);
        acc_sq(acc, D, obs[2 * (T + 1) + day + 1]);
      }
    }
  }
  if (last) {
    last[0] = A;
    last[1] = R;
    last[2] = D;
  }
  return acc;
}

// Gaussian toy: x = theta + z, distance ||x - x_obs|| in fp64
__device__ double toy_dist(const SimParams& p, const float th[8], uint32_t c0, uint32_t c1,
                           uint32_t tag) {
  double acc = 0.0;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const u32x4 w = philox4x32_10(c0, c1, static_cast<uint32_t>(b), tag, p.k0, p.k1);
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int d = 2 * b + h;
      const float z = dev_normal(unif(ws[2 * h]), unif(ws[2 * h + 1]));
      const float xv = __fadd_rn(th[d], z);
      const double e = __dsub_rn(static_cast<double>(xv), static_cast<double>(p.x_obs[d]));
      acc = __dadd_rn(acc, __dmul_rn(e, e));
    }
  }
  return __dsqrt_rn(acc);
}

__global__ void __launch_bounds__(256, 4)
k_simulate(SimParams p, const int32_t* __restrict__ obs,
                           const float* __restrict__ u, int64_t n,
                           const uint32_t* __restrict__ c0_idx, uint32_t c1, uint32_t tag,
                           const uint8_t* __restrict__ skip, double* __restrict__ dist,
                           int32_t* __restrict__ traj, const uint32_t* __restrict__ c1_dev,
                           const int* __restrict__ off_dev, int32_t* __restrict__ ard_last,
                           int64_t m_sub, const int* __restrict__ n_dev,
                           const int32_t* __restrict__ perm) {
  extern __shared__ int32_t s_obs[];
  if (off_dev && *off_dev) return;  // run finished: nothing to simulate
  if (c1_dev) c1 = *c1_dev;         // counter word set on the device (graph launches)
  const int nobs = (p.model == ABC_MODEL_SAIRD && obs) ? 3 * (p.T + 1) : 0;
  int obs_ok = 1;
  for (int i = threadIdx.x; i < nobs; i += blockDim.x) {
    s_obs[i] = obs[i];
    obs_ok &= s_obs[i] >= 0;
  }
  // the warps' inversion queues follow the observations (16-byte aligned)
  BinvJob* bq = reinterpret_cast<BinvJob*>(s_obs + ((nobs + 3) & ~3)) +
                (threadIdx.x >> 5) * kBinvQueue;
  // every observation non-negative (block-uniform): the days' squared errors
  // go in with one carry each
  const bool obs_nonneg = __syncthreads_and(obs_ok) != 0;
  // perm (nullable): thread t runs slot perm[t] (an order that groups similar
  // trajectories into warps); every slot keeps its own counters and outputs
  // (with n_dev, over the slots in use only; the others keep their place)
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  int64_t i = t;
  if (perm && t < n && t < (n_dev ? static_cast<int64_t>(*n_dev) : n)) i = perm[t];
  // n_dev (nullable): the slots in use, counted on the device (a compacted
  // list of capacity n); the others get distance +inf
  const bool live = i < n && !(n_dev && i >= *n_dev) && !(skip && skip[i]);
  // lanes that simulate (the block size is a multiple of 32)
  const unsigned mask = __ballot_sync(0xffffffffu, live);
  if (i >= n) return;
  if (!live) {
    dist[i] = __longlong_as_double(0x7ff0000000000000ll);
    return;
  }
  float th[8];
#pragma unroll
  for (int d = 0; d < 8; ++d) th[d] = theta_of(p, d, u[static_cast<int64_t>(d) * n + i]);
  // slots of several batches at once (m_sub > 0): slot is of batch c1 + kb
  int64_t is = i;
  if (m_sub > 0) {
    const int64_t kb = i / m_sub;
    is = i - kb * m_sub;
    c1 += static_cast<uint32_t>(kb);
  }
  const uint32_t c0 = c0_idx ? c0_idx[is] : static_cast<uint32_t>(is);
  if (p.model == ABC_MODEL_GAUSS_TOY) {
    dist[i] = toy_dist(p, th, c0, c1, tag);
    if (ard_last) {  // the toy has no compartments
      ard_last[0 * n + i] = 0;
      ard_last[1 * n + i] = 0;
      ard_last[2 * n + i] = 0;
    }
  } else {
    int32_t last[3];
    const U128 a = saird_path(p, th, c0, c1, tag, nobs ? s_obs : nullptr, traj, n, i, nullptr,
                              mask, bq, last, obs_nonneg);
    dist[i] = __dsqrt_rn(u128_to_double(a.hi, a.lo));
    if (ard_last) {
      ard_last[0 * n + i] = last[0];
      ard_last[1 * n + i] = last[1];
      ard_last[2 * n + i] = last[2];
    }
  }
}

__global__ void k_prior(SimParams p, int64_t n, float* __restrict__ u) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const u32x4 a = philox4x32_10(static_cast<uint32_t>(j), 0u, 0u, ABC_TAG_PRIOR, p.k0, p.k1);
  const u32x4 b = philox4x32_10(static_cast<uint32_t>(j), 0u, 1u, ABC_TAG_PRIOR, p.k0, p.k1);
  const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
  for (int d = 0; d < 8; ++d) u[static_cast<int64_t>(d) * n + j] = unif(w[d]);
}

// A0: one thread draws theta* in the sub-box and simulates it (A_T > A0 wanted)
__global__ void k_synth_obs(SimParams p, float4 lo0, float4 lo1, float4 hi0, float4 hi1,
                            int32_t* __restrict__ obs, float* __restrict__ theta_star,
                            int32_t* __restrict__ attempts) {
  __shared__ BinvJob bq[kBinvQueue];
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const float lo[8] = {lo0.x, lo0.y, lo0.z, lo0.w, lo1.x, lo1.y, lo1.z, lo1.w};
  const float hi[8] = {hi0.x, hi0.y, hi0.z, hi0.w, hi1.x, hi1.y, hi1.z, hi1.w};
  const int T = p.T;
  int a;
  for (a = 0; a < 64; ++a) {
    const u32x4 wa = philox4x32_10(0u, static_cast<uint32_t>(a), 0u, ABC_TAG_OBS_THETA, p.k0, p.k1);
    const u32x4 wb = philox4x32_10(0u, static_cast<uint32_t>(a), 1u, ABC_TAG_OBS_THETA, p.k0, p.k1);
    const uint32_t w[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
    float th[8];
    for (int d = 0; d < 8; ++d)
      th[d] = __fadd_rn(lo[d], __fmul_rn(unif(w[d]), __fsub_rn(hi[d], lo[d])));
    obs[0 * (T + 1)] = p.A0;
    obs[1 * (T + 1)] = p.R0;
    obs[2 * (T + 1)] = p.D0;
    saird_path(p, th, 0u, static_cast<uint32_t>(a), ABC_TAG_OBS, nullptr, nullptr, 0, 0, obs, 1u,
               bq);
    for (int d = 0; d < 8; ++d) theta_star[d] = th[d];
    if (obs[0 * (T + 1) + T] > p.A0) break;
  }
  *attempts = a < 64 ? a + 1 : -64;
}

__global__ void k_philox(const uint32_t* __restrict__ ctr, uint32_t k0, uint32_t k1, int64_t n,
                         uint32_t* __restrict__ out) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const u32x4 r = philox4x32_10(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3], k0, k1);
  out[4 * i] = r.x;
  out[4 * i + 1] = r.y;
  out[4 * i + 2] = r.z;
  out[4 * i + 3] = r.w;
}

// ---- simulation order ------------------------------------------------------
// The lanes of a warp run their trajectories in lockstep, so lanes whose
// binomial draws fall in different regimes (normal approximation, inversion
// loop, trivial) serialise.  Slots are therefore simulated in the order of a
// key that predicts their regime mix.  The key is a heuristic only: every
// slot keeps its own Philox counters and writes its own outputs, so the
// order changes no result.
//
// Key of a slot: its expected-value path (each day's draws replaced by
// their means n p; Euler steps of three days, fast-math arithmetic) over the T
// days; c counts the draws of that path whose n min(p, 1 - p) is below 10
// (the sampler's inversion regime, trivial draws included) and dpk is the
// day of its largest I; key = min(c, 511) << 7 | min(dpk, 127).  Skipped
// slots sort last.
__global__ void k_sim_order_key(SimParams p, const float* __restrict__ u, int64_t n,
                                const uint8_t* __restrict__ skip, const int* __restrict__ off_dev,
                                const int* __restrict__ n_dev, uint32_t* __restrict__ key) {
  if (off_dev && *off_dev) return;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n || (n_dev && i >= *n_dev)) return;
  if (skip && skip[i]) {
    key[i] = 0xFFFFu;
    return;
  }
  float th[8];
#pragma unroll
  for (int d = 0; d < 8; ++d) th[d] = theta_of(p, d, u[static_cast<int64_t>(d) * n + i]);
  const float a0 = th[0], al = th[1], nn = th[2], be = th[3], ga = th[4], de = th[5],
              et = th[6], ka = th[7];
  const float Pf = static_cast<float>(p.P);
  float A = static_cast<float>(p.A0), R = static_cast<float>(p.R0), D = static_cast<float>(p.D0);
  float I = ka * A;
  float S = fmaxf(Pf - (A + R + D + I), 0.0f);
  const float lamI = ga + be * et, lamA = be + de;
  const float pI = 1.0f - __expf(-lamI), pA = 1.0f - __expf(-lamA);
  const float fI = lamI > 0.0f ? __fdividef(ga, lamI) : 0.0f;
  const float fA = lamA > 0.0f ? __fdividef(be, lamA) : 0.0f;
  const float qpI = fminf(pI, 1.0f - pI), qpA = fminf(pA, 1.0f - pA);
  const float qI = fminf(fI, 1.0f - fI), qA = fminf(fA, 1.0f - fA);
  int c = 0, dpk = 0;
  float peak = 0.0f;
  const float invP = 1.0f / Pf;
  for (int day = 0; day < p.T; day += 3) {
    const float x = fmaxf(A + R + D, 1.0f);
    const float g = a0 + __fdividef(al, 1.0f + __expf(nn * __logf(x)));
    const float pSI = 1.0f - __expf(-g * (I * invP));
    const float LI = I * pI, LA = A * pA;
    c += 3 * ((S * fminf(pSI, 1.0f - pSI) < 10.0f) + (I * qpI < 10.0f) + (A * qpA < 10.0f) +
              (LI * qI < 10.0f) + (LA * qA < 10.0f));
    const float k1 = S * pSI;
    S = fmaxf(S - 3.0f * k1, 0.0f);
    I = fmaxf(I + 3.0f * (k1 - LI), 0.0f);
    A = fmaxf(A + 3.0f * (LI * fI - LA), 0.0f);
    R += 3.0f * LA * fA;
    D += 3.0f * LA * (1.0f - fA);
    if (I > peak) {
      peak = I;
      dpk = day;
    }
  }
  key[i] = (static_cast<uint32_t>(min(c, 511)) << 7) | static_cast<uint32_t>(min(dpk, 127));
}

// ---- host launchers (called by the C ABI layer) --------------------------
int launch_simulate(const SimParams& p, const int32_t* obs, const float* u, int64_t n,
                    const uint32_t* c0_idx, uint32_t c1, uint32_t tag, const uint8_t* skip,
                    double* dist, int32_t* traj, cudaStream_t st, const uint32_t* c1_dev,
                    const int* off_dev, int threads, int32_t* ard_last, int64_t m_sub,
                    const int* n_dev, const int32_t* perm) {
  if (n <= 0) return ABC_OK;
  if (m_sub < 0) return ABC_E_INVAL;
  // 64 registers per thread (__launch_bounds__(256, 4)): up to 8 CTAs of
  // 128 threads per SM; blocks of at most 256 threads
  if (threads != 64 && threads != 128 && threads != 256) return ABC_E_INVAL;
  const size_t nobs = (p.model == ABC_MODEL_SAIRD && obs) ? 3 * static_cast<size_t>(p.T + 1) : 0;
  const size_t smem = sizeof(int32_t) * ((nobs + 3) & ~static_cast<size_t>(3)) +
                      sizeof(BinvJob) * kBinvQueue * static_cast<size_t>(threads / 32);
  k_simulate<<<static_cast<unsigned>(ceil_div(n, threads)), threads, smem, st>>>(
      p, obs, u, n, c0_idx, c1, tag, skip, dist, traj, c1_dev, off_dev, ard_last, m_sub, n_dev,
      perm);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

namespace {
struct SimOrderLayout {
  size_t key, key_s, perm, sort, total;
};
SimOrderLayout sim_order_layout(int64_t n) {
  SimOrderLayout l{};
  const size_t w = align256(sizeof(uint32_t) * static_cast<size_t>(n));
  l.key = 0;
  l.key_s = w;
  l.perm = 2 * w;
  l.sort = 3 * w;
  l.total = l.sort + radix_sort_scratch_bytes(n);
  return l;
}
}  // namespace

size_t sim_order_scratch_bytes(int64_t n) {
  return n >= kSimOrderMin ? sim_order_layout(n).total : 0;
}

int launch_simulate_ordered(const SimParams& p, const int32_t* obs, const float* u, int64_t n,
                            uint32_t c1, const uint8_t* skip, double* dist, void* scratch,
                            size_t bytes, cudaStream_t st, const uint32_t* c1_dev,
                            const int* off_dev, int threads, int64_t m_sub,
                            const uint32_t* c0_idx, const int* n_dev, int32_t* ard_last) {
  if (p.model != ABC_MODEL_SAIRD || n < kSimOrderMin || !obs)
    return launch_simulate(p, obs, u, n, c0_idx, c1, ABC_TAG_SIM, skip, dist, nullptr, st,
                           c1_dev, off_dev, threads, ard_last, m_sub, n_dev);
  const SimOrderLayout l = sim_order_layout(n);
  if (!scratch || bytes < l.total) return ABC_E_SCRATCH;
  char* b = static_cast<char*>(scratch);
  uint32_t* key = reinterpret_cast<uint32_t*>(b + l.key);
  uint32_t* key_s = reinterpret_cast<uint32_t*>(b + l.key_s);
  int32_t* perm = reinterpret_cast<int32_t*>(b + l.perm);
  k_sim_order_key<<<static_cast<unsigned>(ceil_div(n, 256)), 256, 0, st>>>(p, u, n, skip, off_dev,
                                                                            n_dev, key);
  ABC_LAUNCH_CHECK();
  int rc = launch_radix_sort(key, nullptr, key_s, perm, n, n_dev, 16, b + l.sort,
                             l.total - l.sort, st);
  if (rc) return rc;
  return launch_simulate(p, obs, u, n, c0_idx, c1, ABC_TAG_SIM, skip, dist, nullptr, st, c1_dev,
                         off_dev, threads, ard_last, m_sub, n_dev, perm);
}

int launch_prior(const SimParams& p, int64_t n, float* u, cudaStream_t st) {
  if (n <= 0) return ABC_OK;
  k_prior<<<static_cast<unsigned>(ceil_div(n, 256)), 256, 0, st>>>(p, n, u);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

int launch_synth_obs(const SimParams& p, const float* lo, const float* hi, int32_t* obs,
                     float* theta_star, int32_t* attempts, cudaStream_t st) {
  k_synth_obs<<<1, 32, 0, st>>>(p, make_float4(lo[0], lo[1], lo[2], lo[3]),
                                make_float4(lo[4], lo[5], lo[6], lo[7]),
                                make_float4(hi[0], hi[1], hi[2], hi[3]),
                                make_float4(hi[4], hi[5], hi[6], hi[7]), obs, theta_star,
                                attempts);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

int launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, int64_t n, uint32_t* out,
                  cudaStream_t st) {
  if (n <= 0) return ABC_OK;
  k_philox<<<static_cast<unsigned>(ceil_div(n, 256)), 256, 0, st>>>(ctr, k0, k1, n, out);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

}  // namespace abc
