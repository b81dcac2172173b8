// common.cuh -- internal types and helpers shared by the kernels and the
// C ABI layer (never exposed in the public header).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/abcsmc.h"

namespace abc {

// Model parameters as the kernels see them (by value, ~220 bytes).
struct SimParams {
  int32_t model, sampler, T, pad;
  int32_t A0, R0, D0, pad2;
  int64_t P;
  float lo[8], hi[8], x_obs[8];
  uint32_t k0, k1;  // Philox key
  // the key of each of the ten Philox rounds (k + r * Weyl constant), read
  // from the kernel-parameter bank by the simulator's generator
  uint32_t rk0[10], rk1[10];
};

inline SimParams make_params(const abc_config& c) {
  SimParams p{};
  p.model = c.model;
  p.sampler = c.sampler;
  p.T = c.n_days;
  p.A0 = c.init_ard[0];
  p.R0 = c.init_ard[1];
  p.D0 = c.init_ard[2];
  p.P = c.population;
  for (int d = 0; d < 8; ++d) {
    p.lo[d] = c.theta_lo[d];
    p.hi[d] = c.theta_hi[d];
    p.x_obs[d] = c.x_obs[d];
  }
  p.k0 = static_cast<uint32_t>(c.seed & 0xFFFFFFFFull);
  p.k1 = static_cast<uint32_t>(c.seed >> 32) ^ c.run_id;
  for (int r = 0; r < 10; ++r) {
    p.rk0[r] = p.k0 + static_cast<uint32_t>(r) * 0x9E3779B9u;
    p.rk1[r] = p.k1 + static_cast<uint32_t>(r) * 0xBB67AE85u;
  }
  return p;
}

#define ABC_CUDA_TRY(expr)                                  \
  do {                                                      \
    cudaError_t abc_err_ = (expr);                          \
    if (abc_err_ != cudaSuccess) return ABC_E_CUDA;         \
  } while (0)

// Every kernel launch is followed by ABC_LAUNCH_CHECK(), which also counts
// the launch (reported per generation).
int64_t count_launch();
int64_t launch_count();  // launches counted so far (no increment)
#define ABC_LAUNCH_CHECK()      \
  do {                          \
    ::abc::count_launch();      \
    ABC_CUDA_TRY(cudaGetLastError()); \
  } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// round up to 256 bytes so that sub-buffers of one scratch area stay aligned
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// ---- block-level scans and reductions (blockDim.x a multiple of 32) ------
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

// inclusive scan over the block; smem needs blockDim.x / 32 elements
template <typename T>
__device__ __forceinline__ T block_incl_scan(T v, T* smem) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  v = warp_incl_scan(v);
  if (lane == 31) smem[warp] = v;
  __syncthreads();
  if (warp == 0) {
    T w = lane < nw ? smem[lane] : T(0);
    w = warp_incl_scan(w);
    if (lane < nw) smem[lane] = w;
  }
  __syncthreads();
  T off = warp > 0 ? smem[warp - 1] : T(0);
  __syncthreads();
  return v + off;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* smem) {
  T inc = block_incl_scan(v, smem);
  __shared__ T last;
  if (threadIdx.x == blockDim.x - 1) last = inc;
  __syncthreads();
  T r = last;
  __syncthreads();
  return r;
}

// Where the rows of a weight pass came from (all members nullable together):
// row j was proposed from particle anc[j] of the previous population
// u_prev [8][n_prev], whose quantised stage-prior weight q_prev[anc[j]] is
// non-zero (the ancestor was drawn in proportion to it).
// Optional timing of the two kernels of a weight pass: events recorded
// around the tensor-core kernel (tc0/tc1) and the FP32 kernel (fp0/fp1);
// counts (out) points at the device pair [FP32 rows, tensor-core rows].
struct WeightTiming {
  cudaEvent_t tc0 = nullptr, tc1 = nullptr, fp0 = nullptr, fp1 = nullptr;
  const int* counts = nullptr;
  const unsigned long long* tiles = nullptr;  // tile products of the tensor-core kernel
};

// Step-size Beta rule of stage t (Eq. 16 and the mean-variance and
// mode-concentration parameterisations of Sec. 3.2): mode ABC_BETA_*, the
// fixed shapes (a, b) and the real-shape parameters p1, p2.
struct BetaRule {
  int32_t mode;
  float a;
  int32_t b;
  float p1, p2;
};

// The MCMC baseline's single step (ABC_STEP_MCMC, Sec. 2.4.1 and 3.1), kept
// on the device so that graph-captured batch loops adapt it between batches.
struct McmcDev {
  double s;            // current step (variance, unit-cube coordinates)
  long long k;         // adaptations made so far
  long long batches;   // batches walked with the step so far (generations >= 1)
  long long window;    // batches of the run that adapt
  long long acc_prev;  // the generation's accepted / exhausted counters after
  long long exh_prev;  //   the previous batch
  float s_f;           // (float) s, the step the next batch walks with
  float s_start;       // the step of the generation's first batch
};

// Shapes of a real-shape rule (ABC_BETA_REAL, _MEAN_VAR, _MODE_CONC) at stage
// t >= 1 with ratio = eps_t / eps_1 in fp32:
//   real:  (p1, p2);
//   mean-variance: mu = p1 ratio, v = p2 / t, nu = max(mu (1 - mu) / v - 1,
//     1/16), (a, b) = (mu nu, (1 - mu) nu);
//   mode-concentration: w = p1 ratio, k = p2 t, (a, b) = (w (k - 2) + 1,
//     (1 - w) (k - 2) + 1);
// the last two clamped to [2^-20, 2^20].  Plain fp32 operations, each
// rounded once (the library is built without contraction on host and device).
__host__ __device__ inline void beta_real_shape(const BetaRule& r, float ratio, int32_t t,
                                                float* a_out, float* b_out) {
  float a, b;
  if (r.mode == ABC_BETA_PAPER) {
    // Eq. 16 beyond the product form's 1024 uniforms (stage 513 on)
    a = ratio;
    if (!(a >= 0x1p-20f)) a = 0x1p-20f;
    if (a > 0x1p20f) a = 0x1p20f;
    b = static_cast<float>(2 * t);
  } else if (r.mode == ABC_BETA_REAL) {
    a = r.p1;
    b = r.p2;
  } else {
    if (r.mode == ABC_BETA_MEAN_VAR) {
      const float mu = r.p1 * ratio;
      const float v = r.p2 / static_cast<float>(t);
      float nu = (mu * (1.0f - mu)) / v - 1.0f;
      if (!(nu >= 0.0625f)) nu = 0.0625f;
      a = mu * nu;
      b = (1.0f - mu) * nu;
    } else {
      const float w = r.p1 * ratio;
      const float k2 = r.p2 * static_cast<float>(t) - 2.0f;
      a = w * k2 + 1.0f;
      b = (1.0f - w) * k2 + 1.0f;
    }
    if (!(a >= 0x1p-20f)) a = 0x1p-20f;
    if (!(b >= 0x1p-20f)) b = 0x1p-20f;
    if (a > 0x1p20f) a = 0x1p20f;
    if (b > 0x1p20f) b = 0x1p20f;
  }
  *a_out = a;
  *b_out = b;
}

struct AncInfo {
  const int32_t* anc = nullptr;
  const float* u_prev = nullptr;
  const uint32_t* q_prev = nullptr;
  int64_t n_prev = 0;
};

}  // namespace abc
