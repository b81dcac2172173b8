// numcheck.cu -- device-side exhaustive checks of the short arithmetic
// sequences that stand in for longer exact forms: CUDA's correctly rounded
// division and square root on bounded domains (div_nr, sqrt_nr in
// numerics.cuh) and the uniform's construction from bits (unif): each check
// runs both on every operand of the domain on this GPU and counts the
// results that differ in any bit.
#include <cstring>

#include "common.cuh"
#include "numerics.cuh"

namespace abc {

// domain 0: n = m - 1, d = m + 1 for every float m in [sqrt(1/2), sqrt(2)]
// (the logarithm's reduced argument: m or m / 2 as dev_log_core forms it)
__global__ void k_check_div_log(uint32_t lo, uint32_t hi, unsigned long long* bad) {
  unsigned long long c = 0;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t b = lo + blockIdx.x * blockDim.x + threadIdx.x; b <= hi && b >= lo; b += stride) {
    const float m = __uint_as_float(b);
    const float n = __fsub_rn(m, 1.0f), d = __fadd_rn(m, 1.0f);
    c += __float_as_uint(div_nr(n, d)) != __float_as_uint(__fdiv_rn(n, d));
  }
  if (c) atomicAdd(bad, c);
}

// domain 1: a / k for every float a in [2^-100, 2^100] and k = 2..111 (BINV's
// step factor)
__global__ void k_check_div_binv(uint32_t lo, uint32_t hi, unsigned long long* bad) {
  unsigned long long c = 0;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t b = lo + blockIdx.x * blockDim.x + threadIdx.x; b <= hi && b >= lo; b += stride) {
    const float a = __uint_as_float(b);
    for (int k = 2; k <= 111; ++k) {
      const float kf = static_cast<float>(k);
      c += __float_as_uint(div_nr(a, kf)) != __float_as_uint(__fdiv_rn(a, kf));
    }
  }
  if (c) atomicAdd(bad, c);
}

static uint32_t bits_of(float x) {
  uint32_t b;
  std::memcpy(&b, &x, sizeof b);
  return b;
}

// domain 2: every float x in [2^-24, 2^32) (the square roots of the
// binomial draw and of the Box-Muller radius)
__global__ void k_check_sqrt(uint32_t lo, uint32_t hi, unsigned long long* bad) {
  unsigned long long c = 0;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t b = lo + blockIdx.x * blockDim.x + threadIdx.x; b <= hi && b >= lo; b += stride) {
    const float x = __uint_as_float(b);
    c += __float_as_uint(sqrt_nr(x)) != __float_as_uint(__fsqrt_rn(x));
  }
  if (c) atomicAdd(bad, c);
}

// domain 3: every 23-bit significand m (the uniform of any word x with
// x >> 9 = m): unif against (m + 1/2) 2^-23 by conversion, addition and scaling
__global__ void k_check_unif(uint32_t lo, uint32_t hi, unsigned long long* bad) {
  unsigned long long c = 0;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t m = lo + blockIdx.x * blockDim.x + threadIdx.x; m <= hi && m >= lo; m += stride) {
    const float direct = __fmul_rn(__fadd_rn(__uint2float_rn(m), 0.5f), 0x1p-23f);
    c += __float_as_uint(unif((m << 9) | (m & 0x1FFu))) != __float_as_uint(direct);
  }
  if (c) atomicAdd(bad, c);
}

int numerics_check(int which, unsigned long long* bad_host, cudaStream_t st) {
  uint32_t lo, hi;
  if (which == 0) {
    lo = bits_of(kSqrt2 * 0.5f);  // the reduced argument lies in (kSqrt2 / 2, kSqrt2]
    hi = bits_of(kSqrt2);
  } else if (which == 1) {
    lo = bits_of(0x1p-100f);
    hi = bits_of(0x1p100f);
  } else if (which == 2) {
    lo = bits_of(0x1p-24f);
    hi = bits_of(0x1p32f) - 1u;
  } else if (which == 3) {
    lo = 0u;
    hi = (1u << 23) - 1u;
  } else {
    return ABC_E_INVAL;
  }
  unsigned long long* bad = nullptr;
  ABC_CUDA_TRY(cudaMallocAsync(&bad, sizeof *bad, st));
  int rc = ABC_OK;
  if (cudaMemsetAsync(bad, 0, sizeof *bad, st) != cudaSuccess) rc = ABC_E_CUDA;
  if (rc == ABC_OK) {
    if (which == 0) k_check_div_log<<<152 * 8, 256, 0, st>>>(lo, hi, bad);
    else if (which == 1) k_check_div_binv<<<152 * 8, 256, 0, st>>>(lo, hi, bad);
    else if (which == 2) k_check_sqrt<<<152 * 8, 256, 0, st>>>(lo, hi, bad);
    else k_check_unif<<<152 * 8, 256, 0, st>>>(lo, hi, bad);
    if (cudaGetLastError() != cudaSuccess) rc = ABC_E_CUDA;
  }
  if (rc == ABC_OK &&
      (cudaMemcpyAsync(bad_host, bad, sizeof *bad, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    rc = ABC_E_CUDA;
  cudaFreeAsync(bad, st);
  return rc;
}

}  // namespace abc
