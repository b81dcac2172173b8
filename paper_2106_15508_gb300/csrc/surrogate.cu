// surrogate.cu -- MLP surrogate u (8) -> 256 -> 256 -> 4 (tanh-form GELU)
// for delayed-acceptance pre-screening (an extension beyond the paper; the paper
// simulates every proposal).
//
// Parameters: fp32 master copy (Adam updates it) and a bf16 copy that every
// product uses (BF16 weights, FP32 accumulation).  Layouts, row = output:
// W1[256][8], b1[256], W2[256][256], b2[256], W3[4][256], b3[4].
// Outputs are the standardised summaries y = [log1p d, log1p A_T, log1p R_T,
// log1p D_T]; the per-output mean and standard deviation live beside the
// parameters.
//
// Training: the three 256-wide products of a step on tcgen05 (bf16 operands,
// fp32 accumulation) with fused epilogues, layers 1 and 3 and the gradient
// reductions on CUDA cores, Adam in fp32.
// Inference: one persistent kernel per call; per tile of 128 samples the
// input layer runs on tcgen05 from the standardised inputs split into three
// bf16 parts (K = 32), its bias + GELU form the bf16 hidden layer in shared
// memory, layer 2 runs on tcgen05 (M = 128, N = 256, K = 256) and bias +
// GELU + layer 3 are fused into the epilogue.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "numerics.cuh"
#include "surrogate.cuh"
#include "tcgen05.cuh"

namespace abc {

// ---- GELU (tanh form, Hendrycks & Gimpel) -------------------------------
// tanh by the hardware approximation (tanh.approx.f32, absolute error about
// 2^-11): the surrogate works at bf16 precision, and this keeps its
// activations cheap.  Beyond |x| = 5 the tanh form is within 1e-6 of its
// limits (x and 1 for x > 0, 0 for x < 0), which are used there.
__device__ __forceinline__ float tanh_fast(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float gelu_f(float x) {
  if (!(fabsf(x) < 5.0f)) return x > 0.0f ? x : 0.0f;
  const float c = 0.7978845608028654f;
  const float t = tanh_fast(c * (x + 0.044715f * x * x * x));
  return 0.5f * x * (1.0f + t);
}

__device__ __forceinline__ float gelu_grad_f(float x) {
  if (!(fabsf(x) < 5.0f)) return x > 0.0f ? 1.0f : 0.0f;
  const float c = 0.7978845608028654f;
  const float t = tanh_fast(c * (x + 0.044715f * x * x * x));
  return 0.5f * (1.0f + t) + 0.5f * x * (1.0f - t * t) * c * (1.0f + 3.0f * 0.044715f * x * x);
}

// ---- parameters ------------------------------------------------------------
__global__ void k_mlp_init(float* __restrict__ w, uint32_t k0, uint32_t k1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpParams) return;
  // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights from Philox, zero biases
  float bound = 0.0f;
  if (i < kOffB1) bound = 0.35355339f;                       // 1/sqrt(8)
  else if (i >= kOffW2 && i < kOffB2) bound = 0.0625f;       // 1/sqrt(256)
  else if (i >= kOffW3 && i < kOffB3) bound = 0.0625f;
  if (bound == 0.0f) {
    w[i] = 0.0f;
    return;
  }
  const uint32_t r = philox4x32_10(static_cast<uint32_t>(i), 0u, 0u, kTagMlpInit, k0, k1).x;
  const float v = (static_cast<float>(r >> 8) + 0.5f) * 0x1p-24f;
  w[i] = bound * (2.0f * v - 1.0f);
}

__global__ void k_mlp_to_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kMlpParams) wb[i] = __float2bfloat16_rn(w[i]);
}

// out[i] = sum_z P[z * n + i], z in order (deterministic split-K reduction)
__global__ void k_splitk_sum(const float* __restrict__ P, int splits, int64_t n,
                             float* __restrict__ out) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float v = 0.0f;
  for (int z = 0; z < splits; ++z) v += P[z * n + i];
  out[i] = v;
}

// ---- training pieces -------------------------------------------------------
// step_dev (nullable): the bias corrections use the step *step_dev + koff + 1
// counted on the device (graph launches), computed in fp64 and rounded
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1,
                       float c2, const uint32_t* __restrict__ step_dev, uint32_t koff) {
  __shared__ float sc[2];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (step_dev) {
    // bias corrections, once per block (fp64 powers are slow on this GPU)
    if (threadIdx.x == 0) {
      const double t = static_cast<double>(*step_dev) + static_cast<double>(koff) + 1.0;
      sc[0] = static_cast<float>(1.0 - pow(0.9, t));
      sc[1] = static_cast<float>(1.0 - pow(0.999, t));
    }
    __syncthreads();
    c1 = sc[0];
    c2 = sc[1];
  }
  if (i >= kMlpParams) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

int mlp_adam(const MlpState& s, const float* grad, int64_t step, float lr, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.0f - std::pow(b1, static_cast<float>(step));
  const float c2 = 1.0f - std::pow(b2, static_cast<float>(step));
  const unsigned g = (kMlpParams + 255) / 256;
  k_adam<<<g, 256, 0, st>>>(s.w, grad, s.m, s.v, lr, b1, b2, eps, c1, c2, nullptr, 0u);
  ABC_LAUNCH_CHECK();
  k_mlp_to_bf16<<<g, 256, 0, st>>>(s.w, s.wb);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

int mlp_init(const MlpState& s, uint32_t k0, uint32_t k1, cudaStream_t st) {
  const unsigned g = (kMlpParams + 255) / 256;
  k_mlp_init<<<g, 256, 0, st>>>(s.w, k0, k1);
  ABC_LAUNCH_CHECK();
  ABC_CUDA_TRY(cudaMemsetAsync(s.m, 0, sizeof(float) * kMlpParams, st));
  ABC_CUDA_TRY(cudaMemsetAsync(s.v, 0, sizeof(float) * kMlpParams, st));
  k_mlp_to_bf16<<<g, 256, 0, st>>>(s.w, s.wb);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

int mlp_refresh_bf16(const MlpState& s, cudaStream_t st) {
  k_mlp_to_bf16<<<(kMlpParams + 255) / 256, 256, 0, st>>>(s.w, s.wb);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}


// ---- inference on tensor cores ------------------------------------------------
constexpr int kMlpM = 128;                                  // samples per CTA
constexpr uint32_t kMlpATile = kMlpM * kMlpH * 2;           // 64 KB: h1 tile
constexpr uint32_t kMlpBBytes = kMlpH * kMlpH * 2;          // 128 KB: W2
// tensor-core MLP kernels: 16 epilogue warps (warp w reads TMEM lanes
// 32 (w % 4) .. + 31 and columns 64 (w / 4) .. + 63), one bulk-copy warp,
// one MMA warp
constexpr int kMlpEpiWarps = 16;
constexpr int kMlpThreads = 32 * (kMlpEpiWarps + 2);
constexpr size_t kMlpSmem = 1024 + kMlpATile + kMlpBBytes + (4 * kMlpH + kMlpH) * 4 +
                            4 * kMlpM * 4 * 4 + 256;
constexpr uint32_t kMlpIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                               (static_cast<uint32_t>(kMlpH >> 3) << 17) |
                               (static_cast<uint32_t>(kMlpM >> 4) << 24);

// element index of (row r, k) in a K = 256 tile: 8 x 8 core matrices, the 32
// of a row group consecutive along K (LBO 128 B), row groups 4096 B apart
__host__ __device__ __forceinline__ int mlp_packed_index(int r, int k) {
  return ((((r >> 3) << 5) + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7);
}

// W2 (bf16, [out][in]) as the B operand: rows = out, K = in
__global__ void k_mlp_pack_w2(const __nv_bfloat16* __restrict__ wb, __nv_bfloat16* __restrict__ W2pk) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kMlpH * kMlpH) return;
  const int o = idx / kMlpH, k = idx % kMlpH;
  W2pk[mlp_packed_index(o, k)] = wb[kOffW2 + o * kMlpH + k];
}

// epilogue barrier of the 16 epilogue warps (named barrier 1)
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 512;" ::: "memory"); }

// the hidden-layer tile is in shared memory: the 16 epilogue warps and the
// MMA warp (named barrier 2)
__device__ __forceinline__ void tile_ready_sync() { asm volatile("bar.sync 2, 544;" ::: "memory"); }

// generic-proxy writes to shared memory made visible to the tensor cores
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// The input layer as a tensor-core product: K = 32 tiles (8 x 8 core
// matrices, 4 along K, row groups 512 B apart).  The A operand holds each
// sample's standardised input split into three bf16 parts (x = hi + mid +
// lo exactly for normal fp32 x: 3 x 8 significant bits), k = 8 s + d for
// part s of feature d, zeros for s = 3; the B operand holds W1 (bf16) in
// the three part slots, so the fp32 accumulation over k forms W1 x.
__host__ __device__ __forceinline__ int mlp_packed_index32(int r, int k) {
  return ((((r >> 3) << 2) + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7);
}
constexpr uint32_t kMlpXTile = kMlpM * 32 * 2;    // 8 KB: split inputs of a tile
constexpr uint32_t kMlpW1Bytes = kMlpH * 32 * 2;  // 16 KB: W1 in the three part slots

__global__ void k_mlp_pack_w1(const __nv_bfloat16* __restrict__ wb,
                              __nv_bfloat16* __restrict__ W1pk) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kMlpH * 32) return;
  const int o = idx >> 5, k = idx & 31;
  W1pk[mlp_packed_index32(o, k)] = (k >> 3) < 3 ? wb[kOffW1 + o * 8 + (k & 7)]
                                                : __float2bfloat16_rn(0.0f);
}

// shared memory of the inference kernel: the hidden-layer tile, W2, W1 in
// the part slots, the split-input tile (reused for the epilogue's partial
// outputs once the input product has run), b1, b2, W3, barriers
constexpr size_t kMlpInfSmem = 1024 + kMlpATile + kMlpBBytes + kMlpW1Bytes + kMlpXTile +
                               (kMlpH + kMlpH + 4 * kMlpH) * 4 + 64;

// the split input tile is ready (named barrier 2), the hidden-layer tile
// is ready (named barrier 3): the 16 epilogue warps and the MMA warp
__device__ __forceinline__ void x_ready_sync() { asm volatile("bar.sync 2, 544;" ::: "memory"); }
__device__ __forceinline__ void h_ready_sync() { asm volatile("bar.sync 3, 544;" ::: "memory"); }

// Y[j][0..3] = W3 gelu(W2 gelu(W1 x_j + b1) + b2) + b3 for u [8][n] (x = the
// standardised u when xstat is given: (u - mean) / sd).  Persistent CTAs;
// W2 and the packed W1 are loaded once per CTA by bulk copies.  Per tile of
// 128 samples:
//   1. the 16 epilogue warps write the split inputs (warp group g = w / 4
//      writes part g of the 32 rows of its lane quarter q = w % 4; group 3
//      the zero part);
//   2. the MMA warp runs the input layer, 128 x 256 x 32, into TMEM columns
//      0..255;
//   3. the epilogue warps add b1, apply GELU, round to bf16 and write the
//      hidden-layer tile in the UMMA operand layout (warp w: TMEM lanes
//      32 q .. + 31, columns 64 g .. + 63);
//   4. the MMA warp runs layer 2, 128 x 256 x 256, into columns 256..511;
//   5. the epilogue warps add b2, apply GELU and form layer 3, the four
//      column groups' partial outputs added in order.
// Every wait is bounded; a wait that gives up records its code in *err and
// the CTA runs to its end without further waits.
__global__ void __launch_bounds__(kMlpThreads, 1)
k_mlp_infer_tc(const float* __restrict__ u, int64_t n, int64_t ntiles,
               const uint8_t* __restrict__ W2pk, const uint8_t* __restrict__ W1pk,
               const float* __restrict__ w, const __nv_bfloat16* __restrict__ wb,
               const float* __restrict__ xstat, float* __restrict__ Y, unsigned* err) {
  extern __shared__ uint8_t mlp_smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(mlp_smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  uint8_t* sA = base;                       // hidden layer, K = 256
  uint8_t* sB = sA + kMlpATile;             // W2
  uint8_t* sW1 = sB + kMlpBBytes;           // W1, K = 32
  uint8_t* sX = sW1 + kMlpW1Bytes;          // split inputs, K = 32
  float* sY = reinterpret_cast<float*>(sX);  // [4 column groups][128 rows][4], after step 2
  float* sb1 = reinterpret_cast<float*>(sX + kMlpXTile);
  float* sb2 = sb1 + kMlpH;
  float4* sW3 = reinterpret_cast<float4*>(sb2 + kMlpH);  // [256] (W3[0..3][col])
  uint64_t* bars = reinterpret_cast<uint64_t*>(sW3 + kMlpH);
  uint64_t* full = bars;
  uint64_t* t1full = bars + 1;
  uint64_t* t2full = bars + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kMlpH; i += blockDim.x) {
    sb1[i] = w[kOffB1 + i];
    sb2[i] = w[kOffB2 + i];
    sW3[i] = make_float4(__bfloat162float(wb[kOffW3 + i]), __bfloat162float(wb[kOffW3 + kMlpH + i]),
                         __bfloat162float(wb[kOffW3 + 2 * kMlpH + i]),
                         __bfloat162float(wb[kOffW3 + 3 * kMlpH + i]));
  }
  if (threadIdx.x == 0) {
    mbar_init(full, 1);
    mbar_init(t1full, 1);
    mbar_init(t2full, 1);
    fence_mbar_init();
  }
  if (warp == kMlpEpiWarps + 1) {
    tmem_alloc(tmem_slot, 2 * kMlpH);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t acc1 = tmem, acc2 = tmem + kMlpH;
  if (warp == kMlpEpiWarps) {
    // W2 and W1, once per CTA
    if (lane == 0) {
      mbar_expect_tx(full, kMlpBBytes + kMlpW1Bytes);
      bulk_g2s(sB, W2pk, kMlpBBytes, full);
      bulk_g2s(sW1, W1pk, kMlpW1Bytes, full);
      mbar_wait(full, 0u, err, 31u);  // the copies landed before the CTA can exit
    }
  } else if (warp == kMlpEpiWarps + 1) {
    bool ok = lane == 0 ? mbar_wait(full, 0u, err, 32u) : true;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    int committed = -1;
    const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB), x0 = smem_u32(sX), w0 = smem_u32(sW1);
    int it = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      x_ready_sync();
      tc_fence_after();
      if (lane == 0 && ok) {
#pragma unroll
        for (int kk = 0; kk < 2; ++kk)
          umma_bf16(acc1, smem_desc(x0 + kk * 256, 128, 512), smem_desc(w0 + kk * 256, 128, 512),
                    kMlpIdesc, kk > 0 ? 1u : 0u);
        umma_commit(t1full);
      }
      __syncwarp();
      h_ready_sync();
      tc_fence_after();
      if (lane == 0 && ok) {
#pragma unroll
        for (int kk = 0; kk < kMlpH / 16; ++kk)
          umma_bf16(acc2, smem_desc(a0 + kk * 256, 128, 4096),
                    smem_desc(b0 + kk * 256, 128, 4096), kMlpIdesc, kk > 0 ? 1u : 0u);
        umma_commit(t2full);
        committed = it;
      }
      __syncwarp();
    }
    // the last products completed before the tensor memory is released
    if (lane == 0 && committed >= 0) mbar_wait(t2full, static_cast<uint32_t>(committed) & 1u, err, 33u);
    __syncwarp();
  } else {
    const int q = warp & 3, g = warp >> 2;
    const int r = q * 32 + lane;
    const uint32_t lanes = static_cast<uint32_t>(q * 32) << 16;
    bool ok = true;
    int it = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      const int64_t j = t * kMlpM + r;
      // 1. part g of row r's split input (zeros for g = 3 and padding rows)
      {
        uint32_t hv[4] = {0u, 0u, 0u, 0u};
        if (g < 3 && j < n) {
          uint32_t pb[8];
#pragma unroll
          for (int d = 0; d < 8; ++d) {
            float x = u[d * n + j];
            if (xstat) x = __fdiv_rn(__fsub_rn(x, xstat[d]), xstat[8 + d]);
            const __nv_bfloat16 hi = __float2bfloat16_rn(x);
            const float r1 = __fsub_rn(x, __bfloat162float(hi));
            const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
            const __nv_bfloat16 lo = __float2bfloat16_rn(__fsub_rn(r1, __bfloat162float(mid)));
            pb[d] = __bfloat16_as_ushort(g == 0 ? hi : (g == 1 ? mid : lo));
          }
#pragma unroll
          for (int e = 0; e < 4; ++e) hv[e] = pb[2 * e] | (pb[2 * e + 1] << 16);
        }
        *reinterpret_cast<uint4*>(sX + 2 * mlp_packed_index32(r, 8 * g)) =
            make_uint4(hv[0], hv[1], hv[2], hv[3]);
      }
      fence_proxy_async_smem();
      tc_fence_before();  // this thread's reads of the previous tile's TMEM
      x_ready_sync();
      // 3. the hidden layer from the input product
      ok = __all_sync(0xffffffffu, ok && mbar_wait(t1full, static_cast<uint32_t>(it) & 1u, err, 34u));
      tc_fence_after();
      if (ok) {
        for (int cc = 0; cc < 2; ++cc) {
          const int cb = 2 * g + cc;
          float v[32];
          tmem_ld32(acc1 + lanes + cb * 32, v);
#pragma unroll
          for (int c8 = 0; c8 < 4; ++c8) {
            uint32_t hh[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int col = cb * 32 + c8 * 8 + 2 * e;
              const float h0 = gelu_f(v[c8 * 8 + 2 * e] + sb1[col]);
              const float h1 = gelu_f(v[c8 * 8 + 2 * e + 1] + sb1[col + 1]);
              hh[e] = __bfloat16_as_ushort(__float2bfloat16_rn(j < n ? h0 : 0.0f)) |
                      (static_cast<uint32_t>(__bfloat16_as_ushort(
                           __float2bfloat16_rn(j < n ? h1 : 0.0f))) << 16);
            }
            *reinterpret_cast<uint4*>(sA + 2 * mlp_packed_index(r, cb * 32 + c8 * 8)) =
                make_uint4(hh[0], hh[1], hh[2], hh[3]);
          }
        }
      }
      fence_proxy_async_smem();
      tc_fence_before();
      h_ready_sync();
      // 5. layer 2's activation and layer 3
      ok = __all_sync(0xffffffffu, ok && mbar_wait(t2full, static_cast<uint32_t>(it) & 1u, err, 35u));
      tc_fence_after();
      float y[4] = {0.f, 0.f, 0.f, 0.f};
      if (ok) {
        for (int cc = 0; cc < 2; ++cc) {
          const int cb = 2 * g + cc;
          float v[32];
          tmem_ld32(acc2 + lanes + cb * 32, v);
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int col = cb * 32 + i;
            const float hh = gelu_f(v[i] + sb2[col]);
            const float4 w3 = sW3[col];
            y[0] = __fmaf_rn(hh, w3.x, y[0]);
            y[1] = __fmaf_rn(hh, w3.y, y[1]);
            y[2] = __fmaf_rn(hh, w3.z, y[2]);
            y[3] = __fmaf_rn(hh, w3.w, y[3]);
          }
        }
      }
#pragma unroll
      for (int o = 0; o < 4; ++o) sY[(g * kMlpM + r) * 4 + o] = y[o];
      epi_sync();
      if (g == 0 && j < n) {
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          float tt = sY[r * 4 + o];  // column groups added in order
          for (int gg = 1; gg < 4; ++gg) tt += sY[(gg * kMlpM + r) * 4 + o];
          Y[j * 4 + o] = tt + w[kOffB3 + o];
        }
      }
      epi_sync();  // the partial outputs are read before the next tile's inputs overwrite them
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kMlpEpiWarps + 1) tmem_dealloc(tmem, 2 * kMlpH);
}

size_t mlp_infer_scratch_bytes(int64_t) {
  return align256(kMlpBBytes) + align256(kMlpW1Bytes) + align256(16);
}

int mlp_infer_prepare() {
  ABC_CUDA_TRY(cudaFuncSetAttribute(k_mlp_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(kMlpInfSmem)));
  return ABC_OK;
}

// the error word of mlp_infer inside its scratch
unsigned* mlp_infer_err(void* scratch, int64_t) {
  return reinterpret_cast<unsigned*>(static_cast<char*>(scratch) + align256(kMlpBBytes) +
                                     align256(kMlpW1Bytes));
}

namespace {
int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      n = v;
    else
      return 1;
  }
  return n;
}
}  // namespace

// Y [n][4] (standardised outputs) for u [8][n]; the error word lives in scratch
int mlp_infer(const MlpState& s, const float* u, int64_t n, float* Y, void* scratch, size_t bytes,
              unsigned** err_out, cudaStream_t st, bool reset_err, unsigned* err_word,
              const float* xstat) {
  if (n <= 0) return ABC_OK;
  if (bytes < mlp_infer_scratch_bytes(n)) return ABC_E_SCRATCH;
  const int64_t ntiles = ceil_div(n, kMlpM);
  auto* W2pk = reinterpret_cast<__nv_bfloat16*>(scratch);
  auto* W1pk = reinterpret_cast<__nv_bfloat16*>(static_cast<char*>(scratch) + align256(kMlpBBytes));
  unsigned* err = err_word ? err_word : mlp_infer_err(scratch, n);
  if (err_out) *err_out = err;
  if (reset_err) ABC_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(unsigned), st));
  k_mlp_pack_w2<<<(kMlpH * kMlpH + 255) / 256, 256, 0, st>>>(s.wb, W2pk);
  ABC_LAUNCH_CHECK();
  k_mlp_pack_w1<<<(kMlpH * 32 + 255) / 256, 256, 0, st>>>(s.wb, W1pk);
  ABC_LAUNCH_CHECK();
  const unsigned grid = static_cast<unsigned>(std::min<int64_t>(ntiles, sm_count()));
  k_mlp_infer_tc<<<grid, kMlpThreads, kMlpInfSmem, st>>>(
      u, n, ntiles, reinterpret_cast<const uint8_t*>(W2pk), reinterpret_cast<const uint8_t*>(W1pk),
      s.w, s.wb, xstat, Y, err);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

// ---- training on tensor cores -------------------------------------------------
// Packed bf16 operands (8 x 8 core matrices, K-major, 256 K-elements per tile,
// the inference layout):
//   R-layout (samples x features): tile t holds samples 128 t .. 128 t + 127,
//     64 KB, element (b, k) at t * 32768 + mlp_packed_index(b % 128, k);
//   T-layout (features x samples): tile c holds samples 256 c .. 256 c + 255,
//     128 KB, element (k, b) at c * 65536 + mlp_packed_index(k, b % 256).
// One kernel runs the three products of a training step, each a
// 128 x 256 x 256 UMMA per CTA with operands staged by two bulk copies:
//   kTrFwd: Z2 = H1 W2^T (A = H1 R-tile, B = W2 packed by output row); the
//     epilogue adds b2, applies GELU, forms layer 3, the loss and dY, then
//     back through layer 3 and GELU: dZ2 = (dY W3) gelu'(Z2), written in
//     both layouts and in fp32 (feature-major), and H2 in fp32 (feature-major);
//   kTrBwd: dH1 = dZ2 W2 (A = dZ2 R-tile, B = W2^T packed); the epilogue
//     recomputes Z1 from X and forms dZ1 = dH1 gelu'(Z1) in fp32
//     (feature-major);
//   kTrGw2: gW2 = dZ2^T H1 over one 256-sample tile c (A = rows 128 m .. of
//     the dZ2 T-tile, B = the H1 T-tile); the epilogue writes the tile's
//     fp32 partial, summed over tiles in order afterwards (deterministic).
// Rows past the batch (padding to a multiple of 256) carry dY = 0.
enum TrMode { kTrFwd = 0, kTrBwd = 1, kTrGw2 = 2 };

struct TrArgs {
  int B;                      // samples (rows past B are padding)
  const float* w;             // fp32 parameters (biases)
  const __nv_bfloat16* wb;    // bf16 parameters (W3)
  int Bp;                     // padded batch (a multiple of 256): the stride of [256][Bp]
  const float* T;             // targets [B][4] (kTrFwd)
  float* H2;                  // [256][Bp] fp32 (kTrFwd)
  float* dY;                  // [Bp][4] (kTrFwd)
  float* lossp;               // [Bp] squared errors (kTrFwd)
  float* dZ2f;                // [256][Bp] fp32 (kTrFwd)
  __nv_bfloat16* dZ2R;        // R-layout (kTrFwd)
  __nv_bfloat16* dZ2T;        // T-layout (kTrFwd)
  const float* X;             // inputs [B][8] (kTrBwd: Z1 recomputed)
  float* dZ1;                 // [256][Bp] fp32 (kTrBwd)
  float* gW2p;                // [tiles][256][256] (kTrGw2)
};

template <int MODE>
__global__ void __launch_bounds__(kMlpThreads, 1)
k_mlp_train_tc(const uint8_t* __restrict__ Abase, const uint8_t* __restrict__ Bbase, TrArgs a,
               unsigned* err) {
  extern __shared__ uint8_t mlp_smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(mlp_smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  uint8_t* sA = base;
  uint8_t* sB = base + kMlpATile;
  float* sW3 = reinterpret_cast<float*>(sB + kMlpBBytes);
  float* sb2 = sW3 + 4 * kMlpH;
  float* sY = sb2 + kMlpH;  // [4 column groups][128 rows][4] partial outputs
  uint64_t* bars = reinterpret_cast<uint64_t*>(sY + 4 * kMlpM * 4);
  uint64_t* full = bars;
  uint64_t* tfull = bars + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (MODE == kTrFwd) {
    for (int i = threadIdx.x; i < 4 * kMlpH; i += blockDim.x)
      sW3[i] = __bfloat162float(a.wb[kOffW3 + i]);
    for (int i = threadIdx.x; i < kMlpH; i += blockDim.x) sb2[i] = a.w[kOffB2 + i];
  } else if (MODE == kTrBwd) {
    // layer 1 (W1 as its bf16 values, b1) to recompute Z1: 9 KB over the
    // W3 / b2 / partial-output area, which this mode does not use
    for (int i = threadIdx.x; i < 8 * kMlpH; i += blockDim.x)
      sW3[i] = __bfloat162float(a.wb[kOffW1 + i]);
    for (int i = threadIdx.x; i < kMlpH; i += blockDim.x) sW3[8 * kMlpH + i] = a.w[kOffB1 + i];
  }
  if (threadIdx.x == 0) {
    mbar_init(full, 1);
    mbar_init(tfull, 1);
    fence_mbar_init();
  }
  if (warp == kMlpEpiWarps + 1) {
    tmem_alloc(tmem_slot, kMlpH);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // operand tiles of this CTA
  const uint8_t* gA;
  const uint8_t* gB;
  if (MODE == kTrGw2) {
    gA = Abase + static_cast<size_t>(blockIdx.y) * (2 * kMlpATile) +
         static_cast<size_t>(blockIdx.x) * kMlpATile;
    gB = Bbase + static_cast<size_t>(blockIdx.y) * kMlpBBytes;
  } else {
    gA = Abase + static_cast<size_t>(blockIdx.x) * kMlpATile;
    gB = Bbase;
  }
  if (warp == kMlpEpiWarps) {
    if (lane == 0) {
      mbar_expect_tx(full, kMlpATile + kMlpBBytes);
      bulk_g2s(sA, gA, kMlpATile, full);
      bulk_g2s(sB, gB, kMlpBBytes, full);
      mbar_wait(full, 0u, err, 31u);  // both copies landed before the CTA can exit
    }
  } else if (warp == kMlpEpiWarps + 1) {
    if (lane == 0 && mbar_wait(full, 0u, err, 32u)) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
      for (int kk = 0; kk < kMlpH / 16; ++kk)
        umma_bf16(tmem, smem_desc(a0 + kk * 256, 128, 4096), smem_desc(b0 + kk * 256, 128, 4096),
                  kMlpIdesc, kk > 0 ? 1u : 0u);
      umma_commit(tfull);
      mbar_wait(tfull, 0u, err, 33u);
    }
    __syncwarp();
  } else {
    // epilogue: warp w takes accumulator rows 32 (w % 4) .. + 31 (its TMEM
    // lanes) and columns 64 (w / 4) .. + 63
    const bool ok = __all_sync(0xffffffffu, mbar_wait(tfull, 0u, err, 34u));
    tc_fence_after();
    const int q = warp & 3, g = warp >> 2;
    const int r = q * 32 + lane;  // 0..127
    const uint32_t lane_base = tmem + (static_cast<uint32_t>(q * 32) << 16);
    if (MODE == kTrFwd) {
      const int64_t b = static_cast<int64_t>(blockIdx.x) * kMlpM + r;
      const bool live = b < a.B;
      float y[4] = {0.f, 0.f, 0.f, 0.f};
      if (ok) {
        for (int cc = 0; cc < 2; ++cc) {
          const int c = 2 * g + cc;
          float v[32];
          tmem_ld32(lane_base + c * 32, v);
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int col = c * 32 + i;
            const float h = gelu_f(v[i] + sb2[col]);
            a.H2[static_cast<int64_t>(col) * a.Bp + b] = h;
#pragma unroll
            for (int o = 0; o < 4; ++o) y[o] = __fmaf_rn(sW3[o * kMlpH + col], h, y[o]);
          }
        }
      }
#pragma unroll
      for (int o = 0; o < 4; ++o) sY[(g * kMlpM + r) * 4 + o] = y[o];
      epi_sync();
      // the row's outputs (column groups added in order), loss and dY
      float dy[4], l = 0.f;
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        float t = sY[r * 4 + o];
        for (int gg = 1; gg < 4; ++gg) t += sY[(gg * kMlpM + r) * 4 + o];
        const float e = live ? (t + a.w[kOffB3 + o]) - a.T[b * 4 + o] : 0.0f;
        l += e * e;
        dy[o] = 2.0f * e / (4.0f * static_cast<float>(a.B));
        if (g == 0) a.dY[b * 4 + o] = dy[o];
      }
      if (g == 0) a.lossp[b] = l;
      const int64_t tT = b / 256, bT = b % 256;  // T-layout tile and column of this sample
      if (ok) {
        for (int cc = 0; cc < 2; ++cc) {
          const int c = 2 * g + cc;
          float v[32];
          tmem_ld32(lane_base + c * 32, v);
#pragma unroll
          for (int gr = 0; gr < 4; ++gr) {
            uint32_t hb[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const int col = c * 32 + gr * 8 + e;
              float dh = 0.f;
#pragma unroll
              for (int o = 0; o < 4; ++o) dh = __fmaf_rn(dy[o], sW3[o * kMlpH + col], dh);
              const float dz = dh * gelu_grad_f(v[gr * 8 + e] + sb2[col]);
              a.dZ2f[static_cast<int64_t>(col) * a.Bp + b] = dz;
              const __nv_bfloat16 qz = __float2bfloat16_rn(dz);
              hb[e] = __bfloat16_as_ushort(qz);
              a.dZ2T[tT * (kMlpH * 256) + mlp_packed_index(col, static_cast<int>(bT))] = qz;
            }
            uint4 pk;
            pk.x = hb[0] | (hb[1] << 16);
            pk.y = hb[2] | (hb[3] << 16);
            pk.z = hb[4] | (hb[5] << 16);
            pk.w = hb[6] | (hb[7] << 16);
            *reinterpret_cast<uint4*>(a.dZ2R + (b / kMlpM) * (kMlpM * kMlpH) +
                                      mlp_packed_index(r, c * 32 + gr * 8)) = pk;
          }
        }
      }
    } else if (ok && MODE == kTrBwd) {
      const int64_t b = static_cast<int64_t>(blockIdx.x) * kMlpM + r;
      float x[8];
#pragma unroll
      for (int d = 0; d < 8; ++d) x[d] = b < a.B ? a.X[b * 8 + d] : 0.0f;
      for (int cc = 0; cc < 2; ++cc) {
        const int c = 2 * g + cc;
        float v[32];
        tmem_ld32(lane_base + c * 32, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int col = c * 32 + i;
          float z = sW3[8 * kMlpH + col];  // Z1 as layer 1 forms it
#pragma unroll
          for (int d = 0; d < 8; ++d) z = __fmaf_rn(sW3[col * 8 + d], x[d], z);
          a.dZ1[static_cast<int64_t>(col) * a.Bp + b] = v[i] * gelu_grad_f(z);
        }
      }
    } else if (ok && MODE == kTrGw2) {
      const int64_t n = static_cast<int64_t>(blockIdx.x) * kMlpM + r;
      float* out = a.gW2p + static_cast<int64_t>(blockIdx.y) * kMlpH * kMlpH + n * kMlpH;
      for (int cc = 0; cc < 2; ++cc) {
        const int c = 2 * g + cc;
        float v[32];
        tmem_ld32(lane_base + c * 32, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) out[c * 32 + i] = v[i];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kMlpEpiWarps + 1) tmem_dealloc(tmem, kMlpH);
}

// layer 1 of a training step: H1 = gelu(X W1^T + b1) as bf16 in both
// layouts, one thread per (sample, 8 features); rows past B (padding) are zero
__global__ void k_tr_l1(const float* __restrict__ X, int B, int Bp,
                        const __nv_bfloat16* __restrict__ wb, const float* __restrict__ w,
                        __nv_bfloat16* __restrict__ H1R, __nv_bfloat16* __restrict__ H1T) {
  const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= static_cast<int64_t>(Bp) * (kMlpH / 8)) return;
  // consecutive threads take consecutive samples of one feature chunk
  const int b = static_cast<int>(idx % Bp), c = static_cast<int>(idx / Bp);
  float x[8];
#pragma unroll
  for (int d = 0; d < 8; ++d) x[d] = b < B ? X[b * 8 + d] : 0.0f;
  const int tR = b / kMlpM, rR = b % kMlpM, tT = b / 256, bT = b % 256;
  uint32_t hb[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int o = 8 * c + e;
    float z = w[kOffB1 + o];
#pragma unroll
    for (int k = 0; k < 8; ++k) z = __fmaf_rn(__bfloat162float(wb[kOffW1 + o * 8 + k]), x[k], z);
    const __nv_bfloat16 q = __float2bfloat16_rn(b < B ? gelu_f(z) : 0.0f);
    hb[e] = __bfloat16_as_ushort(q);
    H1T[static_cast<int64_t>(tT) * (kMlpH * 256) + mlp_packed_index(o, bT)] = q;
  }
  uint4 v;
  v.x = hb[0] | (hb[1] << 16);
  v.y = hb[2] | (hb[3] << 16);
  v.z = hb[4] | (hb[5] << 16);
  v.w = hb[6] | (hb[7] << 16);
  *reinterpret_cast<uint4*>(H1R + static_cast<int64_t>(tR) * (kMlpM * kMlpH) +
                            mlp_packed_index(rR, 8 * c)) = v;
}

// W2^T (bf16) as the B operand of dH1 = dZ2 W2: rows = input feature k, K = output o
__global__ void k_mlp_pack_w2t(const __nv_bfloat16* __restrict__ wb, __nv_bfloat16* __restrict__ Wpk) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kMlpH * kMlpH) return;
  const int o = idx / kMlpH, k = idx % kMlpH;
  Wpk[mlp_packed_index(k, o)] = wb[kOffW2 + o * kMlpH + k];
}

int mlp_train_prepare() {
  ABC_CUDA_TRY(cudaFuncSetAttribute(k_mlp_train_tc<kTrFwd>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(kMlpSmem)));
  ABC_CUDA_TRY(cudaFuncSetAttribute(k_mlp_train_tc<kTrBwd>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(kMlpSmem)));
  ABC_CUDA_TRY(cudaFuncSetAttribute(k_mlp_train_tc<kTrGw2>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(kMlpSmem)));
  return ABC_OK;
}

// Gradient reductions over the (padded) batch, each output summed by one
// block in a fixed order (deterministic).  Layer 3 and layer 2's bias: block
// k < 256 forms gW3[o][k] = sum_b dY[b][o] H2[k][b] and gb2[k] = sum_b
// dZ2[k][b]; block 256 forms gb3[o] = sum_b dY[b][o] and the loss sum.
__global__ void __launch_bounds__(256)
k_red_l3(const float* __restrict__ dY, const float* __restrict__ H2T,
         const float* __restrict__ dZ2T, const float* __restrict__ lossp, int Bp,
         float* __restrict__ grad, float* __restrict__ loss_dev) {
  __shared__ float sm[32];
  const int k = blockIdx.x;
  if (k < kMlpH) {
    float g[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    const float* h = H2T + static_cast<int64_t>(k) * Bp;
    const float* z = dZ2T + static_cast<int64_t>(k) * Bp;
    for (int b = threadIdx.x; b < Bp; b += blockDim.x) {
      const float4 dy = *reinterpret_cast<const float4*>(dY + b * 4);
      const float hv = h[b];
      g[0] = __fmaf_rn(dy.x, hv, g[0]);
      g[1] = __fmaf_rn(dy.y, hv, g[1]);
      g[2] = __fmaf_rn(dy.z, hv, g[2]);
      g[3] = __fmaf_rn(dy.w, hv, g[3]);
      g[4] += z[b];
    }
#pragma unroll
    for (int o = 0; o < 5; ++o) {
      const float t = block_sum<float>(g[o], sm);
      if (threadIdx.x == 0) {
        if (o < 4) grad[kOffW3 + o * kMlpH + k] = t;
        else grad[kOffB2 + k] = t;
      }
    }
  } else {
    float g[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (int b = threadIdx.x; b < Bp; b += blockDim.x) {
      const float4 dy = *reinterpret_cast<const float4*>(dY + b * 4);
      g[0] += dy.x;
      g[1] += dy.y;
      g[2] += dy.z;
      g[3] += dy.w;
      g[4] += lossp[b];
    }
#pragma unroll
    for (int o = 0; o < 5; ++o) {
      const float t = block_sum<float>(g[o], sm);
      if (threadIdx.x == 0) {
        if (o < 4) grad[kOffB3 + o] = t;
        else *loss_dev = t;
      }
    }
  }
}

// Layer 1: block o forms gW1[o][k] = sum_b dZ1[o][b] X[b][k] (b < B) and
// gb1[o] = sum_b dZ1[o][b].
__global__ void __launch_bounds__(256)
k_red_l1(const float* __restrict__ dZ1T, const float* __restrict__ X, int B, int Bp,
         float* __restrict__ grad) {
  __shared__ float sm[32];
  const int o = blockIdx.x;
  float g[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const float* z = dZ1T + static_cast<int64_t>(o) * Bp;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const float zv = z[b];
#pragma unroll
    for (int k = 0; k < 8; ++k) g[k] = __fmaf_rn(zv, X[b * 8 + k], g[k]);  // X: caller's buffer
    g[8] += zv;
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const float t = block_sum<float>(g[k], sm);
    if (threadIdx.x == 0) {
      if (k < 8) grad[kOffW1 + o * 8 + k] = t;
      else grad[kOffB1 + o] = t;
    }
  }
}

// scratch of one training step on B samples (padded to Bp, a multiple of 256)
struct TrLayout {
  size_t H2, dZ2f, dZ1, dY, lossp, gW2p, H1R, H1T, dZ2R, dZ2T, W2pk, W2Tpk, err, total;
};

static TrLayout tr_layout(int B) {
  const size_t Bp = static_cast<size_t>(ceil_div(std::max(B, 1), 256)) * 256;
  const size_t BH = Bp * kMlpH;
  TrLayout l{};
  size_t o = 0;
  auto take = [&](size_t& f, size_t bytes) {
    f = o;
    o += align256(bytes);
  };
  take(l.H2, 4 * BH);
  take(l.dZ2f, 4 * BH);
  take(l.dZ1, 4 * BH);
  take(l.dY, 4 * 4 * Bp);
  take(l.lossp, 4 * Bp);
  take(l.gW2p, 4 * (Bp / 256) * kMlpH * kMlpH);
  take(l.H1R, 2 * BH);
  take(l.H1T, 2 * BH);
  take(l.dZ2R, 2 * BH);
  take(l.dZ2T, 2 * BH);
  take(l.W2pk, 2 * kMlpH * kMlpH);
  take(l.W2Tpk, 2 * kMlpH * kMlpH);
  take(l.err, 16);
  l.total = o + 1024;
  return l;
}

size_t mlp_train_scratch_bytes(int B) { return tr_layout(B).total; }

// One forward + backward pass on X [B][8], T [B][4] (standardised targets).
// The three 256-wide products run on tcgen05 with bf16 operands (weights,
// H1 and dZ2 rounded to bf16) and fp32 accumulation; layers 1 and 3 and the
// bias sums on CUDA cores in fp32.  Writes the gradients into
// grad[kMlpParams] and the sum of squared errors into *loss_dev; a
// tensor-core wait that timed out sets *err (nullable: the scratch's own).
int mlp_grad(const MlpState& s, const float* X, const float* T, int B, float* grad,
             float* loss_dev, void* scratch, size_t bytes, cudaStream_t st, unsigned* err) {
  if (B <= 0) return ABC_E_INVAL;
  const TrLayout l = tr_layout(B);
  if (bytes < l.total) return ABC_E_SCRATCH;
  char* c = static_cast<char*>(scratch);
  const int Bp = static_cast<int>(ceil_div(B, 256) * 256);
  float* H2 = reinterpret_cast<float*>(c + l.H2);
  float* dZ2f = reinterpret_cast<float*>(c + l.dZ2f);
  float* dZ1 = reinterpret_cast<float*>(c + l.dZ1);
  float* dY = reinterpret_cast<float*>(c + l.dY);
  float* lossp = reinterpret_cast<float*>(c + l.lossp);
  float* gW2p = reinterpret_cast<float*>(c + l.gW2p);
  auto* H1R = reinterpret_cast<__nv_bfloat16*>(c + l.H1R);
  auto* H1T = reinterpret_cast<__nv_bfloat16*>(c + l.H1T);
  auto* dZ2R = reinterpret_cast<__nv_bfloat16*>(c + l.dZ2R);
  auto* dZ2T = reinterpret_cast<__nv_bfloat16*>(c + l.dZ2T);
  auto* W2pk = reinterpret_cast<__nv_bfloat16*>(c + l.W2pk);
  auto* W2Tpk = reinterpret_cast<__nv_bfloat16*>(c + l.W2Tpk);
  if (!err) {
    err = reinterpret_cast<unsigned*>(c + l.err);
    ABC_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(unsigned), st));
  }
  const __nv_bfloat16* wb = s.wb;
  k_tr_l1<<<static_cast<unsigned>(Bp / 8), 256, 0, st>>>(X, B, Bp, wb, s.w, H1R, H1T);
  ABC_LAUNCH_CHECK();
  k_mlp_pack_w2<<<(kMlpH * kMlpH + 255) / 256, 256, 0, st>>>(wb, W2pk);
  ABC_LAUNCH_CHECK();
  k_mlp_pack_w2t<<<(kMlpH * kMlpH + 255) / 256, 256, 0, st>>>(wb, W2Tpk);
  ABC_LAUNCH_CHECK();
  TrArgs a{};
  a.B = B;
  a.Bp = Bp;
  a.w = s.w;
  a.wb = wb;
  a.T = T;
  a.H2 = H2;
  a.dY = dY;
  a.lossp = lossp;
  a.dZ2f = dZ2f;
  a.dZ2R = dZ2R;
  a.dZ2T = dZ2T;
  a.X = X;
  a.dZ1 = dZ1;
  a.gW2p = gW2p;
  // forward through layers 2 and 3, loss, back through layer 3
  k_mlp_train_tc<kTrFwd><<<static_cast<unsigned>(Bp / kMlpM), kMlpThreads, kMlpSmem, st>>>(
      reinterpret_cast<const uint8_t*>(H1R), reinterpret_cast<const uint8_t*>(W2pk), a, err);
  ABC_LAUNCH_CHECK();
  // layer 3 and the layer-2 bias, the loss
  k_red_l3<<<kMlpH + 1, 256, 0, st>>>(dY, H2, dZ2f, lossp, Bp, grad, loss_dev);
  ABC_LAUNCH_CHECK();
  // dZ1 = (dZ2 W2) gelu'(Z1)
  k_mlp_train_tc<kTrBwd><<<static_cast<unsigned>(Bp / kMlpM), kMlpThreads, kMlpSmem, st>>>(
      reinterpret_cast<const uint8_t*>(dZ2R), reinterpret_cast<const uint8_t*>(W2Tpk), a, err);
  ABC_LAUNCH_CHECK();
  // gW2 = dZ2^T H1: one partial per 256-sample tile, summed in tile order
  k_mlp_train_tc<kTrGw2><<<dim3(2, static_cast<unsigned>(Bp / 256)), kMlpThreads, kMlpSmem,
                          st>>>(
      reinterpret_cast<const uint8_t*>(dZ2T), reinterpret_cast<const uint8_t*>(H1T), a, err);
  ABC_LAUNCH_CHECK();
  {
    const int64_t n = static_cast<int64_t>(kMlpH) * kMlpH;
    k_splitk_sum<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(gW2p, Bp / 256, n,
                                                                        grad + kOffW2);
    ABC_LAUNCH_CHECK();
  }
  // layer 1 and its bias
  k_red_l1<<<kMlpH, 256, 0, st>>>(dZ1, X, B, Bp, grad);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

// the scratch's own error word of mlp_grad(B)
unsigned* mlp_grad_err(void* scratch, int B) {
  return reinterpret_cast<unsigned*>(static_cast<char*>(scratch) + tr_layout(B).err);
}

// ---- screening (delayed acceptance) ---------------------------------------------
// For each proposal with pflag 0: y0 = mean + std * Y[i][0] predicts log1p d;
// rho = clamp(1 / (1 + exp(-(log1p eps - y0) / tau)), rho_min, 1) in fp32
// with the library's own exp and log1p (every step correctly rounded, so the
// decision is reproducible off the device); simulated and acceptable when
// U < rho (SCREEN stream), else simulated for the audit with probability
// audit_frac (AUDIT stream) and never accepted.
// sflag: 0 acceptable, 1 exhausted (not simulated), 2 audit only, 3 screened out
__device__ __forceinline__ float screen_rho(float y, const float* ystat, float le, float tau,
                                            float rho_min) {
  const float y0 = __fadd_rn(ystat[0], __fmul_rn(ystat[4], y));
  const float z = __fdiv_rn(__fsub_rn(le, y0), tau);
  const float r = __fdiv_rn(1.0f, __fadd_rn(1.0f, dev_exp(-z)));
  return fminf(fmaxf(r, rho_min), 1.0f);  // a NaN prediction gets rho_min
}

// c1_dev (nullable): the counter word read on the device (graph launches);
// on_dev (nullable): 0 there means no screening yet (every proposal passes
// with rho = 1 and no uniform is drawn), as before the surrogate is trained
__global__ void k_screen(const float* __restrict__ Y, const float* __restrict__ ystat,
                         const uint8_t* __restrict__ pflag, int64_t M, const double* eps_p,
                         uint32_t k0, uint32_t k1, uint32_t c1, float tau, float rho_min,
                         float audit_frac, float* __restrict__ rho, uint8_t* __restrict__ sflag,
                         unsigned long long* __restrict__ exhausted,
                         const uint32_t* __restrict__ c1_dev, const int* __restrict__ on_dev) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool ex = i < M && pflag && pflag[i];
  if (exhausted) {
    const unsigned nx = __popc(__ballot_sync(0xffffffffu, ex));
    if ((threadIdx.x & 31) == 0 && nx) atomicAdd(exhausted, static_cast<unsigned long long>(nx));
  }
  if (i >= M) return;
  if (ex) {
    sflag[i] = 1;
    rho[i] = 1.0f;
    return;
  }
  if (on_dev && !*on_dev) {
    sflag[i] = 0;
    rho[i] = 1.0f;
    return;
  }
  if (c1_dev) c1 = *c1_dev;
  const float le = dev_log1p(__double2float_rn(*eps_p));
  const float r = screen_rho(Y[i * 4], ystat, le, tau, rho_min);
  rho[i] = r;
  const float u1 = unif(philox4x32_10(static_cast<uint32_t>(i), c1, 0u, kTagScreen, k0, k1).x);
  if (u1 < r) {
    sflag[i] = 0;
    return;
  }
  const float u2 = unif(philox4x32_10(static_cast<uint32_t>(i), c1, 0u, kTagAudit, k0, k1).x);
  sflag[i] = u2 < audit_frac ? 2 : 3;
}

int screen(const float* Y, const float* ystat, const uint8_t* pflag, int64_t M, const double* eps,
           uint32_t k0, uint32_t k1, uint32_t c1, float tau, float rho_min, float audit_frac,
           float* rho, uint8_t* sflag, cudaStream_t st, unsigned long long* exhausted,
           const uint32_t* c1_dev, const int* on_dev) {
  if (M <= 0) return ABC_OK;
  k_screen<<<static_cast<unsigned>(ceil_div(M, 256)), 256, 0, st>>>(Y, ystat, pflag, M, eps, k0, k1,
                                                                     c1, tau, rho_min, audit_frac,
                                                                     rho, sflag, exhausted, c1_dev,
                                                                     on_dev);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

// compaction of the simulated slots (sflag 0 or 2), in slot order
constexpr int kCTile = 1024;

__global__ void k_cmp_count(const uint8_t* __restrict__ sflag, int64_t M, int* __restrict__ cnt) {
  __shared__ int sm[32];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kCTile + 4 * threadIdx.x;
  int c = 0;
#pragma unroll
  for (int e = 0; e < 4; ++e) c += (base + e < M && (sflag[base + e] == 0 || sflag[base + e] == 2));
  c = block_sum<int>(c, sm);
  if (threadIdx.x == 0) cnt[blockIdx.x] = c;
}

__global__ void k_cmp_scan(const int* __restrict__ cnt, int ntiles, int* __restrict__ off,
                           int* __restrict__ total, long long* __restrict__ acc = nullptr) {
  __shared__ int sm[32];
  __shared__ int last;
  int carry = 0;
  for (int b = 0; b < ntiles; b += blockDim.x) {
    const int i = b + threadIdx.x;
    const int v = i < ntiles ? cnt[i] : 0;
    const int inc = block_incl_scan<int>(v, sm);
    if (i < ntiles) off[i] = carry + inc - v;
    if (threadIdx.x == blockDim.x - 1) last = inc;
    __syncthreads();
    carry += last;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *total = carry;
    if (acc) *acc += carry;  // running count over the generation's batches
  }
}

__global__ void k_cmp_scatter(const uint8_t* __restrict__ sflag, int64_t M, const int* __restrict__ off,
                              const float* __restrict__ up, const float* __restrict__ sp,
                              const int32_t* __restrict__ ap, const float* __restrict__ rho,
                              float* __restrict__ cu, float* __restrict__ cs,
                              int32_t* __restrict__ ca, float* __restrict__ crho,
                              uint8_t* __restrict__ cflag, uint32_t* __restrict__ cslot,
                              int64_t stride) {
  __shared__ int sm[32];
  // the compacted list is [8][stride] (stride = the batch size M, so that the
  // consumers -- simulator, acceptance, training ring -- take n = M with the
  // count Mc on the device)
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kCTile + 4 * threadIdx.x;
  bool keep[4];
  int c = 0;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    keep[e] = base + e < M && (sflag[base + e] == 0 || sflag[base + e] == 2);
    c += keep[e];
  }
  const int inc = block_incl_scan<int>(c, sm);
  int64_t pos = off[blockIdx.x] + inc - c;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if (!keep[e]) continue;
    const int64_t i = base + e;
#pragma unroll
    for (int d = 0; d < 8; ++d) cu[d * stride + pos] = up[d * M + i];
    cs[pos] = sp[i];
    ca[pos] = ap[i];
    crho[pos] = rho[i];
    cflag[pos] = sflag[i];
    cslot[pos] = static_cast<uint32_t>(i);
    ++pos;
  }
}

int screen_and_compact(const float* Y, const float* ystat, const uint8_t* pflag, int64_t M,
                       const double* eps, uint32_t k0, uint32_t k1, uint32_t c1, float tau,
                       float rho_min, float audit_frac, float* rho, uint8_t* sflag,
                       const float* up, const float* sp, const int32_t* ap, float* cu, float* cs,
                       int32_t* ca, float* crho, uint8_t* cflag, uint32_t* cslot, int* Mc_dev,
                       void* scratch, cudaStream_t st, unsigned long long* exhausted,
                       const uint32_t* c1_dev, const int* on_dev, long long* sim_acc) {
  const int64_t nt = ceil_div(M, kCTile);
  int* cnt = static_cast<int*>(scratch);
  int* off = cnt + align256(4 * nt) / 4;
  int rc = screen(Y, ystat, pflag, M, eps, k0, k1, c1, tau, rho_min, audit_frac, rho, sflag, st,
                  exhausted, c1_dev, on_dev);
  if (rc) return rc;
  k_cmp_count<<<static_cast<unsigned>(nt), 256, 0, st>>>(sflag, M, cnt);
  ABC_LAUNCH_CHECK();
  k_cmp_scan<<<1, 1024, 0, st>>>(cnt, static_cast<int>(nt), off, Mc_dev, sim_acc);
  ABC_LAUNCH_CHECK();
  k_cmp_scatter<<<static_cast<unsigned>(nt), 256, 0, st>>>(sflag, M, off, up, sp, ap, rho, cu, cs, ca,
                                                           crho, cflag, cslot, M);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

size_t screen_scratch_bytes(int64_t M) { return 2 * align256(4 * ceil_div(std::max<int64_t>(M, 1), kCTile)); }

// ---- training data ring ----------------------------------------------------------
// Appends n simulated samples (u [8][n] stride n, d, final A, R, D [3][n])
// as x = u and y = [log1p d, log1p A_T, log1p R_T, log1p D_T] at ring
// positions (*head + i) mod cap; valid (nullable) selects samples in order.
__global__ void k_ring_count(const uint8_t* __restrict__ invalid, int64_t n,
                             const int* __restrict__ n_dev, int* __restrict__ cnt) {
  __shared__ int sm[32];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kCTile + 4 * threadIdx.x;
  const int64_t lim = n_dev ? static_cast<int64_t>(*n_dev) : n;
  int c = 0;
#pragma unroll
  for (int e = 0; e < 4; ++e)
    c += (base + e < n && base + e < lim && (!invalid || invalid[base + e] == 0));
  c = block_sum<int>(c, sm);
  if (threadIdx.x == 0) cnt[blockIdx.x] = c;
}

__global__ void k_ring_put(const uint8_t* __restrict__ invalid, int64_t n,
                           const int* __restrict__ n_dev, const int* __restrict__ off,
                           const float* __restrict__ u, const double* __restrict__ d,
                           const int32_t* __restrict__ ard, const long long* __restrict__ head,
                           int64_t cap, float* __restrict__ RX, float* __restrict__ RY) {
  __shared__ int sm[32];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kCTile + 4 * threadIdx.x;
  const int64_t lim = n_dev ? static_cast<int64_t>(*n_dev) : n;
  bool keep[4];
  int c = 0;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    keep[e] = base + e < n && base + e < lim && (!invalid || invalid[base + e] == 0);
    c += keep[e];
  }
  const int inc = block_incl_scan<int>(c, sm);
  int64_t pos = off[blockIdx.x] + inc - c;
  const long long h = *head;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if (!keep[e]) continue;
    const int64_t i = base + e;
    const int64_t r = (h + pos) % cap;
#pragma unroll
    for (int k = 0; k < 8; ++k) RX[r * 8 + k] = u[k * n + i];
    RY[r * 4 + 0] = static_cast<float>(log1p(d[i]));
    RY[r * 4 + 1] = log1pf(static_cast<float>(ard[0 * n + i]));
    RY[r * 4 + 2] = log1pf(static_cast<float>(ard[1 * n + i]));
    RY[r * 4 + 3] = log1pf(static_cast<float>(ard[2 * n + i]));
    ++pos;
  }
}

__global__ void k_ring_advance(long long* head, const int* added) { *head += *added; }

int ring_append(const uint8_t* invalid, int64_t n, const float* u, const double* d,
                const int32_t* ard, long long* head, int64_t cap, float* RX, float* RY,
                void* scratch, cudaStream_t st, const int* n_dev) {
  if (n <= 0) return ABC_OK;
  const int64_t nt = ceil_div(n, kCTile);
  int* cnt = static_cast<int*>(scratch);
  int* off = cnt + align256(4 * nt) / 4;
  int* added = off + align256(4 * nt) / 4;
  k_ring_count<<<static_cast<unsigned>(nt), 256, 0, st>>>(invalid, n, n_dev, cnt);
  ABC_LAUNCH_CHECK();
  k_cmp_scan<<<1, 1024, 0, st>>>(cnt, static_cast<int>(nt), off, added);
  ABC_LAUNCH_CHECK();
  k_ring_put<<<static_cast<unsigned>(nt), 256, 0, st>>>(invalid, n, n_dev, off, u, d, ard, head, cap,
                                                        RX, RY);
  ABC_LAUNCH_CHECK();
  k_ring_advance<<<1, 1, 0, st>>>(head, added);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

size_t ring_scratch_bytes(int64_t n) { return 3 * align256(4 * ceil_div(std::max<int64_t>(n, 1), kCTile)); }

// mean and standard deviation over the filled ring (fp64): each thread sums
// whole samples (4 outputs, 8 inputs), the blocks write partial sums, and one
// warp adds them in block order (deterministic).  Outputs: ystat[o],
// ystat[4 + o]; inputs: ystat[8 + d], ystat[16 + d], standard deviations
// floored at 1e-6 so that a collapsed population keeps finite standardised
// inputs.
constexpr int kStatBlocks = 256;

__global__ void __launch_bounds__(256)
k_ring_stats_part(const float* __restrict__ RX, const float* __restrict__ RY,
                  const long long* __restrict__ head, int64_t cap, double* __restrict__ part) {
  __shared__ double sm[32];
  const int64_t m = *head < cap ? *head : cap;
  double s1[12], s2[12];
#pragma unroll
  for (int j = 0; j < 12; ++j) s1[j] = s2[j] = 0.0;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < m;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float4 y = *reinterpret_cast<const float4*>(RY + i * 4);
    const float4 x0 = *reinterpret_cast<const float4*>(RX + i * 8);
    const float4 x1 = *reinterpret_cast<const float4*>(RX + i * 8 + 4);
    const float v[12] = {y.x, y.y, y.z, y.w, x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
    for (int j = 0; j < 12; ++j) {
      const double d = v[j];
      s1[j] += d;
      s2[j] += d * d;
    }
  }
#pragma unroll
  for (int j = 0; j < 12; ++j) {
    const double a = block_sum<double>(s1[j], sm);
    const double b = block_sum<double>(s2[j], sm);
    if (threadIdx.x == 0) {
      part[blockIdx.x * 24 + j] = a;
      part[blockIdx.x * 24 + 12 + j] = b;
    }
  }
}

__global__ void k_ring_stats_final(const double* __restrict__ part, int nblk,
                                   const long long* __restrict__ head, int64_t cap,
                                   float* __restrict__ ystat) {
  const int j = threadIdx.x;
  if (j >= 12) return;
  const int64_t m = *head < cap ? *head : cap;
  double s1 = 0.0, s2 = 0.0;
  for (int b = 0; b < nblk; ++b) {
    s1 += part[b * 24 + j];
    s2 += part[b * 24 + 12 + j];
  }
  const double mean = m > 0 ? s1 / static_cast<double>(m) : 0.0;
  const double var = m > 1 ? s2 / static_cast<double>(m) - mean * mean : 1.0;
  if (j < 4) {
    ystat[j] = static_cast<float>(mean);
    ystat[4 + j] = static_cast<float>(var > 1e-12 ? sqrt(var) : 1.0);
  } else {
    ystat[8 + (j - 4)] = static_cast<float>(mean);
    ystat[16 + (j - 4)] = static_cast<float>(fmax(var > 0.0 ? sqrt(var) : 1.0, 1e-6));
  }
}

size_t ring_stats_scratch_bytes() { return align256(sizeof(double) * 24 * kStatBlocks); }

// a minibatch of B samples drawn uniformly from the filled ring (TRAIN stream)
__global__ void k_ring_batch(const float* __restrict__ RX, const float* __restrict__ RY,
                             const long long* __restrict__ head, int64_t cap,
                             const float* __restrict__ ystat, int B, uint32_t step, uint32_t k0,
                             uint32_t k1, float* __restrict__ X, float* __restrict__ T,
                             const uint32_t* __restrict__ step_dev) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B) return;
  if (step_dev) step += *step_dev;  // the run's Adam steps so far (device counter)
  const int64_t m = *head < cap ? *head : cap;
  const u32x4 r = philox4x32_10(static_cast<uint32_t>(i), step, 0u, kTagTrain, k0, k1);
  const uint64_t U = (static_cast<uint64_t>(r.y) << 32) | r.x;
  const int64_t src = m > 0 ? static_cast<int64_t>(__umul64hi(U, static_cast<uint64_t>(m))) : 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) X[i * 8 + k] = (RX[src * 8 + k] - ystat[8 + k]) / ystat[16 + k];
#pragma unroll
  for (int o = 0; o < 4; ++o) T[i * 4 + o] = (RY[src * 4 + o] - ystat[o]) / ystat[4 + o];
}

__global__ void k_step_advance(uint32_t* step_dev, uint32_t steps, const int* off_dev) {
  if (!(off_dev && *off_dev)) *step_dev += steps;
}

// `steps` Adam steps on minibatches of the ring; the step count lives on the
// device (*step_dev, advanced here), so the sequence is the same whether the
// host loop runs once per generation or is captured in a graph
int mlp_train(const MlpState& s, const float* RX, const float* RY, const long long* head,
              int64_t cap, const float* ystat, int B, int steps, uint32_t* step_dev, float lr,
              uint32_t k0, uint32_t k1, float* grad, float* X, float* T, float* loss_dev,
              void* scratch, size_t bytes, cudaStream_t st, const int* off_dev, unsigned* err) {
  int rc;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const unsigned g = (kMlpParams + 255) / 256;
  for (int k = 0; k < steps; ++k) {
    k_ring_batch<<<(B + 255) / 256, 256, 0, st>>>(RX, RY, head, cap, ystat, B,
                                                  static_cast<uint32_t>(k), k0, k1, X, T, step_dev);
    ABC_LAUNCH_CHECK();
    if ((rc = mlp_grad(s, X, T, B, grad, loss_dev, scratch, bytes, st, err))) return rc;
    k_adam<<<g, 256, 0, st>>>(s.w, grad, s.m, s.v, lr, b1, b2, eps, 1.0f, 1.0f, step_dev,
                              static_cast<uint32_t>(k));
    ABC_LAUNCH_CHECK();
    k_mlp_to_bf16<<<g, 256, 0, st>>>(s.w, s.wb);
    ABC_LAUNCH_CHECK();
  }
  k_step_advance<<<1, 1, 0, st>>>(step_dev, static_cast<uint32_t>(steps), off_dev);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

// screening from the generation `start` on once the surrogate has been
// trained: *on = t >= start && *step_dev > 0 (t from t_dev when given)
__global__ void k_sur_gate(const uint32_t* t_dev, uint32_t t, int start,
                           const uint32_t* step_dev, int* on) {
  if (t_dev) t = *t_dev;
  *on = (t >= static_cast<uint32_t>(start) && *step_dev > 0u) ? 1 : 0;
}

int sur_gate(const uint32_t* t_dev, uint32_t t, int start, const uint32_t* step_dev, int* on,
             cudaStream_t st) {
  k_sur_gate<<<1, 1, 0, st>>>(t_dev, t, start, step_dev, on);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

// audited (cflag 2) and audited-with-d<=eps counts over the compacted list
__global__ void k_audit_count(const uint8_t* __restrict__ cflag, const double* __restrict__ cd,
                              const int* __restrict__ Mc, const double* __restrict__ eps_p,
                              unsigned long long* __restrict__ counts) {
  const double eps = *eps_p;
  const int m = *Mc;
  unsigned long long a = 0, b = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    if (cflag[i] == 2) {
      ++a;
      b += cd[i] <= eps;
    }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0 && (a || b)) {
    atomicAdd(&counts[0], a);
    atomicAdd(&counts[1], b);
  }
}

int audit_count(const uint8_t* cflag, const double* cd, const int* Mc, const double* eps,
                unsigned long long* counts, cudaStream_t st) {
  k_audit_count<<<152, 256, 0, st>>>(cflag, cd, Mc, eps, counts);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

// delayed-acceptance correction of importance weights: log W -= log rho
__global__ void k_rho_correct(double* __restrict__ logW, const float* __restrict__ rho, int64_t n,
                              const int* __restrict__ off_dev) {
  if (off_dev && *off_dev) return;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) logW[i] -= log(static_cast<double>(rho[i]));
}

int rho_correct(double* logW, const float* rho, int64_t n, cudaStream_t st, const int* off_dev) {
  k_rho_correct<<<static_cast<unsigned>(ceil_div(n, 256)), 256, 0, st>>>(logW, rho, n, off_dev);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

__global__ void k_stats_init(float* ystat) {
  const int i = threadIdx.x;
  if (i < 24) ystat[i] = ((i >= 4 && i < 8) || i >= 16) ? 1.0f : 0.0f;
}

int stats_init(float* ystat, cudaStream_t st) {
  k_stats_init<<<1, 32, 0, st>>>(ystat);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

int ring_stats(const float* RX, const float* RY, const long long* head, int64_t cap, float* ystat,
               void* scratch, cudaStream_t st) {
  double* part = static_cast<double*>(scratch);
  k_ring_stats_part<<<kStatBlocks, 256, 0, st>>>(RX, RY, head, cap, part);
  ABC_LAUNCH_CHECK();
  k_ring_stats_final<<<1, 32, 0, st>>>(part, kStatBlocks, head, cap, ystat);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

}  // namespace abc
