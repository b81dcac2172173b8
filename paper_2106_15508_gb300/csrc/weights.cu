// weights.cu -- A9 importance weights, FP32 CUDA-core path.
//
//   log W_j = 4 ln(2 pi s_j) - ln sum_k (q_k / total) exp(-|u'_j - u_k|^2 / (2 s_j))
//
// over the surviving columns (q_k > 0), compacted beforehand into cu [8][nc]
// and c_k = log2(q_k) - 32 (in [-32, 0), so the dominant terms carry small
// absolute rounding error).  Work is in base 2: e_jk = c_k - D_jk log2(e) /
// (2 s_j), an online row maximum m and a running sum of 2^(e - m).
// Accuracy: D_jk from direct differences (no |a|^2 + |b|^2 - 2ab
// cancellation), formed with packed fp32x2 arithmetic: dimensions (0,2,4,6)
// and (1,3,5,7) accumulate in the two lanes (one product, three fused
// multiply-adds), then one add; each 128-column tile is summed locally and
// folded into the row total with Kahan compensation.  Columns are split into
// chunks over grid.y; a combine kernel merges the (m, S) partials in fp64.  The kernel
// variance is floored at 1e-30 (1/(2s) must stay finite in fp32; such rows
// carry negligible weight).
#include <algorithm>

#include "common.cuh"

namespace abc {

constexpr int kWThreads = 128;  // threads per CTA
constexpr int kWRows = 4;       // rows per thread
constexpr int kWTile = 128;     // columns per shared-memory tile
constexpr float kSMin = 1e-30f; // floor of the kernel variance s_j

// packed fp32x2 arithmetic (two independent IEEE fp32 lanes per instruction)
__device__ __forceinline__ unsigned long long pk2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ float hsum2(unsigned long long a) {
  float lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a));
  return __fadd_rn(lo, hi);
}
// 2^x (ex2.approx.ftz: about 2 ulp; results below 2^-126 flush to zero,
// i.e. terms under 2^-126 of the row maximum are dropped)
__device__ __forceinline__ float ex2f(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__global__ void __launch_bounds__(kWThreads)
k_weights_fp32(const float* __restrict__ up, const float* __restrict__ s, int64_t rows,
               const float* __restrict__ cu, const float* __restrict__ cc,
               const int* __restrict__ nc_p, int64_t ncap,
               float2* __restrict__ part, const int* __restrict__ off_dev,
               const int* __restrict__ rows_dev) {
  // column coordinates as four pairs: su2[h][k] = (u_2h, u_2h+1) of column k
  __shared__ __align__(16) unsigned long long su2[4][kWTile];
  __shared__ float sc[kWTile];
  if (off_dev && *off_dev) return;  // run finished or its generation stopped
  // rows is the stride (capacity); rows_dev, when given, the rows in use
  const int64_t nrows = rows_dev ? static_cast<int64_t>(*rows_dev) : rows;
  const int64_t nc = *nc_p;
  // the columns in use (nc, known only on the device) split evenly over grid.y
  const int64_t chunk_cols = ceil_div(ceil_div(nc, static_cast<int64_t>(gridDim.y)),
                                      static_cast<int64_t>(kWTile)) * kWTile;
  const int64_t c_begin = static_cast<int64_t>(blockIdx.y) * chunk_cols;
  const int64_t c_end = nc < c_begin + chunk_cols ? nc : c_begin + chunk_cols;
  // row blocks of 512 rows, grid-strided (the grid may be smaller than the
  // capacity when the rows in use are counted on the device)
  for (int64_t rb = blockIdx.x; rb * (kWThreads * kWRows) < nrows; rb += gridDim.x) {
  const int64_t row0 = rb * (kWThreads * kWRows) + threadIdx.x;
  unsigned long long x[kWRows][4];
  float ninv[kWRows], m[kWRows], S[kWRows], cS[kWRows], t[kWRows];
#pragma unroll
  for (int r = 0; r < kWRows; ++r) {
    const int64_t j = row0 + r * kWThreads;
    const bool live = j < nrows;
    // kernel variance floored at 1e-30 so that 1/(2 s) stays finite
    const float sj = live ? fmaxf(s[j], kSMin) : 1.0f;
#pragma unroll
    for (int h = 0; h < 4; ++h)
      x[r][h] = pk2(live ? up[static_cast<int64_t>(2 * h) * rows + j] : 0.0f,
                    live ? up[static_cast<int64_t>(2 * h + 1) * rows + j] : 0.0f);
    ninv[r] = -1.4426950408889634f / (2.0f * sj);  // -log2(e) / (2 s_j)
    m[r] = -INFINITY;
    S[r] = 0.0f;
    cS[r] = 0.0f;
    t[r] = 0.0f;
  }
  for (int64_t c0 = c_begin; c0 < c_end; c0 += kWTile) {
    const int cnt = static_cast<int>(c_end - c0 < kWTile ? c_end - c0 : kWTile);
    __syncthreads();
    for (int i = threadIdx.x; i < kWTile; i += kWThreads) {
      const bool in = i < cnt;
#pragma unroll
      for (int h = 0; h < 4; ++h)
        su2[h][i] = pk2(in ? cu[static_cast<int64_t>(2 * h) * ncap + c0 + i] : 0.0f,
                        in ? cu[static_cast<int64_t>(2 * h + 1) * ncap + c0 + i] : 0.0f);
      sc[i] = in ? cc[c0 + i] : -INFINITY;
    }
    __syncthreads();
    for (int k = 0; k < cnt; ++k) {
      unsigned long long uk[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) uk[h] = su2[h][k];
      const float ck = sc[k];
#pragma unroll
      for (int r = 0; r < kWRows; ++r) {
        // lane 0: dimensions 0, 2, 4, 6; lane 1: 1, 3, 5, 7
        const unsigned long long a0 = sub2(x[r][0], uk[0]);
        const unsigned long long a1 = sub2(x[r][1], uk[1]);
        const unsigned long long a2 = sub2(x[r][2], uk[2]);
        const unsigned long long a3 = sub2(x[r][3], uk[3]);
        unsigned long long q = mul2(a0, a0);
        q = fma2(a1, a1, q);
        q = fma2(a2, a2, q);
        q = fma2(a3, a3, q);
        const float D = hsum2(q);
        const float e = __fmaf_rn(D, ninv[r], ck);
        if (e > m[r]) {
          const float f = ex2f(m[r] - e);
          S[r] *= f;
          cS[r] *= f;
          t[r] *= f;
          m[r] = e;
        }
        t[r] += ex2f(e - m[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < kWRows; ++r) {
      const float y = t[r] - cS[r];
      const float tt = S[r] + y;
      cS[r] = (tt - S[r]) - y;
      S[r] = tt;
      t[r] = 0.0f;
    }
  }
#pragma unroll
  for (int r = 0; r < kWRows; ++r) {
    const int64_t j = row0 + r * kWThreads;
    if (j < nrows) part[static_cast<int64_t>(blockIdx.y) * rows + j] = make_float2(m[r], S[r]);
  }
  __syncthreads();  // the shared tiles are refilled for the next row block
  }
}

__global__ void k_weights_combine(const float2* __restrict__ part, int nchunks,
                                  const float* __restrict__ s, int64_t rows,
                                  const uint64_t* __restrict__ total_p, double* __restrict__ logW,
                                  const int* __restrict__ off_dev, const int* __restrict__ rows_dev) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= (rows_dev ? static_cast<int64_t>(*rows_dev) : rows) || (off_dev && *off_dev)) return;
  const double sj = static_cast<double>(fmaxf(s[j], kSMin));
  double M = -INFINITY;
  for (int c = 0; c < nchunks; ++c) M = fmax(M, static_cast<double>(part[static_cast<int64_t>(c) * rows + j].x));
  double S = 0.0;
  for (int c = 0; c < nchunks; ++c) {
    const float2 p = part[static_cast<int64_t>(c) * rows + j];
    if (p.y > 0.0f) S += static_cast<double>(p.y) * exp2(static_cast<double>(p.x) - M);
  }
  // ln sum_k rhat_k exp(.) = ln2 (M + log2 S + 32 - log2 total)
  const double lse = 0.6931471805599453 * (M + log2(S) + 32.0 - log2(static_cast<double>(*total_p)));
  logW[j] = 4.0 * log(6.283185307179586 * sj) - lse;
}

// column chunks: about 16 CTAs per SM in total, times a tuning multiplier
static int weight_chunks(int64_t rows, int64_t ncap, int mult) {
  const int64_t gx = ceil_div(std::max<int64_t>(rows, 1), kWThreads * kWRows);
  const int64_t want = std::max<int64_t>(1, 2432 / gx) * std::max(1, mult);
  const int64_t maxc = std::max<int64_t>(1, ceil_div(ncap, kWTile));
  return static_cast<int>(std::min<int64_t>(want, maxc));
}

size_t weights_fp32_scratch_bytes(int64_t rows, int64_t ncap, int mult) {
  return align256(sizeof(float2) * static_cast<size_t>(weight_chunks(rows, ncap, mult)) * rows);
}

// cu/cc/nc_dev: compacted survivor columns (capacity ncap); total_p: device u64
int launch_weights_fp32(const float* up, const float* s, int64_t rows, const float* cu,
                        const float* cc, const int* nc_dev, int64_t ncap,
                        const uint64_t* total_p, double* logW, void* scratch, size_t bytes,
                        cudaStream_t st, const int* off_dev, int mult, const int* rows_dev,
                        const WeightTiming* wt) {
  if (rows <= 0) return ABC_OK;
  if (bytes < weights_fp32_scratch_bytes(rows, ncap, mult)) return ABC_E_SCRATCH;
  const int nch = weight_chunks(rows, ncap, mult);
  float2* part = static_cast<float2*>(scratch);
  // with a device-side row count the rows in use are often few: a capped,
  // grid-strided grid keeps the launch from spawning thousands of idle CTAs
  int64_t gx = ceil_div(rows, kWThreads * kWRows);
  if (rows_dev) gx = std::min<int64_t>(gx, 304);
  dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(nch));
  if (wt && wt->fp0) ABC_CUDA_TRY(cudaEventRecord(wt->fp0, st));
  k_weights_fp32<<<grid, kWThreads, 0, st>>>(up, s, rows, cu, cc, nc_dev, ncap, part,
                                             off_dev, rows_dev);
  ABC_LAUNCH_CHECK();
  if (wt && wt->fp1) ABC_CUDA_TRY(cudaEventRecord(wt->fp1, st));
  k_weights_combine<<<static_cast<unsigned>(ceil_div(rows, 256)), 256, 0, st>>>(part, nch, s, rows,
                                                                                total_p, logW, off_dev,
                                                                                rows_dev);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

}  // namespace abc
