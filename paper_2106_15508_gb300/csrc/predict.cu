// predict.cu -- posterior-predictive simulation (Sec. 4.2): the learned
// samples, drawn in proportion to their weights, simulated from day zero
// over the training window and the days ahead; per day and series (A, R, D)
// the order statistics at the requested levels (median and central 99%
// range in the paper's figures).
//
//   1. weights quantised and prefixed like the stage prior (Eq. 10-11):
//      every particle survives (d = 0 <= eps = 0) with r = W, or all q = 1
//      when W is absent;
//   2. R ancestors, U from Philox block (j, 0, 0, PREDICT), first k with
//      prefix_k > floor(U total / 2^64);
//   3. the simulator over `days` days with the PREDICT_SIM stream, full
//      trajectories;
//   4. one block per (day, series, level): radix select (4 passes of 8 bits
//      on the non-negative counts) of the k-th smallest, k = ceil(q R).
#include <algorithm>
#include <cmath>
#include <vector>

#include "batch.cuh"
#include "common.cuh"
#include "numerics.cuh"

namespace abc {

size_t prefix_scratch_bytes(int64_t);

__global__ void k_pred_draw(SimParams p, const float* __restrict__ u, int64_t N,
                            const uint64_t* __restrict__ prefix, int64_t R,
                            float* __restrict__ ur) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= R) return;
  const uint64_t total = prefix[N - 1];
  const u32x4 w = philox4x32_10(static_cast<uint32_t>(j), 0u, 0u, ABC_TAG_PREDICT, p.k0, p.k1);
  const uint64_t U = (static_cast<uint64_t>(w.y) << 32) | w.x;
  const uint64_t x = __umul64hi(U, total);
  int64_t lo = 0, hi = N - 1;
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (prefix[mid] > x) hi = mid;
    else lo = mid + 1;
  }
#pragma unroll
  for (int d = 0; d < 8; ++d) ur[static_cast<int64_t>(d) * R + j] = u[static_cast<int64_t>(d) * N + lo];
}

// out[(t * 3 + c) * nq + i] = k_i-th smallest of traj[t][series c][0..R)
__global__ void __launch_bounds__(256)
k_pred_select(const int32_t* __restrict__ traj, int64_t R, int32_t days,
              const long long* __restrict__ ks, int32_t nq, int32_t* __restrict__ out) {
  __shared__ unsigned hist[256];
  __shared__ unsigned s_digit;
  __shared__ long long s_k;
  const int idx = blockIdx.x;  // (t * 3 + c) * nq + i
  const int i = idx % nq;
  const int tc = idx / nq;
  const int t = tc / 3, c = tc % 3;
  if (t > days) return;
  const int32_t* col = traj + (static_cast<int64_t>(t) * 6 + 2 + c) * R;  // A, R, D
  unsigned want = 0u, mask = 0u;
  if (threadIdx.x == 0) s_k = ks[i];
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0u;
    __syncthreads();
    for (int64_t e = threadIdx.x; e < R; e += blockDim.x) {
      const unsigned v = static_cast<unsigned>(col[e]);
      if ((v & mask) == want) atomicAdd(&hist[(v >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      long long k = s_k, cum = 0;
      unsigned digit = 255u;
      for (unsigned b = 0; b < 256u; ++b) {
        if (cum + hist[b] >= k) {
          digit = b;
          break;
        }
        cum += hist[b];
      }
      s_k = k - cum;
      s_digit = digit;
    }
    __syncthreads();
    want |= s_digit << shift;
    mask |= 255u << shift;
    __syncthreads();
  }
  if (threadIdx.x == 0) out[idx] = static_cast<int32_t>(want);
}

struct PredLayout {
  size_t d0, eps, q, prefix, pscr, ur, traj, dist, ks, total;
};

static PredLayout pred_layout(int64_t N, int64_t R, int32_t days, int32_t nq) {
  PredLayout l{};
  size_t o = 0;
  auto take = [&](size_t& f, size_t bytes) {
    f = o;
    o += align256(bytes);
  };
  take(l.d0, 8 * static_cast<size_t>(N));
  take(l.eps, 8);
  take(l.q, 4 * static_cast<size_t>(N));
  take(l.prefix, 8 * static_cast<size_t>(N));
  take(l.pscr, prefix_scratch_bytes(N));
  take(l.ur, 32 * static_cast<size_t>(R));
  take(l.traj, 4 * static_cast<size_t>(days + 1) * 6 * static_cast<size_t>(R));
  take(l.dist, 8 * static_cast<size_t>(R));
  take(l.ks, 8 * static_cast<size_t>(std::max(nq, 1)));
  l.total = o;
  return l;
}

size_t predict_scratch_bytes(int64_t N, int64_t R, int32_t days, int32_t nq) {
  return pred_layout(N, R, days, nq).total;
}

int launch_predict(const SimParams& p0, const float* u, const double* W, int64_t N, int64_t R,
                   int32_t days, const double* quant, int32_t nq, int32_t* out, void* scratch,
                   size_t bytes, cudaStream_t st) {
  const PredLayout l = pred_layout(N, R, days, nq);
  if (bytes < l.total) return ABC_E_SCRATCH;
  char* b = static_cast<char*>(scratch);
  auto* d0 = reinterpret_cast<double*>(b + l.d0);
  auto* eps = reinterpret_cast<double*>(b + l.eps);
  auto* q = reinterpret_cast<uint32_t*>(b + l.q);
  auto* prefix = reinterpret_cast<uint64_t*>(b + l.prefix);
  auto* ur = reinterpret_cast<float*>(b + l.ur);
  auto* traj = reinterpret_cast<int32_t*>(b + l.traj);
  auto* dist = reinterpret_cast<double*>(b + l.dist);
  auto* ks = reinterpret_cast<long long*>(b + l.ks);
  // ranks k = ceil(q R) clamped to [1, R], computed as the oracle does
  std::vector<long long> kh(static_cast<size_t>(nq));
  for (int i = 0; i < nq; ++i) {
    long long k = static_cast<long long>(std::ceil(quant[i] * static_cast<double>(R)));
    kh[static_cast<size_t>(i)] = std::min<long long>(std::max<long long>(k, 1), R);
  }
  ABC_CUDA_TRY(cudaMemcpyAsync(ks, kh.data(), 8 * kh.size(), cudaMemcpyHostToDevice, st));
  ABC_CUDA_TRY(cudaMemsetAsync(d0, 0, 8 * static_cast<size_t>(N), st));
  ABC_CUDA_TRY(cudaMemsetAsync(eps, 0, 8, st));
  int rc = launch_resample_prefix(d0, W, N, eps, W ? ABC_W_IMPORTANCE : ABC_W_PAPER, q, prefix,
                                  b + l.pscr, l.ur - l.pscr, st);
  if (rc) return rc;
  k_pred_draw<<<static_cast<unsigned>(ceil_div(R, 256)), 256, 0, st>>>(p0, u, N, prefix, R, ur);
  ABC_LAUNCH_CHECK();
  SimParams p = p0;
  p.T = days;
  rc = launch_simulate(p, nullptr, ur, R, nullptr, 0u, ABC_TAG_PREDICT_SIM, nullptr, dist, traj,
                       st);
  if (rc) return rc;
  const int64_t nblocks = static_cast<int64_t>(days + 1) * 3 * nq;
  k_pred_select<<<static_cast<unsigned>(nblocks), 256, 0, st>>>(traj, R, days, ks, nq, out);
  ABC_LAUNCH_CHECK();
  // the host rank vector must outlive the copy
  ABC_CUDA_TRY(cudaStreamSynchronize(st));
  return ABC_OK;
}

}  // namespace abc
