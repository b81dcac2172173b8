// sort.cu -- stable LSD radix sort of 32-bit keys with int32 payloads, 8 bits
// per pass.  Used to put the weight pass's rows and columns in spatial order
// (Morton keys); stability keeps every order, and so every result,
// deterministic.
//
// One pass over n elements in tiles of kRsTile:
//   k_rs_count   per tile, the count of each digit       cnt[digit][tile]
//   k_rs_scan    per digit, exclusive offsets over tiles  (in place) + totals
//   k_rs_base    exclusive offsets of the digits          base[digit]
//   k_rs_scatter element -> base + tile offset + rank among the tile's earlier
//                elements with the same digit (warp match + per-warp counts)
// The element count may live on the device (n_dev); the host size is then a
// capacity, and elements at or beyond *n_dev are left out.
#include "batch.cuh"
#include "common.cuh"

namespace abc {

constexpr int kRsTile = 1024;
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;

__device__ __forceinline__ int64_t rs_count(int64_t cap, const int* n_dev) {
  return n_dev ? static_cast<int64_t>(*n_dev) : cap;
}

__global__ void __launch_bounds__(kRsThreads)
k_rs_count(const uint32_t* __restrict__ keys, int64_t cap, const int* __restrict__ n_dev,
           int shift, int ntiles, int* __restrict__ cnt) {
  __shared__ int h[256];
  const int64_t n = rs_count(cap, n_dev);
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kRsTile;
  for (int e = threadIdx.x; e < kRsTile; e += kRsThreads) {
    const int64_t i = base + e;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
  }
  __syncthreads();
  cnt[static_cast<int64_t>(threadIdx.x) * ntiles + blockIdx.x] = h[threadIdx.x];
}

// one block per digit: exclusive scan of cnt[digit][0..ntiles) in place
__global__ void __launch_bounds__(1024)
k_rs_scan(int* __restrict__ cnt, int ntiles, int* __restrict__ total) {
  __shared__ int sm[32];
  __shared__ int last;
  int* row = cnt + static_cast<int64_t>(blockIdx.x) * ntiles;
  int carry = 0;
  for (int b = 0; b < ntiles; b += blockDim.x) {
    const int i = b + threadIdx.x;
    const int v = i < ntiles ? row[i] : 0;
    const int inc = block_incl_scan<int>(v, sm);
    if (i < ntiles) row[i] = carry + inc - v;
    if (threadIdx.x == blockDim.x - 1) last = inc;
    __syncthreads();
    carry += last;
    __syncthreads();
  }
  if (threadIdx.x == 0) total[blockIdx.x] = carry;
}

__global__ void k_rs_base(const int* __restrict__ total, int* __restrict__ base) {
  __shared__ int sm[32];
  const int v = total[threadIdx.x];
  base[threadIdx.x] = block_incl_scan<int>(v, sm) - v;
}

__global__ void __launch_bounds__(kRsThreads)
k_rs_scatter(const uint32_t* __restrict__ kin, const int32_t* __restrict__ vin, int64_t cap,
             const int* __restrict__ n_dev, int shift, int ntiles, const int* __restrict__ cnt,
             const int* __restrict__ base, uint32_t* __restrict__ kout,
             int32_t* __restrict__ vout) {
  __shared__ int run[256];            // earlier sub-rounds of this tile, per digit
  __shared__ int wc[kRsWarps][256];   // this sub-round, per warp and digit
  const int64_t n = rs_count(cap, n_dev);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  run[threadIdx.x] = 0;
#pragma unroll
  for (int w = 0; w < kRsWarps; ++w) wc[w][threadIdx.x] = 0;
  __syncthreads();
  const int64_t tbase = static_cast<int64_t>(blockIdx.x) * kRsTile;
  for (int r = 0; r < kRsTile / kRsThreads; ++r) {
    // sub-round r: elements tbase + r * 256 + threadIdx.x, in index order
    const int64_t i = tbase + static_cast<int64_t>(r) * kRsThreads + threadIdx.x;
    const bool ok = i < n;
    const uint32_t key = ok ? kin[i] : 0u;
    const int dg = ok ? static_cast<int>((key >> shift) & 255u) : 256;
    const unsigned peers = __match_any_sync(0xffffffffu, dg);
    const int rank = __popc(peers & lt);
    if (ok && rank == 0) wc[warp][dg] = __popc(peers);
    __syncthreads();
    if (ok) {
      int pos = base[dg] + cnt[static_cast<int64_t>(dg) * ntiles + blockIdx.x] + run[dg] + rank;
      for (int w = 0; w < warp; ++w) pos += wc[w][dg];
      kout[pos] = key;
      vout[pos] = vin ? vin[i] : static_cast<int32_t>(i);
    }
    __syncthreads();
    int add = 0;
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) {
      add += wc[w][threadIdx.x];
      wc[w][threadIdx.x] = 0;
    }
    run[threadIdx.x] += add;
    __syncthreads();
  }
}

struct RsLayout {
  size_t cnt, total, base, k1, v1, total_bytes;
};

static RsLayout rs_layout(int64_t cap) {
  RsLayout l{};
  const size_t nt = static_cast<size_t>(ceil_div(std::max<int64_t>(cap, 1), kRsTile));
  size_t o = 0;
  auto take = [&](size_t& f, size_t b) {
    f = o;
    o += align256(b);
  };
  take(l.cnt, 4 * 256 * nt);
  take(l.total, 4 * 256);
  take(l.base, 4 * 256);
  take(l.k1, 4 * static_cast<size_t>(std::max<int64_t>(cap, 1)));
  take(l.v1, 4 * static_cast<size_t>(std::max<int64_t>(cap, 1)));
  l.total_bytes = o;
  return l;
}

size_t radix_sort_scratch_bytes(int64_t cap) { return rs_layout(cap).total_bytes; }

// Sorts the first n (n_dev ? *n_dev : cap) keys of kin, with payload vin
// (NULL: the element indices), by their low `bits` bits into kout / vout.
// kin and vin are not modified.
int launch_radix_sort(const uint32_t* kin, const int32_t* vin, uint32_t* kout, int32_t* vout,
                      int64_t cap, const int* n_dev, int bits, void* scratch, size_t bytes,
                      cudaStream_t st) {
  if (cap <= 0) return ABC_OK;
  if (bits < 1 || bits > 32 || cap > (int64_t(1) << 30)) return ABC_E_INVAL;
  const RsLayout l = rs_layout(cap);
  if (bytes < l.total_bytes) return ABC_E_SCRATCH;
  char* b = static_cast<char*>(scratch);
  int* cnt = reinterpret_cast<int*>(b + l.cnt);
  int* total = reinterpret_cast<int*>(b + l.total);
  int* base = reinterpret_cast<int*>(b + l.base);
  uint32_t* k1 = reinterpret_cast<uint32_t*>(b + l.k1);
  int32_t* v1 = reinterpret_cast<int32_t*>(b + l.v1);
  const int passes = (bits + 7) / 8;
  const int ntiles = static_cast<int>(ceil_div(cap, kRsTile));
  // ping-pong so that the last pass writes kout / vout
  const uint32_t* ki = kin;
  const int32_t* vi = vin;
  for (int p = 0; p < passes; ++p) {
    const bool to_out = ((passes - 1 - p) % 2) == 0;
    uint32_t* ko = to_out ? kout : k1;
    int32_t* vo = to_out ? vout : v1;
    const int shift = 8 * p;
    k_rs_count<<<ntiles, kRsThreads, 0, st>>>(ki, cap, n_dev, shift, ntiles, cnt);
    ABC_LAUNCH_CHECK();
    k_rs_scan<<<256, 1024, 0, st>>>(cnt, ntiles, total);
    ABC_LAUNCH_CHECK();
    k_rs_base<<<1, 256, 0, st>>>(total, base);
    ABC_LAUNCH_CHECK();
    k_rs_scatter<<<ntiles, kRsThreads, 0, st>>>(ki, vi, cap, n_dev, shift, ntiles, cnt, base, ko,
                                                vo);
    ABC_LAUNCH_CHECK();
    ki = ko;
    vi = vo;
  }
  return ABC_OK;
}

}  // namespace abc
