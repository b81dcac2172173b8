// particles.cu -- the HBM-bound particle passes of one SMC generation:
//   A4 tolerance: radix select of the k-th smallest distance (Eq. 8)
//   A5 stage-prior weights, u32 quantisation and u64 inclusive prefix
//      (Eq. 9-11) with a reduce-then-scan over 1024-element tiles
//   A6-A7 BDSS proposal: categorical ancestor, Beta step, Gaussian walk and
//      support redraw (Eq. 11, 16, 17)
//   A8 acceptance and in-order append (Sec. 2.3, Sec. 4.1)
//   survivor compaction for the weight pass, A10 fp64 normalisation / ESS
// Every reduction runs in a fixed order (block partials, then one block),
// so results never depend on scheduling.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "numerics.cuh"

namespace abc {

constexpr int kTile = 1024;    // elements per scan tile
constexpr int kTileThr = 256;  // threads per tile (4 elements each)

// --------------------------------------------------------------- A4 select -
struct SelState {
  unsigned long long prefix, mask;
  long long k;
};

__global__ void k_sel_init(SelState* st, unsigned* hist, long long k) {
  if (threadIdx.x == 0) *st = SelState{0ull, 0ull, k};
  for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0u;
}

__global__ void k_sel_hist(const double* __restrict__ d, int64_t n, const SelState* st,
                           int shift, unsigned* hist) {
  __shared__ unsigned sh[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) sh[i] = 0u;
  __syncthreads();
  const unsigned long long prefix = st->prefix, mask = st->mask;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const unsigned long long key = static_cast<unsigned long long>(__double_as_longlong(d[i]));
    if ((key & mask) == prefix) atomicAdd(&sh[(key >> shift) & 255ull], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// 256 threads, one per bin: the digit b of the k-th key is the first bin
// whose inclusive count reaches k (bin 255 if bins 0..254 hold fewer than
// k keys); k becomes its rank inside that bin
__global__ void k_sel_pick(SelState* st, unsigned* hist, int shift, double* out) {
  __shared__ unsigned long long sm[32];
  const unsigned long long k = static_cast<unsigned long long>(st->k);
  const unsigned h = hist[threadIdx.x];
  const unsigned long long inc = block_incl_scan<unsigned long long>(h, sm);
  const unsigned long long below = inc - h;
  const bool pick = threadIdx.x < 255 ? (below < k && inc >= k) : below < k;
  if (pick) {
    st->k = static_cast<long long>(k - below);
    st->prefix |= static_cast<unsigned long long>(threadIdx.x) << shift;
    st->mask |= 255ull << shift;
    if (shift == 0) *out = __longlong_as_double(static_cast<long long>(st->prefix));
  }
  hist[threadIdx.x] = 0u;  // every thread read its bin before the scan's barriers
}

size_t select_scratch_bytes(int64_t) { return align256(sizeof(SelState)) + align256(256 * 4); }

int launch_select(const double* d, int64_t n, int64_t k, double* out, void* scratch,
                  size_t bytes, cudaStream_t st) {
  if (n <= 0 || k < 1 || k > n) return ABC_E_INVAL;
  if (bytes < select_scratch_bytes(n)) return ABC_E_SCRATCH;
  char* base = static_cast<char*>(scratch);
  SelState* s = reinterpret_cast<SelState*>(base);
  unsigned* hist = reinterpret_cast<unsigned*>(base + align256(sizeof(SelState)));
  k_sel_init<<<1, 256, 0, st>>>(s, hist, static_cast<long long>(k));
  ABC_LAUNCH_CHECK();
  const unsigned grid = static_cast<unsigned>(std::min<int64_t>(ceil_div(n, 1024), 152 * 8));
  for (int pass = 0; pass < 8; ++pass) {
    const int shift = 56 - 8 * pass;
    k_sel_hist<<<grid, 256, 0, st>>>(d, n, s, shift, hist);
    ABC_LAUNCH_CHECK();
    k_sel_pick<<<1, 256, 0, st>>>(s, hist, shift, out);
    ABC_LAUNCH_CHECK();
  }
  return ABC_OK;
}

// ------------------------------------------------- A5 weights and prefix ---
// Distances, tolerances, weights and stage weights are >= 0 (or +inf) and
// never NaN, so their IEEE bit patterns order like their values: the
// comparisons and maxima run on the integer pipes (fp64 is slow here).
__device__ __forceinline__ unsigned long long dbits(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x));
}

__device__ __forceinline__ double stage_weight(double d, double w, double eps, int mode) {
  if (dbits(d) > dbits(eps)) return 0.0;  // d > eps
  return mode == ABC_W_PAPER ? __dsub_rn(eps, d) : w;
}

__global__ void k_rmax(const double* __restrict__ d, const double* __restrict__ W, int64_t n,
                       const double* eps_p, int mode, unsigned long long* rmax_bits) {
  const double eps = *eps_p;
  unsigned long long m = 0ull;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const unsigned long long r = dbits(stage_weight(d[i], W ? W[i] : 0.0, eps, mode));
    m = r > m ? r : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(rmax_bits, m);
}

__global__ void k_quantize(const double* __restrict__ d, const double* __restrict__ W, int64_t n,
                           const double* eps_p, int mode, const unsigned long long* rmax_bits,
                           uint32_t* __restrict__ q, unsigned long long* tile_sum) {
  __shared__ unsigned long long sm[32];
  __shared__ double s_scale;
  const double eps = *eps_p;
  const unsigned long long rmb = *rmax_bits;
  const double rmax = __longlong_as_double(static_cast<long long>(rmb));
  const bool proper = rmb > 0ull && rmb < 0x7ff0000000000000ull;  // 0 < max r < inf
  // scale = (2^32 - 1) / max r, one correctly rounded division per block
  if (threadIdx.x == 0) s_scale = proper ? __ddiv_rn(4294967295.0, rmax) : 0.0;
  __syncthreads();
  const double scale = s_scale;
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile;
  unsigned long long s = 0;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int64_t i = base + e * kTileThr + threadIdx.x;
    if (i < n) {
      uint32_t qi;
      if (proper) {
        const double r = stage_weight(d[i], W ? W[i] : 0.0, eps, mode);
        // the largest weight maps to 2^32 - 1 exactly; otherwise floor(r s),
        // the truncating conversion saturating at 2^32 - 1 (r s >= 0)
        qi = dbits(r) == rmb ? 0xFFFFFFFFu : __double2uint_rz(__dmul_rn(r, scale));
      } else {
        qi = dbits(d[i]) <= dbits(eps) ? 1u : 0u;
      }
      q[i] = qi;
      s += qi;
    }
  }
  s = block_sum<unsigned long long>(s, sm);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = s;
}

// exclusive scan of per-tile totals by one block, in chunks of blockDim.x
// exclusive scan of the tile sums in one block; each thread takes 16
// consecutive values per round (a round covers 16 x blockDim tiles)
constexpr int kScanPer = 16;

template <typename T>
__global__ void __launch_bounds__(1024, 1)
k_scan_tiles(const T* __restrict__ in, int64_t ntiles, T* __restrict__ out, T* total) {
  __shared__ T sm[32];
  __shared__ T last;
  T carry = 0;
  for (int64_t b = 0; b < ntiles; b += static_cast<int64_t>(blockDim.x) * kScanPer) {
    const int64_t i0 = b + static_cast<int64_t>(threadIdx.x) * kScanPer;
    T v[kScanPer];
    T s = 0;
#pragma unroll
    for (int e = 0; e < kScanPer; ++e) {
      v[e] = i0 + e < ntiles ? in[i0 + e] : T(0);
      s += v[e];
    }
    const T inc = block_incl_scan<T>(s, sm);
    T run = carry + inc - s;
#pragma unroll
    for (int e = 0; e < kScanPer; ++e) {
      if (i0 + e < ntiles) out[i0 + e] = run;
      run += v[e];
    }
    if (threadIdx.x == blockDim.x - 1) last = inc;
    __syncthreads();
    carry += last;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void k_prefix_tiles(const uint32_t* __restrict__ q, int64_t n,
                               const unsigned long long* __restrict__ tile_off,
                               uint64_t* __restrict__ prefix, bool vec) {
  __shared__ unsigned long long sm[32];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile + 4 * threadIdx.x;
  // four consecutive weights per thread: one 16-byte load and two 16-byte
  // stores where all four exist and the arrays are 16-byte aligned (vec)
  const bool whole = vec && base + 3 < n;
  unsigned long long v[4];
  if (whole) {
    const uint4 w4 = *reinterpret_cast<const uint4*>(q + base);
    v[0] = w4.x;
    v[1] = w4.y;
    v[2] = w4.z;
    v[3] = w4.w;
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = base + e < n ? q[base + e] : 0ull;
  }
  const unsigned long long s = v[0] + v[1] + v[2] + v[3];
  const unsigned long long inc = block_incl_scan<unsigned long long>(s, sm);
  const unsigned long long r0 = tile_off[blockIdx.x] + inc - s + v[0];
  const unsigned long long r1 = r0 + v[1], r2 = r1 + v[2], r3 = r2 + v[3];
  if (whole) {
    *reinterpret_cast<ulonglong2*>(prefix + base) = make_ulonglong2(r0, r1);
    *reinterpret_cast<ulonglong2*>(prefix + base + 2) = make_ulonglong2(r2, r3);
  } else {
    const unsigned long long r[4] = {r0, r1, r2, r3};
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (base + e < n) prefix[base + e] = r[e];
  }
}

// the tile kernel's 16-byte accesses need both arrays 16-byte aligned
static bool prefix_vec_ok(const uint32_t* q, const uint64_t* prefix) {
  return (reinterpret_cast<uintptr_t>(q) & 15u) == 0 && (reinterpret_cast<uintptr_t>(prefix) & 15u) == 0;
}

size_t prefix_scratch_bytes(int64_t n) {
  const int64_t nt = ceil_div(std::max<int64_t>(n, 1), kTile);
  return align256(8) + 2 * align256(8 * nt) + align256(8);
}

int launch_resample_prefix(const double* d, const double* W, int64_t n, const double* eps,
                           int mode, uint32_t* q, uint64_t* prefix, void* scratch, size_t bytes,
                           cudaStream_t st) {
  if (n <= 0) return ABC_E_INVAL;
  if (mode == ABC_W_IMPORTANCE && !W) return ABC_E_INVAL;
  if (bytes < prefix_scratch_bytes(n)) return ABC_E_SCRATCH;
  const int64_t nt = ceil_div(n, kTile);
  char* b = static_cast<char*>(scratch);
  auto* rmax = reinterpret_cast<unsigned long long*>(b);
  auto* tsum = reinterpret_cast<unsigned long long*>(b + align256(8));
  auto* toff = reinterpret_cast<unsigned long long*>(b + align256(8) + align256(8 * nt));
  ABC_CUDA_TRY(cudaMemsetAsync(rmax, 0, 8, st));
  const unsigned g = static_cast<unsigned>(std::min<int64_t>(ceil_div(n, 256), 152 * 8));
  k_rmax<<<g, 256, 0, st>>>(d, mode == ABC_W_PAPER ? nullptr : W, n, eps, mode, rmax);
  ABC_LAUNCH_CHECK();
  k_quantize<<<static_cast<unsigned>(nt), kTileThr, 0, st>>>(
      d, mode == ABC_W_PAPER ? nullptr : W, n, eps, mode, rmax, q, tsum);
  ABC_LAUNCH_CHECK();
  k_scan_tiles<unsigned long long><<<1, 1024, 0, st>>>(tsum, nt, toff, nullptr);
  ABC_LAUNCH_CHECK();
  k_prefix_tiles<<<static_cast<unsigned>(nt), kTileThr, 0, st>>>(q, n, toff, prefix,
                                                               prefix_vec_ok(q, prefix));
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

// ---------------------------- A5 without allocation (fixed device scratch) --
// Some callers cannot allocate device memory at the time they run this step
// (their device memory belongs to a pool or a budget they do not control),
// so this variant takes its scratch from one file-scope array instead of a
// caller buffer.  The array holds the scratch of the largest supported size,
// stays resident on every device that loads the library until the process
// exits, and is shared by every call: concurrent calls race on it.
constexpr int64_t kNoAllocMaxN = int64_t(1) << 24;
constexpr size_t kNoAllocBytes =
    256 + 2 * static_cast<size_t>(8 * (kNoAllocMaxN / kTile)) + 256;  // prefix_scratch_bytes(max)
static __device__ __align__(256) unsigned char g_prefix_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[kNoAllocMaxDevices] = {};

int64_t resample_prefix_noalloc_max_n() { return kNoAllocMaxN; }

// The host-side name of g_prefix_scratch is not a device address: the device
// address is looked up once per device, with that device current.
int launch_resample_prefix_noalloc(const double* d, const double* W, int64_t n,
                                   const double* eps, int mode, uint32_t* q, uint64_t* prefix,
                                   cudaStream_t st) {
  static_assert(kNoAllocBytes >= 256 + 2 * 8 * (kNoAllocMaxN / kTile) + 256, "scratch size");
  if (n > kNoAllocMaxN) return ABC_E_TOO_LARGE;
  int dev = 0;
  ABC_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return ABC_E_INVAL;
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_prefix_scratch) != cudaSuccess) {
        cudaGetLastError();
        return ABC_E_CUDA;
      }
      g_noalloc_addr[dev] = p;
    }
    scratch = g_noalloc_addr[dev];
  }
  if (prefix_scratch_bytes(n) > kNoAllocBytes) return ABC_E_TOO_LARGE;
  return launch_resample_prefix(d, W, n, eps, mode, q, prefix, scratch, kNoAllocBytes, st);
}

// -------------------------------------------------------- A6-A7 propose ---
bool beta_rule_ok(const BetaRule& r) {
  const auto finite = [](float x) { return x == x && x - x == 0.0f; };
  switch (r.mode) {
    case ABC_BETA_PAPER:
      return true;
    case ABC_BETA_FIXED:
      return r.a > 0.0f && finite(r.a);
    case ABC_BETA_REAL:
      return r.p1 >= 0x1p-20f && r.p1 <= 0x1p20f && r.p2 >= 0x1p-20f && r.p2 <= 0x1p20f;
    case ABC_BETA_MEAN_VAR:
      return r.p1 > 0.0f && r.p1 < 1.0f && r.p2 > 0.0f && r.p2 <= 1.0f;
    case ABC_BETA_MODE_CONC:
      return r.p1 >= 0.0f && r.p1 <= 1.0f && r.p2 >= 2.0f && r.p2 <= 0x1p20f;
    case ABC_STEP_MCMC:
      return true;  // the step is checked where it is given
    default:
      return false;
  }
}

// Slots per warp of k_propose: the lanes of a warp take the slots of their
// chunk one after another, each lane moving on to the chunk's next slot when
// its own is done, so a slot that needs many redraws (attempts vary from 1
// to max_redraw) holds up one lane instead of 31.  Every slot's attempts use
// its own counters, so the assignment of slots to lanes changes no result.
__device__ __forceinline__ int64_t propose_chunk(int64_t slots) {
  // at least about 2432 warps (16 per SM) before a warp takes more than 32
  const int64_t mult = slots / (32 * 2432);
  return 32 * (mult < 1 ? 1 : (mult > 8 ? 8 : mult));
}

__global__ void k_propose(SimParams p, const float* __restrict__ u, int64_t n,
                          const uint64_t* __restrict__ prefix, BetaRule rule,
                          const double* eps_p, const double* eps1_p, int64_t slots,
                          const uint32_t* __restrict__ c0_idx, uint32_t c1, int max_redraw,
                          float* __restrict__ u_out, float* __restrict__ s_out,
                          int32_t* __restrict__ anc_out, int32_t* __restrict__ att_out,
                          uint8_t* __restrict__ flag_out, const uint32_t* __restrict__ c1_dev,
                          const int* __restrict__ beta_b_dev, const int* __restrict__ off_dev,
                          int64_t m_sub, const int* __restrict__ k_lim_dev,
                          const float* __restrict__ s_fix_dev) {
  // the warp's chunk of slots [lo, hi); whole warps return together
  const int64_t chunk = propose_chunk(slots);
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t lo = warp * chunk;
  if (lo >= slots) return;
  if (off_dev && *off_dev) return;  // run finished
  const int64_t hi = lo + chunk < slots ? lo + chunk : slots;
  if (c1_dev) c1 = *c1_dev;  // set on the device (graph launches)
  const int k_lim = k_lim_dev ? *k_lim_dev : 0x7fffffff;
  const int beta_b = beta_b_dev ? *beta_b_dev : rule.b;
  const unsigned long long total = prefix[n - 1];
  float a_t = rule.a, b_t = 0.0f;
  float ratio = 1.0f;
  // the MCMC baseline: one step for every slot and attempt (Eq. 12)
  const bool fixed_step = rule.mode == ABC_STEP_MCMC;
  const float s_fix = fixed_step ? (s_fix_dev ? *s_fix_dev : rule.a) : 0.0f;
  if (rule.mode != ABC_BETA_FIXED && rule.mode != ABC_BETA_REAL && !fixed_step) {
    // Eq. 16: eps_t / eps_1 (1 when eps_1 is zero)
    const double e1 = *eps1_p;
    ratio = e1 > 0.0 ? __double2float_rn(__ddiv_rn(*eps_p, e1)) : 1.0f;
  }
  if (rule.mode == ABC_BETA_PAPER) a_t = ratio;
  // the Gamma ratio: the real-shape rules, and the paper schedule once b =
  // 2t passes 1024 (integer b 0); the stage c1 >> 16 is the same for every
  // batch of the launch
  const bool real_shape = (rule.mode >= ABC_BETA_REAL && rule.mode <= ABC_BETA_MODE_CONC) ||
                          (rule.mode == ABC_BETA_PAPER && beta_b == 0);
  if (real_shape) beta_real_shape(rule, ratio, static_cast<int32_t>(c1 >> 16), &a_t, &b_t);
  const unsigned lt = (1u << (threadIdx.x & 31)) - 1u;
  int64_t next = lo;  // the chunk's next slot (the same in every lane)
  int64_t i = -1;     // this lane's slot, -1 for none
  uint32_t j = 0, c1s = c1;
  int a = 0;
  while (true) {
    // lanes without a slot take the chunk's next ones, in lane order
    const unsigned need = __ballot_sync(0xffffffffu, i < 0);
    if (i < 0) {
      const int64_t cand = next + __popc(need & lt);
      if (cand < hi) {
        i = cand;
        a = 0;
        // slots of several batches at once (m_sub > 0): slot i is slot is
        // of batch c1 + kb; batches at or beyond *k_lim_dev are not drawn
        // (flag 3)
        int64_t is = i;
        c1s = c1;
        if (m_sub > 0) {
          const int64_t kb = i / m_sub;
          is = i - kb * m_sub;
          c1s = c1 + static_cast<uint32_t>(kb);
          if (kb >= k_lim) {
            flag_out[i] = 3;
            i = -1;
          }
        }
        j = c0_idx ? c0_idx[is] : static_cast<uint32_t>(is);
      }
    }
    next += __popc(need);
    if (next > hi) next = hi;
    if (__all_sync(0xffffffffu, i < 0) && next >= hi) break;
    if (i < 0) continue;
    // attempt a of slot i
    // Eq. 11: categorical ancestor by inverting the u64 prefix
    const u32x4 wa = philox4x32_10(j, c1s, static_cast<uint32_t>(a), ABC_TAG_ANCESTOR, p.k0, p.k1);
    const unsigned long long U = (static_cast<unsigned long long>(wa.y) << 32) | wa.x;
    const unsigned long long x = __umul64hi(U, total);
    int64_t blo = 0, bhi = n - 1;
    while (blo < bhi) {
      const int64_t mid = blo + ((bhi - blo) >> 1);
      if (prefix[mid] > x) bhi = mid;
      else blo = mid + 1;
    }
    const int64_t anc = blo;
    float s;
    if (fixed_step) {
      s = s_fix;
    } else if (real_shape) {
      // real shapes: the Gamma ratio
      s = dev_beta_real(a_t, b_t, j, c1s, static_cast<uint32_t>(a), p.k0, p.k1);
    } else {
      // Eq. 16: s ~ Beta(a_t, b) as exp(sum_m log(U_m) / (a_t + m))
      float acc = 0.0f;
      u32x4 wb{0u, 0u, 0u, 0u};
      for (int m = 0; m < beta_b; ++m) {
        if ((m & 3) == 0)
          wb = philox4x32_10(j, c1s,
                             (static_cast<uint32_t>(a) << 8) | static_cast<uint32_t>(m >> 2),
                             ABC_TAG_BETA, p.k0, p.k1);
        const uint32_t wm = (m & 3) == 0 ? wb.x : (m & 3) == 1 ? wb.y : (m & 3) == 2 ? wb.z : wb.w;
        acc = __fadd_rn(acc, __fdiv_rn(dev_log_pos(unif(wm)), __fadd_rn(a_t, __int2float_rn(m))));
      }
      s = dev_exp(acc);
    }
    const float sd = __fsqrt_rn(s);
    // Eq. 17: u' = u_anc + sqrt(s) z; the support check covers all 8 coordinates
    float up[8];
    bool ok = true;
#pragma unroll
    for (int blk = 0; blk < 4; ++blk) {
      const u32x4 wz = philox4x32_10(j, c1s, (static_cast<uint32_t>(a) << 8) | blk, ABC_TAG_WALK,
                                     p.k0, p.k1);
      const float z0 = dev_normal(unif(wz.x), unif(wz.y));
      const float z1 = dev_normal(unif(wz.z), unif(wz.w));
      const float v0 = __fadd_rn(u[static_cast<int64_t>(2 * blk) * n + anc], __fmul_rn(sd, z0));
      const float v1 = __fadd_rn(u[static_cast<int64_t>(2 * blk + 1) * n + anc], __fmul_rn(sd, z1));
      up[2 * blk] = v0;
      up[2 * blk + 1] = v1;
      ok = ok && v0 >= 0.0f && v0 <= 1.0f && v1 >= 0.0f && v1 <= 1.0f;
    }
    if (ok || a + 1 >= max_redraw) {
      // the first u' inside [0,1]^8, or the last attempt's (redraws exhausted)
#pragma unroll
      for (int d = 0; d < 8; ++d) u_out[static_cast<int64_t>(d) * slots + i] = up[d];
      s_out[i] = s;
      anc_out[i] = static_cast<int32_t>(anc);
      att_out[i] = ok ? a + 1 : max_redraw;
      flag_out[i] = ok ? 0 : 1;
      i = -1;
    } else {
      ++a;
    }
  }
}

int launch_propose(const SimParams& p, const float* u, int64_t n, const uint64_t* prefix,
                   const BetaRule& rule, const double* eps, const double* eps1, int64_t slots,
                   const uint32_t* c0_idx, uint32_t c1, int max_redraw, float* u_out,
                   float* s_out, int32_t* anc_out, int32_t* att_out, uint8_t* flag_out,
                   cudaStream_t st, const uint32_t* c1_dev, const int* beta_b_dev,
                   const int* off_dev, int64_t m_sub, const int* k_lim_dev,
                   const float* s_fix_dev) {
  if (n <= 0 || slots < 0 || max_redraw < 1 || !beta_rule_ok(rule) || m_sub < 0)
    return ABC_E_INVAL;
  // the MCMC baseline's step: the device word, or rule.a > 0 (finite)
  if (rule.mode == ABC_STEP_MCMC && !s_fix_dev && !(rule.a > 0.0f && rule.a < INFINITY))
    return ABC_E_INVAL;
  if (rule.mode == ABC_BETA_FIXED && !beta_b_dev && (rule.b < 1 || rule.b > 1024))
    return ABC_E_INVAL;
  // paper schedule: integer b in 1..1024, or 0 for Beta(a_t, 2t) by the
  // Gamma ratio at the stage t = c1 >> 16 >= 1
  if (rule.mode == ABC_BETA_PAPER && !beta_b_dev &&
      (rule.b < 0 || rule.b > 1024 || (rule.b == 0 && !c1_dev && (c1 >> 16) == 0)))
    return ABC_E_INVAL;
  if (rule.mode != ABC_BETA_FIXED && rule.mode != ABC_BETA_REAL && rule.mode != ABC_STEP_MCMC &&
      (!eps || !eps1))
    return ABC_E_INVAL;
  // the scheduled real-shape rules read the stage t = c1 >> 16 >= 1
  if ((rule.mode == ABC_BETA_MEAN_VAR || rule.mode == ABC_BETA_MODE_CONC) && !c1_dev &&
      (c1 >> 16) == 0)
    return ABC_E_INVAL;
  if (slots == 0) return ABC_OK;
  // one warp per chunk of slots (propose_chunk), four warps per block
  const int64_t mult = slots / (32 * 2432);
  const int64_t chunk = 32 * (mult < 1 ? 1 : (mult > 8 ? 8 : mult));
  const int64_t warps = ceil_div(slots, chunk);
  k_propose<<<static_cast<unsigned>(ceil_div(warps, 4)), 128, 0, st>>>(
      p, u, n, prefix, rule, eps, eps1, slots, c0_idx, c1, max_redraw, u_out, s_out, anc_out,
      att_out, flag_out, c1_dev, beta_b_dev, off_dev, m_sub, k_lim_dev, s_fix_dev);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

// ------------------------------------------------ MCMC step adaptation ---
// Start of a generation: its accepted / exhausted counters start at zero,
// and the step of its first batch is recorded for the statistics.
__global__ void k_mcmc_begin(McmcDev* m, const int* off_dev) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (off_dev && *off_dev) return;
  m->acc_prev = 0;
  m->exh_prev = 0;
  m->s_start = m->s_f;
}

// After a batch of M slots (Sec. 3.1 adapts once per batch; Eq. 14-15):
// the batch's accepted and exhausted counts are the growth of the
// generation's counters acc_exh = {accepted, exhausted}; A = accepted /
// simulated (0 if none was simulated); inside the window s <- s (1 + (A -
// A_T) / ((1 - A_T)(k + 1))), A_T = 0.234, each operation rounded once in
// fp64 (no contraction).
__global__ void k_mcmc_adapt(McmcDev* m, const long long* acc_exh, long long M,
                             const int* off_dev) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (off_dev && *off_dev) return;
  const long long acc = acc_exh[0], exh = acc_exh[1];
  const long long acc_b = acc - m->acc_prev, exh_b = exh - m->exh_prev;
  m->acc_prev = acc;
  m->exh_prev = exh;
  if (m->batches < m->window) {
    const double kTarget = 0.234;
    const long long sims = M - exh_b;
    const double A = sims > 0 ? __ddiv_rn(static_cast<double>(acc_b), static_cast<double>(sims))
                              : 0.0;
    const double gain = __dmul_rn(__dsub_rn(1.0, kTarget), static_cast<double>(m->k + 1));
    m->s = __dmul_rn(m->s, __dadd_rn(1.0, __ddiv_rn(__dsub_rn(A, kTarget), gain)));
    m->k += 1;
    m->s_f = __double2float_rn(m->s);
  }
  m->batches += 1;
}

int launch_mcmc_begin(McmcDev* m, const int* off_dev, cudaStream_t st) {
  if (!m) return ABC_E_INVAL;
  k_mcmc_begin<<<1, 32, 0, st>>>(m, off_dev);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

int launch_mcmc_adapt(McmcDev* m, const long long* acc_exh, int64_t M, const int* off_dev,
                      cudaStream_t st) {
  if (!m || !acc_exh || M < 1) return ABC_E_INVAL;
  k_mcmc_adapt<<<1, 32, 0, st>>>(m, acc_exh, M, off_dev);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

// ----------------------------------------------------------- A8 accept ---
__global__ void k_acc_count(const double* __restrict__ dp, const uint8_t* __restrict__ flag,
                            int64_t M, const double* eps_p, int* __restrict__ tile_cnt,
                            long long* counters) {
  __shared__ int sm[32];
  __shared__ int smf[32];
  const double eps = *eps_p;
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile + 4 * threadIdx.x;
  int c = 0, f = 0;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int64_t i = base + e;
    if (i < M) {
      const uint8_t fl = flag[i];  // 1: redraws exhausted; 2: simulated for an audit only
      f += (fl == 1);
      c += (fl == 0 && dp[i] <= eps);
    }
  }
  c = block_sum<int>(c, sm);
  f = block_sum<int>(f, smf);
  if (threadIdx.x == 0) {
    tile_cnt[blockIdx.x] = c;
    if (f && counters)
      atomicAdd(reinterpret_cast<unsigned long long*>(&counters[1]),
                static_cast<unsigned long long>(f));
  }
}

__global__ void k_acc_finish(const int* tile_total, long long* filled, long long* base_out,
                             long long* counters, int64_t N) {
  const long long tot = *tile_total;
  const long long f0 = *filled;
  *base_out = f0;
  counters[0] += tot;
  *filled = f0 + tot < N ? f0 + tot : N;
}

__global__ void k_acc_scatter(const float* __restrict__ up, const double* __restrict__ dp,
                              const float* __restrict__ sp, const int32_t* __restrict__ ap,
                              const uint8_t* __restrict__ flag, int64_t M, const double* eps_p,
                              const int* __restrict__ tile_off, const long long* base_p,
                              int64_t N, float* __restrict__ u_pop, double* __restrict__ d_pop,
                              float* __restrict__ s_pop, int32_t* __restrict__ anc_pop,
                              const float* __restrict__ rho_in, float* __restrict__ rho_pop) {
  __shared__ int sm[32];
  const double eps = *eps_p;
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile + 4 * threadIdx.x;
  bool acc[4];
  int c = 0;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int64_t i = base + e;
    acc[e] = i < M && flag[i] == 0 && dp[i] <= eps;
    c += acc[e];
  }
  const int inc = block_incl_scan<int>(c, sm);
  long long pos = *base_p + tile_off[blockIdx.x] + inc - c;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if (!acc[e]) continue;
    const int64_t i = base + e;
    if (pos < N) {
#pragma unroll
      for (int d = 0; d < 8; ++d) u_pop[static_cast<int64_t>(d) * N + pos] = up[static_cast<int64_t>(d) * M + i];
      d_pop[pos] = dp[i];
      s_pop[pos] = sp[i];
      anc_pop[pos] = ap[i];
      if (rho_pop) rho_pop[pos] = rho_in ? rho_in[i] : 1.0f;
    }
    ++pos;
  }
}

size_t accept_scratch_bytes(int64_t M) {
  const int64_t nt = ceil_div(std::max<int64_t>(M, 1), kTile);
  return 2 * align256(4 * nt) + align256(8) + align256(8);
}

int launch_accept(const float* up, const double* dp, const float* sp, const int32_t* ap,
                  const uint8_t* flag, int64_t M, const double* eps, int64_t N, float* u_pop,
                  double* d_pop, float* s_pop, int32_t* anc_pop, int64_t* filled,
                  int64_t* counters, void* scratch, size_t bytes, cudaStream_t st,
                  const float* rho_in, float* rho_pop) {
  if (M < 0 || N <= 0) return ABC_E_INVAL;
  if (M == 0) return ABC_OK;
  if (bytes < accept_scratch_bytes(M)) return ABC_E_SCRATCH;
  const int64_t nt = ceil_div(M, kTile);
  char* b = static_cast<char*>(scratch);
  int* cnt = reinterpret_cast<int*>(b);
  int* off = reinterpret_cast<int*>(b + align256(4 * nt));
  int* tot = reinterpret_cast<int*>(b + 2 * align256(4 * nt));
  long long* basep = reinterpret_cast<long long*>(b + 2 * align256(4 * nt) + align256(8));
  long long* cnts = reinterpret_cast<long long*>(counters);
  k_acc_count<<<static_cast<unsigned>(nt), kTileThr, 0, st>>>(dp, flag, M, eps, cnt, cnts);
  ABC_LAUNCH_CHECK();
  k_scan_tiles<int><<<1, 1024, 0, st>>>(cnt, nt, off, tot);
  ABC_LAUNCH_CHECK();
  k_acc_finish<<<1, 1, 0, st>>>(tot, reinterpret_cast<long long*>(filled), basep, cnts, N);
  ABC_LAUNCH_CHECK();
  k_acc_scatter<<<static_cast<unsigned>(nt), kTileThr, 0, st>>>(up, dp, sp, ap, flag, M, eps, off,
                                                                basep, N, u_pop, d_pop, s_pop,
                                                                anc_pop, rho_in, rho_pop);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

// ---- several batches accepted at once (graph-captured batches) -----------
// Batches b .. b + K - 1 of M slots each were proposed and simulated
// together; the sequential rule accepts them in (batch, slot) order and
// stops after the batch in which N is reached.  k_spec_count counts each
// batch's acceptances and exhausted slots; k_spec_finish finds that batch,
// adds the counts of the batches up to it (accepted, exhausted) and sets the
// number of batches used; the scatter stores the first N acceptances of the
// whole range in order, which are those of the used batches.
__global__ void __launch_bounds__(256)
k_spec_count(const double* __restrict__ dp, const uint8_t* __restrict__ flag, int64_t M,
             const double* eps_p, int* __restrict__ sub_acc, int* __restrict__ sub_exh) {
  __shared__ int sm[32];
  __shared__ int smf[32];
  const double eps = *eps_p;
  const int64_t b0 = static_cast<int64_t>(blockIdx.x) * M;
  int c = 0, f = 0;
  for (int64_t j = threadIdx.x; j < M; j += blockDim.x) {
    const uint8_t fl = flag[b0 + j];
    f += (fl == 1);
    c += (fl == 0 && dp[b0 + j] <= eps);
  }
  c = block_sum<int>(c, sm);
  f = block_sum<int>(f, smf);
  if (threadIdx.x == 0) {
    sub_acc[blockIdx.x] = c;
    sub_exh[blockIdx.x] = f;
  }
}

__global__ void k_spec_finish(const int* __restrict__ sub_acc, const int* __restrict__ sub_exh,
                              const int* k_lim_dev, long long* filled, long long* base_out,
                              long long* counters, int* used_out, int64_t N) {
  const int klim = *k_lim_dev;
  const long long f0 = *filled;
  *base_out = f0;
  long long f = f0, acc = 0, exh = 0;
  int used = klim;
  for (int k = 0; k < klim; ++k) {
    acc += sub_acc[k];
    exh += sub_exh[k];
    f += sub_acc[k];
    if (f >= N) {
      used = k + 1;
      break;
    }
  }
  counters[0] += acc;
  counters[1] += exh;
  *filled = f < N ? f : N;
  *used_out = used;
}

size_t accept_spec_scratch_bytes(int64_t M, int K) {
  return accept_scratch_bytes(M * K) + 2 * align256(4 * static_cast<size_t>(K));
}

int launch_accept_spec(const float* up, const double* dp, const float* sp, const int32_t* ap,
                       const uint8_t* flag, int64_t M, int K, const int* k_lim_dev,
                       const double* eps, int64_t N, float* u_pop, double* d_pop, float* s_pop,
                       int32_t* anc_pop, int64_t* filled, int64_t* counters, int* used_out,
                       void* scratch, size_t bytes, cudaStream_t st) {
  if (M <= 0 || N <= 0 || K < 1 || !k_lim_dev || !used_out) return ABC_E_INVAL;
  if (bytes < accept_spec_scratch_bytes(M, K)) return ABC_E_SCRATCH;
  const int64_t MK = M * K;
  const int64_t nt = ceil_div(MK, kTile);
  char* b = static_cast<char*>(scratch);
  int* cnt = reinterpret_cast<int*>(b);
  int* off = reinterpret_cast<int*>(b + align256(4 * nt));
  int* tot = reinterpret_cast<int*>(b + 2 * align256(4 * nt));
  long long* basep = reinterpret_cast<long long*>(b + 2 * align256(4 * nt) + align256(8));
  char* tail = b + accept_scratch_bytes(MK);
  int* sub_acc = reinterpret_cast<int*>(tail);
  int* sub_exh = reinterpret_cast<int*>(tail + align256(4 * static_cast<size_t>(K)));
  k_spec_count<<<static_cast<unsigned>(K), 256, 0, st>>>(dp, flag, M, eps, sub_acc, sub_exh);
  ABC_LAUNCH_CHECK();
  k_acc_count<<<static_cast<unsigned>(nt), kTileThr, 0, st>>>(dp, flag, MK, eps, cnt, nullptr);
  ABC_LAUNCH_CHECK();
  k_scan_tiles<int><<<1, 1024, 0, st>>>(cnt, nt, off, tot);
  ABC_LAUNCH_CHECK();
  k_spec_finish<<<1, 1, 0, st>>>(sub_acc, sub_exh, k_lim_dev, reinterpret_cast<long long*>(filled),
                                 basep, reinterpret_cast<long long*>(counters), used_out, N);
  ABC_LAUNCH_CHECK();
  k_acc_scatter<<<static_cast<unsigned>(nt), kTileThr, 0, st>>>(up, dp, sp, ap, flag, MK, eps, off,
                                                                basep, N, u_pop, d_pop, s_pop,
                                                                anc_pop, nullptr, nullptr);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

// --------------------------------------- survivor columns for the weights -
// Columns with q_k > 0, in index order: cu [8][nc] and c_k = log2(q_k) - 32
// as a double-float, hi in cc[0..ncap) and lo in cc[ncap..2 ncap).
__global__ void k_surv_count(const uint32_t* __restrict__ q, int64_t n, int* __restrict__ cnt) {
  __shared__ int sm[32];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile + 4 * threadIdx.x;
  int c = 0;
#pragma unroll
  for (int e = 0; e < 4; ++e) c += (base + e < n && q[base + e] > 0u);
  c = block_sum<int>(c, sm);
  if (threadIdx.x == 0) cnt[blockIdx.x] = c;
}

__global__ void k_surv_scatter(const float* __restrict__ u, const uint32_t* __restrict__ q,
                               int64_t n, const int* __restrict__ off, float* __restrict__ cu,
                               float* __restrict__ cc, int64_t ncap) {
  __shared__ int sm[32];
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile + 4 * threadIdx.x;
  int c = 0;
  bool keep[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    keep[e] = base + e < n && q[base + e] > 0u;
    c += keep[e];
  }
  const int inc = block_incl_scan<int>(c, sm);
  int64_t pos = static_cast<int64_t>(off[blockIdx.x]) + inc - c;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if (!keep[e]) continue;
    const int64_t i = base + e;
#pragma unroll
    for (int d = 0; d < 8; ++d) cu[static_cast<int64_t>(d) * ncap + pos] = u[static_cast<int64_t>(d) * n + i];
    // c_k as a double-float: hi in cc[pos], lo in cc[ncap + pos]
    const double c = log2(static_cast<double>(q[i])) - 32.0;
    const float ch = __double2float_rn(c);
    cc[pos] = ch;
    cc[ncap + pos] = __double2float_rn(c - static_cast<double>(ch));
    ++pos;
  }
}

size_t survivors_scratch_bytes(int64_t n) {
  const int64_t nt = ceil_div(std::max<int64_t>(n, 1), kTile);
  return 2 * align256(4 * nt) + align256(4);
}

// compacts into cu [8][n] / cc[2 n] (capacity n); *nc_dev receives the count
int launch_survivors(const float* u, const uint32_t* q, int64_t n, float* cu, float* cc,
                     int* nc_dev, void* scratch, cudaStream_t st) {
  const int64_t nt = ceil_div(n, kTile);
  char* b = static_cast<char*>(scratch);
  int* cnt = reinterpret_cast<int*>(b);
  int* off = reinterpret_cast<int*>(b + align256(4 * nt));
  k_surv_count<<<static_cast<unsigned>(nt), kTileThr, 0, st>>>(q, n, cnt);
  ABC_LAUNCH_CHECK();
  k_scan_tiles<int><<<1, 1024, 0, st>>>(cnt, nt, off, nc_dev);
  ABC_LAUNCH_CHECK();
  k_surv_scatter<<<static_cast<unsigned>(nt), kTileThr, 0, st>>>(u, q, n, off, cu, cc, n);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

// ------------------------------------------------------ A10 normalise ----
constexpr int kNormBlocks = 512;

// An unsigned key that orders doubles like their values (on the integer
// pipes: fp64 is slow here); NaN maps to 0, below -inf, so that the maximum
// ignores it as fmax does.
__device__ __forceinline__ unsigned long long ord_key(double x) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  if ((b & 0x7FFFFFFFFFFFFFFFull) > 0x7FF0000000000000ull) return 0ull;
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double ord_value(unsigned long long k) {
  return __longlong_as_double(static_cast<long long>(
      (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k));
}

__global__ void k_nz_max(const double* __restrict__ lw, int64_t n, double* part) {
  __shared__ unsigned long long sm[32];
  unsigned long long m = ord_key(-__longlong_as_double(0x7ff0000000000000ll));
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const unsigned long long k = ord_key(lw[i]);
    m = k > m ? k : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long k = __shfl_xor_sync(0xffffffffu, m, o);
    m = k > m ? k : m;
  }
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (blockDim.x >> 5); ++w) m = sm[w] > m ? sm[w] : m;
    part[blockIdx.x] = ord_value(m);
  }
}

// exp(x) for -700 <= x <= 0 to fp64 precision with five fp64 operations
// (this GPU's fp64 rate is far below its fp32 rate).  Tang's table-driven
// method (ACM TOMS 15(2), 1989): x = (64 e + j) ln2 / 64 + r, |r| <= about
// ln2 / 128, reduced in fp64 by two fma with ln2 / 64 split into a double
// and its tail; r as a float pair (rh + rl); exp(r) - 1 = r + r^2 / 2 + r^3
// (1/6 + r/24 + r^2/120), the first two terms as float pairs through
// error-free fma remainders and sums, the rest in fp32 (below 3e-8); times
// 2^(j/64) from a table of float pairs (tab, made from the fp64 exp2); the
// pair recombined exactly in fp64 and scaled by 2^e in the exponent field.
// Relative error below 1e-14 (tests compare with the host's exp).
__device__ __forceinline__ double exp_tang(double x, const float2* tab) {
  const double kLn2By64 = 0x1.62e42fefa39efp-7;     // ln 2 / 64, nearest double
  const double kLn2By64T = 0x1.abc9e3b39803fp-62;   // ln 2 / 64 - kLn2By64
  const float kf = rintf(__double2float_rn(x) * 92.33248261689366f);  // 64 / ln 2
  const int k = static_cast<int>(kf);
  const double kd = static_cast<double>(k);
  double r = fma(-kd, kLn2By64, x);
  r = fma(-kd, kLn2By64T, r);
  const float rh = __double2float_rn(r);
  const float rl = __double2float_rn(r - static_cast<double>(rh));
  const float t = rh * rh;
  const float te = fmaf(rh, rh, -t);                 // rh^2 = t + te exactly
  const float hh = 0.5f * t;
  const float hl = 0.5f * fmaf(2.0f * rh, rl, te);   // r^2 / 2 = hh + hl
  const float q = t * rh * fmaf(rh, fmaf(rh, 1.0f / 120.0f, 1.0f / 24.0f), 1.0f / 6.0f);
  const float sh = rh + hh;                          // two-sum of rh and hh
  const float bb = sh - rh;
  const float se = (rh - (sh - bb)) + (hh - bb);
  const float sl = se + (rl + (hl + q));             // exp(r) - 1 = sh + sl
  const float2 T = tab[k & 63];                      // 2^(j/64) = T.x + T.y
  const float P = T.x * sh;
  const float Pe = fmaf(T.x, sh, -P);
  const float Rh = T.x + P;                          // T.x >= 1 > |P|
  const float Re = P - (Rh - T.x);
  const float Rl = Re + (Pe + (T.y + fmaf(T.x, sl, T.y * sh)));
  const double w = static_cast<double>(Rh) + static_cast<double>(Rl);
  const long long e = static_cast<long long>(k >> 6);  // floor(k / 64)
  return __longlong_as_double(__double_as_longlong(w) + (e << 52));
}

// mode 0: w = exp(lw - M) written to W and summed (the only exponentials);
// mode 1: W scaled by 1/S in place, W^2 summed
__global__ void k_nz_sum(const double* __restrict__ lw, int64_t n, const double* stat, int mode,
                         double* __restrict__ W, double* part) {
  __shared__ double sm[32];
  __shared__ float2 tab[64];
  if (mode == 0 && threadIdx.x < 64) {
    const double v = exp2(static_cast<double>(threadIdx.x) / 64.0);
    const float h = __double2float_rn(v);
    tab[threadIdx.x] = make_float2(h, __double2float_rn(v - static_cast<double>(h)));
  }
  __syncthreads();
  const double M = stat[0];
  const bool uniform = !(M > -__longlong_as_double(0x7ff0000000000000ll));
  const double inv = mode == 1 ? (uniform ? 1.0 / static_cast<double>(n) : 1.0 / stat[1]) : 0.0;
  double acc = 0.0;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double w;
    if (mode == 0) {
      const double li = lw[i];
      const double x = li - M;
      // NaN weights count as 0; below -700 (weights under 1e-304) the library exp
      w = uniform ? 1.0 : (x >= -700.0 ? exp_tang(x, tab) : (x == x ? exp(x) : 0.0));
      W[i] = w;
    } else {
      w = uniform ? inv : W[i] * inv;
      W[i] = w;
      w = w * w;
    }
    acc += w;
  }
  acc = block_sum<double>(acc, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// one block of kNormBlocks threads folds the partials (np <= kNormBlocks):
// op 0 max -> stat[0], 1 sum -> stat[1], 2 ess
__global__ void k_nz_fold(const double* part, int np, int op, double* stat, double* ess,
                          int64_t n) {
  __shared__ double sm[32];
  const double ninf = -__longlong_as_double(0x7ff0000000000000ll);
  double r = op == 0 ? ninf : 0.0;
  if (static_cast<int>(threadIdx.x) < np) r = part[threadIdx.x];
  if (op == 0) {
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < static_cast<int>(blockDim.x >> 5); ++w) r = fmax(r, sm[w]);
      stat[0] = r;
    }
    return;
  }
  r = block_sum<double>(r, sm);
  if (threadIdx.x != 0) return;
  if (op == 1) stat[1] = r;
  else *ess = stat[0] > ninf ? 1.0 / r : static_cast<double>(n);
}

size_t normalize_scratch_bytes(int64_t) { return align256(8 * kNormBlocks) + align256(16); }

int launch_normalize(const double* lw, int64_t n, double* W, double* ess, void* scratch,
                     size_t bytes, cudaStream_t st) {
  if (n <= 0) return ABC_E_INVAL;
  if (bytes < normalize_scratch_bytes(n)) return ABC_E_SCRATCH;
  char* b = static_cast<char*>(scratch);
  double* part = reinterpret_cast<double*>(b);
  double* stat = reinterpret_cast<double*>(b + align256(8 * kNormBlocks));
  const int g = static_cast<int>(std::min<int64_t>(kNormBlocks, ceil_div(n, 256)));
  k_nz_max<<<g, 256, 0, st>>>(lw, n, part);
  ABC_LAUNCH_CHECK();
  k_nz_fold<<<1, kNormBlocks, 0, st>>>(part, g, 0, stat, ess, n);
  ABC_LAUNCH_CHECK();
  k_nz_sum<<<g, 256, 0, st>>>(lw, n, stat, 0, W, part);
  ABC_LAUNCH_CHECK();
  k_nz_fold<<<1, kNormBlocks, 0, st>>>(part, g, 1, stat, ess, n);
  ABC_LAUNCH_CHECK();
  k_nz_sum<<<g, 256, 0, st>>>(lw, n, stat, 1, W, part);
  ABC_LAUNCH_CHECK();
  k_nz_fold<<<1, kNormBlocks, 0, st>>>(part, g, 2, stat, ess, n);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

__global__ void k_fill_f64(double* p, int64_t n, double v) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

int launch_fill(double* p, int64_t n, double v, cudaStream_t st) {
  if (n <= 0) return ABC_OK;
  k_fill_f64<<<static_cast<unsigned>(ceil_div(n, 256)), 256, 0, st>>>(p, n, v);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

}  // namespace abc
