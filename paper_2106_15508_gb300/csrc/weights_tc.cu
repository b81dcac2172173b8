// weights_tc.cu -- A9 importance weights on the tcgen05 tensor cores.
//
//   log W_j = 4 ln(2 pi s_j) - ln sum_k (q_k / total) exp(-|u'_j - u_k|^2 / (2 s_j))
//
// The exponent (base 2) of every pair is an inner product of a row feature
// vector and a column feature vector.  With centred coordinates x = u' - 1/2,
// y = u - 1/2 and L_j = log2(e) / (2 s_j):
//   e_jk = [2 L_j x_j, -L_j, 1] . [y_k, |y_k|^2, c_k]   (10 features)
//          - L_j |x_j|^2                               (row constant, fp64)
// with c_k = log2(q_k) - 32.  A single bf16 copy of these features would
// carry 2^-9 relative error into terms of size L_j (hundreds to 1e5), so
// each feature is split into three bf16 parts (v = v0 + v1 + v2, 24
// significant bits) and the six products with i + j <= 2 are kept: K = 60
// used of 64.  Products of bf16 values are exact and accumulate in fp32 in
// tensor memory, so the remaining error is the fp32 accumulation of terms of
// size ~L_j |y|^2 (stated in the tests, not a parity gate).
//
// Kernel structure (one CTA = 128 rows, one SM):
//   warp 4  : bulk-copy producer (cp.async.bulk, mbarrier complete_tx):
//             the row tile once, then 256-column tiles through a 4-stage ring
//   warp 5  : tcgen05.mma issuer (one thread), M = 128, N = 256, K = 4 x 16,
//             fp32 accumulators double-buffered in TMEM (2 x 256 columns)
//   warps 0-3: epilogue, one thread per row (TMEM lane): tcgen05.ld 32
//             columns at a time, online max and sum of 2^(e - m)
// Operands are packed by a prep kernel in the canonical K-major layout
// without swizzle: 8 x 8 bf16 core matrices (128 contiguous bytes), the 8
// core matrices of a row group consecutive along K (LBO = 128 B), row groups
// 1024 B apart (SBO).  Every mbarrier wait is bounded in time; on time-out
// the kernel records an error word, lets the other roles finish, waits for
// its own copies and frees its tensor memory.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"

namespace abc {

constexpr int kTcM = 128;                           // rows per CTA (UMMA M)
constexpr int kTcN = 256;                           // columns per tile (UMMA N)
constexpr int kTcK = 64;                            // packed K (60 used)
constexpr int kTcStages = 4;                        // column-tile ring
constexpr uint32_t kATile = kTcM * kTcK * 2;        // 16 KB
constexpr uint32_t kBTile = kTcN * kTcK * 2;        // 32 KB
constexpr uint32_t kTmemCols = 512;                 // two 256-column accumulators
constexpr int kTcThreads = 192;                     // 6 warps
constexpr size_t kTcSmem = 1024 + kATile + kTcStages * kBTile + 256;
constexpr float kSMinTc = 1e-30f;
constexpr float kPadLogit = -1.0e30f;

// instruction descriptor, kind::f16: D f32 (bits 4-5 = 1), A and B bf16
// (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17,
// M >> 4 at bit 24
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                            (static_cast<uint32_t>(kTcN >> 3) << 17) |
                            (static_cast<uint32_t>(kTcM >> 4) << 24);

// element index of (row r, k) inside a packed tile
__host__ __device__ __forceinline__ int packed_index(int r, int k) {
  return ((((r >> 3) << 3) + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7);
}

// ---- PTX wrappers -----------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// wait for the phase of the given parity; gives up after ~2 s and records
// the failure (code) in *err
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned* err,
                                          unsigned code) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > 2000000000ull) {
      atomicCAS(err, 0u, code);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(slot)),
               "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// shared-memory matrix descriptor: start >> 4 (bits 0-13), leading byte
// offset >> 4 (16-29), stride byte offset >> 4 (32-45), the fixed 0b001 at
// bits 46-48, base offset 0, relative LBO, no swizzle (bits 61-63 = 0)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = static_cast<uint64_t>((saddr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= 1ull << 46;
  return d;
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 32 consecutive fp32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ---- operand packing -------------------------------------------------------
// split v into three bf16 parts: v = p0 + p1 + p2 up to 2^-24 relative
__device__ __forceinline__ void split3(float v, __nv_bfloat16 (&p)[3]) {
  p[0] = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(p[0]);
  p[1] = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(p[1]);
  p[2] = __float2bfloat16_rn(r2);
}

// the six (i, j) part pairs with i + j <= 2, in K order:
// (0,0) (0,1) (1,0) (0,2) (1,1) (2,0); the A slot takes part i, B part j
__device__ __forceinline__ int pair_a(int t) { return (t == 2 || t == 4) ? 1 : (t == 5 ? 2 : 0); }
__device__ __forceinline__ int pair_b(int t) { return (t == 1 || t == 4) ? 1 : (t == 3 ? 2 : 0); }

// writes one packed row (64 bf16: feature ft, pair t at K = 6 ft + t, K 60-63
// zero) as eight 16-byte core-matrix rows
template <bool kASide>
__device__ __forceinline__ void store_packed_row(__nv_bfloat16* tile, int r, const float (&f)[10]) {
  uint32_t h[64];
#pragma unroll
  for (int ft = 0; ft < 10; ++ft) {
    __nv_bfloat16 p[3];
    split3(f[ft], p);
#pragma unroll
    for (int t = 0; t < 6; ++t)
      h[ft * 6 + t] = __bfloat16_as_ushort(p[kASide ? pair_a(t) : pair_b(t)]);
  }
#pragma unroll
  for (int k = 60; k < 64; ++k) h[k] = 0u;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    uint4 v;
    v.x = h[8 * c + 0] | (h[8 * c + 1] << 16);
    v.y = h[8 * c + 2] | (h[8 * c + 3] << 16);
    v.z = h[8 * c + 4] | (h[8 * c + 5] << 16);
    v.w = h[8 * c + 6] | (h[8 * c + 7] << 16);
    *reinterpret_cast<uint4*>(tile + packed_index(r, 8 * c)) = v;
  }
}

// rows: features [2 L x (8), -L, 1]; rowc[j] = -L |x|^2 (fp64)
__global__ void k_tc_pack_rows(const float* __restrict__ up, const float* __restrict__ s,
                               int64_t rows, int64_t rows_pad, __nv_bfloat16* __restrict__ Apk,
                               double* __restrict__ rowc) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= rows_pad) return;
  float f[10];
  if (j < rows) {
    const float sj = fmaxf(s[j], kSMinTc);
    const float L = 1.4426950408889634f / (2.0f * sj);
    double xx = 0.0;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      const float x = up[static_cast<int64_t>(d) * rows + j] - 0.5f;
      f[d] = 2.0f * L * x;
      xx += static_cast<double>(x) * static_cast<double>(x);
    }
    f[8] = -L;
    f[9] = 1.0f;
    rowc[j] = -static_cast<double>(L) * xx;
  } else {
#pragma unroll
    for (int d = 0; d < 10; ++d) f[d] = 0.0f;
  }
  store_packed_row<true>(Apk + (j / kTcM) * (kTcM * kTcK), static_cast<int>(j % kTcM), f);
}

// columns: features [y (8), |y|^2, c_k]; columns at or beyond nc are padding
// with c = -1e30 (their exponentials vanish)
__global__ void k_tc_pack_cols(const float* __restrict__ cu, const float* __restrict__ cc,
                               const int* __restrict__ nc_p, int64_t ncap, int64_t cols_pad,
                               __nv_bfloat16* __restrict__ Bpk) {
  const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= cols_pad) return;
  const int64_t nc = *nc_p;
  float f[10];
  if (k < nc) {
    float yy = 0.0f;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      const float y = cu[static_cast<int64_t>(d) * ncap + k] - 0.5f;
      f[d] = y;
      yy = __fmaf_rn(y, y, yy);
    }
    f[8] = yy;
    f[9] = cc[k];
  } else {
#pragma unroll
    for (int d = 0; d < 9; ++d) f[d] = 0.0f;
    f[9] = kPadLogit;
  }
  store_packed_row<false>(Bpk + (k / kTcN) * (kTcN * kTcK), static_cast<int>(k % kTcN), f);
}

// ---- main kernel -------------------------------------------------------------
struct TcSmem {
  uint8_t* a;
  uint8_t* b;
  uint64_t* full;
  uint64_t* empty;
  uint64_t* tfull;
  uint64_t* tempty;
  uint64_t* afull;
  uint32_t* tmem_slot;
};

__device__ __forceinline__ TcSmem tc_carve(uint8_t* raw) {
  TcSmem m;
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
  m.a = base;
  m.b = base + kATile;
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + kATile + kTcStages * kBTile);
  m.full = bars;
  m.empty = bars + kTcStages;
  m.tfull = bars + 2 * kTcStages;
  m.tempty = bars + 2 * kTcStages + 2;
  m.afull = bars + 2 * kTcStages + 4;
  m.tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kTcStages + 5);
  return m;
}

__global__ void __launch_bounds__(kTcThreads, 1)
k_weights_tc(const uint8_t* __restrict__ Apk, const uint8_t* __restrict__ Bpk,
             const int* __restrict__ nc_p, int64_t rows, int tiles_per_chunk,
             float2* __restrict__ part, unsigned* err, const int* __restrict__ off_dev) {
  extern __shared__ uint8_t tc_smem_raw[];
  if (off_dev && *off_dev) return;  // run finished or its generation stopped (block-uniform)
  const TcSmem sm = tc_carve(tc_smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nc = *nc_p;
  const int ntot = static_cast<int>((nc + kTcN - 1) / kTcN);
  const int tb = static_cast<int>(blockIdx.y) * tiles_per_chunk;
  const int te = min(ntot, tb + tiles_per_chunk);
  const int64_t row0 = static_cast<int64_t>(blockIdx.x) * kTcM;
  if (tb >= te) {  // no column tile in this chunk: neutral partials
    if (threadIdx.x < kTcM && row0 + threadIdx.x < rows)
      part[static_cast<int64_t>(blockIdx.y) * rows + row0 + threadIdx.x] = make_float2(-INFINITY, 0.0f);
    return;
  }
  const int ntiles = te - tb;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kTcStages; ++i) {
      mbar_init(&sm.full[i], 1);
      mbar_init(&sm.empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&sm.tfull[i], 1);
      mbar_init(&sm.tempty[i], kTcM);
    }
    mbar_init(sm.afull, 1);
    fence_mbar_init();
  }
  if (warp == 5) {
    tmem_alloc(sm.tmem_slot, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *sm.tmem_slot;

  if (warp == 4) {
    // ---------------- producer ----------------
    if (lane == 0) {
      mbar_expect_tx(sm.afull, kATile);
      bulk_g2s(sm.a, Apk + static_cast<size_t>(blockIdx.x) * kATile, kATile, sm.afull);
      int issued = 0;
      for (int t = 0; t < ntiles; ++t) {
        const int st = t % kTcStages;
        const uint32_t ph = static_cast<uint32_t>(t / kTcStages) & 1u;
        if (!mbar_wait(&sm.empty[st], ph ^ 1u, err, 1u)) break;
        mbar_expect_tx(&sm.full[st], kBTile);
        bulk_g2s(sm.b + st * kBTile, Bpk + static_cast<size_t>(tb + t) * kBTile, kBTile,
                 &sm.full[st]);
        issued = t + 1;
      }
      // every copy this thread started has landed before the CTA can exit
      mbar_wait(sm.afull, 0u, err, 2u);
      for (int t = issued > kTcStages ? issued - kTcStages : 0; t < issued; ++t)
        mbar_wait(&sm.full[t % kTcStages], static_cast<uint32_t>(t / kTcStages) & 1u, err, 2u);
    }
  } else if (warp == 5) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int last = -1;
      if (mbar_wait(sm.afull, 0u, err, 3u)) {
        const uint32_t a0 = smem_u32(sm.a);
        for (int t = 0; t < ntiles; ++t) {
          const int st = t % kTcStages, b = t & 1;
          const uint32_t ph = static_cast<uint32_t>(t / kTcStages) & 1u;
          const uint32_t tph = static_cast<uint32_t>(t >> 1) & 1u;
          if (!mbar_wait(&sm.tempty[b], tph ^ 1u, err, 4u)) break;
          if (!mbar_wait(&sm.full[st], ph, err, 5u)) break;
          tc_fence_after();
          const uint32_t b0 = smem_u32(sm.b + st * kBTile);
          const uint32_t d = tmem + static_cast<uint32_t>(b * kTcN);
#pragma unroll
          for (int kk = 0; kk < kTcK / 16; ++kk)
            umma_bf16(d, smem_desc(a0 + kk * 256, 128, 1024), smem_desc(b0 + kk * 256, 128, 1024),
                      kIdesc, kk > 0 ? 1u : 0u);
          umma_commit(&sm.empty[st]);
          umma_commit(&sm.tfull[b]);
          last = t;
        }
      }
      // the accumulators must be complete before the memory is freed
      if (last >= 0)
        mbar_wait(&sm.tfull[last & 1], static_cast<uint32_t>(last >> 1) & 1u, err, 6u);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: thread = row = TMEM lane ----------------
    const int r = threadIdx.x;
    const uint32_t lane_base = tmem + (static_cast<uint32_t>(warp * 32) << 16);
    float m = -INFINITY, S = 0.0f, cS = 0.0f;
    for (int t = 0; t < ntiles; ++t) {
      const int b = t & 1;
      const uint32_t tph = static_cast<uint32_t>(t >> 1) & 1u;
      if (!mbar_wait(&sm.tfull[b], tph, err, 7u)) break;
      tc_fence_after();
      float ts = 0.0f;
#pragma unroll 1
      for (int c = 0; c < kTcN / 32; ++c) {
        float v[32];
        tmem_ld32(lane_base + static_cast<uint32_t>(b * kTcN + c * 32), v);
        float cm = v[0];
#pragma unroll
        for (int i = 1; i < 32; ++i) cm = fmaxf(cm, v[i]);
        if (cm > m) {
          const float f = ex2(m - cm);
          S *= f;
          cS *= f;
          ts *= f;
          m = cm;
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) ts += ex2(v[i] - m);
      }
      tc_fence_before();
      mbar_arrive(&sm.tempty[b]);
      const float y = ts - cS;
      const float tt = S + y;
      cS = (tt - S) - y;
      S = tt;
    }
    if (row0 + r < rows) part[static_cast<int64_t>(blockIdx.y) * rows + row0 + r] = make_float2(m, S);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 5) tmem_dealloc(tmem, kTmemCols);
}

__global__ void k_weights_tc_combine(const float2* __restrict__ part, int nchunks,
                                     const float* __restrict__ s, const double* __restrict__ rowc,
                                     int64_t rows, const uint64_t* __restrict__ total_p,
                                     double* __restrict__ logW, const int* __restrict__ off_dev) {
  const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= rows || (off_dev && *off_dev)) return;
  const double sj = static_cast<double>(fmaxf(s[j], kSMinTc));
  double M = -INFINITY;
  for (int c = 0; c < nchunks; ++c)
    M = fmax(M, static_cast<double>(part[static_cast<int64_t>(c) * rows + j].x));
  double S = 0.0;
  for (int c = 0; c < nchunks; ++c) {
    const float2 p = part[static_cast<int64_t>(c) * rows + j];
    if (p.y > 0.0f) S += static_cast<double>(p.y) * exp2(static_cast<double>(p.x) - M);
  }
  const double lse2 = rowc[j] + M + log2(S) + 32.0 - log2(static_cast<double>(*total_p));
  logW[j] = 4.0 * log(6.283185307179586 * sj) - 0.6931471805599453 * lse2;
}

// one 128 x 256 x 64 product with the weight kernel's operand layout and
// descriptors (diagnostic): D[i][n] = sum_k A[i][k] B[n][k]
__global__ void __launch_bounds__(kTcThreads, 1)
k_tc_probe(const uint8_t* __restrict__ Apk, const uint8_t* __restrict__ Bpk,
           float* __restrict__ D, unsigned* err) {
  extern __shared__ uint8_t tc_smem_raw[];
  const TcSmem sm = tc_carve(tc_smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(&sm.full[0], 1);
    mbar_init(&sm.tfull[0], 1);
    fence_mbar_init();
  }
  if (warp == 5) {
    tmem_alloc(sm.tmem_slot, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *sm.tmem_slot;
  if (warp == 4 && lane == 0) {
    mbar_expect_tx(&sm.full[0], kATile + kBTile);
    bulk_g2s(sm.a, Apk, kATile, &sm.full[0]);
    bulk_g2s(sm.b, Bpk, kBTile, &sm.full[0]);
    mbar_wait(&sm.full[0], 0u, err, 8u);
  } else if (warp == 5 && lane == 0) {
    if (mbar_wait(&sm.full[0], 0u, err, 9u)) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(sm.a), b0 = smem_u32(sm.b);
#pragma unroll
      for (int kk = 0; kk < kTcK / 16; ++kk)
        umma_bf16(tmem, smem_desc(a0 + kk * 256, 128, 1024), smem_desc(b0 + kk * 256, 128, 1024),
                  kIdesc, kk > 0 ? 1u : 0u);
      umma_commit(&sm.tfull[0]);
      mbar_wait(&sm.tfull[0], 0u, err, 10u);
    }
  } else if (warp < 4) {
    const bool ok = mbar_wait(&sm.tfull[0], 0u, err, 11u);
    tc_fence_after();
    if (ok) {
      for (int c = 0; c < kTcN / 32; ++c) {
        float v[32];
        tmem_ld32(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c * 32, v);
        for (int i = 0; i < 32; ++i) D[static_cast<int64_t>(threadIdx.x) * kTcN + c * 32 + i] = v[i];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 5) tmem_dealloc(tmem, kTmemCols);
}

// ---- host side -----------------------------------------------------------------
// column chunks: about two CTAs per SM in total, times a tuning multiplier
static int tc_chunks(int64_t rows, int64_t ncap, int mult) {
  const int64_t gx = ceil_div(std::max<int64_t>(rows, 1), kTcM);
  const int64_t tiles = std::max<int64_t>(1, ceil_div(ncap, kTcN));
  const int64_t want = std::max<int64_t>(1, ceil_div(2 * 152, gx)) * std::max(1, mult);
  return static_cast<int>(std::min<int64_t>(want, tiles));
}

struct TcLayout {
  size_t apk, bpk, rowc, part, err, total;
};

static TcLayout tc_layout(int64_t rows, int64_t ncap, int mult) {
  TcLayout l{};
  const int64_t rpad = ceil_div(std::max<int64_t>(rows, 1), kTcM) * kTcM;
  const int64_t cpad = ceil_div(std::max<int64_t>(ncap, 1), kTcN) * kTcN;
  size_t o = 0;
  l.apk = o;
  o += align256(static_cast<size_t>(rpad) * kTcK * 2);
  l.bpk = o;
  o += align256(static_cast<size_t>(cpad) * kTcK * 2);
  l.rowc = o;
  o += align256(sizeof(double) * static_cast<size_t>(rows));
  l.part = o;
  o += align256(sizeof(float2) * static_cast<size_t>(tc_chunks(rows, ncap, mult)) * rows);
  l.err = o;
  o += align256(sizeof(unsigned));
  l.total = o;
  return l;
}

int weights_tc_prepare() {
  ABC_CUDA_TRY(cudaFuncSetAttribute(k_weights_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(kTcSmem)));
  return ABC_OK;
}

size_t weights_tc_scratch_bytes(int64_t rows, int64_t ncap, int mult) {
  return tc_layout(rows, ncap, mult).total;
}

// cu/cc/nc_dev: compacted survivor columns (capacity ncap).  The error word
// is written into the scratch area; err_host (nullable) receives it when
// sync_err is set.
int launch_weights_tc(const float* up, const float* s, int64_t rows, const float* cu,
                      const float* cc, const int* nc_dev, int64_t ncap, const uint64_t* total_p,
                      double* logW, void* scratch, size_t bytes, unsigned** err_dev,
                      cudaStream_t st, const int* off_dev, int mult) {
  if (rows <= 0) return ABC_OK;
  const TcLayout l = tc_layout(rows, ncap, mult);
  if (bytes < l.total) return ABC_E_SCRATCH;
  // the kernel's shared-memory opt-in is a function attribute: set it unless
  // the stream is being captured (contexts set it when they are created)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  ABC_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
  if (cs == cudaStreamCaptureStatusNone) {
    const int rc = weights_tc_prepare();
    if (rc) return rc;
  }
  char* b = static_cast<char*>(scratch);
  auto* Apk = reinterpret_cast<__nv_bfloat16*>(b + l.apk);
  auto* Bpk = reinterpret_cast<__nv_bfloat16*>(b + l.bpk);
  auto* rowc = reinterpret_cast<double*>(b + l.rowc);
  auto* part = reinterpret_cast<float2*>(b + l.part);
  auto* err = reinterpret_cast<unsigned*>(b + l.err);
  if (err_dev) *err_dev = err;
  ABC_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(unsigned), st));
  const int64_t rpad = ceil_div(rows, kTcM) * kTcM;
  const int64_t cpad = ceil_div(std::max<int64_t>(ncap, 1), kTcN) * kTcN;
  k_tc_pack_rows<<<static_cast<unsigned>(ceil_div(rpad, 128)), 128, 0, st>>>(up, s, rows, rpad, Apk,
                                                                            rowc);
  ABC_LAUNCH_CHECK();
  k_tc_pack_cols<<<static_cast<unsigned>(ceil_div(cpad, 128)), 128, 0, st>>>(cu, cc, nc_dev, ncap,
                                                                            cpad, Bpk);
  ABC_LAUNCH_CHECK();
  const int nch = tc_chunks(rows, ncap, mult);
  const int tiles = static_cast<int>(ceil_div(std::max<int64_t>(ncap, 1), kTcN));
  const int per = static_cast<int>(ceil_div(tiles, nch));
  dim3 grid(static_cast<unsigned>(rpad / kTcM), static_cast<unsigned>(nch));
  k_weights_tc<<<grid, kTcThreads, kTcSmem, st>>>(reinterpret_cast<const uint8_t*>(Apk),
                                                  reinterpret_cast<const uint8_t*>(Bpk), nc_dev,
                                                  rows, per, part, err, off_dev);
  ABC_LAUNCH_CHECK();
  k_weights_tc_combine<<<static_cast<unsigned>(ceil_div(rows, 256)), 256, 0, st>>>(
      part, nch, s, rowc, rows, total_p, logW, off_dev);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

// Apk/Bpk: packed bf16 tiles (16 KB, 32 KB); D: 128 x 256 fp32; err: u32
int launch_tc_probe(const void* Apk, const void* Bpk, float* D, unsigned* err, cudaStream_t st) {
  ABC_CUDA_TRY(cudaFuncSetAttribute(k_tc_probe, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(kTcSmem)));
  ABC_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(unsigned), st));
  k_tc_probe<<<1, kTcThreads, kTcSmem, st>>>(static_cast<const uint8_t*>(Apk),
                                             static_cast<const uint8_t*>(Bpk), D, err);
  ABC_LAUNCH_CHECK();
  return ABC_OK;
}

}  // namespace abc
