// weights.cu -- A9 importance weights, FP32 CUDA-core path.
//
//   log W_j = 4 ln(2 pi s_j) - ln sum_k (q_k / total) exp(-|u'_j - u_k|^2 / (2 s_j))
//
// over the surviving columns (q_k > 0), compacted beforehand into cu [8][nc]
// and c_k = log2(q_k) - 32 as a double-float (hi in cc[k], lo in
// cc[ncap + k]).  Work is in base 2: e_jk = c_k - L_j D_jk with
// L_j = log2(e) / (2 s_j) (a double-float from one fp64 division per row),
// an integer-valued running row maximum m and sums of 2^(e - m).
//
// Every pair is first evaluated in plain fp32 (direct differences in packed
// fp32x2 lanes, one fused multiply-add with L_hi and c_hi).  A pair whose
// fp32 exponent lies within kNearBits of the running maximum is evaluated
// again in double-float arithmetic: each coordinate difference exactly (two
// terms, Knuth's TwoSum), each square exactly (product plus its FMA
// remainder), the eight squares summed with TwoSum, then L D and c - L D
// with the error-free product and sum (Dekker; Ogita, Rump & Oishi 2005).
// Those terms go into a Kahan sum; the pairs below the threshold, each under
// 2^-40 of the maximum, go into a plain fp32 sum.  The running maximum moves
// only to integers, so rescaling a sum is an exact power of two.  Rows whose
// exponents reach 2^22 in magnitude keep only the leading fp32 part (their
// relative precision is that of fp32 already).  Columns are split into
// chunks over grid.y; a combine kernel merges the partials in fp64.  The
// kernel variance is floored at 1e-30 (1/(2s) must stay finite in fp32; such
// rows carry negligible weight).
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

__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ void unpk2(unsigned long long a, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a));
}

constexpr float kNearBits = 40.0f;     // exponents within 40 bits of the maximum: exact path
constexpr float kHugeExp = 4194304.0f;  // 2^22: beyond it a term keeps its fp32 part only

// Knuth's TwoSum: s + e = a + b exactly (any magnitudes)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// The exponent e = c - L D of one pair as a double-float (eh + el), with
// D = |x - y|^2 over the eight coordinates: x, y as four packed pairs of
// coordinates, (lh, ll) = L, (ch, cl) = c.  Differences and squares are
// exact; their sums carry errors of a few 2^-48 relative.
__device__ __forceinline__ void exact_exponent(const unsigned long long (&x)[4],
                                               const unsigned long long (&y)[4], float lh, float ll,
                                               float ch, float cl, float& eh, float& el) {
  unsigned long long hs = 0, he = 0, cr = 0, pn = 0;
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    // d = x - y = ds + de exactly (TwoSum of x and -y, two lanes at once)
    const unsigned long long ds = sub2(x[h], y[h]);
    const unsigned long long bb = sub2(ds, x[h]);
    const unsigned long long de = sub2(sub2(x[h], sub2(ds, bb)), add2(y[h], bb));
    // d^2 = ph + pl exactly: pl = ds^2 - ph from the fused remainder (taken
    // negated with -ds = y - x, also exact), plus the cross term 2 ds de
    const unsigned long long ph = mul2(ds, ds);
    const unsigned long long pln = fma2(sub2(y[h], x[h]), ds, ph);  // = -pl
    const unsigned long long c = mul2(ds, de);
    if (h == 0) {
      hs = ph;
      cr = c;
      pn = pln;
    } else {
      // hs + ph with its rounding error (TwoSum, both lanes)
      const unsigned long long t = add2(hs, ph);
      const unsigned long long b2 = sub2(t, hs);
      he = add2(he, add2(sub2(hs, sub2(t, b2)), sub2(ph, b2)));
      hs = t;
      cr = add2(cr, c);
      pn = add2(pn, pln);
    }
  }
  float h0, h1, e0, e1, c0, c1, n0, n1;
  unpk2(hs, h0, h1);
  unpk2(he, e0, e1);
  unpk2(cr, c0, c1);
  unpk2(pn, n0, n1);
  float dh, de2;
  two_sum(h0, h1, dh, de2);
  // low part: rounding errors of the sums, 2 sum(ds de) and sum(pl)
  const float lo = __fadd_rn(__fadd_rn(de2, __fadd_rn(e0, e1)),
                             __fsub_rn(__fmul_rn(2.0f, __fadd_rn(c0, c1)), __fadd_rn(n0, n1)));
  // renormalise D = dh + dl
  const float Dh = __fadd_rn(dh, lo);
  const float Dl = __fsub_rn(lo, __fsub_rn(Dh, dh));
  // L D = P + Pe (Dekker's product with the fused remainder)
  const float P = __fmul_rn(lh, Dh);
  float Pe = __fmaf_rn(lh, Dh, -P);
  Pe = __fmaf_rn(lh, Dl, Pe);
  Pe = __fmaf_rn(ll, Dh, Pe);
  // c - L D
  float s0, s1;
  two_sum(ch, -P, s0, s1);
  const float lo2 = __fsub_rn(__fadd_rn(s1, cl), Pe);
  eh = __fadd_rn(s0, lo2);
  el = __fsub_rn(lo2, __fsub_rn(eh, s0));
}

// 2^k for an integer-valued k <= 0 (0 below 2^-126, and for k = -inf or NaN)
__device__ __forceinline__ float exact_pow2(float k) {
  if (!(k >= -126.0f)) return 0.0f;
  return __int_as_float((127 + static_cast<int>(k)) << 23);
}

__global__ void __launch_bounds__(kWThreads)
k_weights_fp32(const float* __restrict__ up, const float* __restrict__ s, int64_t rows,
               const float* __restrict__ cu, const float* __restrict__ cc,
               const int* __restrict__ nc_p, int64_t ncap,
               float4* __restrict__ part, const int* __restrict__ off_dev,
               const int* __restrict__ rows_dev) {
  // column coordinates as four pairs: su2[h][k] = (u_2h, u_2h+1) of column k;
  // c_k as (hi, lo)
  __shared__ __align__(16) unsigned long long su2[4][kWTile];
  __shared__ float2 sc[kWTile];
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
  // per row: L = lh + ll, running maximum m (integer-valued), Kahan sum
  // (S, cS) of the exactly evaluated terms, plain sum F of the others
  float lh[kWRows], ll[kWRows], m[kWRows], S[kWRows], cS[kWRows], F[kWRows];
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
    const double L = 1.4426950408889634 / (2.0 * static_cast<double>(sj));  // log2(e) / (2 s_j)
    lh[r] = __double2float_rn(L);
    ll[r] = __double2float_rn(L - static_cast<double>(lh[r]));
    m[r] = -INFINITY;
    S[r] = 0.0f;
    cS[r] = 0.0f;
    F[r] = 0.0f;
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
      sc[i] = in ? make_float2(cc[c0 + i], cc[ncap + c0 + i]) : make_float2(-INFINITY, 0.0f);
    }
    __syncthreads();
    for (int k = 0; k < cnt; ++k) {
      unsigned long long uk[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) uk[h] = su2[h][k];
      const float2 ck = sc[k];
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
        const float e = __fmaf_rn(D, -lh[r], ck.x);
        if (e > m[r] - kNearBits) {
          float eh, el;
          exact_exponent(x[r], uk, lh[r], ll[r], ck.x, ck.y, eh, el);
          if (!(fabsf(eh) < kHugeExp)) el = 0.0f;
          const float mn = ceilf(eh);
          if (mn > m[r]) {
            const float f = exact_pow2(m[r] - mn);
            S[r] *= f;
            cS[r] *= f;
            F[r] *= f;
            m[r] = mn;
          }
          // Kahan: S - cS is the sum
          const float y = ex2f(__fadd_rn(__fsub_rn(eh, m[r]), el)) - cS[r];
          const float t = S[r] + y;
          cS[r] = (t - S[r]) - y;
          S[r] = t;
        } else {
          F[r] += ex2f(e - m[r]);
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < kWRows; ++r) {
    const int64_t j = row0 + r * kWThreads;
    if (j < nrows)
      part[static_cast<int64_t>(blockIdx.y) * rows + j] = make_float4(m[r], S[r], cS[r], F[r]);
  }
  __syncthreads();  // the shared tiles are refilled for the next row block
  }
}

// log W from the chunk partials: sum_c 2^(m_c - M) (S_c - cS_c + F_c) in fp64
// (m_c integer-valued, so the factors are exact)
__global__ void k_weights_combine(const float4* __restrict__ part, int nchunks,
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
    const float4 p = part[static_cast<int64_t>(c) * rows + j];
    const double v = (static_cast<double>(p.y) - static_cast<double>(p.z)) + static_cast<double>(p.w);
    if (v > 0.0) S += v * exp2(static_cast<double>(p.x) - M);
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
  return align256(sizeof(float4) * static_cast<size_t>(weight_chunks(rows, ncap, mult)) * rows);
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
  float4* part = static_cast<float4*>(scratch);
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
