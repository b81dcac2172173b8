// api.cu -- the C ABI: argument checks, step entry points and the context
// that runs whole SMC generations (Sec. 2.4 and 3.2 of arXiv 2106.15508).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cuda_bf16.h>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "batch.cuh"
#include "common.cuh"
#include "surrogate.cuh"

namespace abc {
// launchers not declared in batch.cuh
int launch_prior(const SimParams&, int64_t, float*, cudaStream_t);
int launch_synth_obs(const SimParams&, const float*, const float*, int32_t*, float*, int32_t*,
                     cudaStream_t);
int launch_philox(const uint32_t*, uint32_t, uint32_t, int64_t, uint32_t*, cudaStream_t);
size_t select_scratch_bytes(int64_t);
size_t prefix_scratch_bytes(int64_t);
int launch_resample_prefix_noalloc(const double*, const double*, int64_t, const double*, int,
                                   uint32_t*, uint64_t*, cudaStream_t);
size_t accept_scratch_bytes(int64_t);
size_t survivors_scratch_bytes(int64_t);
size_t weights_fp32_scratch_bytes(int64_t, int64_t, int mult = 1);
size_t weights_tc_scratch_bytes(int64_t, int64_t, int mult = 1);
int64_t weights_tc_tile_pairs();
int ex2_probe(double* rate, cudaStream_t st);
int numerics_check(int which, unsigned long long* bad_host, cudaStream_t st);
size_t predict_scratch_bytes(int64_t N, int64_t R, int32_t days, int32_t nq);
int launch_predict(const SimParams& p, const float* u, const double* W, int64_t N, int64_t R,
                   int32_t days, const double* quant, int32_t nq, int32_t* out, void* scratch,
                   size_t bytes, cudaStream_t st);
int launch_tc_probe(const void*, const void*, float*, unsigned*, cudaStream_t);
size_t normalize_scratch_bytes(int64_t);
int launch_fill(double*, int64_t, double, cudaStream_t);
void set_tc_wait_limit(uint64_t ns);
}  // namespace abc

namespace abc {
static std::atomic<int64_t> g_launches{0};
int64_t count_launch() { return g_launches.fetch_add(1, std::memory_order_relaxed) + 1; }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace abc

using namespace abc;

namespace {
// Test hook: context allocations left before an injected failure (-1: none).
// Failure detection is exercised on the host, without making a device fail.
std::atomic<long long> g_alloc_fail_after{-1};
bool alloc_fails_now() {
  long long left = g_alloc_fail_after.load();
  while (left > 0 && !g_alloc_fail_after.compare_exchange_weak(left, left - 1)) {
  }
  return left == 0;
}
}  // namespace

namespace {

constexpr int64_t kMaxIndex = 0x7fffffffLL;

int check_config(const abc_config* c) {
  if (!c) return ABC_E_INVAL;
  if (c->model != ABC_MODEL_SAIRD && c->model != ABC_MODEL_GAUSS_TOY) return ABC_E_INVAL;
  if (c->sampler != ABC_SIM_BINOMIAL && c->sampler != ABC_SIM_PAPER_NORMAL) return ABC_E_INVAL;
  if (c->model == ABC_MODEL_SAIRD) {
    if (c->n_days < 1 || c->n_days > 16383) return ABC_E_INVAL;  // 4 day + block < 2^16
    if (c->population < 1 || c->population > kMaxIndex) return ABC_E_INVAL;
    int64_t s = 0;
    for (int i = 0; i < 3; ++i) {
      if (c->init_ard[i] < 0) return ABC_E_INVAL;
      s += c->init_ard[i];
    }
    if (s > c->population) return ABC_E_INVAL;
  }
  for (int d = 0; d < 8; ++d)
    if (!(c->theta_hi[d] >= c->theta_lo[d]) || !std::isfinite(c->theta_lo[d]) ||
        !std::isfinite(c->theta_hi[d]))
      return ABC_E_INVAL;
  return ABC_OK;
}

BetaRule beta_rule(const abc_config& c) {
  return BetaRule{c.beta_mode, c.beta_a, c.beta_b, c.beta_p1, c.beta_p2};
}

// (a_t, b_t as fp32, integer b_t or 0) of stage t >= 1 as the proposal kernel
// derives them, for the generation statistics
void stage_shapes(const abc_config& c, double eps, double eps1, int32_t t, int32_t bb,
                  abc_gen_stats* g) {
  const float ratio = eps1 > 0.0 ? static_cast<float>(eps / eps1) : 1.0f;
  const BetaRule r = beta_rule(c);
  if (c.beta_mode == ABC_STEP_MCMC) {
    // the step itself is read from the device (mcmc_stats)
    g->beta_a = 0.0f;
    g->beta_b = 0;
    g->beta_bf = 0.0f;
  } else if (c.beta_mode >= ABC_BETA_REAL || (c.beta_mode == ABC_BETA_PAPER && bb == 0)) {
    beta_real_shape(r, ratio, t, &g->beta_a, &g->beta_bf);
    g->beta_b = 0;
  } else {
    g->beta_a = c.beta_mode == ABC_BETA_PAPER ? ratio : c.beta_a;
    g->beta_b = bb;
    g->beta_bf = static_cast<float>(bb);
  }
}

int check_smc(const abc_config* c) {
  if (c->n_particles < 1 || c->batch_size < 0) return ABC_E_INVAL;
  if (!(c->survival_alpha > 0.0 && c->survival_alpha <= 1.0)) return ABC_E_INVAL;
  if (!beta_rule_ok(beta_rule(*c))) return ABC_E_INVAL;
  if (c->beta_mode == ABC_BETA_FIXED && (c->beta_b < 1 || c->beta_b > 1024)) return ABC_E_INVAL;
  if (c->weight_mode != ABC_W_PAPER && c->weight_mode != ABC_W_IMPORTANCE) return ABC_E_INVAL;
  if (c->weight_prec != ABC_P_FP32 && c->weight_prec != ABC_P_BF16_TC) return ABC_E_INVAL;
  if (c->max_batches < 1 || c->max_batches > 65535) return ABC_E_INVAL;
  if (c->max_total_batches < 0) return ABC_E_INVAL;
  if (!(c->eps_stop >= 0.0f && c->eps_stop < INFINITY)) return ABC_E_INVAL;
  if (c->spec_batches < 0 || c->spec_batches > 256) return ABC_E_INVAL;
  if (c->max_redraw < 1 || c->max_redraw > (1 << 23)) return ABC_E_INVAL;
  if (c->beta_mode == ABC_STEP_MCMC &&
      (!(c->mcmc_s0 > 0.0f && c->mcmc_s0 < INFINITY) || c->mcmc_adapt < 0 || c->surrogate))
    return ABC_E_INVAL;
  if (c->surrogate) {
    if (c->surrogate != 1 || c->surrogate_start < 1 || c->surrogate_steps < 0 ||
        c->surrogate_batch < 32 || c->surrogate_batch > 65536 || !(c->surrogate_lr > 0.0f) ||
        !(c->surrogate_tau > 0.0f) || !(c->surrogate_rho_min > 0.0f) ||
        !(c->surrogate_rho_min <= 1.0f) || !(c->audit_frac >= 0.0f && c->audit_frac <= 1.0f) ||
        c->surrogate_ring < 0)
      return ABC_E_INVAL;
  }
  return ABC_OK;
}

}  // namespace

// ---------------------------------------------------------------- steps ---
extern "C" {

ABC_API void abc_config_default(abc_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof *c);
  c->model = ABC_MODEL_SAIRD;
  c->sampler = ABC_SIM_BINOMIAL;
  c->n_days = 120;
  c->init_ard[0] = 10;
  c->population = 100000;
  const float hi[8] = {1.f, 100.f, 2.f, 1.f, 1.f, 1.f, 1.f, 2.f};  // Eq. 2
  for (int d = 0; d < 8; ++d) c->theta_hi[d] = hi[d];
  c->seed = 1;
  c->n_particles = 1000;
  c->survival_alpha = 0.5;
  c->beta_mode = ABC_BETA_PAPER;
  c->mcmc_s0 = 0.1f;
  c->beta_a = 2.0f;
  c->beta_b = 5;
  c->weight_mode = ABC_W_PAPER;
  c->weight_prec = ABC_P_FP32;
  c->max_batches = 64;
  c->max_redraw = 64;
  c->surrogate = 0;
  c->surrogate_start = 3;
  c->surrogate_steps = 64;
  c->surrogate_batch = 8192;
  c->surrogate_lr = 1e-3f;
  c->surrogate_tau = 0.5f;
  c->surrogate_rho_min = 0.05f;
  c->audit_frac = 0.01f;
  c->surrogate_ring = 0;
  c->spec_batches = 1;
}

ABC_API const char* abc_strerror(int code) {
  switch (code) {
    case ABC_OK: return "ok";
    case ABC_STOP_BUDGET: return "generation stopped: batch budget used before N acceptances";
    case ABC_STOP_TARGET: return "run stopped: tolerance target reached";
    case ABC_STOP_TOTAL: return "run stopped: run budget of batches used";
    case ABC_E_INVAL: return "invalid argument or configuration";
    case ABC_E_NOMEM: return "device allocation failed";
    case ABC_E_CUDA: return "CUDA runtime error";
    case ABC_E_DEVICE: return "device-side bound check failed";
    case ABC_E_SCRATCH: return "scratch buffer too small";
    case ABC_E_STATE: return "malformed or mismatched state";
    case ABC_E_TOO_LARGE: return "size above the fixed scratch of the allocation-free entry point";
    default: return "unknown status";
  }
}

ABC_API int abc_philox(const uint32_t* ctr, uint32_t key0, uint32_t key1, int64_t n, uint32_t* out,
                       void* stream) {
  if (n < 0 || (n > 0 && (!ctr || !out))) return ABC_E_INVAL;
  return launch_philox(ctr, key0, key1, n, out, as_stream(stream));
}

ABC_API int abc_synth_obs(const abc_config* cfg, const float* box_lo, const float* box_hi,
                          int32_t* obs, float* theta_star, int32_t* attempts, void* stream) {
  int rc = check_config(cfg);
  if (rc) return rc;
  if (cfg->model != ABC_MODEL_SAIRD || !box_lo || !box_hi || !obs || !theta_star || !attempts)
    return ABC_E_INVAL;
  return launch_synth_obs(make_params(*cfg), box_lo, box_hi, obs, theta_star, attempts,
                          as_stream(stream));
}

ABC_API int abc_prior(const abc_config* cfg, int64_t n, float* u, void* stream) {
  int rc = check_config(cfg);
  if (rc) return rc;
  if (n < 0 || n > kMaxIndex || (n > 0 && !u)) return ABC_E_INVAL;
  return launch_prior(make_params(*cfg), n, u, as_stream(stream));
}

ABC_API int abc_simulate(const abc_config* cfg, const int32_t* obs, const float* u, int64_t n,
                         const uint32_t* c0_idx, uint32_t c1, uint32_t tag, const uint8_t* skip,
                         double* dist, int32_t* traj, void* stream) {
  int rc = check_config(cfg);
  if (rc) return rc;
  if (n < 0 || n > kMaxIndex || (n > 0 && (!u || !dist))) return ABC_E_INVAL;
  return launch_simulate(make_params(*cfg), obs, u, n, c0_idx, c1, tag, skip, dist, traj,
                         as_stream(stream));
}

ABC_API size_t abc_select_scratch_bytes(int64_t n) { return select_scratch_bytes(n); }

ABC_API int abc_select_kth(const double* d, int64_t n, int64_t k, double* out, void* scratch,
                           size_t scratch_bytes, void* stream) {
  if (!d || !out || !scratch) return ABC_E_INVAL;
  return launch_select(d, n, k, out, scratch, scratch_bytes, as_stream(stream));
}

ABC_API size_t abc_prefix_scratch_bytes(int64_t n) { return prefix_scratch_bytes(n); }

ABC_API int abc_resample_prefix(const double* d, const double* W, int64_t n, const double* eps,
                                int32_t mode, uint32_t* q, uint64_t* prefix, void* scratch,
                                size_t scratch_bytes, void* stream) {
  if (!d || !eps || !q || !prefix || !scratch || n > kMaxIndex) return ABC_E_INVAL;
  if (mode != ABC_W_PAPER && mode != ABC_W_IMPORTANCE) return ABC_E_INVAL;
  return launch_resample_prefix(d, W, n, eps, mode, q, prefix, scratch, scratch_bytes,
                                as_stream(stream));
}

ABC_API int abc_resample_prefix_noalloc(const double* d, const double* W, int64_t n,
                                        const double* eps, int32_t mode, uint32_t* q,
                                        uint64_t* prefix, void* stream) {
  if (!d || !eps || !q || !prefix || n <= 0) return ABC_E_INVAL;
  if (mode != ABC_W_PAPER && mode != ABC_W_IMPORTANCE) return ABC_E_INVAL;
  if (n > ABC_NOALLOC_MAX_N) return ABC_E_TOO_LARGE;
  return launch_resample_prefix_noalloc(d, W, n, eps, mode, q, prefix, as_stream(stream));
}

ABC_API int abc_propose(const abc_config* cfg, const float* u, int64_t n, const uint64_t* prefix,
                        const double* eps, const double* eps1, float beta_a, int32_t beta_b,
                        int64_t slots, const uint32_t* c0_idx, uint32_t c1, float* u_out,
                        float* s_out, int32_t* anc_out, int32_t* attempts_out, uint8_t* flag_out,
                        void* stream) {
  int rc = check_config(cfg);
  if (rc) return rc;
  if (!u || !prefix || n < 1 || n > kMaxIndex || slots < 0 || slots > kMaxIndex) return ABC_E_INVAL;
  if (slots > 0 && (!u_out || !s_out || !anc_out || !attempts_out || !flag_out)) return ABC_E_INVAL;
  if (cfg->max_redraw < 1 || cfg->max_redraw > (1 << 23)) return ABC_E_INVAL;
  BetaRule rule = beta_rule(*cfg);
  rule.a = beta_a;
  rule.b = beta_b;
  return launch_propose(make_params(*cfg), u, n, prefix, rule, eps, eps1, slots, c0_idx, c1,
                        cfg->max_redraw, u_out, s_out, anc_out, attempts_out, flag_out,
                        as_stream(stream));
}

ABC_API size_t abc_accept_scratch_bytes(int64_t M) { return accept_scratch_bytes(M); }

ABC_API int abc_accept_append(const float* up, const double* dp, const float* sp,
                              const int32_t* ap, const uint8_t* flag, int64_t M,
                              const double* eps, int64_t N, float* u_pop, double* d_pop,
                              float* s_pop, int32_t* anc_pop, int64_t* filled, int64_t* counters,
                              void* scratch, size_t scratch_bytes, void* stream) {
  if (M > kMaxIndex || N > kMaxIndex) return ABC_E_INVAL;
  if (M > 0 && (!up || !dp || !sp || !ap || !flag || !eps || !u_pop || !d_pop || !s_pop ||
                !anc_pop || !filled || !counters || !scratch))
    return ABC_E_INVAL;
  return launch_accept(up, dp, sp, ap, flag, M, eps, N, u_pop, d_pop, s_pop, anc_pop, filled,
                       counters, scratch, scratch_bytes, as_stream(stream));
}

// scratch layout of abc_weights: [cu 8n][cc 2n][nc][compaction][weight pass]
static size_t weights_layout(int64_t rows, int64_t n, size_t* off_cc, size_t* off_nc,
                             size_t* off_comp, size_t* off_w) {
  size_t o = align256(sizeof(float) * 8 * static_cast<size_t>(n));
  *off_cc = o;
  o += align256(sizeof(float) * 2 * static_cast<size_t>(n));
  *off_nc = o;
  o += align256(sizeof(int));
  *off_comp = o;
  o += align256(survivors_scratch_bytes(n));
  *off_w = o;
  o += align256(std::max(weights_fp32_scratch_bytes(rows, n), weights_tc_scratch_bytes(rows, n)));
  return o;
}

// reads a device error word after the stream drains; nonzero -> ABC_E_DEVICE
static int check_device_error(const unsigned* err, cudaStream_t st) {
  unsigned h = 0;
  ABC_CUDA_TRY(cudaMemcpyAsync(&h, err, sizeof h, cudaMemcpyDeviceToHost, st));
  ABC_CUDA_TRY(cudaStreamSynchronize(st));
  return h ? ABC_E_DEVICE : ABC_OK;
}

ABC_API size_t abc_weights_scratch_bytes(int64_t rows, int64_t n) {
  size_t a, b, c, d;
  return weights_layout(rows, n, &a, &b, &c, &d);
}

ABC_API int abc_weights(const float* up, const float* s, int64_t rows, const float* u,
                        const uint32_t* q, const uint64_t* prefix, int64_t n, int32_t prec,
                        double* logW, void* scratch, size_t scratch_bytes, void* stream) {
  if (rows < 0 || n < 1 || rows > kMaxIndex || n > kMaxIndex) return ABC_E_INVAL;
  if (!up || !s || !u || !q || !prefix || !logW || !scratch) return ABC_E_INVAL;
  if (prec != ABC_P_FP32 && prec != ABC_P_BF16_TC) return ABC_E_INVAL;
  size_t occ, onc, ocomp, ow;
  const size_t need = weights_layout(rows, n, &occ, &onc, &ocomp, &ow);
  if (scratch_bytes < need) return ABC_E_SCRATCH;
  char* b = static_cast<char*>(scratch);
  cudaStream_t st = as_stream(stream);
  float* cu = reinterpret_cast<float*>(b);
  float* cc = reinterpret_cast<float*>(b + occ);
  int* nc = reinterpret_cast<int*>(b + onc);
  int rc = launch_survivors(u, q, n, cu, cc, nc, b + ocomp, st);
  if (rc) return rc;
  if (prec == ABC_P_FP32)
    return launch_weights_fp32(up, s, rows, cu, cc, nc, n, prefix + (n - 1), logW, b + ow,
                               scratch_bytes - ow, st);
  unsigned* err = nullptr;
  rc = launch_weights_tc(up, s, rows, cu, cc, nc, n, prefix + (n - 1), logW, b + ow,
                         scratch_bytes - ow, &err, st);
  if (rc) return rc;
  return check_device_error(err, st);
}

ABC_API int abc_tc_probe(const void* A, const void* B, float* D, void* stream) {
  if (!A || !B || !D) return ABC_E_INVAL;
  cudaStream_t st = as_stream(stream);
  unsigned* err = nullptr;
  ABC_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&err), sizeof(unsigned), st));
  int rc = launch_tc_probe(A, B, D, err, st);
  if (rc == ABC_OK) rc = check_device_error(err, st);
  cudaFreeAsync(err, st);
  cudaStreamSynchronize(st);
  return rc;
}

static int check_predict(const abc_config* cfg, int64_t N, int64_t R, int32_t days,
                         const double* quant, int32_t nq) {
  int rc = check_config(cfg);
  if (rc) return rc;
  if (cfg->model != ABC_MODEL_SAIRD) return ABC_E_INVAL;
  if (N < 1 || N > kMaxIndex || R < 1 || R > kMaxIndex || days < 0 || days > 100000) return ABC_E_INVAL;
  if (!quant || nq < 1 || nq > 64) return ABC_E_INVAL;
  for (int i = 0; i < nq; ++i)
    if (!(quant[i] > 0.0 && quant[i] <= 1.0)) return ABC_E_INVAL;
  return ABC_OK;
}

ABC_API size_t abc_predict_scratch_bytes(int64_t N, int64_t R, int32_t days, int32_t nq) {
  if (N < 1 || R < 1 || days < 0 || nq < 1) return 0;
  return predict_scratch_bytes(N, R, days, nq);
}

ABC_API int abc_predict(const abc_config* cfg, const float* u, const double* W, int64_t N,
                        int64_t R, int32_t days, const double* quant, int32_t nq, int32_t* out,
                        void* scratch, size_t scratch_bytes, void* stream) {
  int rc = check_predict(cfg, N, R, days, quant, nq);
  if (rc) return rc;
  if (!u || !out || !scratch) return ABC_E_INVAL;
  return launch_predict(make_params(*cfg), u, W, N, R, days, quant, nq, out, scratch,
                        scratch_bytes, as_stream(stream));
}

ABC_API int abc_radix_sort(const uint32_t* keys, const int32_t* vals, int64_t n, int32_t bits,
                           uint32_t* keys_out, int32_t* vals_out, void* stream) {
  if (n < 0 || n > (int64_t(1) << 30) || bits < 1 || bits > 32) return ABC_E_INVAL;
  if (n == 0) return ABC_OK;
  if (!keys || !keys_out || !vals_out || keys == keys_out ||
      (vals && reinterpret_cast<const void*>(vals) == reinterpret_cast<const void*>(vals_out)))
    return ABC_E_INVAL;
  cudaStream_t st = as_stream(stream);
  const size_t sb = radix_sort_scratch_bytes(n);
  void* buf = nullptr;
  if (cudaMallocAsync(&buf, sb, st) != cudaSuccess) {
    cudaGetLastError();
    return ABC_E_NOMEM;
  }
  const int rc = launch_radix_sort(keys, vals, keys_out, vals_out, n, nullptr, bits, buf, sb, st);
  cudaFreeAsync(buf, st);
  return rc;
}

ABC_API int abc_ex2_probe(double* ex2_per_second, void* stream) {
  if (!ex2_per_second) return ABC_E_INVAL;
  return ex2_probe(ex2_per_second, as_stream(stream));
}

ABC_API int abc_numerics_check(int32_t which, uint64_t* mismatches, void* stream) {
  if (!mismatches) return ABC_E_INVAL;
  unsigned long long bad = 0;
  const int rc = numerics_check(which, &bad, as_stream(stream));
  *mismatches = bad;
  return rc;
}

ABC_API size_t abc_normalize_scratch_bytes(int64_t n) { return normalize_scratch_bytes(n); }

ABC_API int abc_normalize(const double* logW, int64_t n, double* W, double* ess, void* scratch,
                          size_t scratch_bytes, void* stream) {
  if (!logW || !W || !ess || !scratch) return ABC_E_INVAL;
  return launch_normalize(logW, n, W, ess, scratch, scratch_bytes, as_stream(stream));
}

ABC_API int abc_screen(const abc_config* cfg, const float* Y, const float* ystat,
                       const uint8_t* flag, int64_t M, const double* eps, uint32_t c1, float* rho,
                       uint8_t* sflag, void* stream) {
  int rc = check_config(cfg);
  if (rc) return rc;
  if (M < 0 || M > kMaxIndex) return ABC_E_INVAL;
  if (!(cfg->surrogate_tau > 0.0f) || !(cfg->surrogate_rho_min > 0.0f) ||
      !(cfg->surrogate_rho_min <= 1.0f) || !(cfg->audit_frac >= 0.0f && cfg->audit_frac <= 1.0f))
    return ABC_E_INVAL;
  if (M > 0 && (!Y || !ystat || !eps || !rho || !sflag)) return ABC_E_INVAL;
  const SimParams p = make_params(*cfg);
  return screen(Y, ystat, flag, M, eps, p.k0, p.k1, c1, cfg->surrogate_tau, cfg->surrogate_rho_min,
                cfg->audit_frac, rho, sflag, as_stream(stream), nullptr);
}

ABC_API void abc_set_wait_limit_ns(uint64_t ns) { set_tc_wait_limit(ns); }

ABC_API void abc_inject_alloc_failure(int64_t after) {
  g_alloc_fail_after.store(after < 0 ? -1 : after);
}

}  // extern "C"

// -------------------------------------------------------------- context ---
struct abc_ctx {
  abc_config cfg{};
  SimParams p{};
  cudaStream_t st = nullptr;
  int64_t N = 0, M = 0;
  int32_t T = 0;
  int cur = 0;
  int32_t gen = 0;
  double eps1_host = 0.0;
  int64_t batches_total = 0;  // run budget count (Sec. 4.1 simulation runs)
  std::vector<abc_gen_stats> stats;
  std::vector<void*> allocs;
  // device buffers
  int* spec_dev = nullptr;  // batches of the round, batches it used (spec_batches)
  int32_t* obs = nullptr;
  float* u[2] = {nullptr, nullptr};
  double* d[2] = {nullptr, nullptr};
  double* W[2] = {nullptr, nullptr};
  float* s[2] = {nullptr, nullptr};
  int32_t* anc[2] = {nullptr, nullptr};
  float* up = nullptr;
  double* dp = nullptr;
  float* sp = nullptr;
  int32_t* ap = nullptr;
  int32_t* att = nullptr;
  uint8_t* flag = nullptr;
  uint32_t* q = nullptr;
  uint64_t* prefix = nullptr;
  double* logW = nullptr;
  float* cu = nullptr;
  float* cc = nullptr;
  int* nc = nullptr;
  double* scal = nullptr;  // [0] eps, [1] eps1, [2] ess
  int64_t* cnt = nullptr;  // [0] filled, [1] accepted, [2] exhausted
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // whole generation
  cudaEvent_t es0 = nullptr, es1 = nullptr;  // one simulator launch
  cudaEvent_t ew0 = nullptr, ew1 = nullptr;  // the weight pass
  cudaEvent_t ek[4] = {nullptr, nullptr, nullptr, nullptr};  // its TC / FP32 kernels
  // surrogate (delayed-acceptance pre-screen)
  MlpState mlp{};
  float* grad = nullptr;
  float* RX = nullptr;            // ring of inputs [cap][8]
  float* RY = nullptr;            // ring of summaries [cap][4]
  long long* ring_head = nullptr; // samples appended so far
  int64_t ring_cap = 0;
  int64_t ring_host = 0;
  float* ystat = nullptr;         // output mean[4], sd[4]; input mean[8], sd[8]
  float* Yp = nullptr;            // predictions [M][4]
  float* rho = nullptr;           // pass probability per slot
  uint8_t* sflag = nullptr;
  float* cmp_u = nullptr;         // compacted simulated slots
  float* cmp_s = nullptr;
  int32_t* cmp_a = nullptr;
  float* cmp_rho = nullptr;
  uint8_t* cmp_flag = nullptr;
  uint32_t* cmp_slot = nullptr;
  double* cmp_d = nullptr;
  int32_t* ard = nullptr;         // final A, R, D [3][M]
  int* Mc = nullptr;
  float* rho_pop[2] = {nullptr, nullptr};
  float* trX = nullptr;
  float* trT = nullptr;
  float* loss = nullptr;
  unsigned long long* audit = nullptr;  // audited, audited with d <= eps
  void* sscratch = nullptr;       // surrogate scratch (training / inference / screening)
  size_t sscratch_bytes = 0;
  uint32_t* train_step = nullptr; // Adam steps so far (device)
  int* screen_on = nullptr;       // this generation screens (device)
  long long* simulated = nullptr; // slots simulated in this generation (device)
  unsigned* inf_err = nullptr;    // error word of the tensor-core inference (device)
  cudaEvent_t eq0 = nullptr, eq1 = nullptr, et0 = nullptr, et1 = nullptr;
  McmcDev* mcmc = nullptr;        // ABC_STEP_MCMC: the run's tuned step (device)

  template <typename T>
  int alloc(T** ptr, size_t count) {
    void* p = nullptr;
    if (alloc_fails_now()) return ABC_E_NOMEM;
    if (cudaMalloc(&p, std::max<size_t>(count * sizeof(T), 256)) != cudaSuccess) {
      cudaGetLastError();
      return ABC_E_NOMEM;
    }
    allocs.push_back(p);
    *ptr = static_cast<T*>(p);
    return ABC_OK;
  }
  ~abc_ctx() {
    for (void* p : allocs) cudaFree(p);
    for (cudaEvent_t e : {ev0, ev1, es0, es1, ew0, ew1, eq0, eq1, et0, et1, ek[0], ek[1], ek[2],
                          ek[3]})
      if (e) cudaEventDestroy(e);
  }
};

namespace {

// batches per device loop round of graph-captured batches (spec_batches);
// the MCMC baseline's step changes between batches: one per round
int spec_k(const abc_config& c) {
  return c.spec_batches > 1 && c.beta_mode != ABC_STEP_MCMC ? c.spec_batches : 1;
}

// The MCMC baseline's step state after generation 0: s = mcmc_s0, no
// adaptation and no batch walked with the step yet; the window is
// mcmc_adapt, or a tenth of the run budget.
McmcDev mcmc_start(const abc_config& c) {
  McmcDev m{};
  m.s = static_cast<double>(c.mcmc_s0);
  m.k = 0;
  m.batches = 0;
  m.window = c.mcmc_adapt > 0 ? c.mcmc_adapt : ceil_div(int64_t(c.max_total_batches), int64_t(10));
  m.s_f = c.mcmc_s0;
  m.s_start = c.mcmc_s0;
  return m;
}

// beta_a = the step of the generation's first batch, mcmc_s = the step after it
int mcmc_stats(const abc_ctx* c, abc_gen_stats* g) {
  if (!c->mcmc) return ABC_OK;
  McmcDev m{};
  ABC_CUDA_TRY(cudaMemcpyAsync(&m, c->mcmc, sizeof m, cudaMemcpyDeviceToHost, c->st));
  ABC_CUDA_TRY(cudaStreamSynchronize(c->st));
  g->beta_a = m.s_start;
  g->beta_b = 0;
  g->beta_bf = 0.0f;
  g->mcmc_s = m.s_f;
  return ABC_OK;
}

int ctx_alloc(abc_ctx* c) {
  const size_t N = static_cast<size_t>(c->N);
  // the proposal buffers hold the slots of spec_batches batches
  const size_t M = static_cast<size_t>(c->M) * static_cast<size_t>(spec_k(c->cfg));
  int rc = ABC_OK;
#define ABC_ALLOC(ptr, n) \
  if ((rc = c->alloc(&(ptr), (n))) != ABC_OK) return rc
  if (c->cfg.model == ABC_MODEL_SAIRD) ABC_ALLOC(c->obs, 3 * static_cast<size_t>(c->T + 1));
  for (int b = 0; b < 2; ++b) {
    ABC_ALLOC(c->u[b], 8 * N);
    ABC_ALLOC(c->d[b], N);
    ABC_ALLOC(c->W[b], N);
    ABC_ALLOC(c->s[b], N);
    ABC_ALLOC(c->anc[b], N);
  }
  ABC_ALLOC(c->spec_dev, 2);
  ABC_ALLOC(c->up, 8 * M);
  ABC_ALLOC(c->dp, M);
  ABC_ALLOC(c->sp, M);
  ABC_ALLOC(c->ap, M);
  ABC_ALLOC(c->att, M);
  ABC_ALLOC(c->flag, M);
  ABC_ALLOC(c->q, N);
  ABC_ALLOC(c->prefix, N);
  ABC_ALLOC(c->logW, N);
  if (c->cfg.weight_mode == ABC_W_IMPORTANCE) {
    ABC_ALLOC(c->cu, 8 * N);
    ABC_ALLOC(c->cc, 2 * N);  // c_k as a double-float (hi, lo halves)
    ABC_ALLOC(c->nc, 1);
  }
  ABC_ALLOC(c->scal, 4);
  ABC_ALLOC(c->cnt, 4);
  if (c->cfg.beta_mode == ABC_STEP_MCMC) ABC_ALLOC(c->mcmc, 1);
  if (c->cfg.surrogate) {
    const int B = c->cfg.surrogate_batch;
    c->ring_cap = c->cfg.surrogate_ring > 0
                      ? c->cfg.surrogate_ring
                      : std::min<int64_t>(int64_t(1) << 21, 16 * std::max<int64_t>(c->N, 4096));
    ABC_ALLOC(c->mlp.w, kMlpParams);
    ABC_ALLOC(c->mlp.wb, kMlpParams);
    ABC_ALLOC(c->mlp.m, kMlpParams);
    ABC_ALLOC(c->mlp.v, kMlpParams);
    ABC_ALLOC(c->grad, kMlpParams);
    ABC_ALLOC(c->RX, 8 * static_cast<size_t>(c->ring_cap));
    ABC_ALLOC(c->RY, 4 * static_cast<size_t>(c->ring_cap));
    ABC_ALLOC(c->ring_head, 1);
    ABC_ALLOC(c->ystat, 24);
    ABC_ALLOC(c->Yp, 4 * M);
    ABC_ALLOC(c->rho, M);
    ABC_ALLOC(c->sflag, M);
    ABC_ALLOC(c->cmp_u, 8 * M);
    ABC_ALLOC(c->cmp_s, M);
    ABC_ALLOC(c->cmp_a, M);
    ABC_ALLOC(c->cmp_rho, M);
    ABC_ALLOC(c->cmp_flag, M);
    ABC_ALLOC(c->cmp_slot, M);
    ABC_ALLOC(c->cmp_d, M);
    ABC_ALLOC(c->ard, 3 * std::max(M, N));
    ABC_ALLOC(c->Mc, 1);
    ABC_ALLOC(c->rho_pop[0], N);
    ABC_ALLOC(c->rho_pop[1], N);
    ABC_ALLOC(c->trX, 8 * static_cast<size_t>(B));
    ABC_ALLOC(c->trT, 4 * static_cast<size_t>(B));
    ABC_ALLOC(c->loss, 1);
    ABC_ALLOC(c->audit, 2);
    ABC_ALLOC(c->train_step, 1);
    ABC_ALLOC(c->screen_on, 1);
    ABC_ALLOC(c->simulated, 1);
    ABC_ALLOC(c->inf_err, 1);
    c->sscratch_bytes = std::max({mlp_train_scratch_bytes(B), mlp_infer_scratch_bytes(c->M),
                                  ring_stats_scratch_bytes(),
                                  screen_scratch_bytes(c->M),
                                  ring_scratch_bytes(std::max(c->M, c->N))});
    char* ss = nullptr;
    if ((rc = c->alloc(&ss, c->sscratch_bytes)) != ABC_OK) return rc;
    c->sscratch = ss;
  }
#undef ABC_ALLOC
  size_t sb = std::max({select_scratch_bytes(c->N), prefix_scratch_bytes(c->N),
                        accept_scratch_bytes(c->M), survivors_scratch_bytes(c->N),
                        spec_k(c->cfg) > 1 ? accept_spec_scratch_bytes(c->M, spec_k(c->cfg))
                                           : size_t(0),
                        normalize_scratch_bytes(c->N), sim_order_scratch_bytes(c->N),
                        sim_order_scratch_bytes(c->M * spec_k(c->cfg))});
  if (c->cfg.weight_mode == ABC_W_IMPORTANCE)  // room for the tuner's chunk multipliers (<= 4)
    sb = std::max(sb, c->cfg.weight_prec == ABC_P_BF16_TC ? weights_tc_scratch_bytes(c->N, c->N, 4)
                                                          : weights_fp32_scratch_bytes(c->N, c->N, 4));
  c->scratch_bytes = sb;
  char* sc = nullptr;
  if ((rc = c->alloc(&sc, sb)) != ABC_OK) return rc;
  c->scratch = sc;
  return ABC_OK;
}

// the surrogate buffers of a context; rho_pop of population buffer `nxt`
SurView sur_view(abc_ctx* c, int nxt) {
  SurView v;
  if (!c->cfg.surrogate) return v;
  v.on = true;
  v.mlp = c->mlp;
  v.ystat = c->ystat;
  v.Yp = c->Yp;
  v.rho = c->rho;
  v.sflag = c->sflag;
  v.cmp_u = c->cmp_u;
  v.cmp_s = c->cmp_s;
  v.cmp_rho = c->cmp_rho;
  v.cmp_a = c->cmp_a;
  v.cmp_flag = c->cmp_flag;
  v.cmp_slot = c->cmp_slot;
  v.cmp_d = c->cmp_d;
  v.ard = c->ard;
  v.Mc = c->Mc;
  v.rho_pop = c->rho_pop[nxt];
  v.RX = c->RX;
  v.RY = c->RY;
  v.ring_head = c->ring_head;
  v.ring_cap = c->ring_cap;
  v.grad = c->grad;
  v.trX = c->trX;
  v.trT = c->trT;
  v.loss = c->loss;
  v.audit = c->audit;
  v.inf_err = c->inf_err;
  v.simulated = c->simulated;
  v.train_step = c->train_step;
  v.screen_on = c->screen_on;
  v.sscratch = c->sscratch;
  v.sscratch_bytes = c->sscratch_bytes;
  v.start = c->cfg.surrogate_start;
  v.steps = c->cfg.surrogate_steps;
  v.batch = c->cfg.surrogate_batch;
  v.lr = c->cfg.surrogate_lr;
  v.tau = c->cfg.surrogate_tau;
  v.rho_min = c->cfg.surrogate_rho_min;
  v.audit_frac = c->cfg.audit_frac;
  return v;
}

int generation0(abc_ctx* c) {
  cudaStream_t st = c->st;
  const int cur = c->cur;
  int rc = launch_prior(c->p, c->N, c->u[cur], st);
  if (rc) return rc;
  ABC_CUDA_TRY(cudaEventRecord(c->es0, st));
  rc = launch_simulate_ordered(c->p, c->obs, c->u[cur], c->N, 0u, nullptr, c->d[cur], c->scratch,
                               c->scratch_bytes, st, nullptr, nullptr, 128, 0, nullptr, nullptr,
                               c->cfg.surrogate ? c->ard : nullptr);
  if (rc) return rc;
  ABC_CUDA_TRY(cudaEventRecord(c->es1, st));
  if (c->cfg.surrogate &&
      (rc = ring_append(nullptr, c->N, c->u[cur], c->d[cur], c->ard, c->ring_head, c->ring_cap, c->RX,
                        c->RY, c->sscratch, st)))
    return rc;
  if ((rc = launch_fill(c->W[cur], c->N, 1.0 / static_cast<double>(c->N), st))) return rc;
  ABC_CUDA_TRY(cudaMemsetAsync(c->anc[cur], 0xFF, sizeof(int32_t) * c->N, st));
  ABC_CUDA_TRY(cudaMemsetAsync(c->s[cur], 0, sizeof(float) * c->N, st));
  McmcDev m0{};
  if (c->mcmc) {
    m0 = mcmc_start(c->cfg);
    ABC_CUDA_TRY(cudaMemcpyAsync(c->mcmc, &m0, sizeof m0, cudaMemcpyHostToDevice, st));
  }
  abc_gen_stats g{};
  g.generation = 0;
  g.status = ABC_OK;
  g.eps = INFINITY;
  g.ess = static_cast<double>(c->N);
  g.beta_b = 0;
  g.batches = 1;
  g.sims = c->N;
  g.sim_days = c->N * static_cast<int64_t>(c->cfg.model == ABC_MODEL_SAIRD ? c->T : 1);
  g.accepted = c->N;
  ABC_CUDA_TRY(cudaEventSynchronize(c->es1));
  float ms = 0.f;
  ABC_CUDA_TRY(cudaEventElapsedTime(&ms, c->es0, c->es1));
  g.ms_sim = ms;
  c->stats.push_back(g);
  return ABC_OK;
}

int generation_t(abc_ctx* c) {
  cudaStream_t st = c->st;
  const int32_t t = c->gen;
  const int cur = c->cur, nxt = 1 - c->cur;
  const int paper_beta = c->cfg.beta_mode == ABC_BETA_PAPER;
  // paper schedule: integer b = 2t up to stage 512, then 0 (the Gamma ratio)
  const int32_t bb = paper_beta ? (t <= 512 ? 2 * t : 0)
                                : c->cfg.beta_mode == ABC_BETA_FIXED ? c->cfg.beta_b : 0;
  if (t > 32767) return ABC_E_INVAL;
  BetaRule rule = beta_rule(c->cfg);
  rule.b = bb;
  double* eps = c->scal + 0;
  double* eps1 = c->scal + 1;
  double* ess = c->scal + 2;
  int64_t k = static_cast<int64_t>(std::ceil(c->cfg.survival_alpha * static_cast<double>(c->N)));
  k = std::min<int64_t>(std::max<int64_t>(k, 1), c->N);
  int rc = launch_select(c->d[cur], c->N, k, eps, c->scratch, c->scratch_bytes, st);
  if (rc) return rc;
  if (t == 1) ABC_CUDA_TRY(cudaMemcpyAsync(eps1, eps, sizeof(double), cudaMemcpyDeviceToDevice, st));
  rc = launch_resample_prefix(c->d[cur], c->W[cur], c->N, eps, c->cfg.weight_mode, c->q, c->prefix,
                              c->scratch, c->scratch_bytes, st);
  if (rc) return rc;
  ABC_CUDA_TRY(cudaMemsetAsync(c->cnt, 0, 4 * sizeof(int64_t), st));
  const bool sur = c->cfg.surrogate != 0;
  const SurView sv = sur_view(c, nxt);
  unsigned* inf_err = nullptr;
  unsigned h_inf_err = 0;
  if (sur) {
    // screening from generation surrogate_start once the surrogate has been
    // trained (decided on the device); this generation's counters
    if ((rc = sur_gate(nullptr, static_cast<uint32_t>(t), sv.start, sv.train_step, sv.screen_on,
                       st)))
      return rc;
    ABC_CUDA_TRY(cudaMemsetAsync(c->audit, 0, 2 * sizeof(unsigned long long), st));
    ABC_CUDA_TRY(cudaMemsetAsync(c->simulated, 0, sizeof(long long), st));
    inf_err = c->inf_err;
    ABC_CUDA_TRY(cudaMemsetAsync(inf_err, 0, sizeof(unsigned), st));
  }
  if (c->mcmc && (rc = launch_mcmc_begin(c->mcmc, nullptr, st))) return rc;
  const float* s_fix = c->mcmc ? &c->mcmc->s_f : nullptr;
  int64_t filled = 0;
  double ms_sim = 0.0, ms_screen = 0.0;
  int32_t b = 0;
  // several batches per round (spec_batches, without the surrogate): K M
  // slots proposed and simulated together, accepted in (batch, slot) order
  const int K = sur ? 1 : spec_k(c->cfg);
  int used = 1;
  for (b = 0; b < c->cfg.max_batches && filled < c->N; b += used) {
    const uint32_t c1 = (static_cast<uint32_t>(t) << 16) | static_cast<uint32_t>(b);
    used = 1;
    if (K > 1) {
      const int klim = std::min(K, c->cfg.max_batches - b);
      ABC_CUDA_TRY(cudaMemcpyAsync(c->spec_dev, &klim, sizeof klim, cudaMemcpyHostToDevice, st));
      rc = launch_propose(c->p, c->u[cur], c->N, c->prefix, rule, eps, eps1, c->M * K, nullptr,
                          c1, c->cfg.max_redraw, c->up, c->sp, c->ap, c->att, c->flag, st,
                          nullptr, nullptr, nullptr, c->M, c->spec_dev);
      if (rc) return rc;
      ABC_CUDA_TRY(cudaEventRecord(c->es0, st));
      rc = launch_simulate_ordered(c->p, c->obs, c->up, c->M * K, c1, c->flag, c->dp, c->scratch,
                                   c->scratch_bytes, st, nullptr, nullptr, 128, c->M);
      if (rc) return rc;
      ABC_CUDA_TRY(cudaEventRecord(c->es1, st));
      rc = launch_accept_spec(c->up, c->dp, c->sp, c->ap, c->flag, c->M, K, c->spec_dev, eps,
                              c->N, c->u[nxt], c->d[nxt], c->s[nxt], c->anc[nxt], c->cnt,
                              c->cnt + 1, c->spec_dev + 1, c->scratch, c->scratch_bytes, st);
      if (rc) return rc;
      ABC_CUDA_TRY(cudaMemcpyAsync(&filled, c->cnt, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
      ABC_CUDA_TRY(cudaMemcpyAsync(&used, c->spec_dev + 1, sizeof used, cudaMemcpyDeviceToHost,
                                   st));
      ABC_CUDA_TRY(cudaStreamSynchronize(st));
      float ms = 0.f;
      ABC_CUDA_TRY(cudaEventElapsedTime(&ms, c->es0, c->es1));
      ms_sim += ms;
      continue;
    }
    rc = launch_propose(c->p, c->u[cur], c->N, c->prefix, rule, eps, eps1, c->M, nullptr, c1,
                        c->cfg.max_redraw, c->up, c->sp, c->ap, c->att, c->flag, st, nullptr,
                        nullptr, nullptr, 0, nullptr, s_fix);
    if (rc) return rc;
    if (sur) {
      // delayed acceptance (a pass-all until the surrogate is trained):
      // predict, screen, simulate only the compacted slots
      const cudaEvent_t ev[3] = {c->eq0, c->es0, c->es1};
      rc = screened_batch(sv, c->p, c->obs, c->up, c->sp, c->ap, c->flag, c->M, eps, c1, nullptr,
                          c->N, c->u[nxt], c->d[nxt], c->s[nxt], c->anc[nxt], c->cnt, c->cnt + 1,
                          reinterpret_cast<unsigned long long*>(c->cnt + 2), c->scratch,
                          c->scratch_bytes, 128, nullptr, st, ev);
      if (rc) return rc;
    } else {
      ABC_CUDA_TRY(cudaEventRecord(c->es0, st));
      rc = launch_simulate_ordered(c->p, c->obs, c->up, c->M, c1, c->flag, c->dp, c->scratch,
                                   c->scratch_bytes, st);
      if (rc) return rc;
      ABC_CUDA_TRY(cudaEventRecord(c->es1, st));
      rc = launch_accept(c->up, c->dp, c->sp, c->ap, c->flag, c->M, eps, c->N, c->u[nxt], c->d[nxt],
                         c->s[nxt], c->anc[nxt], c->cnt, c->cnt + 1, c->scratch, c->scratch_bytes,
                         st);
      if (rc) return rc;
      // the MCMC baseline adapts its step to this batch's acceptance
      if (c->mcmc &&
          (rc = launch_mcmc_adapt(c->mcmc, reinterpret_cast<const long long*>(c->cnt + 1), c->M,
                                  nullptr, st)))
        return rc;
    }
    ABC_CUDA_TRY(cudaMemcpyAsync(&filled, c->cnt, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    ABC_CUDA_TRY(cudaStreamSynchronize(st));
    float ms = 0.f;
    ABC_CUDA_TRY(cudaEventElapsedTime(&ms, c->es0, c->es1));
    ms_sim += ms;
    if (sur) {
      ABC_CUDA_TRY(cudaEventElapsedTime(&ms, c->eq0, c->es0));
      ms_screen += ms;
    }
  }
  int64_t h_cnt[3];
  ABC_CUDA_TRY(cudaMemcpyAsync(h_cnt, c->cnt, sizeof h_cnt, cudaMemcpyDeviceToHost, st));
  unsigned long long h_audit[2] = {0, 0};
  long long simulated = 0;
  if (sur) {
    ABC_CUDA_TRY(cudaMemcpyAsync(h_audit, c->audit, sizeof h_audit, cudaMemcpyDeviceToHost, st));
    ABC_CUDA_TRY(cudaMemcpyAsync(&simulated, c->simulated, sizeof simulated,
                                 cudaMemcpyDeviceToHost, st));
    ABC_CUDA_TRY(cudaMemcpyAsync(&h_inf_err, inf_err, sizeof h_inf_err, cudaMemcpyDeviceToHost,
                                 st));
  }
  ABC_CUDA_TRY(cudaStreamSynchronize(st));
  if (h_inf_err) return ABC_E_DEVICE;
  abc_gen_stats g{};
  g.generation = t;
  g.batches = b;
  g.accepted = h_cnt[1];
  g.ms_screen = ms_screen;
  if (sur) {
    // every slot is exhausted (never simulated), passed, or screened out;
    // audited slots were screened out and simulated anyway
    g.exhausted = h_cnt[2];
    g.sims = simulated;
    g.audited = static_cast<int64_t>(h_audit[0]);
    g.audit_accepted = static_cast<int64_t>(h_audit[1]);
    g.screened = static_cast<int64_t>(b) * c->M - g.exhausted - (simulated - g.audited);
  } else {
    g.exhausted = h_cnt[2];
    g.sims = static_cast<int64_t>(b) * c->M - h_cnt[2];
  }
  g.sim_days = g.sims * static_cast<int64_t>(c->cfg.model == ABC_MODEL_SAIRD ? c->T : 1);
  g.ms_sim = ms_sim;
  int h_nc = 0;
  int h_counts[4] = {0, 0, 0, 0};
  unsigned long long h_tiles = 0;
  WeightTiming wt;
  wt.tc0 = c->ek[0];
  wt.tc1 = c->ek[1];
  wt.fp0 = c->ek[2];
  wt.fp1 = c->ek[3];
  bool weighted = false;
  unsigned* tc_err = nullptr;
  unsigned h_err = 0;
  if (filled < c->N) {
    g.status = ABC_STOP_BUDGET;
  } else {
    g.status = ABC_OK;
    if (c->cfg.weight_mode == ABC_W_IMPORTANCE) {
      rc = launch_survivors(c->u[cur], c->q, c->N, c->cu, c->cc, c->nc, c->scratch, st);
      if (rc) return rc;
      ABC_CUDA_TRY(cudaEventRecord(c->ew0, st));
      if (c->cfg.weight_prec == ABC_P_BF16_TC)
        rc = launch_weights_tc(c->u[nxt], c->s[nxt], c->N, c->cu, c->cc, c->nc, c->N,
                               c->prefix + (c->N - 1), c->logW, c->scratch, c->scratch_bytes,
                               &tc_err, st, nullptr, 1, nullptr,
                               AncInfo{c->anc[nxt], c->u[cur], c->q, c->N}, &wt);
      else
        rc = launch_weights_fp32(c->u[nxt], c->s[nxt], c->N, c->cu, c->cc, c->nc, c->N,
                                 c->prefix + (c->N - 1), c->logW, c->scratch, c->scratch_bytes,
                                 st, nullptr, 1, nullptr, &wt);
      if (rc) return rc;
      ABC_CUDA_TRY(cudaEventRecord(c->ew1, st));
      if (tc_err) ABC_CUDA_TRY(cudaMemcpyAsync(&h_err, tc_err, sizeof h_err, cudaMemcpyDeviceToHost, st));
      ABC_CUDA_TRY(cudaMemcpyAsync(&h_nc, c->nc, sizeof(int), cudaMemcpyDeviceToHost, st));
      if (wt.counts)
        ABC_CUDA_TRY(cudaMemcpyAsync(h_counts, wt.counts, sizeof h_counts, cudaMemcpyDeviceToHost, st));
      if (wt.tiles)
        ABC_CUDA_TRY(cudaMemcpyAsync(&h_tiles, wt.tiles, sizeof h_tiles, cudaMemcpyDeviceToHost, st));
      weighted = true;
      // delayed acceptance: a proposal simulated with probability rho carries 1/rho
      if (sur && (rc = rho_correct(c->logW, sv.rho_pop, c->N, st))) return rc;
      rc = launch_normalize(c->logW, c->N, c->W[nxt], ess, c->scratch, c->scratch_bytes, st);
      if (rc) return rc;
    } else {
      if ((rc = launch_fill(c->W[nxt], c->N, 1.0 / static_cast<double>(c->N), st))) return rc;
      if ((rc = launch_fill(ess, 1, static_cast<double>(c->N), st))) return rc;
    }
  }
  double h_scal[3];
  ABC_CUDA_TRY(cudaMemcpyAsync(h_scal, c->scal, sizeof h_scal, cudaMemcpyDeviceToHost, st));
  ABC_CUDA_TRY(cudaStreamSynchronize(st));
  if (h_err) return ABC_E_DEVICE;
  if (weighted) {
    float ms = 0.f;
    ABC_CUDA_TRY(cudaEventElapsedTime(&ms, c->ew0, c->ew1));
    g.ms_weights = ms;
    g.pairs = c->N * static_cast<int64_t>(h_nc);
    // per-kernel split of the pass (FP32 only: every row on the FP32 kernel)
    const bool tc = c->cfg.weight_prec == ABC_P_BF16_TC;
    g.rows_tc = tc ? h_counts[1] : 0;
    g.rows_exp = tc ? h_counts[2] : 0;
    g.pairs_tc = tc ? static_cast<int64_t>(h_tiles) * weights_tc_tile_pairs() : 0;
    if (tc && h_counts[1] > 0) {
      ABC_CUDA_TRY(cudaEventElapsedTime(&ms, c->ek[0], c->ek[1]));
      g.ms_tc = ms;
    }
    if (!tc || h_counts[0] > 0) {
      ABC_CUDA_TRY(cudaEventElapsedTime(&ms, c->ek[2], c->ek[3]));
      g.ms_fp32 = ms;
    }
  }
  g.eps = h_scal[0];
  g.eps1 = h_scal[1];
  g.ess = g.status == ABC_OK ? h_scal[2] : 0.0;
  stage_shapes(c->cfg, h_scal[0], h_scal[1], t, bb, &g);
  if ((rc = mcmc_stats(c, &g))) return rc;
  c->eps1_host = h_scal[1];
  if (sur && g.status == ABC_OK && c->cfg.surrogate_steps > 0) {
    // train on everything simulated so far (the ring keeps the latest pairs)
    ABC_CUDA_TRY(cudaEventRecord(c->et0, st));
    if ((rc = sur_train(sv, c->p, nullptr, st))) return rc;
    ABC_CUDA_TRY(cudaEventRecord(c->et1, st));
    float lh = 0.f, mt = 0.f;
    ABC_CUDA_TRY(cudaMemcpyAsync(&lh, c->loss, sizeof lh, cudaMemcpyDeviceToHost, st));
    ABC_CUDA_TRY(cudaMemcpyAsync(&h_inf_err, inf_err, sizeof h_inf_err, cudaMemcpyDeviceToHost, st));
    ABC_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_inf_err) return ABC_E_DEVICE;
    ABC_CUDA_TRY(cudaEventElapsedTime(&mt, c->et0, c->et1));
    g.train_loss = lh / (4.0 * c->cfg.surrogate_batch);
    g.ms_train = mt;
  }
  c->stats.push_back(g);
  if (g.status == ABC_OK) c->cur = nxt;
  return g.status;
}

}  // namespace

extern "C" {

ABC_API int abc_init(const abc_config* cfg, const int32_t* obs, void* stream, abc_ctx** out) {
  if (!out) return ABC_E_INVAL;
  *out = nullptr;
  int rc = check_config(cfg);
  if (rc) return rc;
  if ((rc = check_smc(cfg))) return rc;
  if (cfg->model == ABC_MODEL_SAIRD && !obs) return ABC_E_INVAL;
  abc_ctx* c = new (std::nothrow) abc_ctx();
  if (!c) return ABC_E_NOMEM;
  c->cfg = *cfg;
  c->p = make_params(*cfg);
  c->st = as_stream(stream);
  c->N = cfg->n_particles;
  c->M = cfg->batch_size > 0 ? cfg->batch_size : cfg->n_particles;
  c->T = cfg->model == ABC_MODEL_SAIRD ? cfg->n_days : 0;
  if (c->M * spec_k(*cfg) > kMaxIndex) {
    delete c;
    return ABC_E_INVAL;
  }
  if ((rc = ctx_alloc(c)) != ABC_OK) {
    delete c;
    return rc;
  }
  if (cfg->weight_mode == ABC_W_IMPORTANCE && cfg->weight_prec == ABC_P_BF16_TC &&
      (rc = weights_tc_prepare()) != ABC_OK) {
    delete c;
    return rc;
  }
  if (cfg->surrogate) {
    if (cudaEventCreate(&c->eq0) != cudaSuccess || cudaEventCreate(&c->eq1) != cudaSuccess ||
        cudaEventCreate(&c->et0) != cudaSuccess || cudaEventCreate(&c->et1) != cudaSuccess ||
        cudaMemsetAsync(c->ring_head, 0, sizeof(long long), c->st) != cudaSuccess ||
        cudaMemsetAsync(c->train_step, 0, sizeof(uint32_t), c->st) != cudaSuccess ||
        // compacted slots past a batch's count are read as flags: never 1
        cudaMemsetAsync(c->cmp_flag, 0, static_cast<size_t>(c->M), c->st) != cudaSuccess) {
      delete c;
      return ABC_E_CUDA;
    }
    if ((rc = mlp_infer_prepare()) != ABC_OK || (rc = mlp_train_prepare()) != ABC_OK ||
        (rc = mlp_init(c->mlp, c->p.k0, c->p.k1, c->st)) != ABC_OK ||
        (rc = stats_init(c->ystat, c->st)) != ABC_OK) {
      delete c;
      return rc;
    }
  }
  if (c->obs) {
    if (cudaMemcpyAsync(c->obs, obs, sizeof(int32_t) * 3 * (c->T + 1), cudaMemcpyHostToDevice,
                        c->st) != cudaSuccess) {
      delete c;
      return ABC_E_CUDA;
    }
  }
  if (cudaMemsetAsync(c->scal, 0, 4 * sizeof(double), c->st) != cudaSuccess ||
      cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess ||
      cudaEventCreate(&c->es0) != cudaSuccess || cudaEventCreate(&c->es1) != cudaSuccess ||
      cudaEventCreate(&c->ew0) != cudaSuccess || cudaEventCreate(&c->ew1) != cudaSuccess ||
      cudaEventCreate(&c->ek[0]) != cudaSuccess || cudaEventCreate(&c->ek[1]) != cudaSuccess ||
      cudaEventCreate(&c->ek[2]) != cudaSuccess || cudaEventCreate(&c->ek[3]) != cudaSuccess ||
      cudaStreamSynchronize(c->st) != cudaSuccess) {
    delete c;
    return ABC_E_CUDA;
  }
  *out = c;
  return ABC_OK;
}

ABC_API int abc_generation(abc_ctx* c) {
  if (!c) return ABC_E_INVAL;
  // run budget: the generation that reached it was the last
  if (c->gen > 0 && c->cfg.max_total_batches > 0 &&
      c->batches_total >= c->cfg.max_total_batches)
    return ABC_STOP_TOTAL;
  // tolerance target reached by the last generation
  if (c->gen > 1 && c->cfg.eps_stop > 0.0f &&
      c->stats.back().eps <= static_cast<double>(c->cfg.eps_stop))
    return ABC_STOP_TARGET;
  ABC_CUDA_TRY(cudaEventRecord(c->ev0, c->st));
  const int64_t l0 = g_launches.load();
  const bool first = c->gen == 0;
  const int rc = first ? generation0(c) : generation_t(c);
  if (rc < 0) return rc;
  // stage 0 stands for its N prior draws in batches of M simulations
  c->batches_total += first ? ceil_div(c->N, c->M) : c->stats.back().batches;
  c->stats.back().launches = g_launches.load() - l0;
  ABC_CUDA_TRY(cudaEventRecord(c->ev1, c->st));
  ABC_CUDA_TRY(cudaEventSynchronize(c->ev1));
  float ms = 0.f;
  ABC_CUDA_TRY(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  c->stats.back().ms = ms;
  if (rc == ABC_OK) c->gen += 1;
  return rc;
}

ABC_API int abc_run(abc_ctx* c, int32_t n_generations, double eps_target) {
  if (!c || n_generations < 0) return ABC_E_INVAL;
  int rc = ABC_OK;
  while (c->gen < n_generations) {
    rc = abc_generation(c);
    if (rc != ABC_OK) return rc;
    if (eps_target > 0.0 && c->gen > 1 && c->stats.back().eps <= eps_target) return ABC_STOP_TARGET;
  }
  return rc;
}

ABC_API int abc_reset(abc_ctx* c, uint32_t run_id) {
  if (!c) return ABC_E_INVAL;
  ABC_CUDA_TRY(cudaStreamSynchronize(c->st));
  c->cfg.run_id = run_id;
  c->p = make_params(c->cfg);
  c->gen = 0;
  c->cur = 0;
  c->eps1_host = 0.0;
  c->batches_total = 0;
  c->stats.clear();
  ABC_CUDA_TRY(cudaMemsetAsync(c->scal, 0, 4 * sizeof(double), c->st));
  if (c->cfg.surrogate) {
    ABC_CUDA_TRY(cudaMemsetAsync(c->train_step, 0, sizeof(uint32_t), c->st));
    ABC_CUDA_TRY(cudaMemsetAsync(c->ring_head, 0, sizeof(long long), c->st));
    int rc = mlp_init(c->mlp, c->p.k0, c->p.k1, c->st);
    if (!rc) rc = stats_init(c->ystat, c->st);
    if (rc) return rc;
  }
  ABC_CUDA_TRY(cudaStreamSynchronize(c->st));
  return ABC_OK;
}

ABC_API int abc_get_population(abc_ctx* c, float* u, double* dist, double* W, float* s,
                               int32_t* anc, int32_t on_device) {
  if (!c || c->gen == 0) return ABC_E_INVAL;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  const int k = c->cur;
  const size_t N = static_cast<size_t>(c->N);
  if (u) ABC_CUDA_TRY(cudaMemcpyAsync(u, c->u[k], 8 * N * sizeof(float), kind, c->st));
  if (dist) ABC_CUDA_TRY(cudaMemcpyAsync(dist, c->d[k], N * sizeof(double), kind, c->st));
  if (W) ABC_CUDA_TRY(cudaMemcpyAsync(W, c->W[k], N * sizeof(double), kind, c->st));
  if (s) ABC_CUDA_TRY(cudaMemcpyAsync(s, c->s[k], N * sizeof(float), kind, c->st));
  if (anc) ABC_CUDA_TRY(cudaMemcpyAsync(anc, c->anc[k], N * sizeof(int32_t), kind, c->st));
  if (!on_device) ABC_CUDA_TRY(cudaStreamSynchronize(c->st));
  return ABC_OK;
}

ABC_API int abc_get_stats(abc_ctx* c, int32_t t, abc_gen_stats* out) {
  if (!c || !out || t < 0 || t >= static_cast<int32_t>(c->stats.size())) return ABC_E_INVAL;
  *out = c->stats[static_cast<size_t>(t)];
  return ABC_OK;
}

ABC_API int abc_predict_population(abc_ctx* c, int64_t R, int32_t days, const double* quant,
                                   int32_t nq, int32_t* out_host) {
  if (!c || !out_host) return ABC_E_INVAL;
  int rc = check_predict(&c->cfg, c->N, R, days, quant, nq);
  if (rc) return rc;
  const size_t sb = predict_scratch_bytes(c->N, R, days, nq);
  const size_t ob = sizeof(int32_t) * static_cast<size_t>(days + 1) * 3 * nq;
  char* buf = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&buf), sb + align256(ob), c->st) != cudaSuccess)
    return ABC_E_NOMEM;
  auto* out = reinterpret_cast<int32_t*>(buf + sb);
  const bool weighted = c->cfg.weight_mode == ABC_W_IMPORTANCE;
  rc = launch_predict(c->p, c->u[c->cur], weighted ? c->W[c->cur] : nullptr, c->N, R, days, quant,
                      nq, out, buf, sb, c->st);
  if (rc == ABC_OK &&
      (cudaMemcpyAsync(out_host, out, ob, cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
       cudaStreamSynchronize(c->st) != cudaSuccess))
    rc = ABC_E_CUDA;
  cudaFreeAsync(buf, c->st);
  cudaStreamSynchronize(c->st);
  return rc;
}

ABC_API int32_t abc_generations(const abc_ctx* c) { return c ? c->gen : 0; }

namespace {
struct StateHeader {
  char magic[8];
  int64_t N, T;
  uint64_t seed;
  uint32_t run_id;
  int32_t gen;
  double eps1;
  int64_t batches_total;  // run budget count
};
// ABC_STEP_MCMC state after the population: s (f64), k and batches (i64)
constexpr size_t kMcmcTrailer = sizeof(double) + 2 * sizeof(long long);
}  // namespace

ABC_API int abc_get_state(abc_ctx* c, void* buf, size_t* len) {
  if (!c || !len) return ABC_E_INVAL;
  const size_t N = static_cast<size_t>(c->N);
  // the MCMC baseline's step state (s, adaptations, batches) trails the population
  const size_t need = sizeof(StateHeader) +
                      N * (8 * sizeof(float) + 2 * sizeof(double) + sizeof(float) +
                           sizeof(int32_t)) +
                      (c->mcmc ? kMcmcTrailer : 0);
  if (!buf) {
    *len = need;
    return ABC_OK;
  }
  if (*len < need || c->gen == 0) return ABC_E_INVAL;
  StateHeader h{};
  std::memcpy(h.magic, "ABCSMC02", 8);
  h.N = c->N;
  h.T = c->T;
  h.seed = c->cfg.seed;
  h.run_id = c->cfg.run_id;
  h.gen = c->gen;
  h.eps1 = c->eps1_host;
  h.batches_total = c->batches_total;
  char* p = static_cast<char*>(buf);
  std::memcpy(p, &h, sizeof h);
  p += sizeof h;
  const int k = c->cur;
  ABC_CUDA_TRY(cudaMemcpyAsync(p, c->u[k], 8 * N * sizeof(float), cudaMemcpyDeviceToHost, c->st));
  p += 8 * N * sizeof(float);
  ABC_CUDA_TRY(cudaMemcpyAsync(p, c->d[k], N * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  p += N * sizeof(double);
  ABC_CUDA_TRY(cudaMemcpyAsync(p, c->W[k], N * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  p += N * sizeof(double);
  ABC_CUDA_TRY(cudaMemcpyAsync(p, c->s[k], N * sizeof(float), cudaMemcpyDeviceToHost, c->st));
  p += N * sizeof(float);
  ABC_CUDA_TRY(cudaMemcpyAsync(p, c->anc[k], N * sizeof(int32_t), cudaMemcpyDeviceToHost, c->st));
  McmcDev m{};
  if (c->mcmc)
    ABC_CUDA_TRY(cudaMemcpyAsync(&m, c->mcmc, sizeof m, cudaMemcpyDeviceToHost, c->st));
  ABC_CUDA_TRY(cudaStreamSynchronize(c->st));
  if (c->mcmc) {
    p += N * sizeof(int32_t);
    const long long kb[2] = {m.k, m.batches};
    std::memcpy(p, &m.s, sizeof(double));
    std::memcpy(p + sizeof(double), kb, sizeof kb);
  }
  *len = need;
  return ABC_OK;
}

ABC_API int abc_set_state(abc_ctx* c, const void* buf, size_t len) {
  if (!c || !buf || len < sizeof(StateHeader)) return ABC_E_INVAL;
  StateHeader h;
  std::memcpy(&h, buf, sizeof h);
  const size_t N = static_cast<size_t>(c->N);
  const size_t need = sizeof(StateHeader) +
                      N * (8 * sizeof(float) + 2 * sizeof(double) + sizeof(float) +
                           sizeof(int32_t)) +
                      (c->mcmc ? kMcmcTrailer : 0);
  if (std::memcmp(h.magic, "ABCSMC02", 8) != 0 || h.N != c->N || h.T != c->T || len < need ||
      h.gen < 1 || h.gen > 32767 || h.batches_total < 0)
    return ABC_E_STATE;
  const char* p = static_cast<const char*>(buf) + sizeof h;
  const int k = c->cur;
  ABC_CUDA_TRY(cudaMemcpyAsync(c->u[k], p, 8 * N * sizeof(float), cudaMemcpyHostToDevice, c->st));
  p += 8 * N * sizeof(float);
  ABC_CUDA_TRY(cudaMemcpyAsync(c->d[k], p, N * sizeof(double), cudaMemcpyHostToDevice, c->st));
  p += N * sizeof(double);
  ABC_CUDA_TRY(cudaMemcpyAsync(c->W[k], p, N * sizeof(double), cudaMemcpyHostToDevice, c->st));
  p += N * sizeof(double);
  ABC_CUDA_TRY(cudaMemcpyAsync(c->s[k], p, N * sizeof(float), cudaMemcpyHostToDevice, c->st));
  p += N * sizeof(float);
  ABC_CUDA_TRY(cudaMemcpyAsync(c->anc[k], p, N * sizeof(int32_t), cudaMemcpyHostToDevice, c->st));
  McmcDev m{};
  if (c->mcmc) {
    p += N * sizeof(int32_t);
    long long kb[2];
    m = mcmc_start(c->cfg);
    std::memcpy(&m.s, p, sizeof(double));
    std::memcpy(kb, p + sizeof(double), sizeof kb);
    if (!(m.s > 0.0 && m.s < INFINITY) || kb[0] < 0 || kb[1] < 0) return ABC_E_STATE;
    m.k = kb[0];
    m.batches = kb[1];
    m.s_f = static_cast<float>(m.s);
    m.s_start = m.s_f;
    ABC_CUDA_TRY(cudaMemcpyAsync(c->mcmc, &m, sizeof m, cudaMemcpyHostToDevice, c->st));
  }
  ABC_CUDA_TRY(cudaMemcpyAsync(c->scal + 1, &h.eps1, sizeof(double), cudaMemcpyHostToDevice, c->st));
  ABC_CUDA_TRY(cudaStreamSynchronize(c->st));
  c->gen = h.gen;
  c->eps1_host = h.eps1;
  c->batches_total = h.batches_total;
  c->stats.resize(static_cast<size_t>(h.gen));
  return ABC_OK;
}

ABC_API void abc_free(abc_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  delete c;
}

}  // extern "C"

// ------------------------------------------------------------ batched runs ---
namespace {

RunCtxView ctx_view(abc_ctx* c) {
  RunCtxView v{};
  v.p = c->p;
  v.N = c->N;
  v.M = c->M;
  v.K = spec_k(c->cfg);
  v.mcmc = c->mcmc;
  int64_t k = static_cast<int64_t>(std::ceil(c->cfg.survival_alpha * static_cast<double>(c->N)));
  v.rank = std::min<int64_t>(std::max<int64_t>(k, 1), c->N);
  v.beta = beta_rule(c->cfg);
  v.max_redraw = c->cfg.max_redraw;
  v.weight_mode = c->cfg.weight_mode;
  v.weight_prec = c->cfg.weight_prec;
  v.obs = c->obs;
  v.u_cur = c->u[0];
  v.u_nxt = c->u[1];
  v.s_cur = c->s[0];
  v.s_nxt = c->s[1];
  v.d_cur = c->d[0];
  v.d_nxt = c->d[1];
  v.W_cur = c->W[0];
  v.W_nxt = c->W[1];
  v.a_cur = c->anc[0];
  v.a_nxt = c->anc[1];
  v.up = c->up;
  v.sp = c->sp;
  v.dp = c->dp;
  v.ap = c->ap;
  v.att = c->att;
  v.flag = c->flag;
  v.q = c->q;
  v.prefix = c->prefix;
  v.logW = c->logW;
  v.cu = c->cu;
  v.cc = c->cc;
  v.nc = c->nc;
  v.scratch = c->scratch;
  v.scratch_bytes = c->scratch_bytes;
  // the graph writes the new population to buffer 1 and commits it to 0
  v.sur = sur_view(c, 1);
  if (v.sur.on) v.K = 1;  // screened generations run one batch per round
  return v;
}

}  // namespace

struct abc_batch {
  std::vector<abc_ctx*> runs;
  std::vector<BatchRun> br;
  std::vector<RunDev> host;
  RunDev* dev = nullptr;
  cudaStream_t st = nullptr;        // caller's stream
  cudaStream_t cap = nullptr;       // capture origin
  std::vector<cudaStream_t> rs;     // one per run during capture
  cudaStream_t body = nullptr;
  std::vector<cudaEvent_t> evs;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int32_t gen = 0;
  std::vector<std::vector<abc_gen_stats>> stats;
  ~abc_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (cudaStream_t s : rs) if (s) cudaStreamDestroy(s);
    if (cap) cudaStreamDestroy(cap);
    if (body) cudaStreamDestroy(body);
    for (cudaEvent_t e : evs) if (e) cudaEventDestroy(e);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (dev) cudaFree(dev);
    for (abc_ctx* c : runs) delete c;
  }
};

namespace {

int batch_destroy_graph(abc_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  return ABC_OK;
}

// one graph for a whole generation of every run (branches joined at the end)
int batch_build_graph(abc_batch* b) {
  batch_destroy_graph(b);
  const size_t R = b->runs.size();
  // branches in decreasing particle-days (N T): the longest runs are
  // captured, and so launched, first, which shortens the tail of the graph
  std::vector<size_t> order(R);
  for (size_t r = 0; r < R; ++r) order[r] = r;
  std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
    const abc_ctx* cx = b->runs[x];
    const abc_ctx* cy = b->runs[y];
    return cx->N * std::max(cx->T, 1) > cy->N * std::max(cy->T, 1);
  });
  ABC_CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
  int rc = ABC_OK;
  cudaError_t e = cudaEventRecord(b->evs[0], b->cap);
  for (size_t i = 0; i < R && rc == ABC_OK && e == cudaSuccess; ++i) {
    const size_t r = order[i];
    e = cudaStreamWaitEvent(b->rs[r], b->evs[0], 0);
    if (e == cudaSuccess) rc = batch_capture_run(b->br[r], b->rs[r], b->body);
    if (rc == ABC_OK && e == cudaSuccess) e = cudaEventRecord(b->evs[1 + r], b->rs[r]);
    if (rc == ABC_OK && e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->evs[1 + r], 0);
  }
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(b->cap, &g);
  if (rc != ABC_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess || ee != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return ABC_E_CUDA;
  }
  b->graph = g;
  ABC_CUDA_TRY(cudaGraphInstantiate(&b->exec, g, 0));
  return ABC_OK;
}

std::string tune_key(const abc_ctx* c, int sms) {
  int nb = 0;
  while ((int64_t(1) << (nb + 1)) <= c->N) ++nb;
  char buf[96];
  std::snprintf(buf, sizeof buf, "sm%d_n%d_t%d_w%d%d", sms, nb, c->T / 30, c->cfg.weight_mode,
                c->cfg.weight_prec);
  return buf;
}

// times fn() with CUDA events on st (median of 3, after one warm-up)
template <typename F>
int time_ms(cudaStream_t st, cudaEvent_t a, cudaEvent_t bev, F fn, float* out) {
  float v[3];
  int rc = fn();
  if (rc) return rc;
  for (int i = 0; i < 3; ++i) {
    ABC_CUDA_TRY(cudaEventRecord(a, st));
    if ((rc = fn())) return rc;
    ABC_CUDA_TRY(cudaEventRecord(bev, st));
    ABC_CUDA_TRY(cudaEventSynchronize(bev));
    ABC_CUDA_TRY(cudaEventElapsedTime(&v[i], a, bev));
  }
  std::sort(v, v + 3);
  *out = v[1];
  return ABC_OK;
}

}  // namespace

extern "C" {

ABC_API int abc_batch_init(const abc_config* cfgs, int32_t n_runs, const int32_t* const* obs,
                           void* stream, abc_batch** out) {
  if (!out || !cfgs || n_runs < 1 || n_runs > 4096) return ABC_E_INVAL;
  *out = nullptr;
  abc_batch* b = new (std::nothrow) abc_batch();
  if (!b) return ABC_E_NOMEM;
  b->st = as_stream(stream);
  int rc = ABC_OK;
  for (int32_t r = 0; r < n_runs && rc == ABC_OK; ++r) {
    abc_ctx* c = nullptr;
    rc = abc_init(&cfgs[r], obs ? obs[r] : nullptr, stream, &c);
    if (rc == ABC_OK) b->runs.push_back(c);
  }
  if (rc != ABC_OK) {
    delete b;
    return rc;
  }
  b->host.resize(n_runs);
  b->br.resize(n_runs);
  b->stats.resize(n_runs);
  if (cudaMalloc(&b->dev, sizeof(RunDev) * n_runs) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return ABC_E_NOMEM;
  }
  for (int32_t r = 0; r < n_runs; ++r) {
    std::memset(&b->host[r], 0, sizeof(RunDev));
    b->host[r].max_batches = cfgs[r].max_batches;
    b->host[r].max_total = cfgs[r].max_total_batches;
    b->host[r].eps_stop = static_cast<double>(cfgs[r].eps_stop);
    b->br[r].v = ctx_view(b->runs[r]);
    b->br[r].dev = b->dev + r;
  }
  b->rs.assign(n_runs, nullptr);
  b->evs.assign(n_runs + 1, nullptr);
  bool ok = cudaMemcpy(b->dev, b->host.data(), sizeof(RunDev) * n_runs, cudaMemcpyHostToDevice) ==
                cudaSuccess &&
            cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&b->body, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreate(&b->e0) == cudaSuccess && cudaEventCreate(&b->e1) == cudaSuccess;
  for (int32_t r = 0; ok && r < n_runs; ++r)
    ok = cudaStreamCreateWithFlags(&b->rs[r], cudaStreamNonBlocking) == cudaSuccess;
  for (int32_t r = 0; ok && r <= n_runs; ++r)
    ok = cudaEventCreateWithFlags(&b->evs[r], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    delete b;
    return ABC_E_CUDA;
  }
  *out = b;
  return ABC_OK;
}

ABC_API int abc_batch_generation(abc_batch* b) {
  if (!b) return ABC_E_INVAL;
  const size_t R = b->runs.size();
  if (b->gen == 0) {
    for (size_t r = 0; r < R; ++r) {
      const int rc = abc_generation(b->runs[r]);
      if (rc != ABC_OK) return rc < 0 ? rc : ABC_E_CUDA;
      b->stats[r].push_back(b->runs[r]->stats.back());
      b->host[r].t = 1;
      b->host[r].batches_total = b->runs[r]->batches_total;
      // a run budget used up by stage 0 alone: no generation runs
      if (b->host[r].max_total > 0 && b->host[r].batches_total >= b->host[r].max_total)
        b->host[r].done = 1;
    }
    ABC_CUDA_TRY(cudaMemcpyAsync(b->dev, b->host.data(), sizeof(RunDev) * R,
                                 cudaMemcpyHostToDevice, b->st));
    ABC_CUDA_TRY(cudaStreamSynchronize(b->st));
    b->gen = 1;
    return ABC_OK;
  }
  if (b->gen > 32767) return ABC_E_INVAL;  // the stage fills 16 counter bits
  if (!b->exec) {
    const int rc = batch_build_graph(b);
    if (rc) return rc;
  }
  const int64_t l0 = launch_count();
  ABC_CUDA_TRY(cudaStreamSynchronize(b->st));
  ABC_CUDA_TRY(cudaEventRecord(b->e0, b->cap));
  ABC_CUDA_TRY(cudaGraphLaunch(b->exec, b->cap));
  ABC_CUDA_TRY(cudaEventRecord(b->e1, b->cap));
  ABC_CUDA_TRY(cudaEventSynchronize(b->e1));
  float ms = 0.f;
  ABC_CUDA_TRY(cudaEventElapsedTime(&ms, b->e0, b->e1));
  (void)l0;
  std::vector<RunDev> prev = b->host;
  ABC_CUDA_TRY(cudaMemcpy(b->host.data(), b->dev, sizeof(RunDev) * R, cudaMemcpyDeviceToHost));
  int any_err = 0;
  for (size_t r = 0; r < R; ++r) {
    for (unsigned* e : {b->br[r].tc_err, b->br[r].inf_err}) {
      if (!e) continue;
      unsigned h = 0;
      ABC_CUDA_TRY(cudaMemcpy(&h, e, sizeof h, cudaMemcpyDeviceToHost));
      any_err |= h != 0;
    }
    const RunDev& d = b->host[r];
    if (prev[r].done) continue;  // stopped earlier: nothing ran
    abc_ctx* c = b->runs[r];
    abc_gen_stats g{};
    g.generation = static_cast<int32_t>(prev[r].t);
    g.status = d.status;
    g.eps = d.eps;
    g.eps1 = d.eps1;
    g.ess = d.status == ABC_OK ? d.ess : 0.0;
    stage_shapes(c->cfg, d.eps, d.eps1, g.generation, d.beta_b, &g);
    if (int rc = mcmc_stats(c, &g)) return rc;
    g.batches = d.batches;
    g.accepted = d.accepted;
    g.exhausted = d.exhausted;
    g.sims = d.batches * c->M - d.exhausted;
    if (c->cfg.surrogate) {
      // screened: the simulated slots and the audit counts of the generation
      long long sim = 0;
      unsigned long long aud[2] = {0, 0};
      ABC_CUDA_TRY(cudaMemcpy(&sim, c->simulated, sizeof sim, cudaMemcpyDeviceToHost));
      ABC_CUDA_TRY(cudaMemcpy(aud, c->audit, sizeof aud, cudaMemcpyDeviceToHost));
      g.sims = sim;
      g.audited = static_cast<int64_t>(aud[0]);
      g.audit_accepted = static_cast<int64_t>(aud[1]);
      g.screened = d.batches * c->M - d.exhausted - (sim - g.audited);
    }
    g.sim_days = g.sims * static_cast<int64_t>(c->cfg.model == ABC_MODEL_SAIRD ? c->T : 1);
    g.launches = b->br[r].fixed_launches + d.rounds * b->br[r].body_launches;
    g.ms = ms;  // the whole graph (all runs)
    b->stats[r].push_back(g);
    c->batches_total = d.batches_total;
    if (d.status == ABC_OK) {
      c->gen += 1;
      c->eps1_host = d.eps1;
    }
  }
  if (any_err) return ABC_E_DEVICE;
  b->gen += 1;
  return ABC_OK;
}

ABC_API int abc_batch_run(abc_batch* b, int32_t n_generations) {
  if (!b) return ABC_E_INVAL;
  while (b->gen < n_generations && (b->gen == 0 || abc_batch_active(b) > 0)) {
    const int rc = abc_batch_generation(b);
    if (rc != ABC_OK) return rc;
  }
  return ABC_OK;
}

ABC_API int32_t abc_batch_active(const abc_batch* b) {
  if (!b) return 0;
  if (b->gen == 0) return static_cast<int32_t>(b->runs.size());
  int32_t n = 0;
  for (const RunDev& d : b->host) n += d.done ? 0 : 1;
  return n;
}

ABC_API int32_t abc_batch_runs(const abc_batch* b) {
  return b ? static_cast<int32_t>(b->runs.size()) : 0;
}

ABC_API int32_t abc_batch_generations(const abc_batch* b) { return b ? b->gen : 0; }

ABC_API int abc_batch_get_stats(abc_batch* b, int32_t run, int32_t t, abc_gen_stats* out) {
  if (!b || !out || run < 0 || run >= static_cast<int32_t>(b->runs.size())) return ABC_E_INVAL;
  const auto& v = b->stats[static_cast<size_t>(run)];
  if (t < 0 || t >= static_cast<int32_t>(v.size())) return ABC_E_INVAL;
  *out = v[static_cast<size_t>(t)];
  return ABC_OK;
}

ABC_API int abc_batch_get_population(abc_batch* b, int32_t run, float* u, double* dist, double* W,
                                     float* s, int32_t* anc, int32_t on_device) {
  if (!b || run < 0 || run >= static_cast<int32_t>(b->runs.size())) return ABC_E_INVAL;
  return abc_get_population(b->runs[static_cast<size_t>(run)], u, dist, W, s, anc, on_device);
}

ABC_API int abc_batch_autotune(abc_batch* b, const char* cache_path) {
  if (!b || b->gen < 1) return ABC_E_INVAL;
  int dev = 0, sms = 0;
  ABC_CUDA_TRY(cudaGetDevice(&dev));
  ABC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  std::map<std::string, std::pair<int, int>> cache;
  if (cache_path) {
    std::ifstream in(cache_path);
    std::string line;
    while (std::getline(in, line)) {
      char key[96];
      int th = 0, wm = 0;
      if (std::sscanf(line.c_str(), " \"%95[^\"]\": {\"sim_threads\": %d, \"w_mult\": %d}", key, &th,
                      &wm) == 3)
        cache[key] = {th, wm};
    }
  }
  for (size_t r = 0; r < b->runs.size(); ++r) {
    abc_ctx* c = b->runs[r];
    const std::string key = tune_key(c, sms);
    auto it = cache.find(key);
    if (it == cache.end()) {
      RunCtxView& v = b->br[r].v;
      int best_th = 128, best_m = 1;
      float best = 1e30f;
      // simulator block size, on this run's current population
      for (int th : {64, 128, 256}) {
        float ms = 0.f;
        const int rc = time_ms(b->st, b->e0, b->e1, [&] {
          return launch_simulate(v.p, v.obs, v.u_cur, v.N, nullptr, 0xFFFF0000u, ABC_TAG_SIM,
                                 nullptr, v.dp, nullptr, b->st, nullptr, nullptr, th);
        }, &ms);
        if (rc) return rc;
        if (ms < best) {
          best = ms;
          best_th = th;
        }
      }
      // column chunks of the weight pass, on the current population
      if (c->cfg.weight_mode == ABC_W_IMPORTANCE) {
        double* eps = c->scal;
        int rc = launch_select(v.d_cur, v.N, ctx_view(c).rank, eps, v.scratch, v.scratch_bytes, b->st);
        if (!rc) rc = launch_resample_prefix(v.d_cur, v.W_cur, v.N, eps, v.weight_mode, v.q,
                                             v.prefix, v.scratch, v.scratch_bytes, b->st);
        if (!rc) rc = launch_survivors(v.u_cur, v.q, v.N, v.cu, v.cc, v.nc, v.scratch, b->st);
        if (rc) return rc;
        best = 1e30f;
        for (int m : {1, 2, 4}) {
          float ms = 0.f;
          unsigned* err = nullptr;
          rc = time_ms(b->st, b->e0, b->e1, [&] {
            return v.weight_prec == ABC_P_BF16_TC
                       ? launch_weights_tc(v.u_cur, v.s_cur, v.N, v.cu, v.cc, v.nc, v.N,
                                           v.prefix + (v.N - 1), v.logW, v.scratch,
                                           v.scratch_bytes, &err, b->st, nullptr, m)
                       : launch_weights_fp32(v.u_cur, v.s_cur, v.N, v.cu, v.cc, v.nc, v.N,
                                             v.prefix + (v.N - 1), v.logW, v.scratch,
                                             v.scratch_bytes, b->st, nullptr, m);
          }, &ms);
          if (rc) return rc;
          if (ms < best) {
            best = ms;
            best_m = m;
          }
        }
      }
      it = cache.emplace(key, std::make_pair(best_th, best_m)).first;
    }
    b->br[r].sim_threads = it->second.first;
    b->br[r].w_mult = it->second.second;
  }
  if (cache_path) {
    std::ofstream out(cache_path);
    out << "{\n";
    size_t i = 0;
    for (const auto& kv : cache) {
      out << "  \"" << kv.first << "\": {\"sim_threads\": " << kv.second.first
          << ", \"w_mult\": " << kv.second.second << "}" << (++i < cache.size() ? "," : "") << "\n";
    }
    out << "}\n";
  }
  return batch_destroy_graph(b);  // the next generation captures with the new shapes
}

ABC_API int abc_batch_tuning(const abc_batch* b, int32_t run, int32_t* sim_threads,
                             int32_t* w_mult) {
  if (!b || run < 0 || run >= static_cast<int32_t>(b->runs.size())) return ABC_E_INVAL;
  if (sim_threads) *sim_threads = b->br[static_cast<size_t>(run)].sim_threads;
  if (w_mult) *w_mult = b->br[static_cast<size_t>(run)].w_mult;
  return ABC_OK;
}

ABC_API void abc_batch_free(abc_batch* b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  delete b;
}

}  // extern "C"

// ---------------------------------------------------------------- MLP ABI ---
struct abc_mlp {
  MlpState s{};
  void* mem = nullptr;
  ~abc_mlp() {
    if (mem) cudaFree(mem);
  }
};

extern "C" {

ABC_API int32_t abc_mlp_param_count(void) { return kMlpParams; }

ABC_API int abc_mlp_create(uint64_t seed, abc_mlp** out) {
  if (!out) return ABC_E_INVAL;
  *out = nullptr;
  abc_mlp* m = new (std::nothrow) abc_mlp();
  if (!m) return ABC_E_NOMEM;
  const size_t P = kMlpParams;
  if (cudaMalloc(&m->mem, P * (3 * sizeof(float) + sizeof(__nv_bfloat16)) + 256) != cudaSuccess) {
    cudaGetLastError();
    delete m;
    return ABC_E_NOMEM;
  }
  char* b = static_cast<char*>(m->mem);
  m->s.w = reinterpret_cast<float*>(b);
  m->s.m = m->s.w + P;
  m->s.v = m->s.m + P;
  m->s.wb = reinterpret_cast<__nv_bfloat16*>(m->s.v + P);
  int rc = mlp_init(m->s, static_cast<uint32_t>(seed & 0xFFFFFFFFu),
                    static_cast<uint32_t>(seed >> 32), nullptr);
  if (rc == ABC_OK) rc = mlp_infer_prepare();
  if (rc == ABC_OK) rc = mlp_train_prepare();
  if (rc == ABC_OK && cudaDeviceSynchronize() != cudaSuccess) rc = ABC_E_CUDA;
  if (rc != ABC_OK) {
    delete m;
    return rc;
  }
  *out = m;
  return ABC_OK;
}

ABC_API int abc_mlp_set_params(abc_mlp* m, const float* host_params) {
  if (!m || !host_params) return ABC_E_INVAL;
  ABC_CUDA_TRY(cudaMemcpy(m->s.w, host_params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice));
  const int rc = mlp_refresh_bf16(m->s, nullptr);
  if (rc) return rc;
  ABC_CUDA_TRY(cudaDeviceSynchronize());
  return ABC_OK;
}

ABC_API int abc_mlp_get_params(abc_mlp* m, float* host_params, uint16_t* host_bf16) {
  if (!m) return ABC_E_INVAL;
  if (host_params)
    ABC_CUDA_TRY(cudaMemcpy(host_params, m->s.w, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost));
  if (host_bf16)
    ABC_CUDA_TRY(cudaMemcpy(host_bf16, m->s.wb, 2 * kMlpParams, cudaMemcpyDeviceToHost));
  return ABC_OK;
}

ABC_API size_t abc_mlp_scratch_bytes(int32_t batch, int64_t n) {
  return std::max(mlp_train_scratch_bytes(std::max(batch, 1)), mlp_infer_scratch_bytes(n));
}

ABC_API int abc_mlp_grad(abc_mlp* m, const float* X, const float* T, int32_t B, float* grad,
                         float* sse, void* scratch, size_t scratch_bytes, void* stream) {
  if (!m || !X || !T || !grad || !sse || !scratch || B < 1 || B > (1 << 22)) return ABC_E_INVAL;
  cudaStream_t st = as_stream(stream);
  const int rc = mlp_grad(m->s, X, T, B, grad, sse, scratch, scratch_bytes, st);
  if (rc) return rc;
  return check_device_error(mlp_grad_err(scratch, B), st);
}

ABC_API int abc_mlp_adam(abc_mlp* m, const float* grad, int64_t step, float lr, void* stream) {
  if (!m || !grad || step < 1 || !(lr > 0.0f)) return ABC_E_INVAL;
  return mlp_adam(m->s, grad, step, lr, as_stream(stream));
}

ABC_API int abc_mlp_forward(abc_mlp* m, const float* u, int64_t n, float* Y, void* scratch,
                            size_t scratch_bytes, void* stream) {
  if (!m || !u || !Y || !scratch || n < 1 || n > kMaxIndex) return ABC_E_INVAL;
  cudaStream_t st = as_stream(stream);
  unsigned* err = nullptr;
  int rc = mlp_infer(m->s, u, n, Y, scratch, scratch_bytes, &err, st);
  if (rc) return rc;
  return check_device_error(err, st);
}

ABC_API void abc_mlp_free(abc_mlp* m) {
  if (m) {
    cudaDeviceSynchronize();
    delete m;
  }
}

}  // extern "C"
