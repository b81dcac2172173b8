// api.cu -- the C ABI: argument checks, step entry points and the context
// that runs whole SMC generations (Sec. 2.4 and 3.2 of arXiv 2106.15508).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

namespace abc {
int launch_simulate(const SimParams&, const int32_t*, const float*, int64_t, const uint32_t*,
                    uint32_t, uint32_t, const uint8_t*, double*, int32_t*, cudaStream_t);
int launch_prior(const SimParams&, int64_t, float*, cudaStream_t);
int launch_synth_obs(const SimParams&, const float*, const float*, int32_t*, float*, int32_t*,
                     cudaStream_t);
int launch_philox(const uint32_t*, uint32_t, uint32_t, int64_t, uint32_t*, cudaStream_t);
size_t select_scratch_bytes(int64_t);
int launch_select(const double*, int64_t, int64_t, double*, void*, size_t, cudaStream_t);
size_t prefix_scratch_bytes(int64_t);
int launch_resample_prefix(const double*, const double*, int64_t, const double*, int, uint32_t*,
                           uint64_t*, void*, size_t, cudaStream_t);
int launch_resample_prefix_noalloc(const double*, const double*, int64_t, const double*, int,
                                   uint32_t*, uint64_t*, cudaStream_t);
int launch_propose(const SimParams&, const float*, int64_t, const uint64_t*, int, const double*,
                   const double*, float, int, int64_t, const uint32_t*, uint32_t, int, float*,
                   float*, int32_t*, int32_t*, uint8_t*, cudaStream_t);
size_t accept_scratch_bytes(int64_t);
int launch_accept(const float*, const double*, const float*, const int32_t*, const uint8_t*,
                  int64_t, const double*, int64_t, float*, double*, float*, int32_t*, int64_t*,
                  int64_t*, void*, size_t, cudaStream_t);
size_t survivors_scratch_bytes(int64_t);
int launch_survivors(const float*, const uint32_t*, int64_t, float*, float*, int*, void*,
                     cudaStream_t);
size_t weights_fp32_scratch_bytes(int64_t, int64_t);
int launch_weights_fp32(const float*, const float*, int64_t, const float*, const float*,
                        const int*, int64_t, const uint64_t*, double*, void*, size_t,
                        cudaStream_t);
size_t weights_tc_scratch_bytes(int64_t, int64_t);
int launch_weights_tc(const float*, const float*, int64_t, const float*, const float*, const int*,
                      int64_t, const uint64_t*, double*, void*, size_t, unsigned**,
                      cudaStream_t);
int launch_tc_probe(const void*, const void*, float*, unsigned*, cudaStream_t);
size_t normalize_scratch_bytes(int64_t);
int launch_normalize(const double*, int64_t, double*, double*, void*, size_t, cudaStream_t);
int launch_fill(double*, int64_t, double, cudaStream_t);
}  // namespace abc

namespace abc {
static std::atomic<int64_t> g_launches{0};
int64_t count_launch() { return g_launches.fetch_add(1, std::memory_order_relaxed) + 1; }
}  // namespace abc

using namespace abc;

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

int check_smc(const abc_config* c) {
  if (c->n_particles < 1 || c->batch_size < 0) return ABC_E_INVAL;
  if (!(c->survival_alpha > 0.0 && c->survival_alpha <= 1.0)) return ABC_E_INVAL;
  if (c->beta_mode != ABC_BETA_PAPER && c->beta_mode != ABC_BETA_FIXED) return ABC_E_INVAL;
  if (c->beta_mode == ABC_BETA_FIXED &&
      (!(c->beta_a > 0.0f) || c->beta_b < 1 || c->beta_b > 1024))
    return ABC_E_INVAL;
  if (c->weight_mode != ABC_W_PAPER && c->weight_mode != ABC_W_IMPORTANCE) return ABC_E_INVAL;
  if (c->weight_prec != ABC_P_FP32 && c->weight_prec != ABC_P_BF16_TC) return ABC_E_INVAL;
  if (c->max_batches < 1 || c->max_batches > 65535) return ABC_E_INVAL;
  if (c->max_redraw < 1 || c->max_redraw > (1 << 23)) return ABC_E_INVAL;
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
  c->beta_a = 2.0f;
  c->beta_b = 5;
  c->weight_mode = ABC_W_PAPER;
  c->weight_prec = ABC_P_FP32;
  c->max_batches = 64;
  c->max_redraw = 64;
}

ABC_API const char* abc_strerror(int code) {
  switch (code) {
    case ABC_OK: return "ok";
    case ABC_STOP_BUDGET: return "generation stopped: batch budget used before N acceptances";
    case ABC_STOP_TARGET: return "run stopped: tolerance target reached";
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
  const int paper = cfg->beta_mode == ABC_BETA_PAPER;
  if (!paper && !(beta_a > 0.0f)) return ABC_E_INVAL;
  return launch_propose(make_params(*cfg), u, n, prefix, paper, eps, eps1, beta_a, beta_b, slots,
                        c0_idx, c1, cfg->max_redraw, u_out, s_out, anc_out, attempts_out,
                        flag_out, as_stream(stream));
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

// scratch layout of abc_weights: [cu 8n][cc n][nc][compaction][weight pass]
static size_t weights_layout(int64_t rows, int64_t n, size_t* off_cc, size_t* off_nc,
                             size_t* off_comp, size_t* off_w) {
  size_t o = align256(sizeof(float) * 8 * static_cast<size_t>(n));
  *off_cc = o;
  o += align256(sizeof(float) * static_cast<size_t>(n));
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

ABC_API size_t abc_normalize_scratch_bytes(int64_t n) { return normalize_scratch_bytes(n); }

ABC_API int abc_normalize(const double* logW, int64_t n, double* W, double* ess, void* scratch,
                          size_t scratch_bytes, void* stream) {
  if (!logW || !W || !ess || !scratch) return ABC_E_INVAL;
  return launch_normalize(logW, n, W, ess, scratch, scratch_bytes, as_stream(stream));
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
  std::vector<abc_gen_stats> stats;
  std::vector<void*> allocs;
  // device buffers
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

  template <typename T>
  int alloc(T** ptr, size_t count) {
    void* p = nullptr;
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
    for (cudaEvent_t e : {ev0, ev1, es0, es1, ew0, ew1})
      if (e) cudaEventDestroy(e);
  }
};

namespace {

int ctx_alloc(abc_ctx* c) {
  const size_t N = static_cast<size_t>(c->N), M = static_cast<size_t>(c->M);
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
    ABC_ALLOC(c->cc, N);
    ABC_ALLOC(c->nc, 1);
  }
  ABC_ALLOC(c->scal, 4);
  ABC_ALLOC(c->cnt, 4);
#undef ABC_ALLOC
  size_t sb = std::max({select_scratch_bytes(c->N), prefix_scratch_bytes(c->N),
                        accept_scratch_bytes(c->M), survivors_scratch_bytes(c->N),
                        normalize_scratch_bytes(c->N)});
  if (c->cfg.weight_mode == ABC_W_IMPORTANCE)
    sb = std::max(sb, c->cfg.weight_prec == ABC_P_BF16_TC ? weights_tc_scratch_bytes(c->N, c->N)
                                                          : weights_fp32_scratch_bytes(c->N, c->N));
  c->scratch_bytes = sb;
  char* sc = nullptr;
  if ((rc = c->alloc(&sc, sb)) != ABC_OK) return rc;
  c->scratch = sc;
  return ABC_OK;
}

int generation0(abc_ctx* c) {
  cudaStream_t st = c->st;
  const int cur = c->cur;
  int rc = launch_prior(c->p, c->N, c->u[cur], st);
  if (rc) return rc;
  ABC_CUDA_TRY(cudaEventRecord(c->es0, st));
  rc = launch_simulate(c->p, c->obs, c->u[cur], c->N, nullptr, 0u, ABC_TAG_SIM, nullptr, c->d[cur],
                       nullptr, st);
  if (rc) return rc;
  ABC_CUDA_TRY(cudaEventRecord(c->es1, st));
  if ((rc = launch_fill(c->W[cur], c->N, 1.0 / static_cast<double>(c->N), st))) return rc;
  ABC_CUDA_TRY(cudaMemsetAsync(c->anc[cur], 0xFF, sizeof(int32_t) * c->N, st));
  ABC_CUDA_TRY(cudaMemsetAsync(c->s[cur], 0, sizeof(float) * c->N, st));
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
  const int32_t bb = paper_beta ? 2 * t : c->cfg.beta_b;
  if (bb > 1024 || t > 32767) return ABC_E_INVAL;
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
  int64_t filled = 0;
  double ms_sim = 0.0;
  int32_t b = 0;
  for (b = 0; b < c->cfg.max_batches && filled < c->N; ++b) {
    const uint32_t c1 = (static_cast<uint32_t>(t) << 16) | static_cast<uint32_t>(b);
    rc = launch_propose(c->p, c->u[cur], c->N, c->prefix, paper_beta, eps, eps1, c->cfg.beta_a, bb,
                        c->M, nullptr, c1, c->cfg.max_redraw, c->up, c->sp, c->ap, c->att,
                        c->flag, st);
    if (rc) return rc;
    ABC_CUDA_TRY(cudaEventRecord(c->es0, st));
    rc = launch_simulate(c->p, c->obs, c->up, c->M, nullptr, c1, ABC_TAG_SIM, c->flag, c->dp,
                         nullptr, st);
    if (rc) return rc;
    ABC_CUDA_TRY(cudaEventRecord(c->es1, st));
    rc = launch_accept(c->up, c->dp, c->sp, c->ap, c->flag, c->M, eps, c->N, c->u[nxt], c->d[nxt],
                       c->s[nxt], c->anc[nxt], c->cnt, c->cnt + 1, c->scratch, c->scratch_bytes,
                       st);
    if (rc) return rc;
    ABC_CUDA_TRY(cudaMemcpyAsync(&filled, c->cnt, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    ABC_CUDA_TRY(cudaStreamSynchronize(st));
    float ms = 0.f;
    ABC_CUDA_TRY(cudaEventElapsedTime(&ms, c->es0, c->es1));
    ms_sim += ms;
  }
  int64_t h_cnt[3];
  ABC_CUDA_TRY(cudaMemcpyAsync(h_cnt, c->cnt, sizeof h_cnt, cudaMemcpyDeviceToHost, st));
  ABC_CUDA_TRY(cudaStreamSynchronize(st));
  abc_gen_stats g{};
  g.generation = t;
  g.batches = b;
  g.accepted = h_cnt[1];
  g.exhausted = h_cnt[2];
  g.sims = static_cast<int64_t>(b) * c->M - h_cnt[2];
  g.sim_days = g.sims * static_cast<int64_t>(c->cfg.model == ABC_MODEL_SAIRD ? c->T : 1);
  g.beta_b = bb;
  g.ms_sim = ms_sim;
  int h_nc = 0;
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
                               &tc_err, st);
      else
        rc = launch_weights_fp32(c->u[nxt], c->s[nxt], c->N, c->cu, c->cc, c->nc, c->N,
                                 c->prefix + (c->N - 1), c->logW, c->scratch, c->scratch_bytes,
                                 st);
      if (rc) return rc;
      ABC_CUDA_TRY(cudaEventRecord(c->ew1, st));
      if (tc_err) ABC_CUDA_TRY(cudaMemcpyAsync(&h_err, tc_err, sizeof h_err, cudaMemcpyDeviceToHost, st));
      ABC_CUDA_TRY(cudaMemcpyAsync(&h_nc, c->nc, sizeof(int), cudaMemcpyDeviceToHost, st));
      weighted = true;
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
  }
  g.eps = h_scal[0];
  g.eps1 = h_scal[1];
  g.ess = g.status == ABC_OK ? h_scal[2] : 0.0;
  g.beta_a = paper_beta ? (h_scal[1] > 0.0 ? static_cast<float>(h_scal[0] / h_scal[1]) : 1.0f)
                        : c->cfg.beta_a;
  c->eps1_host = h_scal[1];
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
  if ((rc = ctx_alloc(c)) != ABC_OK) {
    delete c;
    return rc;
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
      cudaStreamSynchronize(c->st) != cudaSuccess) {
    delete c;
    return ABC_E_CUDA;
  }
  *out = c;
  return ABC_OK;
}

ABC_API int abc_generation(abc_ctx* c) {
  if (!c) return ABC_E_INVAL;
  ABC_CUDA_TRY(cudaEventRecord(c->ev0, c->st));
  const int64_t l0 = g_launches.load();
  const int rc = c->gen == 0 ? generation0(c) : generation_t(c);
  if (rc < 0) return rc;
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

ABC_API int32_t abc_generations(const abc_ctx* c) { return c ? c->gen : 0; }

namespace {
struct StateHeader {
  char magic[8];
  int64_t N, T;
  uint64_t seed;
  uint32_t run_id;
  int32_t gen;
  double eps1;
};
}  // namespace

ABC_API int abc_get_state(abc_ctx* c, void* buf, size_t* len) {
  if (!c || !len) return ABC_E_INVAL;
  const size_t N = static_cast<size_t>(c->N);
  const size_t need = sizeof(StateHeader) + N * (8 * sizeof(float) + 2 * sizeof(double) +
                                                 sizeof(float) + sizeof(int32_t));
  if (!buf) {
    *len = need;
    return ABC_OK;
  }
  if (*len < need || c->gen == 0) return ABC_E_INVAL;
  StateHeader h{};
  std::memcpy(h.magic, "ABCSMC01", 8);
  h.N = c->N;
  h.T = c->T;
  h.seed = c->cfg.seed;
  h.run_id = c->cfg.run_id;
  h.gen = c->gen;
  h.eps1 = c->eps1_host;
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
  ABC_CUDA_TRY(cudaStreamSynchronize(c->st));
  *len = need;
  return ABC_OK;
}

ABC_API int abc_set_state(abc_ctx* c, const void* buf, size_t len) {
  if (!c || !buf || len < sizeof(StateHeader)) return ABC_E_INVAL;
  StateHeader h;
  std::memcpy(&h, buf, sizeof h);
  const size_t N = static_cast<size_t>(c->N);
  const size_t need = sizeof(StateHeader) + N * (8 * sizeof(float) + 2 * sizeof(double) +
                                                 sizeof(float) + sizeof(int32_t));
  if (std::memcmp(h.magic, "ABCSMC01", 8) != 0 || h.N != c->N || h.T != c->T || len < need ||
      h.gen < 1)
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
  ABC_CUDA_TRY(cudaMemcpyAsync(c->scal + 1, &h.eps1, sizeof(double), cudaMemcpyHostToDevice, c->st));
  ABC_CUDA_TRY(cudaStreamSynchronize(c->st));
  c->gen = h.gen;
  c->eps1_host = h.eps1;
  c->stats.resize(static_cast<size_t>(h.gen));
  return ABC_OK;
}

ABC_API void abc_free(abc_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  delete c;
}

}  // extern "C"
