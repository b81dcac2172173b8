// batch.cuh -- internal types of the batched (many-run) graph path.
#pragma once
#include "common.cuh"
#include "surrogate.cuh"

namespace abc {

// Per-run state read and written by the graph's kernels.  accepted and
// exhausted must stay adjacent: the acceptance kernel takes them as a pair.
struct RunDev {
  uint32_t t;           // generation being run
  uint32_t b;           // batch index inside the generation
  uint32_t c1;          // Philox counter word (t << 16) | b
  int32_t beta_b;       // Beta shape b of this generation
  int32_t done;         // the run has stopped (batch budget)
  int32_t off;          // skip the rest of this generation
  int32_t status;       // of the last generation
  int32_t max_batches;
  long long filled;
  long long accepted;
  long long exhausted;
  long long batches;
  long long batches_total;  // run budget count: ceil(N / M) for stage 0, then every batch
  long long rounds;         // device loop rounds of this generation
  int32_t max_total;        // run budget (0: none)
  int32_t k_lim;            // batches proposed in this round (several: spec_batches)
  int32_t used;             // batches the round used (up to the one that filled N)
  int32_t pad;
  double eps, eps1, ess;
  double eps_stop;          // tolerance target (0: none)
};

// Buffers and settings of a run's surrogate pre-screen (borrowed from its
// context); used by single-run contexts and graph branches alike.
struct SurView {
  bool on = false;                 // the run uses the surrogate
  MlpState mlp{};
  float* ystat = nullptr;          // output means, sds [4 + 4]; input means, sds [8 + 8]
  float* Yp = nullptr;             // predictions [M][4]
  float* rho = nullptr;            // pass probability per slot
  uint8_t* sflag = nullptr;        // 0 acceptable, 1 exhausted, 2 audit only, 3 screened out
  float *cmp_u = nullptr, *cmp_s = nullptr, *cmp_rho = nullptr;  // compacted slots, stride M
  int32_t* cmp_a = nullptr;
  uint8_t* cmp_flag = nullptr;
  uint32_t* cmp_slot = nullptr;
  double* cmp_d = nullptr;
  int32_t* ard = nullptr;          // final A, R, D of each simulated slot [3][M]
  int* Mc = nullptr;               // simulated slots of the batch
  float* rho_pop = nullptr;        // rho of each accepted particle of the new population
  float *RX = nullptr, *RY = nullptr;  // training ring [cap][8], [cap][4]
  long long* ring_head = nullptr;
  int64_t ring_cap = 0;
  float *grad = nullptr, *trX = nullptr, *trT = nullptr, *loss = nullptr;
  unsigned long long* audit = nullptr;  // audited, audited with d <= eps (this generation)
  unsigned* inf_err = nullptr;     // error word of the tensor-core inference and training
  long long* simulated = nullptr;  // simulated slots (this generation)
  uint32_t* train_step = nullptr;  // Adam steps so far (device)
  int* screen_on = nullptr;        // this generation screens
  void* sscratch = nullptr;
  size_t sscratch_bytes = 0;
  int start = 1, steps = 0, batch = 0;
  float lr = 0.f, tau = 1.f, rho_min = 1.f, audit_frac = 0.f;
};

// Device buffers and settings of one run (borrowed from its context).
struct RunCtxView {
  SimParams p;
  int64_t N, M, rank;
  int K;  // batches per device loop round (spec_batches)
  BetaRule beta;
  int max_redraw, weight_mode, weight_prec;
  const int32_t* obs;
  float *u_cur, *u_nxt, *s_cur, *s_nxt, *up, *sp, *cu, *cc;
  double *d_cur, *d_nxt, *W_cur, *W_nxt, *dp, *logW;
  int32_t *a_cur, *a_nxt, *ap, *att;
  uint8_t* flag;
  uint32_t* q;
  uint64_t* prefix;
  int* nc;
  void* scratch;
  size_t scratch_bytes;
  SurView sur;
  McmcDev* mcmc;  // ABC_STEP_MCMC: the run's tuned step (else null)
};

struct BatchRun {
  RunCtxView v;
  RunDev* dev = nullptr;      // this run's slot in the device state array
  int sim_threads = 128;      // autotuned simulator block size
  int w_mult = 1;             // autotuned column-chunk multiplier of the weight pass
  unsigned* tc_err = nullptr; // error word of the tensor-core pass (when used)
  unsigned* inf_err = nullptr; // error word of the surrogate's tensor-core inference
  int64_t fixed_launches = 0; // kernels per generation outside the batch loop
  int64_t body_launches = 0;  // kernels per batch
};

int batch_capture_run(BatchRun& br, cudaStream_t st, cudaStream_t body_st);

// One batch of M proposals (up, sp, ap, flag) screened by the surrogate:
// inference, screen (a pass-all when *screen_on is 0), compaction of the
// simulated slots, their simulation with their own counters, acceptance into
// the new population in slot order, audit counts, training-ring append.
// c1 / c1_dev: the batch's counter word (host value or device word);
// filled, counters (accepted, exhausted adjacent) and exhausted: device
// counters; the screen counts redraw-exhausted slots into *exhausted.  ev
// (nullable): three events recorded before the inference, before and after
// the simulation.  No host synchronisation.
int screened_batch(const SurView& s, const SimParams& p, const int32_t* obs, const float* up,
                   const float* sp, const int32_t* ap, const uint8_t* flag, int64_t M,
                   const double* eps, uint32_t c1, const uint32_t* c1_dev, int64_t N,
                   float* u_pop, double* d_pop, float* s_pop, int32_t* a_pop, int64_t* filled,
                   int64_t* counters, unsigned long long* exhausted, void* scratch,
                   size_t scratch_bytes, int sim_threads, unsigned** inf_err, cudaStream_t st,
                   const cudaEvent_t* ev = nullptr);
// After a generation: the surrogate's training (ring statistics, `steps`
// Adam steps on ring minibatches); off_dev (graph branches): a run whose
// generation stopped does not advance its step count.
int sur_train(const SurView& s, const SimParams& p, const int* off_dev, cudaStream_t st);

// launchers shared with the single-run context
int launch_simulate(const SimParams&, const int32_t*, const float*, int64_t, const uint32_t*,
                    uint32_t, uint32_t, const uint8_t*, double*, int32_t*, cudaStream_t,
                    const uint32_t* c1_dev = nullptr, const int* off_dev = nullptr,
                    int threads = 128, int32_t* ard_last = nullptr, int64_t m_sub = 0,
                    const int* n_dev = nullptr, const int32_t* perm = nullptr);
// A batch of n SAIRD slots (the SIM stream; c0 = c0_idx[i] or the slot
// index) simulated in the order of a key that groups similar trajectories
// into warps (same results as launch_simulate; with n_dev the first *n_dev
// slots are ordered among themselves); below kSimOrderMin slots, for the
// toy model or without observations it is launch_simulate.  scratch: at
// least sim_order_scratch_bytes(n), free until the simulation has run.
constexpr int64_t kSimOrderMin = 16384;
size_t sim_order_scratch_bytes(int64_t n);
int launch_simulate_ordered(const SimParams& p, const int32_t* obs, const float* u, int64_t n,
                            uint32_t c1, const uint8_t* skip, double* dist, void* scratch,
                            size_t bytes, cudaStream_t st, const uint32_t* c1_dev = nullptr,
                            const int* off_dev = nullptr, int threads = 128, int64_t m_sub = 0,
                            const uint32_t* c0_idx = nullptr, const int* n_dev = nullptr,
                            int32_t* ard_last = nullptr);
int launch_select(const double*, int64_t, int64_t, double*, void*, size_t, cudaStream_t);
int launch_resample_prefix(const double*, const double*, int64_t, const double*, int, uint32_t*,
                           uint64_t*, void*, size_t, cudaStream_t);
bool beta_rule_ok(const BetaRule&);
size_t radix_sort_scratch_bytes(int64_t cap);
int launch_radix_sort(const uint32_t* kin, const int32_t* vin, uint32_t* kout, int32_t* vout,
                      int64_t cap, const int* n_dev, int bits, void* scratch, size_t bytes,
                      cudaStream_t st);
int launch_propose(const SimParams&, const float*, int64_t, const uint64_t*, const BetaRule&,
                   const double*, const double*, int64_t, const uint32_t*, uint32_t, int, float*,
                   float*, int32_t*, int32_t*, uint8_t*, cudaStream_t,
                   const uint32_t* c1_dev = nullptr, const int* beta_b_dev = nullptr,
                   const int* off_dev = nullptr, int64_t m_sub = 0,
                   const int* k_lim_dev = nullptr, const float* s_fix_dev = nullptr);
// The MCMC baseline's step (ABC_STEP_MCMC): the start of a generation, and
// the adaptation after a batch of M slots given the generation's {accepted,
// exhausted} counters.  off_dev (nullable): a finished run does nothing.
int launch_mcmc_begin(McmcDev* m, const int* off_dev, cudaStream_t st);
int launch_mcmc_adapt(McmcDev* m, const long long* acc_exh, int64_t M, const int* off_dev,
                      cudaStream_t st);
size_t accept_spec_scratch_bytes(int64_t M, int K);
int launch_accept_spec(const float*, const double*, const float*, const int32_t*,
                       const uint8_t*, int64_t M, int K, const int* k_lim_dev, const double*,
                       int64_t N, float*, double*, float*, int32_t*, int64_t* filled,
                       int64_t* counters, int* used_out, void*, size_t, cudaStream_t);
int launch_accept(const float*, const double*, const float*, const int32_t*, const uint8_t*,
                  int64_t, const double*, int64_t, float*, double*, float*, int32_t*, int64_t*,
                  int64_t*, void*, size_t, cudaStream_t, const float* rho_in = nullptr,
                  float* rho_pop = nullptr);
int launch_survivors(const float*, const uint32_t*, int64_t, float*, float*, int*, void*,
                     cudaStream_t);
int launch_weights_fp32(const float*, const float*, int64_t, const float*, const float*,
                        const int*, int64_t, const uint64_t*, double*, void*, size_t,
                        cudaStream_t, const int* off_dev = nullptr, int mult = 1,
                        const int* rows_dev = nullptr, const WeightTiming* wt = nullptr);
int launch_weights_tc(const float*, const float*, int64_t, const float*, const float*, const int*,
                      int64_t, const uint64_t*, double*, void*, size_t, unsigned**,
                      cudaStream_t, const int* off_dev = nullptr, int mult = 1,
                      const int* rows_dev = nullptr, const AncInfo& ai = AncInfo(),
                      WeightTiming* wt = nullptr);
int launch_normalize(const double*, int64_t, double*, double*, void*, size_t, cudaStream_t);
int weights_tc_prepare();

}  // namespace abc
