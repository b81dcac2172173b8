/*
 * abcsmc.h -- C ABI of the GB300 (sm_103a) implementation of P-ABC-SMC with
 * Beta-distributed step sizes (BDSS), arXiv 2106.15508.
 *
 * Two layers:
 *   - step entry points (abc_prior, abc_simulate, abc_select_kth, ...): one
 *     hot-path step each, on caller-owned DEVICE buffers, stream-ordered on
 *     the given cudaStream_t (passed as void*; NULL = legacy default stream);
 *   - a context (abc_init / abc_generation / abc_run / abc_get_*) that owns
 *     its device buffers and runs whole SMC generations (Sec. 2.4, 3.2).
 *
 * Conventions (all entry points):
 *   - return ABC_OK (0) on success, a positive ABC_STOP_* code for a normal
 *     early stop, or a negative ABC_E_* code; abc_strerror() names it;
 *   - pointers marked "device" must be device (or managed) memory; "host"
 *     pointers are read or written synchronously before return;
 *   - caller buffers are borrowed and never freed by the library;
 *   - arrays of particles are structure-of-arrays: u[d * n + j] holds
 *     coordinate d of particle j (d = 0..7), in unit-cube coordinates
 *     u = (theta - theta_lo) / (theta_hi - theta_lo) (the paper's
 *     reparameterisation, Sec. 3.1);
 *   - theta = [alpha0, alpha, n, beta, gamma, delta, eta, kappa] (Eq. 1);
 *   - random numbers come from Philox4x32-10 (Salmon et al., SC'11) with key
 *     (seed_lo, seed_hi ^ run_id) and counter (c0, c1, c2, tag); c0 is the
 *     slot, c1 = (generation << 16) | batch, c2 and the tag are fixed per
 *     stream (ABC_TAG_*).  Results depend only on the counters, never on
 *     launch geometry.
 * Scratch: entry points that take (scratch, scratch_bytes) need at least
 * the matching abc_*_scratch_bytes() of device memory; contents on entry
 * are ignored.
 */
#ifndef ABCSMC_H
#define ABCSMC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define ABC_API __attribute__((visibility("default")))
#else
#define ABC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define ABC_OK 0
#define ABC_STOP_BUDGET 1       /* a generation used max_batches batches before N acceptances */
#define ABC_STOP_TARGET 2       /* abc_run reached eps_target, or the run its eps_stop   */
#define ABC_STOP_TOTAL 3        /* the run used max_total_batches batches (Sec. 4.1)     */
#define ABC_E_INVAL (-1)        /* bad argument or configuration                         */
#define ABC_E_NOMEM (-2)        /* device allocation failed                              */
#define ABC_E_CUDA (-3)         /* a CUDA runtime call or kernel launch failed           */
#define ABC_E_DEVICE (-4)       /* a device-side bound check tripped                     */
#define ABC_E_SCRATCH (-5)      /* scratch buffer smaller than required                  */
#define ABC_E_STATE (-6)        /* malformed or mismatched state blob                    */
#define ABC_E_TOO_LARGE (-7)    /* size above the fixed scratch of an allocation-free call */

/* ---- enumerations ------------------------------------------------------ */
#define ABC_MODEL_SAIRD 0       /* stochastic S/I/A/R/D/Ru model (Sec. 2.2)              */
#define ABC_MODEL_GAUSS_TOY 1   /* x ~ N(theta, I8), distance ||x - x_obs|| (test model)  */
#define ABC_SIM_BINOMIAL 0      /* exact-count binomial competing risks (default)        */
#define ABC_SIM_PAPER_NORMAL 1  /* the paper's floor(Normal(h, sqrt h)) flows (Sec. 2.2) */
#define ABC_BETA_PAPER 0        /* s ~ Beta(eps_t/eps_1, 2t)  (Eq. 16); product form up  */
                                /*   to t = 512, the Gamma ratio from t = 513 on          */
#define ABC_BETA_FIXED 1        /* s ~ Beta(beta_a, beta_b)                               */
/* Real-shape rules (Sec. 3.2 names the mean-variance and mode-concentration
 * parameterisations beside Eq. 16 without their schedules; here the location
 * follows eps_t/eps_1 as a_t does and the spread follows the stage count as
 * b_t = 2t does).  Sampled by the Gamma ratio X/(X+Y) with Marsaglia-Tsang
 * Gamma variates; t is the stage, ratio = (float)(eps_t / eps_1), 1 when
 * eps_1 = 0. */
#define ABC_BETA_REAL 2         /* s ~ Beta(beta_p1, beta_p2), real shapes in [2^-20, 2^20] */
#define ABC_BETA_MEAN_VAR 3     /* mean p1 ratio, variance p2 / t; a + b at least 1/16    */
#define ABC_BETA_MODE_CONC 4    /* mode p1 ratio, concentration a + b = p2 t              */
/* Not a Beta rule: the paper's comparison method, P-ABC-SMC MCMC (Sec.
 * 2.4.1, 3.1).  Every proposal walks with the run's single step s (Eq. 12;
 * a variance in unit-cube coordinates), starting at mcmc_s0 and adapted
 * after each batch during the adaptation window (Eq. 14-15, see
 * mcmc_adapt).  With the uniform prior and the symmetric walk the
 * Metropolis-Hastings ratio of Eq. 13 is the support indicator, so its
 * accept/reject step is the redraw of proposals outside [0,1]^8.  Runs one
 * batch per round (spec_batches is ignored) and takes no surrogate. */
#define ABC_STEP_MCMC 5
#define ABC_W_PAPER 0           /* resampling weights eps_t - d (Eq. 10), W = 1/N         */
#define ABC_W_IMPORTANCE 1      /* importance weights with the O(N^2) kernel sum          */
#define ABC_P_FP32 0            /* O(N^2) weight sum on CUDA cores in fp32                */
#define ABC_P_BF16_TC 1         /* O(N^2) weight sum on tcgen05 tensor cores, bf16 inputs */

/* Philox stream tags (fourth counter word) */
#define ABC_TAG_PRIOR 0
#define ABC_TAG_ANCESTOR 1
#define ABC_TAG_BETA 2
#define ABC_TAG_WALK 3
#define ABC_TAG_SIM 4
#define ABC_TAG_SCREEN 5
#define ABC_TAG_AUDIT 6
#define ABC_TAG_OBS 7
#define ABC_TAG_OBS_THETA 8
#define ABC_TAG_PREDICT 11
#define ABC_TAG_PREDICT_SIM 12

/* ---- configuration ----------------------------------------------------- */
typedef struct {
  int32_t model;            /* ABC_MODEL_*                                              */
  int32_t sampler;          /* ABC_SIM_*                                                */
  int32_t n_days;           /* T >= 1 for SAIRD (days 1..T are compared)                 */
  int32_t init_ard[3];      /* A0, R0, D0: observed day-0 state (Sec. 2.2)               */
  int64_t population;       /* P, 1 <= P <= 2^31 - 1 (counts are int32)                 */
  float theta_lo[8];        /* prior U(theta_lo, theta_hi) (Eq. 2): lo = 0,              */
  float theta_hi[8];        /*   hi = [1, 100, 2, 1, 1, 1, 1, 2] for SAIRD               */
  float x_obs[8];           /* observation of the Gaussian toy model                    */
  uint64_t seed;            /* Philox key = (seed lo 32, seed hi 32 ^ run_id)            */
  uint32_t run_id;
  int32_t n_particles;      /* N: population kept per generation (Sec. 4.1: samples)    */
  int32_t batch_size;       /* M: proposals per batch (Sec. 3.1: parallel simulations); */
                            /*   0 means M = N                                           */
  int32_t beta_mode;        /* ABC_BETA_*                                               */
  double survival_alpha;    /* alpha of Eq. 8 (0.5 in the paper)                        */
  float beta_a;             /* fixed-mode shape a > 0                                    */
  int32_t beta_b;           /* fixed-mode shape b, integer 1..1024                       */
  int32_t weight_mode;      /* ABC_W_*                                                  */
  int32_t weight_prec;      /* ABC_P_*                                                  */
  int32_t max_batches;      /* per-generation batch budget (<= 65535)                   */
  int32_t max_redraw;       /* proposal redraws when u' leaves [0,1]^8                   */
  /* Surrogate pre-screen (an extension beyond the paper; the paper simulates every
   * proposal): an MLP u -> [log1p d, log1p A_T, log1p R_T, log1p D_T],
   * 8 -> 256 -> 256 -> 4 with GELU, bf16 weights and fp32 accumulation,
   * trained after every generation on the (u, summary) pairs simulated so
   * far, screens proposals by delayed acceptance: a proposal is simulated
   * with probability rho = clamp(sigmoid((log1p eps_t - y0) / tau), rho_min,
   * 1) and its importance weight divided by rho; screened-out proposals are
   * simulated anyway with probability audit_frac to estimate the
   * false-rejection rate (never accepted).  Single-run contexts and
   * batched runs (abc_batch_init) alike.  Not with ABC_STEP_MCMC. */
  int32_t surrogate;        /* 0 off, 1 on                                              */
  int32_t surrogate_start;  /* first generation that screens (>= 1)                      */
  int32_t surrogate_steps;  /* Adam steps after each generation                          */
  int32_t surrogate_batch;  /* minibatch size (<= 65536)                                 */
  float surrogate_lr;       /* Adam learning rate                                       */
  float surrogate_tau;      /* screen temperature in log1p-distance units               */
  float surrogate_rho_min;  /* floor of the pass probability (0 < rho_min <= 1)          */
  float audit_frac;         /* audit probability of a screened-out proposal             */
  int32_t surrogate_ring;   /* training pairs kept; 0 = min(2^21, 16 N)                 */
  /* Real-shape Beta rules: REAL (a, b) = (p1, p2), both in [2^-20, 2^20];
   * MEAN_VAR 0 < p1 < 1 (stage-1 mean), 0 < p2 <= 1 (stage-1 variance);
   * MODE_CONC 0 <= p1 <= 1 (stage-1 mode), 2 <= p2 <= 2^20 (stage-1
   * concentration).  (1/3, 1/18) and (0, 3) give Beta(1, 2) at stage 1, the
   * paper's a_1 = 1, b_1 = 2.  Shapes derived at later stages are clamped to
   * [2^-20, 2^20]. */
  float beta_p1;
  float beta_p2;
  /* Run budget (Sec. 4.1: each trial stops on the stage that reached 1000
   * simulation runs, a simulation run being one batch of M parallel
   * simulations, and that stage finishes): generation 0 counts ceil(N / M)
   * batches, generation t its own; once a generation ends with the count at
   * or above max_total_batches, later generations do not run
   * (ABC_STOP_TOTAL).  0: no budget. */
  int32_t max_total_batches;
  /* Batches simulated together per round, 1..256 (0 means 1): the batches
   * of a stage depend on the stage's state only, so K of them are proposed
   * and simulated at once and accepted in (batch, slot) order; the batches
   * after the one that fills N are discarded, uncounted.  Results and
   * statistics equal those of K = 1 bit for bit; small M (latency-bound
   * rounds) run faster.  The proposal buffers hold K M slots.  Generations
   * that screen with the surrogate run one batch per round. */
  int32_t spec_batches;
  /* Tolerance target: once a generation t >= 1 ends with eps_t <= eps_stop
   * the run is finished -- abc_generation returns ABC_STOP_TARGET and runs
   * nothing, and a batched run stops like one whose run budget is used up.
   * 0: no target.  (abc_run's eps_target does the same for one call.) */
  float eps_stop;
  /* ABC_STEP_MCMC: initial step s0 > 0 (variance in unit-cube coordinates),
   * and the adaptation window in batches that walk with the step (those of
   * generations t >= 1; generation 0 has no step).  After each such batch
   * b = 0, 1, ... with b < window, s <- s (1 + (A - A_T) / ((1 - A_T)(k + 1)))
   * in fp64, A = accepted / simulated slots of the batch (0 if none),
   * A_T = 0.234, k = adaptations so far; proposals use (float) s.  Eq. 15 as
   * printed would make s negative whenever A < A_T: this is its reading as
   * a multiplicative Robbins-Monro step.  mcmc_adapt = 0 gives the paper's
   * window, 10% of the run budget: ceil(max_total_batches / 10) (0, no
   * adaptation, without a budget). */
  float mcmc_s0;
  int32_t mcmc_adapt;
} abc_config;

/* Fill a config with the paper's defaults (SAIRD, binomial flows, alpha 0.5,
 * paper Beta schedule, paper weights, FP32, 64 batches, 64 redraws). */
ABC_API void abc_config_default(abc_config* cfg);

/* ---- step entry points (device buffers, stream-ordered) ---------------- */

/* Philox4x32-10 blocks: out[4i..4i+3] = philox(ctr[4i..4i+3], key).
 * ctr, out: device, n blocks.  For pinning the generator against others. */
ABC_API int abc_philox(const uint32_t* ctr, uint32_t key0, uint32_t key1, int64_t n, uint32_t* out,
               void* stream);

/* A0 synthetic observations (stand-in for the JHU series, Sec. 2.2 and 4):
 * theta* = lo + v (hi - lo) with v from the OBS_THETA stream (c0 = 0,
 * c1 = attempt, c2 = 0..1), simulated with the OBS stream (c1 = attempt),
 * redrawn until A_T > A0, at most 64 attempts.  box_lo/hi: host float[8].
 * obs: device int32 [3][T+1] (rows A, R, D; column t = day t, day 0 =
 * init_ard); theta_star: device float[8]; attempts: device int32[1]
 * (attempts used, or -64 when none grew). */
ABC_API int abc_synth_obs(const abc_config* cfg, const float* box_lo, const float* box_hi, int32_t* obs,
                  float* theta_star, int32_t* attempts, void* stream);

/* Stage 0 (Sec. 2.4): u_j ~ U(0,1)^8 from the PRIOR stream (c0 = j, c1 = 0,
 * c2 = 0..1).  u: device float [8][n]. */
ABC_API int abc_prior(const abc_config* cfg, int64_t n, float* u, void* stream);

/* A2-A3 simulator (Sec. 2.2, Eq. 3-5) and Euclidean distance (Sec. 2.3):
 * for each i < n, theta = lo + u_i (hi - lo), simulate T days with the
 * Philox counters (c0_idx ? c0_idx[i] : i, c1, 4 day + block, tag) and
 * return dist[i] = sqrt(sum_t sum_{A,R,D} (sim - obs)^2) over days 1..T
 * (exact integer sum, one correctly rounded conversion and sqrt).
 * obs: device int32 [3][T+1] (SAIRD; NULL gives distance 0); u: device
 * float [8][n]; c0_idx: device u32[n] or NULL; skip: device u8[n] or NULL
 * (skip[i] != 0 gives +inf and no simulation); dist: device double[n];
 * traj: device int32 [T+1][6][n] (S, I, A, R, D, Ru per day) or NULL. */
ABC_API int abc_simulate(const abc_config* cfg, const int32_t* obs, const float* u, int64_t n,
                 const uint32_t* c0_idx, uint32_t c1, uint32_t tag, const uint8_t* skip,
                 double* dist, int32_t* traj, void* stream);

/* A4 tolerance (Eq. 8): *out = the k-th smallest of d[0..n) (1 <= k <= n),
 * the lower order statistic, ties kept.  d: device double[n], all >= 0 or
 * +inf (no NaN); out: device double[1].  Radix select on the bit patterns. */
ABC_API size_t abc_select_scratch_bytes(int64_t n);
ABC_API int abc_select_kth(const double* d, int64_t n, int64_t k, double* out, void* scratch,
                   size_t scratch_bytes, void* stream);

/* A5 stage prior, weights and prefix (Eq. 9-11): survivors d_j <= *eps;
 * r_j = *eps - d_j (mode ABC_W_PAPER) or W_j (ABC_W_IMPORTANCE), 0 for
 * non-survivors; q_j = floor(r_j * s) with s = (2^32 - 1) / max r in fp64
 * (the largest weight gets 2^32 - 1 exactly, none more; q_j = 1 for every
 * survivor when max r is 0); prefix = inclusive sum of q as u64, so the
 * total is prefix[n-1].  d, W: device double[n] (W unused in paper mode,
 * may be NULL); eps: device double[1]; q: device u32[n]; prefix: device
 * u64[n]. */
ABC_API size_t abc_prefix_scratch_bytes(int64_t n);
ABC_API int abc_resample_prefix(const double* d, const double* W, int64_t n, const double* eps,
                        int32_t mode, uint32_t* q, uint64_t* prefix, void* scratch,
                        size_t scratch_bytes, void* stream);

/* Allocation-free variant of abc_resample_prefix (the paper has no
 * counterpart; it exists for callers that cannot allocate device memory when
 * they run this step -- for example code whose device memory is owned by a
 * pool or a fixed budget it does not control).  Same arguments and results as
 * abc_resample_prefix, without the scratch buffer: the scratch lives in one
 * fixed array inside the library (257 KB per device, held until the process
 * exits), which is enough for n <= ABC_NOALLOC_MAX_N = 2^24; larger n returns
 * ABC_E_TOO_LARGE.  The first call on a device looks up that array's device
 * address, so make it before any stream capture; the address is kept for the
 * life of the process, so do not call this entry point again on a device
 * after cudaDeviceReset() there (the array is reloaded at another address
 * with the new context).  Every call shares the one
 * array: calls that overlap on the GPU (other streams, other threads) race
 * and must be serialised by the caller.  No device memory is allocated. */
#define ABC_NOALLOC_MAX_N (1LL << 24)
ABC_API int abc_resample_prefix_noalloc(const double* d, const double* W, int64_t n,
                                        const double* eps, int32_t mode, uint32_t* q,
                                        uint64_t* prefix, void* stream);

/* A6-A7 BDSS proposal (Eq. 11, 16, 17): for each slot i < slots with
 * c0 = c0_idx ? c0_idx[i] : i and attempt a = 0..max_redraw-1: ancestor =
 * first k with prefix[k] > floor(U64 * total / 2^64) (ANCESTOR stream, c2 =
 * a), s ~ Beta(a_t, b) (BETA stream, c2 = a << 8 | block), z ~ N(0, I8)
 * (WALK stream), u' = u_anc + sqrt(s) z; the first u' inside [0,1]^8 is kept,
 * else flag = 1.  a_t = beta_a, or in paper mode (cfg->beta_mode) a_t =
 * (float)(*eps / *eps1) (1 when *eps1 is 0) and b = beta_b as given (integer
 * b, product form; in paper mode 0 means Beta(a_t, 2t) by the Gamma ratio,
 * a_t clamped to [2^-20, 2^20], t = c1 >> 16 >= 1, as generations from 513
 * on draw it).  Under the real-shape rules (ABC_BETA_REAL, _MEAN_VAR,
 * _MODE_CONC) beta_a and beta_b are ignored: the shapes follow from
 * cfg->beta_p1, cfg->beta_p2, the ratio and the stage t = c1 >> 16 (t >= 1
 * for the last two), and s is drawn by the Gamma ratio (BETA stream, c2 =
 * a << 8 | block, blocks 0..63 for X and 64..127 for Y).  Under
 * ABC_STEP_MCMC every slot walks with s = beta_a > 0 and no BETA block is
 * read (beta_b ignored).
 * u: device float [8][n]; prefix: device u64[n]; eps, eps1: device double[1]
 * (read by the paper, mean-variance and mode-concentration rules; may be
 * NULL otherwise); outputs: device
 * u_out [8][slots], s_out[slots], anc_out, attempts_out (int32), flag_out (u8). */
ABC_API int abc_propose(const abc_config* cfg, const float* u, int64_t n, const uint64_t* prefix,
                const double* eps, const double* eps1, float beta_a, int32_t beta_b,
                int64_t slots, const uint32_t* c0_idx, uint32_t c1, float* u_out, float* s_out,
                int32_t* anc_out, int32_t* attempts_out, uint8_t* flag_out, void* stream);

/* A8 acceptance and assembly (Sec. 2.3, Sec. 4.1): proposals i < M with
 * flag[i] == 0 and dp[i] <= *eps are appended to the population in slot
 * order at positions *filled, *filled + 1, ... while below N.  On return
 * *filled = min(N, *filled + accepted), counters[0] += accepted,
 * counters[1] += number of flagged (redraw-exhausted) slots.
 * up [8][M], dp, sp, ap, flag: device proposal arrays; eps: device double[1];
 * u_pop [8][N], d_pop, s_pop, anc_pop: device population arrays;
 * filled: device int64[1]; counters: device int64[2]. */
ABC_API size_t abc_accept_scratch_bytes(int64_t M);
ABC_API int abc_accept_append(const float* up, const double* dp, const float* sp, const int32_t* ap,
                      const uint8_t* flag, int64_t M, const double* eps, int64_t N, float* u_pop,
                      double* d_pop, float* s_pop, int32_t* anc_pop, int64_t* filled,
                      int64_t* counters, void* scratch, size_t scratch_bytes, void* stream);

/* A9 importance weights (an extension beyond the paper; the paper's weights are
 * Eq. 10): for each row j < rows,
 *   logW[j] = 4 log(2 pi s_j) - log sum_k (q_k / total) exp(-|u'_j - u_k|^2 / (2 s_j))
 * = -log sum_k rhat_k N(u'_j; u_k, s_j I8) (uniform prior on the unit cube),
 * over columns k < n with q_k > 0; total = prefix[n-1]; s_j == 0 gives
 * -inf.  prec: ABC_P_FP32 (CUDA cores) or ABC_P_BF16_TC (tensor cores).
 * up [8][rows], s[rows], u [8][n], q[n], prefix[n]: device; logW: device
 * double[rows]. */
/* ABC_P_BF16_TC: the exponent of each pair is an inner product of row and
 * column feature vectors, evaluated by tcgen05.mma with every feature split
 * into three bf16 parts (24 significant bits) and fp32 accumulation in tensor
 * memory; the per-row log-sum-exp runs in fp32 with an fp64 combine.  The
 * call synchronises the stream to read the kernel's error word (a wait that
 * timed out gives ABC_E_DEVICE). */
ABC_API size_t abc_weights_scratch_bytes(int64_t rows, int64_t n);
ABC_API int abc_weights(const float* up, const float* s, int64_t rows, const float* u, const uint32_t* q,
                const uint64_t* prefix, int64_t n, int32_t prec, double* logW, void* scratch,
                size_t scratch_bytes, void* stream);

/* Diagnostic of the tensor-core path: one 128 x 256 x 64 bf16 product
 * D[i][n] = sum_k A[i][k] B[n][k] (fp32) with the operand layout and
 * descriptors the weight kernel uses.  A, B: device bf16 tiles packed as
 * 8 x 8 core matrices, element (r, k) at index ((r/8)*8 + k/8)*64 + (r%8)*8
 * + k%8 (A: 128 rows, 16 KB; B: 256 rows, 32 KB); D: device float [128][256].
 * Synchronises the stream; ABC_E_DEVICE if a wait timed out. */
ABC_API int abc_tc_probe(const void* A, const void* B, float* D, void* stream);

/* Posterior-predictive simulation (Sec. 4.2: the learned samples simulated
 * from day zero over the training window plus the days ahead, summarised
 * per day by the median and the central 99% range).  R draws from the
 * population u (device float [8][N]) in proportion to W (device double[N];
 * NULL: equal weights), quantised and drawn like the stage prior
 * (Eq. 10-11) with Philox block (j, 0, 0, ABC_TAG_PREDICT); each draw is
 * simulated for `days` days (cfg n_days and observations are not used) with
 * counters (j, 0, 4 day + block, ABC_TAG_PREDICT_SIM); out (device int32
 * [days + 1][3][nq], series A, R, D) receives for every day and series the
 * order statistic of rank ceil(quant[i] R), clamped to [1, R] (the lower
 * order statistic, as Eq. 8).  quant: host double[nq], levels in (0, 1].
 * SAIRD model only.  Synchronises the stream. */
ABC_API size_t abc_predict_scratch_bytes(int64_t N, int64_t R, int32_t days, int32_t nq);
ABC_API int abc_predict(const abc_config* cfg, const float* u, const double* W, int64_t N,
                        int64_t R, int32_t days, const double* quant, int32_t nq, int32_t* out,
                        void* scratch, size_t scratch_bytes, void* stream);

/* Measurement helper (no counterpart in the paper): the sustained rate of
 * ex2.approx.f32 on this GPU in exponentials per second, from a saturating
 * microbenchmark (eight independent chains per thread, 8 blocks of 256 per
 * SM, best of three timed launches).  The tensor-core weight kernel is bound
 * by this unit; bench.py quotes its roofline against this rate.
 * Synchronises the stream. */
ABC_API int abc_ex2_probe(double* ex2_per_second, void* stream);

/* Self-check (no counterpart in the paper): the simulator and the logarithm
 * replace two correctly rounded divisions on bounded operand domains by a
 * shorter sequence (the quotient by the hardware reciprocal approximation,
 * corrected once by its exact remainder, after Markstein).  which = 0 enumerates the
 * logarithm's domain (n = m - 1, d = m + 1, every float m in
 * [sqrt(2)/2, sqrt(2)], 8.4e6 pairs); which = 1 BINV's (a / k, every float a
 * in [2^-100, 2^100], k = 2..111, 1.8e11 pairs); which = 2 the square root
 * that replaces __fsqrt_rn in the binomial and Box-Muller draws the same way
 * (every float in [2^-24, 2^32), 4.7e8 values); which = 3 the uniform built
 * from a Philox word's bits (1.m - (1 - 2^-24)) against its direct form
 * ((x >> 9) + 1/2) 2^-23 by conversion (all 2^23 significands).
 * *mismatches receives the count of operands whose result differs in any bit
 * from the exact form's (0 expected).  ABC_E_INVAL for another which.
 * Synchronises the stream. */
ABC_API int abc_numerics_check(int32_t which, uint64_t* mismatches, void* stream);

/* Stable LSD radix sort (no counterpart in the paper; the weight pass uses it
 * to put its rows and columns in spatial order): keys_out / vals_out = the n
 * pairs (keys[i], vals ? vals[i] : i) ordered by the low `bits` bits of the
 * key (1 <= bits <= 32), equal keys in input order.  keys, vals, keys_out,
 * vals_out: device arrays of n uint32 / int32 (the outputs must not alias the
 * inputs); 0 <= n <= 2^30.  Scratch is allocated on the stream and freed
 * after the sort (stream-ordered); ABC_E_NOMEM if that fails. */
ABC_API int abc_radix_sort(const uint32_t* keys, const int32_t* vals, int64_t n, int32_t bits,
                           uint32_t* keys_out, int32_t* vals_out, void* stream);

/* Test hooks for failure detection (no counterpart in the paper).  Both make
 * a failure happen on the host side of a call, never a device fault.
 * abc_set_wait_limit_ns: time limit of the tensor-core weight kernel's
 * pipeline waits (mbarrier phases of its copy / MMA / epilogue roles) for
 * launches made from now on; 0 restores the default of 2 s.  A wait that
 * runs out records an error word and its role stops; the waits for the
 * CTA's own copies and products before it exits keep the 2 s limit, so
 * nothing is in flight when it ends, and the call returns ABC_E_DEVICE with
 * the context still usable.  A shortened limit only serves to test that
 * path.  abc_inject_alloc_failure: the device allocation of a context
 * (abc_init) after `after` successful ones fails as if cudaMalloc had,
 * giving ABC_E_NOMEM with everything allocated so far released; every later
 * one fails too until the hook is reset with a negative value.  Neither is
 * thread-safe against concurrent calls in other threads. */
ABC_API void abc_set_wait_limit_ns(uint64_t ns);
ABC_API void abc_inject_alloc_failure(int64_t after);

/* A10 normalisation (fp64): W_j = exp(logW_j - max) / sum, *ess = 1 / sum W^2;
 * all -inf gives W = 1/n, ess = n.  logW: device double[n]; W: device
 * double[n]; ess: device double[1]. */
ABC_API size_t abc_normalize_scratch_bytes(int64_t n);
ABC_API int abc_normalize(const double* logW, int64_t n, double* W, double* ess, void* scratch,
                  size_t scratch_bytes, void* stream);

/* A11 delayed-acceptance screen (an extension beyond the paper; the paper simulates
 * every proposal; two-stage acceptance after Christen & Fox 2005).  For
 * slot i < M with flag[i] == 0 the surrogate's prediction of log1p d is
 * y0 = ystat[0] + ystat[4] * Y[4 i] (fp32 product, then sum) and
 *   rho[i] = min(max(1 / (1 + exp(-(log1p((float) *eps) - y0) / tau)), rho_min), 1)
 * in fp32 with the library's own exp and log1p (a NaN prediction gives
 * rho_min).  sflag[i] = 0 (simulate; may be accepted) when
 * U(i, c1, 0, ABC_TAG_SCREEN) < rho[i]; else 2 (simulate for the audit of
 * the false-rejection rate; never accepted) when
 * U(i, c1, 0, ABC_TAG_AUDIT) < audit_frac; else 3 (screened out).
 * flag[i] != 0 (redraw-exhausted) gives sflag 1 and rho 1.  tau = cfg
 * surrogate_tau, rho_min = cfg surrogate_rho_min, audit_frac = cfg
 * audit_frac, the Philox key from cfg seed and run_id; U(.) is the first
 * word of the block, mapped as everywhere.  Y: device float [M][4];
 * ystat: device float[8] (means, then standard deviations); flag: device
 * u8[M] or NULL (all 0); eps: device double[1]; rho: device float[M];
 * sflag: device u8[M].  ABC_E_INVAL for bad sizes or parameters. */
ABC_API int abc_screen(const abc_config* cfg, const float* Y, const float* ystat,
                       const uint8_t* flag, int64_t M, const double* eps, uint32_t c1, float* rho,
                       uint8_t* sflag, void* stream);

/* ---- context: whole generations ---------------------------------------- */
typedef struct abc_ctx abc_ctx;

typedef struct {
  int32_t generation;       /* index t of the generation these stats describe       */
  int32_t status;           /* ABC_OK or ABC_STOP_BUDGET                             */
  double eps;               /* eps_t used for acceptance (+inf for t = 0)           */
  double eps1;              /* eps_1 (0 before generation 1)                        */
  double ess;               /* effective sample size of the new population          */
  float beta_a;             /* step-size Beta shape used (a_t, b_t); ABC_STEP_MCMC:  */
  int32_t beta_b;           /*   beta_a = s of the first batch, beta_b = 0           */
  int64_t batches;          /* batches of M proposals run                           */
  int64_t sims;             /* simulations run (flagged slots excluded)             */
  int64_t sim_days;         /* particle-days simulated                              */
  int64_t exhausted;        /* slots whose redraws were exhausted                   */
  int64_t accepted;         /* acceptances, including those beyond N                */
  int64_t pairs;            /* rows x surviving columns of the O(N^2) weight pass    */
  int64_t launches;         /* kernels this library launched for the generation     */
  double ms;                /* device time of the generation (CUDA events)          */
  double ms_sim;            /* of which the simulator launches (all batches)        */
  double ms_weights;        /* of which the O(N^2) weight pass                      */
  int64_t screened;         /* proposals the surrogate did not pass                 */
  int64_t audited;          /* of which simulated for the audit                     */
  int64_t audit_accepted;   /* audited proposals with d <= eps (false rejections)   */
  double train_loss;        /* surrogate minibatch loss after the generation        */
  double ms_screen;         /* device time of the screening inference               */
  double ms_train;          /* device time of the surrogate training                */
  int64_t rows_tc;          /* weight rows on the tensor cores (the rest on FP32)    */
  double ms_tc;             /* device time of the tensor-core weight kernel          */
  double ms_fp32;           /* device time of the FP32 weight kernel                 */
  float beta_bf;            /* b_t as fp32 (beta_b is 0 under the real-shape rules)  */
  float mcmc_s;             /* ABC_STEP_MCMC: the step s after the generation's      */
                            /*   batches (beta_a: s of its first batch)              */
  int64_t rows_exp;         /* rows whose tensor-core sums were kept (error bound    */
                            /*   small enough); the rest of rows_tc were refined    */
  int64_t pairs_tc;         /* (row, column) pairs in the tiles the tensor-core      */
                            /*   kernel multiplied (column tiles beyond every       */
                            /*   candidate radius of a class-1 row tile are skipped) */
} abc_gen_stats;

/* Validate cfg, allocate every device buffer (owned by the context), copy
 * obs (host int32 [3][T+1]; NULL for the toy model) and bind the stream. */
ABC_API int abc_init(const abc_config* cfg, const int32_t* obs, void* stream, abc_ctx** out);
/* Run one generation: the first call runs stage 0 (prior); later calls
 * run t = 1, 2, ...  Returns ABC_STOP_BUDGET (population unchanged) when
 * max_batches batches did not yield N acceptances, and ABC_STOP_TOTAL
 * (nothing runs) once the run budget max_total_batches is used up. */
ABC_API int abc_generation(abc_ctx* ctx);
/* Run generations until n_generations exist or eps_t <= eps_target
 * (eps_target <= 0 disables it) or the run budget is used up; returns the
 * last generation's status (ABC_STOP_TOTAL for the budget). */
ABC_API int abc_run(abc_ctx* ctx, int32_t n_generations, double eps_target);
/* Start the context over at stage 0 as a new run with the given run_id (the
 * Philox key becomes (seed_lo, seed_hi ^ run_id)), keeping its buffers,
 * observed series and stream: statistics, generation count, run budget
 * count and eps_1 are cleared, and the surrogate (if any) is re-initialised
 * from the new key.  The next abc_generation runs stage 0; the results equal
 * those of a fresh context whose config carries that run_id.  Synchronises
 * the stream. */
ABC_API int abc_reset(abc_ctx* ctx, uint32_t run_id);
/* Copy the population: u [8][N] float, dist, W double[N], s float[N] and
 * anc int32[N] (ancestor index in the previous population, -1 at t = 0);
 * any pointer may be NULL; on_device != 0 means the pointers are device
 * memory (device-to-device copy on the context stream), else host. */
ABC_API int abc_get_population(abc_ctx* ctx, float* u, double* dist, double* W, float* s, int32_t* anc,
                       int32_t on_device);
/* Stats of generation t: 0 <= t < abc_generations(ctx) (the completed
 * generations), and t = abc_generations(ctx) when the last generation stopped
 * on its batch budget (recorded with status ABC_STOP_BUDGET, not counted;
 * batched runs record it the same way). */
ABC_API int abc_get_stats(abc_ctx* ctx, int32_t t, abc_gen_stats* out);
ABC_API int32_t abc_generations(const abc_ctx* ctx);
/* abc_predict on the context's current population (its weights, its
 * model and key); out_host: host int32 [days + 1][3][nq].  Allocates its
 * scratch for the call. */
ABC_API int abc_predict_population(abc_ctx* ctx, int64_t R, int32_t days, const double* quant,
                                   int32_t nq, int32_t* out_host);
/* Checkpoint: serialise (or restore) the generation index, eps_1 and the
 * population.  Philox is stateless, so a restored context continues
 * bit-identically.  get: *len is in/out (call with buf NULL for the size). */
ABC_API int abc_get_state(abc_ctx* ctx, void* buf, size_t* len);
ABC_API int abc_set_state(abc_ctx* ctx, const void* buf, size_t len);
ABC_API void abc_free(abc_ctx* ctx);
ABC_API const char* abc_strerror(int code);

/* ---- surrogate MLP (an extension beyond the paper; the paper has no surrogate) ----
 * 8 -> 256 -> 256 -> 4 with tanh-form GELU; parameters in one fp32 array
 * (row = output): W1[256][8], b1[256], W2[256][256], b2[256], W3[4][256],
 * b3[4] (69124 values); every product uses their bf16 rounding with fp32
 * accumulation.  These entry points expose the kernels the context uses. */
typedef struct abc_mlp abc_mlp;
ABC_API int32_t abc_mlp_param_count(void);
/* Weights U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from Philox (key = seed), zero
 * biases, zero Adam moments. */
ABC_API int abc_mlp_create(uint64_t seed, abc_mlp** out);
ABC_API int abc_mlp_set_params(abc_mlp* m, const float* host_params);
/* host_params: fp32 master values; host_bf16 (nullable): the bf16 copy's bits */
ABC_API int abc_mlp_get_params(abc_mlp* m, float* host_params, uint16_t* host_bf16);
ABC_API size_t abc_mlp_scratch_bytes(int32_t batch, int64_t n);
/* Gradient of the mean squared error over B samples and 4 outputs: the
 * three 256-wide products (layer 2 forward, its input gradient and its
 * weight gradient) on tcgen05 tensor cores with bf16 operands -- weights,
 * hidden activations and hidden gradients rounded to bf16 -- and fp32
 * accumulation; layers 1 and 3 and the bias sums on CUDA cores in fp32; all
 * reductions in a fixed order (deterministic).  X device [B][8], T device
 * [B][4]; grad device [69124]; sse device float[1] receives the sum of
 * squared errors.  Synchronises the stream; ABC_E_DEVICE if a tensor-core
 * wait timed out. */
ABC_API int abc_mlp_grad(abc_mlp* m, const float* X, const float* T, int32_t B, float* grad,
                         float* sse, void* scratch, size_t scratch_bytes, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, step >= 1) on the fp32
 * parameters; refreshes the bf16 copy. */
ABC_API int abc_mlp_adam(abc_mlp* m, const float* grad, int64_t step, float lr, void* stream);
/* Inference on tensor cores: Y device [n][4] for u device [8][n] (the input
 * layer and layer 2 on tcgen05 with fp32 accumulation, the input split into
 * three bf16 parts so that the input layer is fp32-accurate, the hidden layer
 * rounded to bf16, GELU and layer 3 fused into the epilogue).  Synchronises
 * the stream. */
ABC_API int abc_mlp_forward(abc_mlp* m, const float* u, int64_t n, float* Y, void* scratch,
                            size_t scratch_bytes, void* stream);
ABC_API void abc_mlp_free(abc_mlp* m);

/* ---- batched runs (batched form, an extension; the paper runs one problem at
 * a time) ------------------------------------------------------------------
 * n_runs independent runs (own config, seed, size, horizon and observed
 * series each) advanced together.  After stage 0, every generation of every
 * run is ONE CUDA graph launch: an independent branch per run whose batch
 * loop is a device-side conditional WHILE node, so no host round trip
 * happens inside a generation and runs of different sizes overlap on the
 * GPU.  Results equal those of separate contexts with the same configs bit
 * for bit (same kernels, same Philox counters).  A run whose generation uses
 * up its batch budget stops (status ABC_STOP_BUDGET in its stats) and is
 * skipped afterwards; the others continue.  A run whose run budget
 * (max_total_batches) is used up stops the same way after its last
 * generation (status ABC_OK there; the start kernel of the next launch
 * skips it).  The branches share the process's hardware work queues: with
 * many runs, set CUDA_DEVICE_MAX_CONNECTIONS (e.g. 32; the default is 8)
 * before the first CUDA call. */
typedef struct abc_batch abc_batch;
/* cfgs: host array of n_runs configs; obs: host array of n_runs host
 * pointers to int32 [3][T_r+1] series (entries may be NULL for the toy).
 * A run with surrogate != 0 screens inside its graph branch (inference,
 * screen, compaction and simulation of the passed slots per batch; training
 * after the generation), with the results of a single context of that
 * config. */
ABC_API int abc_batch_init(const abc_config* cfgs, int32_t n_runs, const int32_t* const* obs,
                           void* stream, abc_batch** out);
/* First call: stage 0 of every run; later calls: one graph launch. */
ABC_API int abc_batch_generation(abc_batch* b);
/* Generations until n_generations exist or no run is active. */
ABC_API int abc_batch_run(abc_batch* b, int32_t n_generations);
/* Runs that have not stopped (budget, run budget); before stage 0 all. */
ABC_API int32_t abc_batch_active(const abc_batch* b);
ABC_API int32_t abc_batch_runs(const abc_batch* b);
ABC_API int32_t abc_batch_generations(const abc_batch* b);
ABC_API int abc_batch_get_stats(abc_batch* b, int32_t run, int32_t t, abc_gen_stats* out);
ABC_API int abc_batch_get_population(abc_batch* b, int32_t run, float* u, double* dist, double* W,
                                     float* s, int32_t* anc, int32_t on_device);
/* Autotuner: for each run's shape class (log2 N, T / 30, weight mode and
 * precision, SM count) times the simulator at 64/128/256 threads per block
 * and the weight pass at 1/2/4 times its default column chunks on the run's
 * current population (CUDA events, median of 3), keeps the fastest, and
 * reads/writes the choices as JSON at cache_path (NULL: no cache).  Call
 * after stage 0; the graph is rebuilt with the chosen shapes.  Launch shapes
 * never change results. */
ABC_API int abc_batch_autotune(abc_batch* b, const char* cache_path);
ABC_API int abc_batch_tuning(const abc_batch* b, int32_t run, int32_t* sim_threads,
                             int32_t* w_mult);
ABC_API void abc_batch_free(abc_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* ABCSMC_H */
