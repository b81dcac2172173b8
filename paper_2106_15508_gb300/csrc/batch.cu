// batch.cu -- many independent ABC-SMC runs advanced together (a batched
// form, an extension: the paper runs one problem at a time).
//
// Each run keeps its own buffers (an abc_ctx).  One generation of every run
// is one CUDA graph launch: the graph holds an independent branch per run --
//   tolerance select -> eps_1 on the first generation -> stage-prior prefix
//   -> start kernel -> WHILE(not filled and budget left) { propose ->
//   simulate -> accept -> condition kernel } -> finish kernel -> survivor
//   columns -> O(N^2) weights -> normalisation -> commit (copy the new
//   population over the current one)
// -- so the data-dependent batch loops run on the device (conditional WHILE
// nodes set by cudaGraphSetConditional) with no host round trip, and the
// branches of runs of different sizes and horizons overlap on the GPU.  All
// Philox counters (generation, batch) are read from per-run device state, so
// one instantiated graph serves every generation.  A run whose generation
// exhausts its batch budget stops: its later branches are skipped by a flag,
// and so are those of a run whose run budget (batches over all generations)
// is used up.
//
// Launch shapes (simulator block size, column chunks of the weight pass) are
// picked per shape class by a small autotuner that times the candidates on
// the runs' own data and caches the choice in a JSON text file.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "batch.cuh"

namespace abc {

__global__ void k_run_start(RunDev* r, int paper_beta, int fixed_b, int K,
                            cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  r->off = r->done;
  r->b = 0;
  r->c1 = r->t << 16;
  // batches of the first round (K at most, within the batch budget)
  r->k_lim = K < r->max_batches ? K : r->max_batches;
  r->used = 1;
  r->rounds = 0;
  // integer b of the product form (0: the Gamma ratio, under the real-shape
  // rules and for the paper's b = 2t above 1024)
  r->beta_b = paper_beta ? (r->t <= 512u ? static_cast<int>(2 * r->t) : 0) : fixed_b;
  r->filled = 0;
  r->accepted = 0;
  r->exhausted = 0;
  r->batches = 0;
  r->status = 0;
  if (r->t == 1 && !r->done) r->eps1 = r->eps;  // eps_1 is the first generation's eps
  cudaGraphSetConditional(h, r->done ? 0u : 1u);
}

// after a round: advance by the batches it used (1, or up to K when several
// batches run per round: the one that filled N is the last counted)
__global__ void k_run_cond(RunDev* r, long long N, int K, cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int used = r->used;
  r->rounds += 1;
  r->batches += used;
  r->b += static_cast<uint32_t>(used);
  r->c1 = (r->t << 16) | r->b;
  const int left = r->max_batches - static_cast<int>(r->b);
  r->k_lim = K < left ? K : left;
  const bool more = r->filled < N && r->b < static_cast<uint32_t>(r->max_batches);
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

__global__ void k_run_finish(RunDev* r, long long N) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (r->done) return;
  const bool ok = r->filled >= N;
  r->status = ok ? ABC_OK : ABC_STOP_BUDGET;
  r->off = ok ? 0 : 1;
  if (!ok) r->done = 1;
  // run budget (Sec. 4.1): this generation is kept, later ones are skipped
  r->batches_total += r->batches;
  if (ok && r->max_total > 0 && r->batches_total >= r->max_total) r->done = 1;
  // tolerance target: this generation is kept, later ones are skipped
  if (ok && r->eps_stop > 0.0 && r->eps <= r->eps_stop) r->done = 1;
}

// the new population becomes the current one (skipped when the run is off)
__global__ void k_run_commit(RunDev* r, int64_t N, float* __restrict__ u_cur,
                             const float* __restrict__ u_nxt, double* __restrict__ d_cur,
                             const double* __restrict__ d_nxt, double* __restrict__ W_cur,
                             const double* __restrict__ W_nxt, float* __restrict__ s_cur,
                             const float* __restrict__ s_nxt, int32_t* __restrict__ a_cur,
                             const int32_t* __restrict__ a_nxt) {
  if (r->off) return;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < N;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
#pragma unroll
    for (int d = 0; d < 8; ++d) u_cur[d * N + i] = u_nxt[d * N + i];
    d_cur[i] = d_nxt[i];
    W_cur[i] = W_nxt[i];
    s_cur[i] = s_nxt[i];
    a_cur[i] = a_nxt[i];
  }
}

__global__ void k_run_advance(RunDev* r) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && !r->off) r->t += 1;
}

__global__ void k_run_fill_paper(RunDev* r, double* __restrict__ W, int64_t N) {
  if (r->off) return;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < N) W[i] = 1.0 / static_cast<double>(N);
  if (i == 0) r->ess = static_cast<double>(N);
}

int screened_batch(const SurView& s, const SimParams& p, const int32_t* obs, const float* up,
                   const float* sp, const int32_t* ap, const uint8_t* flag, int64_t M,
                   const double* eps, uint32_t c1, const uint32_t* c1_dev, int64_t N,
                   float* u_pop, double* d_pop, float* s_pop, int32_t* a_pop, int64_t* filled,
                   int64_t* counters, unsigned long long* exhausted, void* scratch,
                   size_t scratch_bytes, int sim_threads, unsigned** inf_err, cudaStream_t st,
                   const cudaEvent_t* ev) {
  int rc;
  if (ev) ABC_CUDA_TRY(cudaEventRecord(ev[0], st));
  // predictions of the proposals (the error word is reset once per generation)
  if ((rc = mlp_infer(s.mlp, up, M, s.Yp, s.sscratch, s.sscratch_bytes, inf_err, st, false,
                      s.inf_err, s.ystat + 8)))
    return rc;
  // delayed acceptance: rho and the pass / audit decision, then the slots to
  // simulate in slot order (stride M, count *Mc on the device)
  if ((rc = screen_and_compact(s.Yp, s.ystat, flag, M, eps, p.k0, p.k1, c1, s.tau, s.rho_min,
                               s.audit_frac, s.rho, s.sflag, up, sp, ap, s.cmp_u, s.cmp_s, s.cmp_a,
                               s.cmp_rho, s.cmp_flag, s.cmp_slot, s.Mc, s.sscratch, st, exhausted,
                               c1_dev, s.screen_on, s.simulated)))
    return rc;
  // each simulated slot with its own Philox counters; the rest get +inf
  if (ev) ABC_CUDA_TRY(cudaEventRecord(ev[1], st));
  if ((rc = launch_simulate_ordered(p, obs, s.cmp_u, M, c1, nullptr, s.cmp_d, scratch,
                                    scratch_bytes, st, c1_dev, nullptr, sim_threads, 0, s.cmp_slot,
                                    s.Mc, s.ard)))
    return rc;
  if (ev) ABC_CUDA_TRY(cudaEventRecord(ev[2], st));
  // audited slots (flag 2) are never accepted; each accepted particle keeps its rho
  if ((rc = launch_accept(s.cmp_u, s.cmp_d, s.cmp_s, s.cmp_a, s.cmp_flag, M, eps, N, u_pop, d_pop,
                          s_pop, a_pop, filled, counters, scratch, scratch_bytes, st, s.cmp_rho,
                          s.rho_pop)))
    return rc;
  if ((rc = audit_count(s.cmp_flag, s.cmp_d, s.Mc, eps, s.audit, st))) return rc;
  return ring_append(nullptr, M, s.cmp_u, s.cmp_d, s.ard, s.ring_head, s.ring_cap, s.RX, s.RY,
                     s.sscratch, st, s.Mc);
}

int sur_train(const SurView& s, const SimParams& p, const int* off_dev, cudaStream_t st) {
  if (s.steps <= 0) return ABC_OK;
  // the statistics' partial sums use the scratch before training reuses it
  int rc = ring_stats(s.RX, s.RY, s.ring_head, s.ring_cap, s.ystat, s.sscratch, st);
  if (rc) return rc;
  return mlp_train(s.mlp, s.RX, s.RY, s.ring_head, s.ring_cap, s.ystat, s.batch, s.steps,
                   s.train_step, s.lr, p.k0, p.k1, s.grad, s.trX, s.trT, s.loss, s.sscratch,
                   s.sscratch_bytes, st, off_dev, s.inf_err);
}

int batch_capture_run(BatchRun& br, cudaStream_t st, cudaStream_t body_st) {
  const int64_t l0 = launch_count();
  int64_t l_body0 = 0, l_body1 = 0;
  RunCtxView& v = br.v;
  RunDev* r = br.dev;
  int rc;
  // tolerance eps_t (Eq. 8) into the run state
  if ((rc = launch_select(v.d_cur, v.N, v.rank, &r->eps, v.scratch, v.scratch_bytes, st))) return rc;
  if ((rc = launch_resample_prefix(v.d_cur, v.W_cur, v.N, &r->eps, v.weight_mode, v.q, v.prefix,
                                   v.scratch, v.scratch_bytes, st)))
    return rc;
  // the start kernel sets the loop condition, so the WHILE node's handle is
  // created on the graph being captured before the node itself is added
  cudaGraphConditionalHandle h;
  cudaGraph_t body = nullptr;
  {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    ABC_CUDA_TRY(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, nullptr, nullptr, nullptr));
    if (cs != cudaStreamCaptureStatusActive) return ABC_E_CUDA;
    ABC_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
  }
  const int fixed_b = v.beta.mode == ABC_BETA_FIXED ? v.beta.b : 0;
  k_run_start<<<1, 32, 0, st>>>(r, v.beta.mode == ABC_BETA_PAPER, fixed_b, v.K, h);
  ABC_LAUNCH_CHECK();
  if (v.mcmc && (rc = launch_mcmc_begin(v.mcmc, &r->off, st))) return rc;
  const SurView& sv = v.sur;
  if (sv.on) {
    // screening from generation `start` once trained; this generation's counters
    if ((rc = sur_gate(&r->t, 0u, sv.start, sv.train_step, sv.screen_on, st))) return rc;
    ABC_CUDA_TRY(cudaMemsetAsync(sv.audit, 0, 2 * sizeof(unsigned long long), st));
    ABC_CUDA_TRY(cudaMemsetAsync(sv.simulated, 0, sizeof(long long), st));
    br.inf_err = sv.inf_err;
    ABC_CUDA_TRY(cudaMemsetAsync(sv.inf_err, 0, sizeof(unsigned), st));
  }
  {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t ndeps = 0;
    ABC_CUDA_TRY(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &edges, &ndeps));
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};  // the rest zero
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    ABC_CUDA_TRY(cudaGraphAddNode(&node, g, deps, edges, ndeps, &np));
    body = np.conditional.phGraph_out[0];
    ABC_CUDA_TRY(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1,
                                                     cudaStreamSetCaptureDependencies));
  }
  // loop body: one batch of M proposals, or K batches (K M slots, batch c1 +
  // slot / M) accepted in (batch, slot) order
  ABC_CUDA_TRY(cudaStreamBeginCaptureToGraph(body_st, body, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeRelaxed));
  l_body0 = launch_count();
  const bool spec = v.K > 1;
  const int64_t slots = v.M * v.K;
  rc = launch_propose(v.p, v.u_cur, v.N, v.prefix, v.beta, &r->eps, &r->eps1, slots, nullptr, 0u,
                      v.max_redraw, v.up, v.sp, v.ap, v.att, v.flag, body_st, &r->c1, &r->beta_b,
                      &r->off, spec ? v.M : 0, spec ? &r->k_lim : nullptr,
                      v.mcmc ? &v.mcmc->s_f : nullptr);
  if (!rc && sv.on) {
    // the surrogate screens the batch (a pass-all until it is trained)
    rc = screened_batch(sv, v.p, v.obs, v.up, v.sp, v.ap, v.flag, v.M, &r->eps, 0u, &r->c1, v.N,
                        v.u_nxt, v.d_nxt, v.s_nxt, v.a_nxt, reinterpret_cast<int64_t*>(&r->filled),
                        reinterpret_cast<int64_t*>(&r->accepted),
                        reinterpret_cast<unsigned long long*>(&r->exhausted), v.scratch,
                        v.scratch_bytes, br.sim_threads, nullptr, body_st);
  } else if (!rc) {
    rc = launch_simulate_ordered(v.p, v.obs, v.up, slots, 0u, v.flag, v.dp, v.scratch,
                                 v.scratch_bytes, body_st, &r->c1, &r->off, br.sim_threads,
                                 spec ? v.M : 0);
    if (!rc && spec)
      rc = launch_accept_spec(v.up, v.dp, v.sp, v.ap, v.flag, v.M, v.K, &r->k_lim, &r->eps, v.N,
                              v.u_nxt, v.d_nxt, v.s_nxt, v.a_nxt,
                              reinterpret_cast<int64_t*>(&r->filled),
                              reinterpret_cast<int64_t*>(&r->accepted), &r->used, v.scratch,
                              v.scratch_bytes, body_st);
    else if (!rc)
      rc = launch_accept(v.up, v.dp, v.sp, v.ap, v.flag, v.M, &r->eps, v.N, v.u_nxt, v.d_nxt,
                         v.s_nxt, v.a_nxt, reinterpret_cast<int64_t*>(&r->filled),
                         reinterpret_cast<int64_t*>(&r->accepted), v.scratch, v.scratch_bytes,
                         body_st);
    // the MCMC baseline adapts its step to this batch's acceptance
    if (!rc && v.mcmc) rc = launch_mcmc_adapt(v.mcmc, &r->accepted, v.M, &r->off, body_st);
  }
  if (!rc) {
    k_run_cond<<<1, 32, 0, body_st>>>(r, v.N, v.K, h);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) rc = ABC_E_CUDA;
  }
  l_body1 = launch_count();
  cudaGraph_t done_body = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(body_st, &done_body);
  if (rc) return rc;
  if (ec != cudaSuccess) return ABC_E_CUDA;
  // after the loop
  k_run_finish<<<1, 32, 0, st>>>(r, v.N);
  ABC_LAUNCH_CHECK();
  if (v.weight_mode == ABC_W_IMPORTANCE) {
    if ((rc = launch_survivors(v.u_cur, v.q, v.N, v.cu, v.cc, v.nc, v.scratch, st))) return rc;
    if (v.weight_prec == ABC_P_BF16_TC)
      rc = launch_weights_tc(v.u_nxt, v.s_nxt, v.N, v.cu, v.cc, v.nc, v.N, v.prefix + (v.N - 1),
                             v.logW, v.scratch, v.scratch_bytes, &br.tc_err, st, &r->off,
                             br.w_mult, nullptr, AncInfo{v.a_nxt, v.u_cur, v.q, v.N});
    else
      rc = launch_weights_fp32(v.u_nxt, v.s_nxt, v.N, v.cu, v.cc, v.nc, v.N, v.prefix + (v.N - 1),
                               v.logW, v.scratch, v.scratch_bytes, st, &r->off, br.w_mult);
    if (rc) return rc;
    // delayed acceptance: a particle simulated with probability rho carries 1 / rho
    if (sv.on && (rc = rho_correct(v.logW, sv.rho_pop, v.N, st, &r->off))) return rc;
    if ((rc = launch_normalize(v.logW, v.N, v.W_nxt, &r->ess, v.scratch, v.scratch_bytes, st)))
      return rc;
  } else {
    k_run_fill_paper<<<static_cast<unsigned>(ceil_div(v.N, 256)), 256, 0, st>>>(r, v.W_nxt, v.N);
    ABC_LAUNCH_CHECK();
  }
  if (sv.on && (rc = sur_train(sv, v.p, &r->off, st))) return rc;
  k_run_commit<<<static_cast<unsigned>(std::min<int64_t>(ceil_div(v.N, 256), 1024)), 256, 0, st>>>(
      r, v.N, v.u_cur, v.u_nxt, v.d_cur, v.d_nxt, v.W_cur, v.W_nxt, v.s_cur, v.s_nxt, v.a_cur,
      v.a_nxt);
  ABC_LAUNCH_CHECK();
  k_run_advance<<<1, 32, 0, st>>>(r);
  ABC_LAUNCH_CHECK();
  br.body_launches = l_body1 - l_body0;
  br.fixed_launches = launch_count() - l0 - br.body_launches;
  return ABC_OK;
}

}  // namespace abc
