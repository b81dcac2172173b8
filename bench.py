"""Benchmark: P-ABC-SMC with Beta-distributed step sizes on one GB300.

A step is one whole run of the single-run workload at scale (Sec. 2.4,
3.2): 2^20 particles, population 1e7, 120 days, G = 20 generations (stage 0
and 19 perturbed generations), importance weights with the O(N^2) kernel
sum, the paper's Beta(eps_t/eps_1, 2t) step schedule, on synthetic
observations simulated from a seeded theta*.  Every generation runs the whole
hot path: select eps_t, stage-prior prefix, batches of proposals (ancestor,
Beta step, walk, support check), simulation, acceptance, O(N^2) weights,
fp64 normalisation.  Step k is run k (Philox key (seed_lo, seed_hi ^ k)).

value: simulated particle-days per second over K runs with inputs resident
in HBM (CUDA events on the library's stream); ms_per_step is the wall-time
of one run.  e2e: the same metric through the public C ABI per run --
abc_init from the pinned host series, abc_run, the final population read
back to pinned host memory, abc_free.
cpu_baseline and --impl reference: the CPU oracle on the host cores, each
step one whole run of the same workload at a bounded sample size (8192
particles; same days, population, schedule, weights and generations),
measured, not extrapolated.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sim-days/s; wall-time to ε_final per run, surrogate+batched vs plain"
UNIT = "sim-days/s"
MUFU_EX2_PER_CLK_PER_SM = 16  # 32-bit exp2 issue rate of one SM (4 SMSPs x 4 lanes)
TC_K_USED = 60  # split-bf16 products per pair in the tensor-core weight GEMM (10 features x 6)
K_EFF = 10  # features of the weight pass's inner product (its algorithmic K)
# k_simulate per particle-day, from one ncu capture of every simulator launch of a whole
# 20-generation run of the 262,144-particle case of the workload (58 launches, 1.824e9
# particle-days): smsp__thread_inst_executed.sum / particle-days, and DRAM read + write bytes
SIM_THREAD_INST_PER_DAY = 941.7
SIM_DRAM_BYTES_PER_DAY = 0.3115


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def rank_config(w, rank, **over):
    """Each rank runs its own independent run (seed + rank): weak scaling,
    no data-path collective."""
    return w.config(seed=w.seed + rank, **over)


def job_totals(ms, sim_days, e2e_days, e2e_s, ws, device="cuda"):
    """Whole-job throughput over ws ranks: the units of all ranks over the
    slowest rank's time (max over ranks of the device time and of the host
    end-to-end time).  Returns (value, e2e_value, ms_max)."""
    if ws == 1:
        return sim_days / (ms / 1e3), e2e_days / e2e_s, ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms), float(e2e_s)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    tot = torch.tensor([float(sim_days), float(e2e_days)], device=device, dtype=torch.float64)
    dist.all_reduce(tot)
    return float(tot[0]) / (float(t[0]) / 1e3), float(tot[1]) / float(t[1]), float(t[0])


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu, self.proc, self.path = gpu, None, None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        busy = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def synthetic_obs(G, WL, cfg, torch):
    T = cfg.n_days
    obs = torch.empty((3, T + 1), dtype=torch.int32, device="cuda")
    th = torch.empty(8, dtype=torch.float32, device="cuda")
    att = torch.empty(1, dtype=torch.int32, device="cuda")
    G.abc_synth_obs(cfg, WL.OBS_BOX_LO, WL.OBS_BOX_HI, obs, th, att)
    torch.cuda.synchronize()
    return obs.cpu().numpy(), th.cpu().numpy()


def _nvtx(torch, name):
    """Push (name) or pop (None) an NVTX range; a no-op where torch lacks NVTX."""
    try:
        if name is None:
            torch.cuda.nvtx.range_pop()
        else:
            torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def bench_config(w, G_run, prec):
    """The config object of the single-run workload, shared by both arms."""
    return {"workload": w.name, "particles": w.N, "days": w.T, "population": w.P,
            "generations_per_run": G_run,
            "step": "one whole run (stage 0 + %d perturbed generations)" % (G_run - 1),
            "weights": "importance O(N^2), " + (
                "bf16 tcgen05 (rows with log W error bound <= 0.0166) + exact refinement"
                if prec else "fp32 (double-float near the row maximum)"),
            "beta_schedule": "paper (eps_t/eps_1, 2t)",
            "l2": "flushed between steps (256 MB write)"}


def run_gpu(args):
    import numpy as np
    import torch

    import paper_2106_15508_gb300 as G
    from paper_2106_15508_gb300 import build as B
    from paper_2106_15508_gb300 import workloads as WL

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0:
        B.build()
    if ws > 1:
        torch.distributed.barrier()
    G.lib()
    w = WL.LARGE
    if args.particles:  # a smaller case of the same workload (profiling)
        import dataclasses
        w = dataclasses.replace(w, N=args.particles, name="saird_n%d_t120_p1e7" % args.particles)
    G_run = args.generations or w.G
    # independent runs per rank (weak scaling, no data-path collective)
    cfg = rank_config(w, rank, weight_prec=args.prec)
    obs, theta_star = synthetic_obs(G, WL, cfg, torch)
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    ctx = G.abc_init(cfg, obs, stream=sp)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    N = w.N

    def one_run(run_id):
        G.abc_reset(ctx, run_id)
        rc = G.abc_run(ctx, G_run)
        if rc != G.ABC_OK or G.abc_generations(ctx) != G_run:
            raise RuntimeError("run %d stopped at generation %d: %s" % (
                run_id, G.abc_generations(ctx), G.strerror(rc)))
        return [G.abc_get_stats(ctx, t) for t in range(G_run)]

    try:
        for k in range(args.warmup):  # warm-up runs (their own run ids)
            one_run(1000 + k)
        flush.zero_()  # loads the flush kernel's module before the timed region
        torch.cuda.synchronize()
        clocks = Clocks(local)
        clocks.start()
        time.sleep(0.3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        runs = []
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            # NVTX range "timed" (host calls outside the events): lets a profiler
            # keep the timed runs only
            _nvtx(torch, "timed")
            e0.record(stream)
            for k in range(args.steps):
                if k:
                    flush.zero_()  # L2 (129 MB) flushed between steps
                runs.append(one_run(k))
            e1.record(stream)
            _nvtx(torch, None)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        clk = clocks.stop()
    finally:
        G.abc_free(ctx)
    stats = [s for r in runs for s in r]
    sim_days = sum(s.sim_days for s in stats)
    launches = sum(s.launches for s in stats)
    # end to end through the C ABI per run: the observed series from pinned
    # host memory (abc_init copies it to the device), the whole run, the
    # final population back to pinned host memory
    obs_h = torch.from_numpy(np.ascontiguousarray(obs)).pin_memory()
    pop_h = dict(u=torch.empty((8, N), dtype=torch.float32, pin_memory=True),
                 d=torch.empty(N, dtype=torch.float64, pin_memory=True),
                 W=torch.empty(N, dtype=torch.float64, pin_memory=True),
                 s=torch.empty(N, dtype=torch.float32, pin_memory=True),
                 anc=torch.empty(N, dtype=torch.int32, pin_memory=True))
    e2e_days = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        c_k = rank_config(w, rank, weight_prec=args.prec, run_id=k)
        h = G.abc_init_ptr(c_k, obs_h.data_ptr(), stream=sp)
        try:
            if G.abc_run(h, G_run) != G.ABC_OK:
                raise RuntimeError("e2e run %d stopped" % k)
            e2e_days += sum(G.abc_get_stats(h, t).sim_days for t in range(G_run))
            G.abc_get_population(h, pop_h["u"].data_ptr(), pop_h["d"].data_ptr(),
                                 pop_h["W"].data_ptr(), pop_h["s"].data_ptr(),
                                 pop_h["anc"].data_ptr(), on_device=False)
        finally:
            G.abc_free(h)
    e2e_s = time.perf_counter() - t0
    d2h = sum(t.numel() * t.element_size() for t in pop_h.values())
    h2d = obs_h.numel() * obs_h.element_size()
    rank_ms = ms
    value, e2e_value, ms = job_totals(ms, sim_days, e2e_days, e2e_s, ws)
    if rank != 0:
        return None
    K = args.steps
    peaks, src = _peaks()
    pairs = sum(s.pairs for s in stats)
    wms = sum(s.ms_weights for s in stats)
    sim_ms = sum(s.ms_sim for s in stats)
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    clk_mhz = float(clk.get("sm_mhz") or sm_mhz) if isinstance(clk, dict) else sm_mhz
    # the exp unit's rate, measured on this GPU by the library's probe
    exp_peak = G.abc_ex2_probe()
    exp_nominal = n_sm * MUFU_EX2_PER_CLK_PER_SM * sm_mhz * 1e6
    exp_src = ("measured ex2.approx.f32 rate (abc_ex2_probe: saturating microbenchmark on "
               "this GPU); %d SMs x %d ex2/clk x %.0f MHz would be %.0f Gexp/s" % (
                   n_sm, MUFU_EX2_PER_CLK_PER_SM, sm_mhz, exp_nominal / 1e9))
    tc_peak = float(peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])) * 1e12
    fb_name = "k_fb_rows" if args.prec else "k_weights_fp32"
    roofs = {}
    # simulator: lane-level issue slots (SMs x 4 warp instructions/clk x 32
    # lanes at the median SM clock sampled under load); the work unit is the
    # thread instructions per particle-day counted by ncu over whole runs
    lane_peak = n_sm * 4 * 32 * clk_mhz * 1e6
    sim_rate = SIM_THREAD_INST_PER_DAY * sim_days / (sim_ms / 1e3) if sim_ms > 0 else 0.0
    n_sim_launches = sum(s.batches for s in stats)
    roofs["k_simulate"] = {
        "bound": "alu", "kernel": "k_simulate", "achieved": sim_rate / 1e12,
        "peak": lane_peak / 1e12, "unit": "Tinst/s (thread-level)", "frac": sim_rate / lane_peak,
        "ms_per_step": sim_ms / K,
        "peak_source": "%d SMs x 4 warp-instructions/clk x 32 lanes x %.0f MHz (median SM "
                       "clock sampled under load)" % (n_sm, clk_mhz),
        "work": "%.1f thread instructions per particle-day (ncu over the simulator launches "
                "of whole runs)" % SIM_THREAD_INST_PER_DAY,
        "traffic": SIM_DRAM_BYTES_PER_DAY * sim_days / n_sim_launches if n_sim_launches else None,
        "traffic_note": "DRAM bytes per launch, per particle-day from the same capture"}
    # tensor-core weight kernel: the split-bf16 GEMM over the tiles it visits
    # (2 x 60 flops per pair: 10 features x 6 split products) and one
    # exponential per pair of the rows whose sums it keeps; its roofline is
    # the larger of the two lower bounds on its time.  The algorithmic count
    # of the survey (2 K_eff = 20 flops per pair of all N x N_surv pairs) is
    # given beside it.
    tc_ms = sum(s.ms_tc for s in stats)
    if tc_ms > 0:
        tc_flops = sum(2 * TC_K_USED * s.pairs_tc for s in stats)
        alg_flops = sum(2 * K_EFF * s.pairs for s in stats)
        tc_exps = sum(s.rows_exp * (s.pairs // N) for s in stats)
        t_tensor, t_exp = tc_flops / tc_peak, tc_exps / exp_peak
        common = {"kernel": "k_weights_tc", "ms_per_step": tc_ms / K,
                  "pairs_per_step": pairs / K,
                  "visited_pairs_per_step": sum(s.pairs_tc for s in stats) / K,
                  "kept_row_exps_per_step": tc_exps / K,
                  "algorithmic_tflops": alg_flops / (tc_ms / 1e3) / 1e12,
                  "algorithmic_tensor_frac": alg_flops / (tc_ms / 1e3) / tc_peak,
                  "traffic": None}
        if t_tensor >= t_exp:
            a = tc_flops / (tc_ms / 1e3)
            roofs["k_weights_tc"] = dict(common, bound="tensor", achieved=a / 1e12,
                                         peak=tc_peak / 1e12, unit="TFLOP/s", frac=a / tc_peak,
                                         peak_source="%s bf16 dense GEMM, sustained (cuBLAS)" % src,
                                         work="2 x 60 flops per pair of the visited tiles",
                                         exp_frac=tc_exps / (tc_ms / 1e3) / exp_peak)
        else:
            a = tc_exps / (tc_ms / 1e3)
            roofs["k_weights_tc"] = dict(common, bound="alu", achieved=a / 1e9,
                                         peak=exp_peak / 1e9, unit="Gexp/s", frac=a / exp_peak,
                                         peak_source=exp_src,
                                         work="one exp2 per pair of the kept rows",
                                         tensor_frac=tc_flops / (tc_ms / 1e3) / tc_peak)
    fb_ms = sum(s.ms_fp32 for s in stats)
    if fb_ms > 0:
        fb_pairs = sum((N - s.rows_tc) * (s.pairs // N) for s in stats)
        a = fb_pairs / (fb_ms / 1e3)
        roofs[fb_name] = {"bound": "alu", "kernel": fb_name, "achieved": a / 1e9,
                          "peak": exp_peak / 1e9, "unit": "Gexp/s", "frac": a / exp_peak,
                          "ms_per_step": fb_ms / K, "peak_source": exp_src,
                          "work": "one exp2 per pair", "traffic": None}
    # the roofline line is the dominant kernel's: the largest device time per step
    roofline = max(roofs.values(), key=lambda r: r["ms_per_step"])
    ess = [s.ess / N for s in stats if s.generation > 0]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(bench_config(w, G_run, args.prec),
                       theta_star=[round(float(x), 6) for x in theta_star]),
        "roofline": roofline,
        "rooflines": roofs,
        "wall_time_per_run_s": ms / K / 1e3,
        "pairs_per_step": pairs / K,
        "ess_over_n": {"median": float(np.median(ess)), "min": float(np.min(ess)),
                       "max": float(np.max(ess))},
        "weight_pass_gexp_s": pairs / (wms / 1e3) / 1e9 if wms > 0 else 0.0,
        "phases_ms_per_step": {"weights": wms / K, "simulator": sim_ms / K,
                               "rest": (rank_ms - wms - sim_ms) / K},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
        "generations_of_last_run": [
            {"t": s.generation, "eps": s.eps, "ess_over_n": s.ess / N, "batches": s.batches,
             "sim_days": s.sim_days, "pairs": s.pairs, "pairs_tc": s.pairs_tc, "ms": s.ms,
             "ms_sim": s.ms_sim, "ms_tc": s.ms_tc, "ms_fb": s.ms_fp32, "rows_exp": s.rows_exp}
            for s in runs[-1]],
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, G_run)
    return line


def run_batched(args):
    """64 independent runs (16K-256K particles, 60-180 days, P 1e6-1e8): one
    CUDA graph launch per generation of all runs, against the same runs as
    separate contexts driven one after another from the host ("plain")."""
    import torch

    import paper_2106_15508_gb300 as G
    from paper_2106_15508_gb300 import build as B
    from paper_2106_15508_gb300 import workloads as WL

    B.build()
    G.lib()
    runs = WL.batched_runs(args.runs, weight_prec=args.prec)
    cfgs = [w.config() for w in runs]
    obs = [synthetic_obs(G, WL, c, torch)[0] for c in cfgs]
    stream = torch.cuda.Stream()
    b = G.abc_batch_init(cfgs, obs, stream=stream.cuda_stream)
    tuning = None
    try:
        G.abc_batch_generation(b)
        if args.autotune:
            cache = os.path.join(ROOT, "_build", "autotune.json")
            os.makedirs(os.path.dirname(cache), exist_ok=True)
            t0 = time.perf_counter()
            G.abc_batch_autotune(b, cache)
            tuning = {"seconds": time.perf_counter() - t0,
                      "choices": sorted({G.abc_batch_tuning(b, r) for r in range(len(cfgs))})}
        for _ in range(args.warmup):
            G.abc_batch_generation(b)
        torch.cuda.synchronize()
        _nvtx(torch, "timed")
        t0 = time.perf_counter()
        first = G.abc_batch_generations(b)
        for _ in range(args.steps):
            G.abc_batch_generation(b)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        _nvtx(torch, None)
        days = launches = 0
        for r in range(len(cfgs)):
            for t in range(first, G.abc_batch_generations(b)):
                try:
                    st = G.abc_batch_get_stats(b, r, t)
                except G.AbcError:
                    continue
                days += st.sim_days
                launches += st.launches
    finally:
        G.abc_batch_free(b)
    # plain: every run in its own context, generations driven from the host
    ctxs = [G.abc_init(c, o, stream=stream.cuda_stream) for c, o in zip(cfgs, obs)]
    try:
        for ctx in ctxs:
            G.abc_run(ctx, 1 + args.warmup)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pdays = 0
        for ctx in ctxs:
            for _ in range(args.steps):
                if G.abc_generation(ctx) != G.ABC_OK:
                    break
                pdays += G.abc_get_stats(ctx, G.abc_generations(ctx) - 1).sim_days
        torch.cuda.synchronize()
        psecs = time.perf_counter() - t0
    finally:
        for ctx in ctxs:
            G.abc_free(ctx)
    value = days / secs
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "batched_%d_runs" % len(cfgs),
                       "particles_total": sum(w.N for w in runs),
                       "weights": "importance O(N^2), " + ("bf16 tcgen05" if args.prec else "fp32"),
                       "generations_timed": args.steps},
            "plain": {"value": pdays / psecs, "ms_per_step": psecs * 1e3 / args.steps,
                      "mode": "separate contexts, host-driven batch loops"},
            "wall_time_per_run_per_generation_ms": {"batched": secs * 1e3 / args.steps / len(cfgs),
                                                    "plain": psecs * 1e3 / args.steps / len(cfgs)},
            "speedup_vs_plain": (days / secs) / (pdays / psecs), "gpu_launches": launches,
            "autotune": tuning}


def run_sweep_bench(args):
    """Parallelism sweep (Sec. 4.1): levels x trials runs of 1000 samples,
    120 days, P = 1e7, each stopped on the stage that reached 1000 simulation
    runs; a step is one whole sweep.  Reports the simulated particle-days per
    second over the sweep and the per-level summary of the last sweep."""
    import torch

    import paper_2106_15508_gb300 as G
    from paper_2106_15508_gb300 import build as B
    from paper_2106_15508_gb300 import sweep as S
    from paper_2106_15508_gb300 import workloads as WL

    B.build()
    G.lib()
    levels = tuple(args.levels) if args.levels else S.LEVELS
    cfgs = [c for m in args.methods
            for c in S.sweep_configs(levels, args.trials, spec_target=args.spec_target, method=m,
                                     mcmc_s0=args.mcmc_s0)]
    obs = synthetic_obs(G, WL, cfgs[0], torch)[0]
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        S.run_sweep(cfgs, obs, stream=stream.cuda_stream, grouping=args.grouping)
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    t0 = time.perf_counter()
    days = launches = 0
    for _ in range(args.steps):
        flush.fill_(1)  # L2 flush between steps
        curves = S.run_sweep(cfgs, obs, stream=stream.cuda_stream, grouping=args.grouping)
        days += sum(c.sim_days for c in curves)
        launches += sum(c.launches for c in curves)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    clk = clocks.stop()
    summ = S.summarise_methods(curves)
    if args.grouping == "level":
        for meth, sm in summ.items():
            for M, v in sm.items():
                v["level_s"] = next(c.group_s for c in curves if c.M == M and c.method == meth)
    return {"metric": METRIC, "value": days / secs, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "sweep_%s_levels%s_trials%d_n1000_t120_p1e7_budget1000" % (
                           "-".join(args.methods), "-".join(str(m) for m in levels), args.trials),
                       "step": "one whole sweep (every trial to its stopping stage)",
                       "grouping": args.grouping,
                       "batches_per_round": "about %d simulations in flight, 1 to 64" % (
                           args.spec_target) if args.spec_target else "1",
                       "l2": "flushed between steps (256 MB write)"},
            "gpu_launches": launches, "clocks": clk,
            "sweep": {meth: {str(k): v for k, v in sm.items()} for meth, sm in summ.items()}}


ORACLE_SAMPLE_N = 8192  # particles of the oracle's sample runs


def oracle_sample_run(w, G_run, run_id, cores):
    """One whole run of the workload by the CPU oracle at ORACLE_SAMPLE_N
    particles (same days, population, observed series, paper schedule,
    importance weights and generations), on `cores` threads.  Returns
    (simulated particle-days, seconds)."""
    import oracle as O
    from paper_2106_15508_gb300 import workloads as WL

    A0 = WL.initial_active(w.P)
    m0 = O.OracleModel(T=w.T, P=w.P, A0=A0, seed=w.seed)
    obs, _, _ = O.synth_obs(m0)
    m = O.OracleModel(T=w.T, P=w.P, A0=A0, seed=w.seed, run=run_id)
    m.set_obs(obs)
    c = O.make_smc(ORACLE_SAMPLE_N, beta_mode=w.beta_mode, weight_mode=w.weight_mode,
                   alpha=w.alpha, max_batches=w.max_batches, nthreads=cores)
    t0 = time.perf_counter()
    _, stats = O.run(m, c, G_run)
    secs = time.perf_counter() - t0
    days = ORACLE_SAMPLE_N * w.T + sum((s.sims - s.exhausted) * w.T for s in stats)
    return days, secs


def cpu_baseline(w, G_run):
    """The oracle as it stands on the host cores: one sample run (the same
    function as the reference arm's steps)."""
    cores = os.cpu_count() or 1
    days, secs = oracle_sample_run(w, G_run, 0, cores)
    return {"value": days / secs, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "one whole %d-generation run at %d particles (%.3g sim-days in %.2f s); "
                      "the O(N^2) weight pass is a smaller share at this size than at %d "
                      "particles, so this rate is above the oracle's full-size rate" % (
                          G_run, ORACLE_SAMPLE_N, days, secs, w.N)}


def _f32_at_least(x):
    """The smallest float32 >= x (a tolerance target that x itself meets)."""
    import numpy as np
    f = np.float32(x)
    return float(f if float(f) >= x else np.nextafter(f, np.float32(np.inf)))


def run_eps_final(args):
    """Wall-time to eps_final per run, four forms of the same runs.
    (1) plain: each run alone in its own context, one after another, G
    generations; eps_final of a run is its tolerance at generation G.
    (2) batched: all runs in one graph launch per generation (bit-identical
    results, so the same G generations).  (3) surrogate + batched: every run
    screened by its own surrogate, all runs in one graph, each run stopping
    at its eps_final (abc_config.eps_stop), at most 3 G generations.  (4)
    surrogate alone: the screened runs in their own contexts one after
    another.  Reported: mean wall-time per run of each form (host clock
    around device-synchronised calls; a batch's time is shared by its runs),
    simulations per run, false-rejection rate, runs that reached eps_final."""
    import numpy as np
    import torch

    import paper_2106_15508_gb300 as G
    from paper_2106_15508_gb300 import build as B
    from paper_2106_15508_gb300 import workloads as WL

    B.build()
    G.lib()
    runs = (WL.stress_runs(args.runs, weight_prec=args.prec) if args.stress
            else WL.batched_runs(args.runs, weight_prec=args.prec))
    cfgs = [w.config() for w in runs]
    obs = [synthetic_obs(G, WL, c, torch)[0] for c in cfgs]
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    gens = args.generations or 8
    R = len(cfgs)

    def stats_of(get, n):
        return [get(t) for t in range(n)]

    def ctx_stats(ctx):
        # recorded generations of a context: the completed ones, and a last
        # one that stopped on its batch budget (recorded, not counted)
        n = G.abc_generations(ctx)
        try:
            G.abc_get_stats(ctx, n)
            return n + 1
        except G.AbcError:
            return n

    # (1) plain
    eps_final, t_plain, sims_plain, gens_plain = [], [], [], []
    for c, o in zip(cfgs, obs):
        ctx = G.abc_init(c, o, stream=sp)
        try:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            G.abc_run(ctx, gens + 1)
            torch.cuda.synchronize()
            t_plain.append(time.perf_counter() - t0)
            st = stats_of(lambda t: G.abc_get_stats(ctx, t), ctx_stats(ctx))
            eps_final.append(st[-1].eps)
            sims_plain.append(sum(x.sims for x in st))
            gens_plain.append(len(st) - 1)
        finally:
            G.abc_free(ctx)
    def batch_gens(b, r):
        # generations run r of batch b completed (a run can stop before the
        # others: its stage budget exhausted, or its stop rule met)
        n = 0
        while True:
            try:
                G.abc_batch_get_stats(b, r, n)
                n += 1
            except G.AbcError:
                return n

    # (2) batched
    b = G.abc_batch_init(cfgs, obs, stream=sp)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G.abc_batch_run(b, gens + 1)
        torch.cuda.synchronize()
        t_batch = time.perf_counter() - t0
        eps_b = [G.abc_batch_get_stats(b, r, batch_gens(b, r) - 1).eps for r in range(R)]
    finally:
        G.abc_batch_free(b)

    def sur_cfg(c, ef):
        sc = G.config(**{f: getattr(c, f) if not hasattr(getattr(c, f), "_length_")
                         else list(getattr(c, f)) for f, _ in c._fields_})
        sc.surrogate, sc.surrogate_start, sc.surrogate_steps = 1, 2, args.surrogate_steps
        sc.surrogate_batch, sc.surrogate_tau = args.surrogate_batch, args.surrogate_tau
        sc.surrogate_lr = 1e-3
        sc.surrogate_rho_min, sc.audit_frac = args.surrogate_rho_min, 0.01
        sc.eps_stop = _f32_at_least(ef)
        # screened-out proposals use up batches: a larger per-stage budget
        sc.max_batches = max(c.max_batches, 512)
        if args.surrogate_ring_mult > 0:
            sc.surrogate_ring = args.surrogate_ring_mult * c.n_particles
        return sc

    scfgs = [sur_cfg(c, ef) for c, ef in zip(cfgs, eps_final)]

    def sur_summary(get_stats, ngen):
        st = stats_of(get_stats, ngen)
        aud = sum(x.audited for x in st)
        return dict(eps=st[-1].eps, gens=ngen - 1, sims=sum(x.sims for x in st),
                    screened=sum(x.screened for x in st), audited=aud,
                    audit_accepted=sum(x.audit_accepted for x in st),
                    ms_train=sum(x.ms_train for x in st), ms_screen=sum(x.ms_screen for x in st))

    # (3) surrogate + batched
    b = G.abc_batch_init(scfgs, obs, stream=sp)
    sb = []
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G.abc_batch_run(b, 3 * gens + 1)
        torch.cuda.synchronize()
        t_sur_batch = time.perf_counter() - t0
        for r in range(R):
            sb.append(sur_summary(lambda t, r=r: G.abc_batch_get_stats(b, r, t), batch_gens(b, r)))
    finally:
        G.abc_batch_free(b)
    # (4) surrogate alone
    t_sur, ss = [], []
    for sc, o in zip([] if args.no_surrogate else scfgs, obs):
        ctx = G.abc_init(sc, o, stream=sp)
        try:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            G.abc_run(ctx, 3 * gens + 1)
            torch.cuda.synchronize()
            t_sur.append(time.perf_counter() - t0)
            ss.append(sur_summary(lambda t: G.abc_get_stats(ctx, t), ctx_stats(ctx)))
        finally:
            G.abc_free(ctx)
    per = lambda xs: float(np.mean(xs)) if len(xs) else None
    reached = lambda xs: int(sum(x["eps"] <= sc.eps_stop for x, sc in zip(xs, scfgs)))
    frr = lambda xs: (sum(x["audit_accepted"] for x in xs) / max(1, sum(x["audited"] for x in xs))
                      if xs else None)
    return {"metric": "wall-time to eps_final per run", "unit": "s", "higher_is_better": False,
            "n_gpus": 1, "data": "synthetic",
            "config": {"workload": ("stress_" if args.stress else "") + "eps_final_%d_runs" % R,
                       "generations": gens,
                       "weights": "importance O(N^2), " + ("bf16 tcgen05" if args.prec else "fp32"),
                       "particles": [w.N for w in runs], "days": [w.T for w in runs],
                       "populations": [w.P for w in runs]},
            "plain_s_per_run": per(t_plain),
            "batched_s_per_run": t_batch / R,
            "batched_same_eps": bool(np.all(np.array(eps_b) == np.array(eps_final))),
            "plain_generations": gens_plain,
            "surrogate_batched_s_per_run": t_sur_batch / R,
            "surrogate_batched_reached": reached(sb),
            "surrogate_batched_generations": per([x["gens"] for x in sb]),
            "surrogate_s_per_run": per(t_sur),
            "surrogate_reached": reached(ss) if ss else None,
            "surrogate_generations": per([x["gens"] for x in ss]),
            "sims_per_run": {"plain": per(sims_plain),
                             "surrogate_batched": per([x["sims"] for x in sb]),
                             "surrogate": per([x["sims"] for x in ss])},
            "screened_per_run": {"surrogate_batched": per([x["screened"] for x in sb])},
            "false_rejection_rate": {"surrogate_batched": frr(sb), "surrogate": frr(ss)},
            "train_ms_per_run": {"surrogate": per([x["ms_train"] for x in ss])},
            "screen_ms_per_run": {"surrogate": per([x["ms_screen"] for x in ss])},
            "surrogate_settings": {"start": 2, "steps": args.surrogate_steps,
                                   "ring_mult": args.surrogate_ring_mult,
                                   "batch": args.surrogate_batch, "tau": args.surrogate_tau,
                                   "rho_min": args.surrogate_rho_min, "audit": 0.01, "lr": 1e-3}}


def run_passes(args):
    """The HBM-bound passes at N = 2^28 (inputs 4x+ the 129 MB L2): tolerance
    select (A4), stage-prior weights and prefix (A5, importance mode) and the
    fp64 normalisation (A10), each timed alone with CUDA events (best of 5
    after 2 warm-ups).  Bytes per element are those the kernels move:
    select 8 passes x 8 B; prefix 16 B (max) + 20 B (quantise) + 12 B
    (scan); normalise 3 x 8 B read + 8 B written."""
    import torch

    import paper_2106_15508_gb300 as G
    from paper_2106_15508_gb300 import build as B

    B.build()
    G.lib()
    n = args.pass_n
    dev = "cuda"
    gen = torch.Generator(device=dev).manual_seed(1)
    d = torch.rand(n, dtype=torch.float64, device=dev, generator=gen) * 1e6
    W = torch.rand(n, dtype=torch.float64, device=dev, generator=gen) + 0.1
    lw = torch.randn(n, dtype=torch.float64, device=dev, generator=gen)
    q = torch.empty(n, dtype=torch.int32, device=dev)
    pre = torch.empty(n, dtype=torch.int64, device=dev)
    Wn = torch.empty(n, dtype=torch.float64, device=dev)
    out = torch.empty(4, dtype=torch.float64, device=dev)
    eps = torch.tensor([5e5], dtype=torch.float64, device=dev)
    sc = torch.empty(max(G.abc_select_scratch_bytes(n), G.abc_prefix_scratch_bytes(n),
                         G.abc_normalize_scratch_bytes(n)), dtype=torch.uint8, device=dev)
    peaks, src = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    passes = {
        "select_kth": (64, lambda: G.abc_select_kth(d, n, n // 2, out, sc, sc.numel())),
        "resample_prefix": (48, lambda: G.abc_resample_prefix(d, W, n, eps, G.ABC_W_IMPORTANCE,
                                                              q, pre, sc, sc.numel())),
        "normalize": (32, lambda: G.abc_normalize(lw, n, Wn, out[1:], sc, sc.numel())),
    }
    res = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, (bpe, fn) in passes.items():
        best = 1e30
        for rep in range(7):
            torch.cuda.synchronize()
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            if rep >= 2:
                best = min(best, e0.elapsed_time(e1))
        gbs = bpe * n / (best / 1e3) / 1e9
        res[name] = {"ms": best, "bytes_per_element": bpe, "GB/s": gbs, "frac_of_hbm": gbs / hbm}
    return {"metric": "HBM pass bandwidth", "unit": "GB/s", "n_gpus": 1, "data": "synthetic",
            "config": {"workload": "passes_n%d" % n, "peak": hbm, "peak_source": src},
            "passes": res}


def run_reference(args):
    """The oracle arm: each step is one whole run of the same workload by the
    CPU oracle at a bounded sample size (oracle_sample_run), measured."""
    from paper_2106_15508_gb300 import workloads as WL

    ws, rank = _dist()
    if rank != 0:
        return None
    w = WL.LARGE
    G_run = args.generations or w.G
    cores = os.cpu_count() or 1
    for k in range(args.warmup):
        oracle_sample_run(w, G_run, 1000 + k, cores)
    days = secs = 0.0
    for k in range(args.steps):
        d, t = oracle_sample_run(w, G_run, k, cores)
        days += d
        secs += t
    value = days / secs
    sample = ("each step one whole %d-generation run at %d particles (of %d), measured; the "
              "O(N^2) weight pass is a smaller share at this size, so this rate is above the "
              "oracle's full-size rate" % (G_run, ORACLE_SAMPLE_N, w.N))
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": bench_config(w, G_run, args.prec),
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": cores,
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--prec", type=int, default=1,
                    help="1: tcgen05 (bf16 x3 split, fp32 accumulation; rows with a large "
                         "error bound recomputed exactly); 0: FP32 CUDA cores only")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="single",
                    choices=["single", "batched", "eps_final", "passes", "sweep"])
    ap.add_argument("--levels", type=int, nargs="*", default=None,
                    help="sweep: simulations per batch (default 10 100 1000 10000 100000)")
    ap.add_argument("--trials", type=int, default=10, help="sweep: trials per level")
    ap.add_argument("--spec-target", type=int, default=65536,
                    help="sweep: simulations in flight per round of small levels (0: one batch)")
    ap.add_argument("--grouping", default="all", choices=["all", "level", "run"],
                    help="sweep: one batch of all runs, one per level, or one per run")
    ap.add_argument("--methods", nargs="+", default=["bdss"], choices=["bdss", "mcmc"],
                    help="sweep: BDSS and/or the MCMC-tuned single-step baseline")
    ap.add_argument("--mcmc-s0", type=float, default=0.1,
                    help="sweep: the MCMC baseline's initial step (unit-cube variance)")
    ap.add_argument("--pass-n", type=int, default=1 << 28)
    ap.add_argument("--generations", type=int, default=0,
                    help="generations per run (single: 20, the workload's G; eps_final: 8)")
    ap.add_argument("--surrogate-steps", type=int, default=32)
    ap.add_argument("--surrogate-tau", type=float, default=0.25)
    ap.add_argument("--surrogate-batch", type=int, default=4096)
    ap.add_argument("--surrogate-rho-min", type=float, default=0.05)
    ap.add_argument("--surrogate-ring-mult", type=int, default=2,
                    help="training ring of this many times N samples (0: the library default)")
    ap.add_argument("--stress", action="store_true",
                    help="eps_final on the stress runs (2^20 particles, 365 days, P 3.3e8)")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--particles", type=int, default=0,
                    help="override the particle count (smaller cases for profiling)")
    ap.add_argument("--runs", type=int, default=64)
    ap.add_argument("--autotune", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.workload in ("batched", "sweep"):
        # a batch's graph runs one branch per run: give the process more
        # hardware work queues than the default 8, before CUDA starts
        os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    if args.impl == "reference":
        line = run_reference(args)
    elif args.workload == "batched":
        line = run_batched(args)
    elif args.workload == "eps_final":
        line = run_eps_final(args)
    elif args.workload == "passes":
        line = run_passes(args)
    elif args.workload == "sweep":
        line = run_sweep_bench(args)
    else:
        line = run_gpu(args)
    if line is not None:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
