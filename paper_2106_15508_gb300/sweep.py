"""Parallelism sweep (Sec. 4.1, experiment setup and Fig. 3).

The paper runs P-ABC-SMC BDSS and its baseline P-ABC-SMC MCMC (one
MH-tuned step, Sec. 2.4.1 and 3.1) at five degrees of parallelism (10, 100,
1k, 10k and 100k simulations per simulation run, i.e. per batch of M
parallel simulations), ten independent trials each, collecting 1000
samples.  Each
trial stops on the stage that reached 1000 simulation runs and lets that
stage finish.  Per stage it records the tolerance reached, and it judges the
levels by the best tolerance, the simulation runs needed to reach it and the
spread of both over the trials (Sec. 4, evaluation metrics).

Here every trial is one run of a graph-captured batch (abc_batch_*), with
the run budget in abc_config.max_total_batches; the runs of a batch advance
together, one graph launch per stage, their branches overlapping on the GPU.
By default the whole sweep is one batch: the low levels' runs are chains of
small, latency-bound batches that then overlap the high levels' large ones.
Synthetic observations stand in for the Italy series.

This module holds host logic only (configs, the driver loop, the summary);
every step of every run executes in the library's kernels.
"""
import dataclasses
import math

import numpy as np

from . import (ABC_OK, ABC_STEP_MCMC, ABC_STOP_BUDGET, ABC_W_PAPER, AbcError, abc_batch_free,
               abc_batch_get_stats, abc_batch_init, abc_batch_run)
from . import workloads as WL

LEVELS = (10, 100, 1000, 10000, 100000)
METHODS = ("bdss", "mcmc")


@dataclasses.dataclass
class Curve:
    """One trial: after each stage t >= 1, the simulation runs so far (stage 0
    counting ceil(N / M)) and the tolerance eps_t its acceptance used."""
    M: int
    trial: int
    runs: np.ndarray
    eps: np.ndarray
    sim_days: int      # simulated particle-days, stage 0 included
    launches: int      # kernels launched for the run
    status: int        # of the last stage: ABC_OK, or ABC_STOP_BUDGET
    group_s: float = 0.0  # wall time of the batch the run was part of
    method: str = "bdss"  # "bdss" (Beta step sizes) or "mcmc" (one tuned step)


def spec_for(M, target=65536, cap=64):
    """Batches per device loop round for M simulations per batch: enough to
    put about `target` simulations in flight (a batch of M <= 10^4 is a
    chain of dependent trajectories, latency-bound), at most `cap`."""
    return max(1, min(cap, -(-target // M)))


def sweep_configs(levels=LEVELS, trials=10, N=1000, budget=1000, T=120, P=10_000_000, seed=1,
                  max_batches=65535, spec_target=65536, method="bdss", mcmc_s0=0.1):
    """One config per (level, trial): N samples, M = level, the run budget,
    the paper's weights (Eq. 10) and, for method "bdss", its Beta schedule
    (Eq. 16); for "mcmc" the baseline's single step, started at mcmc_s0 and
    adapted during the first tenth of the run budget (Sec. 2.4.1, 3.1).
    Run ids 0, 1, ... give every trial of a method its own Philox key.
    Small BDSS levels run several batches per round (spec_for; results
    unchanged); spec_target 0 runs one.  The baseline runs one batch per
    round (its step changes between batches)."""
    if method not in METHODS:
        raise ValueError("method must be one of %s" % (METHODS,))
    w = WL.Workload("sweep", N=N, T=T, P=P, G=0, weight_mode=ABC_W_PAPER,
                    max_batches=max_batches, seed=seed)
    extra = dict(beta_mode=ABC_STEP_MCMC, mcmc_s0=mcmc_s0, mcmc_adapt=0) \
        if method == "mcmc" else {}
    return [w.config(batch_size=M, max_total_batches=budget, run_id=li * trials + k,
                     spec_batches=spec_for(M, spec_target) if spec_target and method == "bdss"
                     else 1, **extra)
            for li, M in enumerate(levels) for k in range(trials)]


def method_of(cfg):
    return "mcmc" if cfg.beta_mode == ABC_STEP_MCMC else "bdss"


def _curve(b, r, cfg, trial):
    st0 = abc_batch_get_stats(b, r, 0)
    runs = -(-cfg.n_particles // cfg.batch_size)
    days, launches = st0.sim_days, st0.launches
    rr, ee, status = [], [], ABC_OK
    t = 1
    while True:
        try:
            st = abc_batch_get_stats(b, r, t)
        except AbcError:
            break
        runs += st.batches
        days += st.sim_days
        launches += st.launches
        status = st.status
        if st.status == ABC_OK:
            rr.append(runs)
            ee.append(st.eps)
        t += 1
    return Curve(cfg.batch_size, trial, np.array(rr, np.int64), np.array(ee, np.float64), days,
                 launches, status, method=method_of(cfg))


def run_sweep(cfgs, obs, stream=None, max_stages=32767, grouping="all"):
    """Runs every config on the observed series obs (host int32 [3][T+1])
    until each run has stopped; returns the curves in config order (a
    trial's index counts the earlier configs of its level).  grouping:
    "all", one batch of every run; "level", one batch per level, one after
    another; "run", one batch per run, each driven by a host thread of its
    own, so that no run waits at a stage boundary for the slowest run of its
    batch."""
    import time

    groups = {}
    for i, c in enumerate(cfgs):
        key = 0 if grouping == "all" else c.batch_size if grouping == "level" else i
        groups.setdefault(key, []).append(i)
    curves = [None] * len(cfgs)

    def one(idx):
        sub = [cfgs[i] for i in idx]
        t0 = time.perf_counter()
        b = abc_batch_init(sub, [obs] * len(sub), stream=stream)
        try:
            abc_batch_run(b, max_stages + 1)
            secs = time.perf_counter() - t0
            for k, i in enumerate(idx):
                trial = sum(c.batch_size == cfgs[i].batch_size and
                            method_of(c) == method_of(cfgs[i]) for c in cfgs[:i])
                curves[i] = _curve(b, k, cfgs[i], trial)
                curves[i].group_s = secs
        finally:
            abc_batch_free(b)

    if grouping == "run":
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(max_workers=len(groups)) as ex:
            for f in [ex.submit(one, idx) for idx in groups.values()]:
                f.result()
    else:
        for idx in groups.values():
            one(idx)
    return curves


def summarise_methods(curves):
    """summarise() for the curves of each method: {method: {M: ...}}."""
    return {m: summarise([c for c in curves if c.method == m])
            for m in METHODS if any(c.method == m for c in curves)}


def summarise(curves):
    """Per level (ascending M) of the curves of one method: the best tolerance of each trial (its
    smallest eps_t), the simulation runs at the first stage that reached it,
    the runs in all, the runs at the first stage within a factor 2 of the
    trial's best, with medians, quartiles and the spread of log10 of the
    best tolerance over the trials; trials that ended on a stage which used
    up its per-stage batch budget are counted as stuck."""
    out = {}
    for M in sorted({c.M for c in curves}):
        cs = [c for c in curves if c.M == M]
        done = [c for c in cs if len(c.eps)]
        best = np.array([c.eps.min() for c in done], np.float64)
        to_best = np.array([c.runs[int(np.argmax(c.eps == c.eps.min()))] for c in done],
                           np.float64)
        total = np.array([c.runs[-1] if len(c.runs) else 0 for c in cs], np.float64)
        to_2x = np.array([c.runs[int(np.argmax(c.eps <= 2.0 * c.eps.min()))] for c in done],
                         np.float64)

        def q(a, p):
            return float(np.percentile(a, p)) if len(a) else math.nan

        lb = np.log10(np.maximum(best, 1.0))
        out[M] = {"trials": len(cs), "with_stages": len(done),
                  "stuck": sum(c.status == ABC_STOP_BUDGET for c in cs),
                  "best_eps_median": q(best, 50), "best_eps_q25": q(best, 25),
                  "best_eps_q75": q(best, 75),
                  "log10_best_eps_std": float(lb.std()) if len(lb) else math.nan,
                  "runs_to_best_median": q(to_best, 50), "runs_to_best_q25": q(to_best, 25),
                  "runs_to_best_q75": q(to_best, 75), "runs_to_2x_best_median": q(to_2x, 50),
                  "runs_total_median": q(total, 50),
                  "stages_median": q(np.array([len(c.eps) for c in cs], np.float64), 50),
                  "sim_days": int(sum(c.sim_days for c in cs))}
    return out


def main(argv=None):
    """python -m paper_2106_15508_gb300.sweep [--levels ...] [--trials K]
    [--out file.json]: runs the sweep on cuda:0 and writes the curves and
    the summary as JSON."""
    import argparse
    import json
    import time

    import torch

    from . import abc_synth_obs
    from .build import build

    ap = argparse.ArgumentParser()
    ap.add_argument("--levels", type=int, nargs="+", default=list(LEVELS))
    ap.add_argument("--trials", type=int, default=10)
    ap.add_argument("--samples", type=int, default=1000)
    ap.add_argument("--budget", type=int, default=1000)
    ap.add_argument("--days", type=int, default=120)
    ap.add_argument("--population", type=int, default=10_000_000)
    ap.add_argument("--methods", nargs="+", default=["bdss"], choices=METHODS)
    ap.add_argument("--mcmc-s0", type=float, default=0.1)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    # one graph branch per run: more hardware work queues than the default 8
    # (read when CUDA starts, so set before the first CUDA call)
    import os
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    build()
    cfgs = [c for m in a.methods
            for c in sweep_configs(a.levels, a.trials, a.samples, a.budget, a.days, a.population,
                                   method=m, mcmc_s0=a.mcmc_s0)]
    obs = torch.empty((3, a.days + 1), dtype=torch.int32, device="cuda")
    th = torch.empty(8, dtype=torch.float32, device="cuda")
    att = torch.empty(1, dtype=torch.int32, device="cuda")
    abc_synth_obs(cfgs[0], WL.OBS_BOX_LO, WL.OBS_BOX_HI, obs, th, att)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    curves = run_sweep(cfgs, obs.cpu().numpy())
    secs = time.perf_counter() - t0
    res = {"seconds": secs,
           "summary": {m: {str(k): v for k, v in sm.items()}
                       for m, sm in summarise_methods(curves).items()},
           "curves": [{"method": c.method, "M": c.M, "trial": c.trial, "runs": c.runs.tolist(),
                       "eps": c.eps.tolist(), "status": c.status} for c in curves]}
    text = json.dumps(res)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text)
    else:
        print(json.dumps(res["summary"], indent=1))
    return res


if __name__ == "__main__":
    main()
