"""Batched runs (abc_batch_*): many independent runs, one CUDA graph launch
per generation with device-side batch loops.

* Paper weights: every run of a heterogeneous batch (different particle
  counts, horizons, populations, seeds and Beta settings) reproduces the
  oracle's populations and statistics bit for bit, generation by generation.
* Importance weights: each run equals a separate single-run context bit for
  bit (same kernels, same counters).
* A run that exhausts its batch budget stops alone; autotuning changes launch
  shapes only, never results, and writes its cache.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
import paper_2106_15508_gb300 as G
from paper_2106_15508_gb300 import build as B

from helpers import get_population, oracle_model, oracle_obs, oracle_smc, saird_config

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    G.lib()


def _cfgs(weight_mode, weight_prec=G.ABC_P_FP32):
    specs = [(2048, 40, 100_000, 1, G.ABC_BETA_FIXED), (4096, 25, 1_000_000, 2, G.ABC_BETA_PAPER),
             (1024, 60, 50_000, 3, G.ABC_BETA_PAPER), (3000, 33, 2_000_000, 4, G.ABC_BETA_FIXED)]
    return [saird_config(N, T, P, seed=seed, beta_mode=bm, beta_a=2.0, beta_b=5,
                         weight_mode=weight_mode, weight_prec=weight_prec)
            for N, T, P, seed, bm in specs]


def _batch_pop(b, r, N):
    u = np.zeros((8, N), np.float32)
    d = np.zeros(N)
    W = np.zeros(N)
    s = np.zeros(N, np.float32)
    a = np.zeros(N, np.int32)
    G.abc_batch_get_population(b, r, u, d, W, s, a)
    return dict(u=u, d=d, W=W, s=s, anc=a)


def test_batch_paper_weights_match_oracle():
    cfgs = _cfgs(G.ABC_W_PAPER)
    obs = [oracle_obs(c)[0] for c in cfgs]
    b = G.abc_batch_init(cfgs, obs)
    try:
        models = [oracle_model(c, o) for c, o in zip(cfgs, obs)]
        smcs = [oracle_smc(c) for c in cfgs]
        pops = [O.generation0(m, c) for m, c in zip(models, smcs)]
        eps1 = [0.0] * len(cfgs)
        G.abc_batch_generation(b)
        for t in range(1, 5):
            G.abc_batch_generation(b)
            for r, cfg in enumerate(cfgs):
                new, st = O.generation(models[r], smcs[r], t, eps1[r], pops[r])
                assert st.status == 0
                gp = _batch_pop(b, r, cfg.n_particles)
                for k, ok in (("u", new.u), ("d", new.d), ("s", new.s), ("anc", new.anc)):
                    assert np.array_equal(gp[k].view(np.uint8),
                                          np.ascontiguousarray(ok).view(np.uint8)), (t, r, k)
                g = G.abc_batch_get_stats(b, r, t)
                assert g.eps == st.eps and g.batches == st.batches
                assert g.accepted == st.accepted_total and g.beta_b == st.beta_b
                eps1[r], pops[r] = st.eps1, new
    finally:
        G.abc_batch_free(b)


@pytest.mark.parametrize("prec", [G.ABC_P_FP32, G.ABC_P_BF16_TC])
def test_batch_importance_weights_equal_single_contexts(prec):
    cfgs = _cfgs(G.ABC_W_IMPORTANCE, prec)
    obs = [oracle_obs(c)[0] for c in cfgs]
    b = G.abc_batch_init(cfgs, obs)
    singles = [G.abc_init(c, o) for c, o in zip(cfgs, obs)]
    try:
        G.abc_batch_run(b, 5)
        for ctx in singles:
            G.abc_run(ctx, 5)
        for r, cfg in enumerate(cfgs):
            gb = _batch_pop(b, r, cfg.n_particles)
            gs = get_population(singles[r], cfg.n_particles)
            for k in gb:
                assert np.array_equal(gb[k].view(np.uint8), gs[k].view(np.uint8)), (r, k)
            for t in range(1, 5):
                x, y = G.abc_batch_get_stats(b, r, t), G.abc_get_stats(singles[r], t)
                assert x.eps == y.eps and x.ess == y.ess and x.batches == y.batches
    finally:
        G.abc_batch_free(b)
        for ctx in singles:
            G.abc_free(ctx)


def test_batch_budget_stop_is_per_run():
    cfgs = _cfgs(G.ABC_W_PAPER)
    cfgs[1].batch_size = 512      # M < N: one batch can never fill N = 4096
    cfgs[1].max_batches = 1
    obs = [oracle_obs(c)[0] for c in cfgs]
    b = G.abc_batch_init(cfgs, obs)
    ctx = G.abc_init(cfgs[1], obs[1])
    try:
        G.abc_batch_run(b, 4)
        assert G.abc_batch_get_stats(b, 1, 1).status == G.ABC_STOP_BUDGET
        with pytest.raises(G.AbcError):
            G.abc_batch_get_stats(b, 1, 2)    # the stopped run records nothing more
        for r in (0, 2, 3):
            assert G.abc_batch_get_stats(b, r, 3).status == 0
        # the run alone in a context: the same stopped generation, recorded
        # after the completed ones (and not counted by abc_generations)
        assert G.abc_run(ctx, 4) == G.ABC_STOP_BUDGET
        assert G.abc_generations(ctx) == 1
        x, y = G.abc_get_stats(ctx, 1), G.abc_batch_get_stats(b, 1, 1)
        assert (x.status, x.eps, x.batches, x.sims) == (y.status, y.eps, y.batches, y.sims)
        with pytest.raises(G.AbcError):
            G.abc_get_stats(ctx, 2)
    finally:
        G.abc_batch_free(b)
        G.abc_free(ctx)


def test_autotune_keeps_results_and_writes_cache(tmp_path):
    cfgs = _cfgs(G.ABC_W_IMPORTANCE)
    obs = [oracle_obs(c)[0] for c in cfgs]
    a = G.abc_batch_init(cfgs, obs)
    b = G.abc_batch_init(cfgs, obs)
    cache = str(tmp_path / "tune.json")
    try:
        G.abc_batch_generation(a)
        G.abc_batch_generation(b)
        G.abc_batch_autotune(b, cache)
        for r in range(len(cfgs)):
            th, wm = G.abc_batch_tuning(b, r)
            assert th in (64, 128, 256) and wm in (1, 2, 4)
        tuned = json.load(open(cache))
        assert len(tuned) >= 1
        G.abc_batch_run(a, 4)
        G.abc_batch_run(b, 4)
        for r, cfg in enumerate(cfgs):
            pa, pb = _batch_pop(a, r, cfg.n_particles), _batch_pop(b, r, cfg.n_particles)
            for k in pa:
                assert np.array_equal(pa[k].view(np.uint8), pb[k].view(np.uint8)), (r, k)
    finally:
        G.abc_batch_free(a)
        G.abc_batch_free(b)


def _sur_batch_cfgs():
    """Runs with the surrogate pre-screen (delayed acceptance) beside one
    without: a SAIRD run with importance weights, a SAIRD run with the paper's
    weights, the Gaussian toy with importance weights, and a plain run."""
    sur = dict(surrogate=1, surrogate_start=2, surrogate_steps=16, surrogate_batch=1024,
               surrogate_lr=1e-3, surrogate_tau=0.3, surrogate_rho_min=0.05, audit_frac=0.05)
    return [
        saird_config(2048, 40, 100_000, seed=21, weight_mode=G.ABC_W_IMPORTANCE,
                     weight_prec=G.ABC_P_BF16_TC, **sur),
        saird_config(3000, 30, 1_000_000, seed=22, weight_mode=G.ABC_W_PAPER,
                     beta_mode=G.ABC_BETA_FIXED, beta_a=2.0, beta_b=5, **sur),
        G.config(model=G.ABC_MODEL_GAUSS_TOY, n_days=1, population=1, init_ard=[0, 0, 0],
                 theta_lo=[-10.0] * 8, theta_hi=[10.0] * 8, seed=23, n_particles=2048,
                 beta_mode=G.ABC_BETA_FIXED, beta_a=8.0, beta_b=1000,
                 weight_mode=G.ABC_W_IMPORTANCE, max_batches=400, **sur),
        saird_config(1024, 50, 100_000, seed=24, weight_mode=G.ABC_W_IMPORTANCE),
    ]


def test_batch_with_surrogate_equals_single_contexts():
    """The surrogate inside the graph branches (inference, screen, compacted
    simulation, audits, training ring, 1/rho correction and Adam training
    after each generation, all with device-side counts): every run equals its
    own single-run context bit for bit -- populations, tolerances, batches,
    simulations, screened / audited counts -- through generations that screen."""
    cfgs = _sur_batch_cfgs()
    obs = [None if c.model == G.ABC_MODEL_GAUSS_TOY else oracle_obs(c)[0] for c in cfgs]
    gens = 6
    b = G.abc_batch_init(cfgs, obs)
    ctxs = [G.abc_init(c, o) for c, o in zip(cfgs, obs)]
    try:
        G.abc_batch_run(b, gens)
        for ctx in ctxs:
            G.abc_run(ctx, gens)
        screened_any = 0
        for r, (cfg, ctx) in enumerate(zip(cfgs, ctxs)):
            N = cfg.n_particles
            gp, sp = _batch_pop(b, r, N), get_population(ctx, N)
            for k in gp:
                assert np.array_equal(gp[k].view(np.uint8), sp[k].view(np.uint8)), (r, k)
            for t in range(gens):
                g, s = G.abc_batch_get_stats(b, r, t), G.abc_get_stats(ctx, t)
                assert (g.eps, g.batches, g.sims, g.exhausted, g.accepted) == \
                       (s.eps, s.batches, s.sims, s.exhausted, s.accepted), (r, t)
                assert (g.screened, g.audited, g.audit_accepted) == \
                       (s.screened, s.audited, s.audit_accepted), (r, t)
                if cfg.weight_mode == G.ABC_W_IMPORTANCE:
                    assert g.ess == s.ess, (r, t)
                screened_any += g.screened
        assert screened_any > 0  # the screen did run in the graph
    finally:
        G.abc_batch_free(b)
        for ctx in ctxs:
            G.abc_free(ctx)


def test_tolerance_target_stops_runs():
    """eps_stop: a run whose generation ends at or below its target is done --
    a single context returns ABC_STOP_TARGET afterwards, and in a graph batch
    that run stops while the others go on, its population kept."""
    base = [saird_config(2048, 30, 100_000, seed=31, weight_mode=G.ABC_W_IMPORTANCE),
            saird_config(1024, 30, 100_000, seed=32, weight_mode=G.ABC_W_IMPORTANCE)]
    obs = [oracle_obs(c)[0] for c in base]
    ref = G.abc_init(base[0], obs[0])
    try:
        G.abc_run(ref, 6)
        target = G.abc_get_stats(ref, 3).eps
        ref_pop = None
        G.abc_reset(ref, base[0].run_id)
        G.abc_run(ref, 4)
        ref_pop = get_population(ref, 2048)
    finally:
        G.abc_free(ref)
    f = np.float32(target)  # the smallest float32 at or above the target (compared in fp64)
    if float(f) < target:
        f = np.nextafter(f, np.float32(np.inf))
    stop = saird_config(2048, 30, 100_000, seed=31, weight_mode=G.ABC_W_IMPORTANCE,
                        eps_stop=float(f))
    ctx = G.abc_init(stop, obs[0])
    try:
        assert G.abc_run(ctx, 10) == G.ABC_STOP_TARGET
        assert G.abc_generations(ctx) == 4
        assert G.abc_generation(ctx) == G.ABC_STOP_TARGET
    finally:
        G.abc_free(ctx)
    b = G.abc_batch_init([stop, base[1]], obs)
    try:
        G.abc_batch_run(b, 7)
        assert G.abc_batch_active(b) == 1
        assert G.abc_batch_generations(b) == 7
        gp = _batch_pop(b, 0, 2048)
        for k in gp:
            assert np.array_equal(gp[k].view(np.uint8), ref_pop[k].view(np.uint8)), k
    finally:
        G.abc_batch_free(b)
