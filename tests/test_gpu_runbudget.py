"""The run budget of Sec. 4.1 (each trial stops on the stage that reached a
count of simulation runs, i.e. batches of M parallel simulations, and that
stage finishes) and the paper's step-size schedule past stage 512, on the
GPU against the oracle's run driver, bit for bit: single-run contexts, the
checkpoint, and graph-captured batches."""
import numpy as np
import pytest

import oracle as O
import paper_2106_15508_gb300 as G
from paper_2106_15508_gb300 import build as B

from helpers import get_population, oracle_model, oracle_obs, oracle_smc, saird_config, state_blob

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    G.lib()


def _same(a, b):
    return np.array_equal(np.ascontiguousarray(a).view(np.uint8),
                          np.ascontiguousarray(b).view(np.uint8))


def _counts(cfg, stats):
    """Batches so far after each generation t >= 1 (stage 0: ceil(N / M))."""
    M = cfg.batch_size or cfg.n_particles
    return -(-cfg.n_particles // M) + np.cumsum([s.batches for s in stats])


BUDGET_CASES = [(256, 64, 20), (256, 256, 9), (512, 32, 40), (256, 32, 8), (256, 128, 1)]


@pytest.mark.parametrize("N,M,budget", BUDGET_CASES)
def test_context_run_budget_matches_oracle(N, M, budget):
    cfg = saird_config(N, 30, 100_000, seed=21, batch_size=M, max_total_batches=budget,
                       max_batches=4096)
    obs, _, _ = oracle_obs(cfg)
    pop, ost = O.run(oracle_model(cfg, obs), oracle_smc(cfg), 60)
    assert all(s.status == 0 for s in ost)
    counts = _counts(cfg, ost)
    if -(-N // M) >= budget:
        assert len(ost) == 0
    else:
        assert counts[-1] >= budget and (len(ost) == 1 or counts[-2] < budget)
    ctx = G.abc_init(cfg, obs)
    try:
        rc = G.abc_run(ctx, 60)
        assert rc == G.ABC_STOP_TOTAL
        assert G.abc_generations(ctx) == len(ost) + 1
        for t, s in enumerate(ost, start=1):
            g = G.abc_get_stats(ctx, t)
            assert g.eps == s.eps and g.batches == s.batches and g.status == 0
        if ost:
            gp = get_population(ctx, N)
            for k, ok in (("u", pop.u), ("d", pop.d), ("s", pop.s), ("anc", pop.anc)):
                assert _same(gp[k], ok), k
        assert G.abc_generation(ctx) == G.ABC_STOP_TOTAL   # nothing more runs
    finally:
        G.abc_free(ctx)


def test_checkpoint_carries_the_run_budget():
    """A context restored from generation 2 with the count so far stops where
    the uninterrupted run stops."""
    N, M, budget = 256, 64, 30
    cfg = saird_config(N, 30, 100_000, seed=22, batch_size=M, max_total_batches=budget,
                       max_batches=4096)
    obs, _, _ = oracle_obs(cfg)
    m, c = oracle_model(cfg, obs), oracle_smc(cfg)
    pop_end, ost = O.run(m, c, 60)
    assert len(ost) >= 3
    pop = O.generation0(m, c)
    eps1 = 0.0
    for t in (1, 2):
        pop, st = O.generation(m, c, t, eps1, pop)
        eps1 = st.eps1
    count = -(-N // M) + ost[0].batches + ost[1].batches
    ctx = G.abc_init(cfg, obs)
    try:
        G.abc_set_state(ctx, state_blob(cfg, 3, eps1, pop, batches_total=count))
        assert G.abc_run(ctx, 60) == G.ABC_STOP_TOTAL
        assert G.abc_generations(ctx) == len(ost) + 1
        gp = get_population(ctx, N)
        assert _same(gp["u"], pop_end.u) and _same(gp["d"], pop_end.d)
        # the blob written back carries the count
        blob = G.abc_get_state(ctx)
        assert blob[:8] == b"ABCSMC02"
        assert int(np.frombuffer(blob[48:56], np.int64)[0]) == int(_counts(cfg, ost)[-1])
    finally:
        G.abc_free(ctx)


def test_batch_run_budgets_match_oracle():
    """Runs of one batch with different M and budgets stop on their own
    stages (one of them on stage 0 alone); abc_batch_run ends once none is
    active."""
    specs = [(256, 64, 20, 31), (256, 256, 9, 32), (512, 32, 40, 33), (256, 128, 1, 34),
             (256, 16, 100, 35)]
    cfgs = [saird_config(N, 30, 100_000, seed=sd, batch_size=M, max_total_batches=bud,
                         max_batches=4096) for N, M, bud, sd in specs]
    obs = [oracle_obs(c)[0] for c in cfgs]
    b = G.abc_batch_init(cfgs, obs)
    try:
        G.abc_batch_generation(b)
        assert G.abc_batch_active(b) == 4   # the budget of 1 is used by stage 0
        G.abc_batch_run(b, 200)
        assert G.abc_batch_active(b) == 0 and G.abc_batch_generations(b) < 200
        for r, cfg in enumerate(cfgs):
            pop, ost = O.run(oracle_model(cfg, obs[r]), oracle_smc(cfg), 200)
            assert all(s.status == 0 for s in ost)
            for t, s in enumerate(ost, start=1):
                g = G.abc_batch_get_stats(b, r, t)
                assert g.eps == s.eps and g.batches == s.batches and g.status == s.status
            with pytest.raises(G.AbcError):
                G.abc_batch_get_stats(b, r, len(ost) + 1)   # nothing after the last stage
            if ost:
                u = np.zeros((8, cfg.n_particles), np.float32)
                d = np.zeros(cfg.n_particles)
                G.abc_batch_get_population(b, r, u, d)
                assert _same(u, pop.u) and _same(d, pop.d), r
    finally:
        G.abc_batch_free(b)


def _toy_cfg(seed, N=32, M=32, **kw):
    lo, hi = [-10.0] * 8, [10.0] * 8
    return G.config(model=G.ABC_MODEL_GAUSS_TOY, n_days=1, population=1, init_ard=[0, 0, 0],
                    theta_lo=lo, theta_hi=hi, x_obs=[0.5] * 8, seed=seed, n_particles=N,
                    batch_size=M, survival_alpha=1.0, max_batches=64, **kw)


def test_batch_paper_schedule_past_stage_512_matches_oracle():
    """Survival ratio 1 (and N in the hundreds) keeps the toy's acceptance high, so 516 generations
    run in a few batches each; generations 513 on draw Beta(eps_t/eps_1, 2t)
    by the Gamma ratio, on the GPU as in the oracle."""
    cfgs = [_toy_cfg(41, N=256, M=256), _toy_cfg(42, N=192, M=64)]
    b = G.abc_batch_init(cfgs, [None, None])
    try:
        G.abc_batch_run(b, 517)
        for r, cfg in enumerate(cfgs):
            pop, ost = O.run(oracle_model(cfg), oracle_smc(cfg), 517)
            assert len(ost) == 516 and all(s.status == 0 for s in ost)
            assert ost[511].beta_b == 1024 and ost[512].beta_b == 0 and ost[512].beta_bf == 1026
            for t in (512, 513, 516):
                g = G.abc_batch_get_stats(b, r, t)
                s = ost[t - 1]
                assert g.eps == s.eps and g.batches == s.batches
                assert g.beta_b == s.beta_b and g.beta_bf == s.beta_bf and g.beta_a == s.beta_a
            u = np.zeros((8, cfg.n_particles), np.float32)
            d = np.zeros(cfg.n_particles)
            s_ = np.zeros(cfg.n_particles, np.float32)
            G.abc_batch_get_population(b, r, u, d, None, s_)
            assert _same(u, pop.u) and _same(d, pop.d) and _same(s_, pop.s), r
    finally:
        G.abc_batch_free(b)


def test_context_generation_513_matches_oracle():
    cfg = _toy_cfg(43, N=64, M=64)
    m, c = oracle_model(cfg), oracle_smc(cfg)
    pop = O.generation0(m, c)
    pop, st = O.generation(m, c, 1, 0.0, pop)
    eps1 = st.eps1
    new, st = O.generation(m, c, 513, eps1, pop)
    assert st.status == 0 and st.beta_b == 0
    ctx = G.abc_init(cfg, None)
    try:
        G.abc_set_state(ctx, state_blob(cfg, 513, eps1, pop))
        assert G.abc_generation(ctx) == G.ABC_OK
        g = G.abc_get_stats(ctx, 513)
        assert g.beta_b == 0 and g.beta_bf == 1026.0 and g.beta_a == st.beta_a
        gp = get_population(ctx, 64)
        for k, ok in (("u", new.u), ("d", new.d), ("s", new.s), ("anc", new.anc)):
            assert _same(gp[k], ok), k
    finally:
        G.abc_free(ctx)
