"""Several batches per device loop round (abc_config.spec_batches) in
graph-captured batches: the batches of a stage depend on the stage's state
only, so K of them are proposed and simulated together and accepted in
(batch, slot) order.  Every run must equal the oracle's sequential run bit
for bit: populations, tolerances, batches used, accepted and exhausted
counts, budget stops and run budgets."""
import numpy as np
import pytest

import oracle as O
import paper_2106_15508_gb300 as G
from paper_2106_15508_gb300 import build as B

from helpers import oracle_model, oracle_obs, oracle_smc, saird_config

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


# (N, M, K, max_batches, run budget, seed, weight mode)
SPECS = [(64, 8, 16, 4096, 60, 51, G.ABC_W_PAPER),
         (256, 16, 64, 4096, 0, 52, G.ABC_W_PAPER),
         (256, 100, 4, 4096, 40, 53, G.ABC_W_IMPORTANCE),
         (128, 32, 7, 4096, 0, 54, G.ABC_W_PAPER),
         (256, 8, 16, 30, 0, 55, G.ABC_W_PAPER)]     # a stage outgrows 30 batches


def test_speculative_rounds_match_oracle():
    cfgs = [saird_config(N, 30, 100_000, seed=sd, batch_size=M, spec_batches=K, max_batches=mb,
                         max_total_batches=bud, weight_mode=wm)
            for N, M, K, mb, bud, sd, wm in SPECS]
    obs = [oracle_obs(c)[0] for c in cfgs]
    G_MAX = 8
    b = G.abc_batch_init(cfgs, obs)
    try:
        G.abc_batch_run(b, G_MAX)
        for r, cfg in enumerate(cfgs):
            pop, ost = O.run(oracle_model(cfg, obs[r]), oracle_smc(cfg), G_MAX)
            assert len(ost) >= 1
            for t, s in enumerate(ost, start=1):
                g = G.abc_batch_get_stats(b, r, t)
                assert (g.status, g.eps, g.batches, g.accepted, g.exhausted) == \
                    (s.status, s.eps, s.batches, s.accepted_total, s.exhausted), (r, t)
            with pytest.raises(G.AbcError):
                G.abc_batch_get_stats(b, r, len(ost) + 1)
            u = np.zeros((8, cfg.n_particles), np.float32)
            d = np.zeros(cfg.n_particles)
            W = np.zeros(cfg.n_particles)
            s_ = np.zeros(cfg.n_particles, np.float32)
            a = np.zeros(cfg.n_particles, np.int32)
            G.abc_batch_get_population(b, r, u, d, W, s_, a)
            assert _same(u, pop.u) and _same(d, pop.d) and _same(s_, pop.s), r
            assert _same(a, pop.anc), r
            if cfg.weight_mode == G.ABC_W_PAPER:
                assert _same(W, pop.W), r
            if r == 4:   # a stage that needed more than 30 batches stopped the run
                assert ost[-1].status == G.ABC_STOP_BUDGET
    finally:
        G.abc_batch_free(b)


@pytest.mark.parametrize("N,M,K,mb,bud,seed", [(64, 8, 16, 4096, 60, 61), (256, 16, 64, 4096, 0, 62),
                                                (256, 8, 16, 30, 0, 63)])
def test_context_speculative_rounds_match_oracle(N, M, K, mb, bud, seed):
    cfg = saird_config(N, 30, 100_000, seed=seed, batch_size=M, spec_batches=K, max_batches=mb,
                       max_total_batches=bud)
    obs = oracle_obs(cfg)[0]
    pop, ost = O.run(oracle_model(cfg, obs), oracle_smc(cfg), 8)
    ctx = G.abc_init(cfg, obs)
    try:
        G.abc_run(ctx, 8)
        assert G.abc_generations(ctx) == 1 + sum(s.status == 0 for s in ost)
        for t, s in enumerate(ost, start=1):
            g = G.abc_get_stats(ctx, t)
            assert (g.status, g.eps, g.batches, g.accepted, g.exhausted) == \
                (s.status, s.eps, s.batches, s.accepted_total, s.exhausted), t
        u = np.zeros((8, N), np.float32)
        d = np.zeros(N)
        G.abc_get_population(ctx, u, d)
        assert _same(u, pop.u) and _same(d, pop.d)
    finally:
        G.abc_free(ctx)


def test_spec_batches_validated():
    for bad in (-1, 257):
        cfg = saird_config(64, 10, 1000, batch_size=8, spec_batches=bad)
        with pytest.raises(G.AbcError):
            G.abc_init(cfg, oracle_obs(saird_config(64, 10, 1000))[0])


def _toy(seed, N, M, K):
    lo, hi = [-10.0] * 8, [10.0] * 8
    return G.config(model=G.ABC_MODEL_GAUSS_TOY, n_days=1, population=1, init_ard=[0, 0, 0],
                    theta_lo=lo, theta_hi=hi, x_obs=[0.5] * 8, seed=seed, n_particles=N,
                    batch_size=M, spec_batches=K, max_batches=4096)


def test_speculative_rounds_other_models_and_rules():
    """The Gaussian toy, the paper's floor-normal flows and a real-shape Beta
    rule (the stage t = c1 >> 16 must not see the batch offset) under K > 1."""
    cfgs = [_toy(71, 128, 16, 8),
            saird_config(128, 30, 100_000, seed=72, batch_size=16, spec_batches=12,
                         sampler=G.ABC_SIM_PAPER_NORMAL, max_batches=4096),
            saird_config(128, 30, 100_000, seed=73, batch_size=16, spec_batches=12,
                         beta_mode=G.ABC_BETA_MODE_CONC, beta_p1=0.2, beta_p2=10.0,
                         max_batches=4096)]
    obs = [None, oracle_obs(cfgs[1])[0], oracle_obs(cfgs[2])[0]]
    b = G.abc_batch_init(cfgs, obs)
    try:
        G.abc_batch_run(b, 6)
        for r, cfg in enumerate(cfgs):
            m = oracle_model(cfg, obs[r]) if obs[r] is not None else oracle_model(cfg)
            pop, ost = O.run(m, oracle_smc(cfg), 6)
            for t, s in enumerate(ost, start=1):
                g = G.abc_batch_get_stats(b, r, t)
                assert (g.status, g.eps, g.batches, g.accepted, g.exhausted) == \
                    (s.status, s.eps, s.batches, s.accepted_total, s.exhausted), (r, t)
            u = np.zeros((8, cfg.n_particles), np.float32)
            s_ = np.zeros(cfg.n_particles, np.float32)
            G.abc_batch_get_population(b, r, u, None, None, s_)
            assert _same(u, pop.u) and _same(s_, pop.s), r
    finally:
        G.abc_batch_free(b)
