"""The parallelism sweep (Sec. 4.1) on the GPU: every trial's curve (the
simulation runs so far and eps_t after each stage) equals the oracle run's
with the same config, bit for bit, on a reduced sweep -- for BDSS and for
the MCMC baseline arm, alone and in one batch together."""
import numpy as np
import pytest

import oracle as O
import paper_2106_15508_gb300 as G
from paper_2106_15508_gb300 import build as B
from paper_2106_15508_gb300 import sweep as S

from helpers import oracle_model, oracle_obs, oracle_smc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    G.lib()


@pytest.mark.parametrize("grouping", ["all", "level", "run"])
def test_reduced_sweep_matches_oracle_runs(grouping):
    cfgs = S.sweep_configs(levels=(8, 32, 256), trials=3, N=64, budget=24, T=30, P=100_000,
                           max_batches=4096)
    obs, _, _ = oracle_obs(cfgs[0])
    curves = S.run_sweep(cfgs, obs, grouping=grouping)
    for cfg, cv in zip(cfgs, curves):
        _, ost = O.run(oracle_model(cfg, obs), oracle_smc(cfg), 10_000)
        ok = [s for s in ost if s.status == 0]
        runs = -(-cfg.n_particles // cfg.batch_size) + np.cumsum([s.batches for s in ost])
        assert cv.M == cfg.batch_size and cv.trial == cfg.run_id % 3
        assert np.array_equal(cv.eps, np.array([s.eps for s in ok]))
        assert np.array_equal(cv.runs, runs[:len(ok)])
        assert cv.status == (ost[-1].status if ost else G.ABC_OK)
        if ok:
            assert cv.runs[-1] >= 24 and (len(ok) == 1 or cv.runs[-2] < 24)
    s = S.summarise(curves)
    assert sorted(s) == [8, 32, 256] and all(v["trials"] == 3 for v in s.values())


def test_reduced_sweep_both_methods_match_oracle_runs():
    """Both arms of the paper's comparison in one graph batch: the baseline's
    trials adapt their step over a tenth of the run budget (their first 3
    batches after the prior stage) inside the graph, and every curve equals
    the oracle's."""
    cfgs = [c for m in S.METHODS
            for c in S.sweep_configs(levels=(8, 64), trials=2, N=64, budget=24, T=30,
                                     P=100_000, max_batches=4096, method=m, mcmc_s0=0.05)]
    obs, _, _ = oracle_obs(cfgs[0])
    curves = S.run_sweep(cfgs, obs)
    for cfg, cv in zip(cfgs, curves):
        _, ost = O.run(oracle_model(cfg, obs), oracle_smc(cfg), 10_000)
        ok = [s for s in ost if s.status == 0]
        runs = -(-cfg.n_particles // cfg.batch_size) + np.cumsum([s.batches for s in ost])
        assert cv.method == S.method_of(cfg) and cv.trial == cfg.run_id % 2
        assert np.array_equal(cv.eps, np.array([s.eps for s in ok])), (cv.method, cv.M)
        assert np.array_equal(cv.runs, runs[:len(ok)])
    s = S.summarise_methods(curves)
    assert sorted(s) == ["bdss", "mcmc"] and sorted(s["mcmc"]) == [8, 64]
