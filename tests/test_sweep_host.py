"""Host logic of the parallelism sweep (Sec. 4.1): the per-trial configs and
the per-level summary, on hand-made curves whose answers are known."""
import math

import numpy as np

import paper_2106_15508_gb300 as G
from paper_2106_15508_gb300 import sweep as S


def test_sweep_configs_cover_levels_and_trials():
    cfgs = S.sweep_configs(levels=(10, 100, 1000), trials=4, N=1000, budget=1000)
    assert len(cfgs) == 12
    assert [c.batch_size for c in cfgs] == [10] * 4 + [100] * 4 + [1000] * 4
    assert len({c.run_id for c in cfgs}) == 12          # independent Philox keys
    for c in cfgs:
        assert c.n_particles == 1000 and c.max_total_batches == 1000
        assert c.weight_mode == G.ABC_W_PAPER and c.beta_mode == G.ABC_BETA_PAPER
        assert c.n_days == 120 and c.population == 10_000_000
        assert c.max_batches == 65535
    # batches per round: about 65536 simulations in flight, 1 to 64
    assert [c.spec_batches for c in cfgs[::4]] == [64, 64, 64]
    assert S.spec_for(100000) == 1 and S.spec_for(10000) == 7
    assert all(c.spec_batches == 1 for c in S.sweep_configs(levels=(10,), trials=2,
                                                            spec_target=0))


def _c(M, trial, runs, eps, status=G.ABC_OK, days=0):
    return S.Curve(M, trial, np.array(runs, np.int64), np.array(eps, np.float64), days, 0,
                   status)


def test_summary_on_known_curves():
    curves = [
        _c(10, 0, [300, 700, 1100], [50.0, 20.0, 20.0], days=5),
        _c(10, 1, [250, 1200], [40.0, 10.0], days=7),
        _c(10, 2, [], [], status=G.ABC_STOP_BUDGET),
        _c(100, 0, [11, 12, 13], [9.0, 4.0, 1000.0]),
    ]
    s = S.summarise(curves)
    assert sorted(s) == [10, 100]
    a = s[10]
    assert a["trials"] == 3 and a["with_stages"] == 2 and a["stuck"] == 1
    # best tolerances 20 and 10; first stage reaching them at 700 and 1200 runs
    assert a["best_eps_median"] == 15.0
    assert a["runs_to_best_median"] == 950.0
    # within 2x of the best (40 and 20): 700 and 1200 runs
    assert a["runs_to_2x_best_median"] == 950.0
    assert a["runs_total_median"] == 1100.0           # totals 1100, 1200, 0
    assert a["stages_median"] == 2.0
    assert math.isclose(a["log10_best_eps_std"], np.std(np.log10([20.0, 10.0])))
    assert a["sim_days"] == 12
    b = s[100]
    assert b["best_eps_median"] == 4.0 and b["runs_to_best_median"] == 12.0
    assert b["runs_to_2x_best_median"] == 12.0
    assert b["log10_best_eps_std"] == 0.0


def test_mcmc_arm_configs():
    """The baseline arm: the single tuned step with the paper's adaptation
    window (0 = the first tenth of the run budget), one batch per round, the
    same levels, trials, budget and run ids as the BDSS arm."""
    b = S.sweep_configs(levels=(10, 1000), trials=3, N=1000, budget=1000)
    m = S.sweep_configs(levels=(10, 1000), trials=3, N=1000, budget=1000, method="mcmc",
                        mcmc_s0=0.05)
    assert [c.run_id for c in m] == [c.run_id for c in b]
    assert [c.batch_size for c in m] == [c.batch_size for c in b]
    for c in m:
        assert c.beta_mode == G.ABC_STEP_MCMC and math.isclose(c.mcmc_s0, 0.05, rel_tol=1e-7)
        assert c.mcmc_adapt == 0 and c.max_total_batches == 1000 and c.spec_batches == 1
        assert S.method_of(c) == "mcmc"
    assert all(S.method_of(c) == "bdss" for c in b)
    try:
        S.sweep_configs(levels=(10,), trials=1, method="abc")
        raise AssertionError("an unknown method must be refused")
    except ValueError:
        pass


def test_summary_per_method():
    curves = [_c(10, 0, [300, 700], [50.0, 20.0]), _c(10, 1, [250], [40.0])]
    mc = S.Curve(10, 0, np.array([400], np.int64), np.array([60.0]), 0, 0, G.ABC_OK,
                 method="mcmc")
    s = S.summarise_methods(curves + [mc])
    assert sorted(s) == ["bdss", "mcmc"]
    assert s["bdss"][10]["trials"] == 2 and s["mcmc"][10]["trials"] == 1
    assert s["mcmc"][10]["best_eps_median"] == 60.0
    assert S.summarise_methods(curves).keys() == {"bdss"}
