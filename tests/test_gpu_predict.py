"""Posterior-predictive simulation (Sec. 4.2) on the GPU against the oracle:
resampled draws, trajectories over the training window and the days ahead
and the per-day order statistics (median, central 99% range and others) are
integers, so the GPU must match bit for bit."""
import numpy as np
import pytest

import oracle as O
import paper_2106_15508_gb300 as G
from paper_2106_15508_gb300 import build as B

import inputs as IN
from helpers import dev, empty, host, oracle_model, oracle_obs, saird_config

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

Q = [0.005, 0.25, 0.5, 0.995]


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    G.lib()


def _gpu_predict(cfg, u, W, R, days, q=Q):
    N = u.shape[1]
    sb = G.abc_predict_scratch_bytes(N, R, days, len(q))
    sc = empty(sb, torch.uint8)
    out = empty((days + 1, 3, len(q)), torch.int32)
    G.abc_predict(cfg, dev(u), None if W is None else dev(W), N, R, days, q, out, sc, sb)
    return host(out)


@pytest.mark.parametrize("N,R,days,weighted", [(4096, 3001, 90, True), (777, 1, 30, True),
                                               (4096, 2048, 150, False)])
def test_predict_bitexact(N, R, days, weighted):
    cfg = saird_config(N, 60, 100_000, seed=21)
    u = IN.clustered_particles(N, 22, 0.4, 0.15)
    W = None
    if weighted:
        W = np.exp(IN.rng(23).normal(0, 2, N))
        W /= W.sum()
    got = _gpu_predict(cfg, u, W, R, days)
    want = O.predict(oracle_model(cfg), u, W, R, days, Q)
    assert np.array_equal(got, want)
    assert np.all(got[:, :, 0] <= got[:, :, 2]) and np.all(got[:, :, 2] <= got[:, :, 3])


def test_predict_population_of_a_context():
    """abc_predict_population on a run's population equals abc_predict on
    the population read back from the context, and the oracle's."""
    cfg = saird_config(4096, 60, 100_000, seed=5, weight_mode=G.ABC_W_IMPORTANCE,
                       beta_mode=G.ABC_BETA_FIXED, beta_a=2.0, beta_b=5)
    obs, _, _ = oracle_obs(cfg)
    ctx = G.abc_init(cfg, obs)
    try:
        G.abc_run(ctx, 4)
        out = G.abc_predict_population(ctx, 5000, 90, Q)
        u = np.zeros((8, 4096), np.float32)
        d = np.zeros(4096)
        W = np.zeros(4096)
        s = np.zeros(4096, np.float32)
        a = np.zeros(4096, np.int32)
        G.abc_get_population(ctx, u, d, W, s, a)
    finally:
        G.abc_free(ctx)
    assert np.array_equal(out, _gpu_predict(cfg, u, W, 5000, 90))
    assert np.array_equal(out, O.predict(oracle_model(cfg, obs), u, W, 5000, 90, Q))
    # the first 60 days are the training window: the median of A stays in
    # the range the observed series spans
    med = out[1:61, 0, 2]
    assert med.max() >= 0.5 * obs[0, 1:61].min()


def test_predict_rejects_bad_levels():
    cfg = saird_config(64, 10, 1000)
    with pytest.raises(G.AbcError):
        _gpu_predict(cfg, IN.unit_particles(64, 1), None, 10, 5, q=[0.0, 0.5])
