"""Pins of the oracle's delayed-acceptance screen (surrogate pre-screen;
an extension beyond the paper, not in the paper): the pass probability against the
logistic function in fp64, its clamps, the exhausted-slot rule, and the
frequencies of the two Bernoulli draws (pass with probability rho, audit with
probability audit_frac among the rest) against their binomial laws, plus the
two-stage acceptance identity that justifies the 1/rho weight factor."""
import math

import numpy as np

import oracle as O


def _model(seed=3):
    return O.OracleModel(T=1, P=100, A0=1, seed=seed)


def _rho_fp64(y, ystat, eps, tau, rho_min):
    y0 = np.float64(ystat[0]) + np.float64(ystat[4]) * y.astype(np.float64)
    r = 1.0 / (1.0 + np.exp(-(math.log1p(eps) - y0) / tau))
    return np.clip(r, rho_min, 1.0)


def test_rho_is_the_clamped_logistic():
    rng = np.random.default_rng(1)
    M = 20000
    Y = rng.normal(0, 2, (M, 4)).astype(np.float32)
    ystat = np.array([12.0, 0, 0, 0, 1.5, 1, 1, 1], np.float32)
    eps = 4.0e5
    rho, sf = O.screen(_model(), Y, ystat, None, eps, 7, 0.5, 0.05, 0.01)
    want = _rho_fp64(Y[:, 0], ystat, eps, 0.5, 0.05)
    # fp32 arithmetic: a few roundings of the logistic's argument (|z| <= ~50)
    # move rho by at most ~|z| rho (1 - rho) 2^-21 plus the final ulps
    z = np.abs((math.log1p(eps) - (12.0 + 1.5 * Y[:, 0].astype(np.float64))) / 0.5)
    tol = want * (1 - want) * (z + 4) * 2.0**-21 + 4 * 2.0**-24
    assert np.all(np.abs(rho - want) <= tol)
    assert np.all((rho >= np.float32(0.05)) & (rho <= 1.0))
    assert set(np.unique(sf)) <= {0, 2, 3}


def test_clamps_nan_and_exhausted_slots():
    ystat = np.array([0.0, 0, 0, 0, 1.0, 1, 1, 1], np.float32)
    Y = np.zeros((6, 4), np.float32)
    Y[:, 0] = [1e6, -1e6, np.nan, np.inf, -np.inf, 0.0]
    flag = np.array([0, 0, 0, 0, 0, 1], np.uint8)
    rho, sf = O.screen(_model(), Y, ystat, flag, 10.0, 1, 0.25, 0.1, 0.0)
    assert rho[0] == np.float32(0.1) and rho[1] == 1.0   # predicted far above / below eps
    assert rho[2] == np.float32(0.1)                       # NaN prediction: the floor
    assert rho[3] == np.float32(0.1) and rho[4] == 1.0
    assert rho[5] == 1.0 and sf[5] == 1                    # redraw-exhausted: not simulated
    assert sf[1] == 0 and sf[4] == 0                       # rho 1 always passes
    assert np.all(sf[:5] != 2)                             # audit_frac 0: no audits


def test_pass_and_audit_frequencies():
    """With a constant prediction rho is constant: passes ~ Bin(M, rho);
    audits ~ Bin(M - passes, audit_frac); both within 5 standard deviations."""
    M = 200000
    ystat = np.array([0.0, 0, 0, 0, 1.0, 1, 1, 1], np.float32)
    le = math.log1p(50.0)
    for target in (0.05, 0.3, 0.77):
        y = le + 0.5 * math.log(1 / target - 1)  # logistic((le - y) / 0.5) = target
        Y = np.full((M, 4), y, np.float32)
        rho, sf = O.screen(_model(5), Y, ystat, None, 50.0, 11, 0.5, 0.01, 0.2)
        r = float(rho[0])
        assert abs(r - target) < 1e-5 and np.all(rho == rho[0])
        npass = int(np.sum(sf == 0))
        assert abs(npass - M * r) < 5 * math.sqrt(M * r * (1 - r))
        rest = M - npass
        naud = int(np.sum(sf == 2))
        assert abs(naud - rest * 0.2) < 5 * math.sqrt(rest * 0.2 * 0.8)
        assert npass + naud + int(np.sum(sf == 3)) == M


def test_draws_follow_the_counters():
    """The uniforms are Philox blocks (slot, c1, 0, SCREEN / AUDIT): the same
    counters give the same decisions, another c1 or key other ones, and a
    slot's decision does not depend on M."""
    rng = np.random.default_rng(4)
    Y = rng.normal(0, 1, (5000, 4)).astype(np.float32)
    ystat = np.array([3.0, 0, 0, 0, 1.0, 1, 1, 1], np.float32)
    a = O.screen(_model(3), Y, ystat, None, 20.0, (4 << 16) | 2, 1.0, 0.05, 0.5)[1]
    b = O.screen(_model(3), Y, ystat, None, 20.0, (4 << 16) | 2, 1.0, 0.05, 0.5)[1]
    c = O.screen(_model(3), Y, ystat, None, 20.0, (4 << 16) | 3, 1.0, 0.05, 0.5)[1]
    d = O.screen(_model(4), Y, ystat, None, 20.0, (4 << 16) | 2, 1.0, 0.05, 0.5)[1]
    e = O.screen(_model(3), Y[:777], ystat, None, 20.0, (4 << 16) | 2, 1.0, 0.05, 0.5)[1]
    assert np.array_equal(a, b) and np.array_equal(a[:777], e)
    assert np.mean(a != c) > 0.2 and np.mean(a != d) > 0.2
    # the pass uniform is the first word of the SCREEN block
    key = _model(3).key
    for i in (0, 1, 4999):
        w = O.philox([i, (4 << 16) | 2, 0, O.TAG_SCREEN], key)
        rho = O.screen(_model(3), Y[i:i + 1], ystat, None, 20.0, (4 << 16) | 2, 1.0, 0.05, 0.5)[0]
        assert (a[i] == 0) == (O.uniform(int(w[0])) < rho[0])


def test_two_stage_acceptance_identity():
    """Proposals x ~ q, kept with probability rho(x): weighting the kept ones
    by 1/rho(x) gives unbiased q-expectations (the reason accepted particles
    carry the factor 1/rho).  x ~ U(0,1) stands in for the proposal."""
    M = 400000
    rng = np.random.default_rng(9)
    x = rng.random(M)
    ystat = np.array([0.0, 0, 0, 0, 1.0, 1, 1, 1], np.float32)
    Y = np.zeros((M, 4), np.float32)
    Y[:, 0] = (4.0 * x - 1.0).astype(np.float32)  # the screen prefers small x
    rho, sf = O.screen(_model(8), Y, ystat, None, 0.5, 1, 0.7, 0.05, 0.0)
    keep = sf == 0
    w = 1.0 / rho[keep].astype(np.float64)
    for f in (lambda v: v, lambda v: v * v, lambda v: np.cos(3 * v)):
        fx = f(x)
        est = np.sum(w * fx[keep]) / M
        se = math.sqrt(np.var(np.where(keep, fx / np.maximum(rho, 1e-9), 0.0)) / M)
        assert abs(est - fx.mean()) < 5 * se
    # unweighted, the kept sample is biased towards small x
    assert x[keep].mean() < x.mean() - 0.05
