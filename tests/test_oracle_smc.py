"""Pins of the oracle's ABC-SMC steps (Sec. 2.3-2.4, 3.2): percentile,
stage prior and categorical draw, Beta step and Gaussian walk, importance
weights against scipy's Gaussian densities, normalisation, generation
invariants and the Gaussian toy's closed-form ABC posterior."""
import json
import math
import os

import numpy as np
import pytest
import scipy.stats as st
from scipy.special import logsumexp

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def test_paper_constants_fixture():
    g = json.load(open(GOLDEN))
    assert list(O.SAIRD_THETA_MAX) == g["prior_upper"]["value"]
    m = O.OracleModel(T=1, P=100, A0=1, seed=1)
    u = O.prior(m, 5000)
    assert np.all((u > 0) & (u < 1))
    th = u * O.SAIRD_THETA_MAX[:, None]
    assert np.all(th.max(axis=1) <= O.SAIRD_THETA_MAX)
    # prior sample is uniform on the box (Eq. 2)
    for d in range(8):
        assert st.kstest(u[d], "uniform").pvalue > 1e-3


@pytest.mark.parametrize("n,alpha", [(1, 0.5), (7, 0.5), (4096, 0.5), (1000, 0.1), (10, 0.99)])
def test_percentile_is_lower_order_statistic(n, alpha):
    """Eq. 8: eps = k-th smallest distance, k = ceil(alpha N)."""
    rng = np.random.default_rng(n)
    d = rng.integers(0, 50, n).astype(np.float64)  # with ties
    k = O.rank(alpha, n)
    assert k == max(1, min(n, math.ceil(alpha * n)))
    assert O.kth(d, k) == np.sort(d)[k - 1]


def test_stage_prior_weights_and_prefix():
    """Eq. 9-10: survivors d <= eps; mode 0 weight eps - d, mode 1 the
    previous weight; u32 quantisation relative to the largest weight."""
    rng = np.random.default_rng(5)
    d = rng.uniform(0, 10, 1000)
    W = rng.uniform(0, 1, 1000)
    eps = 5.0
    for mode in (0, 1):
        q, pre, tot = O.resample_prefix(d, W, eps, mode)
        r = np.where(d <= eps, eps - d if mode == 0 else W, 0.0)
        assert np.all(q[d > eps] == 0)
        assert q[np.argmax(r)] == 2**32 - 1
        assert np.all(np.abs(q / 4294967295.0 - r / r.max()) <= 2.0**-32 + 1e-15)
        assert np.array_equal(pre, np.cumsum(q.astype(np.uint64)))
        assert tot == int(pre[-1])
    # degenerate: every survivor at exactly eps (all mode-0 weights zero)
    q, pre, tot = O.resample_prefix(np.full(10, 3.0), None, 3.0, 0)
    assert np.all(q == 1) and tot == 10


def _center_population(n, seed=0):
    rng = np.random.default_rng(seed)
    return (0.5 + 0.01 * rng.standard_normal((8, n))).astype(np.float32)


def test_categorical_ancestor_frequencies():
    """Eq. 11: ancestors are drawn with probability q_k / total."""
    n = 50
    m = O.OracleModel(T=1, P=100, A0=1, seed=3)
    u = _center_population(n)
    rng = np.random.default_rng(1)
    q = rng.integers(0, 2**32, n).astype(np.uint32)
    q[[3, 17]] = 0
    pre = np.cumsum(q.astype(np.uint64))
    slots = 60000
    out = O.propose(m, u, pre, int(pre[-1]), 1.0, 1000, slots, c1=(1 << 16), nthreads=4)
    assert np.all(out["flag"] == 0)
    cnt = np.bincount(out["anc"], minlength=n)
    assert cnt[3] == 0 and cnt[17] == 0
    exp = q / q.sum() * slots
    m_ = exp > 0
    chi = ((cnt[m_] - exp[m_]) ** 2 / exp[m_]).sum()
    assert st.chi2.sf(chi, m_.sum() - 1) > 1e-3


@pytest.mark.parametrize("a,b", [(1.0, 2), (0.5, 5), (2.0, 5)])
def test_walk_is_gaussian_with_beta_variance(a, b):
    """Eq. 16-17: s ~ Beta(a, b) and u' = u_anc + sqrt(s) z, z ~ N(0, I);
    checked where the first attempt succeeded (population at the centre)."""
    n = 20
    m = O.OracleModel(T=1, P=100, A0=1, seed=int(a * 10) + b)
    u = _center_population(n, 2)
    q = np.ones(n, np.uint32)
    pre = np.cumsum(q.astype(np.uint64))
    slots = 20000
    out = O.propose(m, u, pre, n, a, b, slots, c1=(2 << 16) | 1, nthreads=4)
    ok = (out["flag"] == 0)
    up, s, anc = out["u"], out["s"], out["anc"]
    assert np.all((up[:, ok] >= 0) & (up[:, ok] <= 1))
    first = ok & (out["attempts"] == 1)
    # s of first-attempt draws is biased to small values by the support check;
    # the walk, given s, is not
    z = (up[:, first] - u[:, anc[first]]) / np.sqrt(s[first])[None, :]
    # condition on s small enough that the support is never reached
    small = s[first] < 0.0025
    if small.sum() > 200:
        assert st.kstest(z[:, small].ravel(), "norm").pvalue > 1e-3
    # the step sizes of all attempts are Beta(a, b): re-draw them directly
    s_all = np.array([O.beta(m.key, a, b, j, (2 << 16) | 1, 0) for j in range(3000)])
    assert st.kstest(s_all, st.beta(a, b).cdf).pvalue > 1e-3


def test_redraw_exhaustion_is_flagged():
    """Proposals that leave [0,1]^8 are redrawn; after max_redraw attempts the
    slot is flagged and its attempt count equals max_redraw."""
    n = 10
    m = O.OracleModel(T=1, P=100, A0=1, seed=4)
    u = np.full((8, n), 0.999, np.float32)
    pre = np.arange(1, n + 1, dtype=np.uint64)
    out = O.propose(m, u, pre, n, 5.0, 1, 500, c1=(1 << 16), max_redraw=2)
    assert out["flag"].sum() > 0
    assert np.all(out["attempts"][out["flag"] == 1] == 2)
    assert np.all(out["attempts"][out["flag"] == 0] <= 2)


def test_weights_single_survivor_closed_form():
    """One survivor: log W = -log N(u'; u_1, s I8) (scipy's density)."""
    rng = np.random.default_rng(7)
    u = rng.uniform(0, 1, (8, 4)).astype(np.float32)
    q = np.array([0, 12345, 0, 0], np.uint32)
    up = rng.uniform(0, 1, (8, 50)).astype(np.float32)
    s = rng.uniform(0.001, 0.3, 50).astype(np.float32)
    lw = O.weights(up, s, u, q, 12345)
    for j in range(50):
        want = -st.multivariate_normal(u[:, 1].astype(np.float64),
                                       float(s[j]) * np.eye(8)).logpdf(up[:, j].astype(np.float64))
        assert abs(lw[j] - want) <= 1e-10 * max(1, abs(want))


def test_weights_mixture_against_scipy():
    """log W_j = -log sum_k (q_k / total) N(u'_j; u_k, s_j I8)."""
    rng = np.random.default_rng(8)
    n, rows = 300, 40
    u = rng.uniform(0, 1, (8, n)).astype(np.float32)
    q = rng.integers(0, 2**32, n).astype(np.uint32)
    q[::7] = 0
    tot = int(q.astype(np.uint64).sum())
    up = rng.uniform(0, 1, (8, rows)).astype(np.float32)
    s = np.exp(rng.uniform(np.log(1e-4), np.log(0.5), rows)).astype(np.float32)
    lw = O.weights(up, s, u, q, tot)
    for j in range(rows):
        keep = q > 0
        comp = [st.multivariate_normal(u[:, k].astype(np.float64), float(s[j]) * np.eye(8))
                .logpdf(up[:, j].astype(np.float64)) for k in np.where(keep)[0]]
        want = -logsumexp(np.array(comp) + np.log(q[keep].astype(np.float64) / tot))
        assert abs(lw[j] - want) <= 1e-9 * max(1, abs(want)), (j, lw[j], want)
    # the kernel variance is floored at 1e-30: s = 0 and s = 1e-30 agree
    w0 = O.weights(up[:, :3], np.zeros(3, np.float32), u, q, tot)
    w1 = O.weights(up[:, :3], np.full(3, 1e-30, np.float32), u, q, tot)
    assert np.array_equal(w0, w1) and np.all(np.isfinite(w0))


def test_normalize_and_ess():
    W, ess = O.normalize(np.zeros(100))
    assert np.allclose(W, 0.01) and abs(ess - 100) < 1e-9
    W, ess = O.normalize(np.array([0.0, -1000.0, -1000.0]))
    assert abs(ess - 1) < 1e-9 and abs(W.sum() - 1) < 1e-15
    rng = np.random.default_rng(0)
    lw = rng.normal(0, 3, 1000)
    W, ess = O.normalize(lw)
    p = np.exp(lw - logsumexp(lw))
    assert np.allclose(W, p, rtol=1e-12)
    assert abs(ess - 1 / np.sum(p**2)) < 1e-9 * ess
    W, ess = O.normalize(np.full(4, -np.inf))
    assert np.allclose(W, 0.25) and ess == 4
    W, ess = O.normalize(np.array([0.0, np.nan, 0.0]))  # NaN counts as weight 0
    assert np.allclose(W, [0.5, 0.0, 0.5]) and abs(ess - 2) < 1e-12


def _small_saird(seed=1, T=30, P=100000):
    A0 = max(10, round(1e-4 * P))
    m = O.OracleModel(T=T, P=P, A0=A0, seed=seed)
    obs, _, _ = O.synth_obs(m)
    m.set_obs(obs)
    return m


@pytest.mark.parametrize("weight_mode", [0, 1])
def test_generation_invariants(weight_mode):
    """eps non-increasing (Sec. 2.4), accepted d <= eps_t, paper Beta
    schedule a_1 = eps_1/eps_1 = 1, b_1 = 2 (Eq. 16, Sec. 3.2.2's Beta(1,2)),
    ancestors are survivors with positive weight, weights sum to one."""
    m = _small_saird()
    c = O.make_smc(512, weight_mode=weight_mode, nthreads=4)
    pop = O.generation0(m, c)
    eps1, prev_eps = 0.0, math.inf
    for t in range(1, 6):
        q, pre, tot = O.resample_prefix(pop.d, pop.W, O.kth(pop.d, O.rank(0.5, 512)),
                                        weight_mode)
        new, stt = O.generation(m, c, t, eps1, pop)
        assert stt.status == 0
        if t == 1:
            assert stt.beta_a == 1.0 and stt.beta_b == 2
            eps1 = stt.eps1
        else:
            assert stt.beta_b == 2 * t and stt.beta_a == np.float32(stt.eps / eps1)
        assert stt.eps <= prev_eps
        prev_eps = stt.eps
        assert np.all(new.d <= stt.eps)
        assert np.all(pop.d[new.anc] <= stt.eps) and np.all(q[new.anc] > 0)
        assert abs(new.W.sum() - 1) < 1e-12
        assert stt.total == tot
        pop = new


def test_oracle_is_deterministic_and_thread_invariant():
    m = _small_saird(seed=2, T=20)
    r1 = O.run(m, O.make_smc(256, weight_mode=1, nthreads=1), 4)
    r2 = O.run(m, O.make_smc(256, weight_mode=1, nthreads=4), 4)
    assert np.array_equal(r1[0].u, r2[0].u) and np.array_equal(r1[0].d, r2[0].d)
    assert np.array_equal(r1[0].W, r2[0].W)


def test_gaussian_toy_closed_form_posterior():
    """Conjugate toy (x ~ N(theta, I8), flat box prior, x_obs = 0): the ABC
    posterior at tolerance eps is Y - Z with Y uniform on the eps-ball and
    Z ~ N(0, I8): mean 0, variance 1 + eps^2/10 per coordinate.  Importance
    weights (mode 1) with a narrow fixed Beta(8, 1000) step; 10 independent
    runs (seeds 1..10).  Per run, the weighted mean and the weighted variance
    over v0 = 1 + eps^2/10 are averaged over the 8 exchangeable coordinates;
    over the 10 runs both must lie within 2 Monte-Carlo standard errors
    (the runs' standard deviation / sqrt 10) of 0 and 1."""
    lo, hi = np.full(8, -10, np.float32), np.full(8, 10, np.float32)
    means, ratios = [], []
    for seed in range(1, 11):
        m = O.OracleModel(model=1, T=0, P=1, theta_lo=lo, theta_hi=hi, seed=seed)
        c = O.make_smc(2048, beta_mode=1, beta_a=8.0, beta_b=1000, weight_mode=1,
                       max_batches=400, nthreads=4)
        pop, stats = O.run(m, c, 10)
        assert all(s.status == 0 for s in stats)
        eps = stats[-1].eps
        th = lo[:, None] + pop.u * (hi - lo)[:, None]
        mean = (th * pop.W).sum(1)
        var = (th**2 * pop.W).sum(1) - mean**2
        means.append(mean.mean())
        ratios.append(var.mean() / (1 + eps**2 / 10))
    means, ratios = np.array(means), np.array(ratios)
    se_m = means.std(ddof=1) / math.sqrt(len(means))
    se_v = ratios.std(ddof=1) / math.sqrt(len(ratios))
    assert abs(means.mean()) < 2 * se_m, (means, se_m)
    assert abs(ratios.mean() - 1) < 2 * se_v, (ratios, se_v)
