"""The MCMC baseline in the oracle (Sec. 2.4.1 Eq. 12-15, Sec. 3.1): one
tuned step s for every proposal, adapted once per batch toward the target
acceptance A_T = 0.234 during the first 10% of the run.

Pins that do not restate the update: its fixed point, direction and bounds;
a Robbins-Monro run on a stationary stage that must settle at the target
acceptance; a whole generation replayed from the oracle's single steps; and
the conjugate Gaussian toy's closed-form ABC posterior reached with the
baseline's proposals and importance weights."""
import math

import numpy as np
import pytest

import oracle as O

A_T = 0.234


def test_adapt_fixed_point_direction_and_bounds():
    s = 0.05
    # 117 / 500 rounds to the same double as the literal 0.234: no change
    assert O.mcmc_adapt(s, 0, 117, 500) == s
    assert O.mcmc_adapt(s, 7, 117, 500) == s
    for k in (0, 1, 5, 100):
        up, down = O.mcmc_adapt(s, k, 400, 500), O.mcmc_adapt(s, k, 10, 500)
        assert up > s > down > 0
        # all accepted doubles the step at k = 0; none accepted shrinks it by
        # A_T / (1 - A_T) of the gain, never to zero or below
        hi, lo = O.mcmc_adapt(s, k, 500, 500), O.mcmc_adapt(s, k, 0, 500)
        assert math.isclose(hi / s, 1 + 1 / (k + 1), rel_tol=1e-15)
        assert math.isclose(lo / s, 1 - A_T / (1 - A_T) / (k + 1), rel_tol=1e-15)
        assert lo > 0.69 * s
        # nothing simulated counts as nothing accepted
        assert O.mcmc_adapt(s, k, 0, 0) == lo
    # the gain falls as 1 / (k + 1)
    steps = [abs(math.log(O.mcmc_adapt(1.0, k, 450, 500))) for k in range(6)]
    assert all(a > b for a, b in zip(steps, steps[1:]))


def test_window_is_a_tenth_of_the_run_budget():
    assert O.mcmc_window(O.make_smc(100, max_total=1000)) == 100
    assert O.mcmc_window(O.make_smc(100, max_total=1001)) == 101
    assert O.mcmc_window(O.make_smc(100, max_total=0)) == 0
    assert O.mcmc_window(O.make_smc(100, max_total=1000, mcmc_adapt=7)) == 7


def _toy(seed):
    lo, hi = np.full(8, -10, np.float32), np.full(8, 10, np.float32)
    return O.OracleModel(model=1, T=0, P=1, theta_lo=lo, theta_hi=hi, seed=seed), lo, hi


def test_robbins_monro_approaches_the_target_acceptance_from_both_sides():
    """A stationary stage (fixed population, tolerance at the 5% quantile of
    the prior draws' distances, fixed stage prior) of the Gaussian toy: the
    acceptance falls from about 0.8 for s -> 0 to about 0.15 at s = 0.1, so
    it crosses A_T once, near s = 0.06.  From a step too small (0.02) and one
    too large (0.15), 400 adapted batches of 1024 each move the acceptance
    toward A_T: the last 100 batches' mean acceptances bracket A_T, lie
    within 0.06 of it and closer than the first 10 batches', and the two
    steps, 7.5x apart at the start, end less than 2x apart on either side of
    the crossing.  (With gain 1 / (k + 1) the approach is slow: the step can
    grow by at most a factor k + 1 in k batches.)"""
    m, _, _ = _toy(5)
    c = O.make_smc(1024, max_batches=1, nthreads=4)
    pop = O.generation0(m, c)
    eps = O.kth(pop.d, O.rank(0.05, c.N))
    q, pre, tot = O.resample_prefix(pop.d, pop.W, eps, 0)
    ends, first, last = [], [], []
    for s0 in (0.02, 0.15):
        s, acc_rate = s0, []
        for k in range(400):
            c1 = (1 << 16) | k
            o = O.propose(m, pop.u, pre, tot, 1.0, 1, 1024, c1, nthreads=4,
                          s_fixed=float(np.float32(s)))
            d = O.simulate(m, o["u"], c1=c1, skip=o["flag"])
            ok = o["flag"] == 0
            acc = int(((d <= eps) & ok).sum())
            acc_rate.append(acc / max(int(ok.sum()), 1))
            s = O.mcmc_adapt(s, k, acc, int(ok.sum()))
        ends.append(s)
        first.append(np.mean(acc_rate[:10]))
        last.append(np.mean(acc_rate[-100:]))
    assert last[0] > A_T > last[1], last
    for f, l in zip(first, last):
        assert abs(l - A_T) < 0.06 and abs(l - A_T) < abs(f - A_T), (first, last)
    assert ends[0] < ends[1] < 2 * ends[0], ends


def _replay_generation(m, c, t, eps1, pop, ms):
    """Generation t of the MCMC baseline from the oracle's single steps."""
    N, M = c.N, c.M
    eps = O.kth(pop.d, O.rank(c.alpha, N))
    q, pre, tot = O.resample_prefix(pop.d, pop.W, eps, c.weight_mode)
    u_new, d_new, s_new = [], [], []
    window = O.mcmc_window(c)
    s, k, nb = ms
    b = 0
    while b < c.max_batches and len(d_new) < N:
        c1 = (t << 16) | b
        o = O.propose(m, pop.u, pre, tot, 0.0, 0, M, c1, s_fixed=float(np.float32(s)))
        d = O.simulate(m, o["u"], c1=c1, skip=o["flag"])
        ok = o["flag"] == 0
        acc = np.nonzero(ok & (d <= eps))[0]
        for j in acc[: N - len(d_new)]:
            u_new.append(o["u"][:, j])
            d_new.append(d[j])
            s_new.append(o["s"][j])
        if nb < window:
            s = O.mcmc_adapt(s, k, len(acc), int(ok.sum()))
            k += 1
        nb += 1
        b += 1
    return np.array(u_new).T, np.array(d_new), np.array(s_new, np.float32), (s, k, nb), eps


@pytest.mark.parametrize("adapt", [0, 3, 1000])
def test_generation_equals_its_single_steps(adapt):
    """or_generation in MCMC mode: the proposals walk with (float) s of the
    batch, s adapts after each batch inside the window, and the state
    (s, k, batches) crosses generations; a replay from or_propose,
    or_simulate and or_mcmc_adapt must give the same populations and state
    bit for bit (windows closed from the start, closing mid-run, open)."""
    m, _, _ = _toy(2)
    c = O.make_smc(300, M=200, beta_mode=O.MCMC_MODE, max_batches=200, mcmc_s0=0.02,
                   mcmc_adapt=adapt, max_total=0 if adapt == 0 else 10**6, nthreads=4)
    pop = O.generation0(m, c)
    ms = O.mcmc_start(c)
    assert (ms.s, ms.k, ms.batches) == (float(np.float32(0.02)), 0, 0)
    state = (ms.s, ms.k, ms.batches)
    eps1 = 0.0
    for t in range(1, 5):
        u, d, s, state, eps = _replay_generation(m, c, t, eps1, pop, state)
        s_start = ms.s
        new, st = O.generation(m, c, t, eps1, pop, ms)
        assert st.status == 0
        assert (ms.s, ms.k, ms.batches) == state
        assert st.beta_a == np.float32(s_start) and st.mcmc_s == np.float32(ms.s)
        assert st.eps == eps
        assert np.array_equal(new.u, u) and np.array_equal(new.d, d)
        assert np.array_equal(new.s, s)
        if adapt == 0:
            assert np.all(new.s == np.float32(0.02))
        eps1 = st.eps1
        pop = new
    if adapt == 3:
        assert ms.k == 3  # the first three batches of generation 1
    if adapt == 1000:
        assert ms.k == ms.batches


def test_mcmc_generation_needs_its_state():
    m, _, _ = _toy(1)
    c = O.make_smc(64, beta_mode=O.MCMC_MODE, nthreads=1)
    pop = O.generation0(m, c)
    with pytest.raises(ValueError):
        O.generation(m, c, 1, 0.0, pop)


def test_gaussian_toy_closed_form_posterior_mcmc_step():
    """The conjugate toy of test_oracle_smc (x ~ N(theta, I8), flat box
    prior, x_obs = 0; ABC posterior at eps: mean 0, variance 1 + eps^2/10 per
    coordinate), reached with the baseline's single step (started at
    s0 = 4e-3, adapted over its first 5 batches) and importance weights whose
    kernel variance is each particle's own step: over 10 runs the weighted
    mean and the variance ratio lie within 2 Monte-Carlo standard errors of
    0 and 1."""
    means, ratios = [], []
    for seed in range(1, 11):
        m, lo, hi = _toy(seed)
        c = O.make_smc(2048, beta_mode=O.MCMC_MODE, weight_mode=1, max_batches=400,
                       mcmc_s0=4e-3, mcmc_adapt=5, max_total=10**6, nthreads=4)
        pop, stats = O.run(m, c, 10)
        assert all(s.status == 0 for s in stats)
        assert len({float(s.beta_a) for s in stats}) > 1  # the step adapted
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
