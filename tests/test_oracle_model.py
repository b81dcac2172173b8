"""Pins of the oracle's simulator (Sec. 2.2): compartment conservation,
brute-force enumeration of exact trajectory probabilities at tiny population
and horizon, the deterministic mean-field limit at large population, the
paper's floor-normal flow law, and the Gaussian toy's distance law."""
import itertools
import math

import numpy as np
import pytest
import scipy.stats as st

import oracle as O

THETA_MAX = O.SAIRD_THETA_MAX.astype(np.float64)


def _u_of(theta):
    return (np.asarray(theta, np.float64) / THETA_MAX).astype(np.float32)


def _theta_of(u):
    return (u.astype(np.float32) * O.SAIRD_THETA_MAX).astype(np.float32)


def test_conservation_and_nonnegativity():
    """S+I+A+R+D+Ru = P and every compartment >= 0 on every day (Sec. 2.2)."""
    for sampler in (0, 1):
        m = O.OracleModel(T=40, P=50000, A0=200, R0=30, D0=4, seed=5, sampler=sampler)
        u = O.prior(m, 2000)
        _, tr = O.simulate(m, u, traj=True)
        assert np.all(tr >= 0)
        tot = tr.astype(np.int64).sum(axis=1)
        assert np.all(tot == 50000)
        # R and D never decrease (they only receive flows)
        assert np.all(np.diff(tr[:, 3, :], axis=0) >= 0)
        assert np.all(np.diff(tr[:, 4, :], axis=0) >= 0)


def _exact_step(state, th, P):
    """Exact law of one day under binomial competing risks, fp64 (Eq. 4-5)."""
    S, I, A, R, D, Ru = state
    a0, al, n, be, ga, de, et, ka = [float(v) for v in th]
    x = A + R + D
    xn = (0.0 if n > 0 else 1.0) if x == 0 else x ** n
    g = a0 + al / (1.0 + xn)
    pSI = -math.expm1(-np.float32(np.float32(g) * np.float32(I)) / np.float32(P))
    lamI, lamA = ga + be * et, be + de
    pI, pA = -math.expm1(-lamI), -math.expm1(-lamA)
    fI, fA = ga / lamI, be / lamA
    out = {}
    for k1 in range(S + 1):
        p1 = st.binom.pmf(k1, S, pSI)
        for LI in range(I + 1):
            p2 = p1 * st.binom.pmf(LI, I, pI)
            for k2 in range(LI + 1):
                p3 = p2 * st.binom.pmf(k2, LI, fI)
                for LA in range(A + 1):
                    p4 = p3 * st.binom.pmf(LA, A, pA)
                    for k3 in range(LA + 1):
                        p5 = p4 * st.binom.pmf(k3, LA, fA)
                        nxt = (S - k1, I + k1 - LI, A + k2 - LA, R + k3, D + LA - k3,
                               Ru + LI - k2)
                        out[nxt] = out.get(nxt, 0.0) + p5
    return out


def test_brute_force_enumeration_tiny_population():
    """Exact probabilities of every 2-day trajectory at P = 6 (products of
    binomial pmfs) against 300k oracle trajectories: G-test."""
    P, T = 6, 2
    theta = np.array([0.5, 20.0, 1.0, 0.3, 0.4, 0.1, 0.5, 1.5])
    u = _u_of(theta)
    th = _theta_of(u)
    m = O.OracleModel(T=T, P=P, A0=1, R0=0, D0=0, seed=11)
    nsamp = 300000
    U = np.repeat(u[:, None], nsamp, axis=1)
    _, tr = O.simulate(m, U, traj=True, nthreads=4)
    I0 = int(math.floor(np.float32(th[7]) * np.float32(1)))
    s0 = (P - 1 - I0, I0, 1, 0, 0, 0)
    assert tuple(tr[0, :, 0]) == s0
    exact = {}
    for s1, p1 in _exact_step(s0, th, P).items():
        for s2, p2 in _exact_step(s1, th, P).items():
            exact[(s1, s2)] = exact.get((s1, s2), 0.0) + p1 * p2
    assert abs(sum(exact.values()) - 1) < 1e-9
    keys = list(exact)
    index = {k: i for i, k in enumerate(keys)}
    counts = np.zeros(len(keys))
    for j in range(nsamp):
        k = (tuple(int(v) for v in tr[1, :, j]), tuple(int(v) for v in tr[2, :, j]))
        assert k in index, k  # never an impossible trajectory
        counts[index[k]] += 1
    e = np.array([exact[k] for k in keys]) * nsamp
    big = e >= 5
    obs = np.append(counts[big], counts[~big].sum())
    exp = np.append(e[big], e[~big].sum())
    mask = exp > 0
    g = 2 * np.sum(np.where(obs[mask] > 0, obs[mask] * np.log(obs[mask] / exp[mask]), 0))
    dof = mask.sum() - 1
    assert st.chi2.sf(g, dof) > 1e-3, (g, dof)


def test_mean_field_limit_large_population():
    """At P = 1e9 (A0 = 1e5) the ensemble mean of 64 trajectories follows the
    deterministic recurrence with flows n p (normal branch of the sampler).
    Individual paths carry early Poisson noise that the epidemic's growth
    amplifies (about 0.5% at day 30), so the ensemble mean is compared: its
    standard error is about 6e-4, a wrong flow or split is off by far more."""
    P, T, K = 10**9, 30, 64
    theta = np.array([0.35, 40.0, 0.8, 0.05, 0.2, 0.01, 0.4, 1.2])
    u = _u_of(theta)
    th = _theta_of(u).astype(np.float64)
    m = O.OracleModel(T=T, P=P, A0=100000, R0=0, D0=0, seed=3)
    _, tr = O.simulate(m, np.repeat(u[:, None], K, axis=1), traj=True, nthreads=4)
    a0, al, n, be, ga, de, et, ka = th
    I0 = math.floor(np.float32(ka) * np.float32(100000))
    S, I, A, R, D, Ru = P - 100000 - I0, I0, 1e5, 0.0, 0.0, 0.0
    lamI, lamA = ga + be * et, be + de
    pI, pA = -math.expm1(-lamI), -math.expm1(-lamA)
    for day in range(1, T + 1):
        g = a0 + al / (1 + (A + R + D) ** n)
        pSI = -math.expm1(-g * I / P)
        k1, LI, LA = S * pSI, I * pI, A * pA
        S, I, A = S - k1, I + k1 - LI, A + LI * ga / lamI - LA
        R, D, Ru = R + LA * be / lamA, D + LA * de / lamA, Ru + LI * be * et / lamI
        mf = np.array([S, I, A, R, D, Ru])
        sim = tr[day].astype(np.float64)
        big = mf > 1e5
        rel = (sim[big] - mf[big, None]) / mf[big, None]
        assert np.all(np.abs(rel.mean(axis=1)) < 3e-3), (day, rel.mean(axis=1))
        assert np.all(np.abs(rel) < 3e-2), day


def test_paper_mode_first_flow_law():
    """Paper mode (Sec. 2.2): k1 = floor(N(h, sd sqrt h)) clamped to [0, S];
    the first day's S->I flow is compared with the exact Phi differences."""
    P, T = 100000, 1
    theta = np.array([0.5, 20.0, 1.0, 0.3, 0.4, 0.1, 0.5, 1.5])
    u = _u_of(theta)
    th = _theta_of(u).astype(np.float64)
    m = O.OracleModel(T=T, P=P, A0=50, R0=0, D0=0, seed=2, sampler=1)
    nsamp = 100000
    _, tr = O.simulate(m, np.repeat(u[:, None], nsamp, axis=1), traj=True, nthreads=4)
    S0, I0 = int(tr[0, 0, 0]), int(tr[0, 1, 0])
    k1 = S0 - tr[1, 0, :].astype(np.int64)
    g = th[0] + th[1] / (1 + 50 ** th[2])
    h = g * S0 * (I0 / P)
    ks = np.arange(int(h - 8 * math.sqrt(h)) - 1, int(h + 8 * math.sqrt(h)) + 2)
    ks = ks[ks >= 0]
    pk = st.norm.cdf((ks + 1 - h) / math.sqrt(h)) - st.norm.cdf((ks - h) / math.sqrt(h))
    pk[0] += st.norm.cdf((ks[0] - h) / math.sqrt(h))
    obs = np.array([(k1 == k).sum() for k in ks], float)
    exp = pk * nsamp
    big = exp > 5
    chi = ((obs[big] - exp[big]) ** 2 / exp[big]).sum()
    assert st.chi2.sf(chi, big.sum() - 1) > 1e-3


def test_gaussian_toy_distance_law():
    """Toy model: ||theta + z - x_obs||^2 is noncentral chi^2_8."""
    lo, hi = np.full(8, -10, np.float32), np.full(8, 10, np.float32)
    m = O.OracleModel(model=1, T=0, P=1, theta_lo=lo, theta_hi=hi, seed=4)
    theta = np.array([1.0, -0.5, 0.3, 2.0, 0.0, -1.5, 0.7, 0.2])
    u = ((theta - lo) / (hi - lo)).astype(np.float32)
    th = (lo + u * (hi - lo)).astype(np.float64)
    d = O.simulate(m, np.repeat(u[:, None], 20000, axis=1))
    lam = float((th ** 2).sum())
    assert st.kstest(d ** 2, st.ncx2(8, lam).cdf).pvalue > 1e-3


def test_resimulation_by_counter_index_is_identical():
    """A particle's trajectory depends only on its counters: re-simulating a
    sample of slots by c0 index reproduces the batch distances bit for bit."""
    m = O.OracleModel(T=30, P=100000, A0=10, seed=9)
    obs, _, _ = O.synth_obs(O.OracleModel(T=30, P=100000, A0=10, seed=9))
    m.set_obs(obs)
    u = O.prior(m, 1000)
    d = O.simulate(m, u, c1=(3 << 16) | 2)
    idx = np.array([5, 17, 999, 0, 500], np.uint32)
    d2 = O.simulate(m, u[:, idx], c1=(3 << 16) | 2, c0_idx=idx)
    assert np.array_equal(d[idx], d2)


def test_synthetic_observations():
    """A0 = max(10, round(1e-4 P)), R0 = D0 = 0; theta* in the sub-box; the
    epidemic grows (A_T > A0); deterministic in the seed."""
    for P, T, seed in ((100000, 60, 1), (10**7, 120, 2)):
        A0 = max(10, round(1e-4 * P))
        m = O.OracleModel(T=T, P=P, A0=A0, seed=seed)
        obs, th, att = O.synth_obs(m)
        assert att >= 1
        assert tuple(obs[:, 0]) == (A0, 0, 0)
        assert obs[0, T] > A0
        assert np.all(th >= O.OBS_BOX_LO) and np.all(th <= O.OBS_BOX_HI)
        obs2, th2, _ = O.synth_obs(O.OracleModel(T=T, P=P, A0=A0, seed=seed))
        assert np.array_equal(obs, obs2) and np.array_equal(th, th2)
        assert np.all(np.diff(obs[1]) >= 0) and np.all(np.diff(obs[2]) >= 0)
