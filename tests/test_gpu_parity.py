"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer, index and random-number work is compared bit for bit: Philox
blocks, prior draws, trajectories, distances (exact integer sums, one
correctly rounded conversion and sqrt), order statistics, quantised weights
and prefixes, ancestors, Beta steps, walks and whole populations.  The FP32
weight path is compared with the fp64 oracle within the tolerance derived in
test_weights_fp32_vs_oracle.  Sizes span several tiles with ragged tails;
the 2^20-particle, 120-day, P = 1e7 workload is checked on sampled outputs.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import paper_2106_15508_gb300 as G
from paper_2106_15508_gb300 import build as B
from paper_2106_15508_gb300 import workloads as WL

import inputs as IN
from helpers import (get_population, oracle_model, oracle_obs, oracle_smc, saird_config,
                     state_blob)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REPORT = {}


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    G.lib()
    yield
    out = os.environ.get("ABC_PARITY_REPORT")
    if out:
        with open(out, "w") as f:
            json.dump(REPORT, f, indent=1, default=float)


_VIEW = {np.dtype(np.uint32): np.int32, np.dtype(np.uint64): np.int64}


def dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype in _VIEW:
        a = a.view(_VIEW[a.dtype])
    return torch.from_numpy(a).cuda()


def host(t, dtype=None):
    torch.cuda.synchronize()
    a = t.cpu().numpy()
    return a.view(dtype) if dtype is not None else a


def empty(shape, dtype):
    return torch.empty(shape, dtype=dtype, device="cuda")


def scratch(nbytes):
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device="cuda")


# ------------------------------------------------------------- RNG, prior ---
def test_philox_blocks_bitexact():
    ctr = IN.counters(4099, 1)
    for key in ((0, 0), (0x12345678, 0x9ABCDEF0)):
        out = empty((4099, 4), torch.int32)
        G.abc_philox(dev(ctr), key[0], key[1], 4099, out)
        got = host(out, np.uint32)
        for i in range(0, 4099, 37):
            assert np.array_equal(got[i], O.philox(ctr[i], key)), i


@pytest.mark.parametrize("n", [1, 1000, 4097])
def test_prior_bitexact(n):
    cfg = saird_config(n, 60, 100000, seed=3, run_id=5)
    u = empty((8, n), torch.float32)
    G.abc_prior(cfg, n, u)
    assert np.array_equal(host(u).view(np.uint32), O.prior(oracle_model(cfg), n).view(np.uint32))


@pytest.mark.parametrize("P,T,seed", [(100_000, 60, 1), (10_000_000, 120, 2), (10**6, 180, 9)])
def test_synthetic_observations_bitexact(P, T, seed):
    cfg = saird_config(16, T, P, seed=seed)
    obs = empty((3, T + 1), torch.int32)
    th = empty(8, torch.float32)
    att = empty(1, torch.int32)
    G.abc_synth_obs(cfg, WL.OBS_BOX_LO, WL.OBS_BOX_HI, obs, th, att)
    o_obs, o_th, o_att = oracle_obs(cfg)
    assert np.array_equal(host(obs), o_obs)
    assert np.array_equal(host(th).view(np.uint32), o_th.view(np.uint32))
    assert int(host(att)[0]) == o_att


# --------------------------------------------------------------- simulator -
def _sim_gpu(cfg, obs, u, c1=0, c0_idx=None, skip=None, traj=False, tag=G.TAG_SIM):
    n = u.shape[1]
    d = empty(n, torch.float64)
    T = cfg.n_days
    tr = empty((T + 1, 6, n), torch.int32) if traj else None
    G.abc_simulate(cfg, None if obs is None else dev(obs), dev(u), n,
                   None if c0_idx is None else dev(c0_idx), c1, tag,
                   None if skip is None else dev(skip), d, tr)
    return (host(d), host(tr)) if traj else host(d)


@pytest.mark.parametrize("sampler", [G.ABC_SIM_BINOMIAL, G.ABC_SIM_PAPER_NORMAL])
def test_simulate_trajectories_bitexact_4096_particles(sampler):
    """N = 4096, P = 1e5, 60 days: every compartment of every day and every
    distance identical to the oracle, for prior draws and clustered draws."""
    cfg = saird_config(4096, 60, 100_000, seed=1, sampler=sampler)
    obs, _, _ = oracle_obs(cfg)
    m = oracle_model(cfg, obs)
    for u, c1 in ((O.prior(m, 4096), 0), (IN.clustered_particles(4096, 5, 0.3, 0.1), (2 << 16) | 3)):
        d, tr = _sim_gpu(cfg, obs, u, c1=c1, traj=True)
        od, otr = O.simulate(m, u, c1=c1, traj=True, nthreads=8)
        assert np.array_equal(tr, otr)
        assert np.array_equal(d.view(np.uint64), od.view(np.uint64))
        tot = tr.astype(np.int64).sum(axis=1)
        assert np.all(tot == cfg.population) and np.all(tr >= 0)


@pytest.mark.parametrize("n", [1, 33, 4097])
def test_simulate_ragged_skip_and_counter_index(n):
    cfg = saird_config(n, 30, 50_000, seed=4)
    obs, _, _ = oracle_obs(cfg)
    m = oracle_model(cfg, obs)
    u = IN.unit_particles(n, 11)
    skip = (IN.rng(3).random(n) < 0.2).astype(np.uint8)
    c0 = IN.rng(4).integers(0, 2**32, n, dtype=np.uint64).astype(np.uint32)
    d = _sim_gpu(cfg, obs, u, c1=77, c0_idx=c0, skip=skip)
    od = O.simulate(m, u, c1=77, c0_idx=c0, skip=skip)
    assert np.array_equal(d.view(np.uint64), od.view(np.uint64))
    assert np.all(np.isinf(d[skip == 1]))


@pytest.mark.parametrize("kind", ["negative", "extreme"])
def test_simulate_distance_with_unusual_observations(kind):
    """The day's three squared errors go into the 128-bit distance with one
    carry when every observation is a count (non-negative); a series with
    negative entries takes the three-carry path.  Both must equal the
    oracle's exact integer sum: negative entries down to INT32_MIN (squares
    up to 2^64 - 2^33 + 1), and counts up to INT32_MAX (the one-carry path
    at its bound: three squares near 2^62 per day)."""
    cfg = saird_config(4097, 40, 100_000, seed=12)
    obs, _, _ = oracle_obs(cfg)
    obs = obs.copy()
    r = IN.rng(13)
    if kind == "negative":
        obs[:, 1::3] = -obs[:, 1::3]
        obs[0, 5] = np.iinfo(np.int32).min
        obs[2, 7] = -1
    else:
        obs[:, 2::4] = np.iinfo(np.int32).max
        obs[1, 3::5] = r.integers(2**30, 2**31 - 1, obs[1, 3::5].shape)
    m = oracle_model(cfg, obs)
    u = IN.unit_particles(4097, 14)
    d = _sim_gpu(cfg, obs, u, c1=5)
    od = O.simulate(m, u, c1=5, nthreads=8)
    assert np.array_equal(d.view(np.uint64), od.view(np.uint64))


def test_simulate_gaussian_toy_bitexact():
    lo, hi = [-10.0] * 8, [10.0] * 8
    cfg = G.config(model=G.ABC_MODEL_GAUSS_TOY, n_days=1, population=1, init_ard=[0, 0, 0],
                   theta_lo=lo, theta_hi=hi, x_obs=[0.5] * 8, seed=6, n_particles=1000)
    u = IN.unit_particles(3000, 2)
    d = _sim_gpu(cfg, None, u, c1=9)
    od = O.simulate(oracle_model(cfg), u, c1=9)
    assert np.array_equal(d.view(np.uint64), od.view(np.uint64))


def test_simulate_full_size_sampled():
    """2^20 particles, 120 days, P = 1e7 (the large single-run workload) in
    the launch the context uses; 2048 sampled particles re-simulated by the
    oracle through their counters must match bit for bit."""
    w = WL.LARGE
    cfg = w.config()
    obs, _, _ = oracle_obs(cfg)
    n = w.N
    u = empty((8, n), torch.float32)
    G.abc_prior(cfg, n, u)
    d = empty(n, torch.float64)
    c1 = (5 << 16) | 1
    G.abc_simulate(cfg, dev(obs), u, n, None, c1, G.TAG_SIM, None, d, None)
    uh, dh = host(u), host(d)
    idx = np.sort(IN.rng(7).choice(n, 2048, replace=False)).astype(np.uint32)
    m = oracle_model(cfg, obs)
    assert np.array_equal(uh[:, idx].view(np.uint32), O.prior(m, n)[:, idx].view(np.uint32))
    od = O.simulate(m, uh[:, idx], c1=c1, c0_idx=idx, nthreads=8)
    assert np.array_equal(dh[idx].view(np.uint64), od.view(np.uint64))
    REPORT["full_size_sim_median_dist"] = float(np.median(dh))


# ------------------------------------------------------------- select ------
@pytest.mark.parametrize("n,alpha,ties,inf", [(1, 0.5, False, False), (4097, 0.5, True, False),
                                              (100_003, 0.1, False, True),
                                              ((1 << 20) + 17, 0.5, False, False)])
def test_select_kth_matches_oracle(n, alpha, ties, inf):
    d = IN.distances(n, n, ties=ties, with_inf=inf)
    k = O.rank(alpha, n)
    out = empty(1, torch.float64)
    sc = scratch(G.abc_select_scratch_bytes(n))
    G.abc_select_kth(dev(d), n, k, out, sc, sc.numel())
    assert host(out)[0] == O.kth(d, k)


# ------------------------------------------------------- weights + prefix --
@pytest.mark.parametrize("n", [4096 + 1000, 1 << 20])
@pytest.mark.parametrize("mode", [G.ABC_W_PAPER, G.ABC_W_IMPORTANCE])
def test_resample_prefix_bitexact(n, mode):
    d = IN.distances(n, 1, ties=True)
    W = IN.weights(n, 2)
    eps = O.kth(d, O.rank(0.5, n))
    q = empty(n, torch.int32)
    pre = empty(n, torch.int64)
    sc = scratch(G.abc_prefix_scratch_bytes(n))
    G.abc_resample_prefix(dev(d), dev(W), n, dev(np.array([eps])), mode, q, pre, sc, sc.numel())
    oq, opre, otot = O.resample_prefix(d, W, eps, mode)
    assert np.array_equal(host(q, np.uint32), oq)
    assert np.array_equal(host(pre, np.uint64), opre)


@pytest.mark.parametrize("n", [4099, 100_003])
def test_resample_prefix_unaligned_outputs(n):
    """q and prefix at 4- and 8-byte offsets (not 16-byte aligned): the scan
    takes its element-wise path and the result is the same."""
    d = IN.distances(n, 3, ties=True)
    W = IN.weights(n, 4)
    eps = O.kth(d, O.rank(0.5, n))
    qb = empty(n + 1, torch.int32)
    pb = empty(n + 1, torch.int64)
    q, pre = qb[1:], pb[1:]
    sc = scratch(G.abc_prefix_scratch_bytes(n))
    G.abc_resample_prefix(dev(d), dev(W), n, dev(np.array([eps])), G.ABC_W_IMPORTANCE, q, pre,
                          sc, sc.numel())
    oq, opre, _ = O.resample_prefix(d, W, eps, 1)
    assert np.array_equal(host(q, np.uint32), oq)
    assert np.array_equal(host(pre, np.uint64), opre)


def test_resample_prefix_degenerate():
    n = 3000
    d = np.full(n, 7.0)
    d[::3] = 9.0
    q = empty(n, torch.int32)
    pre = empty(n, torch.int64)
    sc = scratch(G.abc_prefix_scratch_bytes(n))
    G.abc_resample_prefix(dev(d), None, n, dev(np.array([7.0])), G.ABC_W_PAPER, q, pre, sc,
                          sc.numel())
    oq, opre, _ = O.resample_prefix(d, None, 7.0, 0)
    assert np.array_equal(host(q, np.uint32), oq) and oq.sum() == np.sum(d <= 7.0)
    assert np.array_equal(host(pre, np.uint64), opre)


# ------------------------------------------------------------- propose -----
@pytest.mark.parametrize("mode,a,b,eps,eps1", [(G.ABC_BETA_FIXED, 2.0, 5, 0, 0),
                                               (G.ABC_BETA_PAPER, 0.0, 2, 4.0, 4.0),
                                               (G.ABC_BETA_PAPER, 0.0, 14, 2.0, 4.0),
                                               (G.ABC_BETA_FIXED, 0.1, 15, 0, 0)])
def test_propose_bitexact(mode, a, b, eps, eps1):
    n, slots = 3000, 5003
    cfg = saird_config(n, 10, 1000, seed=8, beta_mode=mode, beta_a=a or 2.0, beta_b=b)
    m = oracle_model(cfg)
    u = IN.clustered_particles(n, 3, 0.5, 0.2)
    q = IN.quantised_weights(n, 4)
    pre = np.cumsum(q.astype(np.uint64))
    c1 = (3 << 16) | 2
    outs = dict(u=empty((8, slots), torch.float32), s=empty(slots, torch.float32),
                anc=empty(slots, torch.int32), att=empty(slots, torch.int32),
                flag=empty(slots, torch.uint8))
    G.abc_propose(cfg, dev(u), n, dev(pre), dev(np.array([eps])), dev(np.array([eps1])),
                  a, b, slots, None, c1, outs["u"], outs["s"], outs["anc"], outs["att"],
                  outs["flag"])
    a_t = np.float32(eps / eps1) if mode == G.ABC_BETA_PAPER else np.float32(a)
    o = O.propose(m, u, pre, int(pre[-1]), float(a_t), b, slots, c1, nthreads=8)
    assert np.array_equal(host(outs["anc"]), o["anc"])
    assert np.array_equal(host(outs["s"]).view(np.uint32), o["s"].view(np.uint32))
    assert np.array_equal(host(outs["u"]).view(np.uint32), o["u"].view(np.uint32))
    assert np.array_equal(host(outs["att"]), o["attempts"])
    assert np.array_equal(host(outs["flag"]), o["flag"])


def test_propose_redraw_exhaustion_bitexact():
    n, slots = 64, 3000
    cfg = saird_config(n, 10, 1000, seed=9, beta_mode=G.ABC_BETA_FIXED, beta_a=5.0, beta_b=1,
                       max_redraw=2)
    u = np.full((8, n), 0.999, np.float32)
    pre = np.arange(1, n + 1, dtype=np.uint64)
    c0 = IN.rng(1).integers(0, 2**32, slots, dtype=np.uint64).astype(np.uint32)
    outs = [empty((8, slots), torch.float32), empty(slots, torch.float32),
            empty(slots, torch.int32), empty(slots, torch.int32), empty(slots, torch.uint8)]
    G.abc_propose(cfg, dev(u), n, dev(pre), None, None, 5.0, 1, slots, dev(c0), 65537, *outs)
    o = O.propose(oracle_model(cfg), u, pre, n, 5.0, 1, slots, 65537, max_redraw=2, c0_idx=c0)
    assert host(outs[4]).sum() > 0
    assert np.array_equal(host(outs[4]), o["flag"])
    assert np.array_equal(host(outs[0]).view(np.uint32), o["u"].view(np.uint32))


# --------------------------------------------------------------- accept ----
@pytest.mark.parametrize("M,N,filled0", [(5000, 1000, 0), (5000, 4000, 3500), (777, 10_000, 12)])
def test_accept_append_in_slot_order(M, N, filled0):
    r = IN.rng(M + N)
    up = r.random((8, M)).astype(np.float32)
    dp = r.gamma(2.0, 10.0, M)
    sp = r.random(M).astype(np.float32)
    ap = r.integers(0, 100, M).astype(np.int32)
    fl = (r.random(M) < 0.1).astype(np.uint8)
    eps = float(np.median(dp))
    pop = [empty((8, N), torch.float32), empty(N, torch.float64), empty(N, torch.float32),
           empty(N, torch.int32)]
    for t in pop:
        t.zero_()
    filled = dev(np.array([filled0], np.int64))
    counters = dev(np.array([0, 0], np.int64))
    sc = scratch(G.abc_accept_scratch_bytes(M))
    G.abc_accept_append(dev(up), dev(dp), dev(sp), dev(ap), dev(fl), M, dev(np.array([eps])), N,
                        *pop, filled, counters, sc, sc.numel())
    acc = np.where((fl == 0) & (dp <= eps))[0]
    take = acc[: max(0, N - filled0)]
    sl = slice(filled0, filled0 + len(take))
    assert int(host(filled)[0]) == min(N, filled0 + len(acc))
    assert list(host(counters)) == [len(acc), int(fl.sum())]
    assert np.array_equal(host(pop[0])[:, sl], up[:, take])
    assert np.array_equal(host(pop[1])[sl], dp[take])
    assert np.array_equal(host(pop[3])[sl], ap[take])


# ------------------------------------------------------------ weights ------
def _weights_gpu(up, s, u, q):
    rows, n = up.shape[1], u.shape[1]
    pre = np.cumsum(q.astype(np.uint64))
    lw = empty(rows, torch.float64)
    sc = scratch(G.abc_weights_scratch_bytes(rows, n))
    G.abc_weights(dev(up), dev(s), rows, dev(u), dev(q), dev(pre), n, G.ABC_P_FP32, lw, sc,
                  sc.numel())
    return host(lw), int(pre[-1])


def logw_tolerance_direct_fp32(s, olw):
    """Bound on |log W - log W_fp64| for rows evaluated directly in fp32 (the
    tensor-core precision's recomputed rows).

    With a = 4 ln(2 pi s) and LSE = a - log W (natural log) the per-column
    exponent e = c_k - D log2(e)/(2 s) carries at most ~10 ulp of the
    magnitudes involved (fp32 differences: 1, squares and sums in two fp32x2
    lanes of four terms plus the final add: 5, the scale 1/(2s): 2, the fused
    product-add: 1, rounding of c_k: 1), i.e. <= 10 * 2^-24 * (|LSE| + |a|)
    after the ln 2 < 1 change of base, with a factor 1.6 margin; summing
    2^(e - m) (ex2.approx, ~2 ulp per term) in fp32 tiles of 128 terms plus a
    Kahan fold adds <= 132 * 2^-24 relative to the row sum, i.e. absolute in
    log W; the fp64 combine adds ~1e-15.  Together:
        |d log W| <= 2^-24 (16 (|LSE| + |a|) + 160)."""
    s_eff = np.maximum(np.asarray(s, np.float32), np.float32(1e-30)).astype(np.float64)
    a = 4.0 * np.log(2.0 * np.pi * s_eff)
    lse = a - olw
    return 2.0**-24 * (16.0 * (np.abs(lse) + np.abs(a)) + 160.0)


def logw_tolerance(s, olw):
    """Bound on |log W_fp32 - log W_fp64| for the FP32 precision.

    Every term within 40 bits of the row maximum has its exponent evaluated
    in double-float arithmetic (exact differences and squares, error-free
    product and sum): its error is a few 2^-44 of |e|, and 2^-24 |e| for
    terms with |e| >= 2^22, which keep their fp32 part only.  Each such term
    is then exponentiated by ex2.approx (relative error <= 2^-22) and added
    in a Kahan sum (<= 2 * 2^-24); the terms below the threshold, each under
    2^-40 of the maximum, sum to at most n 2^-40 of it, so even an fp32
    exponent error on all of them stays below 2^-24 for n <= 2^20 and
    |e| < 2^21.  The fp64 combine adds ~1e-15.  So, in natural-log units
    (ln 2 < 1):
        |d log W| <= 2^-21 + 2^-23 |LSE| [|LSE| >= 2^21 ln 2]
    with LSE = 4 ln(2 pi s) - log W.  Besides this bound the test asserts the
    1e-6 relative bar max |d log W| / max(|log W|, 1) <= 1e-6."""
    s_eff = np.maximum(np.asarray(s, np.float32), np.float32(1e-30)).astype(np.float64)
    lse = np.abs(4.0 * np.log(2.0 * np.pi * s_eff) - olw)
    return 2.0**-21 + np.where(lse >= 2.0**21 * math.log(2.0), 2.0**-23 * lse, 0.0)


REL_BAR = 1e-6  # FP32 weights against the fp64 oracle, relative on log W


def _compare_logw(lw, olw, s, name):
    assert np.all(np.isfinite(lw)) and np.all(np.isfinite(olw))
    err = np.abs(lw - olw)
    tol = logw_tolerance(s, olw)
    rel = err / np.maximum(np.abs(olw), 1.0)
    REPORT[name] = dict(max_abs=float(err.max()), median_abs=float(np.median(err)),
                        max_rel=float(rel.max()), max_err_over_tol=float((err / tol).max()),
                        rows=int(len(err)))
    print(name, REPORT[name])
    assert np.all(err <= tol), REPORT[name]
    assert rel.max() <= REL_BAR, REPORT[name]
    return err


@pytest.mark.parametrize("rows,n", [(4096, 4096), (777, 5003), (1, 300)])
def test_weights_fp32_vs_oracle(rows, n):
    up = IN.clustered_particles(rows, rows, 0.5, 0.15)
    u = IN.clustered_particles(n, n + 1, 0.5, 0.15)
    s = IN.step_sizes(rows, 3, 1e-4, 0.3)
    if rows > 10:
        s[::97] = 0.0        # floored to 1e-30 on both sides
        s[1::97] = 1e-40     # subnormal step: no overflow, no NaN
        up[:, 1::97] = u[:, 5][:, None]  # exactly on a column
    q = IN.quantised_weights(n, 5)
    lw, tot = _weights_gpu(up, s, u, q)
    olw = O.weights(up, s, u, q, tot, nthreads=8)
    _compare_logw(lw, olw, s, "weights_fp32_%dx%d" % (rows, n))


def test_weights_fp32_full_size_sampled_rows():
    """2^20 rows x 2^20 columns (about half surviving): 48 sampled rows
    against the fp64 oracle over every column."""
    n = 1 << 20
    up = IN.clustered_particles(n, 21, 0.5, 0.1)
    u = IN.clustered_particles(n, 22, 0.5, 0.1)
    s = IN.step_sizes(n, 23, 1e-4, 0.05)
    q = IN.quantised_weights(n, 24, zero_frac=0.5)
    lw, tot = _weights_gpu(up, s, u, q)
    idx = np.sort(IN.rng(25).choice(n, 48, replace=False))
    olw = O.weights(up[:, idx], s[idx], u, q, tot, nthreads=8)
    _compare_logw(lw[idx], olw, s[idx], "weights_fp32_full_sampled")


def test_normalize_matches_oracle():
    for n, seed in ((1, 1), (4097, 2), (1 << 20, 3)):
        lw = IN.rng(seed).normal(-20, 15, n)
        lw[IN.rng(seed).random(n) < 0.01] = -np.inf
        W = empty(n, torch.float64)
        ess = empty(1, torch.float64)
        sc = scratch(G.abc_normalize_scratch_bytes(n))
        G.abc_normalize(dev(lw), n, W, ess, sc, sc.numel())
        oW, oess = O.normalize(lw)
        assert np.allclose(host(W), oW, rtol=1e-12, atol=0)
        assert abs(host(ess)[0] - oess) <= 1e-12 * oess
    W = empty(5, torch.float64)
    G.abc_normalize(dev(np.full(5, -np.inf)), 5, W, ess, sc, sc.numel())
    assert np.allclose(host(W), 0.2) and host(ess)[0] == 5
    lw = np.array([0.0, np.nan, -1.0, np.nan])
    W = empty(4, torch.float64)
    G.abc_normalize(dev(lw), 4, W, ess, sc, sc.numel())
    oW, oess = O.normalize(lw)
    assert np.allclose(host(W), oW, rtol=1e-12, atol=0) and oW[1] == 0.0


def test_normalize_exponentials_across_the_range():
    """The normalisation's table-driven exponential over log-weight gaps
    from 0 to -720 (-700 and below take the library exp), against the
    oracle's libm exp: the weights relative to the largest one (exp of the
    gap, free of the sum's rounding; gaps down to -690, whose weights stay
    clear of fp64's subnormal range) within 5e-14, the weights themselves
    within 1e-12 (the sums are added in different orders)."""
    n = (1 << 16) + 3
    r = IN.rng(77)
    lw = -720.0 * r.random(n)
    lw[0] = 0.0
    lw[1:50] = -r.random(49) * 1e-6      # tiny reductions
    lw[50:60] = -700.0 + r.random(10) * 1e-9  # at the switch
    W = empty(n, torch.float64)
    ess = empty(1, torch.float64)
    sc = scratch(G.abc_normalize_scratch_bytes(n))
    G.abc_normalize(dev(lw), n, W, ess, sc, sc.numel())
    oW, oess = O.normalize(lw)
    got = host(W)
    ok = lw >= -690.0  # weights / S far from fp64's subnormal range
    rel = np.abs(got[ok] / got[0] - np.exp(lw[ok])) / np.exp(lw[ok])
    REPORT["normalize_exp_max_rel"] = float(rel.max())
    assert rel.max() <= 5e-14, rel.max()
    assert np.allclose(got, oW, rtol=1e-12, atol=0)
    assert abs(host(ess)[0] - oess) <= 1e-12 * oess


# ---------------------------------------------------------- context --------
def _stats_match(g, o):
    assert g.eps == o.eps and g.eps1 == o.eps1
    assert g.batches == o.batches and g.accepted == o.accepted_total
    assert g.exhausted == o.exhausted and g.sims == o.sims - o.exhausted
    assert g.beta_b == o.beta_b and np.float32(g.beta_a) == np.float32(o.beta_a)


def test_context_paper_weights_bitexact_small_workload():
    """The 4096-particle, 60-day, P = 1e5 workload with Beta(2, 5) steps and
    the paper's weights (Eq. 10), 8 generations through abc_init /
    abc_generation: every generation's population and statistics equal the
    oracle's bit for bit."""
    w = WL.SMALL
    cfg = w.config(weight_mode=G.ABC_W_PAPER)
    obs, _, _ = oracle_obs(cfg)
    m, c = oracle_model(cfg, obs), oracle_smc(cfg)
    ctx = G.abc_init(cfg, obs)
    try:
        pop = O.generation0(m, c)
        G.abc_generation(ctx)
        gp = get_population(ctx, w.N)
        assert np.array_equal(gp["u"], pop.u) and np.array_equal(gp["d"], pop.d)
        eps1 = 0.0
        for t in range(1, w.G):
            new, st = O.generation(m, c, t, eps1, pop)
            rc = G.abc_generation(ctx)
            assert rc == st.status == 0
            gp = get_population(ctx, w.N)
            for k, ok in (("u", new.u), ("d", new.d), ("s", new.s), ("anc", new.anc)):
                assert np.array_equal(gp[k].view(np.uint8), np.ascontiguousarray(ok).view(np.uint8)), (t, k)
            _stats_match(G.abc_get_stats(ctx, t), st)
            eps1, pop = st.eps1, new
        REPORT["small_paper_eps"] = [G.abc_get_stats(ctx, t).eps for t in range(1, w.G)]
    finally:
        G.abc_free(ctx)


def test_context_importance_generation_from_oracle_state():
    """Importance weights: the oracle's population after generation t is
    loaded with abc_set_state; the CUDA generation t+1 then reproduces the
    oracle's proposals, distances and ancestors bit for bit and its weights
    within the FP32 tolerance."""
    cfg = saird_config(4096, 60, 100_000, seed=2, weight_mode=G.ABC_W_IMPORTANCE,
                       beta_mode=G.ABC_BETA_PAPER)
    obs, _, _ = oracle_obs(cfg)
    m, c = oracle_model(cfg, obs), oracle_smc(cfg)
    pop = O.generation0(m, c)
    eps1 = 0.0
    for t in range(1, 3):
        pop, st = O.generation(m, c, t, eps1, pop)
        eps1 = st.eps1
    new, st = O.generation(m, c, 3, eps1, pop)
    assert st.status == 0
    ctx = G.abc_init(cfg, obs)
    try:
        G.abc_set_state(ctx, state_blob(cfg, 3, eps1, pop))
        assert G.abc_generation(ctx) == 0
        gp = get_population(ctx, cfg.n_particles)
        for k, ok in (("u", new.u), ("d", new.d), ("s", new.s), ("anc", new.anc)):
            assert np.array_equal(gp[k].view(np.uint8), np.ascontiguousarray(ok).view(np.uint8)), k
        _stats_match(G.abc_get_stats(ctx, 3), st)
        # W_j = exp(log W_j - max) / sum: relative error <= twice the log W bound
        tol = 2 * logw_tolerance(new.s, new.logW)
        err = np.abs(gp["W"] - new.W)
        REPORT["ctx_importance_W_maxerr_rel_to_max"] = float(err.max() / new.W.max())
        assert np.all(err <= tol * new.W + 1e-15)
        g = G.abc_get_stats(ctx, 3)
        assert abs(g.ess - st.ess) <= 2 * tol.max() * st.ess
    finally:
        G.abc_free(ctx)


def test_checkpoint_resume_is_bit_identical():
    cfg = saird_config(2048, 40, 100_000, seed=5, weight_mode=G.ABC_W_IMPORTANCE)
    obs, _, _ = oracle_obs(cfg)
    a = G.abc_init(cfg, obs)
    b = G.abc_init(cfg, obs)
    try:
        G.abc_run(a, 3)
        blob = G.abc_get_state(a)
        G.abc_run(a, 5)
        G.abc_set_state(b, blob)
        assert G.abc_generations(b) == 3
        G.abc_run(b, 5)
        pa, pb = get_population(a, 2048), get_population(b, 2048)
        for k in pa:
            assert np.array_equal(pa[k].view(np.uint8), pb[k].view(np.uint8)), k
    finally:
        G.abc_free(a)
        G.abc_free(b)


@pytest.mark.parametrize("prec", [G.ABC_P_FP32, G.ABC_P_BF16_TC])
def test_reset_starts_a_new_run_equal_to_a_fresh_context(prec):
    """abc_reset(ctx, r) after a run: the next generations equal those of a
    fresh context whose config carries run_id r, bit for bit, statistics
    included."""
    cfg = saird_config(2048, 40, 100_000, seed=6, weight_mode=G.ABC_W_IMPORTANCE,
                       weight_prec=prec)
    obs, _, _ = oracle_obs(cfg)
    fresh_cfg = saird_config(2048, 40, 100_000, seed=6, weight_mode=G.ABC_W_IMPORTANCE,
                             weight_prec=prec, run_id=7)
    a = G.abc_init(cfg, obs)
    b = G.abc_init(fresh_cfg, obs)
    try:
        G.abc_run(a, 4)
        G.abc_reset(a, 7)
        assert G.abc_generations(a) == 0
        G.abc_run(a, 4)
        G.abc_run(b, 4)
        pa, pb = get_population(a, 2048), get_population(b, 2048)
        for k in pa:
            assert np.array_equal(pa[k].view(np.uint8), pb[k].view(np.uint8)), k
        for t in range(4):
            sa, sb = G.abc_get_stats(a, t), G.abc_get_stats(b, t)
            assert (sa.eps, sa.batches, sa.sims, sa.ess) == (sb.eps, sb.batches, sb.sims, sb.ess)
    finally:
        G.abc_free(a)
        G.abc_free(b)


def test_batch_budget_stop_keeps_population():
    """M < N with a budget of one batch cannot fill the population: the
    generation reports ABC_STOP_BUDGET and leaves the population unchanged."""
    cfg = saird_config(4096, 20, 100_000, seed=3, batch_size=512, max_batches=1)
    obs, _, _ = oracle_obs(cfg)
    ctx = G.abc_init(cfg, obs)
    try:
        G.abc_generation(ctx)
        before = get_population(ctx, 4096)
        assert G.abc_generation(ctx) == G.ABC_STOP_BUDGET
        assert G.abc_generations(ctx) == 1
        after = get_population(ctx, 4096)
        assert np.array_equal(before["u"], after["u"])
        assert G.abc_get_stats(ctx, 1).status == G.ABC_STOP_BUDGET
    finally:
        G.abc_free(ctx)


def test_errors_are_reported_not_faulted():
    n = 1000
    d = dev(IN.distances(n, 1))
    out = empty(1, torch.float64)
    small = scratch(8)
    with pytest.raises(G.AbcError) as e:
        G.abc_select_kth(d, n, 1, out, small, 8)
    assert e.value.code == -5
    with pytest.raises(G.AbcError):
        G.abc_select_kth(d, n, n + 1, out, scratch(1 << 16), 1 << 16)
    with pytest.raises(G.AbcError):
        G.abc_init(G.config(n_particles=-1), np.zeros((3, 121), np.int32))


def test_gaussian_toy_closed_form_on_gpu():
    """Ten independent importance-weighted GPU runs of the conjugate toy
    (seeds 1..10, 4096 particles, 10 generations, Beta(8, 1000) steps, FP32
    weights): per run the weighted mean and the weighted variance over
    v0 = 1 + eps^2/10 are averaged over the 8 exchangeable coordinates, and
    over the 10 runs they must lie within 2 Monte-Carlo standard errors (the
    runs' standard deviation / sqrt 10) of the closed form's 0 and 1."""
    means, ratios, ess = [], [], []
    for seed in range(1, 11):
        cfg = G.config(model=G.ABC_MODEL_GAUSS_TOY, n_days=1, population=1, init_ard=[0, 0, 0],
                       theta_lo=[-10.0] * 8, theta_hi=[10.0] * 8, seed=seed, n_particles=4096,
                       beta_mode=G.ABC_BETA_FIXED, beta_a=8.0, beta_b=1000,
                       weight_mode=G.ABC_W_IMPORTANCE, max_batches=400)
        ctx = G.abc_init(cfg, None)
        try:
            G.abc_run(ctx, 10)
            st = G.abc_get_stats(ctx, 9)
            p = get_population(ctx, 4096)
        finally:
            G.abc_free(ctx)
        th = -10 + 20 * p["u"].astype(np.float64)
        mean = (th * p["W"]).sum(1)
        var = (th**2 * p["W"]).sum(1) - mean**2
        means.append(mean.mean())
        ratios.append(var.mean() / (1 + st.eps**2 / 10))
        ess.append(st.ess)
    means, ratios = np.array(means), np.array(ratios)
    se_m = means.std(ddof=1) / math.sqrt(len(means))
    se_v = ratios.std(ddof=1) / math.sqrt(len(ratios))
    REPORT["toy_10_runs"] = dict(mean=float(means.mean()), se_mean=float(se_m),
                                 var_ratio=float(ratios.mean()), se_var_ratio=float(se_v),
                                 ess_median=float(np.median(ess)))
    assert abs(means.mean()) < 2 * se_m, (means, se_m)
    assert abs(ratios.mean() - 1) < 2 * se_v, (ratios, se_v)


@pytest.mark.parametrize("M,K", [(0, 1), (4096, 8)])
def test_context_ordered_simulation_bitexact(M, K):
    """Batches of at least 16384 slots are simulated in the order of the
    regime key (k_sim_order_key, a radix sort, k_simulate through the
    permutation): 32768 particles with one batch of N slots, and batches of
    4096 slots run 8 per round (32768 slots in one ordered launch); three
    generations and stage 0 equal the oracle bit for bit."""
    cfg = saird_config(32768, 40, 100_000, seed=12, weight_mode=G.ABC_W_PAPER, batch_size=M,
                       spec_batches=K, max_batches=400)
    obs, _, _ = oracle_obs(cfg)
    m, c = oracle_model(cfg, obs), oracle_smc(cfg)
    ctx = G.abc_init(cfg, obs)
    try:
        pop = O.generation0(m, c)
        G.abc_generation(ctx)
        gp = get_population(ctx, cfg.n_particles)
        assert np.array_equal(gp["d"].view(np.uint64), pop.d.view(np.uint64))
        eps1 = 0.0
        for t in range(1, 4):
            new, st = O.generation(m, c, t, eps1, pop)
            assert G.abc_generation(ctx) == st.status == 0
            gp = get_population(ctx, cfg.n_particles)
            for k, ok in (("u", new.u), ("d", new.d), ("s", new.s), ("anc", new.anc)):
                assert np.array_equal(gp[k].view(np.uint8),
                                      np.ascontiguousarray(ok).view(np.uint8)), (t, k)
            _stats_match(G.abc_get_stats(ctx, t), st)
            eps1, pop = st.eps1, new
    finally:
        G.abc_free(ctx)
