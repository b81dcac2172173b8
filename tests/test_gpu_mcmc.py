"""The MCMC baseline (ABC_STEP_MCMC; Sec. 2.4.1 Eq. 12-15, Sec. 3.1) on the
GPU against the oracle: proposals with the single step, the per-batch step
adaptation inside its window, whole runs through single contexts and graph
batches, and checkpoints that carry the step state -- bit for bit."""
import numpy as np
import pytest

import oracle as O
import paper_2106_15508_gb300 as G
from paper_2106_15508_gb300 import build as B

import inputs as IN
from helpers import get_population, oracle_model, oracle_obs, oracle_smc, saird_config

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    G.lib()


def _dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("s,slots,max_redraw", [(0.01, 5003, 64), (0.7, 3001, 3)])
def test_propose_fixed_step_bitexact(s, slots, max_redraw):
    """abc_propose under ABC_STEP_MCMC with beta_a = s: ancestors, walks,
    steps, attempts and flags equal or_propose with s_fixed = s (a wide step
    with 3 redraws exhausts many slots)."""
    cfg = saird_config(4099, 30, 100_000, seed=3, beta_mode=G.ABC_STEP_MCMC,
                       max_redraw=max_redraw)
    m = oracle_model(cfg)
    n = cfg.n_particles
    u = IN.unit_particles(n, seed=11)
    d = IN.distances(n, seed=12)
    eps = float(np.median(d))
    q, pre, tot = O.resample_prefix(d, None, eps, 0)
    c1 = (3 << 16) | 7
    o = O.propose(m, u, pre, tot, 0.0, 0, slots, c1, max_redraw=max_redraw, nthreads=8,
                  s_fixed=s)
    out = {k: torch.empty(sh, dtype=dt, device="cuda") for k, sh, dt in
           (("u", (8, slots), torch.float32), ("s", slots, torch.float32),
            ("anc", slots, torch.int32), ("att", slots, torch.int32), ("flag", slots, torch.uint8))}
    G.abc_propose(cfg, _dev(u), n, _dev(pre), None, None, s, 0, slots, None, c1, out["u"],
                  out["s"], out["anc"], out["att"], out["flag"])
    for k, ok in (("u", o["u"]), ("s", o["s"]), ("anc", o["anc"]), ("att", o["attempts"]),
                  ("flag", o["flag"])):
        assert np.array_equal(_host(out[k]).view(np.uint8),
                              np.ascontiguousarray(ok).view(np.uint8)), k
    assert np.all(o["s"] == np.float32(s))
    if max_redraw == 3:
        assert o["flag"].sum() > 0


def _mcmc_cfg(N, T, P, seed, adapt, M=0, budget=0, s0=0.05, **kw):
    return saird_config(N, T, P, seed=seed, beta_mode=G.ABC_STEP_MCMC, mcmc_s0=s0,
                        mcmc_adapt=adapt, batch_size=M, max_total_batches=budget,
                        weight_mode=G.ABC_W_PAPER, max_batches=400, **kw)


def _compare_generation(gp, g, new, st, tag):
    for k, ok in (("u", new.u), ("d", new.d), ("s", new.s), ("anc", new.anc)):
        assert np.array_equal(gp[k].view(np.uint8), np.ascontiguousarray(ok).view(np.uint8)), \
            (tag, k)
    assert g.eps == st.eps and g.batches == st.batches, tag
    assert g.accepted == st.accepted_total and g.exhausted == st.exhausted, tag
    assert np.float32(g.beta_a) == np.float32(st.beta_a), tag
    assert np.float32(g.mcmc_s) == np.float32(st.mcmc_s), tag


@pytest.mark.parametrize("adapt,M,budget", [(0, 0, 0), (5, 1024, 0), (0, 512, 300)])
def test_context_mcmc_runs_bitexact(adapt, M, budget):
    """Six generations of the baseline through abc_init / abc_generation with
    the paper's weights: a fixed step (no window), a window of 5 batches
    closing during generation 2 or so, and the paper's window (the first
    tenth of a 300-batch run budget): every population, tolerance, batch
    count and step equals the oracle's."""
    cfg = _mcmc_cfg(2048, 40, 100_000, seed=4, adapt=adapt, M=M, budget=budget)
    obs, _, _ = oracle_obs(cfg)
    m, c = oracle_model(cfg, obs), oracle_smc(cfg)
    ctx = G.abc_init(cfg, obs)
    try:
        pop = O.generation0(m, c)
        ms = O.mcmc_start(c)
        assert G.abc_generation(ctx) == 0
        eps1 = 0.0
        for t in range(1, 7):
            new, st = O.generation(m, c, t, eps1, pop, ms)
            assert G.abc_generation(ctx) == st.status == 0
            _compare_generation(get_population(ctx, cfg.n_particles), G.abc_get_stats(ctx, t),
                                new, st, t)
            eps1, pop = st.eps1, new
        if adapt or budget:
            assert ms.k > 0 and ms.s != float(np.float32(cfg.mcmc_s0))
        else:
            assert ms.k == 0
    finally:
        G.abc_free(ctx)


def test_batch_mcmc_runs_equal_oracle_and_mix_with_bdss():
    """A graph batch holding three baseline runs (different windows, seeds,
    sizes) and one BDSS run: each baseline run's generations equal the
    oracle's bit for bit (the step adapts inside the graph's device-side
    batch loop), and the BDSS run equals its single context."""
    cfgs = [_mcmc_cfg(2048, 40, 100_000, seed=1, adapt=8, M=700),
            _mcmc_cfg(1500, 25, 1_000_000, seed=2, adapt=0, M=0, budget=200, s0=0.02),
            _mcmc_cfg(3000, 33, 2_000_000, seed=3, adapt=0),
            saird_config(2048, 40, 100_000, seed=9, weight_mode=G.ABC_W_PAPER)]
    obs = [oracle_obs(c)[0] for c in cfgs]
    b = G.abc_batch_init(cfgs, obs)
    single = G.abc_init(cfgs[3], obs[3])
    try:
        models = [oracle_model(c, o) for c, o in zip(cfgs, obs)]
        smcs = [oracle_smc(c) for c in cfgs]
        pops = [O.generation0(m, c) for m, c in zip(models, smcs)]
        states = [O.mcmc_start(c) for c in smcs[:3]]
        eps1 = [0.0] * 3
        G.abc_batch_generation(b)
        G.abc_run(single, 6)
        for t in range(1, 6):
            G.abc_batch_generation(b)
            for r in range(3):
                new, st = O.generation(models[r], smcs[r], t, eps1[r], pops[r], states[r])
                assert st.status == 0
                u = np.zeros((8, cfgs[r].n_particles), np.float32)
                d = np.zeros(cfgs[r].n_particles)
                W = np.zeros(cfgs[r].n_particles)
                s = np.zeros(cfgs[r].n_particles, np.float32)
                a = np.zeros(cfgs[r].n_particles, np.int32)
                G.abc_batch_get_population(b, r, u, d, W, s, a)
                _compare_generation(dict(u=u, d=d, s=s, anc=a), G.abc_batch_get_stats(b, r, t),
                                    new, st, (t, r))
                eps1[r], pops[r] = st.eps1, new
        N = cfgs[3].n_particles
        u = np.zeros((8, N), np.float32)
        d, W = np.zeros(N), np.zeros(N)
        s, a = np.zeros(N, np.float32), np.zeros(N, np.int32)
        G.abc_batch_get_population(b, 3, u, d, W, s, a)
        gp = get_population(single, N)
        for k, v in (("u", u), ("d", d), ("s", s), ("anc", a)):
            assert np.array_equal(gp[k].view(np.uint8), v.view(np.uint8)), k
    finally:
        G.abc_batch_free(b)
        G.abc_free(single)


def test_checkpoint_carries_the_step_state():
    """abc_get_state of a baseline run holds its step, adaptation count and
    batch count: a context restored from it after generation 2 continues
    exactly as the uninterrupted run (window still open at the cut)."""
    cfg = _mcmc_cfg(2048, 40, 100_000, seed=6, adapt=30, M=512)
    obs, _, _ = oracle_obs(cfg)
    a = G.abc_init(cfg, obs)
    b = G.abc_init(cfg, obs)
    try:
        G.abc_run(a, 3)
        blob = G.abc_get_state(a)
        G.abc_run(a, 6)
        G.abc_set_state(b, blob)
        G.abc_run(b, 6)
        pa, pb = get_population(a, 2048), get_population(b, 2048)
        for k in pa:
            assert np.array_equal(pa[k].view(np.uint8), pb[k].view(np.uint8)), k
        for t in range(3, 6):
            assert G.abc_get_stats(a, t).mcmc_s == G.abc_get_stats(b, t).mcmc_s
    finally:
        G.abc_free(a)
        G.abc_free(b)


def test_mcmc_importance_weights_match_oracle():
    """Importance weights with the baseline's step (each particle's own s as
    kernel variance; the step changes between batches inside the window,
    and the restored state carries it into generation 3):
    generation 3 from the oracle's state equals the oracle's proposals bit
    for bit and its weights within the FP32 bound."""
    from helpers import state_blob
    from test_gpu_parity import logw_tolerance
    cfg = _mcmc_cfg(4096, 60, 100_000, seed=2, adapt=40, M=1024, s0=0.01)
    cfg.weight_mode = G.ABC_W_IMPORTANCE
    obs, _, _ = oracle_obs(cfg)
    m, c = oracle_model(cfg, obs), oracle_smc(cfg)
    pop = O.generation0(m, c)
    ms = O.mcmc_start(c)
    eps1 = 0.0
    for t in range(1, 3):
        pop, st = O.generation(m, c, t, eps1, pop, ms)
        eps1 = st.eps1
    cut = (ms.s, ms.k, ms.batches)
    new, st = O.generation(m, c, 3, eps1, pop, ms)
    assert st.status == 0
    ctx = G.abc_init(cfg, obs)
    try:
        G.abc_set_state(ctx, state_blob(cfg, 3, eps1, pop, mcmc=cut))
        assert G.abc_generation(ctx) == 0
        gp = get_population(ctx, cfg.n_particles)
        for k, ok in (("u", new.u), ("d", new.d), ("s", new.s), ("anc", new.anc)):
            assert np.array_equal(gp[k].view(np.uint8), np.ascontiguousarray(ok).view(np.uint8)), k
        tol = 2 * logw_tolerance(new.s, new.logW)
        assert np.all(np.abs(gp["W"] - new.W) <= tol * new.W + 1e-15)
    finally:
        G.abc_free(ctx)
