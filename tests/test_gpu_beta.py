"""Parity of the real-shape step-size rules (Sec. 3.2: fixed real shapes, the
mean-variance and the mode-concentration parameterisations beside Eq. 16)
with the CPU oracle, bit for bit: single proposals through abc_propose, whole
generations through a context, and runs inside a graph-captured batch."""
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


def dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


RULES = [
    (G.ABC_BETA_REAL, 0.4, 2.6, 3),
    (G.ABC_BETA_REAL, 2.5, 0.4, 1),
    (G.ABC_BETA_REAL, 2.0 ** -20, 2.0 ** -20, 1),
    (G.ABC_BETA_MEAN_VAR, 1 / 3, 1 / 18, 1),
    (G.ABC_BETA_MEAN_VAR, 1 / 3, 1 / 18, 6),   # a + b at the 1/16 floor
    (G.ABC_BETA_MODE_CONC, 0.2, 10.0, 3),
    (G.ABC_BETA_MODE_CONC, 0.0, 3.0, 9),
]


@pytest.mark.parametrize("mode,p1,p2,t", RULES)
def test_propose_real_shape_rules_bitexact(mode, p1, p2, t):
    n, slots = 3000, 5003
    cfg = saird_config(n, 10, 1000, seed=12, beta_mode=mode, beta_p1=p1, beta_p2=p2)
    m = oracle_model(cfg)
    u = IN.clustered_particles(n, 3, 0.5, 0.2)
    q = IN.quantised_weights(n, 4)
    pre = np.cumsum(q.astype(np.uint64))
    eps, eps1 = 1.5, 4.0
    c1 = (t << 16) | 2
    outs = dict(u=torch.empty((8, slots), dtype=torch.float32, device="cuda"),
                s=torch.empty(slots, dtype=torch.float32, device="cuda"),
                anc=torch.empty(slots, dtype=torch.int32, device="cuda"),
                att=torch.empty(slots, dtype=torch.int32, device="cuda"),
                flag=torch.empty(slots, dtype=torch.uint8, device="cuda"))
    G.abc_propose(cfg, dev(u), n, dev(pre), dev(np.array([eps])), dev(np.array([eps1])),
                  0.0, 0, slots, None, c1, outs["u"], outs["s"], outs["anc"], outs["att"],
                  outs["flag"])
    a, b, bi = O.beta_shape(mode, np.float32(eps / eps1), t, p1=p1, p2=p2)
    assert bi == 0
    o = O.propose(m, u, pre, int(pre[-1]), a, 0, slots, c1, nthreads=8, beta_bf=b)
    assert np.array_equal(host(outs["anc"]), o["anc"])
    assert np.array_equal(host(outs["s"]).view(np.uint32), o["s"].view(np.uint32))
    assert np.array_equal(host(outs["u"]).view(np.uint32), o["u"].view(np.uint32))
    assert np.array_equal(host(outs["att"]), o["attempts"])
    assert np.array_equal(host(outs["flag"]), o["flag"])


@pytest.mark.parametrize("t,eps", [(513, 1.5), (2000, 0.0)])
def test_propose_paper_schedule_beyond_1024_bitexact(t, eps):
    """Eq. 16 after stage 512: integer b 0 selects Beta(eps/eps1, 2t) by the
    Gamma ratio (ratio 0 clamped to 2^-20)."""
    n, slots = 2000, 3001
    cfg = saird_config(n, 10, 1000, seed=13, beta_mode=G.ABC_BETA_PAPER)
    m = oracle_model(cfg)
    u = IN.clustered_particles(n, 5, 0.5, 0.2)
    q = IN.quantised_weights(n, 6)
    pre = np.cumsum(q.astype(np.uint64))
    eps1 = 4.0
    c1 = (t << 16) | 5
    outs = dict(u=torch.empty((8, slots), dtype=torch.float32, device="cuda"),
                s=torch.empty(slots, dtype=torch.float32, device="cuda"),
                anc=torch.empty(slots, dtype=torch.int32, device="cuda"),
                att=torch.empty(slots, dtype=torch.int32, device="cuda"),
                flag=torch.empty(slots, dtype=torch.uint8, device="cuda"))
    G.abc_propose(cfg, dev(u), n, dev(pre), dev(np.array([eps])), dev(np.array([eps1])),
                  0.0, 0, slots, None, c1, outs["u"], outs["s"], outs["anc"], outs["att"],
                  outs["flag"])
    a, b, bi = O.beta_shape(G.ABC_BETA_PAPER, np.float32(eps / eps1), t)
    assert bi == 0 and b == 2 * t
    o = O.propose(m, u, pre, int(pre[-1]), a, 0, slots, c1, nthreads=8, beta_bf=b)
    assert np.array_equal(host(outs["anc"]), o["anc"])
    assert np.array_equal(host(outs["s"]).view(np.uint32), o["s"].view(np.uint32))
    assert np.array_equal(host(outs["u"]).view(np.uint32), o["u"].view(np.uint32))
    assert np.array_equal(host(outs["flag"]), o["flag"])


def test_propose_rejects_stage_zero_for_scheduled_rules():
    cfg = saird_config(64, 10, 1000, beta_mode=G.ABC_BETA_MODE_CONC, beta_p1=0.2, beta_p2=10.0)
    u = np.full((8, 64), 0.5, np.float32)
    pre = np.arange(1, 65, dtype=np.uint64)
    e = dev(np.array([1.0]))
    outs = [torch.empty((8, 8), dtype=torch.float32, device="cuda"),
            torch.empty(8, dtype=torch.float32, device="cuda"),
            torch.empty(8, dtype=torch.int32, device="cuda"),
            torch.empty(8, dtype=torch.int32, device="cuda"),
            torch.empty(8, dtype=torch.uint8, device="cuda")]
    with pytest.raises(G.AbcError):
        G.abc_propose(cfg, dev(u), 64, dev(pre), e, e, 0.0, 0, 8, None, 5, *outs)


def _check_stats(g, o):
    assert g.eps == o.eps and g.eps1 == o.eps1
    assert g.batches == o.batches and g.accepted == o.accepted_total
    assert g.beta_b == o.beta_b == 0
    assert np.float32(g.beta_a) == np.float32(o.beta_a)
    assert np.float32(g.beta_bf) == np.float32(o.beta_bf)


@pytest.mark.parametrize("mode,p1,p2", [(G.ABC_BETA_MEAN_VAR, 1 / 3, 1 / 18),
                                        (G.ABC_BETA_MODE_CONC, 0.1, 6.0)])
def test_context_real_shape_rules_bitexact(mode, p1, p2):
    """4096 particles, 60 days, P = 1e5, the paper's weights (Eq. 10), 6
    generations: populations and shapes equal the oracle's bit for bit."""
    cfg = saird_config(4096, 60, 100_000, seed=21, beta_mode=mode, beta_p1=p1, beta_p2=p2,
                       weight_mode=G.ABC_W_PAPER)
    obs, _, _ = oracle_obs(cfg)
    m, c = oracle_model(cfg, obs), oracle_smc(cfg)
    ctx = G.abc_init(cfg, obs)
    try:
        pop = O.generation0(m, c)
        G.abc_generation(ctx)
        eps1 = 0.0
        for t in range(1, 6):
            new, st = O.generation(m, c, t, eps1, pop)
            assert G.abc_generation(ctx) == st.status == 0
            gp = get_population(ctx, 4096)
            for k, ok in (("u", new.u), ("d", new.d), ("s", new.s), ("anc", new.anc)):
                assert np.array_equal(gp[k].view(np.uint8),
                                      np.ascontiguousarray(ok).view(np.uint8)), (t, k)
            _check_stats(G.abc_get_stats(ctx, t), st)
            eps1, pop = st.eps1, new
    finally:
        G.abc_free(ctx)


def test_batch_mixed_beta_rules_match_oracle():
    """Four runs with four rules inside one graph-captured batch, 4 generations,
    the paper's weights (Eq. 10): populations equal the oracle's bit for bit."""
    specs = [(2048, 30, 100_000, 31, G.ABC_BETA_REAL, 0.5, 3.5),
             (1024, 45, 500_000, 32, G.ABC_BETA_MEAN_VAR, 0.3, 0.02),
             (3000, 20, 50_000, 33, G.ABC_BETA_MODE_CONC, 0.05, 4.0),
             (1500, 25, 1_000_000, 34, G.ABC_BETA_PAPER, 0.0, 0.0)]
    cfgs = [saird_config(N, T, P, seed=s, beta_mode=bm, beta_p1=p1, beta_p2=p2,
                         weight_mode=G.ABC_W_PAPER) for N, T, P, s, bm, p1, p2 in specs]
    obs = [oracle_obs(c)[0] for c in cfgs]
    b = G.abc_batch_init(cfgs, obs)
    try:
        models = [oracle_model(c, o) for c, o in zip(cfgs, obs)]
        smcs = [oracle_smc(c) for c in cfgs]
        pops = [O.generation0(m, c) for m, c in zip(models, smcs)]
        eps1 = [0.0] * len(cfgs)
        G.abc_batch_generation(b)
        for t in range(1, 5):
            G.abc_batch_generation(b)
            for r, cfg in enumerate(cfgs):
                new, st = O.generation(models[r], smcs[r], t, eps1[r], pops[r])
                assert st.status == 0
                N = cfg.n_particles
                u = np.zeros((8, N), np.float32)
                d, W = np.zeros(N), np.zeros(N)
                s = np.zeros(N, np.float32)
                a = np.zeros(N, np.int32)
                G.abc_batch_get_population(b, r, u, d, W, s, a)
                for k, got, ok in (("u", u, new.u), ("d", d, new.d), ("s", s, new.s),
                                   ("anc", a, new.anc)):
                    assert np.array_equal(got.view(np.uint8),
                                          np.ascontiguousarray(ok).view(np.uint8)), (t, r, k)
                g = G.abc_batch_get_stats(b, r, t)
                assert g.eps == st.eps and g.beta_b == st.beta_b
                assert np.float32(g.beta_a) == np.float32(st.beta_a)
                assert np.float32(g.beta_bf) == np.float32(st.beta_bf)
                eps1[r], pops[r] = st.eps1, new
    finally:
        G.abc_batch_free(b)
