"""The tensor-core (tcgen05) weight path.

1. abc_tc_probe: one 128 x 256 x 64 bf16 product with the weight kernel's
   operand layout and descriptors.  Small-integer operands make every
   product and partial sum exact in fp32, so D must equal A B^T exactly.
2. abc_weights with ABC_P_BF16_TC against the fp64 oracle: the error is
   stated (written to the parity report) and bounded by the error model of
   the fp32 tensor-memory accumulation (logw_tc_bound); rows whose model
   bound is too large are recomputed exactly and take the FP32 bound.
3. A generation of the context on the tensor-core path reproduces the
   oracle's proposals and distances bit for bit; its weights follow (2).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import paper_2106_15508_gb300 as G
from paper_2106_15508_gb300 import build as B

import inputs as IN
from helpers import get_population, oracle_model, oracle_obs, oracle_smc, saird_config, state_blob

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
    out = os.environ.get("ABC_TC_REPORT")
    if out:
        with open(out, "w") as f:
            json.dump(REPORT, f, indent=1, default=float)


def packed_index(r, k):
    """Core-matrix layout of abc_tc_probe's operands (8 x 8 bf16 blocks)."""
    return (((r // 8) * 8 + k // 8) * 64) + (r % 8) * 8 + (k % 8)


def pack(M):
    rows, K = M.shape
    out = np.zeros(rows * K, np.float32)
    for r in range(rows):
        for k in range(K):
            out[packed_index(r, k)] = M[r, k]
    return out


def to_bf16_bits(x):
    """float32 values exactly representable in bf16 -> raw 16-bit patterns."""
    b = np.asarray(x, np.float32).view(np.uint32)
    assert np.all((b & 0xFFFF) == 0)
    return (b >> 16).astype(np.uint16)


def test_tc_probe_exact_small_integers():
    rng = np.random.default_rng(0)
    A = rng.integers(-8, 9, (128, 64)).astype(np.float32)
    Bm = rng.integers(-8, 9, (256, 64)).astype(np.float32)
    a = torch.from_numpy(to_bf16_bits(pack(A)).view(np.int16)).cuda()
    b = torch.from_numpy(to_bf16_bits(pack(Bm)).view(np.int16)).cuda()
    D = torch.empty((128, 256), dtype=torch.float32, device="cuda")
    G.abc_tc_probe(a, b, D)
    got = D.cpu().numpy()
    want = A.astype(np.float64) @ Bm.astype(np.float64).T
    dump = os.environ.get("ABC_TC_DUMP")
    if dump:
        np.savez(dump, A=A, B=Bm, D=got)
    REPORT["probe_exact_fraction"] = float(np.mean(got == want))
    assert np.array_equal(got, want)


TC_BOUND_MAX = 2.0**-24 * (64.0 * (6.0 * 721.34752 + 32.0) + 160.0)


def tc_row_bound(up, s, u, q):
    """Error model of the tensor-core precision for row j.  The pair exponent
    (log2) is an fp32 sum of up to 64 exact bf16 products of total size
    L (2 |x| Y + Y^2) + |c| <= L (2 |x| Y + Y^2) + 32, with coordinates
    centred on the mean of the columns (q > 0), x = u'_j - mean,
    Y^2 = max_k |u_k - mean|^2 and L = log2(e) / (2 s_j) (the three-way split
    represents every factor to 2^-24 relative); with up to 64 roundings of
    2^-24 of that size plus the fp32 row sums of the FP32 path:
        B_j = 2^-24 (64 (L (2 |x| Y + Y^2) + 32) + 160)   (natural log, ln 2 < 1)."""
    keep = q > 0
    m = u[:, keep].astype(np.float64).mean(1).astype(np.float32).astype(np.float64)
    y2 = ((u[:, keep].astype(np.float64) - m[:, None]) ** 2).sum(0).max()
    x = np.sqrt(((up.astype(np.float64) - m[:, None]) ** 2).sum(0))
    L = 1.4426950408889634 / (2.0 * np.maximum(np.asarray(s, np.float64), 1e-30))
    return 2.0**-24 * (64.0 * (L * (2.0 * x * math.sqrt(y2) + y2) + 32.0) + 160.0)


def logw_tc_bound(up, s, olw, u, q):
    """Rows whose bound B_j is at most TC_BOUND_MAX (the bound at s = 1e-3
    with |x|, |y| <= sqrt 2) keep their tensor-core value and take B_j.  The
    others are recomputed exactly from the columns that can lie within 45
    bits of the row maximum (or by the FP32 kernel): they take the FP32
    tolerance plus the dropped columns' share, at most nc 2^-45 of the row
    sum.  A row within 1% of the cut may be on either side (the library
    evaluates B_j in fp32)."""
    from test_gpu_parity import logw_tolerance_direct_fp32
    B = tc_row_bound(up, s, u, q)
    fp = logw_tolerance_direct_fp32(s, olw) + int(np.sum(q > 0)) * 2.0**-45
    return np.where(B <= 1.01 * TC_BOUND_MAX, np.maximum(B, fp), fp)


def _weights(up, s, u, q, prec):
    rows, n = up.shape[1], u.shape[1]
    pre = np.cumsum(q.astype(np.uint64))
    lw = torch.empty(rows, dtype=torch.float64, device="cuda")
    sc = torch.empty(G.abc_weights_scratch_bytes(rows, n), dtype=torch.uint8, device="cuda")
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x).view(
        {np.dtype(np.uint32): np.int32, np.dtype(np.uint64): np.int64}.get(x.dtype, x.dtype))).cuda()
    G.abc_weights(dev(up), dev(s), rows, dev(u), dev(q), dev(pre), n, prec, lw, sc, sc.numel())
    torch.cuda.synchronize()
    return lw.cpu().numpy(), int(pre[-1])


def _state_errors(name, lw, olw, s, up, u, q):
    err = np.abs(lw - olw)
    bound = logw_tc_bound(up, s, olw, u, q)
    W = np.exp(olw - olw.max())
    W /= W.sum()
    Wg = np.exp(lw - lw.max())
    Wg /= Wg.sum()
    relW = np.abs(Wg - W) / np.maximum(W, 1e-300)
    big = W >= 1e-6 * W.max()  # weights that carry mass
    ess, essg = 1.0 / np.sum(W**2), 1.0 / np.sum(Wg**2)
    REPORT[name] = dict(max_abs=float(err.max()), median_abs=float(np.median(err)),
                        p99_abs=float(np.quantile(err, 0.99)),
                        max_err_over_bound=float((err / bound).max()),
                        tv_normalised_W=float(0.5 * np.abs(W - Wg).sum()),
                        max_rel_W=float(relW[big].max()), median_rel_W=float(np.median(relW[big])),
                        ess_rel_err=float(abs(essg - ess) / ess),
                        rows=int(len(err)),
                        fraction_exact=float(np.mean(tc_row_bound(up, s, u, q) > TC_BOUND_MAX)))
    print(name, REPORT[name])
    assert np.all(np.isfinite(lw))
    assert np.all(err <= bound), REPORT[name]


@pytest.mark.parametrize("rows,n,slo,shi", [(4096, 4096, 1e-4, 0.3), (777, 5003, 1e-4, 0.3),
                                             (130, 300, 1e-4, 0.3),
                                             (1000, 2000, 2e-3, 0.3),     # every row on tcgen05
                                             (1000, 2000, 1e-7, 9e-4)])   # mostly recomputed
def test_weights_tc_vs_oracle(rows, n, slo, shi):
    up = IN.clustered_particles(rows, rows, 0.5, 0.15)
    u = IN.clustered_particles(n, n + 1, 0.5, 0.15)
    s = IN.step_sizes(rows, 3, slo, shi)
    q = IN.quantised_weights(n, 5)
    lw, tot = _weights(up, s, u, q, G.ABC_P_BF16_TC)
    olw = O.weights(up, s, u, q, tot, nthreads=8)
    _state_errors("weights_tc_%dx%d_s%g" % (rows, n, slo), lw, olw, s, up, u, q)


def test_weights_tc_tiny_steps_recomputed():
    """Steps of 1e-20..1e-9 (far below any tensor-core precision): every row
    is recomputed exactly from the few columns near it."""
    rows, n = 600, 3001
    up = IN.clustered_particles(rows, 31, 0.5, 0.15)
    u = IN.clustered_particles(n, 32, 0.5, 0.15)
    s = IN.step_sizes(rows, 33, 1e-20, 1e-9)
    q = IN.quantised_weights(n, 34)
    lw, tot = _weights(up, s, u, q, G.ABC_P_BF16_TC)
    olw = O.weights(up, s, u, q, tot, nthreads=8)
    _state_errors("weights_tc_tiny_s", lw, olw, s, up, u, q)


def test_weights_tc_dense_cluster_falls_back_to_direct_rows():
    """Two dense column clusters far apart put the centre between them, so
    rows inside one cluster have large error bounds while thousands of
    columns lie within the listing margin: the lists overflow and the rows
    go through the per-row direct-difference kernel."""
    r = np.random.default_rng(35)
    n = 6000
    u = np.empty((8, n), np.float32)
    u[:, :3000] = np.clip(0.9 + 0.01 * r.standard_normal((8, 3000)), 0, 1)
    u[:, 3000:] = np.clip(0.1 + 0.01 * r.standard_normal((8, 3000)), 0, 1)
    rows = 700
    up = np.clip(0.9 + 0.01 * r.standard_normal((8, rows)), 0, 1).astype(np.float32)
    s = np.exp(r.uniform(np.log(5e-5), np.log(2e-4), rows)).astype(np.float32)
    q = IN.quantised_weights(n, 36, zero_frac=0.0)
    lw, tot = _weights(up, s, u, q, G.ABC_P_BF16_TC)
    olw = O.weights(up, s, u, q, tot, nthreads=8)
    _state_errors("weights_tc_dense_cluster", lw, olw, s, up, u, q)


def test_weights_tc_full_size_sampled_rows():
    n = 1 << 20
    up = IN.clustered_particles(n, 21, 0.5, 0.1)
    u = IN.clustered_particles(n, 22, 0.5, 0.1)
    s = IN.step_sizes(n, 23, 1e-4, 0.05)
    q = IN.quantised_weights(n, 24, zero_frac=0.5)
    lw, tot = _weights(up, s, u, q, G.ABC_P_BF16_TC)
    idx = np.sort(IN.rng(25).choice(n, 48, replace=False))
    olw = O.weights(up[:, idx], s[idx], u, q, tot, nthreads=8)
    _state_errors("weights_tc_full_sampled", lw[idx], olw, s[idx], up[:, idx], u, q)


def test_context_generation_on_tensor_cores():
    cfg = saird_config(4096, 60, 100_000, seed=2, weight_mode=G.ABC_W_IMPORTANCE,
                       weight_prec=G.ABC_P_BF16_TC)
    obs, _, _ = oracle_obs(cfg)
    m, c = oracle_model(cfg, obs), oracle_smc(cfg)
    pop = O.generation0(m, c)
    eps1 = 0.0
    for t in range(1, 3):
        pop, st = O.generation(m, c, t, eps1, pop)
        eps1 = st.eps1
    new, st = O.generation(m, c, 3, eps1, pop)
    ctx = G.abc_init(cfg, obs)
    try:
        G.abc_set_state(ctx, state_blob(cfg, 3, eps1, pop))
        assert G.abc_generation(ctx) == 0
        gp = get_population(ctx, cfg.n_particles)
        for k, ok in (("u", new.u), ("d", new.d), ("s", new.s), ("anc", new.anc)):
            assert np.array_equal(gp[k].view(np.uint8), np.ascontiguousarray(ok).view(np.uint8)), k
        REPORT["ctx_tc_tv_normalised_W"] = float(0.5 * np.abs(gp["W"] - new.W).sum())
        REPORT["ctx_tc_ess"] = [float(G.abc_get_stats(ctx, 3).ess), float(st.ess)]
        assert REPORT["ctx_tc_tv_normalised_W"] < 1e-3
    finally:
        G.abc_free(ctx)


@pytest.mark.parametrize("prec", [G.ABC_P_FP32, G.ABC_P_BF16_TC])
def test_late_generation_weights_with_paper_schedule(prec):
    """A later generation of the paper's Beta(eps_t/eps_1, 2t) schedule puts
    part of the steps far below 1e-3 (a_t < 1): starting from the oracle's
    population after generation 5 (16384 particles), the generation's
    normalised weights and ESS agree with the fp64 oracle on both precisions
    (the tensor-core precision sends the rows with large error bounds to the
    FP32 path)."""
    cfg = saird_config(16384, 60, 1_000_000, seed=7, weight_mode=G.ABC_W_IMPORTANCE,
                       beta_mode=G.ABC_BETA_PAPER, weight_prec=prec)
    obs, _, _ = oracle_obs(cfg)
    m, c = oracle_model(cfg, obs), oracle_smc(cfg, nthreads=16)
    pop = O.generation0(m, c)
    eps1 = 0.0
    for t in range(1, 6):
        pop, st = O.generation(m, c, t, eps1, pop)
        assert st.status == 0
        eps1 = st.eps1
    new, st = O.generation(m, c, 6, eps1, pop)
    assert st.status == 0
    small = float(np.mean(new.s < 1e-3))
    ctx = G.abc_init(cfg, obs)
    try:
        G.abc_set_state(ctx, state_blob(cfg, 6, eps1, pop))
        assert G.abc_generation(ctx) == 0
        gp = get_population(ctx, cfg.n_particles)
        assert np.array_equal(gp["anc"], new.anc) and np.array_equal(gp["d"], new.d)
        tv = float(0.5 * np.abs(gp["W"] - new.W).sum())
        ess = (float(G.abc_get_stats(ctx, 6).ess), float(st.ess))
        REPORT["late_gen_prec%d" % prec] = {"tv_normalised_W": tv, "ess_gpu_oracle": ess,
                                            "fraction_s_below_1e-3": small}
        assert tv < 1e-3
        assert abs(ess[0] - ess[1]) <= 1e-3 * ess[1]
    finally:
        G.abc_free(ctx)


@pytest.mark.parametrize("t", [1, 2, 4])
def test_generation_weight_errors_stated(t):
    """Error of the tensor-core precision against the fp64 oracle on the
    weights of real generations (the oracle's population after generation
    t - 1 loaded into a context; 16384 particles, 60 days, P = 1e6, paper
    schedule): generation 1 has every row on the tensor cores (large steps),
    later ones a growing share recomputed exactly.  Stated in the report:
    max / median / p99 of |d log W| and of the relative error of the
    normalised weights carrying mass, the total variation and the ESS error."""
    cfg = saird_config(16384, 60, 1_000_000, seed=11, weight_mode=G.ABC_W_IMPORTANCE,
                       beta_mode=G.ABC_BETA_PAPER, weight_prec=G.ABC_P_BF16_TC)
    obs, _, _ = oracle_obs(cfg)
    m, c = oracle_model(cfg, obs), oracle_smc(cfg, nthreads=16)
    pop = O.generation0(m, c)
    eps1 = 0.0
    for k in range(1, t):
        pop, st = O.generation(m, c, k, eps1, pop)
        assert st.status == 0
        eps1 = st.eps1
    new, st = O.generation(m, c, t, eps1, pop)
    assert st.status == 0
    ctx = G.abc_init(cfg, obs)
    try:
        G.abc_set_state(ctx, state_blob(cfg, t, eps1, pop))
        assert G.abc_generation(ctx) == 0
        gp = get_population(ctx, cfg.n_particles)
        g = G.abc_get_stats(ctx, t)
    finally:
        G.abc_free(ctx)
    assert np.array_equal(gp["anc"], new.anc) and np.array_equal(gp["d"], new.d)
    W, Wg = new.W, gp["W"]
    lw_rel = np.log(np.maximum(Wg, 1e-300)) - np.log(np.maximum(W, 1e-300))
    big = W >= 1e-6 * W.max()
    relW = np.abs(Wg - W)[big] / W[big]
    dlog = np.abs(lw_rel[big] - np.median(lw_rel[big]))
    REPORT["generation_%d_tc" % t] = dict(
        rows_tc=int(g.rows_tc), rows_kept=int(g.rows_exp), rows_with_mass=int(big.sum()),
        max_rel_W=float(relW.max()), median_rel_W=float(np.median(relW)),
        p99_rel_W=float(np.quantile(relW, 0.99)), max_dlogW=float(dlog.max()),
        median_dlogW=float(np.median(dlog)), p99_dlogW=float(np.quantile(dlog, 0.99)),
        tv_normalised_W=float(0.5 * np.abs(Wg - W).sum()),
        ess_gpu=float(g.ess), ess_oracle=float(st.ess),
        ess_rel_err=float(abs(g.ess - st.ess) / st.ess))
    print(REPORT["generation_%d_tc" % t])
    assert REPORT["generation_%d_tc" % t]["tv_normalised_W"] < 1e-3
