"""The surrogate pre-screen (delayed acceptance; an extension beyond the paper, not in
the paper) on the GPU against the oracle.

1. abc_screen equals the oracle's screen rule bit for bit (rho and the
   simulate / audit / screened-out decision), ragged sizes included.
2. The MLP kernels: tensor-core inference, the tensor-core gradient and
   Adam against the fp64 oracle, each within a bound derived from its
   precision.
3. A screened generation of the context keeps only proposals the oracle
   would accept, bit-exact and in (batch, slot) order, and its counters add
   up; the toy model's closed-form posterior survives delayed acceptance
   (the 1/rho factor); the screen saves simulations.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import paper_2106_15508_gb300 as G
from paper_2106_15508_gb300 import build as B

from helpers import (dev, empty, get_population, host, oracle_model, oracle_obs, oracle_smc,
                     saird_config, state_blob)

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
    out = os.environ.get("ABC_SURROGATE_REPORT")
    if out:
        with open(out, "w") as f:
            json.dump(REPORT, f, indent=1, default=float)


# ---- 1. the screen rule ---------------------------------------------------
@pytest.mark.parametrize("M", [1, 255, 4097, 1 << 20])
def test_screen_bit_exact(M):
    rng = np.random.default_rng(M)
    Y = rng.normal(0, 2, (M, 4)).astype(np.float32)
    Y[rng.random(M) < 0.01, 0] = np.nan
    Y[rng.random(M) < 0.01, 0] = 1e30
    flag = (rng.random(M) < 0.05).astype(np.uint8)
    ystat = np.array([12.5, 1, 2, 3, 1.3, 1, 1, 1], np.float32)
    eps = 2.7e5
    c1 = (5 << 16) | 3
    cfg = saird_config(1024, 10, 1000, seed=11, surrogate_tau=0.4, surrogate_rho_min=0.05,
                       audit_frac=0.1)
    rho, sflag = empty(M, torch.float32), empty(M, torch.uint8)
    G.abc_screen(cfg, dev(Y), dev(ystat), dev(flag), M, dev(np.array([eps])), c1, rho, sflag)
    orho, osf = O.screen(oracle_model(cfg), Y, ystat, flag, eps, c1, 0.4, 0.05, 0.1)
    assert np.array_equal(host(rho).view(np.uint32), orho.view(np.uint32))
    assert np.array_equal(host(sflag), osf)
    REPORT["screen_%d" % M] = {k: int(np.sum(osf == k)) for k in range(4)}


def test_screen_rejects_bad_parameters():
    cfg = saird_config(1024, 10, 1000, surrogate_tau=0.0)
    z = empty(4, torch.float32)
    with pytest.raises(G.AbcError):
        G.abc_screen(cfg, empty((4, 4), torch.float32), empty(8, torch.float32), None, 4,
                     dev(np.array([1.0])), 0, z, empty(4, torch.uint8))


# ---- 2. the MLP ---------------------------------------------------------------
def _bf16_rne(x):
    """fp32 -> bf16 -> fp32, round to nearest even (the definition of the cast)."""
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def _split(flat):
    out, o = {}, 0
    for k in O.MLP_ORDER:
        n = int(np.prod(O.MLP_SHAPES[k]))
        out[k] = flat[o:o + n].astype(np.float64).reshape(O.MLP_SHAPES[k])
        o += n
    return out


def _device_params(m):
    """The values the kernels multiply with: bf16 weights, fp32 biases."""
    n = G.lib().abc_mlp_param_count()
    w = np.zeros(n, np.float32)
    wb = np.zeros(n, np.uint16)
    G.abc_mlp_get_params(m, w, wb)
    wbf = (wb.astype(np.uint32) << 16).view(np.float32)
    assert np.array_equal(wbf.view(np.uint32), _bf16_rne(w).view(np.uint32))
    p, pb = _split(w), _split(wbf)
    for k in ("b1", "b2", "b3"):
        pb[k] = p[k]
    return w, pb


def _random_params(seed):
    rng = np.random.default_rng(seed)
    flat = []
    for k in O.MLP_ORDER:
        shp = O.MLP_SHAPES[k]
        fan = shp[1] if len(shp) == 2 else 64
        flat.append(rng.normal(0, 1.2 / math.sqrt(fan), int(np.prod(shp))))
    return np.concatenate(flat).astype(np.float32)


def test_mlp_param_layout_and_init():
    assert G.lib().abc_mlp_param_count() == sum(int(np.prod(s)) for s in O.MLP_SHAPES.values())
    m = G.abc_mlp_create(7)
    try:
        w, _ = _device_params(m)
        p = _split(w)  # fp32 master values
        assert np.all(p["b1"] == 0) and np.all(p["b2"] == 0) and np.all(p["b3"] == 0)
        assert np.abs(p["W1"]).max() <= 1 / math.sqrt(8) and np.abs(p["W2"]).max() <= 1 / 16
        assert np.abs(p["W3"]).max() <= 1 / 16
        assert abs(p["W2"].std() - 1 / 16 / math.sqrt(3)) < 1e-3  # U(-1/16, 1/16)
        assert abs(p["W2"].mean()) < 1e-3
    finally:
        G.abc_mlp_free(m)


@pytest.mark.parametrize("n", [1, 300, 4096, 60001])
def test_mlp_forward_tc_vs_oracle(n):
    """Inference on tcgen05.  Besides fp32 accumulation the kernel rounds the
    first hidden layer to bf16 (relative 2^-9); propagated through layer 2
    (|gelu'| <= 1.13) and layer 3 that bounds the output error by
        sum_o' |W3_oo'| 1.13 sum_k |W2_o'k| |h1_k| 2^-8     (factor 2 margin)
    plus 2^-20 of the magnitudes summed in fp32.  60001 samples are 469
    tiles of 128: every CTA of the persistent kernel runs several."""
    m = G.abc_mlp_create(3)
    try:
        G.abc_mlp_set_params(m, _random_params(5))
        _, p = _device_params(m)
        u = np.random.default_rng(n).random((8, n)).astype(np.float32)
        Y = empty((n, 4), torch.float32)
        sb = G.abc_mlp_scratch_bytes(1, n)
        sc = empty(sb, torch.uint8)
        G.abc_mlp_forward(m, dev(u), n, Y, sc, sb)
        got = host(Y).astype(np.float64)
    finally:
        G.abc_mlp_free(m)
    x = u.T.astype(np.float64)
    want = O.mlp_forward(p, x)
    z1 = x @ p["W1"].T + p["b1"]
    h1 = np.abs(z1 * 0.5 * (1 + np.tanh(0.7978845608028654 * (z1 + 0.044715 * z1**3))))
    # hidden layer 1: bf16 rounding (2^-9 relative, x 1.13 for GELU's slope) and the
    # hardware tanh (absolute error below 2^-10.9, so under 2^-11 |z| in GELU)
    d2 = (h1 * 2.0**-8 * 1.13 + 2.0**-11 * np.abs(z1)) @ np.abs(p["W2"]).T
    z2m = h1 @ np.abs(p["W2"]).T + np.abs(p["b2"])
    # hidden layer 2: the propagated error through GELU plus its own tanh error
    bound = (1.13 * d2 + 2.0**-11 * z2m) @ np.abs(p["W3"]).T
    mag = z2m @ np.abs(p["W3"]).T + np.abs(p["b3"])
    bound = bound + 2.0**-20 * (mag + 1.0)
    err = np.abs(got - want)
    REPORT["mlp_forward_%d" % n] = dict(max_abs=float(err.max()),
                                        max_err_over_bound=float((err / bound).max()),
                                        y_scale=float(np.abs(want).max()))
    assert np.all(np.isfinite(got))
    assert np.all(err <= bound), REPORT["mlp_forward_%d" % n]


def _abs_backward(p, X, T):
    """First-order magnitudes of the training pass in fp64: the backward
    formulas with every factor replaced by its absolute value (|gelu'| <= 1.13,
    |gelu''| <= 0.8).  Each gradient element's rounding error is a sum of
    rounding errors of these products, so it is at most a small multiple of
    the bf16 unit 2^-9 times these magnitudes."""
    gelu = lambda z: 0.5 * z * (1 + np.tanh(0.7978845608028654 * (z + 0.044715 * z**3)))
    def gelu_d(z):
        t = np.tanh(0.7978845608028654 * (z + 0.044715 * z**3))
        return 0.5 * (1 + t) + 0.5 * z * (1 - t * t) * 0.7978845608028654 * (1 + 3 * 0.044715 * z * z)
    B = len(X)
    A = {k: np.abs(v) for k, v in p.items()}
    z1 = X @ p["W1"].T + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = gelu(z2)
    y = h2 @ p["W3"].T + p["b3"]
    dY = np.abs(2 * (y - T) / (4 * B))
    # GELU by the hardware tanh is off by at most 2^-11 |z|: |h| + |z| bounds
    # each hidden value together with that error
    h1 = np.abs(h1) + np.abs(z1)
    h2 = np.abs(h2) + np.abs(z2)
    # |dz2| with the perturbation of gelu' through z2's own magnitude
    mz2 = np.abs(h1) @ A["W2"].T + A["b2"]
    dh2 = dY @ A["W3"]
    dz2 = dh2 * (np.abs(gelu_d(z2)) + 0.8 * mz2)
    dh1 = dz2 @ A["W2"]
    dz1 = dh1 * (np.abs(gelu_d(z1)) + 0.8 * (np.abs(X) @ A["W1"].T + A["b1"]))
    mh2 = np.abs(h2) + 1.13 * mz2
    dYm = dY + np.abs(mh2 @ A["W3"].T) / (4 * B)
    return {"W3": dYm.T @ mh2, "b3": dYm.sum(0), "W2": dz2.T @ np.abs(h1), "b2": dz2.sum(0),
            "W1": dz1.T @ np.abs(X), "b1": dz1.sum(0)}


@pytest.mark.parametrize("Bn", [37, 300, 2048])
def test_mlp_gradient_vs_oracle(Bn):
    """Training pass on tensor cores: the layer-2 forward, input-gradient and
    weight-gradient products take bf16 operands (weights, hidden activations
    H1 and hidden gradients dZ2 rounded to bf16, unit u = 2^-9) with fp32
    accumulation; layers 1 and 3 and the bias sums run in fp32.  Against the
    fp64 oracle (the same bf16 weights as fp64 values): per array the
    max-norm error is at most 2e-2 of the gradient's max-norm (the bf16
    bar), and every element is within 16 u times its first-order magnitude
    (_abs_backward) plus an fp32 floor."""
    m = G.abc_mlp_create(9)
    try:
        G.abc_mlp_set_params(m, _random_params(6))
        _, p = _device_params(m)
        rng = np.random.default_rng(Bn)
        X = rng.random((Bn, 8)).astype(np.float32)
        T = rng.normal(0, 1, (Bn, 4)).astype(np.float32)
        n = G.lib().abc_mlp_param_count()
        g = empty(n, torch.float32)
        sse = empty(1, torch.float32)
        sb = G.abc_mlp_scratch_bytes(Bn, 1)
        sc = empty(sb, torch.uint8)
        G.abc_mlp_grad(m, dev(X), dev(T), Bn, g, sse, sc, sb)
        got = _split(host(g))
        loss = float(host(sse)[0]) / (4 * Bn)
    finally:
        G.abc_mlp_free(m)
    Xd, Td = X.astype(np.float64), T.astype(np.float64)
    oloss, og = O.mlp_backward(p, Xd, Td)
    mag = _abs_backward(p, Xd, Td)
    assert abs(loss - oloss) <= 2.0**-6 * oloss
    rep = {}
    for k in O.MLP_ORDER:
        err = np.abs(got[k] - og[k])
        scale = np.abs(og[k]).max()
        tol = 16 * 2.0**-9 * mag[k] + 2.0**-20 * scale
        rep[k] = dict(rel_maxnorm=float(err.max() / scale), max_err_over_tol=float((err / tol).max()))
        assert err.max() <= 2e-2 * scale, (k, rep[k])
        assert np.all(err <= tol), (k, rep[k])
    REPORT["mlp_grad_%d" % Bn] = rep


def test_mlp_adam_vs_oracle():
    """Three Adam steps in fp32 against the fp64 oracle; the bf16 copy is the
    round-to-nearest-even cast of the fp32 master."""
    m = G.abc_mlp_create(4)
    try:
        w0 = _random_params(8)
        G.abc_mlp_set_params(m, w0)
        n = w0.size
        rng = np.random.default_rng(10)
        ow, om, ov = w0.astype(np.float64), np.zeros(n), np.zeros(n)
        lr = 1e-3
        for step in range(1, 4):
            gr = (rng.normal(0, 1, n) * np.exp(rng.uniform(-8, 2, n))).astype(np.float32)
            G.abc_mlp_adam(m, dev(gr), step, lr)
            O.adam(ow, gr.astype(np.float64), om, ov, lr, 0.9, 0.999, 1e-8, step)
        torch.cuda.synchronize()
        w, _ = _device_params(m)
    finally:
        G.abc_mlp_free(m)
    err = np.abs(w.astype(np.float64) - ow)
    tol = 3 * lr * 1e-5 + 4 * np.spacing(np.abs(ow).astype(np.float32)).astype(np.float64)
    REPORT["adam_max_abs"] = float(err.max())
    assert np.all(err <= tol)


# ---- 3. the context -------------------------------------------------------------
def _sur_config(N, **kw):
    base = dict(weight_mode=G.ABC_W_PAPER, beta_mode=G.ABC_BETA_FIXED, beta_a=2.0, beta_b=5,
                surrogate=1, surrogate_start=1, surrogate_steps=200, surrogate_batch=4096,
                surrogate_tau=0.3, surrogate_rho_min=0.05, audit_frac=0.05)
    base.update(kw)
    return saird_config(N, 60, 100_000, seed=4, **base)


@pytest.mark.parametrize("NN", [4096, 20000])
def test_screened_generation_keeps_oracle_proposals(NN):
    """Paper weights (mode A) keep the run bit-exact before the screen: from
    the oracle's generation-1 population, generation 2 (not screened: nothing
    is trained yet) equals the oracle and trains the surrogate, and
    generation 3 screens.  Every particle of generation 3 is the
    oracle's proposal at some (batch, slot) with d <= eps, bit for bit, in
    (batch, slot) order; the stats add up.  At 20000 slots per batch the
    compacted slots are simulated in the order of the regime key."""
    cfg = _sur_config(NN)
    obs, _, _ = oracle_obs(cfg)
    m, c = oracle_model(cfg, obs), oracle_smc(cfg)
    pop = O.generation0(m, c)
    eps1 = 0.0
    pop, st = O.generation(m, c, 1, eps1, pop)
    eps1 = st.eps1
    ctx = G.abc_init(cfg, obs)
    try:
        G.abc_set_state(ctx, state_blob(cfg, 2, eps1, pop))
        # generation 2: no screen yet (nothing trained); equals the oracle
        assert G.abc_generation(ctx) == 0
        p2, ost = O.generation(m, c, 2, eps1, pop)
        assert ost.status == 0
        g2 = get_population(ctx, NN)
        assert np.array_equal(g2["u"].view(np.uint32), p2.u.view(np.uint32))
        assert np.array_equal(g2["d"], p2.d)
        s2 = G.abc_get_stats(ctx, 2)
        assert s2.screened == 0 and s2.train_loss > 0 and math.isfinite(s2.train_loss)
        # generation 3 screens
        assert G.abc_generation(ctx) == 0
        s3 = G.abc_get_stats(ctx, 3)
        g3 = get_population(ctx, NN)
    finally:
        G.abc_free(ctx)
    N = M = NN
    eps = O.kth(p2.d, O.rank(0.5, N))
    assert s3.eps == eps
    q, pre, tot = O.resample_prefix(p2.d, p2.W, eps, 0)
    acc_u, acc_d, acc_s, acc_a = [], [], [], []
    for b in range(s3.batches):
        c1 = (3 << 16) | b
        o = O.propose(m, p2.u, pre, tot, 2.0, 5, M, c1, nthreads=8)
        d = O.simulate(m, o["u"], c1=c1, nthreads=8)
        d[o["flag"] != 0] = np.inf
        ok = d <= eps
        acc_u.append(o["u"][:, ok])
        acc_d.append(d[ok])
        acc_s.append(o["s"][ok])
        acc_a.append(o["anc"][ok])
    ou = np.concatenate(acc_u, 1)
    od = np.concatenate(acc_d)
    okey = {ou[:, i].tobytes(): i for i in range(ou.shape[1])}
    idx = np.array([okey.get(g3["u"][:, j].tobytes(), -1) for j in range(N)])
    assert np.all(idx >= 0), "a kept particle is not an acceptable oracle proposal"
    assert np.all(np.diff(idx) > 0), "not in (batch, slot) order"
    assert np.array_equal(g3["d"], od[idx])
    assert np.array_equal(g3["s"].view(np.uint32), np.concatenate(acc_s)[idx].view(np.uint32))
    assert np.array_equal(g3["anc"], np.concatenate(acc_a)[idx])
    passed = s3.sims - s3.audited
    assert s3.screened + passed + s3.exhausted == s3.batches * M
    assert 0 <= s3.audit_accepted <= s3.audited <= s3.screened
    frr = s3.audit_accepted / max(s3.audited, 1)
    REPORT["screened_generation_%d" % NN] = dict(
        batches=int(s3.batches), oracle_acceptable=int(ou.shape[1]), screened=int(s3.screened),
        audited=int(s3.audited), audit_accepted=int(s3.audit_accepted),
        false_rejection_rate=frr, train_loss=float(s3.train_loss),
        skipped_fraction=float(s3.screened - s3.audited) / (s3.batches * M))


def _toy_config(seed, surrogate):
    return G.config(model=G.ABC_MODEL_GAUSS_TOY, n_days=1, population=1, init_ard=[0, 0, 0],
                    theta_lo=[-10.0] * 8, theta_hi=[10.0] * 8, seed=seed, n_particles=4096,
                    beta_mode=G.ABC_BETA_FIXED, beta_a=8.0, beta_b=1000,
                    weight_mode=G.ABC_W_IMPORTANCE, max_batches=2000, surrogate=surrogate,
                    surrogate_start=2, surrogate_steps=300, surrogate_batch=4096,
                    surrogate_tau=0.25, surrogate_rho_min=0.05, audit_frac=0.02)


def test_toy_posterior_with_delayed_acceptance():
    """Importance weights times 1/rho keep the conjugate toy's closed-form
    ABC posterior (variance 1 + eps^2/10, mean 0) within 3 Monte-Carlo
    standard errors over 4 seeds, and the screen saves simulations against
    the same seeds without it."""
    ratios, ses, zs, sims = [], [], [], {0: 0, 1: 0}
    for seed in range(1, 5):
        for sur in (1, 0):
            ctx = G.abc_init(_toy_config(seed, sur), None)
            try:
                G.abc_run(ctx, 10)
                st = [G.abc_get_stats(ctx, t) for t in range(1, 10)]
                p = get_population(ctx, 4096)
            finally:
                G.abc_free(ctx)
            assert all(s.status == 0 for s in st)
            sims[sur] += sum(s.sims for s in st[3:])
            if not sur:
                continue
            assert sum(s.screened for s in st) > 0
            last = st[-1]
            th = -10 + 20 * p["u"].astype(np.float64)
            mean = (th * p["W"]).sum(1)
            var = (th**2 * p["W"]).sum(1) - mean**2
            v0 = 1 + last.eps**2 / 10
            ratios.append(var.mean() / v0)
            ses.append(math.sqrt(2.0 / (last.ess * 8)))
            zs.append(mean.mean() / math.sqrt(v0 / last.ess / 8))
    se = math.sqrt(sum(x * x for x in ses)) / len(ses)
    REPORT["toy_delayed_acceptance"] = dict(var_ratio=float(np.mean(ratios)), se=se,
                                            z=[float(z) for z in zs],
                                            sims_gen4_9=dict(surrogate=sims[1], plain=sims[0]))
    assert abs(np.mean(ratios) - 1) < 3 * se, (ratios, se)
    assert abs(np.mean(zs)) * math.sqrt(len(zs)) < 3, zs
    assert sims[1] < sims[0]
