"""The tensor-core (tcgen05) weight path.

1. abc_tc_probe: one 128 x 256 x 64 bf16 product with the weight kernel's
   operand layout and descriptors.  Small-integer operands make every
   product and partial sum exact in fp32, so D must equal A B^T exactly.
2. abc_weights with ABC_P_BF16_TC against the fp64 oracle: the error is
   stated (written to the parity report) and bounded by the error model of
   the fp32 tensor-memory accumulation (logw_tc_bound).
3. A generation of the context on the tensor-core path reproduces the
   oracle's proposals and distances bit for bit; its weights follow (2).
"""
import json
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


def logw_tc_bound(up, s, olw):
    """Error model of the tensor-core path.  The pair exponent (log2) is an
    fp32 sum of 60 exact bf16 products whose magnitudes are bounded by
    L (2 |x| |y| + |y|^2) + |c| <= 6 L + 32 (|x|, |y| <= sqrt 2 after
    centring, L = log2(e) / (2 s)); the three-way split represents each
    factor to 2^-24 relative.  With up to 64 roundings of 2^-24 of that
    magnitude plus the fp32 row sums of the FP32 path:
        |d log W| <= 2^-24 (64 (6 L + 32) + 160)   (natural log, ln 2 < 1)."""
    L = 1.4426950408889634 / (2.0 * np.maximum(np.asarray(s, np.float32), 1e-30))
    return 2.0**-24 * (64.0 * (6.0 * L + 32.0) + 160.0)


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


def _state_errors(name, lw, olw, s, up):
    err = np.abs(lw - olw)
    bound = logw_tc_bound(up, s, olw)
    W = np.exp(olw - olw.max())
    W /= W.sum()
    Wg = np.exp(lw - lw.max())
    Wg /= Wg.sum()
    REPORT[name] = dict(max_abs=float(err.max()), median_abs=float(np.median(err)),
                        p99_abs=float(np.quantile(err, 0.99)),
                        max_err_over_bound=float((err / bound).max()),
                        tv_normalised_W=float(0.5 * np.abs(W - Wg).sum()),
                        rows=int(len(err)))
    print(name, REPORT[name])
    assert np.all(np.isfinite(lw))
    assert np.all(err <= bound), REPORT[name]


@pytest.mark.parametrize("rows,n", [(4096, 4096), (777, 5003), (130, 300)])
def test_weights_tc_vs_oracle(rows, n):
    up = IN.clustered_particles(rows, rows, 0.5, 0.15)
    u = IN.clustered_particles(n, n + 1, 0.5, 0.15)
    s = IN.step_sizes(rows, 3, 1e-4, 0.3)
    q = IN.quantised_weights(n, 5)
    lw, tot = _weights(up, s, u, q, G.ABC_P_BF16_TC)
    olw = O.weights(up, s, u, q, tot, nthreads=8)
    _state_errors("weights_tc_%dx%d" % (rows, n), lw, olw, s, up)


def test_weights_tc_full_size_sampled_rows():
    n = 1 << 20
    up = IN.clustered_particles(n, 21, 0.5, 0.1)
    u = IN.clustered_particles(n, 22, 0.5, 0.1)
    s = IN.step_sizes(n, 23, 1e-4, 0.05)
    q = IN.quantised_weights(n, 24, zero_frac=0.5)
    lw, tot = _weights(up, s, u, q, G.ABC_P_BF16_TC)
    idx = np.sort(IN.rng(25).choice(n, 48, replace=False))
    olw = O.weights(up[:, idx], s[idx], u, q, tot, nthreads=8)
    _state_errors("weights_tc_full_sampled", lw[idx], olw, s[idx], up[:, idx])


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
