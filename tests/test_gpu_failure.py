"""Failure detection in forms that fault no GPU.

1. A pipeline wait of the tensor-core weight kernel that runs out.  The test
   hook abc_set_wait_limit_ns shortens the kernel's wait limit so that its
   copy, MMA and epilogue waits give up almost at once (the waits for the
   CTA's own copies and products before it exits keep their 2 s limit, so
   nothing is left in flight).  The call must return ABC_E_DEVICE from the
   kernel's error word; with the default limit restored, the next call on the
   same stream must succeed and give the results of a call made before.
2. A device allocation that fails.  The test hook abc_inject_alloc_failure
   makes the k-th allocation of abc_init fail on the host as cudaMalloc would;
   abc_init must return ABC_E_NOMEM, give back everything it had allocated,
   and a context created afterwards must run normally.
"""
import numpy as np
import pytest

import paper_2106_15508_gb300 as G
from paper_2106_15508_gb300 import build as B
from paper_2106_15508_gb300 import workloads as WL

import inputs as IN

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    G.lib()
    yield
    G.abc_set_wait_limit_ns(0)
    G.abc_inject_alloc_failure(-1)


def _dev(x):
    x = np.ascontiguousarray(x)
    view = {np.dtype(np.uint32): np.int32, np.dtype(np.uint64): np.int64}.get(x.dtype)
    return torch.from_numpy(x.view(view) if view else x).cuda()


def _tc_weights(args):
    up, s, u, q = args
    rows, n = up.shape[1], u.shape[1]
    pre = np.cumsum(q.astype(np.uint64))
    lw = torch.empty(rows, dtype=torch.float64, device="cuda")
    sc = torch.empty(G.abc_weights_scratch_bytes(rows, n), dtype=torch.uint8, device="cuda")
    G.abc_weights(_dev(up), _dev(s), rows, _dev(u), _dev(q), _dev(pre), n, G.ABC_P_BF16_TC, lw,
                  sc, sc.numel())
    torch.cuda.synchronize()
    return lw.cpu().numpy()


def test_weight_kernel_wait_timeout_is_reported_and_the_context_stays_usable():
    rows, n = 4096, 65536
    args = (IN.clustered_particles(rows, 41, 0.5, 0.15), IN.step_sizes(rows, 42, 1e-3, 0.3),
            IN.clustered_particles(n, 43, 0.5, 0.15), IN.quantised_weights(n, 44))
    before = _tc_weights(args)
    G.abc_set_wait_limit_ns(1)
    try:
        with pytest.raises(G.AbcError) as e:
            _tc_weights(args)
        assert e.value.code == G.ABC_E_DEVICE
    finally:
        G.abc_set_wait_limit_ns(0)
    after = _tc_weights(args)
    assert np.all(np.isfinite(after))
    assert np.allclose(after, before, rtol=1e-12, atol=1e-12)


def _small_config():
    P = 100_000
    return G.config(n_days=30, population=P, init_ard=[WL.initial_active(P), 0, 0], seed=9,
                    n_particles=2048, theta_hi=list(WL.SAIRD_THETA_MAX),
                    weight_mode=G.ABC_W_IMPORTANCE, weight_prec=G.ABC_P_BF16_TC)


def _obs(cfg):
    obs = torch.empty((3, cfg.n_days + 1), dtype=torch.int32, device="cuda")
    th = torch.empty(8, dtype=torch.float32, device="cuda")
    att = torch.empty(1, dtype=torch.int32, device="cuda")
    G.abc_synth_obs(cfg, WL.OBS_BOX_LO, WL.OBS_BOX_HI, obs, th, att)
    return obs.cpu().numpy()


def _run_dist(cfg, obs):
    ctx = G.abc_init(cfg, obs)
    try:
        G.abc_run(ctx, 3)
        d = np.zeros(cfg.n_particles)
        G.abc_get_population(ctx, dist=d)
        return d
    finally:
        G.abc_free(ctx)


def test_injected_allocation_failure_gives_nomem_and_releases_memory():
    cfg = _small_config()
    obs = _obs(cfg)
    ref = _run_dist(cfg, obs)  # also loads every lazily loaded kernel first
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in (0, 1, 7, 20):
        G.abc_inject_alloc_failure(k)
        try:
            with pytest.raises(G.AbcError) as e:
                G.abc_init(cfg, obs)
            assert e.value.code == G.ABC_E_NOMEM, k
        finally:
            G.abc_inject_alloc_failure(-1)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] >= free0 - (4 << 20), k
    assert np.array_equal(_run_dist(cfg, obs), ref)
