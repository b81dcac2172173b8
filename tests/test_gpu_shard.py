"""The sharded-run driver with the CUDA backend (paper_2106_15508_gb300.shard):
on one GPU (a single rank) its generations equal those of a context bit for
bit -- the driver splits slots and weight rows by rank and exchanges them by
all-gathers, and with one rank it runs the same kernels on the same Philox
counters as abc_generation.  (Several ranks need several GPUs; their
exchange logic is tested on CPU ranks in test_shard.py.)"""
import numpy as np
import pytest

import paper_2106_15508_gb300 as G
from paper_2106_15508_gb300 import build as B

from helpers import oracle_obs, saird_config

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    G.lib()


def _device_population(ctx, N):
    from paper_2106_15508_gb300 import shard
    p = shard.Population(torch.empty((8, N), dtype=torch.float32, device="cuda"),
                         torch.empty(N, dtype=torch.float64, device="cuda"),
                         torch.empty(N, dtype=torch.float64, device="cuda"),
                         torch.empty(N, dtype=torch.float32, device="cuda"),
                         torch.empty(N, dtype=torch.int32, device="cuda"))
    G.abc_get_population(ctx, p.u, p.d, p.W, p.s, p.anc, on_device=True)
    torch.cuda.synchronize()
    return p


@pytest.mark.parametrize("weight_mode", [G.ABC_W_PAPER, G.ABC_W_IMPORTANCE])
def test_single_rank_driver_equals_context(weight_mode):
    from paper_2106_15508_gb300 import shard
    N, M = 2048, 1000
    cfg = saird_config(N, 30, 100_000, seed=41, batch_size=M, weight_mode=weight_mode)
    obs = oracle_obs(cfg)[0]
    ctx = G.abc_init(cfg, obs)
    try:
        G.abc_generation(ctx)  # stage 0
        pop = _device_population(ctx, N)
        be = shard.CudaBackend(cfg, obs, N, M)
        comm = shard.Comm(1, 0)
        eps1 = 0.0
        for t in range(1, 5):
            new, st = shard.generation(be, comm, t, eps1, pop, N, M, cfg.survival_alpha,
                                       cfg.weight_mode, cfg.max_batches)
            assert G.abc_generation(ctx) == G.ABC_OK and st.status == 0
            ref = _device_population(ctx, N)
            g = G.abc_get_stats(ctx, t)
            assert (st.eps, st.eps1, st.batches, st.accepted, st.exhausted) == \
                   (g.eps, g.eps1, g.batches, g.accepted, g.exhausted), t
            assert st.ess == g.ess, t
            for a, b in ((new.u, ref.u), (new.d, ref.d), (new.W, ref.W), (new.s, ref.s),
                         (new.anc, ref.anc)):
                assert torch.equal(a.view(torch.uint8), b.view(torch.uint8)), t
            eps1, pop = st.eps1, new
    finally:
        G.abc_free(ctx)


def test_single_rank_driver_mcmc_step_equals_context():
    """The MCMC baseline through the driver: the step adapts on the host
    after every batch (McmcStep, IEEE double) and walks on the device as
    the proposal kernel's fixed step; four generations equal a context whose
    step adapts on the device, bit for bit, the steps included."""
    from paper_2106_15508_gb300 import shard
    N, M = 2048, 700
    cfg = saird_config(N, 30, 100_000, seed=43, batch_size=M, weight_mode=G.ABC_W_PAPER,
                       beta_mode=G.ABC_STEP_MCMC, mcmc_s0=0.03, mcmc_adapt=9, max_batches=400)
    obs = oracle_obs(cfg)[0]
    ctx = G.abc_init(cfg, obs)
    try:
        G.abc_generation(ctx)  # stage 0
        pop = _device_population(ctx, N)
        be = shard.CudaBackend(cfg, obs, N, M)
        comm = shard.Comm(1, 0)
        mcmc = shard.McmcStep.start(cfg)
        eps1 = 0.0
        for t in range(1, 5):
            s_first = mcmc.step32()
            new, st = shard.generation(be, comm, t, eps1, pop, N, M, cfg.survival_alpha,
                                       cfg.weight_mode, cfg.max_batches, mcmc=mcmc)
            assert G.abc_generation(ctx) == G.ABC_OK and st.status == 0
            ref = _device_population(ctx, N)
            g = G.abc_get_stats(ctx, t)
            assert (st.eps, st.batches, st.accepted, st.exhausted) == \
                   (g.eps, g.batches, g.accepted, g.exhausted), t
            assert np.float32(g.beta_a) == np.float32(s_first)
            assert np.float32(g.mcmc_s) == np.float32(mcmc.s), t
            for a, b in ((new.u, ref.u), (new.d, ref.d), (new.s, ref.s), (new.anc, ref.anc)):
                assert torch.equal(a.view(torch.uint8), b.view(torch.uint8)), t
            eps1, pop = st.eps1, new
        assert mcmc.k == 9
    finally:
        G.abc_free(ctx)
