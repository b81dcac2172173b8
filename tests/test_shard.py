"""One run sharded over ranks (paper_2106_15508_gb300.shard): proposal slots
and weight rows in contiguous blocks per rank, the batch and the log
weights all-gathered.  On CPU ranks (gloo, world sizes 2 and 3) with the
oracle's steps as the local backend, three generations must equal the
unsharded oracle's generations bit for bit -- populations, tolerances,
batch counts, weights -- for the paper's weights and for importance
weights, with slot and row blocks of unequal sizes, and for the MCMC
baseline, whose step adapts after every batch on every rank."""
import math
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleBackend:
    """The local steps by the CPU oracle, on torch CPU tensors (test only)."""

    def __init__(self, m, c):
        import oracle as O
        self.O, self.m, self.c = O, m, c

    def empty_population(self, N):
        from paper_2106_15508_gb300 import shard
        return shard.Population(torch.zeros((8, N), dtype=torch.float32),
                                torch.zeros(N, dtype=torch.float64),
                                torch.zeros(N, dtype=torch.float64),
                                torch.zeros(N, dtype=torch.float32),
                                torch.zeros(N, dtype=torch.int32))

    def kth(self, d, k):
        return float(self.O.kth(d.numpy(), k))

    def prefix(self, d, W, eps, mode):
        q, pre, tot = self.O.resample_prefix(d.numpy(), W.numpy(), eps, mode)
        return torch.from_numpy(q.view(np.int32)), torch.from_numpy(pre.view(np.int64)), tot

    def propose(self, u, prefix, total, eps, eps1, t, c1, lo, count, s_fixed=None):
        c = self.c
        ratio = eps / eps1 if eps1 > 0 else 1.0
        if s_fixed is None:
            a, bf, bb = self.O.beta_shape(c.beta_mode, ratio, t, c.beta_a, c.beta_b, c.beta_p1,
                                          c.beta_p2)
        else:
            a, bf, bb = 0.0, 0.0, 0
        o = self.O.propose(self.m, u.numpy(), prefix.numpy().view(np.uint64), total, a, bb, count,
                           c1, c.max_redraw, c0_idx=np.arange(lo, lo + count, dtype=np.uint32),
                           beta_bf=bf, s_fixed=s_fixed or 0.0)
        self._lo = lo
        return {k: torch.from_numpy(np.ascontiguousarray(o[k])) for k in ("u", "s", "anc", "flag")}

    def simulate(self, u, c1, lo, count, flag):
        d = self.O.simulate(self.m, u.numpy(), c1=c1, c0_idx=np.arange(lo, lo + count,
                                                                       dtype=np.uint32),
                            skip=flag.numpy())
        return torch.from_numpy(d)

    def accept(self, batch, eps, new, filled):
        N = new.d.numel()
        fl, d = batch["flag"].numpy(), batch["d"].numpy()
        acc = np.nonzero((fl == 0) & (d <= eps))[0]
        take = acc[: max(0, N - filled)]
        sl = slice(filled, filled + len(take))
        new.u[:, sl] = batch["u"][:, take]
        new.d[sl] = batch["d"][take]
        new.s[sl] = batch["s"][take]
        new.anc[sl] = batch["anc"][take]
        return filled + len(take), len(acc), int((fl == 1).sum())

    def weights(self, up, s, u, q, prefix, total):
        lw = self.O.weights(up.numpy(), s.numpy(), u.numpy(), q.numpy().view(np.uint32), total)
        return torch.from_numpy(lw)

    def normalize(self, logW):
        W, ess = self.O.normalize(logW.numpy())
        return torch.from_numpy(W), float(ess)


def _setup_run(weight_mode, method="bdss"):
    import oracle as O
    from paper_2106_15508_gb300 import workloads as WL
    P, T, N = 100_000, 20, 500
    m = O.OracleModel(T=T, P=P, A0=WL.initial_active(P), seed=3)
    obs, _, _ = O.synth_obs(m)
    m.set_obs(obs)
    # M = 37 slots per batch: blocks of 19/18 (two ranks) or 13/12/12 (three)
    mode = O.MCMC_MODE if method == "mcmc" else 0
    c = O.make_smc(N, M=37, beta_mode=mode, weight_mode=weight_mode, max_batches=400,
                   mcmc_s0=0.02, mcmc_adapt=40)
    return m, c


def _worker(rank, ws, port, weight_mode, method, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import oracle as O
        from paper_2106_15508_gb300 import shard
        m, c = _setup_run(weight_mode, method)
        pop0 = O.generation0(m, c)
        ms = O.mcmc_start(c)
        mcmc = shard.McmcStep(ms.s, 0, 0, O.mcmc_window(c)) if method == "mcmc" else None
        pop = shard.Population(torch.from_numpy(pop0.u.copy()), torch.from_numpy(pop0.d.copy()),
                               torch.from_numpy(pop0.W.copy()), torch.from_numpy(pop0.s.copy()),
                               torch.from_numpy(pop0.anc.copy()))
        be = OracleBackend(m, c)
        comm = shard.Comm(ws, rank)
        eps1, res = 0.0, []
        for t in range(1, 4):
            pop, st = shard.generation(be, comm, t, eps1, pop, c.N, c.M, c.alpha, c.weight_mode,
                                       c.max_batches, mcmc=mcmc)
            assert st.status == 0
            eps1 = st.eps1
            res.append((st.eps, st.eps1, st.batches, st.accepted, st.exhausted, st.ess,
                        pop.u.numpy().copy(), pop.d.numpy().copy(), pop.W.numpy().copy(),
                        pop.s.numpy().copy(), pop.anc.numpy().copy(),
                        (mcmc.s, mcmc.k, mcmc.batches) if mcmc else None))
        out[rank] = res
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws,weight_mode,method", [(2, 0, "bdss"), (3, 1, "bdss"), (2, 1, "bdss"),
                                                    (2, 0, "mcmc"), (3, 1, "mcmc")])
def test_sharded_generations_equal_the_unsharded_oracle(ws, weight_mode, method):
    sys.path.insert(0, ROOT)
    import oracle as O
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(ws, port, weight_mode, method, out), nprocs=ws,
                           join=True, start_method="spawn")
        res = dict(out)
    m, c = _setup_run(weight_mode, method)
    pop = O.generation0(m, c)
    ms = O.mcmc_start(c) if method == "mcmc" else None
    eps1 = 0.0
    for t in range(1, 4):
        new, st = O.generation(m, c, t, eps1, pop, ms)
        assert st.status == 0
        for rank in range(ws):
            eps, e1, batches, acc, exh, ess, u, d, W, s, anc, step = res[rank][t - 1]
            if ms is not None:
                assert step == (ms.s, ms.k, ms.batches), (rank, t)
            assert (eps, e1, batches, acc, exh) == (st.eps, st.eps1, st.batches,
                                                    st.accepted_total, st.exhausted), (rank, t)
            assert ess == st.ess or (math.isnan(ess) and math.isnan(st.ess))
            for g, o in ((u, new.u), (d, new.d), (W, new.W), (s, new.s), (anc, new.anc)):
                assert np.array_equal(np.ascontiguousarray(g).view(np.uint8),
                                      np.ascontiguousarray(o).view(np.uint8)), (rank, t)
        eps1, pop = st.eps1, new


def test_blocks_cover_every_slot_once():
    sys.path.insert(0, ROOT)
    from paper_2106_15508_gb300 import shard
    for n in (0, 1, 7, 37, 1000):
        for ws in (1, 2, 3, 8):
            blocks = [shard.block(n, r, ws) for r in range(ws)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            assert all(b[1] == nb[0] for b, nb in zip(blocks, blocks[1:]))
            sizes = [hi - lo for lo, hi in blocks]
            assert max(sizes) - min(sizes) <= 1
