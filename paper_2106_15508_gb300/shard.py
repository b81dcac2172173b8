"""One ABC-SMC run sharded over several ranks (one GPU each).

Proposal slots and weight rows are split into contiguous blocks, one per
rank; what a generation needs from the other ranks arrives by all-gathers:

  * tolerance (Eq. 8) and stage prior with its prefix (Eq. 9-11): every rank
    holds the whole population, so each computes the same eps_t, q and prefix
    (replicated, cheap next to the simulations);
  * each batch (Sec. 3.1, Eq. 16-17): rank r proposes and simulates slots
    [lo_r, hi_r) of the batch with the global slot indices as Philox
    counters, then the batch is all-gathered in slot order and every rank
    appends the acceptances in (batch, slot) order, so all ranks hold the
    same new population and the same batch count;
  * importance weights (the O(N^2) sum): rank r computes the rows of its
    block against all surviving columns, the log weights are all-gathered
    and every rank normalises them (fp64).

Every Philox counter is the one of the unsharded run, so the result equals
the single-rank generation bit for bit, whatever the number of ranks.  The
MCMC baseline (one tuned step, Sec. 2.4.1 and 3.1) adapts its step after
each batch from the all-gathered batch's counts, on every rank alike.

The local steps come from a backend object (the CUDA library's entry points
on the rank's GPU, `CudaBackend`); the exchanges from torch.distributed
(NCCL between GPUs, gloo between host processes).  Arrays are torch tensors
of the backend's device.
"""
import dataclasses
import math

import torch

from . import (ABC_BETA_PAPER, ABC_OK, ABC_STEP_MCMC, ABC_W_IMPORTANCE, TAG_SIM, abc_accept_append,
               abc_accept_scratch_bytes, abc_normalize, abc_normalize_scratch_bytes, abc_prefix_scratch_bytes,
               abc_propose, abc_resample_prefix, abc_select_kth, abc_select_scratch_bytes, abc_simulate,
               abc_weights, abc_weights_scratch_bytes)


def block(n, rank, world):
    """Contiguous block [lo, hi) of n items for `rank` of `world` (sizes
    differ by at most one, the larger blocks first)."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def rank_of_slots(n, world):
    return [block(n, r, world) for r in range(world)]


class Comm:
    """All-gathers along the last axis over torch.distributed (or a single
    process when world == 1)."""

    def __init__(self, world=1, rank=0, group=None):
        self.world, self.rank, self.group = world, rank, group

    def allgather_last(self, x, n):
        """x: this rank's block (last axis); returns the n items of all ranks
        in rank order."""
        if self.world == 1:
            return x
        import torch.distributed as dist
        blocks = rank_of_slots(n, self.world)
        width = max(hi - lo for lo, hi in blocks)
        pad = torch.zeros(x.shape[:-1] + (width,), dtype=x.dtype, device=x.device)
        pad[..., : x.shape[-1]] = x
        parts = [torch.empty_like(pad) for _ in range(self.world)]
        dist.all_gather(parts, pad.contiguous(), group=self.group)
        return torch.cat([p[..., : hi - lo] for p, (lo, hi) in zip(parts, blocks)], dim=-1)


@dataclasses.dataclass
class Population:
    u: torch.Tensor    # [8][N] float32
    d: torch.Tensor    # [N] float64
    W: torch.Tensor    # [N] float64
    s: torch.Tensor    # [N] float32
    anc: torch.Tensor  # [N] int32


@dataclasses.dataclass
class McmcStep:
    """The MCMC baseline's tuned step across generations: s (a variance in
    unit-cube coordinates, fp64), the adaptations made, the batches walked
    with the step so far and the adaptation window in batches."""
    s: float
    k: int = 0
    batches: int = 0
    window: int = 0

    @classmethod
    def start(cls, cfg):
        """After generation 0: s = mcmc_s0 (as fp32), the window mcmc_adapt
        or a tenth of the run budget."""
        import numpy as np
        window = cfg.mcmc_adapt if cfg.mcmc_adapt > 0 else -(-cfg.max_total_batches // 10)
        return cls(float(np.float32(cfg.mcmc_s0)), 0, 0, window)

    def step32(self):
        import numpy as np
        return float(np.float32(self.s))

    def adapt(self, accepted, simulated):
        """After a batch (Eq. 14-15 as the library reads them): inside the
        window s <- s (1 + (A - A_T) / ((1 - A_T)(k + 1))), A = accepted /
        simulated (0 if none), A_T = 0.234; IEEE double operations in the
        library's order."""
        if self.batches < self.window:
            a_t = 0.234
            a = accepted / simulated if simulated > 0 else 0.0
            gain = (1.0 - a_t) * float(self.k + 1)
            self.s = self.s * (1.0 + (a - a_t) / gain)
            self.k += 1
        self.batches += 1


@dataclasses.dataclass
class GenStats:
    eps: float = 0.0
    eps1: float = 0.0
    batches: int = 0
    accepted: int = 0
    exhausted: int = 0
    ess: float = 0.0
    status: int = ABC_OK


def generation(backend, comm, t, eps1, pop, N, M, alpha, weight_mode, max_batches, mcmc=None):
    """Generation t >= 1 from the (replicated) population `pop`; returns the
    new population (replicated on every rank) and the statistics.  Slots of
    a batch and rows of the weight pass are split over the ranks.  mcmc: the
    McmcStep of an MCMC-baseline run (updated in place), else None."""
    st = GenStats()
    k = min(max(math.ceil(alpha * N), 1), N)  # the lower order statistic of rank ceil(alpha N)
    eps = backend.kth(pop.d, k)
    eps1 = eps if t == 1 else eps1
    st.eps, st.eps1 = eps, eps1
    q, prefix, total = backend.prefix(pop.d, pop.W, eps, weight_mode)
    lo, hi = block(M, comm.rank, comm.world)
    new = backend.empty_population(N)
    filled = 0
    b = 0
    while b < max_batches and filled < N:
        c1 = (t << 16) | b
        mine = backend.propose(pop.u, prefix, total, eps, eps1, t, c1, lo, hi - lo,
                               s_fixed=mcmc.step32() if mcmc is not None else None)
        d_mine = backend.simulate(mine["u"], c1, lo, hi - lo, mine["flag"])
        batch = {"u": comm.allgather_last(mine["u"], M), "d": comm.allgather_last(d_mine, M),
                 "s": comm.allgather_last(mine["s"], M), "anc": comm.allgather_last(mine["anc"], M),
                 "flag": comm.allgather_last(mine["flag"], M)}
        filled, acc, exh = backend.accept(batch, eps, new, filled)
        st.accepted += acc
        st.exhausted += exh
        if mcmc is not None:
            mcmc.adapt(acc, M - exh)
        b += 1
    st.batches = b
    if filled < N:
        st.status = 1  # the batch budget ran out: the population is kept
        return pop, st
    if weight_mode == ABC_W_IMPORTANCE:
        rlo, rhi = block(N, comm.rank, comm.world)
        lw = backend.weights(new.u[:, rlo:rhi], new.s[rlo:rhi], pop.u, q, prefix, total)
        logW = comm.allgather_last(lw, N)
        new.W, st.ess = backend.normalize(logW)
    else:
        new.W = torch.full((N,), 1.0 / N, dtype=torch.float64, device=new.W.device)
        st.ess = float(N)
    return new, st


class CudaBackend:
    """The local steps on this rank's GPU through the library's C ABI (step
    entry points on device buffers of the process's current stream)."""

    def __init__(self, cfg, obs, N, M):
        dev = torch.device("cuda", torch.cuda.current_device())
        self.cfg, self.N, self.M, self.dev = cfg, N, M, dev
        self.obs = torch.as_tensor(obs, dtype=torch.int32).to(dev).contiguous() \
            if obs is not None else None
        nb = max(abc_select_scratch_bytes(N), abc_prefix_scratch_bytes(N),
                 abc_accept_scratch_bytes(M), abc_normalize_scratch_bytes(N),
                 abc_weights_scratch_bytes(N, N))
        self.scratch = torch.empty(nb, dtype=torch.uint8, device=dev)
        self.scal = torch.zeros(4, dtype=torch.float64, device=dev)  # eps, eps1, ess

    def _sc(self):
        return self.scratch, self.scratch.numel()

    def empty_population(self, N):
        d = self.dev
        return Population(torch.zeros((8, N), dtype=torch.float32, device=d),
                          torch.zeros(N, dtype=torch.float64, device=d),
                          torch.zeros(N, dtype=torch.float64, device=d),
                          torch.zeros(N, dtype=torch.float32, device=d),
                          torch.zeros(N, dtype=torch.int32, device=d))

    def kth(self, d, k):
        abc_select_kth(d, d.numel(), k, self.scal[0:1], *self._sc())
        return float(self.scal[0].item())

    def prefix(self, d, W, eps, mode):
        n = d.numel()
        self.scal[0] = eps
        q = torch.empty(n, dtype=torch.int32, device=self.dev)
        pre = torch.empty(n, dtype=torch.int64, device=self.dev)
        abc_resample_prefix(d, W, n, self.scal[0:1], mode, q, pre, *self._sc())
        return q, pre, int(pre[-1].item()) & ((1 << 64) - 1)

    def propose(self, u, prefix, total, eps, eps1, t, c1, lo, count, s_fixed=None):
        self.scal[0], self.scal[1] = eps, eps1
        c0 = torch.arange(lo, lo + count, dtype=torch.int32, device=self.dev)
        out = {"u": torch.empty((8, count), dtype=torch.float32, device=self.dev),
               "s": torch.empty(count, dtype=torch.float32, device=self.dev),
               "anc": torch.empty(count, dtype=torch.int32, device=self.dev),
               "att": torch.empty(count, dtype=torch.int32, device=self.dev),
               "flag": torch.empty(count, dtype=torch.uint8, device=self.dev)}
        paper = self.cfg.beta_mode == ABC_BETA_PAPER
        bb = (2 * t if t <= 512 else 0) if paper else self.cfg.beta_b
        # the MCMC baseline walks with the run's step (beta_a under ABC_STEP_MCMC)
        a = s_fixed if self.cfg.beta_mode == ABC_STEP_MCMC else self.cfg.beta_a
        abc_propose(self.cfg, u, u.shape[1], prefix, self.scal[0:1], self.scal[1:2],
                    a, bb, count, c0, c1, out["u"], out["s"], out["anc"],
                    out["att"], out["flag"])
        self._c0 = c0
        return out

    def simulate(self, u, c1, lo, count, flag):
        d = torch.empty(count, dtype=torch.float64, device=self.dev)
        abc_simulate(self.cfg, self.obs, u, count, self._c0, c1, TAG_SIM, flag, d)
        return d

    def accept(self, batch, eps, new, filled):
        self.scal[0] = eps
        M = batch["d"].numel()
        f = torch.tensor([filled], dtype=torch.int64, device=self.dev)
        cnt = torch.zeros(2, dtype=torch.int64, device=self.dev)
        abc_accept_append(batch["u"].contiguous(), batch["d"], batch["s"], batch["anc"],
                          batch["flag"], M, self.scal[0:1], self.N, new.u, new.d, new.s, new.anc,
                          f, cnt, *self._sc())
        c = cnt.tolist()
        return int(f.item()), int(c[0]), int(c[1])

    def weights(self, up, s, u, q, prefix, total):
        rows = up.shape[1]
        lw = torch.empty(rows, dtype=torch.float64, device=self.dev)
        abc_weights(up.contiguous(), s.contiguous(), rows, u, q, prefix, u.shape[1],
                    self.cfg.weight_prec, lw, *self._sc())
        return lw

    def normalize(self, logW):
        n = logW.numel()
        W = torch.empty(n, dtype=torch.float64, device=self.dev)
        abc_normalize(logW, n, W, self.scal[2:3], *self._sc())
        return W, float(self.scal[2].item())


__all__ = ["block", "Comm", "Population", "GenStats", "McmcStep", "generation", "CudaBackend"]
