"""Glue for the parity tests: one configuration expressed for both the CUDA
library (AbcConfig) and the CPU oracle (Model/Smc), plus torch transfers."""
import ctypes
import struct

import numpy as np

import oracle as O
import paper_2106_15508_gb300 as G
from paper_2106_15508_gb300 import workloads as WL


def oracle_model(cfg, obs=None):
    m = O.OracleModel(model=cfg.model, sampler=cfg.sampler, T=cfg.n_days, P=cfg.population,
                      A0=cfg.init_ard[0], R0=cfg.init_ard[1], D0=cfg.init_ard[2],
                      theta_lo=list(cfg.theta_lo), theta_hi=list(cfg.theta_hi),
                      x_obs=list(cfg.x_obs), seed=cfg.seed, run=cfg.run_id)
    m.set_obs(obs)
    return m


def oracle_smc(cfg, nthreads=8):
    return O.make_smc(cfg.n_particles, M=cfg.batch_size or cfg.n_particles,
                      alpha=cfg.survival_alpha, beta_mode=cfg.beta_mode, beta_a=cfg.beta_a,
                      beta_b=cfg.beta_b, weight_mode=cfg.weight_mode,
                      max_batches=cfg.max_batches, max_redraw=cfg.max_redraw, nthreads=nthreads,
                      beta_p1=cfg.beta_p1, beta_p2=cfg.beta_p2, max_total=cfg.max_total_batches,
                      mcmc_s0=cfg.mcmc_s0, mcmc_adapt=cfg.mcmc_adapt)


def saird_config(N, T, P, seed=1, **kw):
    A0 = WL.initial_active(P)
    base = dict(n_days=T, population=P, init_ard=[A0, 0, 0], seed=seed, n_particles=N,
                theta_hi=list(WL.SAIRD_THETA_MAX))
    base.update(kw)
    return G.config(**base)


def oracle_obs(cfg):
    """Synthetic observations written by the oracle (the CUDA path is checked
    against the same series separately)."""
    obs, th, att = O.synth_obs(oracle_model(cfg))
    return obs, th, att


def state_blob(cfg, gen, eps1, pop, batches_total=0, mcmc=None):
    """abc_set_state layout: magic, N, T, seed, run_id, gen, eps1, the run
    budget count, then u [8][N] f32, dist f64, W f64, s f32, anc i32; for
    the MCMC baseline the step state (s f64, adaptations i64, batches i64)
    follows (mcmc = (s, k, batches))."""
    N = cfg.n_particles
    T = cfg.n_days if cfg.model == G.ABC_MODEL_SAIRD else 0
    head = struct.pack("<8sqqQIidq", b"ABCSMC02", N, T, cfg.seed, cfg.run_id, gen, eps1,
                       batches_total)
    return b"".join([head, np.ascontiguousarray(pop.u, np.float32).tobytes(),
                     np.ascontiguousarray(pop.d, np.float64).tobytes(),
                     np.ascontiguousarray(pop.W, np.float64).tobytes(),
                     np.ascontiguousarray(pop.s, np.float32).tobytes(),
                     np.ascontiguousarray(pop.anc, np.int32).tobytes(),
                     b"" if mcmc is None else struct.pack("<dqq", *mcmc)])


def get_population(ctx, N):
    u = np.zeros((8, N), np.float32)
    d = np.zeros(N, np.float64)
    W = np.zeros(N, np.float64)
    s = np.zeros(N, np.float32)
    anc = np.zeros(N, np.int32)
    G.abc_get_population(ctx, u, d, W, s, anc)
    return dict(u=u, d=d, W=W, s=s, anc=anc)


def dev(a):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def empty(shape, dtype):
    import torch
    return torch.empty(shape, dtype=dtype, device="cuda")
