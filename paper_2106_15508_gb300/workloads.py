"""Synthetic workloads: sizes and input recipe only (no method arithmetic).

The paper fits 120 days of the JHU Italy series (Sec. 4); that data is not
available here, so observed series are simulated from a seeded true theta*
drawn in a growing-epidemic sub-box of the prior (abc_synth_obs), with
A0 = max(10, round(1e-4 P)), R0 = D0 = 0.
"""
import dataclasses

from . import (ABC_BETA_FIXED, ABC_BETA_PAPER, ABC_P_BF16_TC, ABC_P_FP32, ABC_W_IMPORTANCE,
               ABC_W_PAPER, config)

SAIRD_THETA_MAX = (1.0, 100.0, 2.0, 1.0, 1.0, 1.0, 1.0, 2.0)  # Eq. 2
OBS_BOX_LO = (0.2, 10.0, 0.5, 0.02, 0.05, 0.005, 0.2, 0.5)
OBS_BOX_HI = (0.6, 90.0, 1.5, 0.1, 0.3, 0.03, 0.8, 1.5)


def initial_active(P: int) -> int:
    return max(10, int(round(1e-4 * P)))


@dataclasses.dataclass
class Workload:
    name: str
    N: int                 # particles kept per generation
    T: int                 # days
    P: int                 # population
    G: int                 # generations
    beta_mode: int = ABC_BETA_PAPER
    beta_a: float = 2.0
    beta_b: int = 5
    weight_mode: int = ABC_W_IMPORTANCE
    weight_prec: int = ABC_P_FP32
    M: int = 0             # proposals per batch (0: N)
    alpha: float = 0.5
    max_batches: int = 64
    seed: int = 1

    def config(self, **over):
        kw = dict(n_days=self.T, population=self.P, init_ard=[initial_active(self.P), 0, 0],
                  theta_hi=list(SAIRD_THETA_MAX), seed=self.seed, n_particles=self.N,
                  batch_size=self.M, beta_mode=self.beta_mode, beta_a=self.beta_a,
                  beta_b=self.beta_b, weight_mode=self.weight_mode,
                  weight_prec=self.weight_prec, survival_alpha=self.alpha,
                  max_batches=self.max_batches)
        kw.update(over)
        return config(**kw)


# Config 1: plain ABC-SMC, Beta(2,5) steps, 4096 particles, P = 1e5, 60 days, 8 generations
SMALL = Workload("saird_n4096_t60_p1e5", N=4096, T=60, P=100_000, G=8, beta_mode=ABC_BETA_FIXED,
                 beta_a=2.0, beta_b=5)
# Config 2: single run at scale, 2^20 particles, P = 1e7, 120 days, 20 generations
LARGE = Workload("saird_n1048576_t120_p1e7", N=1 << 20, T=120, P=10_000_000, G=20)

WORKLOADS = {w.name: w for w in (SMALL, LARGE)}


def batched_runs(n_runs=64, seed=0, weight_prec=ABC_P_FP32):
    """Batched workload: n_runs independent runs with seeds 1..n_runs,
    N_r = 2^(14 + floor(5 U)) particles (16K-256K), T_r ~ U{60..180} days,
    P_r = 10^(6 + 2 U) (1e6-1e8), paper Beta schedule, importance weights."""
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n_runs):
        N = 1 << (14 + int(np.floor(5 * rng.random())))
        T = int(rng.integers(60, 181))
        P = int(round(10 ** (6 + 2 * rng.random())))
        out.append(Workload("batched_run%d" % r, N=N, T=T, P=P, G=8, seed=r + 1,
                            weight_prec=weight_prec))
    return out

def stress_runs(n_runs=32, weight_prec=ABC_P_BF16_TC):
    """Stress workload: n_runs concurrent runs of 2^20 particles, 365 days,
    P = 3.3e8, seeds 1..n_runs, paper Beta schedule, importance weights."""
    return [Workload("stress_run%d" % r, N=1 << 20, T=365, P=330_000_000, G=25, seed=r + 1,
                     weight_prec=weight_prec) for r in range(n_runs)]


__all__ = ["Workload", "SMALL", "LARGE", "WORKLOADS", "batched_runs", "stress_runs", "OBS_BOX_LO", "OBS_BOX_HI",
           "SAIRD_THETA_MAX", "initial_active", "ABC_W_PAPER", "ABC_P_BF16_TC"]
