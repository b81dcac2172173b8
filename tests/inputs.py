"""Seeded synthetic inputs shared by the oracle and the CUDA path in the
parity tests.  Random arrays only: none of the method's arithmetic lives
here."""
import numpy as np


def rng(seed):
    return np.random.default_rng(seed)


def unit_particles(n, seed, lo=0.0, hi=1.0):
    """[8][n] float32 unit-cube coordinates."""
    return rng(seed).uniform(lo, hi, (8, n)).astype(np.float32)


def clustered_particles(n, seed, centre=0.5, spread=0.05):
    r = rng(seed)
    return np.clip(centre + spread * r.standard_normal((8, n)), 0.0, 1.0).astype(np.float32)


def distances(n, seed, ties=False, with_inf=False):
    r = rng(seed)
    d = r.integers(0, 1000, n).astype(np.float64) if ties else r.gamma(2.0, 1e4, n)
    if with_inf:
        d[r.integers(0, n, max(1, n // 50))] = np.inf
    return d


def weights(n, seed):
    w = rng(seed).lognormal(0.0, 2.0, n)
    return w / w.sum()


def quantised_weights(n, seed, zero_frac=0.3):
    r = rng(seed)
    q = r.integers(1, 2**32, n, dtype=np.uint64).astype(np.uint32)
    q[r.random(n) < zero_frac] = 0
    if q.max() == 0:
        q[0] = 1
    return q


def step_sizes(n, seed, lo=1e-4, hi=0.5):
    return np.exp(rng(seed).uniform(np.log(lo), np.log(hi), n)).astype(np.float32)


def counters(n, seed):
    return rng(seed).integers(0, 2**32, (n, 4), dtype=np.uint64).astype(np.uint32)
