"""CPU oracle for P-ABC-SMC with Beta-distributed step sizes (arXiv 2106.15508).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py.  The product package never imports
it.  This module only marshals numpy arrays into the plain C oracle
(abc_oracle.c); all arithmetic lives there.
"""
import ctypes as C
import math

import numpy as np

from .build import build_oracle

_lib = None

TAG_PRIOR, TAG_ANCESTOR, TAG_BETA, TAG_WALK, TAG_SIM, TAG_SCREEN, TAG_AUDIT = 0, 1, 2, 3, 4, 5, 6
TAG_OBS, TAG_OBS_THETA = 7, 8
TAG_PREDICT, TAG_PREDICT_SIM = 11, 12

SAIRD_THETA_MAX = np.array([1, 100, 2, 1, 1, 1, 1, 2], np.float32)  # Eq. 2
OBS_BOX_LO = np.array([0.2, 10, 0.5, 0.02, 0.05, 0.005, 0.2, 0.5], np.float32)
OBS_BOX_HI = np.array([0.6, 90, 1.5, 0.1, 0.3, 0.03, 0.8, 1.5], np.float32)


class Model(C.Structure):
    _fields_ = [
        ("model", C.c_int32), ("sampler", C.c_int32), ("T", C.c_int32), ("pad0", C.c_int32),
        ("P", C.c_int64), ("A0", C.c_int32), ("R0", C.c_int32), ("D0", C.c_int32),
        ("pad1", C.c_int32), ("theta_lo", C.c_float * 8), ("theta_hi", C.c_float * 8),
        ("obs", C.POINTER(C.c_int32)), ("x_obs", C.c_float * 8), ("key", C.c_uint32 * 2),
    ]


class Smc(C.Structure):
    _fields_ = [
        ("N", C.c_int32), ("M", C.c_int32), ("max_total", C.c_int32), ("alpha", C.c_double),
        ("beta_mode", C.c_int32),
        ("beta_a", C.c_float), ("beta_b", C.c_int32), ("beta_p1", C.c_float),
        ("beta_p2", C.c_float), ("weight_mode", C.c_int32),
        ("max_batches", C.c_int32), ("max_redraw", C.c_int32), ("nthreads", C.c_int32),
        ("mcmc_s0", C.c_float), ("mcmc_adapt", C.c_int32),
    ]


class McmcState(C.Structure):
    """The MCMC baseline's tuned step across generations (s, adaptations
    made, batches walked with the step so far)."""
    _fields_ = [("s", C.c_double), ("k", C.c_int64), ("batches", C.c_int64)]


class GenStats(C.Structure):
    _fields_ = [
        ("eps", C.c_double), ("eps1", C.c_double), ("ess", C.c_double), ("beta_a", C.c_float),
        ("beta_b", C.c_int32), ("beta_bf", C.c_float), ("mcmc_s", C.c_float),
        ("batches", C.c_int64), ("sims", C.c_int64),
        ("exhausted", C.c_int64), ("accepted_total", C.c_int64), ("total", C.c_uint64),
        ("status", C.c_int32),
    ]


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t)) if a is not None else None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build_oracle())
        L = _lib
        L.or_uniform.restype = C.c_float
        L.or_uniform.argtypes = [C.c_uint32]
        for name in ("or_logf", "or_expf", "or_expm1f", "or_log1pf", "or_cos2pi"):
            getattr(L, name).restype = C.c_float
            getattr(L, name).argtypes = [C.c_float]
        L.or_normal.restype = C.c_float
        L.or_normal.argtypes = [C.c_float, C.c_float]
        L.or_binomial.restype = C.c_int32
        L.or_binomial.argtypes = [C.c_int32, C.c_float, C.c_float, C.c_float]
        L.or_beta.restype = C.c_float
        L.or_beta.argtypes = [C.POINTER(C.c_uint32), C.c_float, C.c_int32, C.c_uint32,
                              C.c_uint32, C.c_uint32]
        L.or_gamma_log.restype = C.c_float
        L.or_gamma_log.argtypes = [C.POINTER(C.c_uint32), C.c_float, C.c_uint32, C.c_uint32,
                                   C.c_uint32, C.c_uint32]
        L.or_beta_real.restype = C.c_float
        L.or_beta_real.argtypes = [C.POINTER(C.c_uint32), C.c_float, C.c_float, C.c_uint32,
                                   C.c_uint32, C.c_uint32]
        L.or_beta_shape.restype = None
        L.or_beta_shape.argtypes = [C.c_int32, C.c_float, C.c_int32, C.c_float, C.c_int32,
                                    C.c_float, C.c_float, C.POINTER(C.c_float),
                                    C.POINTER(C.c_int32)]
        L.or_kth.restype = C.c_double
        L.or_kth.argtypes = [C.POINTER(C.c_double), C.c_int64, C.c_int64]
        L.or_rank.restype = C.c_int64
        L.or_rank.argtypes = [C.c_double, C.c_int64]
        L.or_resample_prefix.restype = C.c_uint64
        L.or_normalize.restype = C.c_double
        L.or_synth_obs.restype = C.c_int32
        L.or_generation.restype = C.c_int32
        L.or_mcmc_adapt.restype = C.c_double
        L.or_mcmc_adapt.argtypes = [C.c_double, C.c_int64, C.c_int64, C.c_int64]
        L.or_mcmc_window.restype = C.c_int64
    return _lib


def make_key(seed: int, run: int = 0):
    return (seed & 0xFFFFFFFF, ((seed >> 32) & 0xFFFFFFFF) ^ (run & 0xFFFFFFFF))


class OracleModel:
    """Owns a Model struct plus the arrays it points to."""

    def __init__(self, *, model=0, sampler=0, T=60, P=100000, A0=10, R0=0, D0=0,
                 theta_lo=None, theta_hi=None, obs=None, x_obs=None, seed=1, run=0):
        self.s = Model()
        self.s.model, self.s.sampler, self.s.T, self.s.P = model, sampler, T, P
        self.s.A0, self.s.R0, self.s.D0 = A0, R0, D0
        lo = np.zeros(8, np.float32) if theta_lo is None else np.asarray(theta_lo, np.float32)
        hi = SAIRD_THETA_MAX if theta_hi is None else np.asarray(theta_hi, np.float32)
        self.s.theta_lo[:] = [float(v) for v in lo]
        self.s.theta_hi[:] = [float(v) for v in hi]
        self.s.x_obs[:] = [0.0] * 8 if x_obs is None else [float(v) for v in x_obs]
        k = make_key(seed, run)
        self.s.key[0], self.s.key[1] = k
        self.key = np.array(k, np.uint32)
        self.T = T
        self.set_obs(obs)

    def set_obs(self, obs):
        if obs is None:
            self.obs = None
            self.s.obs = None
        else:
            self.obs = np.ascontiguousarray(obs, np.int32).reshape(3, self.T + 1)
            self.s.obs = _p(self.obs, C.c_int32)

    def ref(self):
        return C.byref(self.s)


def philox(ctr, key):
    out = np.zeros(4, np.uint32)
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    lib().or_philox(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def constants():
    out = np.zeros(24, np.float32)
    lib().or_constants(_p(out, C.c_float), 24)
    return out


def fn(name):
    f = getattr(lib(), name)
    return lambda x: f(float(np.float32(x)))


def uniform(x):
    return lib().or_uniform(int(x))


def normal(w1, w2):
    return lib().or_normal(float(w1), float(w2))


def binomial(n, p, w1, w2):
    return lib().or_binomial(int(n), float(np.float32(p)), float(np.float32(w1)),
                             float(np.float32(w2)))


def beta(key, a, b, c0, c1, attempt):
    k = np.ascontiguousarray(key, np.uint32)
    return lib().or_beta(_p(k, C.c_uint32), float(np.float32(a)), int(b), c0, c1, attempt)


def gamma_log(key, alpha, c0, c1, attempt, blk0=0):
    k = np.ascontiguousarray(key, np.uint32)
    return lib().or_gamma_log(_p(k, C.c_uint32), float(np.float32(alpha)), c0, c1, attempt, blk0)


def beta_real(key, a, b, c0, c1, attempt):
    k = np.ascontiguousarray(key, np.uint32)
    return lib().or_beta_real(_p(k, C.c_uint32), float(np.float32(a)), float(np.float32(b)),
                              c0, c1, attempt)


BETA_PAPER, BETA_FIXED, BETA_REAL, BETA_MEAN_VAR, BETA_MODE_CONC = 0, 1, 2, 3, 4


def beta_shape(mode, ratio, t, fa=2.0, fb=5, p1=0.0, p2=0.0):
    """(a, b, integer b or 0) of stage t under a step-size Beta rule."""
    out = (C.c_float * 2)()
    bi = C.c_int32()
    lib().or_beta_shape(mode, float(np.float32(ratio)), t, fa, fb, p1, p2, out, C.byref(bi))
    return float(out[0]), float(out[1]), int(bi.value)


def simulate(m: OracleModel, u, c1=0, tag=TAG_SIM, c0_idx=None, skip=None, traj=False,
             nthreads=1):
    u = np.ascontiguousarray(u, np.float32)
    n = u.shape[1]
    dist = np.zeros(n, np.float64)
    tr = np.zeros((m.T + 1, 6, n), np.int32) if traj else None
    c0 = None if c0_idx is None else np.ascontiguousarray(c0_idx, np.uint32)
    sk = None if skip is None else np.ascontiguousarray(skip, np.uint8)
    lib().or_simulate(m.ref(), _p(u, C.c_float), C.c_int64(n), _p(c0, C.c_uint32),
                      C.c_uint32(c1), C.c_uint32(tag), _p(sk, C.c_uint8), _p(dist, C.c_double),
                      _p(tr, C.c_int32), C.c_int(nthreads))
    return (dist, tr) if traj else dist


def synth_obs(m: OracleModel, lo=OBS_BOX_LO, hi=OBS_BOX_HI):
    obs = np.zeros((3, m.T + 1), np.int32)
    th = np.zeros(8, np.float32)
    lo = np.ascontiguousarray(lo, np.float32)
    hi = np.ascontiguousarray(hi, np.float32)
    att = lib().or_synth_obs(m.ref(), _p(lo, C.c_float), _p(hi, C.c_float), _p(obs, C.c_int32),
                             _p(th, C.c_float))
    return obs, th, att


def prior(m: OracleModel, n):
    u = np.zeros((8, n), np.float32)
    lib().or_prior(m.ref(), C.c_int64(n), _p(u, C.c_float))
    return u


def rank(alpha, n):
    return lib().or_rank(float(alpha), int(n))


def kth(d, k):
    d = np.ascontiguousarray(d, np.float64)
    return lib().or_kth(_p(d, C.c_double), len(d), int(k))


def resample_prefix(d, W, eps, mode):
    d = np.ascontiguousarray(d, np.float64)
    W = np.ascontiguousarray(W if W is not None else np.zeros_like(d), np.float64)
    n = len(d)
    q = np.zeros(n, np.uint32)
    pre = np.zeros(n, np.uint64)
    tot = lib().or_resample_prefix(_p(d, C.c_double), _p(W, C.c_double), C.c_int64(n),
                                   C.c_double(eps), C.c_int(mode), _p(q, C.c_uint32),
                                   _p(pre, C.c_uint64))
    return q, pre, int(tot)


def propose(m: OracleModel, u, prefix, total, beta_a, beta_b, slots, c1, max_redraw=64,
            c0_idx=None, nthreads=1, beta_bf=0.0, s_fixed=0.0):
    """beta_b >= 1: s ~ Beta(beta_a, beta_b) by the product form; beta_b = 0:
    s ~ Beta(beta_a, beta_bf) by the Gamma ratio; s_fixed > 0: the MCMC
    baseline's single step s = s_fixed for every slot."""
    u = np.ascontiguousarray(u, np.float32)
    prefix = np.ascontiguousarray(prefix, np.uint64)
    n = u.shape[1]
    up = np.zeros((8, slots), np.float32)
    s = np.zeros(slots, np.float32)
    anc = np.zeros(slots, np.int32)
    att = np.zeros(slots, np.int32)
    fl = np.zeros(slots, np.uint8)
    c0 = None if c0_idx is None else np.ascontiguousarray(c0_idx, np.uint32)
    lib().or_propose(m.ref(), _p(u, C.c_float), C.c_int64(n), _p(prefix, C.c_uint64),
                     C.c_uint64(total), C.c_float(beta_a), C.c_int32(beta_b),
                     C.c_float(beta_bf), C.c_float(s_fixed), C.c_int64(slots),
                     _p(c0, C.c_uint32), C.c_uint32(c1), C.c_int32(max_redraw), _p(up, C.c_float),
                     _p(s, C.c_float), _p(anc, C.c_int32), _p(att, C.c_int32), _p(fl, C.c_uint8),
                     C.c_int(nthreads))
    return dict(u=up, s=s, anc=anc, attempts=att, flag=fl)


def weights(up, s, u, q, total, nthreads=1):
    up = np.ascontiguousarray(up, np.float32)
    s = np.ascontiguousarray(s, np.float32)
    u = np.ascontiguousarray(u, np.float32)
    q = np.ascontiguousarray(q, np.uint32)
    rows, n = up.shape[1], u.shape[1]
    out = np.zeros(rows, np.float64)
    lib().or_weights(_p(up, C.c_float), _p(s, C.c_float), C.c_int64(rows), _p(u, C.c_float),
                     _p(q, C.c_uint32), C.c_int64(n), C.c_uint64(total), _p(out, C.c_double),
                     C.c_int(nthreads))
    return out


def normalize(logW):
    logW = np.ascontiguousarray(logW, np.float64)
    W = np.zeros_like(logW)
    ess = lib().or_normalize(_p(logW, C.c_double), C.c_int64(len(logW)), _p(W, C.c_double))
    return W, ess


def make_smc(N, M=None, alpha=0.5, beta_mode=0, beta_a=2.0, beta_b=5, weight_mode=0,
             max_batches=64, max_redraw=64, nthreads=1, beta_p1=0.0, beta_p2=0.0, max_total=0,
             mcmc_s0=0.1, mcmc_adapt=0):
    c = Smc()
    c.mcmc_s0, c.mcmc_adapt = mcmc_s0, mcmc_adapt
    c.N, c.M = N, (N if M is None else M)
    c.max_total = max_total
    c.alpha, c.beta_mode, c.beta_a, c.beta_b = alpha, beta_mode, beta_a, beta_b
    c.beta_p1, c.beta_p2 = beta_p1, beta_p2
    c.weight_mode, c.max_batches, c.max_redraw, c.nthreads = (weight_mode, max_batches,
                                                              max_redraw, nthreads)
    return c


class Population:
    def __init__(self, N):
        self.u = np.zeros((8, N), np.float32)
        self.d = np.zeros(N, np.float64)
        self.W = np.full(N, 1.0 / N)
        self.s = np.zeros(N, np.float32)
        self.anc = np.full(N, -1, np.int32)
        self.logW = np.zeros(N, np.float64)


def generation0(m: OracleModel, c: Smc):
    pop = Population(c.N)
    lib().or_generation0(m.ref(), C.byref(c), _p(pop.u, C.c_float), _p(pop.d, C.c_double),
                         _p(pop.W, C.c_double))
    return pop


MCMC_MODE = 5  # beta_mode of the MCMC baseline (one tuned step, Sec. 2.4.1)


def mcmc_start(c: Smc):
    """The MCMC baseline's step state after generation 0: s = mcmc_s0, no
    adaptation and no batch walked with the step yet."""
    return McmcState(float(np.float32(c.mcmc_s0)), 0, 0)


def mcmc_adapt(s, k, acc, sims):
    return lib().or_mcmc_adapt(float(s), int(k), int(acc), int(sims))


def mcmc_window(c: Smc):
    return lib().or_mcmc_window(C.byref(c))


def generation(m: OracleModel, c: Smc, t: int, eps1: float, pop: Population, mcmc=None):
    """mcmc: the McmcState of an MCMC-baseline run (updated in place)."""
    if c.beta_mode == MCMC_MODE and mcmc is None:
        raise ValueError("the MCMC baseline needs its step state")
    new = Population(c.N)
    st = GenStats()
    rc = lib().or_generation(m.ref(), C.byref(c), C.c_int32(t), C.c_double(eps1),
                             _p(pop.u, C.c_float), _p(pop.d, C.c_double), _p(pop.W, C.c_double),
                             _p(new.u, C.c_float), _p(new.d, C.c_double), _p(new.W, C.c_double),
                             _p(new.s, C.c_float), _p(new.anc, C.c_int32),
                             _p(new.logW, C.c_double), C.byref(st),
                             C.byref(mcmc) if mcmc is not None else None)
    if rc < 0:
        raise ValueError("or_generation: bad arguments")
    return new, st


def batches_gen0(c: Smc):
    """Simulation batches that generation 0 stands for: its N prior draws in
    batches of M parallel simulations (Sec. 4.1 counts simulation runs)."""
    return -(-c.N // c.M)


def run(m: OracleModel, c: Smc, G: int):
    """Generations 0..G-1; returns the final population and per-generation stats.

    A generation that exhausts its batch budget ends the run.  With
    c.max_total > 0 the run also ends after the first generation at whose end
    the simulation batches so far (generation 0 counting batches_gen0) reach
    max_total: Sec. 4.1 stops each trial on the stage that reached 1000
    simulation runs, and lets that stage finish."""
    pop = generation0(m, c)
    stats = []
    eps1 = 0.0
    total = batches_gen0(c)
    ms = mcmc_start(c) if c.beta_mode == MCMC_MODE else None
    for t in range(1, G):
        if c.max_total > 0 and total >= c.max_total:
            break
        new, st = generation(m, c, t, eps1, pop, ms)
        stats.append(st)
        total += st.batches
        if st.status != 0:
            break
        eps1 = st.eps1
        pop = new
    return pop, stats


# ---- surrogate MLP (8 -> 256 -> 256 -> 4, tanh-form GELU), fp64 -----------
MLP_SHAPES = dict(W1=(256, 8), b1=(256,), W2=(256, 256), b2=(256,), W3=(4, 256), b3=(4,))
MLP_ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


def gelu(x):
    lib().or_gelu.restype = C.c_double
    lib().or_gelu.argtypes = [C.c_double]
    return lib().or_gelu(float(x))


def _mlp_args(params):
    arrs = [np.ascontiguousarray(params[k], np.float64) for k in MLP_ORDER]
    return arrs, [_p(a, C.c_double) for a in arrs]


def mlp_forward(params, x):
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 8)
    y = np.zeros((len(x), 4))
    _, ptrs = _mlp_args(params)
    lib().or_mlp_forward(*ptrs, _p(x, C.c_double), C.c_int64(len(x)), _p(y, C.c_double))
    return y


def mlp_backward(params, x, t):
    x = np.ascontiguousarray(x, np.float64).reshape(-1, 8)
    t = np.ascontiguousarray(t, np.float64).reshape(-1, 4)
    grads = {k: np.zeros(MLP_SHAPES[k]) for k in MLP_ORDER}
    _, ptrs = _mlp_args(params)
    f = lib().or_mlp_backward
    f.restype = C.c_double
    loss = f(*ptrs, _p(x, C.c_double), _p(t, C.c_double), C.c_int64(len(x)),
             *[_p(grads[k], C.c_double) for k in MLP_ORDER])
    return loss, grads


def predict(m: OracleModel, u, W, R, days, quant):
    """Posterior-predictive order statistics: int32 [days + 1][3 (A, R, D)][nq]."""
    u = np.ascontiguousarray(u, np.float32)
    N = u.shape[1]
    Wc = None if W is None else np.ascontiguousarray(W, np.float64)
    qv = np.ascontiguousarray(quant, np.float64)
    out = np.zeros((days + 1, 3, len(qv)), np.int32)
    rc = lib().or_predict(m.ref(), _p(u, C.c_float), _p(Wc, C.c_double), C.c_int64(N),
                          C.c_int64(R), C.c_int32(days), _p(qv, C.c_double), C.c_int32(len(qv)),
                          _p(out, C.c_int32))
    if rc != 0:
        raise ValueError("or_predict: bad arguments")
    return out


def screen(m: OracleModel, Y, ystat, flag, eps, c1, tau, rho_min, audit_frac):
    """Delayed-acceptance screen: returns (rho float32[M], sflag uint8[M])."""
    Y = np.ascontiguousarray(Y, np.float32).reshape(-1, 4)
    M = len(Y)
    ystat = np.ascontiguousarray(ystat, np.float32)
    fl = None if flag is None else np.ascontiguousarray(flag, np.uint8)
    rho = np.zeros(M, np.float32)
    sflag = np.zeros(M, np.uint8)
    lib().or_screen(m.ref(), _p(Y, C.c_float), _p(ystat, C.c_float), _p(fl, C.c_uint8),
                    C.c_int64(M), C.c_double(eps), C.c_uint32(c1), C.c_float(tau),
                    C.c_float(rho_min), C.c_float(audit_frac), _p(rho, C.c_float),
                    _p(sflag, C.c_uint8))
    return rho, sflag


def adam(w, g, m, v, lr, b1, b2, eps, t):
    """in place on float64 arrays"""
    lib().or_adam(_p(w, C.c_double), _p(np.ascontiguousarray(g, np.float64), C.c_double),
                  _p(m, C.c_double), _p(v, C.c_double), C.c_int64(w.size), C.c_double(lr),
                  C.c_double(b1), C.c_double(b2), C.c_double(eps), C.c_int64(t))


__all__ = [n for n in dir() if not n.startswith("_")] + ["math"]
