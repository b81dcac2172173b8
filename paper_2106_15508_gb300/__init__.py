"""Python binding of libabcsmc.so, the GB300 (sm_103a) implementation of
P-ABC-SMC with Beta-distributed step sizes (arXiv 2106.15508).

Argument marshalling only: every step runs in the CUDA library.  Functions
carry the names of the C entry points in include/abcsmc.h and accept device
pointers as ints or as objects with a data_ptr() (torch tensors).  Streams
default to torch's current CUDA stream.  There is no CPU fallback: importing
works without the library, but the first call raises if it is missing.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libabcsmc.so")

ABC_OK, ABC_STOP_BUDGET, ABC_STOP_TARGET, ABC_STOP_TOTAL = 0, 1, 2, 3
ABC_E_INVAL, ABC_E_NOMEM, ABC_E_CUDA, ABC_E_DEVICE, ABC_E_SCRATCH, ABC_E_STATE = -1, -2, -3, -4, -5, -6
ABC_E_TOO_LARGE = -7
ABC_NOALLOC_MAX_N = 1 << 24
ABC_MODEL_SAIRD, ABC_MODEL_GAUSS_TOY = 0, 1
ABC_SIM_BINOMIAL, ABC_SIM_PAPER_NORMAL = 0, 1
ABC_BETA_PAPER, ABC_BETA_FIXED, ABC_BETA_REAL, ABC_BETA_MEAN_VAR, ABC_BETA_MODE_CONC = 0, 1, 2, 3, 4
ABC_STEP_MCMC = 5  # the MCMC-tuned single step (the paper's comparison method)
ABC_W_PAPER, ABC_W_IMPORTANCE = 0, 1
ABC_P_FP32, ABC_P_BF16_TC = 0, 1
TAG_PRIOR, TAG_ANCESTOR, TAG_BETA, TAG_WALK, TAG_SIM, TAG_SCREEN, TAG_AUDIT = 0, 1, 2, 3, 4, 5, 6
TAG_OBS, TAG_OBS_THETA = 7, 8

# every entry point declared in include/abcsmc.h
EXPORTS = (
    "abc_config_default", "abc_philox", "abc_synth_obs", "abc_prior", "abc_simulate",
    "abc_select_scratch_bytes", "abc_select_kth", "abc_prefix_scratch_bytes",
    "abc_resample_prefix", "abc_resample_prefix_noalloc", "abc_propose",
    "abc_accept_scratch_bytes", "abc_accept_append",
    "abc_weights_scratch_bytes", "abc_weights", "abc_tc_probe", "abc_normalize_scratch_bytes",
    "abc_normalize",
    "abc_init", "abc_generation", "abc_run", "abc_get_population", "abc_get_stats",
    "abc_generations", "abc_get_state", "abc_set_state", "abc_free", "abc_strerror",
    "abc_batch_init", "abc_batch_generation", "abc_batch_run", "abc_batch_runs",
    "abc_batch_generations", "abc_batch_active", "abc_batch_get_stats", "abc_batch_get_population",
    "abc_batch_autotune", "abc_batch_tuning", "abc_batch_free",
    "abc_screen", "abc_ex2_probe", "abc_numerics_check", "abc_radix_sort", "abc_predict_scratch_bytes", "abc_predict",
    "abc_predict_population",
    "abc_mlp_param_count", "abc_mlp_create", "abc_mlp_set_params", "abc_mlp_get_params",
    "abc_mlp_scratch_bytes", "abc_mlp_grad", "abc_mlp_adam", "abc_mlp_forward", "abc_mlp_free",
    "abc_set_wait_limit_ns", "abc_inject_alloc_failure", "abc_reset",
)


class AbcConfig(C.Structure):
    _fields_ = [
        ("model", C.c_int32), ("sampler", C.c_int32), ("n_days", C.c_int32),
        ("init_ard", C.c_int32 * 3), ("population", C.c_int64),
        ("theta_lo", C.c_float * 8), ("theta_hi", C.c_float * 8), ("x_obs", C.c_float * 8),
        ("seed", C.c_uint64), ("run_id", C.c_uint32), ("n_particles", C.c_int32),
        ("batch_size", C.c_int32), ("beta_mode", C.c_int32), ("survival_alpha", C.c_double),
        ("beta_a", C.c_float), ("beta_b", C.c_int32), ("weight_mode", C.c_int32),
        ("weight_prec", C.c_int32), ("max_batches", C.c_int32), ("max_redraw", C.c_int32),
        ("surrogate", C.c_int32), ("surrogate_start", C.c_int32), ("surrogate_steps", C.c_int32),
        ("surrogate_batch", C.c_int32), ("surrogate_lr", C.c_float), ("surrogate_tau", C.c_float),
        ("surrogate_rho_min", C.c_float), ("audit_frac", C.c_float), ("surrogate_ring", C.c_int32),
        ("beta_p1", C.c_float), ("beta_p2", C.c_float), ("max_total_batches", C.c_int32),
        ("spec_batches", C.c_int32), ("eps_stop", C.c_float), ("mcmc_s0", C.c_float),
        ("mcmc_adapt", C.c_int32),
    ]


class AbcGenStats(C.Structure):
    _fields_ = [
        ("generation", C.c_int32), ("status", C.c_int32), ("eps", C.c_double),
        ("eps1", C.c_double), ("ess", C.c_double), ("beta_a", C.c_float), ("beta_b", C.c_int32),
        ("batches", C.c_int64), ("sims", C.c_int64), ("sim_days", C.c_int64),
        ("exhausted", C.c_int64), ("accepted", C.c_int64), ("pairs", C.c_int64),
        ("launches", C.c_int64), ("ms", C.c_double), ("ms_sim", C.c_double),
        ("ms_weights", C.c_double), ("screened", C.c_int64), ("audited", C.c_int64),
        ("audit_accepted", C.c_int64), ("train_loss", C.c_double), ("ms_screen", C.c_double),
        ("ms_train", C.c_double), ("rows_tc", C.c_int64), ("ms_tc", C.c_double),
        ("ms_fp32", C.c_double), ("beta_bf", C.c_float), ("mcmc_s", C.c_float),
        ("rows_exp", C.c_int64), ("pairs_tc", C.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class AbcError(RuntimeError):
    def __init__(self, code, where):
        super().__init__("%s failed: %s (%d)" % (where, strerror(code), code))
        self.code = code


_lib = None

_V, _I32, _I64, _U32, _SZ, _D, _F = (C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_size_t,
                                     C.c_double, C.c_float)
_SIGS = {
    "abc_config_default": (None, [C.POINTER(AbcConfig)]),
    "abc_strerror": (C.c_char_p, [C.c_int]),
    "abc_philox": (C.c_int, [_V, _U32, _U32, _I64, _V, _V]),
    "abc_synth_obs": (C.c_int, [C.POINTER(AbcConfig), _V, _V, _V, _V, _V, _V]),
    "abc_prior": (C.c_int, [C.POINTER(AbcConfig), _I64, _V, _V]),
    "abc_simulate": (C.c_int, [C.POINTER(AbcConfig), _V, _V, _I64, _V, _U32, _U32, _V, _V, _V, _V]),
    "abc_select_scratch_bytes": (_SZ, [_I64]),
    "abc_select_kth": (C.c_int, [_V, _I64, _I64, _V, _V, _SZ, _V]),
    "abc_prefix_scratch_bytes": (_SZ, [_I64]),
    "abc_resample_prefix": (C.c_int, [_V, _V, _I64, _V, _I32, _V, _V, _V, _SZ, _V]),
    "abc_resample_prefix_noalloc": (C.c_int, [_V, _V, _I64, _V, _I32, _V, _V, _V]),
    "abc_propose": (C.c_int, [C.POINTER(AbcConfig), _V, _I64, _V, _V, _V, _F, _I32, _I64, _V, _U32,
                              _V, _V, _V, _V, _V, _V]),
    "abc_accept_scratch_bytes": (_SZ, [_I64]),
    "abc_accept_append": (C.c_int, [_V, _V, _V, _V, _V, _I64, _V, _I64, _V, _V, _V, _V, _V, _V, _V,
                                    _SZ, _V]),
    "abc_weights_scratch_bytes": (_SZ, [_I64, _I64]),
    "abc_weights": (C.c_int, [_V, _V, _I64, _V, _V, _V, _I64, _I32, _V, _V, _SZ, _V]),
    "abc_tc_probe": (C.c_int, [_V, _V, _V, _V]),
    "abc_normalize_scratch_bytes": (_SZ, [_I64]),
    "abc_normalize": (C.c_int, [_V, _I64, _V, _V, _V, _SZ, _V]),
    "abc_init": (C.c_int, [C.POINTER(AbcConfig), _V, _V, C.POINTER(C.c_void_p)]),
    "abc_generation": (C.c_int, [_V]),
    "abc_run": (C.c_int, [_V, _I32, _D]),
    "abc_get_population": (C.c_int, [_V, _V, _V, _V, _V, _V, _I32]),
    "abc_get_stats": (C.c_int, [_V, _I32, C.POINTER(AbcGenStats)]),
    "abc_generations": (C.c_int32, [_V]),
    "abc_get_state": (C.c_int, [_V, _V, C.POINTER(C.c_size_t)]),
    "abc_set_state": (C.c_int, [_V, _V, _SZ]),
    "abc_free": (None, [_V]),
    "abc_batch_init": (C.c_int, [C.POINTER(AbcConfig), _I32, _V, _V, C.POINTER(C.c_void_p)]),
    "abc_batch_generation": (C.c_int, [_V]),
    "abc_batch_run": (C.c_int, [_V, _I32]),
    "abc_batch_runs": (C.c_int32, [_V]),
    "abc_batch_generations": (C.c_int32, [_V]),
    "abc_batch_active": (C.c_int32, [_V]),
    "abc_batch_get_stats": (C.c_int, [_V, _I32, _I32, C.POINTER(AbcGenStats)]),
    "abc_batch_get_population": (C.c_int, [_V, _I32, _V, _V, _V, _V, _V, _I32]),
    "abc_batch_autotune": (C.c_int, [_V, C.c_char_p]),
    "abc_batch_tuning": (C.c_int, [_V, _I32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "abc_batch_free": (None, [_V]),
    "abc_screen": (C.c_int, [_V, _V, _V, _V, _I64, _V, C.c_uint32, _V, _V, _V]),
    "abc_ex2_probe": (C.c_int, [C.POINTER(C.c_double), _V]),
    "abc_numerics_check": (C.c_int, [_I32, C.POINTER(C.c_uint64), _V]),
    "abc_radix_sort": (C.c_int, [_V, _V, _I64, _I32, _V, _V, _V]),
    "abc_predict_scratch_bytes": (_SZ, [_I64, _I64, _I32, _I32]),
    "abc_predict": (C.c_int, [_V, _V, _V, _I64, _I64, _I32, _V, _I32, _V, _V, _SZ, _V]),
    "abc_predict_population": (C.c_int, [_V, _I64, _I32, _V, _I32, _V]),
    "abc_mlp_param_count": (C.c_int32, []),
    "abc_mlp_create": (C.c_int, [C.c_uint64, C.POINTER(C.c_void_p)]),
    "abc_mlp_set_params": (C.c_int, [_V, _V]),
    "abc_mlp_get_params": (C.c_int, [_V, _V, _V]),
    "abc_mlp_scratch_bytes": (_SZ, [_I32, _I64]),
    "abc_mlp_grad": (C.c_int, [_V, _V, _V, _I32, _V, _V, _V, _SZ, _V]),
    "abc_mlp_adam": (C.c_int, [_V, _V, _I64, _F, _V]),
    "abc_mlp_forward": (C.c_int, [_V, _V, _I64, _V, _V, _SZ, _V]),
    "abc_mlp_free": (None, [_V]),
    "abc_set_wait_limit_ns": (None, [C.c_uint64]),
    "abc_inject_alloc_failure": (None, [_I64]),
    "abc_reset": (C.c_int, [_V, _U32]),
}


def lib():
    """Load libabcsmc.so (raises if it has not been built: no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libabcsmc.so is missing; run paper_2106_15508_gb300.build.build() "
                              "(or __graft_entry__.build()) first")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def strerror(code):
    return lib().abc_strerror(int(code)).decode()


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(s):
    if s is not None:
        return s if isinstance(s, int) else s.cuda_stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def _check(rc, where, ok=(ABC_OK,)):
    if rc not in ok:
        raise AbcError(rc, where)
    return rc


def config(**kw):
    """abc_config_default() overridden by keyword fields (arrays as lists)."""
    c = AbcConfig()
    lib().abc_config_default(C.byref(c))
    for k, v in kw.items():
        f = getattr(c, k)
        if isinstance(f, C.Array):
            f[:] = list(v)
        else:
            setattr(c, k, v)
    return c


# ---- step entry points (device pointers) -------------------------------
def abc_philox(ctr, key0, key1, n, out, stream=None):
    return _check(lib().abc_philox(_ptr(ctr), key0, key1, n, _ptr(out), _stream(stream)),
                  "abc_philox")


def abc_synth_obs(cfg, box_lo, box_hi, obs, theta_star, attempts, stream=None):
    lo = (C.c_float * 8)(*[float(v) for v in box_lo])
    hi = (C.c_float * 8)(*[float(v) for v in box_hi])
    return _check(lib().abc_synth_obs(C.byref(cfg), C.cast(lo, C.c_void_p), C.cast(hi, C.c_void_p),
                                      _ptr(obs), _ptr(theta_star), _ptr(attempts),
                                      _stream(stream)), "abc_synth_obs")


def abc_prior(cfg, n, u, stream=None):
    return _check(lib().abc_prior(C.byref(cfg), n, _ptr(u), _stream(stream)), "abc_prior")


def abc_simulate(cfg, obs, u, n, c0_idx, c1, tag, skip, dist, traj=None, stream=None):
    return _check(lib().abc_simulate(C.byref(cfg), _ptr(obs), _ptr(u), n, _ptr(c0_idx), c1, tag,
                                     _ptr(skip), _ptr(dist), _ptr(traj), _stream(stream)),
                  "abc_simulate")


def abc_select_scratch_bytes(n):
    return lib().abc_select_scratch_bytes(n)


def abc_select_kth(d, n, k, out, scratch, scratch_bytes, stream=None):
    return _check(lib().abc_select_kth(_ptr(d), n, k, _ptr(out), _ptr(scratch), scratch_bytes,
                                       _stream(stream)), "abc_select_kth")


def abc_prefix_scratch_bytes(n):
    return lib().abc_prefix_scratch_bytes(n)


def abc_resample_prefix(d, W, n, eps, mode, q, prefix, scratch, scratch_bytes, stream=None):
    return _check(lib().abc_resample_prefix(_ptr(d), _ptr(W), n, _ptr(eps), mode, _ptr(q),
                                            _ptr(prefix), _ptr(scratch), scratch_bytes,
                                            _stream(stream)), "abc_resample_prefix")


def abc_resample_prefix_noalloc(d, W, n, eps, mode, q, prefix, stream=None):
    """abc_resample_prefix without a scratch buffer (fixed library scratch,
    n <= 2^24; calls sharing it must not overlap on the GPU)."""
    return _check(lib().abc_resample_prefix_noalloc(_ptr(d), _ptr(W), n, _ptr(eps), mode, _ptr(q),
                                                    _ptr(prefix), _stream(stream)),
                  "abc_resample_prefix_noalloc")


def abc_propose(cfg, u, n, prefix, eps, eps1, beta_a, beta_b, slots, c0_idx, c1, u_out, s_out,
                anc_out, attempts_out, flag_out, stream=None):
    return _check(lib().abc_propose(C.byref(cfg), _ptr(u), n, _ptr(prefix), _ptr(eps), _ptr(eps1),
                                    beta_a, beta_b, slots, _ptr(c0_idx), c1, _ptr(u_out),
                                    _ptr(s_out), _ptr(anc_out), _ptr(attempts_out),
                                    _ptr(flag_out), _stream(stream)), "abc_propose")


def abc_accept_scratch_bytes(M):
    return lib().abc_accept_scratch_bytes(M)


def abc_accept_append(up, dp, sp, ap, flag, M, eps, N, u_pop, d_pop, s_pop, anc_pop, filled,
                      counters, scratch, scratch_bytes, stream=None):
    return _check(lib().abc_accept_append(
        _ptr(up), _ptr(dp), _ptr(sp), _ptr(ap), _ptr(flag), M, _ptr(eps), N, _ptr(u_pop),
        _ptr(d_pop), _ptr(s_pop), _ptr(anc_pop), _ptr(filled), _ptr(counters), _ptr(scratch),
        scratch_bytes, _stream(stream)), "abc_accept_append")


def abc_weights_scratch_bytes(rows, n):
    return lib().abc_weights_scratch_bytes(rows, n)


def abc_weights(up, s, rows, u, q, prefix, n, prec, logW, scratch, scratch_bytes, stream=None):
    return _check(lib().abc_weights(_ptr(up), _ptr(s), rows, _ptr(u), _ptr(q), _ptr(prefix), n,
                                    prec, _ptr(logW), _ptr(scratch), scratch_bytes,
                                    _stream(stream)), "abc_weights")


def abc_tc_probe(A, B, D, stream=None):
    return _check(lib().abc_tc_probe(_ptr(A), _ptr(B), _ptr(D), _stream(stream)), "abc_tc_probe")


def abc_normalize_scratch_bytes(n):
    return lib().abc_normalize_scratch_bytes(n)


def abc_normalize(logW, n, W, ess, scratch, scratch_bytes, stream=None):
    return _check(lib().abc_normalize(_ptr(logW), n, _ptr(W), _ptr(ess), _ptr(scratch),
                                      scratch_bytes, _stream(stream)), "abc_normalize")


# ---- context --------------------------------------------------------------
def abc_init(cfg, obs_host, stream=None):
    """obs_host: host int32 [3][T+1] (numpy or None for the toy model)."""
    h = C.c_void_p()
    ptr = None if obs_host is None else obs_host.ctypes.data
    _check(lib().abc_init(C.byref(cfg), ptr, _stream(stream), C.byref(h)), "abc_init")
    return h


def abc_init_ptr(cfg, obs_host_ptr, stream=None):
    """abc_init with the observed series given by host address (e.g. pinned
    memory; 0 or None for the toy model)."""
    h = C.c_void_p()
    _check(lib().abc_init(C.byref(cfg), obs_host_ptr or None, _stream(stream), C.byref(h)),
           "abc_init")
    return h


def abc_generation(ctx):
    return _check(lib().abc_generation(ctx), "abc_generation",
                  ok=(ABC_OK, ABC_STOP_BUDGET, ABC_STOP_TARGET, ABC_STOP_TOTAL))


def abc_run(ctx, n_generations, eps_target=0.0):
    return _check(lib().abc_run(ctx, n_generations, eps_target), "abc_run",
                  ok=(ABC_OK, ABC_STOP_BUDGET, ABC_STOP_TARGET, ABC_STOP_TOTAL))


def abc_reset(ctx, run_id):
    """Start the context over at stage 0 as run `run_id`."""
    return _check(lib().abc_reset(ctx, int(run_id)), "abc_reset")


def abc_get_population(ctx, u=None, dist=None, W=None, s=None, anc=None, on_device=False):
    def p(x):
        if x is None:
            return None
        return x.ctypes.data if hasattr(x, "ctypes") else _ptr(x)
    return _check(lib().abc_get_population(ctx, p(u), p(dist), p(W), p(s), p(anc),
                                           1 if on_device else 0), "abc_get_population")


def abc_get_stats(ctx, t):
    st = AbcGenStats()
    _check(lib().abc_get_stats(ctx, t, C.byref(st)), "abc_get_stats")
    return st


def abc_generations(ctx):
    return lib().abc_generations(ctx)


def abc_get_state(ctx):
    n = C.c_size_t(0)
    _check(lib().abc_get_state(ctx, None, C.byref(n)), "abc_get_state")
    buf = C.create_string_buffer(n.value)
    _check(lib().abc_get_state(ctx, C.cast(buf, C.c_void_p), C.byref(n)), "abc_get_state")
    return buf.raw[: n.value]


def abc_set_state(ctx, blob: bytes):
    buf = C.create_string_buffer(blob, len(blob))
    return _check(lib().abc_set_state(ctx, C.cast(buf, C.c_void_p), len(blob)), "abc_set_state")


def abc_set_state_ptr(ctx, host_ptr: int, nbytes: int):
    """abc_set_state from a host buffer given by address (e.g. pinned memory)."""
    return _check(lib().abc_set_state(ctx, host_ptr, nbytes), "abc_set_state")


def abc_free(ctx):
    if ctx:
        lib().abc_free(ctx)


# ---- batched runs -----------------------------------------------------------
def abc_batch_init(cfgs, obs_list, stream=None):
    """cfgs: list of AbcConfig; obs_list: list of host int32 [3][T_r+1] numpy
    arrays (None for the toy model)."""
    n = len(cfgs)
    arr = (AbcConfig * n)(*cfgs)
    ptrs = (C.c_void_p * n)(*[None if o is None else o.ctypes.data for o in obs_list])
    h = C.c_void_p()
    _check(lib().abc_batch_init(arr, n, C.cast(ptrs, C.c_void_p), _stream(stream), C.byref(h)),
           "abc_batch_init")
    h._keep = (arr, ptrs, obs_list)
    return h


def abc_batch_generation(b):
    return _check(lib().abc_batch_generation(b), "abc_batch_generation")


def abc_batch_run(b, n_generations):
    return _check(lib().abc_batch_run(b, n_generations), "abc_batch_run")


def abc_batch_runs(b):
    return lib().abc_batch_runs(b)


def abc_batch_generations(b):
    return lib().abc_batch_generations(b)


def abc_batch_active(b):
    return lib().abc_batch_active(b)


def abc_batch_get_stats(b, run, t):
    st = AbcGenStats()
    _check(lib().abc_batch_get_stats(b, run, t, C.byref(st)), "abc_batch_get_stats")
    return st


def abc_batch_get_population(b, run, u=None, dist=None, W=None, s=None, anc=None):
    p = lambda x: None if x is None else x.ctypes.data
    return _check(lib().abc_batch_get_population(b, run, p(u), p(dist), p(W), p(s), p(anc), 0),
                  "abc_batch_get_population")


def abc_batch_autotune(b, cache_path=None):
    return _check(lib().abc_batch_autotune(b, None if cache_path is None else
                                           cache_path.encode()), "abc_batch_autotune")


def abc_batch_tuning(b, run):
    th, wm = C.c_int32(0), C.c_int32(0)
    _check(lib().abc_batch_tuning(b, run, C.byref(th), C.byref(wm)), "abc_batch_tuning")
    return th.value, wm.value


def abc_batch_free(b):
    if b:
        lib().abc_batch_free(b)


# ---- surrogate MLP ------------------------------------------------------------
MLP_SHAPES = dict(W1=(256, 8), b1=(256,), W2=(256, 256), b2=(256,), W3=(4, 256), b3=(4,))
MLP_ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


def abc_screen(cfg, Y, ystat, flag, M, eps, c1, rho, sflag, stream=None):
    return _check(lib().abc_screen(C.byref(cfg), _ptr(Y), _ptr(ystat), _ptr(flag), M, _ptr(eps), c1,
                                   _ptr(rho), _ptr(sflag), _stream(stream)), "abc_screen")


def abc_set_wait_limit_ns(ns):
    """Test hook: time limit of the tensor-core weight kernel's pipeline waits
    (0 restores the default)."""
    lib().abc_set_wait_limit_ns(int(ns))


def abc_inject_alloc_failure(after):
    """Test hook: the context allocation after `after` successful ones fails
    (negative: off)."""
    lib().abc_inject_alloc_failure(int(after))


def abc_ex2_probe(stream=None):
    """Sustained ex2.approx.f32 rate of this GPU (exponentials per second)."""
    r = C.c_double()
    _check(lib().abc_ex2_probe(C.byref(r), _stream(stream)), "abc_ex2_probe")
    return r.value


def abc_numerics_check(which, stream=None):
    """Operand pairs of check `which` whose short division differs from
    __fdiv_rn (0 expected)."""
    r = C.c_uint64()
    _check(lib().abc_numerics_check(which, C.byref(r), _stream(stream)), "abc_numerics_check")
    return r.value


def abc_radix_sort(keys, vals, n, bits, keys_out, vals_out, stream=None):
    return _check(lib().abc_radix_sort(_ptr(keys), _ptr(vals), n, bits, _ptr(keys_out),
                                       _ptr(vals_out), _stream(stream)), "abc_radix_sort")


def abc_predict_scratch_bytes(N, R, days, nq):
    return lib().abc_predict_scratch_bytes(N, R, days, nq)


def abc_predict(cfg, u, W, N, R, days, quant, out, scratch, scratch_bytes, stream=None):
    """Posterior-predictive order statistics into out (device int32
    [days + 1][3][nq]); quant: host sequence of levels in (0, 1]."""
    import numpy as np
    q = np.ascontiguousarray(quant, np.float64)
    return _check(lib().abc_predict(C.byref(cfg), _ptr(u), _ptr(W), N, R, days, q.ctypes.data,
                                    len(q), _ptr(out), _ptr(scratch), scratch_bytes,
                                    _stream(stream)), "abc_predict")


def abc_predict_population(ctx, R, days, quant):
    """abc_predict on the context's population; returns int32 [days + 1][3][nq]."""
    import numpy as np
    q = np.ascontiguousarray(quant, np.float64)
    out = np.zeros((days + 1, 3, len(q)), np.int32)
    _check(lib().abc_predict_population(ctx, R, days, q.ctypes.data, len(q), out.ctypes.data),
           "abc_predict_population")
    return out


def abc_mlp_create(seed=1):
    h = C.c_void_p()
    _check(lib().abc_mlp_create(seed, C.byref(h)), "abc_mlp_create")
    return h


def abc_mlp_set_params(m, params):
    """params: host float32 array of abc_mlp_param_count() values"""
    return _check(lib().abc_mlp_set_params(m, params.ctypes.data), "abc_mlp_set_params")


def abc_mlp_get_params(m, params=None, bf16=None):
    p = lambda x: None if x is None else x.ctypes.data
    return _check(lib().abc_mlp_get_params(m, p(params), p(bf16)), "abc_mlp_get_params")


def abc_mlp_scratch_bytes(batch, n):
    return lib().abc_mlp_scratch_bytes(batch, n)


def abc_mlp_grad(m, X, T, B, grad, sse, scratch, scratch_bytes, stream=None):
    return _check(lib().abc_mlp_grad(m, _ptr(X), _ptr(T), B, _ptr(grad), _ptr(sse), _ptr(scratch),
                                     scratch_bytes, _stream(stream)), "abc_mlp_grad")


def abc_mlp_adam(m, grad, step, lr, stream=None):
    return _check(lib().abc_mlp_adam(m, _ptr(grad), step, lr, _stream(stream)), "abc_mlp_adam")


def abc_mlp_forward(m, u, n, Y, scratch, scratch_bytes, stream=None):
    return _check(lib().abc_mlp_forward(m, _ptr(u), n, _ptr(Y), _ptr(scratch), scratch_bytes,
                                        _stream(stream)), "abc_mlp_forward")


def abc_mlp_free(m):
    if m:
        lib().abc_mlp_free(m)
