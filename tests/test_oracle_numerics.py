"""Pins of the oracle's numerics (CPU, no GPU): Philox against NVIDIA's curand
host generator, constants against their exact definitions, fp32
transcendentals against fp64 library values, samplers against exact
distributions.  Each pin is chosen so that a dropped term, a wrong sign or a
swapped operand in the oracle fails it."""
import ctypes
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.stats as st

import oracle as O


# ---------------------------------------------------------------- Philox ---
def _curand_host(seed, offset, n):
    try:
        lib = ctypes.CDLL("libcurand.so")
    except OSError:
        try:
            lib = ctypes.CDLL("/usr/local/cuda/lib64/libcurand.so")
        except OSError:
            pytest.skip("libcurand not available on this host")
    gen = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) != 0:  # PHILOX4_32_10
        pytest.skip("curand host Philox generator unavailable")
    assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
    assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(offset)) == 0
    buf = (ctypes.c_uint * n)()
    assert lib.curandGenerate(gen, buf, ctypes.c_size_t(n)) == 0
    lib.curandDestroyGenerator(gen)
    return np.array(buf[:], np.uint32).reshape(-1, 4)


@pytest.mark.parametrize("seed,block0", [(0, 0), (0x123456789ABCDEF0, 65530),
                                         (0xDEADBEEF00C0FFEE, 65536 * (2**32 + 3) + 7)])
def test_philox_matches_curand_host_generator(seed, block0):
    """curand's host Philox4_32_10 emits block b = philox((b>>16 lo, b>>16 hi, b&0xffff, 0),
    key=(seed lo, seed hi)); 12 consecutive blocks cross the 65536 boundary."""
    out = _curand_host(seed, 4 * block0, 48)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i, blk in enumerate(out):
        b = block0 + i
        hi = b >> 16
        ctr = [hi & 0xFFFFFFFF, hi >> 32, b & 0xFFFF, 0]
        assert np.array_equal(blk, O.philox(ctr, key)), (seed, b)


def test_philox_counter_word3_and_key_sensitivity():
    """Word 3 of the counter and both key words each change every output word."""
    base = O.philox([1, 2, 3, 4], [5, 6])
    for ctr, key in (([1, 2, 3, 5], [5, 6]), ([1, 2, 3, 4], [5, 7]), ([1, 2, 3, 4], [6, 6])):
        other = O.philox(ctr, key)
        assert np.all(other != base)


def test_uniform_mapping():
    """(x >> 9) + 1/2 over 2^23: strictly inside (0, 1), symmetric, exact."""
    assert O.uniform(0) == 2.0 ** -24
    assert O.uniform(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert O.uniform(0x80000000) == 0.5 + 2.0 ** -24
    rng = np.random.default_rng(0)
    for x in rng.integers(0, 2**32, 1000):
        assert O.uniform(int(x)) == ((int(x) >> 9) + 0.5) / 2**23


# ------------------------------------------------------------- constants ---
def _rn32(x: Fraction) -> float:
    c = np.float32(float(x))
    cands = [np.nextafter(c, np.float32(-np.inf)), c, np.nextafter(c, np.float32(np.inf))]
    return float(min(cands, key=lambda v: (abs(Fraction(float(v)) - x),
                                           int(np.float32(v).view(np.uint32)) & 1)))


def test_constants_are_their_definitions():
    import sympy
    c = O.constants()
    ln2 = Fraction(str(sympy.log(2).evalf(60)))
    assert c[0] == 0.693145751953125  # 15-bit head of ln 2
    assert abs(Fraction(float(c[0])) - ln2) < Fraction(1, 2**16)
    assert c[1] == _rn32(ln2 - Fraction(float(c[0])))
    assert c[2] == _rn32(Fraction(str((1 / sympy.log(2)).evalf(60))))
    assert c[3] == _rn32(Fraction(str((2 * sympy.pi).evalf(60))))
    assert c[4] == _rn32(Fraction(str(sympy.sqrt(2).evalf(60))))
    for k in range(14):
        assert c[5 + k] == _rn32(Fraction(1, math.factorial(k))), k
    for k in range(1, 6):
        assert c[18 + k] == _rn32(Fraction(1, 2 * k + 1)), k


# -------------------------------------------------------- transcendentals --
def _ulp_err(got, want):
    want32 = np.float32(want)
    return abs(got - want) / float(np.spacing(np.abs(want32)))


def _sweep(lo, hi, n=4000, log=False, seed=0):
    rng = np.random.default_rng(seed)
    if log:
        x = np.exp(rng.uniform(np.log(lo), np.log(hi), n))
    else:
        x = rng.uniform(lo, hi, n)
    return np.unique(x.astype(np.float32))


@pytest.mark.parametrize("name,ref,lo,hi,log", [
    ("or_logf", math.log, 2.0**-25, 1.0, True),
    ("or_logf", math.log, 0.5, 2.0, False),
    ("or_logf", math.log, 1.0, 3.3e8, True),
    ("or_expf", math.exp, -87.0, 88.0, False),
    ("or_expf", math.exp, -1.0, 1.0, False),
    ("or_expm1f", math.expm1, -17.0, 10.0, False),
    ("or_expm1f", math.expm1, -0.5, 0.5, False),
    ("or_expm1f", math.expm1, 1e-9, 0.35, True),
    ("or_log1pf", math.log1p, -0.5, 1.0, False),
    ("or_log1pf", math.log1p, 1e-9, 0.1, True),
])
def test_transcendental_ulp_bound(name, ref, lo, hi, log):
    f = O.fn(name)
    worst = 0.0
    for x in _sweep(lo, hi, log=log):
        got = f(x)
        want = ref(float(x))
        worst = max(worst, _ulp_err(got, want))
    # log1p composes log (<= 2 ulp), a division and a product: 3 ulp
    bound = 3.0 if name == "or_log1pf" else 2.0
    assert worst <= bound, (name, worst)


def test_log1p_negative_small():
    f = O.fn("or_log1pf")
    for x in -_sweep(1e-9, 0.5, log=True, seed=3):
        assert _ulp_err(f(x), math.log1p(float(x))) <= 3.0


def test_cos2pi_within_tolerance():
    f = O.fn("or_cos2pi")
    xs = np.concatenate([_sweep(0.0, 1.0, 20000), np.float32([0, 0.125, 0.25, 0.375, 0.5,
                                                              0.625, 0.75, 0.875, 1.0])])
    for w in xs:
        got = f(w)
        want = math.cos(2 * math.pi * float(w))
        # absolute error is what matters for Box-Muller; bound it and the ulp error
        assert abs(got - want) <= 1.5e-7, (w, got, want)
    assert f(0.0) == 1.0 and f(0.5) == -1.0 and f(0.25) == 0.0 and f(0.75) == 0.0


def test_transcendental_special_values():
    assert O.fn("or_logf")(0.0) == -math.inf
    assert math.isnan(O.fn("or_logf")(-1.0))
    assert O.fn("or_logf")(1.0) == 0.0
    assert O.fn("or_expf")(0.0) == 1.0
    assert O.fn("or_expf")(-200.0) == 0.0
    assert O.fn("or_expf")(100.0) == math.inf
    assert O.fn("or_expm1f")(0.0) == 0.0
    assert O.fn("or_expm1f")(-30.0) == -1.0
    # subnormal results are produced by a single rounding
    x = np.float32(-100.0)
    assert abs(O.fn("or_expf")(x) - math.exp(-100.0)) <= float(np.float32(2.0**-149))


# --------------------------------------------------------------- samplers --
def test_normal_is_standard_normal():
    rng = np.random.default_rng(1)
    w = rng.integers(0, 2**32, (20000, 2), dtype=np.uint64)
    z = np.array([O.normal(O.uniform(int(a)), O.uniform(int(b))) for a, b in w])
    assert st.kstest(z, "norm").pvalue > 1e-3
    assert abs(z.mean()) < 4 / math.sqrt(len(z))


@pytest.mark.parametrize("n,p", [(1, 0.3), (7, 0.2), (40, 0.05), (1000, 0.004), (25, 0.7),
                                 (12, 0.999)])
def test_binv_is_exact_inversion(n, p):
    """BINV returns the smallest k with CDF(k) >= u; where fp32 pmf rounding
    could matter (u within 1e-5 of a CDF step) either neighbour is accepted."""
    p32 = float(np.float32(p))
    flip = p32 > 0.5
    q = (1 - p32) if flip else p32
    rng = np.random.default_rng(n)
    cdf = st.binom.cdf(np.arange(n + 1), n, q)
    for x in rng.integers(0, 2**32, 3000):
        u = O.uniform(int(x))
        k = O.binomial(n, p32, u, 0.5)
        want = int(np.searchsorted(cdf, u, side="left"))
        kk = n - k if flip else k
        if kk != want:
            near = min(abs(u - cdf[want - 1]) if want > 0 else 1, abs(u - cdf[min(want, n)]))
            assert near < 1e-5, (n, p, u, k, want)


def test_binomial_chi_square_small_n():
    n, p = 30, 0.13
    rng = np.random.default_rng(2)
    w = rng.integers(0, 2**32, (40000, 2), dtype=np.uint64)
    k = np.array([O.binomial(n, p, O.uniform(int(a)), O.uniform(int(b))) for a, b in w])
    obs = np.bincount(k, minlength=n + 1)
    exp = st.binom.pmf(np.arange(n + 1), n, float(np.float32(p))) * len(k)
    m = exp > 5
    chi = ((obs[m] - exp[m]) ** 2 / exp[m]).sum()
    assert st.chi2.sf(chi, m.sum() - 1) > 1e-3


@pytest.mark.parametrize("n,p", [(100000, 0.3), (5000, 0.01), (10**7, 0.9), (200, 0.5)])
def test_binomial_normal_branch_moments(n, p):
    rng = np.random.default_rng(3)
    w = rng.integers(0, 2**32, (20000, 2), dtype=np.uint64)
    k = np.array([O.binomial(n, p, O.uniform(int(a)), O.uniform(int(b))) for a, b in w],
                 dtype=np.float64)
    p32 = float(np.float32(p))
    mu, var = n * p32, n * p32 * (1 - p32)
    assert abs(k.mean() - mu) < 5 * math.sqrt(var / len(k)) + 0.5
    assert abs(k.var() / var - 1) < 0.05
    assert k.min() >= 0 and k.max() <= n


def test_binomial_trivial_cases():
    assert O.binomial(0, 0.5, 0.3, 0.3) == 0
    assert O.binomial(10, 0.0, 0.3, 0.3) == 0
    assert O.binomial(10, 1.0, 0.3, 0.3) == 10
    assert O.binomial(10, -0.1, 0.3, 0.3) == 0


@pytest.mark.parametrize("a,b", [(1.0, 2), (0.5, 5), (0.1, 15), (2.0, 5)])
def test_beta_sampler_ks(a, b):
    """Shapes of Sec. 3.2.2 (Beta(1,2), Beta(0.5,5), Beta(0.1,15)) and Beta(2,5)."""
    key = [7, 11]
    s = np.array([O.beta(key, a, b, j, 3, 0) for j in range(6000)])
    assert np.all((s >= 0) & (s <= 1))
    assert st.kstest(s, st.beta(a, b).cdf).pvalue > 1e-3
