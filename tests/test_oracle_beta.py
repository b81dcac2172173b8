"""Pins of the oracle's general-shape step-size Beta (Sec. 3.2: Eq. 16 and the
mean-variance and mode-concentration parameterisations the paper names).

* the Gamma sampler (Marsaglia-Tsang) and the Gamma-ratio Beta against the
  scipy distributions by Kolmogorov-Smirnov, including shapes below 1;
* the integer-b product form and the Gamma ratio agree in distribution;
* the shape rules against the closed-form moments and the numerically located
  mode of the Beta density, and their clamps.
"""
import numpy as np
import pytest
import scipy.optimize as so
import scipy.stats as st

import oracle as O

KEY = [0x9E3779B9, 0x243F6A88]


def _gamma_logs(alpha, n=12000, c1=9, blk0=0):
    return np.array([O.gamma_log(KEY, alpha, j, c1, 0, blk0) for j in range(n)], np.float64)


@pytest.mark.parametrize("alpha", [0.05, 0.3, 1.0, 2.5, 17.3, 900.0])
def test_gamma_log_ks(alpha):
    lg = _gamma_logs(alpha)
    assert np.all(np.isfinite(lg))
    x = np.exp(lg)
    assert st.kstest(x, st.gamma(alpha).cdf).pvalue > 1e-3


def test_gamma_log_blocks_independent():
    """X (blocks 0..63) and Y (blocks 64..127) of one slot are uncorrelated."""
    x = _gamma_logs(2.0, 8000, blk0=0)
    y = _gamma_logs(2.0, 8000, blk0=64)
    r = np.corrcoef(x, y)[0, 1]
    assert abs(r) < 4.0 / np.sqrt(len(x))


@pytest.mark.parametrize("a,b", [(0.3, 2.7), (2.5, 0.4), (0.1, 15.5), (5.3, 7.1), (1.0, 1.0),
                                 (40.5, 0.9)])
def test_beta_real_ks(a, b):
    s = np.array([O.beta_real(KEY, a, b, j, 4, 0) for j in range(12000)], np.float64)
    assert np.all((s >= 0) & (s <= 1))
    assert st.kstest(s, st.beta(a, b).cdf).pvalue > 1e-3
    m, v = st.beta(a, b).stats("mv")
    assert abs(s.mean() - m) < 5 * np.sqrt(v / len(s))


def test_beta_real_small_shapes():
    """Beta(0.02, 0.03) puts much of its mass closer to 0 and to 1 than fp32
    resolves (below 2^-128 the ratio underflows to 0; within 2^-25 of 1 it rounds
    to 1).  The draws are compared by the mass of [0, 1e-36), [1e-36, 1/2) and
    [1/2, 1] (chi-square), and inside [1e-36, 1/2) by KS against the
    conditional CDF."""
    a, b = 0.02, 0.03
    s = np.array([O.beta_real(KEY, a, b, j, 6, 0) for j in range(12000)], np.float64)
    B = st.beta(a, b)
    edges = [1e-36, 0.5]
    p = np.diff(np.concatenate([[0.0], B.cdf(edges), [1.0]]))
    n = np.array([np.sum(s < 1e-36), np.sum((s >= 1e-36) & (s < 0.5)), np.sum(s >= 0.5)])
    assert st.chisquare(n, p * len(s)).pvalue > 1e-3
    mid = s[(s >= 1e-36) & (s < 0.5)]
    lo, hi = B.cdf(1e-36), B.cdf(0.5)
    assert st.kstest(mid, lambda x: (B.cdf(x) - lo) / (hi - lo)).pvalue > 1e-3


@pytest.mark.parametrize("a,b", [(1.0, 2), (0.5, 5), (0.1, 15)])
def test_beta_real_matches_product_form(a, b):
    """Shapes of Sec. 3.2 with integer b: the two samplers agree in distribution."""
    s_ratio = np.array([O.beta_real(KEY, a, float(b), j, 21, 0) for j in range(8000)])
    s_prod = np.array([O.beta(KEY, a, b, j, 22, 0) for j in range(8000)])
    assert st.ks_2samp(s_ratio, s_prod).pvalue > 1e-3


def test_beta_real_tiny_shapes_are_defined():
    """At the clamp 2^-20 both shapes: finite, in [0, 1], and nearly Bernoulli."""
    t = 2.0 ** -20
    s = np.array([O.beta_real(KEY, t, t, j, 5, 0) for j in range(2000)])
    assert np.all((s >= 0) & (s <= 1))
    assert np.mean((s < 1e-3) | (s > 1 - 1e-3)) > 0.99
    # Beta(e, e) is symmetric: about half the mass at each end
    assert abs(np.mean(s > 0.5) - 0.5) < 0.05


def test_shape_paper_and_fixed():
    a, b, bi = O.beta_shape(O.BETA_PAPER, 0.25, 7)
    assert (np.float32(a), b, bi) == (np.float32(0.25), 14.0, 14)
    a, b, bi = O.beta_shape(O.BETA_FIXED, 0.25, 7, fa=2.0, fb=5)
    assert (a, b, bi) == (2.0, 5.0, 5)
    a, b, bi = O.beta_shape(O.BETA_REAL, 0.25, 7, p1=0.7, p2=3.5)
    assert (np.float32(a), b, bi) == (np.float32(0.7), 3.5, 0)


def test_shape_paper_beyond_1024_uses_the_gamma_ratio():
    """Eq. 16's b = 2t: the product form up to stage 512 (1024 uniforms),
    then the same Beta(ratio, 2t) by the Gamma ratio, a clamped like the
    real-shape rules."""
    a, b, bi = O.beta_shape(O.BETA_PAPER, 0.25, 512)
    assert (np.float32(a), b, bi) == (np.float32(0.25), 1024.0, 1024)
    a, b, bi = O.beta_shape(O.BETA_PAPER, 0.25, 513)
    assert (np.float32(a), b, bi) == (np.float32(0.25), 1026.0, 0)
    a, b, bi = O.beta_shape(O.BETA_PAPER, 0.0, 2000)
    assert (a, b, bi) == (2.0 ** -20, 4000.0, 0)


@pytest.mark.parametrize("a,b", [(0.2, 1026), (0.9, 1500)])
def test_beta_real_at_paper_shapes_beyond_1024(a, b):
    """The shapes the paper schedule reaches after stage 512 (small a, b in
    the thousands): the Gamma ratio against scipy's Beta."""
    s = np.array([O.beta_real(KEY, a, float(b), j, 23, 0) for j in range(8000)], np.float64)
    B = st.beta(a, b)
    ok = s > 1e-30  # below this fp32 resolves nothing that the KS test could use
    assert abs(np.mean(~ok) - B.cdf(1e-30)) < 0.02
    lo = B.cdf(1e-30)
    assert st.kstest(s[ok], lambda x: (B.cdf(x) - lo) / (1 - lo)).pvalue > 1e-3


@pytest.mark.parametrize("p1,p2,ratio,t", [(0.3, 0.01, 1.0, 1), (0.3, 0.05, 0.5, 3),
                                           (0.6, 0.02, 0.9, 2), (0.1, 0.001, 0.2, 5)])
def test_shape_mean_variance_moments(p1, p2, ratio, t):
    """The shapes reproduce mean p1 ratio and variance p2 / t (closed-form Beta moments)."""
    a, b, bi = O.beta_shape(O.BETA_MEAN_VAR, ratio, t, p1=p1, p2=p2)
    assert bi == 0
    m, v = st.beta(a, b).stats("mv")
    assert m == pytest.approx(p1 * ratio, rel=1e-5)
    assert v == pytest.approx(p2 / t, rel=1e-5)


def test_shape_mean_variance_cap():
    """A variance at or above mu (1 - mu) caps a + b at 1/16, keeping the mean."""
    mu = 0.2
    a, b, _ = O.beta_shape(O.BETA_MEAN_VAR, 1.0, 1, p1=mu, p2=0.5)
    assert a + b == pytest.approx(1 / 16, rel=1e-6)
    assert a / (a + b) == pytest.approx(mu, rel=1e-6)


@pytest.mark.parametrize("p1,p2,ratio,t", [(0.2, 10.0, 1.0, 1), (0.5, 4.0, 0.6, 3),
                                           (0.9, 3.0, 0.5, 7)])
def test_shape_mode_concentration(p1, p2, ratio, t):
    """The Beta density peaks at p1 ratio and a + b = p2 t."""
    a, b, bi = O.beta_shape(O.BETA_MODE_CONC, ratio, t, p1=p1, p2=p2)
    assert bi == 0 and a >= 1 and b >= 1
    assert a + b == pytest.approx(p2 * t, rel=1e-6)
    res = so.minimize_scalar(lambda x: -st.beta(a, b).logpdf(x), bounds=(1e-9, 1 - 1e-9),
                             method="bounded", options={"xatol": 1e-10})
    assert res.x == pytest.approx(p1 * ratio, abs=1e-4)


def test_shape_stage_one_defaults_equal_paper_stage_one():
    """Mean 1/3, variance 1/18 and mode 0, concentration 3 both give Beta(1, 2),
    the paper's stage-1 shape (a_1 = eps_1/eps_1 = 1, b_1 = 2)."""
    a, b, _ = O.beta_shape(O.BETA_MEAN_VAR, 1.0, 1, p1=1 / 3, p2=1 / 18)
    assert (a, b) == pytest.approx((1.0, 2.0), rel=1e-6)
    a, b, _ = O.beta_shape(O.BETA_MODE_CONC, 1.0, 1, p1=0.0, p2=3.0)
    assert (a, b) == (1.0, 2.0)
    # and at stage t the mode-concentration rule stays Beta(1, 3t - 1)
    a, b, _ = O.beta_shape(O.BETA_MODE_CONC, 0.1, 4, p1=0.0, p2=3.0)
    assert (a, b) == (1.0, 11.0)


def test_shape_clamps():
    a, b, _ = O.beta_shape(O.BETA_MEAN_VAR, 0.0, 2, p1=0.3, p2=0.01)
    assert a == 2.0 ** -20 and b == pytest.approx(1 / 16)
    a, b, _ = O.beta_shape(O.BETA_MODE_CONC, 0.5, 60000, p1=0.5, p2=100.0)
    assert a == 2.0 ** 20 and b == 2.0 ** 20


def test_propose_real_shapes_use_gamma_ratio():
    """With beta_b = 0 the proposal's first-attempt s is the Gamma-ratio draw."""
    m = O.OracleModel(model=1, seed=5)
    n = 64
    rng = np.random.default_rng(3)
    u = rng.uniform(0.3, 0.7, (8, n)).astype(np.float32)
    pre = np.cumsum(np.ones(n, np.uint64)).astype(np.uint64)
    c1 = (3 << 16) | 1
    out = O.propose(m, u, pre, n, 0.4, 0, 300, c1, beta_bf=2.6)
    first = out["attempts"] == 1
    assert first.sum() > 50
    ref = np.array([O.beta_real(m.key, 0.4, 2.6, j, c1, 0) for j in np.flatnonzero(first)],
                   np.float32)
    np.testing.assert_array_equal(out["s"][first], ref)


MUTANTS = {
    "9d -> 3d": ("1.0f / sqrtf(9.0f * d)", "1.0f / sqrtf(3.0f * d)"),
    "no shape<1 boost": ("if (alpha < 1.0f) lg = lg +", "if (0) lg = lg +"),
    "x^2 without 1/2": ("0.5f * x2 + d *", "x2 + d *"),
    "log v for log dv": ("lg = or_logf(d * v);", "lg = or_logf(v);"),
    "1/3 -> 1/2": ("al - 0x1.555556p-2f", "al - 0.5f"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_sampler_mistakes_fail_the_ks_pins(name, tmp_path):
    """A copy of the oracle with one plausible mistake in the Gamma sampler
    fails the KS pins above (the oracle under test passes them)."""
    import ctypes as C
    import os
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = open(os.path.join(root, "oracle", "abc_oracle.c")).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1
    c = tmp_path / "mut.c"
    c.write_text(src.replace(old, new))
    so = tmp_path / "mut.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=gnu11", str(c),
                    "-o", str(so), "-lm"], check=True)
    L = C.CDLL(str(so))
    L.or_gamma_log.restype = C.c_float
    L.or_gamma_log.argtypes = [C.POINTER(C.c_uint32), C.c_float] + [C.c_uint32] * 4
    key = (C.c_uint32 * 2)(*KEY)
    worst = 1.0
    for alpha in [0.05, 0.3, 1.0, 2.5, 17.3, 900.0]:
        x = np.exp([L.or_gamma_log(key, alpha, j, 9, 0, 0) for j in range(12000)])
        worst = min(worst, st.kstest(x, st.gamma(alpha).cdf).pvalue)
    assert worst < 1e-3
