"""The fp32 constants of the device numerics (csrc/numerics.cuh) are the
correctly rounded values of their definitions (exact rational arithmetic;
independent of the oracle, which has its own copy and its own pin)."""
import math
import os
import re
from fractions import Fraction

import numpy as np
import sympy

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2106_15508_gb300", "csrc", "numerics.cuh")


def _rn32(x: Fraction) -> np.float32:
    c = np.float32(float(x))
    cands = [np.nextafter(c, np.float32(-np.inf)), c, np.nextafter(c, np.float32(np.inf))]
    return np.float32(min(cands, key=lambda v: (abs(Fraction(float(v)) - x),
                                                int(np.float32(v).view(np.uint32)) & 1)))


def _exact(expr) -> Fraction:
    return Fraction(str(sympy.N(expr, 60)))


def test_device_constants_are_correctly_rounded():
    consts = dict(re.findall(r"constexpr float (k\w+) = ([0-9.eE+-]+)f;", open(SRC).read()))
    head = Fraction(0.693145751953125)
    want = {"kLn2Hi": head, "kLn2Lo": _exact(sympy.log(2)) - head,
            "kLog2e": _exact(1 / sympy.log(2)), "kTwoPi": _exact(2 * sympy.pi),
            "kSqrt2": _exact(sympy.sqrt(2))}
    for k in range(2, 14):
        want["kF%d" % k] = Fraction(1, math.factorial(k))
    for k in (3, 5, 7, 9, 11):
        want["kO%d" % k] = Fraction(1, k)
    assert set(want) <= set(consts)
    for name, v in want.items():
        assert np.float32(float(consts[name])) == _rn32(v), name
    # the 15-bit head makes e * LN2_HI exact for |e| < 2^9
    assert (int(np.float32(0.693145751953125).view(np.uint32)) & 0x1FF) == 0


def test_uniform_from_bits_equals_direct_form():
    """unif() builds ((x >> 9) + 1/2) 2^-23 as 1.m - (1 - 2^-24) from the bits of
    x: the float 1.m is exact and so is the difference, so one rounded
    subtraction gives the direct form exactly, for all 2^23 significands
    (the device check abc_numerics_check(3) repeats this on the GPU)."""
    src = open(SRC).read()
    assert "__uint_as_float((x >> 9) | 0x3F800000u), 0x1.fffffep-1f" in src
    m = np.arange(1 << 23, dtype=np.uint32)
    direct = (m.astype(np.float32) + np.float32(0.5)) * np.float32(2.0**-23)
    one_m = (m | np.uint32(0x3F800000)).view(np.float32)
    bits = one_m - np.float32(1.0 - 2.0**-24)
    assert np.float32(1.0 - 2.0**-24).view(np.uint32) == 0x3F7FFFFF
    assert np.array_equal(direct.view(np.uint32), bits.view(np.uint32))
