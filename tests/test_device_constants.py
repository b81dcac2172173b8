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
