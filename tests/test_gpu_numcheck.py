"""The short division sequence (the quotient by the reciprocal approximation,
corrected once by its exact remainder, after Markstein) that the logarithm and the BINV loop use
on bounded operand domains equals CUDA's correctly rounded __fdiv_rn on
every operand pair of those domains, and the square root of the binomial and
Box-Muller draws (reciprocal-square-root approximation, one remainder
correction) equals __fsqrt_rn on [2^-24, 2^32); and the uniform built from
a Philox word's bits equals its direct form by integer-to-float conversion
for every 23-bit significand; all enumerated on the device."""
import pytest

import paper_2106_15508_gb300 as G
from paper_2106_15508_gb300 import build as B

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    G.lib()


@pytest.mark.parametrize("which", [0, 1, 2, 3])
def test_short_sequences_are_exact_on_their_domains(which):
    assert G.abc_numerics_check(which) == 0


def test_unknown_check_is_rejected():
    with pytest.raises(G.AbcError):
        G.abc_numerics_check(7)
