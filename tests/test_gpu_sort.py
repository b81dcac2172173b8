"""The stable radix sort behind the weight pass's spatial order, through
abc_radix_sort, against numpy's stable argsort: bit-exact keys and payloads
(equal keys keep their input order), ragged sizes, few and many distinct
keys, partial key widths."""
import numpy as np
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


@pytest.mark.parametrize("n,bits,distinct", [(1, 8, 4), (1023, 16, 7), (1025, 18, 1 << 18),
                                             (300_001, 16, 3), (1 << 20, 32, 1 << 32),
                                             (77_777, 12, 1 << 12), (5000, 1, 2)])
def test_radix_sort_matches_stable_argsort(n, bits, distinct):
    rng = np.random.default_rng(n + bits)
    keys = rng.integers(0, min(distinct, 1 << 32), n, dtype=np.uint64).astype(np.uint32)
    vals = rng.integers(-2**31, 2**31 - 1, n, dtype=np.int64).astype(np.int32)
    kd = torch.from_numpy(keys.view(np.int32)).cuda()
    vd = torch.from_numpy(vals).cuda()
    ko = torch.empty_like(kd)
    vo = torch.empty_like(vd)
    G.abc_radix_sort(kd, vd, n, bits, ko, vo)
    masked = keys & np.uint32((1 << bits) - 1) if bits < 32 else keys
    order = np.argsort(masked, kind="stable")
    torch.cuda.synchronize()
    assert np.array_equal(ko.cpu().numpy().view(np.uint32), keys[order])
    assert np.array_equal(vo.cpu().numpy(), vals[order])


def test_radix_sort_default_payload_is_the_index():
    n = 4099
    keys = (np.arange(n, dtype=np.uint32) * 2654435761) >> np.uint32(20)
    kd = torch.from_numpy(keys.view(np.int32)).cuda()
    ko = torch.empty_like(kd)
    vo = torch.empty(n, dtype=torch.int32, device="cuda")
    G.abc_radix_sort(kd, None, n, 12, ko, vo)
    torch.cuda.synchronize()
    assert np.array_equal(vo.cpu().numpy(), np.argsort(keys, kind="stable"))


def test_radix_sort_rejects_bad_arguments():
    kd = torch.zeros(8, dtype=torch.int32, device="cuda")
    vo = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(G.AbcError):
        G.abc_radix_sort(kd, None, 8, 0, kd.clone(), vo)
    with pytest.raises(G.AbcError):
        G.abc_radix_sort(kd, None, 8, 16, kd, vo)  # output aliases the input
