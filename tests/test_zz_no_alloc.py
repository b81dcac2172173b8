"""abc_resample_prefix_noalloc: the stage-prior prefix scan for callers that
cannot allocate device memory when they run it (for example when their
device memory belongs to a pool or a budget they do not control).  It must
give exactly what the allocating entry point gives -- the outputs are
integers, so the tolerance is zero -- on consecutive calls that share the
library's fixed scratch array, and refuse sizes above that array's limit.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import paper_2106_15508_gb300 as G
from paper_2106_15508_gb300 import build as B

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    a = np.ascontiguousarray(a)
    view = {np.dtype(np.uint32): np.int32, np.dtype(np.uint64): np.int64}.get(a.dtype)
    return torch.from_numpy(a.view(view) if view else a).cuda()


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    d = rng.integers(0, 5000, n).astype(np.float64)  # ties at the tolerance
    W = rng.lognormal(0.0, 2.0, n)
    eps = float(np.sort(d)[(n + 1) // 2 - 1])
    return d, W / W.sum(), eps


def _run(n, seed, mode, noalloc):
    d, W, eps = _inputs(n, seed)
    q = torch.empty(n, dtype=torch.int32, device="cuda")
    pre = torch.empty(n, dtype=torch.int64, device="cuda")
    if noalloc:
        G.abc_resample_prefix_noalloc(_dev(d), _dev(W), n, _dev(np.array([eps])), mode, q, pre)
    else:
        sc = torch.empty(G.abc_prefix_scratch_bytes(n), dtype=torch.uint8, device="cuda")
        G.abc_resample_prefix(_dev(d), _dev(W), n, _dev(np.array([eps])), mode, q, pre, sc,
                              sc.numel())
    torch.cuda.synchronize()
    return q.cpu().numpy().view(np.uint32), pre.cpu().numpy().view(np.uint64)


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    G.lib()


@pytest.mark.parametrize("mode", [G.ABC_W_PAPER, G.ABC_W_IMPORTANCE])
def test_noalloc_prefix_matches_allocating_entry_point(mode):
    # two calls in a row on the shared scratch: a large one, then a smaller
    # one that must not see anything the first left behind
    for n, seed in ((3_000_017, 11), (40_961, 12)):
        q_ref, pre_ref = _run(n, seed, mode, noalloc=False)
        q_na, pre_na = _run(n, seed, mode, noalloc=True)
        assert np.array_equal(q_na, q_ref)
        assert np.array_equal(pre_na, pre_ref)
        assert int(pre_na[-1]) == int(q_ref.astype(np.uint64).sum())


def test_noalloc_prefix_at_its_maximum_size():
    # n = 2^24 is the one size whose tile sums fill the whole fixed array;
    # a small call after it must not see what it left there
    for n, seed in ((G.ABC_NOALLOC_MAX_N, 13), (4097, 14)):
        q_ref, pre_ref = _run(n, seed, G.ABC_W_IMPORTANCE, noalloc=False)
        q_na, pre_na = _run(n, seed, G.ABC_W_IMPORTANCE, noalloc=True)
        assert np.array_equal(q_na, q_ref)
        assert np.array_equal(pre_na, pre_ref)


def test_noalloc_prefix_rejects_sizes_above_its_scratch():
    n = G.ABC_NOALLOC_MAX_N + 1
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    q = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(G.AbcError) as e:
        G.abc_resample_prefix_noalloc(x, x, n, x, G.ABC_W_PAPER, q, q)
    assert e.value.code == G.ABC_E_TOO_LARGE
