"""pf_compact_noalloc: compaction for callers that cannot allocate device
memory (a framework-owned allocator, a path that cannot take cudaMalloc's
implicit synchronisation).

It must give exactly what pf_compact gives, call after call, although its
counters live in one fixed device array shared by every call.  This file
runs last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    from paper_1910_03936_gb300 import build
    build.build()
    import paper_1910_03936_gb300 as m
    return m


def _flags(seed, n, p):
    rng = np.random.default_rng(seed)
    f = (rng.random(n) < p).astype(np.uint8) * rng.integers(1, 255, size=n).astype(np.uint8)
    return torch.from_numpy(f).cuda()


def test_noalloc_matches_pf_compact_twice(pf):
    ctx = pf.pf_create(0)
    try:
        # two calls in a row with different data and sizes: the second call
        # must not see anything the first one left in the shared counters
        for seed, n, p in ((1, 1_000_003, 0.3), (2, 250_001, 0.7)):
            f = _flags(seed, n, p)
            idx_a = torch.full((n,), -1, dtype=torch.int64, device="cuda:0")
            idx_b = torch.full((n,), -2, dtype=torch.int64, device="cuda:0")
            k_a = torch.full((1,), -1, dtype=torch.int64, device="cuda:0")
            k_b = torch.full((1,), -2, dtype=torch.int64, device="cuda:0")
            pf.pf_compact(ctx, f, idx_a, k_a, n)
            pf.pf_sync(ctx)
            pf.pf_compact_noalloc(f, idx_b, k_b, n)
            torch.cuda.synchronize()
            k = int(k_a.item())
            assert k == int(k_b.item())
            assert torch.equal(idx_a[:k], idx_b[:k])
            assert k == int(np.count_nonzero(f.cpu().numpy()))
    finally:
        pf.pf_destroy(ctx)


def test_noalloc_rejects_sizes_beyond_its_array(pf):
    # buffers really hold n elements, so that a regression of the host-side
    # size check shows up as a wrong status or result, never as an access
    # outside a buffer
    n = 134_217_728 + 1
    f = torch.zeros(n, dtype=torch.uint8, device="cuda:0")
    f[::1000] = 1
    idx = torch.full((n,), -5, dtype=torch.int64, device="cuda:0")
    k = torch.full((1,), -3, dtype=torch.int64, device="cuda:0")
    with pytest.raises(pf.PFError) as ei:
        pf.pf_compact_noalloc(f, idx, k, n)   # rejected on the host, nothing launched
    assert ei.value.status == 1
    torch.cuda.synchronize()
    assert int(k.item()) == -3                 # nothing was written
    assert bool((idx[:1000] == -5).all()) and bool((idx[-1000:] == -5).all())
    del f, idx
    torch.cuda.empty_cache()
