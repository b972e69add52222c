"""pf_run_host: the whole path on host buffers, chunked over two slots and
replayed as CUDA graphs, bit-exact with the oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    from paper_1910_03936_gb300 import build
    build.build()
    import paper_1910_03936_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(pf):
    c = pf.pf_create(0)
    yield c
    pf.pf_destroy(c)


def expected(P, deciders):
    acc, cnt = oracle.filter_batch(P, deciders=deciders)
    vb = oracle.verify_batch(P)
    return acc, cnt, np.where(acc[0] == 1, vb, P.E.astype(np.int32) + 1)


@pytest.mark.parametrize("chunk", [1000, 4096, 0])
@pytest.mark.parametrize("dec", [3, 1])
def test_ragged_chunks(pf, ctx, chunk, dec):
    P = synth.generate(synth.MIXED, 21, 10007)
    acc, cnt, dist = pf.pf_run_host(ctx, dec, P.reads, P.refs, int(P.E.max()),
                                    byte_off=P.read_off, E=P.E, chunk_pairs=chunk)
    oa, oc, od = expected(P, dec)
    assert np.array_equal(cnt, oc) and np.array_equal(acc, oa)
    assert np.array_equal(dist, od)


@pytest.mark.parametrize("chunk", [777, 5000])
def test_fixed_length_uniform_E(pf, ctx, chunk):
    P = synth.generate(synth.SKEWED, 22, 9001, m=150, E=6)
    acc, cnt, dist = pf.pf_run_host(ctx, 3, P.reads, P.refs, 6, length=150, chunk_pairs=chunk)
    oa, oc, od = expected(P, 3)
    assert np.array_equal(cnt, oc) and np.array_equal(acc, oa)
    assert np.array_equal(dist, od)


def test_pinned_host_buffers(pf, ctx):
    import torch
    P = synth.generate(synth.SKEWED_ALL, 23, 3000, m=250, E=25, kmax=100)
    reads = torch.from_numpy(P.reads).pin_memory().numpy()
    refs = torch.from_numpy(P.refs).pin_memory().numpy()
    acc, cnt, dist = pf.pf_run_host(ctx, 3, reads, refs, 25, length=250, E=P.E, chunk_pairs=1024)
    oa, oc, od = expected(P, 3)
    assert np.array_equal(cnt, oc) and np.array_equal(acc, oa)
    assert np.array_equal(dist, od)


def test_huge_page_host_buffers(pf, ctx):
    """Inputs and outputs in pf_host_alloc memory: the same results; the
    block is page-locked (the CUDA runtime sees host memory) and 256-byte
    aligned; a freed block's space is reused; freeing an unknown pointer is
    refused."""
    import ctypes
    import torch
    P = synth.generate(synth.MIXED, 24, 5003)
    reads = pf.host_empty(P.reads.size, np.uint8)
    reads[:] = P.reads
    refs = pf.host_empty(P.refs.size, np.uint8)
    refs[:] = P.refs
    off = pf.host_empty(P.read_off.size, np.int64)
    off[:] = P.read_off
    E = pf.host_empty(P.E.size, np.int16)
    E[:] = P.E
    out = (pf.host_empty(2 * P.n, np.uint8), pf.host_empty(2 * P.n, np.int16),
           pf.host_empty(P.n, np.int32))
    assert reads.ctypes.data % 256 == 0
    assert torch.from_numpy(reads).is_pinned()
    acc, cnt, dist = pf.pf_run_host(ctx, 3, reads, refs, int(P.E.max()), byte_off=off, E=E,
                                    chunk_pairs=2048, out=out)
    oa, oc, od = expected(P, 3)
    assert np.array_equal(cnt, oc) and np.array_equal(acc, oa)
    assert np.array_equal(dist, od)
    import gc
    gc.collect()
    gc.disable()  # no finalizer frees other blocks between the calls below
    try:
        addr = pf.pf_host_alloc(3 << 20)
        pf.pf_host_free(addr)
        assert pf.pf_host_alloc(3 << 20) == addr  # first fit: the same space again
        pf.pf_host_free(addr)
    finally:
        gc.enable()
    with pytest.raises(pf.PFError):
        pf.pf_host_free(addr)  # already freed: unknown
    pf.pf_host_free(None)
