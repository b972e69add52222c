"""Parity at the workloads' full sizes, in the launch configuration the
benchmark times, on sampled outputs the oracle recomputes one by one.

- 150 bp, E = 6, 20M pairs (the benchmark step: pack, tuned batched filter
  with both deciders, compaction, verification)
- mixed lengths 100/150/250 and thresholds, 50M pairs (one scheduler call
  over ragged arrays), and the same through the chunked host pipeline
- 250 bp, E = 25, 10M pairs: filter + verify, and verification of all pairs
- 100 bp, E = 5, 100k pairs from ASCII: every pair
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu
SAMPLE = 20000


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


def subset(P, idx):
    return synth.Pairs(P.reads, P.refs, P.read_off[idx], P.ref_off[idx], P.lens[idx], P.E[idx])


def expected(P, deciders=3):
    acc, cnt = oracle.filter_batch(P, deciders=deciders)
    vb = oracle.verify_batch(P)
    return acc, cnt, np.where(acc[0] == 1, vb, P.E.astype(np.int32) + 1)


def run_path(pf, ctx, P, fixed=None, E_max=None):
    dev = "cuda:0"
    reads = torch.from_numpy(P.reads).to(dev)
    refs = torch.from_numpy(P.refs).to(dev)
    if fixed:
        pairs = pf.pack_pairs(ctx, reads, refs, length=fixed)
    else:
        pairs = pf.pack_pairs(ctx, reads, refs, byte_off=P.read_off)
    del reads, refs
    n = P.n
    lens = torch.from_numpy(P.lens).to(dev)
    E = torch.from_numpy(P.E).to(dev)
    acc = torch.zeros(2 * n, dtype=torch.uint8, device=dev)
    cnt = torch.zeros(2 * n, dtype=torch.int16, device=dev)
    dist = torch.zeros(n, dtype=torch.int32, device=dev)
    pf.pf_filter_verify(ctx, 3, pairs, lens, E, int(P.E.max()) if E_max is None else E_max,
                        acc, cnt, dist, n)
    pf.pf_sync(ctx)
    return pairs, lens, E, acc.cpu().numpy().reshape(2, n), cnt.cpu().numpy().reshape(2, n), \
        dist.cpu().numpy()


def check_sample(P, acc, cnt, dist, seed):
    idx = np.sort(np.random.default_rng(seed).choice(P.n, size=min(SAMPLE, P.n), replace=False))
    oa, oc, od = expected(subset(P, idx))
    assert np.array_equal(cnt[:, idx], oc)
    assert np.array_equal(acc[:, idx], oa)
    assert np.array_equal(dist[idx], od)


def test_headline_step_20M(pf, ctx):
    P = synth.generate(synth.SKEWED, 0x5EED0001, 20_000_000, m=150, E=6, kmax=60)
    # the benchmark's launch configuration: the autotuner's choice on the
    # first 2M pairs, as the benchmark makes it
    dev = "cuda:0"
    reads = torch.from_numpy(P.reads[:2_000_000 * 150]).to(dev)
    refs = torch.from_numpy(P.refs[:2_000_000 * 150]).to(dev)
    sample = pf.pack_pairs(ctx, reads, refs, length=150)
    lens = torch.full((2_000_000,), 150, dtype=torch.int32, device=dev)
    for dec in (1, 3):
        cfg, chunk, _ = pf.pf_tune(ctx, dec, sample, lens, 6, n=2_000_000, reps=2)
        assert pf.pf_tune_get(ctx, dec, 6) == (cfg, chunk)
    del reads, refs, sample, lens
    _, _, _, acc, cnt, dist = run_path(pf, ctx, P, fixed=150)
    check_sample(P, acc, cnt, dist, 1)
    # accept flags and distances agree with each other everywhere
    assert np.all((dist <= 6) <= (acc[0] == 1))
    # and the fused and two-phase forms of the exact-E6 kernel give the same
    # results on the whole batch
    cfgs = pf.pf_kernel_configs()
    for form in [i for i, c in enumerate(cfgs) if c[3] == 6]:
        pf.pf_tune_set(ctx, 3, 6, form, 64)
        _, _, _, a2, c2, d2 = run_path(pf, ctx, P, fixed=150)
        assert np.array_equal(a2, acc) and np.array_equal(c2, cnt) and np.array_equal(d2, dist)


def test_mixed_50M_device_and_host_pipeline(pf, ctx):
    P = synth.generate(synth.MIXED, 0x5EED0003, 50_000_000, kmax=60)
    _, _, _, acc, cnt, dist = run_path(pf, ctx, P)
    check_sample(P, acc, cnt, dist, 2)
    # the chunked host pipeline on a 5M-pair slice gives the same results
    Q = synth.generate(synth.MIXED, 0x5EED0003, 5_000_000, kmax=60)
    a2, c2, d2 = pf.pf_run_host(ctx, 3, Q.reads, Q.refs, 20, byte_off=Q.read_off, E=Q.E,
                                chunk_pairs=1 << 20)
    assert np.array_equal(a2, acc[:, :Q.n]) and np.array_equal(c2, cnt[:, :Q.n])
    assert np.array_equal(d2, dist[:Q.n])


def test_250bp_E25_10M_filter_verify_and_verify_all(pf, ctx):
    P = synth.generate(synth.SKEWED_ALL, 0x5EED0004, 10_000_000, m=250, E=25, kmax=100)
    pairs, lens, E, acc, cnt, dist = run_path(pf, ctx, P, fixed=250)
    check_sample(P, acc, cnt, dist, 3)
    all_d = torch.zeros(P.n, dtype=torch.int32, device="cuda:0")
    pf.pf_verify(ctx, pairs, lens, E, 25, None, None, all_d, P.n)
    pf.pf_sync(ctx)
    all_d = all_d.cpu().numpy()
    idx = np.sort(np.random.default_rng(4).choice(P.n, size=SAMPLE, replace=False))
    assert np.array_equal(all_d[idx], oracle.verify_batch(subset(P, idx)))
    # filtering never loses a pair within E: the verified distances match
    acc_mask = acc[0] == 1
    assert np.array_equal(dist[acc_mask], all_d[acc_mask])
    assert np.all(all_d[~acc_mask] == 26)


def test_uniform_100bp_E5_100k_every_pair(pf, ctx):
    P = synth.generate(synth.UNIFORM, 0x5EED0000, 100_000, m=100, E=5, kmax=20)
    _, _, _, acc, cnt, dist = run_path(pf, ctx, P, fixed=100)
    oa, oc, od = expected(P)
    assert np.array_equal(cnt, oc) and np.array_equal(acc, oa) and np.array_equal(dist, od)
