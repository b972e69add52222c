"""GPU parity of the thesis's other deciders against the oracle, bit-exact:
SneakySnake on sub-matrices (§8.5), Shouji (Ch. 6) and GateKeeper with
SHD's conventions (Ch. 3).  Every call goes through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import synth
from conftest import ArrayPairs, all_pairs
from gpu_util import DevicePairs, DEV
from test_gpu_parity import edge_items, explicit_pairs

pytestmark = pytest.mark.gpu

PARTITIONS = [(8, 2), (8, 8), (5, 3), (32, 32), (1, 1), (13, 4), (32, 1), (3, 100)]


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


def run(pf, ctx, fn, D, *extra, per_pair_E=True):
    acc = torch.full((max(D.n, 1),), 0xEE, dtype=torch.uint8, device=DEV)
    cnt = torch.full((max(D.n, 1),), -7, dtype=torch.int16, device=DEV)
    fn(ctx, D.pairs, D.lens, D.E if per_pair_E else None, D.E_max, *extra, acc, cnt, D.n)
    pf.pf_sync(ctx)
    return acc.cpu().numpy()[:D.n], cnt.cpu().numpy()[:D.n]


def check(acc, cnt, want, E):
    assert np.array_equal(cnt, want)
    assert np.array_equal(acc, (want <= E).astype(np.uint8))


CASES = [
    ("cfg1_uniform_100bp_E5", synth.UNIFORM, 100, 5, 20, 6000),
    ("cfg2_150bp_E0", synth.SKEWED, 150, 0, 60, 4000),
    ("cfg2_150bp_E6", synth.SKEWED, 150, 6, 60, 8000),
    ("cfg2_150bp_E15", synth.SKEWED, 150, 15, 60, 4000),
    ("cfg3_mixed", synth.MIXED, 0, 0, 60, 8000),
    ("cfg4_250bp_E25", synth.SKEWED_ALL, 250, 25, 100, 2000),
]


@pytest.fixture(scope="module")
def cases(pf, ctx):
    out = {}
    for name, kind, m, E, km, n in CASES:
        P = synth.generate(kind, 0x5EED0700 + n + m + E, n, m=m or 150, E=E, kmax=km)
        out[name] = (P, DevicePairs(ctx, P))
    return out


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_partitioned_matches_oracle(pf, ctx, cases, name):
    P, D = cases[name]
    for t, y in PARTITIONS:
        want = oracle.int_batch("ss_partitioned", P, p0=t, p1=y)
        acc, cnt = run(pf, ctx, pf.pf_filter_partitioned, D, t, y)
        check(acc, cnt, want, P.E)


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_shouji_matches_oracle(pf, ctx, cases, name):
    P, D = cases[name]
    want = oracle.int_batch("shouji", P)
    acc, cnt = run(pf, ctx, pf.pf_filter_shouji, D)
    check(acc, cnt, want, P.E)


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_shd_matches_oracle(pf, ctx, cases, name):
    P, D = cases[name]
    for flags in (0, 1, 2, 3):
        want = oracle.int_batch("gk_shd", P, p0=flags & 1, p1=(flags >> 1) & 1)
        acc, cnt = run(pf, ctx, pf.pf_filter_shd, D, flags)
        check(acc, cnt, want, P.E)
    # no switch: GateKeeper of the fused filter
    _, gk = oracle.filter_batch(P, deciders=oracle.GATEKEEPER)
    _, cnt = run(pf, ctx, pf.pf_filter_shd, D, 0)
    assert np.array_equal(cnt, gk[0])


def test_edge_items(pf, ctx):
    P = explicit_pairs(edge_items())
    D = DevicePairs(ctx, P)
    for t, y in PARTITIONS:
        acc, cnt = run(pf, ctx, pf.pf_filter_partitioned, D, t, y)
        check(acc, cnt, oracle.int_batch("ss_partitioned", P, p0=t, p1=y), P.E)
    acc, cnt = run(pf, ctx, pf.pf_filter_shouji, D)
    check(acc, cnt, oracle.int_batch("shouji", P), P.E)
    for flags in (0, 1, 2, 3):
        acc, cnt = run(pf, ctx, pf.pf_filter_shd, D, flags)
        check(acc, cnt, oracle.int_batch("gk_shd", P, p0=flags & 1, p1=flags >> 1), P.E)


@pytest.mark.parametrize("E", [0, 1, 2, 3])
def test_exhaustive_len4(pf, ctx, E):
    reads, refs = all_pairs("ACGN", 4)
    P = ArrayPairs(reads, refs, E)
    Pd = synth.Pairs(P.reads, P.refs, P.read_off, P.ref_off, P.lens, P.E)
    D = DevicePairs(ctx, Pd, fixed=4)
    for t, y in ((1, 1), (2, 1), (2, 2), (3, 2), (4, 4)):
        acc, cnt = run(pf, ctx, pf.pf_filter_partitioned, D, t, y)
        check(acc, cnt, oracle.int_batch("ss_partitioned", P, p0=t, p1=y), E)
    acc, cnt = run(pf, ctx, pf.pf_filter_shouji, D)
    check(acc, cnt, oracle.int_batch("shouji", P), E)
    for flags in (0, 1, 2, 3):
        acc, cnt = run(pf, ctx, pf.pf_filter_shd, D, flags)
        check(acc, cnt, oracle.int_batch("gk_shd", P, p0=flags & 1, p1=flags >> 1), E)


def test_uniform_threshold_without_E_array(pf, ctx, cases):
    P, D = cases["cfg2_150bp_E6"]
    acc, cnt = run(pf, ctx, pf.pf_filter_shouji, D, per_pair_E=False)
    check(acc, cnt, oracle.int_batch("shouji", P), 6)
    acc, cnt = run(pf, ctx, pf.pf_filter_partitioned, D, 8, 2, per_pair_E=False)
    check(acc, cnt, oracle.int_batch("ss_partitioned", P, p0=8, p1=2), 6)


def test_invalid_arguments(pf, ctx, cases):
    P, D = cases["cfg2_150bp_E6"]
    acc = torch.zeros(D.n, dtype=torch.uint8, device=DEV)
    cnt = torch.zeros(D.n, dtype=torch.int16, device=DEV)
    for t, y in ((0, 1), (33, 1), (8, 0)):
        with pytest.raises(pf.PFError):
            pf.pf_filter_partitioned(ctx, D.pairs, D.lens, D.E, 6, t, y, acc, cnt, D.n)
    with pytest.raises(pf.PFError):
        pf.pf_filter_shd(ctx, D.pairs, D.lens, D.E, 6, 4, acc, cnt, D.n)
    with pytest.raises(pf.PFError):
        pf.pf_filter_shouji(ctx, D.pairs, D.lens, D.E, 32, acc, cnt, D.n)
    # a pair whose E exceeds E_max is marked on the device and reported
    Q = explicit_pairs([("ACGT", "ACGT", 2), ("ACGT", "ACGA", 9), ("ACGT", "ACGT", 1)])
    DQ = DevicePairs(ctx, Q)
    for fn, extra in ((pf.pf_filter_partitioned, (8, 2)), (pf.pf_filter_shouji, ()),
                      (pf.pf_filter_shd, (3,))):
        a = torch.zeros(3, dtype=torch.uint8, device=DEV)
        c = torch.zeros(3, dtype=torch.int16, device=DEV)
        fn(ctx, DQ.pairs, DQ.lens, DQ.E, 3, *extra, a, c, 3)
        with pytest.raises(pf.PFError):
            pf.pf_sync(ctx)
        pf.pf_sync(ctx)
        assert c.cpu().tolist() == [0, -1, 0]


def test_full_size_sampled(pf, ctx):
    """The 20M-pair 150 bp, E = 6 workload: every variant on the whole
    batch, sampled outputs recomputed by the oracle."""
    P = synth.generate(synth.SKEWED, 0x5EED0001, 20_000_000, m=150, E=6, kmax=60)
    reads = torch.from_numpy(P.reads).to(DEV)
    refs = torch.from_numpy(P.refs).to(DEV)
    pairs = pf.pack_pairs(ctx, reads, refs, length=150)
    del reads, refs
    lens = torch.full((P.n,), 150, dtype=torch.int32, device=DEV)
    E = torch.full((P.n,), 6, dtype=torch.int16, device=DEV)
    idx = np.sort(np.random.default_rng(7).choice(P.n, size=20000, replace=False))
    sub = synth.Pairs(P.reads, P.refs, P.read_off[idx], P.ref_off[idx], P.lens[idx], P.E[idx])
    acc = torch.empty(P.n, dtype=torch.uint8, device=DEV)
    cnt = torch.empty(P.n, dtype=torch.int16, device=DEV)
    for fn, extra, kind, p in ((pf.pf_filter_partitioned, (8, 2), "ss_partitioned", (8, 2)),
                               (pf.pf_filter_shouji, (), "shouji", (0, 0)),
                               (pf.pf_filter_shd, (3,), "gk_shd", (1, 1))):
        fn(ctx, pairs, lens, E, 6, *extra, acc, cnt, P.n)
        pf.pf_sync(ctx)
        want = oracle.int_batch(kind, sub, p0=p[0], p1=p[1])
        assert np.array_equal(cnt.cpu().numpy()[idx], want)
        assert np.array_equal(acc.cpu().numpy()[idx], (want <= 6).astype(np.uint8))


def test_false_reject_examples_on_the_gpu(pf, ctx, golden):
    # the hand-traced pairs that GateKeeper and Shouji reject although their
    # edit distance is within E: the kernels reproduce those counts, and
    # SneakySnake and the verifier accept them with their distance
    from gpu_util import filter_dev, verify_dev
    for name, slot in (("gatekeeper_false_reject.txt", "gk"), ("shouji_false_reject.txt", "sh")):
        kv, _ = golden(name)
        E = int(kv["E"])
        reads = np.frombuffer(kv["read"].encode(), np.uint8)[None, :]
        refs = np.frombuffer(kv["ref"].encode(), np.uint8)[None, :]
        D = DevicePairs(ctx, ArrayPairs(reads, refs, E), fixed=reads.shape[1])
        acc, cnt = filter_dev(ctx, D, 3)
        assert cnt[0, 0] <= int(kv["edit_distance"]) and acc[0, 0] == 1
        if slot == "gk":
            assert cnt[1, 0] == int(kv["count"]) and acc[1, 0] == 0
        else:
            a, c = run(pf, ctx, pf.pf_filter_shouji, D)
            assert c[0] == int(kv["count"]) and a[0] == 0
        assert verify_dev(ctx, D)[0] == int(kv["edit_distance"])
