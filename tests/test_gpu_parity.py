"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Sizes span several tiles and warps with ragged tails; every kernel
configuration of the batch scheduler is exercised; edge cases cover empty
pairs, lengths around word boundaries, E = 0, E >= length, all-N and
lower-case input, invalid bytes and invalid per-pair thresholds.  Accept
flags, counts, packed words, indices and distances must be bit-exact.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from conftest import ArrayPairs

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
    pf.pf_set_small_batch(c, 0)  # these batches are small: exercise the scheduler's kernels
    yield c
    pf.pf_destroy(c)


def explicit_pairs(items):
    """synth.Pairs from a list of (read, ref, E)."""
    reads = b"".join(r.encode() for r, _, _ in items)
    refs = b"".join(f.encode() for _, f, _ in items)
    lens = np.array([len(r) for r, _, _ in items], dtype=np.int32)
    off = np.zeros(len(items) + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    E = np.array([e for _, _, e in items], dtype=np.int16)
    return synth.Pairs(np.frombuffer(reads, np.uint8).copy() if reads else np.zeros(0, np.uint8),
                       np.frombuffer(refs, np.uint8).copy() if refs else np.zeros(0, np.uint8),
                       off, off, lens, E)


def edge_items():
    rng = np.random.default_rng(2024)
    items = [("", "", 0), ("", "", 5), ("A", "A", 0), ("A", "C", 0), ("N", "N", 0),
             ("N", "N", 1), ("ACG", "ACG", 9), ("ACG", "TTT", 20), ("acgtn", "ACGTN", 1),
             ("GGTGAGAGTTGT", "GGTGGAGAGATC", 3), ("GGTGAGAGTTGT", "GGTGGAGAGATC", 2),
             ("N" * 40, "N" * 40, 31), ("A" * 64, "A" * 64, 0), ("A" * 64, "A" * 63 + "C", 0)]
    for L in (31, 32, 33, 63, 64, 65, 95, 96, 97, 127, 128, 129, 255, 256, 257, 300, 511, 1000):
        for E in (0, 1, 3, 7, 15, 31):
            ref = "".join(rng.choice(list("ACGT"), size=L))
            read = list(ref)
            for _ in range(int(rng.integers(0, E + 3))):
                pos = int(rng.integers(0, max(len(read), 1)))
                op = rng.random()
                if not read:
                    read.append("A")
                elif op < 0.5:
                    read[pos] = str(rng.choice(list("ACGTN")))
                elif op < 0.75:
                    read.insert(pos, str(rng.choice(list("ACGT"))))
                else:
                    del read[pos]
            read = ("".join(read) + ref)[:L]
            items.append((read, ref, E))
    return items


def oracle_filter(P, deciders):
    return oracle.filter_batch(P, deciders=deciders)


# ---- a1 pack ---------------------------------------------------------------

def test_pack_ragged_matches_oracle(pf, ctx):
    from gpu_util import to_dev
    P = synth.generate(synth.MIXED, 11, 3000)
    P2 = explicit_pairs(edge_items())
    for src, off in ((P.reads, P.read_off), (P2.refs, P2.ref_off)):
        wo, total = pf.pf_pack_layout(off)
        out = pf.Seqs.empty(total, "cuda:0", word_off=to_dev(wo))
        pf.pf_pack(ctx, to_dev(src if len(src) else np.zeros(1, np.uint8)), to_dev(off),
                   to_dev(wo), out)
        pf.pf_sync(ctx)
        owo, lo, hi, nm, bad = oracle.pack_batch(src, off)
        assert bad == 0
        assert np.array_equal(owo, wo)
        for got, want in ((out.lo, lo), (out.hi, hi), (out.nmask, nm)):
            assert np.array_equal(got.cpu().numpy()[:total].view(np.uint32), want)


@pytest.mark.parametrize("length", [1, 31, 32, 33, 100, 150, 250, 257])
def test_pack_fixed_matches_oracle(pf, ctx, length):
    from gpu_util import to_dev
    rng = np.random.default_rng(length)
    n = 777
    src = rng.choice(np.frombuffer(b"ACGTNacgtn", np.uint8), size=n * length)
    W = (length + 31) // 32
    out = pf.Seqs.empty(n * W, "cuda:0", stride_words=W)
    pf.pf_pack_fixed(ctx, to_dev(src), n, length, out)
    pf.pf_sync(ctx)
    off = np.arange(n + 1, dtype=np.int64) * length
    _, lo, hi, nm, _ = oracle.pack_batch(src, off)
    for got, want in ((out.lo, lo), (out.hi, hi), (out.nmask, nm)):
        assert np.array_equal(got.cpu().numpy().view(np.uint32), want)


def test_pack_unaligned_source(pf, ctx):
    from gpu_util import to_dev
    rng = np.random.default_rng(5)
    base = to_dev(rng.choice(np.frombuffer(b"ACGT", np.uint8), size=5000))
    for shift in (1, 2, 3, 5):
        src = base[shift:shift + 150 * 20]
        out = pf.Seqs.empty(20 * 5, "cuda:0", stride_words=5)
        pf.pf_pack_fixed(ctx, src, 20, 150, out)
        pf.pf_sync(ctx)
        host = base.cpu().numpy()[shift:shift + 3000]
        _, lo, hi, nm, _ = oracle.pack_batch(host, np.arange(21, dtype=np.int64) * 150)
        assert np.array_equal(out.lo.cpu().numpy().view(np.uint32), lo)
        assert np.array_equal(out.nmask.cpu().numpy().view(np.uint32), nm)


def test_pack_invalid_bytes_report_and_pack_as_n(pf, ctx):
    from gpu_util import to_dev
    seq = np.frombuffer(b"ACGTXACGT-ACGU" + b"A" * 30, np.uint8).copy()
    off = np.array([0, len(seq)], dtype=np.int64)
    wo, total = pf.pf_pack_layout(off)
    out = pf.Seqs.empty(total, "cuda:0", word_off=to_dev(wo))
    pf.pf_pack(ctx, to_dev(seq), to_dev(off), to_dev(wo), out)
    with pytest.raises(pf.PFError) as ei:
        pf.pf_sync(ctx)
    assert ei.value.status == 7
    _, lo, hi, nm, bad = oracle.pack_batch(seq, off)
    assert bad == 3
    assert np.array_equal(out.nmask.cpu().numpy()[:total].view(np.uint32), nm)
    assert np.array_equal(out.lo.cpu().numpy()[:total].view(np.uint32), lo)


def test_pack_neighbour_bytes_never_leak(pf, ctx):
    """Bytes past a sequence's end (the next sequence's, or whatever follows
    the buffer) never change its planes, and raise the error only when they
    belong to a sequence that holds them."""
    from gpu_util import to_dev
    rng = np.random.default_rng(9)
    acgt = np.frombuffer(b"ACGT", np.uint8)
    # ragged: a valid 40-byte sequence followed by one that starts with bad bytes
    seqs = [rng.choice(acgt, 40), np.frombuffer(b"XY#" + b"C" * 37, np.uint8),
            rng.choice(acgt, 33)]
    src = np.concatenate(seqs)
    off = np.array([0, 40, 80, 113], dtype=np.int64)
    wo, total = pf.pf_pack_layout(off)
    out = pf.Seqs.empty(total, "cuda:0", word_off=to_dev(wo))
    pf.pf_pack(ctx, to_dev(src), to_dev(off), to_dev(wo), out)
    with pytest.raises(pf.PFError):
        pf.pf_sync(ctx)
    _, lo, hi, nm, bad = oracle.pack_batch(src, off)
    assert bad == 3
    for got, want in ((out.lo, lo), (out.hi, hi), (out.nmask, nm)):
        assert np.array_equal(got.cpu().numpy()[:total].view(np.uint32), want)
    # fixed: the buffer is a slice followed by bytes that are not bases
    for length in (37, 150, 250):
        n = 64
        whole = np.concatenate([rng.choice(acgt, n * length), np.frombuffer(b"#" * 64, np.uint8)])
        dev = to_dev(whole)
        W = (length + 31) // 32
        out = pf.Seqs.empty(n * W, "cuda:0", stride_words=W)
        pf.pf_pack_fixed(ctx, dev[:n * length], n, length, out)
        pf.pf_sync(ctx)  # no error: the '#' bytes are outside every sequence
        _, lo, hi, nm, _ = oracle.pack_batch(whole[:n * length],
                                             np.arange(n + 1, dtype=np.int64) * length)
        for got, want in ((out.lo, lo), (out.hi, hi), (out.nmask, nm)):
            assert np.array_equal(got.cpu().numpy().view(np.uint32), want)


@pytest.mark.parametrize("maxlen", [70, 255, 600])
def test_pack_ragged_blocks_and_spare_words(pf, ctx, maxlen):
    """The ragged layout with empty sequences, short and long sequences
    from an unaligned start, bytes that are not bases before the first and
    after the last sequence (never an error) and inside (packed as N, an
    error), and a word_off with a spare word after some sequences (all N)."""
    from gpu_util import to_dev
    rng = np.random.default_rng(maxlen)
    n = 700
    lens = rng.integers(0, maxlen + 1, size=n)
    lens[rng.choice(n, 20, replace=False)] = 0
    pre, post = 13, 40
    body = rng.choice(np.frombuffer(b"ACGTNacgtn", np.uint8), size=int(lens.sum()))
    whole = np.concatenate([np.frombuffer(b"@" * pre, np.uint8), body,
                            np.frombuffer(b"%" * post, np.uint8)])
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    words = (lens + 31) // 32
    spare = (rng.random(n) < 0.1).astype(np.int64)
    wo = np.concatenate([[0], np.cumsum(words + spare)]).astype(np.int64)
    total = int(wo[-1])
    for bad in (False, True):
        src = whole.copy()
        if bad:
            pos = pre + rng.choice(len(body), 2, replace=False)
            src[pos] = np.frombuffer(b"#-", np.uint8)
        dev = to_dev(src)
        out = pf.Seqs.empty(total, "cuda:0", word_off=to_dev(wo))
        for t in (out.lo, out.hi, out.nmask):
            t.fill_(0x5A5A5A5A)
        pf.pf_pack(ctx, dev[1:], to_dev(off + pre - 1), to_dev(wo), out)
        if bad:
            with pytest.raises(pf.PFError):
                pf.pf_sync(ctx)
        else:
            pf.pf_sync(ctx)
        owo, lo, hi, nm, nbad = oracle.pack_batch(src[pre:pre + len(body)], off)
        assert nbad == (2 if bad else 0)
        got = [t.cpu().numpy()[:total].view(np.uint32) for t in (out.lo, out.hi, out.nmask)]
        for s_ in range(n):
            a, b = int(owo[s_]), int(owo[s_ + 1])
            g = int(wo[s_])
            for plane, want in zip(got, (lo, hi, nm)):
                assert np.array_equal(plane[g:g + b - a], want[a:b]), (maxlen, s_)
            if spare[s_]:
                assert got[0][g + b - a] == 0 and got[1][g + b - a] == 0
                assert got[2][g + b - a] == 0xFFFFFFFF


@pytest.mark.parametrize("maxlen", [70, 600, 5000])
def test_pack_starts_grouped_layout(pf, ctx, maxlen):
    """pf_pack_starts with pf_pack_layout_grouped's word starts writes every
    sequence's words (as the oracle packs them) where its start says, for
    empty, short and long sequences from an unaligned start, and reports
    bytes that are not bases inside a sequence."""
    from gpu_util import to_dev
    rng = np.random.default_rng(maxlen + 1)
    n = 900
    lens = rng.integers(0, maxlen + 1, size=n)
    lens[rng.choice(n, 25, replace=False)] = 0
    E = rng.integers(0, pf.PF_MAX_E + 1, size=n).astype(np.int16)
    pre = 7
    body = rng.choice(np.frombuffer(b"ACGTNacgtn", np.uint8), size=int(lens.sum()))
    whole = np.concatenate([np.frombuffer(b"@" * pre, np.uint8), body,
                            np.frombuffer(b"%" * 9, np.uint8)])
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    ws, total = pf.pf_pack_layout_grouped(off, E)
    for bad in (False, True):
        src = whole.copy()
        if bad:
            src[pre + rng.choice(len(body), 3, replace=False)] = np.frombuffer(b"#-*", np.uint8)
        out = pf.Seqs.empty(total, "cuda:0", word_off=to_dev(ws))
        for t in (out.lo, out.hi, out.nmask):
            t.fill_(0x5A5A5A5A)
        pf.pf_pack_starts(ctx, to_dev(src)[1:], to_dev(off + pre - 1), to_dev(ws), out)
        if bad:
            with pytest.raises(pf.PFError) as ei:
                pf.pf_sync(ctx)
            assert ei.value.status == 7
        else:
            pf.pf_sync(ctx)
        owo, lo, hi, nm, nbad = oracle.pack_batch(src[pre:pre + len(body)], off)
        assert nbad == (3 if bad else 0)
        got = [t.cpu().numpy()[:total].view(np.uint32) for t in (out.lo, out.hi, out.nmask)]
        for s_ in range(n):
            a, b = int(owo[s_]), int(owo[s_ + 1])
            g = int(ws[s_])
            for plane, want in zip(got, (lo, hi, nm)):
                assert np.array_equal(plane[g:g + b - a], want[a:b]), (maxlen, s_)
    # the planes are covered exactly: no word left at the fill value
    assert not np.any(got[2] == 0x5A5A5A5A)


@pytest.mark.parametrize("dec", [1, 2, 3])
def test_grouped_layout_whole_path_bit_exact(pf, ctx, case_data, dec):
    """The mixed batch packed in the layout grouped by threshold and length:
    filter and whole path equal the oracle, through the scheduler (every
    configuration the tuner finds on it) and the plain kernel."""
    from gpu_util import to_dev
    P, _, (oa, oc) = case_data["cfg3_mixed"]
    n = P.n
    pairs = pf.pack_pairs(ctx, to_dev(P.reads), to_dev(P.refs), byte_off=P.read_off,
                          group_E=P.E)
    lens, E, Emax = to_dev(P.lens.astype(np.int32)), to_dev(P.E), int(P.E.max())
    slots = 2 if dec == 3 else 1
    want_a = oa if dec == 3 else oa[[dec - 1]]
    want_c = oc if dec == 3 else oc[[dec - 1]]
    before = {e: pf.pf_tune_get(ctx, dec, e) for e in range(Emax + 1)}
    try:
        pf.pf_tune_batch(ctx, dec, pairs, lens, E, Emax, n=n, sample=4096, reps=1)
        for fn in (pf.pf_filter, pf.pf_filter_plain):
            acc = torch.zeros(slots * n, dtype=torch.uint8, device="cuda:0")
            cnt = torch.zeros(slots * n, dtype=torch.int16, device="cuda:0")
            fn(ctx, dec, pairs, lens, E, Emax, acc, cnt, n)
            pf.pf_sync(ctx)
            assert np.array_equal(cnt.cpu().numpy().reshape(slots, n), want_c)
            assert np.array_equal(acc.cpu().numpy().reshape(slots, n), want_a)
        dist = torch.full((n,), -5, dtype=torch.int32, device="cuda:0")
        acc = torch.zeros(slots * n, dtype=torch.uint8, device="cuda:0")
        cnt = torch.zeros(slots * n, dtype=torch.int16, device="cuda:0")
        pf.pf_filter_verify(ctx, dec, pairs, lens, E, Emax, acc, cnt, dist, n)
        pf.pf_sync(ctx)
        first = 0 if dec & 1 else 1  # the first selected decider's accepts are verified
        vb = oracle.verify_batch(P)
        want = np.where(oa[first] == 1, vb, P.E.astype(np.int32) + 1)
        assert np.array_equal(dist.cpu().numpy(), want)
        assert np.array_equal(acc.cpu().numpy().reshape(slots, n), want_a)
    finally:
        for e, (c, k) in before.items():
            pf.pf_tune_set(ctx, dec, e, c, k)


@pytest.mark.parametrize("length,n", [(1, 5000), (2, 3001), (32, 2047), (150, 4000),
                                      (4000, 300), (131072, 3), (131073, 2)])
def test_pack_fixed_across_tiles(pf, ctx, length, n):
    """The fixed layout over many 1023-word tiles with a ragged last one,
    sources starting at every offset within 32 bytes after bytes that are
    not bases, invalid bytes inside (packed as N, error raised), and the
    longest sequences each kernel form takes (4096 words and one more)."""
    from gpu_util import to_dev
    rng = np.random.default_rng(length * 7 + n)
    W = (length + 31) // 32
    for shift in (0, 1, 7, 16, 31) if length < 100000 else (0, 13):
        body = rng.choice(np.frombuffer(b"ACGTNacgtn", np.uint8), size=n * length)
        bad_at = rng.choice(n * length, size=3, replace=False) if shift % 2 else []
        body[bad_at] = np.frombuffer(b"X#-", np.uint8)[:len(bad_at)]
        whole = np.concatenate([np.frombuffer(b"@" * shift, np.uint8), body,
                                np.frombuffer(b"%" * 40, np.uint8)])
        dev = to_dev(whole)
        out = pf.Seqs.empty(n * W, "cuda:0", stride_words=W)
        pf.pf_pack_fixed(ctx, dev[shift:shift + n * length], n, length, out)
        if len(bad_at):
            with pytest.raises(pf.PFError) as ei:
                pf.pf_sync(ctx)
            assert ei.value.status == 7
        else:
            pf.pf_sync(ctx)
        _, lo, hi, nm, bad = oracle.pack_batch(body, np.arange(n + 1, dtype=np.int64) * length)
        assert bad == len(bad_at)
        for got, want in ((out.lo, lo), (out.hi, hi), (out.nmask, nm)):
            assert np.array_equal(got.cpu().numpy().view(np.uint32), want), (shift, length)


# ---- a2-a4 filter ---------------------------------------------------------

CASES = [
    ("cfg1_uniform_100bp_E5", synth.UNIFORM, 100, 5, 20, 20000),
    ("cfg2_150bp_E0", synth.SKEWED, 150, 0, 60, 12000),
    ("cfg2_150bp_E1", synth.SKEWED, 150, 1, 60, 12000),
    ("cfg2_150bp_E6", synth.SKEWED, 150, 6, 60, 20000),
    ("cfg2_150bp_E11", synth.SKEWED, 150, 11, 60, 12000),
    ("cfg2_150bp_E15", synth.SKEWED, 150, 15, 60, 12000),
    ("cfg3_mixed", synth.MIXED, 0, 0, 60, 30000),
    ("cfg4_250bp_E25", synth.SKEWED_ALL, 250, 25, 100, 6000),
]


@pytest.fixture(scope="module")
def case_data(ctx):
    from gpu_util import DevicePairs
    out = {}
    for name, kind, m, E, kmax, n in CASES:
        P = synth.generate(kind, 0x5EED0000 + 17 * E + m, n, m=m, E=E, kmax=kmax)
        fixed = m if kind != synth.MIXED else None
        D = DevicePairs(ctx, P, fixed=fixed)
        out[name] = (P, D, oracle_filter(P, 3))
    return out


@pytest.mark.parametrize("name", [c[0] for c in CASES])
@pytest.mark.parametrize("plain", [True, False])
def test_filter_both_deciders_bit_exact(ctx, case_data, name, plain):
    from gpu_util import filter_dev
    P, D, (oa, oc) = case_data[name]
    a, c = filter_dev(ctx, D, 3, plain=plain)
    assert np.array_equal(c, oc), np.argwhere(c != oc)[:5]
    assert np.array_equal(a, oa)


@pytest.mark.parametrize("name", ["cfg2_150bp_E6", "cfg3_mixed", "cfg4_250bp_E25"])
@pytest.mark.parametrize("dec", [1, 2])
@pytest.mark.parametrize("plain", [True, False])
def test_filter_single_decider(ctx, case_data, name, dec, plain):
    from gpu_util import filter_dev
    P, D, (oa, oc) = case_data[name]
    a, c = filter_dev(ctx, D, dec, plain=plain)
    slot = 0 if dec == 1 else 1
    assert np.array_equal(c[0], oc[slot])
    assert np.array_equal(a[0], oa[slot])


def test_filter_uniform_E_without_array(ctx, case_data):
    from gpu_util import filter_dev
    P, D, (oa, oc) = case_data["cfg2_150bp_E6"]
    for plain in (True, False):
        a, c = filter_dev(ctx, D, 3, plain=plain, per_pair_E=False)
        assert np.array_equal(c, oc) and np.array_equal(a, oa)


@pytest.mark.parametrize("name", ["cfg1_uniform_100bp_E5", "cfg2_150bp_E0", "cfg2_150bp_E1",
                                  "cfg2_150bp_E6", "cfg2_150bp_E11", "cfg2_150bp_E15"])
@pytest.mark.parametrize("dec", [1, 2, 3])
def test_plain_exact_threshold_kernel(pf, ctx, case_data, name, dec):
    # one compile-time threshold for every pair of the batch
    P, D, (oa, oc) = case_data[name]
    E = int(P.E[0])
    slots = 2 if dec == 3 else 1
    acc = torch.full((slots * D.n,), 0xEE, dtype=torch.uint8, device="cuda:0")
    cnt = torch.full((slots * D.n,), -7, dtype=torch.int16, device="cuda:0")
    pf.pf_filter_plain_exact(ctx, dec, D.pairs, D.lens, E, acc, cnt, D.n)
    pf.pf_sync(ctx)
    a = acc.cpu().numpy().reshape(slots, D.n)
    c = cnt.cpu().numpy().reshape(slots, D.n)
    want = [0, 1] if dec == 3 else [dec - 1]
    assert np.array_equal(c, oc[want]) and np.array_equal(a, oa[want])


def test_plain_exact_threshold_rejects_large_E(pf, ctx, case_data):
    P, D, _ = case_data["cfg2_150bp_E6"]
    acc = torch.zeros(D.n, dtype=torch.uint8, device="cuda:0")
    cnt = torch.zeros(D.n, dtype=torch.int16, device="cuda:0")
    with pytest.raises(pf.PFError) as ei:
        pf.pf_filter_plain_exact(ctx, 1, D.pairs, D.lens, 16, acc, cnt, D.n)
    assert ei.value.status == 1


def test_every_batched_configuration(pf, ctx):
    """Each (lanes per pair, slots per lane) kernel, each decider set, at the
    thresholds it serves, against the oracle."""
    from gpu_util import DevicePairs, filter_dev
    cfgs = pf.pf_kernel_configs()
    data = {}
    for E in (0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 20, 31):
        P = synth.generate(synth.SKEWED, 900 + E, 2500, m=150 if E < 20 else 250, E=E,
                           kmax=max(60, 3 * E))
        data[E] = (P, DevicePairs(ctx, P, fixed=int(P.lens[0])), oracle_filter(P, 3))
    for ci, (tpp, dpt, ecap, xe, words) in enumerate(cfgs):
        for E, (P, D, (oa, oc)) in data.items():
            if xe >= 0 and E != xe:
                continue
            if xe < 0 and (E > ecap or E < ecap // 2 - 1):
                continue
            for dec in (1, 2, 3):
                for chunk in (32, 1000):
                    pf.pf_tune_set(ctx, dec, E, ci, chunk)
                    a, c = filter_dev(ctx, D, dec, per_pair_E=False, E_max=E)
                    want_c = oc if dec == 3 else oc[[0 if dec == 1 else 1]]
                    want_a = oa if dec == 3 else oa[[0 if dec == 1 else 1]]
                    assert np.array_equal(c, want_c), (ci, tpp, dpt, E, dec, chunk)
                    assert np.array_equal(a, want_a), (ci, tpp, dpt, E, dec, chunk)


def test_ragged_mixed_E_with_several_configs(pf, ctx, case_data):
    """Per-pair E spread over three kernel configurations in one call."""
    from gpu_util import filter_dev
    P, D, (oa, oc) = case_data["cfg3_mixed"]
    cfgs = pf.pf_kernel_configs()
    pick = {e: next(i for i, c in enumerate(cfgs)
                    if c[3] < 0 and c[2] >= e and c[0] == (4 if e > 7 else 1))
            for e in range(0, 21)}
    for e, ci in pick.items():
        pf.pf_tune_set(ctx, 3, e, ci, 128)
    a, c = filter_dev(ctx, D, 3)
    assert np.array_equal(c, oc) and np.array_equal(a, oa)


def test_edge_cases(ctx):
    from gpu_util import DevicePairs, filter_dev
    P = explicit_pairs(edge_items())
    D = DevicePairs(ctx, P)
    oa, oc = oracle_filter(P, 3)
    for plain in (True, False):
        a, c = filter_dev(ctx, D, 3, plain=plain)
        assert np.array_equal(c, oc), np.argwhere(c != oc)[:5]
        assert np.array_equal(a, oa)
    # worked example of Fig. 8.1/8.2: three obstacles at E = 3
    i = [k for k, it in enumerate(edge_items()) if it[0] == "GGTGAGAGTTGT" and it[2] == 3][0]
    assert c[0][i] == 3 and a[0][i] == 1


def test_invalid_per_pair_threshold(pf, ctx):
    from gpu_util import DevicePairs, filter_dev
    P = explicit_pairs([("ACGT", "ACGT", 2), ("ACGT", "ACGA", 9), ("ACGT", "ACGT", 1)])
    D = DevicePairs(ctx, P)
    D.E_max = 3  # the second pair's E = 9 exceeds it
    for plain in (True, False):
        with pytest.raises(pf.PFError) as ei:
            filter_dev(ctx, D, 3, plain=plain)
        assert ei.value.status == 1
        pf.pf_sync(ctx)
    # the whole path marks the invalid pair (count -1, dist -1) and no other
    n = D.n
    acc = torch.zeros(2 * n, dtype=torch.uint8, device="cuda:0")
    cnt = torch.zeros(2 * n, dtype=torch.int16, device="cuda:0")
    dist = torch.full((n,), -5, dtype=torch.int32, device="cuda:0")
    pf.pf_filter_verify(ctx, 3, D.pairs, D.lens, D.E, D.E_max, acc, cnt, dist, n)
    with pytest.raises(pf.PFError):
        pf.pf_sync(ctx)
    pf.pf_sync(ctx)
    assert dist.cpu().tolist() == [0, -1, 0]
    assert cnt.cpu().tolist() == [0, -1, 0, 0, -1, 0]


def test_host_checks_reject_bad_arguments(pf, ctx, case_data):
    P, D, _ = case_data["cfg2_150bp_E6"]
    acc = torch.zeros(2 * D.n, dtype=torch.uint8, device="cuda:0")
    cnt = torch.zeros(2 * D.n, dtype=torch.int16, device="cuda:0")
    with pytest.raises(pf.PFError):
        pf.pf_filter(ctx, 3, D.pairs, D.lens, D.E, 32, acc, cnt, D.n)
    with pytest.raises(pf.PFError):
        pf.pf_filter(ctx, 4, D.pairs, D.lens, D.E, 6, acc, cnt, D.n)
    with pytest.raises(pf.PFError):
        pf.pf_tune_set(ctx, 1, 20, 0, 64)  # configuration 0 serves E <= 3
    exact6 = [i for i, c in enumerate(pf.pf_kernel_configs()) if c[3] == 6][0]
    with pytest.raises(pf.PFError):
        pf.pf_tune_set(ctx, 1, 5, exact6, 64)  # serves E == 6 only


# ---- a5 compaction ----------------------------------------------------------

@pytest.mark.parametrize("n", [0, 1, 15, 16, 17, 4095, 4096, 4097, 100003])
@pytest.mark.parametrize("offset", [0, 3])
def test_compact_matches_nonzero(pf, ctx, n, offset):
    rng = np.random.default_rng(n + offset)
    flags = (rng.random(n + offset) < 0.3).astype(np.uint8)
    flags[offset:] *= rng.integers(1, 255, size=n).astype(np.uint8)
    f = torch.from_numpy(flags).cuda()[offset:]
    idx = torch.full((max(n, 1),), -1, dtype=torch.int64, device="cuda:0")
    n_out = torch.full((1,), -1, dtype=torch.int64, device="cuda:0")
    pf.pf_compact(ctx, f, idx, n_out, n)
    pf.pf_sync(ctx)
    want = np.nonzero(flags[offset:])[0]
    k = int(n_out.item())
    assert k == len(want)
    assert np.array_equal(idx.cpu().numpy()[:k], want)


# ---- a6 verification -----------------------------------------------------------

@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_verify_all_pairs_bit_exact(ctx, case_data, name):
    from gpu_util import verify_dev
    P, D, _ = case_data[name]
    d = verify_dev(ctx, D)
    assert np.array_equal(d, oracle.verify_batch(P)), name


def test_verify_edge_cases_and_subset(ctx):
    from gpu_util import DevicePairs, verify_dev
    P = explicit_pairs(edge_items())
    D = DevicePairs(ctx, P)
    want = oracle.verify_batch(P)
    assert np.array_equal(verify_dev(ctx, D), want)
    sub = np.arange(0, P.n, 3)
    got = verify_dev(ctx, D, idx=sub)
    assert np.array_equal(got[sub], want[sub])
    rest = np.setdiff1d(np.arange(P.n), sub)
    assert np.all(got[rest] == -9)   # untouched
    # equals the unbanded distance wherever that is <= E
    wf = oracle.int_batch("wf", P)
    assert np.array_equal(np.minimum(wf, P.E.astype(np.int32) + 1), want)


def test_verify_exhaustive_tiny(ctx):
    """All pairs over {A,C,G,N}^4 at E = 0..4 (Levenshtein vs the banded
    bit-vector kernel)."""
    from conftest import all_pairs
    from gpu_util import DevicePairs, verify_dev
    reads, refs = all_pairs("ACGN", 4)
    for E in range(0, 5):
        P = ArrayPairs(reads, refs, E)
        sp = synth.Pairs(P.reads, P.refs, P.read_off, P.ref_off, P.lens, P.E)
        D = DevicePairs(ctx, sp, fixed=4)
        assert np.array_equal(verify_dev(ctx, D), oracle.verify_batch(sp))


# ---- a2-a6 whole path --------------------------------------------------------------

@pytest.mark.parametrize("name", ["cfg2_150bp_E6", "cfg3_mixed", "cfg4_250bp_E25"])
def test_filter_verify_path(pf, ctx, case_data, name):
    P, D, (oa, oc) = case_data[name]
    n = D.n
    acc = torch.zeros(2 * n, dtype=torch.uint8, device="cuda:0")
    cnt = torch.zeros(2 * n, dtype=torch.int16, device="cuda:0")
    dist = torch.full((n,), -5, dtype=torch.int32, device="cuda:0")
    pf.pf_filter_verify(ctx, 3, D.pairs, D.lens, D.E, D.E_max, acc, cnt, dist, n)
    pf.pf_sync(ctx)
    a = acc.cpu().numpy().reshape(2, n)
    assert np.array_equal(a, oa)
    d = dist.cpu().numpy()
    vb = oracle.verify_batch(P)
    E1 = P.E.astype(np.int32) + 1
    want = np.where(oa[0] == 1, vb, E1)
    assert np.array_equal(d, want)
    # zero false rejects: every pair within E survives with its exact distance
    assert np.all(oa[0][vb <= P.E] == 1)


@pytest.mark.parametrize("name", [c[0] for c in CASES])
@pytest.mark.parametrize("small", [0, 1 << 30])
@pytest.mark.parametrize("dec", [1, 3])
def test_resolved_pairs_equal_full_verification(pf, ctx, case_data, name, small, dec):
    """Accepted pairs whose SneakySnake count equals their Hamming distance
    skip verification; their distances (and every other output) equal those
    of verifying every accepted pair, and the oracle's, through the
    scheduler's kernels and through the plain kernel."""
    P, D, (oa, oc) = case_data[name]
    n = D.n
    vb = oracle.verify_batch(P)
    want = np.where(oa[0] == 1, vb, P.E.astype(np.int32) + 1)
    outs, counts = [], []
    pf.pf_set_small_batch(ctx, small)
    try:
        for resolve in (True, False):
            pf.pf_set_resolve_by_bounds(ctx, resolve)
            acc = torch.zeros(2 * n, dtype=torch.uint8, device="cuda:0")
            cnt = torch.zeros(2 * n, dtype=torch.int16, device="cuda:0")
            dist = torch.full((n,), -5, dtype=torch.int32, device="cuda:0")
            pf.pf_filter_verify(ctx, dec, D.pairs, D.lens, D.E, D.E_max, acc, cnt, dist, n)
            pf.pf_sync(ctx)
            outs.append((acc.cpu().numpy(), cnt.cpu().numpy(), dist.cpu().numpy()))
            counts.append(pf.pf_last_verified_count(ctx))
    finally:
        pf.pf_set_resolve_by_bounds(ctx, True)
        pf.pf_set_small_batch(ctx, 0)
    for x, y in zip(outs[0], outs[1]):
        assert np.array_equal(x, y)
    assert np.array_equal(outs[0][2], want)
    slots = 2 if dec == 3 else 1
    assert np.array_equal(outs[0][0][:slots * n].reshape(slots, n), oa[:slots])
    assert np.array_equal(outs[0][1][:slots * n].reshape(slots, n), oc[:slots])
    ham = oracle.int_batch("hamming", P)
    resolved = (oa[0] == 1) & (oc[0] == ham)
    assert np.array_equal(outs[0][2][resolved], ham[resolved])
    assert counts == [int(oa[0].sum() - resolved.sum()), int(oa[0].sum())]


def test_last_verified_count_after_an_empty_batch(pf, ctx, case_data):
    P, D, _ = case_data["cfg2_150bp_E6"]
    acc = torch.zeros(2 * D.n, dtype=torch.uint8, device="cuda:0")
    cnt = torch.zeros(2 * D.n, dtype=torch.int16, device="cuda:0")
    dist = torch.zeros(D.n, dtype=torch.int32, device="cuda:0")
    pf.pf_filter_verify(ctx, 3, D.pairs, D.lens, D.E, D.E_max, acc, cnt, dist, D.n)
    assert pf.pf_last_verified_count(ctx) > 0
    pf.pf_filter_verify(ctx, 3, D.pairs, D.lens, D.E, D.E_max, acc, cnt, dist, 0)
    assert pf.pf_last_verified_count(ctx) == 0


def test_two_phase_configs_on_ragged_pairs(pf, ctx, case_data):
    """The two-phase kernels on mixed lengths and thresholds: pairs longer
    than their shared arrays take the fused loop in the same warps."""
    from gpu_util import filter_dev
    P, D, (oa, oc) = case_data["cfg3_mixed"]
    cfgs = pf.pf_kernel_configs()
    for dec in (1, 3):
        for e in range(0, 21):
            two = [i for i, c in enumerate(cfgs) if c[3] == e and c[4] > 0]
            if two:
                pf.pf_tune_set(ctx, dec, e, two[0], 64)
            else:
                pf.pf_tune_set(ctx, dec, e, next(i for i, c in enumerate(cfgs)
                                                 if c[3] < 0 and c[2] >= e), 64)
        a, c = filter_dev(ctx, D, dec)
        want_c = oc if dec == 3 else oc[[0]]
        want_a = oa if dec == 3 else oa[[0]]
        assert np.array_equal(c, want_c) and np.array_equal(a, want_a)


def test_every_two_phase_config_bit_exact(pf, ctx):
    """Every two-phase configuration, forced for the thresholds it serves,
    on pairs that fit its shared arrays (150 bp; 250 bp for the forms with
    8-word arrays) and on pairs that overflow them (200 bp, 7 words; 300 bp:
    the fused loop in the same warps), both decider sets."""
    from gpu_util import DevicePairs, filter_dev
    cfgs = pf.pf_kernel_configs()
    data = {}
    for i, (tpp, dpt, ecap, xe, words) in enumerate(cfgs):
        if words <= 0:
            continue
        if xe >= 0:
            cases = [(xe, 150), (xe, 200)] + ([(xe, 250), (xe, 300)] if words >= 8 else [])
        else:
            cases = [(ecap, 250), (ecap, 300), (max(ecap // 2, 1), 250)]
        for E, m in cases:
            if (E, m) not in data:
                P = synth.generate(synth.SKEWED, 0x5EED0C00 + 97 * E + m, 1500, m=m, E=E,
                                   kmax=max(40, 3 * E))
                data[(E, m)] = (DevicePairs(ctx, P, fixed=m), oracle_filter(P, 3))
            D, (oa, oc) = data[(E, m)]
            for dec in (1, 3):
                before = pf.pf_tune_get(ctx, dec, E)
                pf.pf_tune_set(ctx, dec, E, i, 64)
                try:
                    a, c = filter_dev(ctx, D, dec)
                finally:
                    pf.pf_tune_set(ctx, dec, E, *before)
                want_c = oc if dec == 3 else oc[[0]]
                want_a = oa if dec == 3 else oa[[0]]
                assert np.array_equal(c, want_c), (i, m, E, dec)
                assert np.array_equal(a, want_a), (i, m, E, dec)


# ---- scheduler tuning ------------------------------------------------------------

def test_tuner_picks_a_valid_config_and_stays_exact(pf, ctx, case_data):
    """pf_tune keeps a configuration serving E (or -1, the plain kernel),
    and the filter stays exact with it; the previous choice is restored so
    that later tests keep exercising the scheduler's kernels."""
    from gpu_util import filter_dev
    P, D, (oa, oc) = case_data["cfg2_150bp_E6"]
    before = pf.pf_tune_get(ctx, 3, 6)
    try:
        cfg, chunk, ms = pf.pf_tune(ctx, 3, D.pairs, D.lens, 6, reps=1)
        assert ms > 0 and chunk in (64, 256, 1024)
        if cfg != -1:
            tpp, dpt, ecap, xe, words = pf.pf_kernel_configs()[cfg]
            assert xe == 6 or (xe < 0 and ecap >= 6)
        assert pf.pf_tune_get(ctx, 3, 6) == (cfg, chunk)
        a, c = filter_dev(ctx, D, 3)
        assert np.array_equal(c, oc) and np.array_equal(a, oa)
    finally:
        pf.pf_tune_set(ctx, 3, 6, *before)
    assert pf.pf_tune_get(ctx, 3, 6) == before


def test_tuner_can_choose_the_plain_kernel(pf, ctx, case_data):
    """At E = 0 (one diagonal, a memory-bound filter) the plain kernel is
    timed too; whatever wins, pf_filter routes uniform-E batches to it and
    stays exact, and pf_tune_set returns the threshold to the scheduler."""
    from gpu_util import filter_dev
    P, D, (oa, oc) = case_data["cfg2_150bp_E0"]
    before = pf.pf_tune_get(ctx, 1, 0)
    try:
        cfg, chunk, ms = pf.pf_tune(ctx, 1, D.pairs, D.lens, 0, reps=1)
        assert pf.pf_tune_get(ctx, 1, 0)[0] == cfg
        a, c = filter_dev(ctx, D, 1)
        assert np.array_equal(c, oc[[0]]) and np.array_equal(a, oa[[0]])
        pf.pf_tune_set(ctx, 1, 0, -1, 64)  # the plain kernel, by hand
        assert pf.pf_tune_get(ctx, 1, 0) == (-1, 64)
        a, c = filter_dev(ctx, D, 1)
        assert np.array_equal(c, oc[[0]]) and np.array_equal(a, oa[[0]])
        with pytest.raises(pf.PFError):
            pf.pf_tune_set(ctx, 1, 0, -2, 64)
    finally:
        pf.pf_tune_set(ctx, 1, 0, *before)
    assert pf.pf_tune_get(ctx, 1, 0) == before


def test_tune_batch_tunes_each_threshold_on_its_own_pairs(pf, ctx, case_data):
    from gpu_util import filter_dev
    P, D, (oa, oc) = case_data["cfg3_mixed"]
    cfgs = pf.pf_kernel_configs()
    pf.pf_tune_batch(ctx, 3, D.pairs, D.lens, D.E, D.E_max, reps=1)
    for e, count in zip(*np.unique(P.E, return_counts=True)):
        cfg, chunk = pf.pf_tune_get(ctx, 3, int(e))
        tpp, dpt, ecap, xe, words = cfgs[cfg]
        assert (xe == e or (xe < 0 and ecap >= e)) and chunk in (64, 256, 1024)
    a, c = filter_dev(ctx, D, 3)
    assert np.array_equal(c, oc) and np.array_equal(a, oa)
    with pytest.raises(pf.PFError):
        pf.pf_tune_batch(ctx, 3, D.pairs, D.lens, D.E, D.E_max, reps=0)


def test_small_batches_take_one_plain_launch(pf, case_data):
    """With the default small-batch rule, pf_filter and pf_filter_verify on
    small batches run the plain kernel; results are the same."""
    P, D, (oa, oc) = case_data["cfg3_mixed"]
    c = pf.pf_create(0)
    try:
        from gpu_util import filter_dev
        a, k = filter_dev(c, D, 3)
        assert np.array_equal(a, oa) and np.array_equal(k, oc)
        n = D.n
        acc = torch.zeros(2 * n, dtype=torch.uint8, device="cuda:0")
        cnt = torch.zeros(2 * n, dtype=torch.int16, device="cuda:0")
        dist = torch.full((n,), -5, dtype=torch.int32, device="cuda:0")
        pf.pf_filter_verify(c, 3, D.pairs, D.lens, D.E, D.E_max, acc, cnt, dist, n)
        pf.pf_sync(c)
        want = np.where(oa[0] == 1, oracle.verify_batch(P), P.E.astype(np.int32) + 1)
        assert np.array_equal(dist.cpu().numpy(), want)
        # one threshold for the whole batch (no per-pair E): the plain kernel
        # with the threshold fixed at compile time (E <= 15), else at run time
        for name in ("cfg1_uniform_100bp_E5", "cfg2_150bp_E0", "cfg2_150bp_E15",
                     "cfg4_250bp_E25"):
            P2, D2, (oa2, oc2) = case_data[name]
            for dec in (1, 2, 3):
                a2, k2 = filter_dev(c, D2, dec, per_pair_E=False)
                rows = [0, 1] if dec == 3 else [dec - 1]
                assert np.array_equal(k2, oc2[rows]) and np.array_equal(a2, oa2[rows]), (name, dec)
        with pytest.raises(pf.PFError):
            pf.pf_set_small_batch(c, -1)
    finally:
        pf.pf_destroy(c)
