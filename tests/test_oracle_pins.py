"""Pins of the CPU oracle against what the thesis and the mathematics fix.

Every check here compares the oracle with something other than itself: a
value printed in the thesis (fixtures under tests/golden/), a textbook
definition restated independently in Python (recursive Levenshtein, a
shortest-path search over the snake's grid graph, pattern rewriting for
the amend rule), closed forms, or properties the thesis states (zero false
rejects of SneakySnake, E = 0 is exact matching, substitution-only pairs
are bounded by the Hamming distance).
"""
import functools
import itertools
import random
from collections import deque

import numpy as np
import pytest

import oracle
import synth
from conftest import ArrayPairs, all_pairs, read_golden


# ---- independent restatements used as pins ---------------------------------

def _match(x, y):
    return x == y and x.upper() != "N"


def lev_recursive(a, b):
    """Textbook recursive definition of the Levenshtein distance."""
    a, b = a.upper(), b.upper()

    @functools.lru_cache(maxsize=None)
    def D(i, j):
        if i == 0:
            return j
        if j == 0:
            return i
        return min(D(i - 1, j) + 1, D(i, j - 1) + 1,
                   D(i - 1, j - 1) + (0 if _match(a[i - 1], b[j - 1]) else 1))

    return D(len(a), len(b))


def snake_graph_min(read, ref, E):
    """Sneaky Snake Problem (§8.2) as a shortest path: states are grid cells
    (column i of the reference, diagonal d); a free cell passes to the next
    column on the same diagonal at no cost, an obstacle (mismatch or cell
    outside the read) passes to the next column on any diagonal at cost 1.
    Returns the fewest obstacles of any path from column 0 to column m."""
    m = len(ref)
    if m == 0:
        return 0
    INF = 1 << 30
    dist = {}
    dq = deque()
    for d in range(-E, E + 1):
        dist[(0, d)] = 0
        dq.append((0, d))
    best = INF
    while dq:
        i, d = dq.popleft()
        c = dist[(i, d)]
        if i == m:
            best = min(best, c)
            continue
        j = i + d
        free = 0 <= j < m and _match(ref[i], read[j])
        if free:
            nxt = [((i + 1, d), c)]
        else:
            nxt = [((i + 1, e), c + 1) for e in range(-E, E + 1)]
        for s, nc in nxt:
            if nc < dist.get(s, INF):
                dist[s] = nc
                if nc == c:
                    dq.appendleft(s)
                else:
                    dq.append(s)
    return best


def gatekeeper_by_patterns(read, ref, E):
    """GateKeeper (§5.2.1-§5.2.3) with the amend step written as string
    rewriting of every "101" and "1001" occurrence of the original mask."""
    m = len(ref)
    if m == 0:
        return 0
    h = sum(0 if _match(ref[i], read[i]) else 1 for i in range(m))
    if h <= E:
        return h
    final = ["1"] * m
    for d in range(-E, E + 1):
        mask = "".join("0" if (0 <= i + d < m and _match(ref[i], read[i + d])) else "1"
                       for i in range(m))
        out = list(mask)
        for p in range(m):
            if mask.startswith("101", p):
                out[p + 1] = "1"
            if mask.startswith("1001", p):
                out[p + 1] = "1"
                out[p + 2] = "1"
        final = ["1" if (f == "1" and o == "1") else "0" for f, o in zip(final, out)]
    return min(final.count("1"), E + 1)


# ---- golden values printed in the thesis -------------------------------------

def test_sneakysnake_worked_example():
    kv, _ = read_golden("sneakysnake_example.txt")
    ref, read, E = kv["reference"], kv["read"], int(kv["E"])
    assert oracle.sneakysnake(read, ref, E) == int(kv["obstacles"])
    assert oracle.sneakysnake_dp(read, ref, E) == int(kv["obstacles"])
    pipes = [ref[s:s + n] for s, n in oracle.sneakysnake_trace(read, ref, E)]
    assert pipes == kv["pipes"].split(",")
    # the example pair is accepted at E = 3 although its Levenshtein distance
    # is 4: a false accept, which the method allows (never a false reject)
    assert lev_recursive(read, ref) == 4 == oracle.wf(read, ref)


def test_shouji_example_subsequences():
    kv, _ = read_golden("shouji_example.txt")
    text, pattern, E = kv["text"], kv["pattern"], int(kv["E"])
    pipes = [text[s:s + n] for s, n in oracle.sneakysnake_trace(pattern, text, E)]
    assert pipes == kv["subsequences"].split(",")


def test_nonadditive_example():
    kv, _ = read_golden("nonadditive.txt")
    assert oracle.wf(kv["a"], kv["b"]) == int(kv["edit_distance"])
    assert oracle.hamming(kv["a"], kv["b"]) == int(kv["per_character_edits"])
    assert oracle.wf_banded(kv["a"], kv["b"], 4) == int(kv["edit_distance"])


def test_amend_golden_patterns():
    _, rows = read_golden("amend_patterns.txt")
    assert len(rows) >= 10
    for row in rows:
        src, dst = [s.strip() for s in row.split("->")]
        got = "".join(str(int(b)) for b in oracle.amend([int(c) for c in src]))
        assert got == dst, (src, got, dst)


def test_pack_golden_words():
    _, rows = read_golden("pack_words.txt")
    for row in rows:
        seq, lo, hi, nm = [s.strip() for s in row.split(":")]
        glo, ghi, gnm, bad = oracle.pack(seq)
        assert bad == 0
        for got, want in ((glo, lo), (ghi, hi), (gnm, nm)):
            assert [int(x) for x in got] == [int(w, 16) for w in want.split(",")], row


def test_pack_rejects_other_bytes():
    lo, hi, nm, bad = oracle.pack("ACXT")
    assert bad == 1
    assert nm[0] & 0b0100  # the bad byte packs as N


# ---- brute force against independent restatements -----------------------------

@pytest.mark.parametrize("L", [1, 2, 3])
def test_sneakysnake_equals_graph_search_exhaustive(L):
    seqs = ["".join(p) for p in itertools.product("ACGN", repeat=L)]
    for read in seqs:
        for ref in seqs:
            for E in range(0, L + 1):
                want = min(snake_graph_min(read, ref, E), E + 1)
                assert oracle.sneakysnake(read, ref, E) == want, (read, ref, E)
                assert oracle.sneakysnake_dp(read, ref, E) == want, (read, ref, E)


def test_sneakysnake_equals_graph_search_random():
    rng = random.Random(1234)
    for _ in range(600):
        L = rng.randint(4, 14)
        ref = "".join(rng.choice("ACGT") for _ in range(L))
        read = list(ref)
        for _ in range(rng.randint(0, 5)):
            op = rng.random()
            pos = rng.randrange(len(read)) if read else 0
            if op < 0.5 and read:
                read[pos] = rng.choice("ACGTN")
            elif op < 0.75:
                read.insert(pos, rng.choice("ACGT"))
            elif read:
                del read[pos]
        read = ("".join(read) + ref)[:L]
        E = rng.randint(0, 4)
        want = min(snake_graph_min(read, ref, E), E + 1)
        assert oracle.sneakysnake(read, ref, E) == want, (read, ref, E)
        assert oracle.sneakysnake_dp(read, ref, E) == want, (read, ref, E)


@pytest.mark.parametrize("L", [1, 2, 3])
def test_levenshtein_equals_recursion_exhaustive(L):
    seqs = ["".join(p) for p in itertools.product("ACGN", repeat=L)]
    for a in seqs:
        for b in seqs:
            d = lev_recursive(a, b)
            assert oracle.wf(a, b) == d
            for E in range(0, L + 1):
                assert oracle.wf_banded(a, b, E) == min(d, E + 1), (a, b, E)


def test_levenshtein_unequal_lengths_and_closed_forms():
    rng = random.Random(7)
    for _ in range(300):
        a = "".join(rng.choice("ACGTN") for _ in range(rng.randint(0, 9)))
        b = "".join(rng.choice("ACGTN") for _ in range(rng.randint(0, 9)))
        assert oracle.wf(a, b) == lev_recursive(a, b)
    assert oracle.wf("ACGTACGT", "") == 8
    assert oracle.wf("", "ACG") == 3
    assert oracle.wf("ACGTACGT", "ACGTACGT") == 0
    assert oracle.wf("AAAA", "CCCC") == 4
    assert oracle.wf("N", "N") == 1          # an N never matches
    assert oracle.wf("ACGT", "CGTA") == 2    # rotation by one: delete + insert


@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_gatekeeper_equals_pattern_rewriting(L):
    rng = random.Random(99 + L)
    seqs = ["".join(p) for p in itertools.product("ACGN", repeat=L)]
    cases = [(a, b) for a in seqs for b in seqs]
    if len(cases) > 4000:
        cases = rng.sample(cases, 4000)
    for read, ref in cases:
        for E in range(0, L + 1):
            assert oracle.gatekeeper(read, ref, E) == gatekeeper_by_patterns(read, ref, E)


def test_gatekeeper_pattern_rewriting_random_long():
    rng = random.Random(5)
    for _ in range(300):
        L = rng.randint(5, 40)
        ref = "".join(rng.choice("ACGT") for _ in range(L))
        read = list(ref)
        for _ in range(rng.randint(0, 8)):
            pos = rng.randrange(L)
            if rng.random() < 0.5:
                read[pos] = rng.choice("ACGTN")
            else:
                read.insert(pos, rng.choice("ACGT"))
        read = "".join(read)[:L]
        E = rng.randint(0, 6)
        assert oracle.gatekeeper(read, ref, E) == gatekeeper_by_patterns(read, ref, E)


def test_neighborhood_map_definition():
    ref, read, E = "GGTGGAGAGATC", "GGTGAGAGTTGT", 3
    M = oracle.neighborhood_map(read, ref, E)
    for d in range(-E, E + 1):
        for i in range(len(ref)):
            j = i + d
            want = 0 if (0 <= j < len(read) and read[j] == ref[i]) else 1
            assert M[d + E, i] == want


# ---- properties the thesis states, exhaustive at C speed ----------------------

@pytest.fixture(scope="module")
def exhaustive_5():
    reads, refs = all_pairs("ACGN", 5)
    return reads, refs


@pytest.mark.parametrize("E", [0, 1, 2, 3, 5])
def test_properties_exhaustive_len5(exhaustive_5, E):
    reads, refs = exhaustive_5
    P = ArrayPairs(reads, refs, E)
    acc, cnt = oracle.filter_batch(P)
    wf = oracle.int_batch("wf", P)
    wfb = oracle.int_batch("wf_banded", P)
    dp = oracle.int_batch("ss_dp", P)
    ss = cnt[0].astype(np.int32)
    # SneakySnake never exceeds the edit distance: zero false rejects (Ch. 8
    # Discussion; Ch. 9 false reject rate)
    assert np.all(ss <= np.minimum(wf, E + 1))
    assert np.all(acc[0][wf <= E] == 1)
    # greedy walk equals the minimum-obstacle formulation of the problem
    assert np.array_equal(ss, dp)
    # Ukkonen's band with saturation equals the full distance, saturated
    assert np.array_equal(wfb, np.minimum(wf, E + 1))
    # accept flags follow the counts (count <= E)
    assert np.array_equal(acc[0], (cnt[0] <= E).astype(np.uint8))
    assert np.array_equal(acc[1], (cnt[1] <= E).astype(np.uint8))
    if E == 0:
        exact = np.all(reads == refs, axis=1) & np.all(reads != ord("N"), axis=1)
        assert np.array_equal(acc[0].astype(bool), exact)
        assert np.array_equal(acc[1].astype(bool), exact)


def test_accept_monotone_in_E(exhaustive_5):
    reads, refs = exhaustive_5
    prev_full = None
    prev_acc = None
    for E in range(0, 6):
        P = ArrayPairs(reads, refs, E)
        full = oracle.int_batch("ss_full", P)
        acc, _ = oracle.filter_batch(P, deciders=oracle.SNEAKYSNAKE)
        if prev_full is not None:
            assert np.all(full <= prev_full)          # more diagonals never hurt
            assert np.all(acc[0] >= prev_acc)         # accept at E => accept at E+1
        prev_full, prev_acc = full, acc[0]


def test_substitution_only_bounded_by_hamming():
    rng = np.random.default_rng(11)
    n, L = 4000, 60
    refs = rng.choice(np.frombuffer(b"ACGT", np.uint8), size=(n, L))
    reads = refs.copy()
    for p in range(n):
        k = rng.integers(0, 12)
        pos = rng.choice(L, size=k, replace=False)
        reads[p, pos] = rng.choice(np.frombuffer(b"ACGTN", np.uint8), size=k)
    for E in (0, 3, 6, 10):
        P = ArrayPairs(reads, refs, E)
        acc, cnt = oracle.filter_batch(P)
        ham = oracle.int_batch("hamming", P)
        assert np.all(cnt[0] <= np.minimum(ham, E + 1))
        # GateKeeper's fast path (§5.2.1): Hamming <= E accepts with count = Hamming
        sel = ham <= E
        assert np.all(acc[1][sel] == 1)
        assert np.array_equal(cnt[1][sel], ham[sel])


@pytest.mark.parametrize("m,E,kind", [(100, 5, synth.UNIFORM), (150, 6, synth.SKEWED),
                                      (250, 25, synth.SKEWED_ALL)])
def test_zero_false_rejects_on_synthetic_reads(m, E, kind):
    P = synth.generate(kind, 0x5EED0000 + m, 400, m=m, E=E, kmax=60 if kind != synth.SKEWED_ALL else 100)
    acc, cnt = oracle.filter_batch(P)
    wf = oracle.int_batch("wf", P)
    assert np.all(acc[0][wf <= E] == 1)
    assert np.all(cnt[0] <= np.minimum(wf, E + 1))
    assert np.array_equal(oracle.verify_batch(P), np.minimum(wf, E + 1))
    assert np.array_equal(cnt[0], oracle.int_batch("ss_dp", P))
