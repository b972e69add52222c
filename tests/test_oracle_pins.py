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


@pytest.mark.parametrize("E", [0, 1, 2, 3, 5])
def test_equal_bounds_give_the_distance(exhaustive_5, E):
    """SneakySnake's count is a lower bound on the banded distance (Ch. 8
    Discussion: the snake underestimates the edits) and the Hamming distance
    an upper one (substitutions alone align the pair), so where the two agree
    at <= E that is the distance: the pairs the path resolves without
    verification."""
    reads, refs = exhaustive_5
    P = ArrayPairs(reads, refs, E)
    _, cnt = oracle.filter_batch(P)
    ham = oracle.int_batch("hamming", P)
    wfb = oracle.int_batch("wf_banded", P)
    ss = cnt[0].astype(np.int32)
    assert np.all(ss <= wfb) and np.all(wfb <= np.minimum(ham, E + 1))
    sel = (ss == ham) & (ham <= E)
    assert sel.any() and np.array_equal(wfb[sel], ham[sel])


def test_equal_bounds_give_the_distance_synthetic():
    P = synth.generate(synth.SKEWED, 0x5EED0B0D, 3000, m=150, E=6, kmax=20)
    _, cnt = oracle.filter_batch(P)
    ham = oracle.int_batch("hamming", P)
    wfb = oracle.verify_batch(P)
    sel = (cnt[0] == ham) & (ham <= 6)
    assert sel.sum() > 100
    assert np.array_equal(wfb[sel], ham[sel])


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


# ---- NEXT rows: partitioned SneakySnake (§8.5), Shouji (Ch. 6), SHD-style
# GateKeeper (Ch. 3) -------------------------------------------------------

def test_partitioned_lzc_example():
    kv, _ = read_golden("lzc_example.txt")
    row = kv["row_msb_first"][::-1]          # column 0 first
    t, y = int(kv["t"]), int(kv["y"])
    ref = "".join("A" for _ in row)
    read = "".join("C" if b == "1" else "A" for b in row)
    assert oracle.sneakysnake_partitioned(read, ref, 0, t, y) == int(kv["obstacles"])
    xs = [int(v) for v in kv["x"].split(",")]
    assert int(kv["obstacles"]) == min(y, t - sum(xs))
    # one replication passes the obstacle and stops: min(1, 8 - 4) = 1
    assert oracle.sneakysnake_partitioned(read, ref, 0, t, 1) == 1


@pytest.mark.parametrize("E", [0, 1, 2, 3])
def test_partitioned_special_cases_exhaustive(exhaustive_5, E):
    reads, refs = exhaustive_5
    P = ArrayPairs(reads, refs, E)
    ss = np.minimum(oracle.int_batch("ss_full", P), E + 1)
    wf = oracle.int_batch("wf", P)
    # one sub-matrix with enough replications is the whole problem
    assert np.array_equal(oracle.int_batch("ss_partitioned", P, p0=5, p1=5), ss)
    # t = 1: a column costs an obstacle exactly when all 2E+1 cells block it
    maps = [oracle.neighborhood_map(r.tobytes(), f.tobytes(), E) for r, f in
            zip(reads[::97], refs[::97])]
    blocked = np.array([int(np.all(M == 1, axis=0).sum()) for M in maps])
    sub = ArrayPairs(reads[::97], refs[::97], E)
    assert np.array_equal(oracle.int_batch("ss_partitioned", sub, p0=1, p1=1),
                          np.minimum(blocked, E + 1))
    prev = None
    for t in (1, 2, 3, 5):
        for y in (1, 2, 3, 6):
            c = oracle.int_batch("ss_partitioned", P, p0=t, p1=y)
            # restarting at sub-matrix borders and capping the replications
            # only removes obstacles: never above SneakySnake or the distance
            assert np.all(c <= ss) and np.all(c <= np.minimum(wf, E + 1))
            if prev is not None and prev[0] == t:
                assert np.all(c >= prev[1])  # more replications find more
            prev = (t, c)


def test_shouji_example_bit_vector():
    kv, _ = read_golden("shouji_example.txt")
    E = int(kv["E"])
    v, ones = oracle.shouji_vector(kv["pattern"], kv["text"], E)
    # zeros of the bit-vector are the common subsequences of Fig. 6.1
    runs, i = [], 0
    while i < len(v):
        if v[i] == 0:
            j = i
            while j < len(v) and v[j] == 0:
                j += 1
            runs.append(kv["text"][i:j])
            i = j
        else:
            i += 1
    assert runs == kv["subsequences"].split(",")
    assert ones == 3 and oracle.shouji(kv["pattern"], kv["text"], E) == 3


@pytest.mark.parametrize("E", [0, 1, 2, 3])
def test_shouji_zero_false_rejects_exhaustive(exhaustive_5, E):
    reads, refs = exhaustive_5
    P = ArrayPairs(reads, refs, E)
    sh = oracle.int_batch("shouji", P)
    wf = oracle.int_batch("wf", P)
    # Ch. 6 analysis and Ch. 9: no similar pair is filtered out.  The thesis
    # observed this on its datasets; it holds for every pair of length 5, but
    # it is not a theorem: at 150 bp, E = 6 about 2.7e-5 of the synthetic
    # pairs within E are rejected (GateKeeper: about 1.6e-4)
    assert np.all(sh <= np.minimum(wf, E + 1))
    if E == 0:
        exact = np.all(reads == refs, axis=1) & np.all(reads != ord("N"), axis=1)
        assert np.array_equal(sh == 0, exact)


def test_shouji_zero_false_rejects_synthetic():
    # small samples of the synthetic workloads (seeded): none of their pairs
    # within E is rejected
    for m, E, kind, km in ((100, 5, synth.UNIFORM, 20), (150, 6, synth.SKEWED, 60)):
        P = synth.generate(kind, 0x5EED0100 + m, 400, m=m, E=E, kmax=km)
        sh = oracle.int_batch("shouji", P)
        wf = oracle.int_batch("wf", P)
        assert np.all(sh <= np.minimum(wf, E + 1))


def test_shd_streak_example():
    kv, _ = read_golden("shd_streak_example.txt")
    E = int(kv["E"])
    assert oracle.gatekeeper_shd(kv["read"], kv["ref"], E, False, False) == int(kv["popcount_count"])
    assert oracle.gatekeeper_shd(kv["read"], kv["ref"], E, False, True) == int(kv["streak_count"])
    assert oracle.wf(kv["read"], kv["ref"]) == int(kv["edit_distance"])


@pytest.mark.parametrize("E", [0, 1, 2, 3])
def test_shd_switches_exhaustive(exhaustive_5, E):
    reads, refs = exhaustive_5
    P = ArrayPairs(reads, refs, E)
    _, cnt = oracle.filter_batch(P)
    gk = cnt[1].astype(np.int32)
    assert np.array_equal(oracle.int_batch("gk_shd", P, p0=0, p1=0), gk)
    vz = oracle.int_batch("gk_shd", P, p0=1, p1=0)
    st = oracle.int_batch("gk_shd", P, p0=0, p1=1)
    both = oracle.int_batch("gk_shd", P, p0=1, p1=1)
    # zero-filled vacant cells and streak counting only lower the count
    assert np.all(vz <= gk) and np.all(st <= gk) and np.all(both <= np.minimum(vz, st))
    # the Hamming fast path is shared: within E, every variant reports it
    ham = oracle.int_batch("hamming", P)
    sel = ham <= E
    assert np.array_equal(both[sel], ham[sel])


def test_shouji_window_width_example():
    kv, _ = read_golden("shouji_width_example.txt")
    v, ones = oracle.shouji_vector(kv["read"], kv["ref"], int(kv["E"]))
    assert "".join(str(int(b)) for b in v) == kv["bit_vector"]
    assert ones == int(kv["count"])
    assert oracle.wf(kv["read"], kv["ref"]) == int(kv["edit_distance"])


def test_shd_vacant_zero_closed_form():
    # reads that mismatch everywhere: every mask is all ones except its
    # vacant cells, which SHD's shifts fill with 0, so the first E and the
    # last E columns of the final bit-vector are 0 (Ch. 3, Leading and
    # Trailing Zeros) and the count is m - 2E; with vacant cells 1 it is m
    for m, E in ((8, 3), (10, 3), (12, 4)):
        read, ref = "A" * m, "C" * m
        assert oracle.gatekeeper_shd(read, ref, E, True, False) == min(m - 2 * E, E + 1)
        assert oracle.gatekeeper_shd(read, ref, E, False, False) == E + 1
        assert oracle.gatekeeper(read, ref, E) == E + 1
        # one streak of m - 2E ones
        assert oracle.gatekeeper_shd(read, ref, E, True, True) == min((m - 2 * E + 2) // 3, E + 1)


# ---- false rejects of GateKeeper and Shouji: hand-traced minimal pairs -------

def _bits(s):
    return [int(c) for c in s]


def test_gatekeeper_false_reject_example():
    kv, _ = read_golden("gatekeeper_false_reject.txt")
    read, ref, E = kv["read"], kv["ref"], int(kv["E"])
    # the map's rows (d = -E..E) and their amends, as traced by hand
    mp = oracle.neighborhood_map(read, ref, E)
    for d in range(-E, E + 1):
        assert mp[d + E].tolist() == _bits(kv["mask_d%d" % d]), d
    assert mp[E].tolist() == _bits(kv["hamming_mask"])
    anded = np.ones(len(read), dtype=np.uint8)
    for d in range(-E, E + 1):
        anded &= oracle.amend(mp[d + E])
    assert anded.tolist() == _bits(kv["and_of_amended"])
    assert oracle.gatekeeper(read, ref, E) == int(kv["count"])
    assert oracle.wf(read, ref) == int(kv["edit_distance"]) <= E
    # SneakySnake accepts it (its count never exceeds the edit distance)
    assert oracle.sneakysnake(read, ref, E) <= int(kv["edit_distance"])


def test_shouji_false_reject_example():
    kv, _ = read_golden("shouji_false_reject.txt")
    read, ref, E = kv["read"], kv["ref"], int(kv["E"])
    mp = oracle.neighborhood_map(read, ref, E)
    for d in range(-E, E + 1):
        assert mp[d + E].tolist() == _bits(kv["map_d%d" % d]), d
    v, ones = oracle.shouji_vector(read, ref, E)
    assert v.tolist() == _bits(kv["bit_vector"])
    assert ones == int(kv["count"]) and oracle.shouji(read, ref, E) == int(kv["count"])
    assert oracle.wf(read, ref) == int(kv["edit_distance"]) <= E
    assert oracle.sneakysnake(read, ref, E) <= int(kv["edit_distance"])


@pytest.mark.parametrize("kind,L,E_first", [("gatekeeper", 4, 2), ("shouji", 6, 2)])
def test_false_reject_examples_are_the_shortest(kind, L, E_first):
    # every shorter pair over {A,C,G,T}, at every E, is accepted whenever its
    # edit distance is within E, and at length L none is rejected below E_first
    for length in range(1, L + 1):
        for E in range(0, length if length < L else E_first):
            reads, refs = all_pairs("ACGT", length)
            P = ArrayPairs(reads, refs, E)
            ed = oracle.int_batch("wf_banded", P)
            if kind == "gatekeeper":
                c = oracle.filter_batch(P, deciders=2)[1][0]
            else:
                c = oracle.int_batch("shouji", P)
            assert not np.any((ed <= E) & (c > E)), (length, E)


# ---- work counts (needed-work roofline; they change no result) --------------

def test_work_counts_worked_example(golden):
    kv, _ = golden("sneakysnake_example.txt")
    F, R, E = kv["reference"], kv["read"], int(kv["E"])
    # Counted by hand on the map of Fig. 8.1/8.2 (12 columns, one word):
    # three deepest-pipe searches (from columns 0, 5 and 10; each ends at an
    # obstacle: columns 4, 9 and 11), so the walk reads all 12 columns.
    # The d = 0 row mismatches at columns 4..11: the Hamming count passes
    # E = 3 at column 7 (8 columns read).  GateKeeper accepts (count 2), so
    # its AND needs every column.
    assert oracle.work_counts(R, F, E) == (3, 12, 8, 12)
    assert oracle.sneakysnake(R, F, E) == 3 and oracle.gatekeeper(R, F, E) == 2


def test_work_counts_are_the_walks_searches():
    # one-word pairs: the walk searches once per obstacle, plus once to leave
    # the grid unless an obstacle step already did; a rejected pair stops at
    # its (E+1)-th obstacle.  Identical pairs need one search and, with the
    # Hamming check accepting, no amended AND.
    rng = np.random.default_rng(11)
    for _ in range(400):
        m = int(rng.integers(1, 33))
        E = int(rng.integers(0, 6))
        R = bytes(int(x) for x in rng.choice(list(b"ACGT"), m))
        F = bytearray(R)
        for _ in range(int(rng.integers(0, 8))):
            F[int(rng.integers(0, m))] = int(rng.choice(list(b"ACGT")))
        F = bytes(F)
        words, cols, ham_cols, and_cols = oracle.work_counts(R, F, E)
        k = oracle.sneakysnake(R, F, E)
        if k > E:
            assert words == E + 1
        else:
            assert words in (k, k + 1) and cols == m
        h = oracle.hamming(R, F)
        assert ham_cols == (m if h <= E else
                            1 + next(i for i in range(m)
                                     if sum(R[j] != F[j] for j in range(i + 1)) > E))
        assert (and_cols == 0) == (h <= E)
    assert oracle.work_counts("ACGTACGT", "ACGTACGT", 2) == (1, 8, 8, 0)
