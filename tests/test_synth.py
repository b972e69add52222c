"""The seeded input generator: determinism, slicing, recipe shapes."""
import numpy as np

import oracle
import synth


def test_stream_matches_published_splitmix64():
    # SplitMix64 (Steele, Lea, Flood 2014) restated: state += golden gamma,
    # then the two xor-shift-multiply rounds of the finaliser.
    def mix(z):
        M = (1 << 64) - 1
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        return z ^ (z >> 31)

    M = (1 << 64) - 1
    seed, pair = 42, 17
    s = mix((seed + 0x632BE59BD9B4E019) & M) ^ mix((pair * 0xD1B54A32D192ED03 + 1) & M)
    want = []
    for _ in range(5):
        s = (s + 0x9E3779B97F4A7C15) & M
        want.append(mix(s))
    assert [int(x) for x in synth.stream(seed, pair, 5)] == want


def test_deterministic_and_sliceable():
    a = synth.generate(synth.MIXED, 99, 300)
    b = synth.generate(synth.MIXED, 99, 100, p0=150)
    c = synth.generate(synth.MIXED, 99, 300, threads=1)
    assert np.array_equal(a.reads, c.reads) and np.array_equal(a.refs, c.refs)
    for p in range(100):
        assert a.read(150 + p) == b.read(p)
        assert a.ref(150 + p) == b.ref(p)
        assert a.E[150 + p] == b.E[p]


def test_mixed_recipe_shapes():
    lens, E = synth.shapes(synth.MIXED, 7, 20000)
    allowed = {100: {2, 5, 8}, 150: {3, 8, 12}, 250: {5, 13, 20}}
    for m in (100, 150, 250):
        assert set(np.unique(E[lens == m]).tolist()) == allowed[m]
    frac = np.array([(lens == m).mean() for m in (100, 150, 250)])
    assert np.allclose(frac, [0.4, 0.4, 0.2], atol=0.02)


def test_serve_recipe_shapes():
    lens, E = synth.shapes(synth.SERVE, 8, 20000)
    assert set(np.unique(lens).tolist()) == {100, 150, 250}
    assert E.min() >= 0 and np.all(E <= np.round(lens * 0.10 + 0.5))


def test_skewed_base_composition():
    P = synth.generate(synth.SKEWED, 3, 2000, m=150, E=6)
    refs = P.refs
    gc = np.isin(refs, np.frombuffer(b"GC", np.uint8)).mean()
    nfrac = (refs == ord("N")).mean()
    assert abs(gc - 0.41) < 0.01
    assert 0.0003 < nfrac < 0.002
    assert set(np.unique(P.reads).tolist()) <= set(b"ACGTN")


def test_skewed_mix_mostly_incorrect():
    # 20% of pairs draw at most E edits, 80% draw more: the fraction within
    # edit distance E must sit below 20% plus a little (edits can cancel).
    E = 6
    P = synth.generate(synth.SKEWED, 4, 3000, m=150, E=E)
    wf = oracle.int_batch("wf", P)
    frac = (wf <= E).mean()
    assert 0.15 < frac < 0.26


def test_uniform_recipe_lengths_exact():
    P = synth.generate(synth.UNIFORM, 5, 500, m=100, E=5, kmax=20)
    assert np.all(P.lens == 100)
    assert len(P.reads) == 500 * 100
    assert set(np.unique(P.reads).tolist()) <= set(b"ACGT")
