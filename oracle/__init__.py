"""CPU oracle for the pre-alignment filtering hot path.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline
leg of the benchmark use it; the product path never does.  The arithmetic
lives in ``pf_oracle.c`` (plain loops over ASCII bytes, each function citing
the thesis passage it restates); this module compiles it with gcc and
marshals numpy arrays into it.

Parity status per function (what pins it, see tests/test_oracle_pins.py):
  sneakysnake     pinned (worked example of Ch. 8, brute-force graph search,
                  DP formulation, zero false rejects vs Wagner-Fischer)
  sneakysnake_dp  pinned (equals the graph search on all tiny inputs)
  gatekeeper      pinned only through the amend golden patterns, an
                  independent pattern-rewriting restatement, E=0 and
                  substitution-only properties
  wf / wf_banded  pinned (textbook recursion, closed forms, example of Ch. 8)
  pack            pinned (hand-written golden words)
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

SNEAKYSNAKE, GATEKEEPER = 1, 2


def build(force=False):
    """Compile ``pf_oracle.c`` into ``_build/liboracle.so`` with gcc."""
    src = os.path.join(_HERE, "pf_oracle.c")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)):
        return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-o", tmp, src])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        p, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint
        for name in ("or_sneakysnake", "or_sneakysnake_full", "or_sneakysnake_dp",
                     "or_gatekeeper", "or_wf_banded"):
            getattr(lib, name).argtypes = [ctypes.c_char_p, ctypes.c_char_p, i32, i32]
            getattr(lib, name).restype = i32
        lib.or_sneakysnake_trace.argtypes = [ctypes.c_char_p, ctypes.c_char_p, i32, i32, p, p, i32]
        lib.or_sneakysnake_trace.restype = i32
        lib.or_hamming.argtypes = [ctypes.c_char_p, ctypes.c_char_p, i32]
        lib.or_hamming.restype = i32
        lib.or_wf.argtypes = [ctypes.c_char_p, i32, ctypes.c_char_p, i32]
        lib.or_wf.restype = i32
        lib.or_amend.argtypes = [p, i32, p]
        lib.or_amend.restype = None
        lib.or_neighborhood_map.argtypes = [ctypes.c_char_p, ctypes.c_char_p, i32, i32, p]
        lib.or_neighborhood_map.restype = None
        lib.or_pack.argtypes = [ctypes.c_char_p, i32, p, p, p]
        lib.or_pack.restype = i32
        lib.or_filter_batch.argtypes = [p, p, p, p, p, p, i32, u32, p, p, i64, i32]
        lib.or_filter_batch.restype = None
        lib.or_int_batch.argtypes = [i32, p, p, p, p, p, p, i32, p, i64, i32, i32, i32]
        lib.or_sneakysnake_partitioned.argtypes = [ctypes.c_char_p, ctypes.c_char_p, i32, i32,
                                                   i32, i32]
        lib.or_shouji.argtypes = [ctypes.c_char_p, ctypes.c_char_p, i32, i32]
        lib.or_shouji_vector.argtypes = [ctypes.c_char_p, ctypes.c_char_p, i32, i32, p]
        lib.or_gatekeeper_shd.argtypes = [ctypes.c_char_p, ctypes.c_char_p, i32, i32, i32, i32]
        lib.or_int_batch.restype = None
        lib.or_pack_batch.argtypes = [p, p, i64, p, p, p, p]
        lib.or_pack_batch.restype = i64
        lib.or_work_counts.argtypes = [ctypes.c_char_p, ctypes.c_char_p, i32, i32, p]
        lib.or_work_counts.restype = None
        _lib = lib
    return _lib


def _b(s):
    return s.encode() if isinstance(s, str) else bytes(s)


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


# ---- single pairs -------------------------------------------------------

def sneakysnake(R, F, E):
    """Saturated SneakySnake obstacle count min(count, E+1)."""
    R, F = _b(R), _b(F)
    assert len(R) == len(F)
    return _load().or_sneakysnake(R, F, len(R), E)


def sneakysnake_full(R, F, E):
    R, F = _b(R), _b(F)
    return _load().or_sneakysnake_full(R, F, len(R), E)


def sneakysnake_dp(R, F, E):
    R, F = _b(R), _b(F)
    return _load().or_sneakysnake_dp(R, F, len(R), E)


def sneakysnake_partitioned(R, F, E, t, y):
    """Partitioned SneakySnake (sub-matrices of t columns, y replications
    each), min(count, E+1)."""
    R, F = _b(R), _b(F)
    assert len(R) == len(F) and t >= 1 and y >= 1
    return _load().or_sneakysnake_partitioned(R, F, len(R), E, t, y)


def shouji(R, F, E):
    """Shouji count min(ones of the Shouji bit-vector, E+1)."""
    R, F = _b(R), _b(F)
    assert len(R) == len(F)
    return _load().or_shouji(R, F, len(R), E)


def shouji_vector(R, F, E):
    """The Shouji bit-vector (uint8[m]) and its number of ones."""
    R, F = _b(R), _b(F)
    v = np.zeros(max(len(R), 1), dtype=np.uint8)
    ones = _load().or_shouji_vector(R, F, len(R), E, _ptr(v))
    return v[:len(R)], ones


def gatekeeper_shd(R, F, E, vacant_zero=True, streak=True):
    """GateKeeper with SHD's vacant-zero masks and/or streak counting."""
    R, F = _b(R), _b(F)
    assert len(R) == len(F)
    return _load().or_gatekeeper_shd(R, F, len(R), E, int(vacant_zero), int(streak))


def sneakysnake_trace(R, F, E):
    """Pipes of the unlimited walk: list of (start column, length)."""
    R, F = _b(R), _b(F)
    cap = len(R) + 1
    st = np.zeros(cap, dtype=np.int32)
    ln = np.zeros(cap, dtype=np.int32)
    k = _load().or_sneakysnake_trace(R, F, len(R), E, _ptr(st), _ptr(ln), cap)
    return [(int(st[i]), int(ln[i])) for i in range(k)]


def gatekeeper(R, F, E):
    R, F = _b(R), _b(F)
    return _load().or_gatekeeper(R, F, len(R), E)


def hamming(R, F):
    R, F = _b(R), _b(F)
    return _load().or_hamming(R, F, len(R))


def wf(a, b):
    a, b = _b(a), _b(b)
    return _load().or_wf(a, len(a), b, len(b))


def wf_banded(R, F, E):
    R, F = _b(R), _b(F)
    return _load().or_wf_banded(R, F, len(R), E)


def amend(bits):
    h = np.ascontiguousarray(np.asarray(bits, dtype=np.uint8))
    out = np.empty_like(h)
    _load().or_amend(_ptr(h), len(h), _ptr(out))
    return out


def neighborhood_map(R, F, E):
    R, F = _b(R), _b(F)
    out = np.empty((2 * E + 1, len(R)), dtype=np.uint8)
    _load().or_neighborhood_map(R, F, len(R), E, _ptr(out))
    return out


def pack(seq):
    """Pack one sequence; returns (lo, hi, nmask, bad) uint32 word arrays."""
    s = _b(seq)
    w = (len(s) + 31) // 32
    lo, hi, nm = (np.zeros(max(w, 1), dtype=np.uint32) for _ in range(3))
    bad = _load().or_pack(s, len(s), _ptr(lo), _ptr(hi), _ptr(nm))
    return lo[:w], hi[:w], nm[:w], bad


# ---- batches ------------------------------------------------------------

def _threads(t):
    return int(t or os.cpu_count() or 1)


def _E_arr(E):
    e = np.ascontiguousarray(np.asarray(E, dtype=np.int16).reshape(-1))
    return e, (1 if e.size > 1 else 0)


def filter_batch(pairs, deciders=SNEAKYSNAKE | GATEKEEPER, E=None, threads=None):
    """Oracle accept/count for a ``synth.Pairs`` batch.

    Returns (accept uint8[s, n], count int16[s, n]) with one slot per
    selected decider, SneakySnake first.
    """
    lib = _load()
    n = pairs.n
    e, stride = _E_arr(pairs.E if E is None else E)
    slots = bin(deciders & 3).count("1")
    acc = np.zeros((slots, n), dtype=np.uint8)
    cnt = np.zeros((slots, n), dtype=np.int16)
    lib.or_filter_batch(_ptr(pairs.reads), _ptr(pairs.read_off), _ptr(pairs.refs),
                        _ptr(pairs.ref_off), _ptr(np.ascontiguousarray(pairs.lens, np.int32)),
                        _ptr(e), stride, deciders, _ptr(acc), _ptr(cnt), n, _threads(threads))
    return acc, cnt


_KINDS = {"wf_banded": 1, "wf": 2, "ss_dp": 3, "ss_full": 4, "hamming": 5,
          "ss_partitioned": 6, "shouji": 7, "gk_shd": 8, "work": 9}


def int_batch(kind, pairs, E=None, threads=None, p0=0, p1=0):
    """Per-pair integers: 'wf_banded' (min(ED, E+1)), 'wf', 'ss_dp',
    'ss_full', 'hamming', 'ss_partitioned' (p0 = t, p1 = y), 'shouji',
    'gk_shd' (p0 = vacant zero, p1 = streak counting)."""
    lib = _load()
    n = pairs.n
    e, stride = _E_arr(pairs.E if E is None else E)
    out = np.zeros(n, dtype=np.int32)
    lib.or_int_batch(_KINDS[kind], _ptr(pairs.reads), _ptr(pairs.read_off), _ptr(pairs.refs),
                     _ptr(pairs.ref_off), _ptr(np.ascontiguousarray(pairs.lens, np.int32)),
                     _ptr(e), stride, _ptr(out), n, _threads(threads), int(p0), int(p1))
    return out


def work_counts(R, F, E):
    """(SneakySnake search words, SneakySnake columns, GateKeeper Hamming
    columns, GateKeeper AND columns) the method needs for one pair."""
    R, F = _b(R), _b(F)
    out = np.zeros(4, dtype=np.int32)
    _load().or_work_counts(R, F, len(R), E, _ptr(out))
    return tuple(int(x) for x in out)


def work_batch(pairs, E=None, threads=None):
    """work_counts for every pair of a batch: int32[n, 4]."""
    lib = _load()
    n = pairs.n
    e, stride = _E_arr(pairs.E if E is None else E)
    out = np.zeros((max(n, 1), 4), dtype=np.int32)
    lib.or_int_batch(9, _ptr(pairs.reads), _ptr(pairs.read_off), _ptr(pairs.refs),
                     _ptr(pairs.ref_off), _ptr(np.ascontiguousarray(pairs.lens, np.int32)),
                     _ptr(e), stride, _ptr(out), n, _threads(threads), 0, 0)
    return out[:n]


def verify_batch(pairs, E=None, threads=None):
    """dist = min(Levenshtein, E+1) per pair (Ukkonen band)."""
    return int_batch("wf_banded", pairs, E, threads)


def pack_batch(ascii_bytes, byte_off):
    """Pack sequences [byte_off[s], byte_off[s+1]); returns
    (word_off int64[nseq+1], lo, hi, nmask, bad)."""
    lib = _load()
    byte_off = np.ascontiguousarray(byte_off, dtype=np.int64)
    nseq = len(byte_off) - 1
    lens = np.diff(byte_off)
    words = (lens + 31) // 32
    word_off = np.zeros(nseq + 1, dtype=np.int64)
    np.cumsum(words, out=word_off[1:])
    total = int(word_off[-1])
    lo, hi, nm = (np.zeros(max(total, 1), dtype=np.uint32) for _ in range(3))
    a = np.ascontiguousarray(ascii_bytes, dtype=np.uint8)
    if a.size == 0:
        a = np.zeros(1, dtype=np.uint8)
    bad = lib.or_pack_batch(_ptr(a), _ptr(byte_off), nseq, _ptr(word_off),
                            _ptr(lo), _ptr(hi), _ptr(nm))
    return word_off, lo[:total], hi[:total], nm[:total], int(bad)
