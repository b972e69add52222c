"""Seeded synthetic read/reference pairs (input generation only).

The C source (``synth.c``) documents the recipes.  Every pair owns a
SplitMix64 stream keyed by (seed, pair index), so a slice of a data set is
regenerated identically on its own.  Outputs are ASCII bytes plus int64 byte
offsets, int32 lengths and int16 thresholds; both the CUDA path and the
oracle consume them.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libsynth.so")
_lib = None

UNIFORM, SKEWED, MIXED, SKEWED_ALL, SERVE = 0, 1, 2, 3, 4


def build(force=False):
    """Compile ``synth.c`` into ``_build/libsynth.so`` with gcc."""
    src = os.path.join(_HERE, "synth.c")
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
        i64, i32, u64, p = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p
        lib.synth_shapes.argtypes = [i32, u64, i32, i32, i64, i64, p, p]
        lib.synth_shapes.restype = None
        lib.synth_fill.argtypes = [i32, u64, i32, i32, i32, i64, i64, p, p, p, p, i32]
        lib.synth_fill.restype = i32
        lib.synth_stream.argtypes = [u64, i64, i64, p]
        lib.synth_stream.restype = None
        _lib = lib
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def stream(seed, pair, count):
    """First ``count`` raw 64-bit draws of the stream of ``pair``."""
    out = np.empty(count, dtype=np.uint64)
    _load().synth_stream(seed, pair, count, _ptr(out))
    return out


def shapes(kind, seed, n, m=0, E=0, p0=0):
    """Per-pair (lens int32[n], E int16[n]) of pairs [p0, p0+n)."""
    lens = np.empty(n, dtype=np.int32)
    es = np.empty(n, dtype=np.int16)
    _load().synth_shapes(kind, seed, m, E, p0, p0 + n, _ptr(lens), _ptr(es))
    return lens, es


class Pairs:
    """A generated batch: ASCII reads and refs with per-pair offsets."""

    def __init__(self, reads, refs, read_off, ref_off, lens, E):
        self.reads, self.refs = reads, refs
        self.read_off, self.ref_off = read_off, ref_off
        self.lens, self.E = lens, E

    @property
    def n(self):
        return len(self.lens)

    def read(self, p):
        return bytes(self.reads[self.read_off[p]:self.read_off[p] + self.lens[p]])

    def ref(self, p):
        return bytes(self.refs[self.ref_off[p]:self.ref_off[p] + self.lens[p]])


def generate(kind, seed, n, m=0, E=0, kmax=60, p0=0, threads=None):
    """Generate pairs [p0, p0+n) of recipe ``kind``.

    Offsets are exclusive prefix sums of the lengths (n+1 entries), reads
    and refs live in separate byte arrays with identical offsets.
    """
    lib = _load()
    lens, es = shapes(kind, seed, n, m, E, p0)
    off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    total = int(off[-1])
    reads = np.empty(max(total, 1), dtype=np.uint8)
    refs = np.empty(max(total, 1), dtype=np.uint8)
    threads = threads or os.cpu_count() or 1
    rc = lib.synth_fill(kind, seed, m, E, kmax, p0, p0 + n, _ptr(off), _ptr(off),
                        _ptr(reads), _ptr(refs), int(threads))
    if rc != 0:
        raise ValueError("synth_fill: length out of range")
    return Pairs(reads[:total], refs[:total], off, off, lens, es)
