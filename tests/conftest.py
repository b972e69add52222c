import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def read_golden(name):
    """Parse a ``key = value`` / ``a -> b`` / ``a : b : c`` fixture."""
    path = os.path.join(ROOT, "tests", "golden", name)
    rows = []
    kv = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if " = " in line:
                k, v = line.split(" = ", 1)
                kv[k.strip()] = v.strip()
            else:
                rows.append(line)
    return kv, rows


class ArrayPairs:
    """Pairs given as two (n, L) uint8 arrays of ASCII bytes, same shape as
    ``synth.Pairs`` so that the oracle batch calls accept them."""

    def __init__(self, reads2d, refs2d, E):
        reads2d = np.ascontiguousarray(reads2d, dtype=np.uint8)
        refs2d = np.ascontiguousarray(refs2d, dtype=np.uint8)
        n, L = reads2d.shape
        self.reads = reads2d.reshape(-1) if n * L else np.zeros(1, np.uint8)
        self.refs = refs2d.reshape(-1) if n * L else np.zeros(1, np.uint8)
        self.read_off = np.arange(n + 1, dtype=np.int64) * L
        self.ref_off = self.read_off
        self.lens = np.full(n, L, dtype=np.int32)
        e = np.asarray(E, dtype=np.int16).reshape(-1)
        self.E = np.full(n, e[0], dtype=np.int16) if e.size == 1 else e

    @property
    def n(self):
        return len(self.lens)


def all_pairs(alphabet, L):
    """Every (read, ref) pair of length L over ``alphabet``: two (n, L)
    uint8 arrays with n = |alphabet|^(2L)."""
    codes = np.frombuffer(alphabet.encode(), dtype=np.uint8)
    a = len(codes)
    seqs = np.array(np.meshgrid(*[np.arange(a)] * L, indexing="ij")).reshape(L, -1).T
    seqs = codes[seqs] if L else np.zeros((1, 0), np.uint8)
    ns = seqs.shape[0]
    ri = np.repeat(np.arange(ns), ns)
    fi = np.tile(np.arange(ns), ns)
    return seqs[ri], seqs[fi]


@pytest.fixture(scope="session")
def golden():
    return read_golden
