"""Helpers for the GPU tests: move generated pairs to the device and run the
library's entry points through the Python binding (which calls the C ABI)."""
import numpy as np
import torch

import paper_1910_03936_gb300 as pf

DEV = "cuda:0"


def to_dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(DEV)


class DevicePairs:
    """A synth.Pairs-like batch on the device, packed by pf_pack."""

    def __init__(self, ctx, P, fixed=None):
        self.n = P.n
        self.lens = to_dev(P.lens.astype(np.int32))
        self.E = to_dev(P.E.astype(np.int16))
        self.E_max = int(P.E.max()) if P.n else 0
        reads = to_dev(P.reads if len(P.reads) else np.zeros(1, np.uint8))
        refs = to_dev(P.refs if len(P.refs) else np.zeros(1, np.uint8))
        if fixed is not None:
            self.pairs = pf.pack_pairs(ctx, reads, refs, length=fixed)
        else:
            assert np.array_equal(P.read_off, P.ref_off)
            self.pairs = pf.pack_pairs(ctx, reads, refs, byte_off=P.read_off)


def filter_dev(ctx, D, deciders, plain=False, per_pair_E=True, E_max=None):
    slots = bin(deciders).count("1")
    acc = torch.full((slots * max(D.n, 1),), 0xEE, dtype=torch.uint8, device=DEV)
    cnt = torch.full((slots * max(D.n, 1),), -7, dtype=torch.int16, device=DEV)
    fn = pf.pf_filter_plain if plain else pf.pf_filter
    E = D.E if per_pair_E else None
    fn(ctx, deciders, D.pairs, D.lens, E, D.E_max if E_max is None else E_max, acc, cnt, D.n)
    pf.pf_sync(ctx)
    a = acc.cpu().numpy()[:slots * D.n].reshape(slots, D.n)
    c = cnt.cpu().numpy()[:slots * D.n].reshape(slots, D.n)
    return a, c


def verify_dev(ctx, D, idx=None):
    dist = torch.full((max(D.n, 1),), -9, dtype=torch.int32, device=DEV)
    if idx is None:
        pf.pf_verify(ctx, D.pairs, D.lens, D.E, D.E_max, None, None, dist, D.n)
    else:
        idx_d = to_dev(np.asarray(idx, dtype=np.int64)) if len(idx) else \
            torch.zeros(1, dtype=torch.int64, device=DEV)
        n_idx = torch.tensor([len(idx)], dtype=torch.int64, device=DEV)
        pf.pf_verify(ctx, D.pairs, D.lens, D.E, D.E_max, idx_d, n_idx, dist, D.n)
    pf.pf_sync(ctx)
    return dist.cpu().numpy()[:D.n]
