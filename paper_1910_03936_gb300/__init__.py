"""GB300-native pre-alignment filtering: neighbourhood map, SneakySnake and
GateKeeper deciders, compaction and banded bit-vector verification, behind
the C ABI of ``include/pf.h``.

This module is argument marshalling only: every function below forwards
torch tensors (device memory) to the function of the same name in
``libpf.so`` and turns a non-OK status into :class:`PFError`.  There is no
CPU fallback: every call raises when the library has not been built.
"""
import ctypes
import os

import torch

from . import build as _build_mod

__all__ = [
    "PFError", "Seqs", "Pairs", "PF_SNEAKYSNAKE", "PF_GATEKEEPER", "PF_MAX_E",
    "pf_create", "pf_destroy", "pf_set_stream", "pf_sync", "pf_last_error",
    "pf_pack_layout", "pf_pack", "pf_pack_fixed", "pf_filter", "pf_filter_plain",
    "pf_compact", "pf_verify", "pf_filter_verify", "library_path", "load", "pack_pairs",
    "pf_kernel_configs", "pf_tune_set", "pf_tune_get", "pf_tune", "pf_compact_noalloc",
    "ServeConfig", "Request", "pf_serve_start", "pf_submit", "pf_poll", "pf_wait",
    "pf_serve_resume", "pf_serve_stats_get", "pf_serve_stop", "pf_serve_replay", "pf_run_host",
    "pf_filter_partitioned", "pf_filter_shouji", "pf_filter_shd", "PF_SHD_VACANT_ZERO",
    "PF_SHD_STREAK", "pf_set_small_batch", "pf_tune_batch", "pf_set_resolve_by_bounds",
    "pf_last_verified_count", "pf_peak_int", "PF_SERVE_BATCHED", "PF_SERVE_DEVICE_LOOP",
    "pf_serve_trace", "pf_filter_plain_exact", "pf_pack_layout_grouped", "pf_pack_starts",
    "pf_host_alloc", "pf_host_free", "host_empty",
]

PF_SNEAKYSNAKE = 1
PF_GATEKEEPER = 2
PF_MAX_E = 31
PF_SHD_VACANT_ZERO = 1
PF_SHD_STREAK = 2
PF_SERVE_BATCHED = 0
PF_SERVE_DEVICE_LOOP = 1

_STATUS = {0: "PF_OK", 1: "PF_EINVAL", 2: "PF_ENOMEM", 3: "PF_ECUDA", 4: "PF_ETIMEOUT",
           5: "PF_EBUSY", 6: "PF_ECANCELLED", 7: "PF_EDATA"}


class PFError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (_STATUS.get(status, status), message))
        self.status = status


class _Config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("hbm_budget", ctypes.c_size_t), ("flags", ctypes.c_uint)]


class _Seqs(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_void_p), ("hi", ctypes.c_void_p), ("nmask", ctypes.c_void_p),
                ("word_off", ctypes.c_void_p), ("stride_words", ctypes.c_int64)]


class _Pairs(ctypes.Structure):
    _fields_ = [("read", _Seqs), ("ref", _Seqs)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("max_requests", ctypes.c_int),
                ("chunk_pairs", ctypes.c_int), ("workers", ctypes.c_int),
                ("idle_exit_us", ctypes.c_int), ("start_paused", ctypes.c_int),
                ("mode", ctypes.c_int), ("batch_pairs", ctypes.c_int),
                ("overlap_pairs", ctypes.c_int)]


class _Request(ctypes.Structure):
    _fields_ = [("deciders", ctypes.c_uint), ("n", ctypes.c_int64),
                ("reads", ctypes.c_void_p), ("refs", ctypes.c_void_p),
                ("byte_off", ctypes.c_void_p), ("E", ctypes.c_void_p),
                ("accept", ctypes.c_void_p), ("count", ctypes.c_void_p),
                ("dist", ctypes.c_void_p)]


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("pairs_completed", ctypes.c_uint64),
                ("loop_launches", ctypes.c_uint64), ("queue_s", ctypes.c_double),
                ("stage_s", ctypes.c_double), ("device_s", ctypes.c_double),
                ("drain_s", ctypes.c_double), ("queue_max_s", ctypes.c_double),
                ("stage_max_s", ctypes.c_double), ("device_max_s", ctypes.c_double),
                ("drain_max_s", ctypes.c_double), ("batch_pairs", ctypes.c_uint64),
                ("batch_pairs_max", ctypes.c_uint64), ("batch_gpu_s", ctypes.c_double),
                ("place_host_s", ctypes.c_double), ("launch_host_s", ctypes.c_double)]


_lib = None


def library_path():
    return _build_mod.LIB


def load():
    """Load ``libpf.so``; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise ImportError("libpf.so is not built (run paper_1910_03936_gb300.build.build())")
    lib = ctypes.CDLL(path)
    P, I, I64, U, S = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint,
                       ctypes.c_int)
    sig = {
        "pf_create": [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(_Config)],
        "pf_destroy": [P],
        "pf_set_stream": [P, P],
        "pf_sync": [P],
        "pf_pack_layout": [P, I64, P, ctypes.POINTER(ctypes.c_int64)],
        "pf_pack": [P, P, P, P, I64, P, P, P],
        "pf_pack_layout_grouped": [P, P, I64, P, ctypes.POINTER(ctypes.c_int64)],
        "pf_host_alloc": [ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)],
        "pf_host_free": [P],
        "pf_pack_starts": [P, P, P, P, I64, P, P, P],
        "pf_pack_fixed": [P, P, I64, I, P, P, P],
        "pf_filter": [P, U, ctypes.POINTER(_Pairs), P, P, I, P, P, I64],
        "pf_filter_plain": [P, U, ctypes.POINTER(_Pairs), P, P, I, P, P, I64],
        "pf_filter_plain_exact": [P, U, ctypes.POINTER(_Pairs), P, I, P, P, I64],
        "pf_filter_partitioned": [P, ctypes.POINTER(_Pairs), P, P, I, I, I, P, P, I64],
        "pf_filter_shouji": [P, ctypes.POINTER(_Pairs), P, P, I, P, P, I64],
        "pf_filter_shd": [P, ctypes.POINTER(_Pairs), P, P, I, U, P, P, I64],
        "pf_compact": [P, P, I64, P, P],
        "pf_compact_noalloc": [P, I64, P, P, P],
        "pf_verify": [P, ctypes.POINTER(_Pairs), P, P, I, P, P, I64, P],
        "pf_filter_verify": [P, U, ctypes.POINTER(_Pairs), P, P, I, P, P, P, I64],
        "pf_kernel_configs": [P, P, P, P, P, I, ctypes.POINTER(ctypes.c_int)],
        "pf_serve_start": [P, ctypes.POINTER(ServeConfig)],
        "pf_submit": [P, ctypes.POINTER(_Request), ctypes.POINTER(ctypes.c_uint64)],
        "pf_poll": [P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)],
        "pf_wait": [P, ctypes.c_uint64, I, ctypes.POINTER(ctypes.c_double)],
        "pf_serve_resume": [P],
        "pf_serve_stats_get": [P, ctypes.POINTER(ServeStats)],
        "pf_serve_stop": [P],
        "pf_serve_trace": [P, P, I, ctypes.POINTER(ctypes.c_int)],
        "pf_run_host": [P, U, P, P, P, I, P, I, P, P, P, I64, I64],
        "pf_serve_replay": [P, P, I, P, I, P, ctypes.POINTER(ctypes.c_double)],
        "pf_tune_set": [P, U, I, I, I],
        "pf_set_small_batch": [P, I64],
        "pf_set_resolve_by_bounds": [P, I],
        "pf_last_verified_count": [P, ctypes.POINTER(ctypes.c_int64)],
        "pf_peak_int": [P, I, I, ctypes.POINTER(ctypes.c_double),
                        ctypes.POINTER(ctypes.c_double)],
        "pf_tune_batch": [P, U, ctypes.POINTER(_Pairs), P, P, I, I64, I64, I],
        "pf_tune_get": [P, U, I, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
        "pf_tune": [P, U, ctypes.POINTER(_Pairs), P, I, I64, I, ctypes.POINTER(ctypes.c_int),
                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = S
    lib.pf_last_error.argtypes = [P]
    lib.pf_last_error.restype = ctypes.c_char_p
    lib.pf_status_string.argtypes = [S]
    lib.pf_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status, ctx=None):
    if status != 0:
        msg = load().pf_last_error(ctx).decode() if ctx is not None else ""
        raise PFError(status, msg)


def _p(t):
    """Device address of a tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _dt(t, dtype, name):
    if t is not None and t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))


class Seqs:
    """Packed sequences: three int32 bit-plane tensors and either int64 word
    offsets (n+1 entries) or a fixed stride in words."""

    def __init__(self, lo, hi, nmask, word_off=None, stride_words=0):
        for t, nm in ((lo, "lo"), (hi, "hi"), (nmask, "nmask")):
            _dt(t, torch.int32, nm)
        _dt(word_off, torch.int64, "word_off")
        self.lo, self.hi, self.nmask = lo, hi, nmask
        self.word_off, self.stride_words = word_off, int(stride_words)

    def _c(self):
        return _Seqs(self.lo.data_ptr(), self.hi.data_ptr(), self.nmask.data_ptr(),
                     self.word_off.data_ptr() if self.word_off is not None else None,
                     self.stride_words)

    @staticmethod
    def empty(total_words, device, word_off=None, stride_words=0):
        mk = lambda: torch.empty(max(int(total_words), 1), dtype=torch.int32, device=device)
        return Seqs(mk(), mk(), mk(), word_off, stride_words)


class Pairs:
    def __init__(self, read, ref):
        self.read, self.ref = read, ref

    def _c(self):
        return _Pairs(self.read._c(), self.ref._c())


class _Ctx:
    """Owning handle of a pf_ctx."""

    def __init__(self, handle, device):
        self.handle, self.device = handle, device

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            try:
                _lib.pf_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


def _cur_stream(ctx):
    st = torch.cuda.current_stream(ctx.device).cuda_stream
    _check(load().pf_set_stream(ctx.handle, ctypes.c_void_p(st)), ctx.handle)


def pf_create(device=0, stream=None, hbm_budget=0):
    lib = load()
    cfg = _Config(device, stream if stream is not None
                  else torch.cuda.current_stream(device).cuda_stream, hbm_budget, 0)
    h = ctypes.c_void_p()
    st = lib.pf_create(ctypes.byref(h), ctypes.byref(cfg))
    if st != 0:
        raise PFError(st, lib.pf_last_error(None).decode())
    return _Ctx(h, device)


def pf_destroy(ctx):
    if ctx.handle:
        st = load().pf_destroy(ctx.handle)
        ctx.handle = None
        _check(st)


def pf_set_stream(ctx, stream):
    _check(load().pf_set_stream(ctx.handle, ctypes.c_void_p(int(stream))), ctx.handle)


def pf_sync(ctx):
    _check(load().pf_sync(ctx.handle), ctx.handle)


def pf_last_error(ctx):
    return load().pf_last_error(ctx.handle).decode()


def pf_pack_layout(byte_off):
    """Host int64 byte offsets (numpy or list, nseq+1) -> (word_off numpy, total)."""
    import numpy as np
    bo = np.ascontiguousarray(byte_off, dtype=np.int64)
    nseq = len(bo) - 1
    wo = np.zeros(nseq + 1, dtype=np.int64)
    total = ctypes.c_int64()
    _check(load().pf_pack_layout(ctypes.c_void_p(bo.ctypes.data), nseq,
                                 ctypes.c_void_p(wo.ctypes.data), ctypes.byref(total)))
    return wo, int(total.value)


def pf_host_alloc(nbytes):
    """Page-locked host block of at least nbytes (huge pages where the
    system has them); returns its address.  Free with pf_host_free."""
    p = ctypes.c_void_p()
    _check(load().pf_host_alloc(ctypes.c_size_t(int(nbytes)), ctypes.byref(p)))
    return p.value


def pf_host_free(addr):
    _check(load().pf_host_free(ctypes.c_void_p(addr)))


def host_empty(count, dtype):
    """A numpy array of `count` elements in pf_host_alloc memory, freed when
    the last view of it goes away."""
    import numpy as np
    import weakref
    dt = np.dtype(dtype)
    nbytes = max(int(count) * dt.itemsize, 1)
    addr = pf_host_alloc(nbytes)
    raw = (ctypes.c_uint8 * nbytes).from_address(addr)
    weakref.finalize(raw, pf_host_free, addr)
    return np.frombuffer(raw, dtype=np.uint8)[:int(count) * dt.itemsize].view(dt)


def pf_pack_layout_grouped(byte_off, E=None):
    """Host int64 byte offsets (nseq+1) and optional host int16 thresholds
    (nseq) -> (word_start numpy int64[nseq], total words)."""
    import numpy as np
    bo = np.ascontiguousarray(byte_off, dtype=np.int64)
    nseq = len(bo) - 1
    Eh = None
    if E is not None:
        Eh = np.ascontiguousarray(E, dtype=np.int16)
        if Eh.shape != (nseq,):
            raise ValueError("E must hold one threshold per sequence")
    ws = np.zeros(max(nseq, 0), dtype=np.int64)
    total = ctypes.c_int64()
    _check(load().pf_pack_layout_grouped(
        ctypes.c_void_p(bo.ctypes.data), ctypes.c_void_p(Eh.ctypes.data) if Eh is not None else None,
        nseq, ctypes.c_void_p(ws.ctypes.data), ctypes.byref(total)))
    return ws, int(total.value)


def pf_pack_starts(ctx, ascii, byte_off, word_start, out):
    """Pack ragged ASCII into ``out`` (a Seqs) at per-sequence first words."""
    _dt(ascii, torch.uint8, "ascii")
    _dt(byte_off, torch.int64, "byte_off")
    _dt(word_start, torch.int64, "word_start")
    nseq = byte_off.numel() - 1
    if word_start.numel() < nseq:
        raise ValueError("word_start needs one entry per sequence")
    _cur_stream(ctx)
    _check(load().pf_pack_starts(ctx.handle, _p(ascii), _p(byte_off), _p(word_start), nseq,
                                 _p(out.lo), _p(out.hi), _p(out.nmask)), ctx.handle)


def pf_pack(ctx, ascii, byte_off, word_off, out):
    """Pack ragged ASCII (uint8 device tensor) into ``out`` (a Seqs)."""
    _dt(ascii, torch.uint8, "ascii")
    _dt(byte_off, torch.int64, "byte_off")
    _dt(word_off, torch.int64, "word_off")
    _cur_stream(ctx)
    nseq = byte_off.numel() - 1
    _check(load().pf_pack(ctx.handle, _p(ascii), _p(byte_off), _p(word_off), nseq,
                          _p(out.lo), _p(out.hi), _p(out.nmask)), ctx.handle)


def pf_pack_fixed(ctx, ascii, nseq, length, out):
    _dt(ascii, torch.uint8, "ascii")
    _cur_stream(ctx)
    _check(load().pf_pack_fixed(ctx.handle, _p(ascii), int(nseq), int(length), _p(out.lo),
                                _p(out.hi), _p(out.nmask)), ctx.handle)


def _filter_call(fn, ctx, deciders, pairs, lens, E, E_max, accept, count, n):
    _dt(lens, torch.int32, "lens")
    _dt(E, torch.int16, "E")
    _dt(accept, torch.uint8, "accept")
    _dt(count, torch.int16, "count")
    _cur_stream(ctx)
    cp = pairs._c()
    _check(fn(ctx.handle, int(deciders), ctypes.byref(cp), _p(lens), _p(E), int(E_max),
              _p(accept), _p(count), int(n)), ctx.handle)


def pf_filter(ctx, deciders, pairs, lens, E, E_max, accept, count, n=None):
    n = lens.numel() if n is None else n
    _filter_call(load().pf_filter, ctx, deciders, pairs, lens, E, E_max, accept, count, n)


def pf_filter_plain(ctx, deciders, pairs, lens, E, E_max, accept, count, n=None):
    n = lens.numel() if n is None else n
    _filter_call(load().pf_filter_plain, ctx, deciders, pairs, lens, E, E_max, accept, count, n)


def pf_filter_plain_exact(ctx, deciders, pairs, lens, E, accept, count, n=None):
    """The plain kernel with one threshold E (0..15) fixed at compile time."""
    _dt(lens, torch.int32, "lens")
    _dt(accept, torch.uint8, "accept")
    _dt(count, torch.int16, "count")
    n = lens.numel() if n is None else n
    _cur_stream(ctx)
    cp = pairs._c()
    _check(load().pf_filter_plain_exact(ctx.handle, int(deciders), ctypes.byref(cp), _p(lens),
                                        int(E), _p(accept), _p(count), int(n)), ctx.handle)


def _variant_call(fn, ctx, pairs, lens, E, E_max, extra, accept, count, n):
    _dt(lens, torch.int32, "lens")
    _dt(E, torch.int16, "E")
    _dt(accept, torch.uint8, "accept")
    _dt(count, torch.int16, "count")
    n = lens.numel() if n is None else n
    _cur_stream(ctx)
    cp = pairs._c()
    _check(fn(ctx.handle, ctypes.byref(cp), _p(lens), _p(E), int(E_max), *extra, _p(accept),
              _p(count), int(n)), ctx.handle)


def pf_filter_partitioned(ctx, pairs, lens, E, E_max, t, y, accept, count, n=None):
    """SneakySnake on sub-matrices of t columns with y replications each."""
    _variant_call(load().pf_filter_partitioned, ctx, pairs, lens, E, E_max, (int(t), int(y)),
                  accept, count, n)


def pf_filter_shouji(ctx, pairs, lens, E, E_max, accept, count, n=None):
    """Shouji: 4-column windows and the Shouji bit-vector."""
    _variant_call(load().pf_filter_shouji, ctx, pairs, lens, E, E_max, (), accept, count, n)


def pf_filter_shd(ctx, pairs, lens, E, E_max, flags, accept, count, n=None):
    """GateKeeper with SHD's vacant-zero masks and/or streak counting."""
    _variant_call(load().pf_filter_shd, ctx, pairs, lens, E, E_max, (int(flags),), accept,
                  count, n)


def _compact_args(flags, idx, n_out, n):
    _dt(flags, torch.uint8, "flags")
    _dt(idx, torch.int64, "idx")
    _dt(n_out, torch.int64, "n_out")
    n = flags.numel() if n is None else int(n)
    if n < 0 or n > flags.numel() or n > idx.numel() or n_out.numel() < 1:
        raise ValueError("n = %d outside the buffers (flags %d, idx %d, n_out %d elements)"
                         % (n, flags.numel(), idx.numel(), n_out.numel()))
    if not (flags.device == idx.device == n_out.device):
        raise ValueError("flags, idx and n_out must be on one device")
    return n


def pf_compact(ctx, flags, idx, n_out, n=None):
    n = _compact_args(flags, idx, n_out, n)
    _cur_stream(ctx)
    _check(load().pf_compact(ctx.handle, _p(flags), n, _p(idx), _p(n_out)), ctx.handle)


def pf_compact_noalloc(flags, idx, n_out, n=None, stream=None):
    """pf_compact without a context and without any device allocation
    (fixed in-library counters, n <= 134,217,728; concurrent calls race).
    Runs with the buffers' device current, on its current stream unless
    ``stream`` is given."""
    n = _compact_args(flags, idx, n_out, n)
    with torch.cuda.device(flags.device):
        if stream is None:
            stream = torch.cuda.current_stream(flags.device).cuda_stream
        _check(load().pf_compact_noalloc(_p(flags), n, _p(idx), _p(n_out),
                                         ctypes.c_void_p(int(stream))))


def pf_verify(ctx, pairs, lens, E, E_max, idx, n_idx, dist, n=None):
    _dt(lens, torch.int32, "lens")
    _dt(E, torch.int16, "E")
    _dt(idx, torch.int64, "idx")
    _dt(n_idx, torch.int64, "n_idx")
    _dt(dist, torch.int32, "dist")
    n = lens.numel() if n is None else n
    _cur_stream(ctx)
    cp = pairs._c()
    _check(load().pf_verify(ctx.handle, ctypes.byref(cp), _p(lens), _p(E), int(E_max), _p(idx),
                            _p(n_idx), int(n), _p(dist)), ctx.handle)


def pf_filter_verify(ctx, deciders, pairs, lens, E, E_max, accept, count, dist, n=None):
    _dt(lens, torch.int32, "lens")
    _dt(E, torch.int16, "E")
    _dt(accept, torch.uint8, "accept")
    _dt(count, torch.int16, "count")
    _dt(dist, torch.int32, "dist")
    n = lens.numel() if n is None else n
    _cur_stream(ctx)
    cp = pairs._c()
    _check(load().pf_filter_verify(ctx.handle, int(deciders), ctypes.byref(cp), _p(lens), _p(E),
                                   int(E_max), _p(accept), _p(count), _p(dist), int(n)),
           ctx.handle)


def pack_pairs(ctx, reads, refs, length=None, byte_off=None, group_E=None):
    """Pack device ASCII reads and refs (uint8 tensors) with pf_pack.

    Fixed length: pass ``length`` (sequence s is bytes [s*length,
    (s+1)*length)).  Ragged: pass ``byte_off`` as host int64 offsets
    (numpy, n+1 entries) shared by reads and refs; word offsets come from
    pf_pack_layout, or, with ``group_E`` (host per-pair thresholds), from
    pf_pack_layout_grouped (packed with pf_pack_starts).  Returns a
    :class:`Pairs`.
    """
    dev = reads.device
    if length is not None:
        n = reads.numel() // length if length else 0
        W = (length + 31) // 32
        out = []
        for src in (reads, refs):
            s = Seqs.empty(n * W, dev, stride_words=W)
            if n and length:
                pf_pack_fixed(ctx, src, n, length, s)
            out.append(s)
        return Pairs(out[0], out[1])
    import numpy as np
    bo_d = torch.from_numpy(np.ascontiguousarray(byte_off, dtype=np.int64)).to(dev)
    if group_E is not None:
        ws, total = pf_pack_layout_grouped(byte_off, group_E)
        ws_d = torch.from_numpy(ws).to(dev)
        out = []
        for src in (reads, refs):
            s = Seqs.empty(total, dev, word_off=ws_d)
            pf_pack_starts(ctx, src, bo_d, ws_d, s)
            out.append(s)
        return Pairs(out[0], out[1])
    wo, total = pf_pack_layout(byte_off)
    wo_d = torch.from_numpy(wo).to(dev)
    out = []
    for src in (reads, refs):
        s = Seqs.empty(total, dev, word_off=wo_d)
        pf_pack(ctx, src, bo_d, wo_d, s)
        out.append(s)
    return Pairs(out[0], out[1])


def pf_kernel_configs():
    """List of (tpp, dpt, ecap, exact_e, words) of the batch scheduler's
    kernels; exact_e >= 0 marks a kernel that serves that threshold only,
    words > 0 its two-phase form (mask words of pairs up to that many
    32-column words kept in shared memory)."""
    import numpy as np
    cnt = ctypes.c_int()
    _check(load().pf_kernel_configs(None, None, None, None, None, 0, ctypes.byref(cnt)))
    a = [np.zeros(cnt.value, dtype=np.int32) for _ in range(5)]
    _check(load().pf_kernel_configs(*[ctypes.c_void_p(x.ctypes.data) for x in a], cnt.value,
                                    ctypes.byref(cnt)))
    return [tuple(int(x[i]) for x in a) for i in range(cnt.value)]


def pf_tune_set(ctx, deciders, E, cfg, chunk):
    _check(load().pf_tune_set(ctx.handle, int(deciders), int(E), int(cfg), int(chunk)), ctx.handle)


def pf_tune_batch(ctx, deciders, pairs, lens, E, E_max, n=None, sample=0, reps=2):
    """Autotune every threshold of this batch on its own pairs."""
    _dt(lens, torch.int32, "lens")
    _dt(E, torch.int16, "E")
    n = lens.numel() if n is None else n
    _cur_stream(ctx)
    cp = pairs._c()
    _check(load().pf_tune_batch(ctx.handle, int(deciders), ctypes.byref(cp), _p(lens), _p(E),
                                int(E_max), int(n), int(sample), int(reps)), ctx.handle)


def pf_set_small_batch(ctx, pairs):
    """Batches below `pairs` take one plain launch (0: always the scheduler)."""
    _check(load().pf_set_small_batch(ctx.handle, int(pairs)), ctx.handle)


def pf_set_resolve_by_bounds(ctx, enable):
    """Skip verifying accepted pairs whose SneakySnake count equals their
    Hamming distance (default on; results are the same either way)."""
    _check(load().pf_set_resolve_by_bounds(ctx.handle, int(bool(enable))), ctx.handle)


def pf_last_verified_count(ctx):
    """Pairs the last pf_filter_verify on ctx sent to verification."""
    v = ctypes.c_int64()
    _check(load().pf_last_verified_count(ctx.handle, ctypes.byref(v)), ctx.handle)
    return v.value


def pf_peak_int(ctx, kind=0, launches=30):
    """Integer-pipe microbenchmark: (instructions/s, ms per launch) of the
    LOP3+SHF mix (kind 0) or POPC+LOP3 (kind 1) over a full-occupancy grid."""
    ops, ms = ctypes.c_double(), ctypes.c_double()
    _cur_stream(ctx)
    _check(load().pf_peak_int(ctx.handle, int(kind), int(launches), ctypes.byref(ops),
                              ctypes.byref(ms)), ctx.handle)
    return ops.value, ms.value


def pf_tune_get(ctx, deciders, E):
    c, k = ctypes.c_int(), ctypes.c_int()
    _check(load().pf_tune_get(ctx.handle, int(deciders), int(E), ctypes.byref(c), ctypes.byref(k)),
           ctx.handle)
    return c.value, k.value


def pf_tune(ctx, deciders, pairs, lens, E, n=None, reps=3):
    """Autotune (deciders, E) on these pairs; returns (cfg, chunk, ms)."""
    _dt(lens, torch.int32, "lens")
    n = lens.numel() if n is None else n
    _cur_stream(ctx)
    cp = pairs._c()
    c, k, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    _check(load().pf_tune(ctx.handle, int(deciders), ctypes.byref(cp), _p(lens), int(E), int(n),
                          int(reps), ctypes.byref(c), ctypes.byref(k), ctypes.byref(ms)),
           ctx.handle)
    return c.value, k.value, ms.value


# ---- a8 serving -----------------------------------------------------------

def pf_serve_start(ctx, hbm_budget=0, max_requests=0, chunk_pairs=0, workers=0,
                   idle_exit_us=0, start_paused=False, mode=0, batch_pairs=0, overlap_pairs=0):
    """Start serving; mode PF_SERVE_BATCHED (0) or PF_SERVE_DEVICE_LOOP (1)."""
    cfg = ServeConfig(hbm_budget, max_requests, chunk_pairs, workers, idle_exit_us,
                      1 if start_paused else 0, int(mode), int(batch_pairs), int(overlap_pairs))
    _check(load().pf_serve_start(ctx.handle, ctypes.byref(cfg)), ctx.handle)


class Request:
    """A request in host memory (numpy arrays).  The arrays are kept
    referenced here until the request is waited for.  pinned=True copies the
    inputs into, and allocates the outputs in, page-locked memory from
    pf_host_alloc (the fast path: asynchronous uploads, results written in
    place by the GPU)."""

    def __init__(self, deciders, reads, refs, byte_off, E, pinned=False):
        import numpy as np

        def host(a, dtype):
            a = np.ascontiguousarray(a, dtype=dtype)
            if pinned:
                h = host_empty(a.size, dtype)
                h[:] = a
                return h
            return a

        def zeros(count, dtype):
            dt = torch.empty(0, dtype=dtype).numpy().dtype
            if pinned:
                h = host_empty(count, dt)
                h[:] = 0
                return h
            return np.zeros(count, dtype=dt)

        self._keep = []
        self.reads = host(reads, np.uint8)
        self.refs = host(refs, np.uint8)
        self.byte_off = host(byte_off, np.int64)
        self.E = host(E, np.int16)
        self.n = len(self.byte_off) - 1
        slots = 2 if deciders == 3 else 1
        self.deciders = deciders
        self.accept = zeros(slots * max(self.n, 1), torch.uint8)
        self.count = zeros(slots * max(self.n, 1), torch.int16)
        self.dist = zeros(max(self.n, 1), torch.int32)
        self.ticket = None

    def _c(self):
        ptr = lambda a: ctypes.c_void_p(a.ctypes.data) if a.size else None
        return _Request(self.deciders, self.n, ptr(self.reads), ptr(self.refs),
                        ptr(self.byte_off), ptr(self.E), ptr(self.accept),
                        ptr(self.count), ptr(self.dist))


def pf_submit(ctx, req):
    t = ctypes.c_uint64()
    c = req._c()
    _check(load().pf_submit(ctx.handle, ctypes.byref(c), ctypes.byref(t)), ctx.handle)
    req.ticket = t.value
    return t.value


def pf_poll(ctx, ticket):
    d = ctypes.c_int()
    _check(load().pf_poll(ctx.handle, ticket, ctypes.byref(d)), ctx.handle)
    return bool(d.value)


def pf_wait(ctx, ticket, timeout_ms=-1):
    """Returns (status, latency_ms); status 0 is PF_OK, 4 PF_ETIMEOUT."""
    lat = ctypes.c_double()
    st = load().pf_wait(ctx.handle, ticket, int(timeout_ms), ctypes.byref(lat))
    return st, lat.value


def pf_serve_resume(ctx):
    _check(load().pf_serve_resume(ctx.handle), ctx.handle)


def pf_serve_stats_get(ctx):
    st = ServeStats()
    _check(load().pf_serve_stats_get(ctx.handle, ctypes.byref(st)), ctx.handle)
    return {f: getattr(st, f) for f, _ in ServeStats._fields_}


def pf_serve_trace(ctx, cap=65536):
    """Batched mode: the most recent device batches as a float64 array of
    shape (k, 13): launch s, completion s, pairs, request parts, ms waiting
    for uploads / the previous batch, GPU ms, enqueue ms, decider set, GPU ms
    of the offsets, pack, filter, compaction + verification and epilogue."""
    import numpy as np
    out = np.zeros((max(cap, 1), 13), dtype=np.float64)
    k = ctypes.c_int()
    _check(load().pf_serve_trace(ctx.handle, ctypes.c_void_p(out.ctypes.data), int(cap),
                                 ctypes.byref(k)), ctx.handle)
    return out[:k.value]


def pf_serve_stop(ctx):
    _check(load().pf_serve_stop(ctx.handle), ctx.handle)


def pf_serve_replay(ctx, pool, arrival_s):
    """Submit pool[i % len(pool)] at arrival_s[i] (seconds from the call)
    from a C thread, wait for all; returns (status, latency_ms[], elapsed_s)."""
    import numpy as np
    arr = (_Request * len(pool))(*[r._c() for r in pool])
    t = np.ascontiguousarray(arrival_s, dtype=np.float64)
    lat = np.zeros(max(len(t), 1), dtype=np.float64)
    el = ctypes.c_double()
    st = load().pf_serve_replay(ctx.handle, ctypes.cast(arr, ctypes.c_void_p), len(pool),
                                ctypes.c_void_p(t.ctypes.data), len(t),
                                ctypes.c_void_p(lat.ctypes.data), ctypes.byref(el))
    return st, lat[:len(t)], el.value


def pf_run_host(ctx, deciders, reads, refs, E_max, byte_off=None, length=0, E=None,
                chunk_pairs=0, out=None):
    """Whole path on host numpy arrays, chunked and graph-replayed on the
    device.  Returns (accept[slots, n], count[slots, n], dist[n])."""
    import numpy as np
    reads = np.ascontiguousarray(reads, dtype=np.uint8)
    refs = np.ascontiguousarray(refs, dtype=np.uint8)
    if byte_off is not None:
        byte_off = np.ascontiguousarray(byte_off, dtype=np.int64)
        n = len(byte_off) - 1
    else:
        n = reads.size // length if length else 0
    slots = 2 if deciders == 3 else 1
    if out is None:
        out = (np.zeros(slots * max(n, 1), np.uint8), np.zeros(slots * max(n, 1), np.int16),
               np.zeros(max(n, 1), np.int32))
    acc, cnt, dist = out
    ptr = lambda a: ctypes.c_void_p(a.ctypes.data) if a is not None else None
    if E is not None:
        E = np.ascontiguousarray(E, dtype=np.int16)
    _check(load().pf_run_host(ctx.handle, int(deciders), ptr(reads), ptr(refs), ptr(byte_off),
                              int(length), ptr(E), int(E_max), ptr(acc), ptr(cnt), ptr(dist),
                              int(n), int(chunk_pairs)), ctx.handle)
    return acc[:slots * n].reshape(slots, n), cnt[:slots * n].reshape(slots, n), dist[:n]
