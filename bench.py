"""Benchmark of the pre-alignment filtering hot path on GB300.

Workload (one GPU): 20,000,000 read/reference pairs of 150 bp, E = 6,
bases 0.1% N and 41% GC, 20% of pairs with at most E edits and 80% with
E+1..60 edits (sub/ins/del 0.6/0.2/0.2), seeded synthetic ASCII resident in
HBM (inputs are far larger than L2, so no flush is needed between steps).

One step = the whole hot path over the batch: pack reads and references to
bit-planes, filter with SneakySnake and GateKeeper (batched persistent
kernels), compact the pairs SneakySnake accepts, verify them with the banded
bit-vector kernel.  value = pairs per second of that step.

Extra keys: per-stage times, the plain vs batched SneakySnake filter kernel
(pairs/s), the roofline of the dominant kernel, the end-to-end figure
(host ASCII in pinned memory -> device -> step -> results back), SM clocks
sampled during the timed region, and the CPU oracle timed on a bounded
sample on the host cores.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank runs an independent replica on its own
GPU and its own shard of pairs (weak scaling); rank 0 prints the line with
the slowest rank's time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

M, E_HEAD, N_PAIRS, KMAX = 150, 6, 20_000_000, 60
SEED = 0x5EED0001
METRIC = "pairs/s (SneakySnake, 150bp, E=6) batched vs plain kernel; serve p50/p99 ms"
WORKLOAD = "cfg2_150bp_E6_20M"



def host_copy(pf, a):
    """A copy of numpy array a in page-locked host memory from pf_host_alloc
    (huge pages: uploads from it do not stall), as a torch tensor."""
    import torch
    h = pf.host_empty(a.size, a.dtype)
    h[:] = a.reshape(-1)
    return torch.from_numpy(h)


def host_zeros(pf, count, dtype):
    import torch
    h = pf.host_empty(count, torch.empty(0, dtype=dtype).numpy().dtype)
    h[:] = 0
    return torch.from_numpy(h)

def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling in the background during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# multi-rank helpers: replicas on their own shards, control-plane reduction

def shard_start(rank, pairs_per_rank):
    """First pair index of a rank's shard (weak scaling: every rank owns
    pairs_per_rank consecutive pairs of the generator's pair space)."""
    return rank * pairs_per_rank


def max_over_ranks(value, dist=None):
    """The slowest rank's time (MAX all-reduce on the host, no GPU data)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def headline_config(n):
    """The workload both arms name (the reference arm times a sample of it)."""
    return {"workload": WORKLOAD, "pairs_per_gpu": n, "read_len": M, "E": E_HEAD,
            "deciders": "SneakySnake+GateKeeper",
            "verify": "SneakySnake accepts whose count differs from their Hamming "
                      "distance (equal bounds resolve the rest)",
            "l2": "inputs larger than L2 (9 GB resident)"}


# ---------------------------------------------------------------------------
# CPU oracle baseline (also the reference arm)

def oracle_step_rate(n_sample, threads=None):
    """Time the oracle on pairs [0, n_sample) of the workload: filter with
    both deciders, then banded Wagner-Fischer on the SneakySnake accepts.
    Returns (pairs/s, seconds, threads)."""
    import oracle
    import synth
    threads = threads or os.cpu_count() or 1
    P = synth.generate(synth.SKEWED, SEED, n_sample, m=M, E=E_HEAD, kmax=KMAX, threads=threads)
    t0 = time.perf_counter()
    acc, _ = oracle.filter_batch(P, deciders=3, threads=threads)
    sel = np.nonzero(acc[0])[0]
    sub = synth.Pairs(P.reads, P.refs, P.read_off[sel], P.ref_off[sel], P.lens[sel], P.E[sel])
    oracle.verify_batch(sub, threads=threads)
    dt = time.perf_counter() - t0
    return n_sample / dt, dt, threads


def needed_ops_per_pair(n_sample):
    """Integer operations the method needs per pair on average, counted on
    the first n_sample pairs of the workload by the oracle's work counters
    (part of the CPU-baseline leg): the per-word figures of the full count,
    applied to the words each decider needs before it is decided (a
    word-parallel kernel stops a pair once both are).  Returns (ops, what)."""
    import oracle
    import synth
    P = synth.generate(synth.SKEWED, SEED, n_sample, m=M, E=E_HEAD, kmax=KMAX)
    w = oracle.work_batch(P).astype(np.int64)
    D = 2 * E_HEAD + 1
    words = lambda cols: (cols + 31) // 32
    w_map = words(np.maximum(w[:, 1], w[:, 3]))
    w_and, w_ham = words(w[:, 3]), words(w[:, 2])
    ops = (5 * D * w_map + 5 * np.maximum(w_ham - w_map, 0)   # map (d = 0 alone past it)
           + 8 * D * w_and + w_ham                            # GateKeeper
           + (3 * D + 1) * w[:, 0])                           # SneakySnake searches
    what = ("oracle work counts on pairs 0..%d: SneakySnake %.2f search-words, map %.2f "
            "words, GateKeeper AND %.2f words, Hamming %.2f words per pair"
            % (n_sample, w[:, 0].mean(), w_map.mean(), w_and.mean(), w_ham.mean()))
    return float(ops.mean()), what


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n_sample = args.ref_sample
    times = []
    rate = None
    for i in range(args.warmup + args.steps):
        r, dt, thr = oracle_step_rate(n_sample)
        if i >= args.warmup:
            times.append(dt)
            rate = r
    ms = 1000.0 * statistics.mean(times)
    value = n_sample / (ms / 1000.0)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": headline_config(args.pairs),
        "sample_pairs_per_step": n_sample,
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": thr, "kind": "oracle",
                         "sample": "each step times pairs 0..%d of the %d-pair workload "
                                   "(filter both deciders + banded WF on SneakySnake "
                                   "accepts); value = sampled pairs / time"
                                   % (n_sample, args.pairs)},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# serving: offered-load replay through the device-resident loop

def serve_pool(pf, seed, count=48, pinned=True):
    """Requests of log-uniform size in [1e3, 2e5] pairs, lengths uniform over
    {100, 150, 250}, E = round(r * len) with r ~ U[0, 0.10), 20/80 mix of
    pairs within / beyond E (the serving recipe of synth), in page-locked
    host memory."""
    import synth
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(1e3), np.log(2e5), size=count)).astype(np.int64)
    pool, p0 = [], 0
    for n in sizes:
        P = synth.generate(synth.SERVE, seed, int(n), kmax=60, p0=p0)
        p0 += int(n)
        pool.append(pf.Request(3, P.reads, P.refs, P.read_off, P.E, pinned=pinned))
    return pool, sizes, rng


def serve_reference_rates(pf, ctx, seed, n=4_000_000):
    """The two numbers the offered loads are stated against: the batched
    path's device throughput on a resident batch of the serving mix (pack +
    filter with both deciders + compaction + verification, the same tuned
    path the batched serving mode runs), and the host link's bound for the
    serving mix (pinned host -> device copy rate / bytes moved per pair)."""
    import torch
    import synth
    dev = torch.device("cuda", 0)
    P = synth.generate(synth.SERVE, seed + 99, n, kmax=60)
    reads_h = host_copy(pf, P.reads)
    reads = reads_h.to(dev)
    refs = torch.from_numpy(P.refs).to(dev)
    wo, total = pf.pf_pack_layout(P.read_off)
    bo_d = torch.from_numpy(P.read_off).to(dev)
    wo_d = torch.from_numpy(wo).to(dev)
    rd = pf.Seqs.empty(total, dev, word_off=wo_d)
    rf = pf.Seqs.empty(total, dev, word_off=wo_d)
    pairs = pf.Pairs(rd, rf)
    lens = torch.from_numpy(P.lens).to(dev)
    E = torch.from_numpy(P.E).to(dev)
    Emax = int(P.E.max())
    acc = torch.empty(2 * n, dtype=torch.uint8, device=dev)
    cnt = torch.empty(2 * n, dtype=torch.int16, device=dev)
    dist = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    pf.pf_pack(ctx, reads, bo_d, wo_d, rd)
    pf.pf_pack(ctx, refs, bo_d, wo_d, rf)
    pf.pf_tune_batch(ctx, 3, pairs, lens, E, Emax, n=n, sample=1 << 18, reps=1)

    def step():
        pf.pf_pack(ctx, reads, bo_d, wo_d, rd)
        pf.pf_pack(ctx, refs, bo_d, wo_d, rf)
        pf.pf_filter_verify(ctx, 3, pairs, lens, E, Emax, acc, cnt, dist, n)

    for _ in range(3):
        step()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(5):
        step()
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / 5
    # host link: pinned -> device copies of the reads buffer
    for _ in range(2):
        reads.copy_(reads_h, non_blocking=True)
    a.record(stream)
    for _ in range(5):
        reads.copy_(reads_h, non_blocking=True)
    b.record(stream)
    torch.cuda.synchronize(dev)
    h2d_gbs = 5 * reads_h.numel() / (a.elapsed_time(b) / 1000.0) / 1e9
    bytes_per_pair = 2.0 * float(P.read_off[-1]) / n + 8 + 2   # ASCII, offset, threshold
    return {"batched_peak_pairs_s": n / (ms / 1000.0), "batched_ms": ms, "batch_pairs": n,
            "h2d_gbs": h2d_gbs, "h2d_bytes_per_pair": bytes_per_pair,
            "link_bound_pairs_s": h2d_gbs * 1e9 / bytes_per_pair}


def serve_measure(pf, ctx, seconds_per_load, seed, mode=0, ref=None, loads=(0.25, 0.5, 0.9)):
    """Serving through pf_serve_replay.  Peak = pairs/s of a burst of every
    request of the pool (16 times over, about 25M pairs) submitted at once,
    the best of three; then Poisson
    arrivals at fractions of that peak and, when it is below the peak, at a
    quarter of the batched path's device throughput (ref).  Latency = submit
    to results in host memory."""
    pool, sizes, rng = serve_pool(pf, seed)
    mean_pairs = float(sizes.mean())
    pf.pf_serve_start(ctx, mode=mode)
    pf.pf_serve_replay(ctx, pool[:8], np.zeros(8))           # warm-up
    burst = np.zeros(16 * len(pool))
    bursts = []
    for _ in range(3):   # the host is shared: the best of three bursts
        st, lat, el = pf.pf_serve_replay(ctx, pool, burst)
        bursts.append(16 * float(sizes.sum()) / el)
    peak = max(bursts)
    out = {"mode": "batched" if mode == 0 else "device_loop", "peak_pairs_s": peak,
           "burst_pairs_s": bursts,
           "requests_pool": len(pool), "mean_request_pairs": mean_pairs, "status": int(st),
           "buffers": "page-locked host"}
    points = [("load_%d" % int(f * 100), f * peak) for f in loads]
    if ref and 0.25 * ref["batched_peak_pairs_s"] < 0.95 * peak:
        points.append(("load_25_of_batched_peak", 0.25 * ref["batched_peak_pairs_s"]))
    for name, offered in points:
        lam = offered / mean_pairs
        count = max(50, int(lam * seconds_per_load))
        arr = np.cumsum(rng.exponential(1.0 / lam, size=count))
        n0 = len(pf.pf_serve_trace(ctx)) if mode == 0 else 0
        st, lat, el = pf.pf_serve_replay(ctx, pool, arr)
        done_pairs = float(sum(sizes[i % len(pool)] for i in range(count)))
        out[name] = {
            "offered_pairs_s": offered, "throughput_pairs_s": done_pairs / el,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "requests": count, "status": int(st)}
        if mode == 0:
            out[name]["batches"] = trace_summary(pf.pf_serve_trace(ctx)[n0:])
    out["stats"] = pf.pf_serve_stats_get(ctx)
    pf.pf_serve_stop(ctx)
    return out


def trace_summary(tr):
    """Per-batch times of a load point (pf_serve_trace): p50 / p99 / max of
    the batch's span (enqueue to completion seen), its wait for uploads, its
    GPU time, and what is left of the span (queued behind the batch before
    it, and the scheduler seeing completion)."""
    if len(tr) == 0:
        return None
    span = (tr[:, 1] - tr[:, 0]) * 1e3
    rest = span - np.maximum(tr[:, 4], 0) - tr[:, 5]
    q = lambda a: [round(float(np.percentile(a, 50)), 3), round(float(np.percentile(a, 99)), 3),
                   round(float(a.max()), 3)]
    return {"count": int(len(tr)), "pairs_p50": float(np.median(tr[:, 2])), "span_ms": q(span),
            "upload_wait_ms": q(tr[:, 4]), "gpu_ms": q(tr[:, 5]), "rest_ms": q(rest)}


def serve_all(pf, seconds_per_load, seed, small_batch=1 << 16):
    """Both serving modes on the same request pool, and the numbers the
    offered loads are stated against.  A context of its own, tuned on a
    resident batch of the serving mix (the batched mode copies its table)."""
    ctx = pf.pf_create(0)
    pf.pf_set_small_batch(ctx, small_batch)
    ref = serve_reference_rates(pf, ctx, seed)
    out = {"reference_rates": ref, "small_batch": small_batch}
    out["batched"] = serve_measure(pf, ctx, seconds_per_load, seed, mode=0, ref=ref)
    out["device_loop"] = serve_measure(pf, ctx, seconds_per_load / 2, seed, mode=1, ref=None)
    pf.pf_destroy(ctx)
    b = out["batched"]
    out["note"] = ("offered loads are fractions of the measured serving peak; the batched "
                   "path's device throughput on the serving mix is %.2fG pairs/s, but the "
                   "requests' ASCII, offsets and thresholds (%.0f bytes per pair) cross a host "
                   "link measured at %.0f GB/s, which bounds any served rate at %.2fG pairs/s "
                   "(the serving peak reached %.0f%% of it), so loads of 50%% and 90%% of the "
                   "batched peak cannot be offered"
                   % (ref["batched_peak_pairs_s"] / 1e9, ref["h2d_bytes_per_pair"],
                      ref["h2d_gbs"], ref["link_bound_pairs_s"] / 1e9,
                      100.0 * b["peak_pairs_s"] / ref["link_bound_pairs_s"]))
    return out


# ---------------------------------------------------------------------------
# the other configurations, compact, on the default line

def filter_ops(lens, E, dec):
    """Integer operations of the method per pair, every word of every pair
    (map 5 D W, GateKeeper 8 D W + W, SneakySnake (E+1)(3D+1), D = 2E+1,
    W = ceil(m/32)), summed over a batch of lengths and thresholds."""
    D = 2 * E.astype(np.int64) + 1
    W = (lens.astype(np.int64) + 31) // 32
    ops = 5 * D * W
    if dec & 2:
        ops = ops + 8 * D * W + W
    if dec & 1:
        ops = ops + (E.astype(np.int64) + 1) * (3 * D + 1)
    return float(ops.sum())


def other_configs(pf, args, rank):
    """Configurations 1, 3 and 4 on one GPU each as a compact row: batched
    (tuned) vs plain filter, the whole step, and the filter's fraction of the
    integer-pipe peak.  Configurations 3 and 4 run a seeded sample of their
    workload (4M and 2M pairs) to keep the run short."""
    import torch
    import synth
    dev = torch.device("cuda", 0)
    ctx = pf.pf_create(0)
    peak = 152 * 64 * 2070.0 * 1e6 / 1e12
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps=5):
        for _ in range(2):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps

    out = {}
    specs = [("cfg1_100bp_E5_100k", synth.UNIFORM, 0x5EED0000, 100_000, 100, 5, 20, 1),
             ("cfg3_mixed_4M_sample_of_50M", synth.MIXED, 0x5EED0003, 4_000_000, 0, 0, 60, 3),
             ("cfg4_250bp_E25_2M_sample_of_10M", synth.SKEWED_ALL, 0x5EED0004, 2_000_000, 250, 25,
              100, 3)]
    for name, kind, seed, n, m, e, kmax, dec in specs:
        P = synth.generate(kind, seed + rank * 7919, n, m=m, E=e, kmax=kmax)
        reads = torch.from_numpy(P.reads).to(dev)
        refs = torch.from_numpy(P.refs).to(dev)
        lens = torch.from_numpy(P.lens).to(dev)
        E = torch.from_numpy(P.E).to(dev)
        Emax = int(P.E.max())
        if m:
            W = (m + 31) // 32
            rd = pf.Seqs.empty(n * W, dev, stride_words=W)
            rf = pf.Seqs.empty(n * W, dev, stride_words=W)
            pack = lambda: (pf.pf_pack_fixed(ctx, reads, n, m, rd),
                            pf.pf_pack_fixed(ctx, refs, n, m, rf))
        else:  # grouped by threshold and length, as the mixed workload's own line
            ws, total = pf.pf_pack_layout_grouped(P.read_off, P.E)
            bo_d = torch.from_numpy(P.read_off).to(dev)
            ws_d = torch.from_numpy(ws).to(dev)
            rd = pf.Seqs.empty(total, dev, word_off=ws_d)
            rf = pf.Seqs.empty(total, dev, word_off=ws_d)
            pack = lambda: (pf.pf_pack_starts(ctx, reads, bo_d, ws_d, rd),
                            pf.pf_pack_starts(ctx, refs, bo_d, ws_d, rf))
        pairs = pf.Pairs(rd, rf)
        pack()
        acc = torch.empty(2 * n, dtype=torch.uint8, device=dev)
        cnt = torch.empty(2 * n, dtype=torch.int16, device=dev)
        dist = torch.empty(n, dtype=torch.int32, device=dev)
        if n >= 1 << 20:
            pf.pf_tune_batch(ctx, 1, pairs, lens, E, Emax, n=n, sample=1 << 19, reps=1)
            pf.pf_tune_batch(ctx, 3, pairs, lens, E, Emax, n=n, sample=1 << 19, reps=1)
        if name.startswith("cfg1"):  # one threshold for the whole batch
            E = None
        ss_b = timed(lambda: pf.pf_filter(ctx, 1, pairs, lens, E, Emax, acc, cnt, n))
        ss_p = timed(lambda: pf.pf_filter_plain(ctx, 1, pairs, lens, E, Emax, acc, cnt, n))
        f_ms = timed(lambda: pf.pf_filter(ctx, dec, pairs, lens, E, Emax, acc, cnt, n))
        if dec == 1:
            step = lambda: (pack(), pf.pf_filter(ctx, 1, pairs, lens, E, Emax, acc, cnt, n))
            what = "pack + SneakySnake"
        else:
            step = lambda: (pack(), pf.pf_filter_verify(ctx, 3, pairs, lens, E, Emax, acc, cnt,
                                                        dist, n))
            what = "pack + filter (both deciders) + compact + verify"
        st_ms = timed(step)
        row = {"pairs": n, "step": what, "step_ms": st_ms, "step_pairs_s": n / (st_ms / 1e3),
               "sneakysnake_batched_pairs_s": n / (ss_b / 1e3),
               "sneakysnake_plain_pairs_s": n / (ss_p / 1e3), "batched_over_plain": ss_p / ss_b,
               "filter_ms": f_ms,
               "filter_frac_of_alu_peak": filter_ops(P.lens, P.E, dec) / (f_ms / 1e3) / 1e12 / peak}
        if dec == 3:
            row["verify_all_ms"] = timed(lambda: pf.pf_verify(ctx, pairs, lens, E, Emax, None, None,
                                                              dist, n))
        out[name] = row
        del reads, refs, rd, rf, pairs, acc, cnt, dist, P
        torch.cuda.empty_cache()
    if not args.no_sweep:
        # configuration 2's sweep of E = 0..15 on 2M-pair samples of its
        # 20M-pair batches (compact: pairs/s only)
        rows = threshold_sweep_rows(pf, ctx, 2_000_000, lambda fn, reps: timed(fn, reps), dev, 5)
        out["cfg2_sweep_2M_samples_of_20M"] = {
            "E": {int(E): {"sneakysnake_batched_pairs_s": r["ss_batched_pairs_s"],
                           "sneakysnake_plain_pairs_s": r["ss_plain_pairs_s"],
                           "batched_over_plain": round(r["batched_over_plain"], 3),
                           "step_pairs_s": r["step_pairs_s"]} for E, r in rows.items()},
            "step": "pack x2 + filter (both deciders) + compact + verify"}
        torch.cuda.empty_cache()
    pf.pf_destroy(ctx)
    return out


# ---------------------------------------------------------------------------
# the other configurations (their own lines; the default line is the
# 150 bp, E = 6 workload above)

def threshold_sweep_rows(pf, ctx, n, timed, dev, reps, emit=None):
    """150 bp pairs at every threshold E = 0..15, one batch of n pairs per E
    (the headline recipe, seed 0x5EED0002 + E): SneakySnake alone batched
    (tuned) vs plain, and the step of both deciders with verification."""
    import torch
    import synth
    W = (M + 31) // 32
    rd = pf.Seqs.empty(n * W, dev, stride_words=W)
    rf = pf.Seqs.empty(n * W, dev, stride_words=W)
    pairs = pf.Pairs(rd, rf)
    lens = torch.full((n,), M, dtype=torch.int32, device=dev)
    acc = torch.empty(2 * n, dtype=torch.uint8, device=dev)
    cnt = torch.empty(2 * n, dtype=torch.int16, device=dev)
    dist = torch.empty(n, dtype=torch.int32, device=dev)
    rows = {}
    for E in range(16):
        P = synth.generate(synth.SKEWED, 0x5EED0002 + E, n, m=M, E=E, kmax=KMAX)
        reads = torch.from_numpy(P.reads).to(dev)
        refs = torch.from_numpy(P.refs).to(dev)
        del P
        Et = torch.full((n,), E, dtype=torch.int16, device=dev)
        pack = lambda: (pf.pf_pack_fixed(ctx, reads, n, M, rd), pf.pf_pack_fixed(ctx, refs, n, M, rf))
        pack()
        tune_n = min(n, 2_000_000)
        t1 = pf.pf_tune(ctx, 1, pairs, lens, E, n=tune_n, reps=2)
        t3 = pf.pf_tune(ctx, 3, pairs, lens, E, n=tune_n, reps=2)
        ss_b = timed(lambda: pf.pf_filter(ctx, 1, pairs, lens, None, E, acc, cnt, n), reps)
        ss_p = timed(lambda: pf.pf_filter_plain(ctx, 1, pairs, lens, None, E, acc, cnt, n), reps)
        step = timed(lambda: (pack(), pf.pf_filter_verify(ctx, 3, pairs, lens, Et, E, acc, cnt,
                                                          dist, n)), reps)
        n_ver = pf.pf_last_verified_count(ctx)
        row = {"E": E, "pairs": n, "ss_batched_pairs_s": n / (ss_b / 1000.0),
               "ss_plain_pairs_s": n / (ss_p / 1000.0), "batched_over_plain": ss_p / ss_b,
               "tuned_cfg_ss": list(t1[:2]), "tuned_cfg_both": list(t3[:2]),
               "step_ms": step, "step_pairs_s": n / (step / 1000.0),
               "accepted_frac": float(acc[:n].float().mean().item()),
               "verified_frac": n_ver / n}
        rows[E] = row
        if emit:
            emit(row)
        del reads, refs
    return rows


def run_threshold_sweep(args, pf, ctx, timed, dev):
    """The sweep of every threshold at the headline size: one JSON line per
    E, then a summary line."""
    n = args.pairs
    rows = threshold_sweep_rows(pf, ctx, n, timed, dev, max(1, args.steps),
                                emit=lambda r: print(json.dumps(r), flush=True))
    print(json.dumps({"workload": "cfg2_sweep", "read_len": M, "pairs_per_E": n,
                      "step": "pack x2 + filter (both deciders) + compact + verify",
                      "rows": rows}), flush=True)
    pf.pf_destroy(ctx)


def run_other_workload(args):
    import torch
    import synth
    import paper_1910_03936_gb300 as pf
    from paper_1910_03936_gb300 import build as pfbuild
    pfbuild.build()
    synth.build()
    dev = torch.device("cuda", 0)
    ctx = pf.pf_create(0)
    stream = torch.cuda.current_stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        for _ in range(args.warmup):
            fn()
        a, b = ev(), ev()
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps

    w = args.workload
    if w == "cfg2_sweep":
        run_threshold_sweep(args, pf, ctx, timed, dev)
        return
    size = args.other_pairs
    if w == "cfg1":   # plain SneakySnake, 100k pairs of 100 bp from ASCII, E = 5
        P = synth.generate(synth.UNIFORM, 0x5EED0000, size or 100_000, m=100, E=5, kmax=20)
        fixed, Emax, kind = 100, 5, "uniform"
    elif w == "cfg3":  # 50M pairs, 100/150/250 bp, E = round(r*len)
        P = synth.generate(synth.MIXED, 0x5EED0003, size or 50_000_000, kmax=60)
        fixed, Emax, kind = None, int(P.E.max()), "mixed"
    else:              # cfg4: 10M pairs of 250 bp, E = 25
        P = synth.generate(synth.SKEWED_ALL, 0x5EED0004, size or 10_000_000, m=250, E=25,
                           kmax=100)
        fixed, Emax, kind = 250, 25, "skewed_all"
    n = P.n
    reads_h = host_copy(pf, P.reads)
    refs_h = host_copy(pf, P.refs)
    reads, refs = reads_h.to(dev), refs_h.to(dev)
    lens = torch.from_numpy(P.lens).to(dev)
    E = torch.from_numpy(P.E).to(dev)
    if fixed:
        W = (fixed + 31) // 32
        rd = pf.Seqs.empty(n * W, dev, stride_words=W)
        rf = pf.Seqs.empty(n * W, dev, stride_words=W)
        pack = lambda: (pf.pf_pack_fixed(ctx, reads, n, fixed, rd),
                        pf.pf_pack_fixed(ctx, refs, n, fixed, rf))
    else:
        # the packed layout grouped by threshold and length: the pairs each
        # bin's launch runs lie together in the planes
        ws, total = pf.pf_pack_layout_grouped(P.read_off, P.E)
        bo_d = torch.from_numpy(P.read_off).to(dev)
        ws_d = torch.from_numpy(ws).to(dev)
        rd = pf.Seqs.empty(total, dev, word_off=ws_d)
        rf = pf.Seqs.empty(total, dev, word_off=ws_d)
        pack = lambda: (pf.pf_pack_starts(ctx, reads, bo_d, ws_d, rd),
                        pf.pf_pack_starts(ctx, refs, bo_d, ws_d, rf))
    pairs = pf.Pairs(rd, rf)
    pack()
    acc = torch.zeros(2 * n, dtype=torch.uint8, device=dev)
    cnt = torch.zeros(2 * n, dtype=torch.int16, device=dev)
    dist = torch.zeros(n, dtype=torch.int32, device=dev)
    out = {"workload": w, "pairs": n, "recipe": kind, "E_max": Emax}
    reps = max(1, args.steps)
    out["pack_ms"] = timed(pack, reps)
    if w == "cfg1":  # one threshold for the whole batch: E passed as a scalar
        out["ss_plain_ms"] = timed(lambda: pf.pf_filter_plain(ctx, 1, pairs, lens, None, 5, acc, cnt, n), reps)
        out["ss_batched_ms"] = timed(lambda: pf.pf_filter(ctx, 1, pairs, lens, None, 5, acc, cnt, n), reps)
        step = lambda: (pack(), pf.pf_filter(ctx, 1, pairs, lens, None, 5, acc, cnt, n))
        out["step"] = "pack + SneakySnake (scheduler: below 2^20 pairs one plain launch, threshold fixed at compile time)"
    else:
        if args.cfg is not None:  # one forced configuration (profiling)
            tpp, dpt, ecap, xe, words = pf.pf_kernel_configs()[args.cfg]
            for e in range(Emax + 1):  # every threshold it serves: one launch
                if (xe == e) or (xe < 0 and e <= ecap):
                    pf.pf_tune_set(ctx, 3, e, args.cfg, args.chunk)
        else:
            # the autotuner on the batch as it is: each threshold timed on up
            # to 1M of its own pairs
            pf.pf_tune_batch(ctx, 3, pairs, lens, E, Emax, n=n, sample=1 << 20, reps=1)
        out["tuned_cfg"] = {int(e): pf.pf_tune_get(ctx, 3, int(e)) for e in np.unique(P.E)}
        if args.stage == "filter_batched":  # the filter alone (profiling)
            out["filter_ms"] = timed(
                lambda: pf.pf_filter(ctx, 3, pairs, lens, E, Emax, acc, cnt, n), reps)
            print(json.dumps(out), flush=True)
            pf.pf_destroy(ctx)
            return
        out["filter_ms"] = timed(lambda: pf.pf_filter(ctx, 3, pairs, lens, E, Emax, acc, cnt, n), reps)
        out["filter_verify_ms"] = timed(
            lambda: pf.pf_filter_verify(ctx, 3, pairs, lens, E, Emax, acc, cnt, dist, n), reps)
        out["verify_all_ms"] = timed(
            lambda: pf.pf_verify(ctx, pairs, lens, E, Emax, None, None, dist, n), reps)
        step = lambda: (pack(), pf.pf_filter_verify(ctx, 3, pairs, lens, E, Emax, acc, cnt, dist, n))
        out["step"] = "pack + batched filter (both deciders) + compact + verify"
    step_ms = timed(step, reps)
    out["ms_per_step"] = step_ms
    out["value"] = n / (step_ms / 1000.0)
    out["unit"] = "pairs/s"
    if w == "cfg3":  # chunked host pipeline, graph replay, pinned host buffers
        import time
        acc_h = host_zeros(pf, 2 * n, torch.uint8).numpy()
        cnt_h = host_zeros(pf, 2 * n, torch.int16).numpy()
        dist_h = host_zeros(pf, n, torch.int32).numpy()
        args_rh = (ctx, 3, reads_h.numpy(), refs_h.numpy(), Emax)
        # offsets and thresholds pinned too: a pageable source makes its
        # upload synchronous and stalls the overlap of the two slots
        off_h = host_copy(pf, P.read_off).numpy()
        E_h = host_copy(pf, P.E).numpy()
        kw = dict(byte_off=off_h, E=E_h, chunk_pairs=1 << 21, out=(acc_h, cnt_h, dist_h))
        pf.pf_run_host(*args_rh, **kw)
        runs = []
        for _ in range(3):
            t = time.perf_counter()
            pf.pf_run_host(*args_rh, **kw)
            runs.append(time.perf_counter() - t)
        out["e2e_host_pipeline_pairs_s"] = n / statistics.median(runs)
        out["e2e_host_pipeline_ms"] = [round(r * 1e3, 2) for r in runs]
    print(json.dumps(out), flush=True)
    pf.pf_destroy(ctx)


# ---------------------------------------------------------------------------
# GPU arm

def main_gpu(args):
    import torch
    import synth
    import paper_1910_03936_gb300 as pf
    from paper_1910_03936_gb300 import build as pfbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pfbuild.build()
    synth.build()

    n = args.pairs
    p0 = shard_start(rank, n)
    # Serving first: its latency tails depend on the host side of the
    # page-locked uploads, which the large page-locked buffers and the host
    # traffic of the measurements below disturb (measured: p99 at 25% load
    # 1.1 ms first in a process, 4.5 ms after the rest of the bench).
    serve = None
    if args.stage == "step" and not args.no_serve and not args.no_extras:
        serve = serve_all(pf, args.serve_seconds, SEED + 5 + rank, args.serve_small_batch)
    t_gen = time.perf_counter()
    P = synth.generate(synth.SKEWED, SEED, n, m=M, E=E_HEAD, kmax=KMAX, p0=p0)
    t_gen = time.perf_counter() - t_gen

    ctx = pf.pf_create(local)
    stream = torch.cuda.current_stream(dev)
    reads_h = host_copy(pf, P.reads)
    refs_h = host_copy(pf, P.refs)
    reads = reads_h.to(dev)
    refs = refs_h.to(dev)
    del P
    W = (M + 31) // 32
    lens = torch.full((n,), M, dtype=torch.int32, device=dev)
    E = torch.full((n,), E_HEAD, dtype=torch.int16, device=dev)
    rd = pf.Seqs.empty(n * W, dev, stride_words=W)
    rf = pf.Seqs.empty(n * W, dev, stride_words=W)
    pairs = pf.Pairs(rd, rf)
    acc = torch.empty(2 * n, dtype=torch.uint8, device=dev)
    cnt = torch.empty(2 * n, dtype=torch.int16, device=dev)
    dist_out = torch.empty(n, dtype=torch.int32, device=dev)
    acc_h = host_zeros(pf, 2 * n, torch.uint8)
    cnt_h = host_zeros(pf, 2 * n, torch.int16)
    dist_h = host_zeros(pf, n, torch.int32)

    # tune the batched kernel for this threshold on a sample of the batch
    pf.pf_pack_fixed(ctx, reads, n, M, rd)
    pf.pf_pack_fixed(ctx, refs, n, M, rf)
    tuned = {}
    if args.cfg is not None:
        for dec in (1, 2, 3):
            pf.pf_tune_set(ctx, dec, E_HEAD, args.cfg, args.chunk)
            tuned[dec] = (args.cfg, args.chunk, None)
    elif not args.no_tune:
        tune_n = min(n, 2_000_000)
        for dec in (1, 3):
            tuned[dec] = pf.pf_tune(ctx, dec, pairs, lens, E_HEAD, n=tune_n, reps=2)
    else:
        for dec in (1, 2, 3):
            c, k = pf.pf_tune_get(ctx, dec, E_HEAD)
            tuned[dec] = (c, k, None)

    ev = lambda: torch.cuda.Event(enable_timing=True)
    stage_names = ("pack", "filter", "compact_verify")

    def step(record=None):
        e = [ev() for _ in range(4)] if record is not None else None
        if e: e[0].record(stream)
        pf.pf_pack_fixed(ctx, reads, n, M, rd)
        pf.pf_pack_fixed(ctx, refs, n, M, rf)
        if e: e[1].record(stream)
        pf.pf_filter_verify(ctx, 3, pairs, lens, E, E_HEAD, acc, cnt, dist_out, n)
        if e: e[3].record(stream)
        if record is not None:
            record.append(e)

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()

    if args.stage == "serve":
        out = serve_all(pf, args.serve_seconds, SEED + 5 + rank, args.serve_small_batch)
        if rank == 0:
            print(json.dumps({"stage": "serve", "serve": out}), flush=True)
        pf.pf_destroy(ctx)
        return
    if args.stage != "step":
        dec = args.deciders
        # one threshold for every pair: no per-pair E array, one kernel launch
        if args.stage in ("filter_plain", "filter_batched"):
            f0 = pf.pf_filter_plain if args.stage == "filter_plain" else pf.pf_filter
            fn = lambda: f0(ctx, dec, pairs, lens, None, E_HEAD, acc, cnt, n)
        elif args.stage == "partitioned":
            fn = lambda: pf.pf_filter_partitioned(ctx, pairs, lens, None, E_HEAD, 8, 2, acc[:n],
                                                  cnt[:n], n)
        elif args.stage == "shouji":
            fn = lambda: pf.pf_filter_shouji(ctx, pairs, lens, None, E_HEAD, acc[:n], cnt[:n], n)
        else:  # shd
            fn = lambda: pf.pf_filter_shd(ctx, pairs, lens, None, E_HEAD,
                                          pf.PF_SHD_VACANT_ZERO | pf.PF_SHD_STREAK, acc[:n],
                                          cnt[:n], n)
        for _ in range(args.warmup):
            fn()
        a0, a1 = ev(), ev()
        a0.record(stream)
        for _ in range(args.steps):
            fn()
        a1.record(stream)
        torch.cuda.synchronize(dev)
        fms = a0.elapsed_time(a1) / args.steps
        if rank == 0:
            print(json.dumps({"stage": args.stage, "deciders": dec, "ms": fms,
                              "pairs_s": n / (fms / 1000.0), "cfg": list(tuned[dec if dec in tuned else 1])}),
                  flush=True)
        pf.pf_destroy(ctx)
        return
    for _ in range(args.warmup):
        step()
    pf.pf_sync(ctx)
    barrier()
    clocks = Clocks(local)
    clocks.start()
    recs = []
    t0, t1 = ev(), ev()
    t0.record(stream)
    for _ in range(args.steps):
        step(recs)
    t1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    pf.pf_sync(ctx)
    ms = max_over_ranks(t0.elapsed_time(t1) / args.steps, dist)
    pack_ms = statistics.mean(r[0].elapsed_time(r[1]) for r in recs)
    fv_ms = statistics.mean(r[1].elapsed_time(r[3]) for r in recs)
    if args.no_extras:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": n * world / (ms / 1000.0),
                              "unit": "pairs/s", "ms_per_step": ms, "pack_ms": pack_ms,
                              "filter_verify_ms": fv_ms, "clocks": clk,
                              "mode": "step only (profiling)"}), flush=True)
        pf.pf_destroy(ctx)
        return

    # per-kernel split of filter vs compact+verify: time them separately
    def timed(fn, reps=args.steps):
        a, b = ev(), ev()
        fn()
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps

    filt_ms = timed(lambda: pf.pf_filter(ctx, 3, pairs, lens, E, E_HEAD, acc, cnt, n))
    idx = torch.empty(n, dtype=torch.int64, device=dev)
    n_idx = torch.empty(1, dtype=torch.int64, device=dev)
    pf.pf_compact(ctx, acc[:n], idx, n_idx, n)
    compact_ms = timed(lambda: pf.pf_compact(ctx, acc[:n], idx, n_idx, n))
    verify_accepted_ms = timed(lambda: pf.pf_verify(ctx, pairs, lens, E, E_HEAD, idx, n_idx,
                                                    dist_out, n))
    n_accepted = int(n_idx.item())
    # The step verifies only the accepted pairs whose SneakySnake count differs
    # from their Hamming distance (the others are resolved by the filter).
    # Rebuild that set here (Hamming distances by torch on the ASCII; N never
    # matches) to time the verification the step runs; its size must equal
    # the library's own count.
    pf.pf_filter_verify(ctx, 3, pairs, lens, E, E_HEAD, acc, cnt, dist_out, n)
    n_verified = pf.pf_last_verified_count(ctx)
    need = torch.empty(n, dtype=torch.uint8, device=dev)
    base = torch.tensor(list(b"ACGT"), dtype=torch.uint8, device=dev)
    for c0 in range(0, n, 1 << 21):
        c1 = min(n, c0 + (1 << 21))
        r = reads[c0 * M:c1 * M].view(-1, M)
        f = refs[c0 * M:c1 * M].view(-1, M)
        ok = torch.isin(r, base) & torch.isin(f, base) & (r == f)
        h = (M - ok.sum(1)).to(torch.int16)
        need[c0:c1] = ((acc[c0:c1] == 1) & (cnt[c0:c1] != h)).to(torch.uint8)
    pf.pf_compact(ctx, need, idx, n_idx, n)
    assert int(n_idx.item()) == n_verified, (int(n_idx.item()), n_verified)
    del need
    verify_ms = timed(lambda: pf.pf_verify(ctx, pairs, lens, E, E_HEAD, idx, n_idx, dist_out, n))
    # the alternative to filtering: the early-exit verifier on every pair
    dist_all = torch.empty(n, dtype=torch.int32, device=dev)
    verify_all_ms = timed(lambda: pf.pf_verify(ctx, pairs, lens, E, E_HEAD, None, None,
                                               dist_all, n))
    del dist_all
    # headline comparison: SneakySnake alone, batched (tuned) vs plain kernel
    ss_batched_ms = timed(lambda: pf.pf_filter(ctx, 1, pairs, lens, E, E_HEAD, acc, cnt, n))
    ss_plain_ms = timed(lambda: pf.pf_filter_plain(ctx, 1, pairs, lens, E, E_HEAD, acc, cnt, n))
    # where the gain comes from: the plain kernel with the threshold fixed at
    # compile time (specialisation alone), the same fused kernel body through
    # the scheduler's persistent launch, and the tuned two-phase form
    ss_plain_exact_ms = timed(lambda: pf.pf_filter_plain_exact(ctx, 1, pairs, lens, E_HEAD, acc,
                                                               cnt, n))
    fused_cfg = [i for i, c in enumerate(pf.pf_kernel_configs())
                 if c[3] == E_HEAD and c[4] == 0][0]
    keep = pf.pf_tune_get(ctx, 1, E_HEAD)
    pf.pf_tune_set(ctx, 1, E_HEAD, fused_cfg, 64)
    ss_fused_ms = timed(lambda: pf.pf_filter(ctx, 1, pairs, lens, None, E_HEAD, acc, cnt, n))
    pf.pf_tune_set(ctx, 1, E_HEAD, keep[0], keep[1])

    # The thesis's other deciders on the same batch: throughput, and accuracy
    # against the exact distances of the step (SneakySnake never rejects a
    # pair within E, so every pair it rejected is beyond E).
    pf.pf_filter_verify(ctx, 3, pairs, lens, E, E_HEAD, acc, cnt, dist_out, n)
    truth = dist_out <= E_HEAD
    n_far = int((~truth).sum().item())

    def accuracy(a):
        a = a.bool()
        return {"accept_frac": a.float().mean().item(),
                "false_accept_rate": int((a & ~truth).sum().item()) / max(n_far, 1),
                "false_rejects": int((truth & ~a).sum().item())}

    variants = {"sneakysnake": accuracy(acc[:n]), "gatekeeper": accuracy(acc[n:2 * n])}
    v_reps = max(3, args.steps // 5)
    for name, fn, extra in (("sneakysnake_t8_y2", pf.pf_filter_partitioned, (8, 2)),
                            ("sneakysnake_t32_y32", pf.pf_filter_partitioned, (32, 32)),
                            ("shouji", pf.pf_filter_shouji, ()),
                            ("gatekeeper_shd", pf.pf_filter_shd,
                             (pf.PF_SHD_VACANT_ZERO | pf.PF_SHD_STREAK,))):
        v_ms = timed(lambda: fn(ctx, pairs, lens, E, E_HEAD, *extra, acc[:n], cnt[:n], n),
                     reps=v_reps)
        variants[name] = dict(accuracy(acc[:n]), pairs_s=n / (v_ms / 1000.0), ms=v_ms)
    variants["sneakysnake"]["pairs_s"] = n / (ss_batched_ms / 1000.0)
    pf.pf_sync(ctx)

    # end to end through the public API: pf_run_host on pinned host ASCII,
    # results into pinned host buffers; chunks of 1M pairs on two slots
    # (upload of one overlapping the device work of the other), each slot's
    # device work replayed as a CUDA graph
    out_bufs = (acc_h.numpy(), cnt_h.numpy(), dist_h.numpy())
    rh, fh = reads_h.numpy(), refs_h.numpy()
    E_h = host_zeros(pf, n, torch.int16).numpy()
    E_h[:] = E_HEAD
    pf.pf_run_host(ctx, 3, rh, fh, E_HEAD, length=M, E=E_h, chunk_pairs=1 << 20, out=out_bufs)
    e2e_steps = max(1, min(args.steps, 3))
    if dist is not None:
        dist.barrier()
    t_e = time.perf_counter()
    for _ in range(e2e_steps):
        pf.pf_run_host(ctx, 3, rh, fh, E_HEAD, length=M, E=E_h, chunk_pairs=1 << 20, out=out_bufs)
    e2e_ms = max_over_ranks((time.perf_counter() - t_e) * 1000.0 / e2e_steps, dist)
    pf.pf_sync(ctx)

    configs = None if args.no_configs else other_configs(pf, args, rank)

    pk, pk_kind = peaks()
    stages = {"pack": pack_ms, "filter": filt_ms, "compact": compact_ms, "verify": verify_ms}
    dominant = max(stages, key=stages.get)
    # Algorithmic work per launch (the per-unit figures of the method): bytes
    # the stage must move, and integer operations of the method counted for
    # every word of every pair (no early exit).
    D, Wd = 2 * E_HEAD + 1, (M + 31) // 32
    ops_filter = 5 * D * Wd + (8 * D * Wd + Wd) + (E_HEAD + 1) * (3 * D + 1)
    alg_bytes = {
        "pack": n * (2 * M + 2 * 3 * M / 8.0),
        "filter": n * (2 * 3 * M / 8.0 + 4 + 2 * 3),
        "compact": n * 1 + n_verified * 8,
        "verify": n_verified * (2 * 3 * M / 8.0 + 4 + 4 + 8),
    }
    alg_ops = {
        "pack": None,
        "filter": n * float(ops_filter),
        "compact": None,
        "verify": n_verified * 20.0 * M,
    }
    # DRAM bytes per launch from one ncu capture of each kernel at 2M pairs
    # (profiles/), scaled to this launch by the units processed; valid for
    # the kernels as captured (the two-phase exact-E6 filter with 5-word
    # arrays that the tuner picks; pack_stream, one launch per 2M sequences,
    # two per pair; verify<u32> on the pairs left after equal bounds)
    traffic_per_pair = {"filter": (248.0896e6 + 10.408448e6) / 2e6,
                        "pack": 2 * (300.054784e6 + 91.782656e6) / 2e6,
                        "verify": (173.886208e6 + 5.08544e6) / 2e6}
    sm_mhz = clk.get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
    alu_peak = 152 * 64 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12  # Top/s, ALU pipe
    ms_dom = stages[dominant]
    hbm_ach = alg_bytes[dominant] / (ms_dom / 1000.0) / 1e9
    if alg_ops[dominant] is not None:
        ach = alg_ops[dominant] / (ms_dom / 1000.0) / 1e12
        roof = {"kernel": dominant, "bound": "alu", "achieved": ach, "peak": alu_peak,
                "unit": "Tops/s", "frac": ach / alu_peak,
                "traffic": (traffic_per_pair[dominant] * n
                            if dominant in traffic_per_pair and M == 150 and E_HEAD == 6 else None),
                "peak_source": "derived: 152 SMs x 64 integer ALU lanes/clk x max SM clock",
                "ops_per_pair": ops_filter if dominant == "filter" else 20 * M,
                "hbm_view": {"achieved_gbs": hbm_ach, "peak_gbs": pk.get("hbm_gbs"),
                             "frac": hbm_ach / pk.get("hbm_gbs"), "peak_source": pk_kind}}
    else:
        roof = {"kernel": dominant, "bound": "hbm", "achieved": hbm_ach,
                "peak": pk.get("hbm_gbs"), "unit": "GB/s", "frac": hbm_ach / pk.get("hbm_gbs"),
                "traffic": None, "peak_source": pk_kind}
    roof["ms_per_launch"] = ms_dom
    roof["sm_mhz_during_step"] = sm_mhz
    if roof["bound"] == "alu":
        # the same peak measured: a LOP3 + funnel-shift loop on every SM
        clk_pk = Clocks(local)
        clk_pk.start()
        pk_ops, pk_ms = pf.pf_peak_int(ctx, 0, 30)
        pk_clk = clk_pk.stop()
        roof["peak_measured"] = pk_ops / 1e12
        roof["frac_of_measured"] = roof["achieved"] / roof["peak_measured"]
        roof["peak_measured_source"] = ("pf_peak_int kind 0 (LOP3 + SHF, full occupancy), "
                                        "%.1f ms per launch x 30, SM clock median %s MHz"
                                        % (pk_ms, pk_clk.get("sm_mhz")))

    total = n * world
    value = total / (ms / 1000.0)
    line = {
        "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": headline_config(n),
        "stages_ms": {"pack": pack_ms, "filter_compact_verify": fv_ms, "filter": filt_ms,
                      "compact": compact_ms, "verify": verify_ms,
                      "verify_every_accepted_pair": verify_accepted_ms,
                      "verify_all_pairs_instead": verify_all_ms},
        "accepted_frac": n_accepted / n,
        "verified_frac": n_verified / n,
        "filter_sneakysnake": {"batched_pairs_s": n / (ss_batched_ms / 1000.0),
                               "plain_pairs_s": n / (ss_plain_ms / 1000.0),
                               "batched_over_plain": ss_plain_ms / ss_batched_ms,
                               "tuned_cfg": list(tuned[1]),
                               "split": {
                                   "plain_runtime_E_ms": ss_plain_ms,
                                   "plain_exact_E_ms": ss_plain_exact_ms,
                                   "scheduler_fused_exact_E_ms": ss_fused_ms,
                                   "scheduler_tuned_two_phase_ms": ss_batched_ms,
                                   "specialisation": ss_plain_ms / ss_plain_exact_ms,
                                   "persistent_launch": ss_plain_exact_ms / ss_fused_ms,
                                   "two_phase": ss_fused_ms / ss_batched_ms}},
        "deciders": variants,
        "configs": configs,
        "roofline": roof,
        "e2e": {"value": total / (e2e_ms / 1000.0), "unit": "pairs/s", "ms_per_step": e2e_ms,
                "call": "pf_run_host (pinned host buffers, 1M-pair chunks, graph replay)",
                "h2d_bytes_per_step": 2 * n * M + 2 * n,
                "d2h_bytes_per_step": n * (2 + 4 + 4)},
        "gpu_launches": None,
        "serve": serve,
        "clocks": clk,
        "gen_s": t_gen,
    }
    # kernels of ours launched per step: 2 pack, binning (init, and with
    # several configurations histogram, scan, scatter), one filter launch per
    # distinct configuration serving E = 0..E_HEAD (a per-pair E array can
    # hold any of them), 3 compaction, 1 verification
    n_cfg = len({pf.pf_tune_get(ctx, 3, e)[0] for e in range(E_HEAD + 1)})
    line["gpu_launches"] = args.steps * (2 + (1 if n_cfg == 1 else 4) + n_cfg + 3 + 1)
    if rank == 0 and world == 1 and not args.no_cpu:
        r, dt, thr = oracle_step_rate(args.cpu_sample)
        r1, dt1, _ = oracle_step_rate(args.cpu_sample_1t, threads=1)
        if roof["bound"] == "alu" and dominant == "filter":
            need, sample = needed_ops_per_pair(args.work_sample)
            roof["ops_per_pair_needed"] = need
            roof["frac_needed"] = n * need / (ms_dom / 1000.0) / 1e12 / roof["peak"]
            roof["needed_sample"] = sample
        line["cpu_baseline"] = {"value": r, "unit": "pairs/s", "cores": thr, "kind": "oracle",
                                "sample": "first %d pairs of the workload (filter both "
                                          "deciders + banded WF on SneakySnake accepts), "
                                          "%.1f s" % (args.cpu_sample, dt),
                                "single_thread": {"value": r1, "unit": "pairs/s", "cores": 1,
                                                  "sample": "first %d pairs, %.1f s"
                                                            % (args.cpu_sample_1t, dt1)}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    pf.pf_destroy(ctx)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--pairs", type=int, default=N_PAIRS)
    ap.add_argument("--other-pairs", type=int, default=None,
                    help="batch size of --workload cfg1/cfg3/cfg4 (default: the "
                         "configuration's own)")
    ap.add_argument("--cpu-sample", type=int, default=8_000_000,
                    help="pairs of the oracle's timed sample for cpu_baseline (about 10 s)")
    ap.add_argument("--cpu-sample-1t", type=int, default=300_000,
                    help="pairs of the single-thread oracle sample (about 5 s)")
    ap.add_argument("--work-sample", type=int, default=200_000,
                    help="pairs of the oracle work-count sample for roofline.frac_needed")
    ap.add_argument("--ref-sample", type=int, default=400_000,
                    help="pairs per step of --impl reference (K + W steps in a few minutes)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the default kernel choice")
    ap.add_argument("--no-extras", action="store_true",
                    help="time the step only (for profiling): no side measurements")
    ap.add_argument("--cfg", type=int, default=None, help="force batch kernel configuration")
    ap.add_argument("--chunk", type=int, default=64)
    ap.add_argument("--stage", default="step",
                    choices=["step", "filter_plain", "filter_batched", "serve", "partitioned",
                             "shouji", "shd"],
                    help="time one filter kernel instead of the step (profiling)")
    ap.add_argument("--deciders", type=int, default=3)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the compact E = 0..15 sweep in the configs block")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the compact rows of configurations 1, 3 and 4")
    ap.add_argument("--workload", default="headline",
                    choices=["headline", "cfg1", "cfg3", "cfg4", "cfg2_sweep"],
                    help="other configurations, each on its own line")
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--serve-small-batch", type=int, default=1 << 16,
                    help="serving batches below this many pairs take the plain kernel")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "headline":
        run_other_workload(args)
    else:
        main_gpu(args)


if __name__ == "__main__":
    main()
