"""Serving (continuous batching) through the C ABI, in both modes: device
batches running the tuned path (PF_SERVE_BATCHED) and the device-resident
loop (PF_SERVE_DEVICE_LOOP).

Results must be bit-exact with the oracle, identical for a request served
alone and in a mix of concurrent requests, correct when the memory budget
admits one request at a time (device loop) or splits requests across
batches (batched); malformed requests are refused on the host; waits are
bounded (timeouts, cancellation on stop, the device loop leaving when idle
and coming back on demand).
"""
import threading
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    from paper_1910_03936_gb300 import build
    build.build()
    import paper_1910_03936_gb300 as m
    return m


@pytest.fixture
def ctx(pf):
    c = pf.pf_create(0)
    yield c
    pf.pf_destroy(c)


MODES = [0, 1]   # PF_SERVE_BATCHED, PF_SERVE_DEVICE_LOOP


def make_request(pf, seed, n, deciders=3, p0=0, pinned=False):
    P = synth.generate(synth.SERVE, seed, n, kmax=60, p0=p0)
    return P, pf.Request(deciders, P.reads, P.refs, P.read_off, P.E, pinned=pinned)


def expected(P, deciders):
    acc, cnt = oracle.filter_batch(P, deciders=deciders)
    vb = oracle.verify_batch(P)
    dist = np.where(acc[0] == 1, vb, P.E.astype(np.int32) + 1)
    return acc.reshape(-1), cnt.reshape(-1), dist


def check(P, R, deciders):
    a, c, d = expected(P, deciders)
    assert np.array_equal(R.count[:len(c)], c)
    assert np.array_equal(R.accept[:len(a)], a)
    assert np.array_equal(R.dist[:P.n], d)


@pytest.mark.parametrize("mode", MODES)
def test_requests_bit_exact(pf, ctx, mode):
    pf.pf_serve_start(ctx, chunk_pairs=512, mode=mode)
    reqs = [make_request(pf, 100 + i, n, deciders=d)
            for i, (n, d) in enumerate([(1000, 3), (5000, 1), (777, 2), (20000, 3), (1, 3), (0, 3)])]
    for _, R in reqs:
        pf.pf_submit(ctx, R)
    for P, R in reqs:
        st, lat = pf.pf_wait(ctx, R.ticket, 60000)
        assert st == 0 and lat > 0
        check(P, R, R.deciders)
    stats = pf.pf_serve_stats_get(ctx)
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    pf.pf_serve_stop(ctx)


@pytest.mark.parametrize("mode", MODES)
def test_alone_and_in_the_mix_are_identical(pf, ctx, mode):
    pf.pf_serve_start(ctx, chunk_pairs=256, mode=mode)
    P, alone = make_request(pf, 7, 6000)
    pf.pf_submit(ctx, alone)
    assert pf.pf_wait(ctx, alone.ticket, 60000)[0] == 0
    others = [make_request(pf, 1000 + i, int(n))[1]
              for i, n in enumerate(np.random.default_rng(3).integers(1000, 30000, 24))]
    _, mixed = make_request(pf, 7, 6000)
    for i, R in enumerate(others):
        pf.pf_submit(ctx, R)
        if i == len(others) // 2:
            pf.pf_submit(ctx, mixed)   # arrives while the others are on the GPU
    assert pf.pf_wait(ctx, mixed.ticket, 60000)[0] == 0
    for R in others:
        assert pf.pf_wait(ctx, R.ticket, 60000)[0] == 0
    assert np.array_equal(alone.accept, mixed.accept)
    assert np.array_equal(alone.count, mixed.count)
    assert np.array_equal(alone.dist, mixed.dist)
    check(P, mixed, 3)
    pf.pf_serve_stop(ctx)


@pytest.mark.parametrize("mode", MODES)
def test_budget_admits_one_request_at_a_time(pf, ctx, mode):
    # device loop: room for two 20k-pair requests at most, the others wait
    # for memory; batched: batches of about 15k pairs, so every request is
    # split across two or three of them
    pf.pf_serve_start(ctx, hbm_budget=24 << 20, max_requests=8, chunk_pairs=1024, mode=mode)
    reqs = [make_request(pf, 300 + i, 20000) for i in range(5)]
    for _, R in reqs:
        pf.pf_submit(ctx, R)
    for P, R in reqs:
        assert pf.pf_wait(ctx, R.ticket, 120000)[0] == 0
        check(P, R, 3)
    pf.pf_serve_stop(ctx)


@pytest.mark.parametrize("mode", MODES)
def test_malformed_requests_are_refused(pf, ctx, mode):
    pf.pf_serve_start(ctx, hbm_budget=8 << 20, mode=mode)
    P, R = make_request(pf, 5, 100)
    bad_E = pf.Request(3, P.reads, P.refs, P.read_off, np.full(100, 40, np.int16))
    with pytest.raises(pf.PFError) as ei:
        pf.pf_submit(ctx, bad_E)
    assert ei.value.status == 1
    off = P.read_off.copy()
    off[50] = off[49] - 1
    bad_off = pf.Request(3, P.reads, P.refs, off, P.E)
    with pytest.raises(pf.PFError) as ei:
        pf.pf_submit(ctx, bad_off)
    assert ei.value.status == 1
    P2, big = make_request(pf, 6, 100000)
    if mode == 1:                              # cannot fit 8 MiB whole
        with pytest.raises(pf.PFError) as ei:
            pf.pf_submit(ctx, big)
        assert ei.value.status == 2
    else:                                      # streams through the batches
        pf.pf_submit(ctx, big)
        assert pf.pf_wait(ctx, big.ticket, 120000)[0] == 0
        check(P2, big, 3)
    pf.pf_submit(ctx, R)                       # the serving loop is unaffected
    assert pf.pf_wait(ctx, R.ticket, 60000)[0] == 0
    check(P, R, 3)
    pf.pf_serve_stop(ctx)


@pytest.mark.parametrize("mode", MODES)
def test_invalid_bytes_report_edata(pf, ctx, mode):
    # paused, so that the bad request and a good one share a batch: the
    # error belongs to the request whose bytes carried it
    pf.pf_serve_start(ctx, mode=mode, start_paused=True)
    P, _ = make_request(pf, 8, 500)
    reads = P.reads.copy()
    reads[10] = ord("X")
    R = pf.Request(3, reads, P.refs, P.read_off, P.E)
    P2, good = make_request(pf, 12, 700)
    pf.pf_submit(ctx, R)
    pf.pf_submit(ctx, good)
    time.sleep(0.05)
    pf.pf_serve_resume(ctx)
    assert pf.pf_wait(ctx, R.ticket, 60000)[0] == 7
    assert pf.pf_wait(ctx, good.ticket, 60000)[0] == 0
    check(P2, good, 3)
    pf.pf_serve_stop(ctx)


@pytest.mark.parametrize("mode", MODES)
def test_paused_wait_times_out_and_stop_cancels(pf, ctx, mode):
    pf.pf_serve_start(ctx, start_paused=True, mode=mode)
    P, R = make_request(pf, 9, 3000)
    pf.pf_submit(ctx, R)
    st, _ = pf.pf_wait(ctx, R.ticket, 200)
    assert st == 4                       # PF_ETIMEOUT: nothing runs while paused
    assert not pf.pf_poll(ctx, R.ticket)
    result = {}
    t = threading.Thread(target=lambda: result.update(st=pf.pf_wait(ctx, R.ticket, -1)[0]))
    t.start()
    time.sleep(0.1)
    pf.pf_serve_stop(ctx)                # the waiter wakes with PF_ECANCELLED
    t.join(10)
    assert not t.is_alive() and result["st"] == 6


def test_device_loop_leaves_when_idle_and_returns(pf, ctx):
    pf.pf_serve_start(ctx, idle_exit_us=1000, mode=1)
    P1, R1 = make_request(pf, 10, 2000)
    pf.pf_submit(ctx, R1)
    assert pf.pf_wait(ctx, R1.ticket, 60000)[0] == 0
    time.sleep(0.2)                      # far beyond the loop's 1 ms idle bound
    P2, R2 = make_request(pf, 11, 2000)
    pf.pf_submit(ctx, R2)
    assert pf.pf_wait(ctx, R2.ticket, 60000)[0] == 0
    check(P1, R1, 3)
    check(P2, R2, 3)
    assert pf.pf_serve_stats_get(ctx)["loop_launches"] >= 2
    pf.pf_serve_stop(ctx)


@pytest.mark.parametrize("mode", MODES)
def test_replay_open_loop_load(pf, ctx, mode):
    pf.pf_serve_start(ctx, mode=mode)
    pool = [make_request(pf, 400 + i, n) for i, n in enumerate((1000, 4000, 12000))]
    arrivals = np.cumsum(np.random.default_rng(1).exponential(0.002, size=30))
    st, lat, el = pf.pf_serve_replay(ctx, [R for _, R in pool], arrivals)
    assert st == 0 and np.all(lat > 0) and el >= arrivals[-1]
    for P, R in pool:
        check(P, R, 3)
    pf.pf_serve_stop(ctx)


# ---- batched mode ------------------------------------------------------------

@pytest.mark.parametrize("pinned", [False, True])
def test_batched_splits_requests_and_mixes_deciders(pf, ctx, pinned):
    # batches of 1,000 pairs at most: every request below is split across
    # several batches, and the decider sets 1, 2 and 3 share batches
    pf.pf_serve_start(ctx, mode=0, batch_pairs=1000, start_paused=True)
    reqs = [make_request(pf, 500 + i, n, deciders=d, pinned=pinned)
            for i, (n, d) in enumerate([(2500, 3), (700, 2), (1, 1), (3001, 1), (999, 2),
                                        (1000, 3), (0, 3), (4321, 2)])]
    for _, R in reqs:
        pf.pf_submit(ctx, R)
    pf.pf_serve_resume(ctx)
    for P, R in reqs:
        assert pf.pf_wait(ctx, R.ticket, 60000)[0] == 0
        check(P, R, R.deciders)
    assert pf.pf_serve_stats_get(ctx)["loop_launches"] >= 13
    pf.pf_serve_stop(ctx)


def test_batched_pinned_and_pageable_agree(pf, ctx):
    pf.pf_serve_start(ctx, mode=0)
    P, a = make_request(pf, 77, 9000, pinned=True)
    _, b = make_request(pf, 77, 9000, pinned=False)
    pf.pf_submit(ctx, a)
    pf.pf_submit(ctx, b)
    assert pf.pf_wait(ctx, a.ticket, 60000)[0] == 0
    assert pf.pf_wait(ctx, b.ticket, 60000)[0] == 0
    for x, y in ((a.accept, b.accept), (a.count, b.count), (a.dist, b.dist)):
        assert np.array_equal(x, y)
    check(P, a, 3)
    pf.pf_serve_stop(ctx)


def test_batched_uses_the_serving_contexts_tuning(pf, ctx):
    # the plain kernel below the small-batch size, the scheduler above it:
    # both give the oracle's results
    for small in (0, 1 << 30):
        pf.pf_set_small_batch(ctx, small)
        pf.pf_serve_start(ctx, mode=0)
        P, R = make_request(pf, 90, 5000)
        pf.pf_submit(ctx, R)
        assert pf.pf_wait(ctx, R.ticket, 60000)[0] == 0
        check(P, R, 3)
        pf.pf_serve_stop(ctx)


def test_batched_trace_accounts_for_every_pair(pf, ctx):
    pf.pf_serve_start(ctx, mode=0, batch_pairs=3000)
    reqs = [make_request(pf, 600 + i, n, pinned=True) for i, n in enumerate((4000, 1500, 9000))]
    for _, R in reqs:
        pf.pf_submit(ctx, R)
    for P, R in reqs:
        assert pf.pf_wait(ctx, R.ticket, 60000)[0] == 0
        check(P, R, 3)
    tr = pf.pf_serve_trace(ctx)
    total = sum(P.n for P, _ in reqs)
    assert len(tr) >= total // 3000 and tr[:, 2].sum() == total
    assert (tr[:, 2] <= 3000).all() and (tr[:, 3] >= 1).all()
    assert (tr[:, 1] >= tr[:, 0]).all() and (tr[:, 5] > 0).all()
    assert (tr[:, 8:13] >= 0).all() and (tr[:, 7] == 3).all()
    st = pf.pf_serve_stats_get(ctx)
    assert st["batch_pairs"] == total and st["loop_launches"] == len(tr)
    pf.pf_serve_stop(ctx)
    with pytest.raises(pf.PFError):
        pf.pf_serve_trace(ctx)           # not serving
    pf.pf_serve_start(ctx, mode=1)
    with pytest.raises(pf.PFError):
        pf.pf_serve_trace(ctx)           # the device loop keeps no batch trace
    pf.pf_serve_stop(ctx)
