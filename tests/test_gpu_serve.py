"""GPU tests of the serving loop (pac_serve_*): continuous batching with
memory admission.

Each query's results are the same when it is served in a mix (submitted
from several host threads while other batches run, admitted as memory and
slots free up) as when it runs alone: integer aggregates, MIN/MAX, meta and
the released cells of integer queries bit-exact; float sums within 1e-6
relative to the world's sum of |v| (global float atomics do not fix the
order of additions).  Batches admitted while others run execute at the same
time on the GPU (their aggregation kernels' device-timer spans intersect).
A tight memory budget forces admission in several rounds; an oversized query
is refused.
"""
import threading
import time

import numpy as np
import pytest

from paper_2603_15023_gb300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    h = B.pac_create(0)
    yield h
    B.pac_destroy(h)


def _queries():
    from test_gpu_batch import ALL, Q
    r = np.random.default_rng(123)
    qs = []
    for i in range(48):
        n = int(r.choice([0, 1, 77, 5000, 40_000, 130_000]))
        G = int(r.choice([1, 3, 8, 40, 900]))
        gdt = np.uint8 if G <= 255 else np.int32
        if i % 3 == 0:
            kinds, vdt, fin = [B.PAC_COUNT, B.PAC_SUM, B.PAC_AVG], np.int64, B.PAC_FIN_ADAPTIVE
        elif i % 3 == 1:
            kinds, vdt, fin = ALL, np.float32, -1
        else:
            kinds, vdt, fin = [B.PAC_COUNT, B.PAC_SUM, B.PAC_MIN, B.PAC_MAX], np.float64, -1
        qs.append(Q(20_000 + i, n, G, None if G == 1 else gdt, kinds, vdt, fin_mode=fin))
    return qs


def _snapshot(q):
    got, meta = q.results()
    return got, meta, q.release()


def _reset(q):
    for t, _ in q.outs:
        t.fill_(-5)
    q.meta.fill_(-5)
    q.noised.fill_(-5)


def _same(q, alone, mixed):
    (ga, ma, ra), (gm, mm, rm) = alone, mixed
    for kind, a, m in zip(q.kinds, ga, gm):
        if q.vt == B.PAC_I64 or kind in (B.PAC_COUNT, B.PAC_MIN, B.PAC_MAX):
            np.testing.assert_array_equal(m, a)
        else:
            # each is within 1e-6 of the FP64 oracle (relative to the world's
            # sum of |v|), so the two agree within twice that
            assert np.all(np.abs(m - a) <= 2e-6 * q.abs_world(kind) + 1e-300)
    np.testing.assert_array_equal(mm, ma)
    if q.fin_mode >= 0:
        for x, y in zip(ra, rm):
            np.testing.assert_array_equal(y, x)


def test_served_results_equal_alone(ctx):
    T = __import__("torch")
    qs = _queries()
    alone = []
    s = T.cuda.current_stream().cuda_stream
    for q in qs:
        assert B.pac_batch_run(ctx, B.make_queries([q.query]), 1, s) == B.PAC_OK
        alone.append(_snapshot(q))
        q.check()
        _reset(q)
    T.cuda.synchronize()
    srv = B.pac_serve_create(ctx, mem_budget=1 << 30, max_inflight=16, max_batch=6, n_streams=3)
    try:
        tickets = [None] * len(qs)

        def client(k):
            r = np.random.default_rng(k)
            for i in range(k, len(qs), 4):
                tickets[i] = B.pac_serve_submit(srv, qs[i].query)
                time.sleep(float(r.uniform(0, 0.002)))

        th = [threading.Thread(target=client, args=(k,)) for k in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        lats = []
        for i, tk in enumerate(tickets):
            lat, st = B.pac_serve_wait(srv, tk)
            assert st == B.PAC_OK, (i, B.status_name(st))
            lats.append(lat)
        assert B.pac_serve_stats(srv, "completed") == len(qs)
        assert B.pac_serve_stats(srv, "batches") >= 2
        assert B.pac_serve_stats(srv, "max_inflight_seen") <= 16
        assert B.pac_serve_stats(srv, "p99_ms") >= B.pac_serve_stats(srv, "p50_ms") > 0
        assert all(x > 0 for x in lats)
    finally:
        B.pac_serve_destroy(srv)
    for q, a in zip(qs, alone):
        _same(q, a, _snapshot(q))
        q.check()


def test_batches_overlap_on_the_device(ctx):
    """Continuous batching overlaps work on the device: one query per batch,
    four streams, queries of 2M rows (about 31 work items, so one batch's
    kernel holds a fraction of the SMs for about a millisecond).  The server
    stamps each batch's aggregation kernel with the GPU's global timer (the
    earliest block start and the latest block end) and reports the most
    batches whose kernels were running at one instant; with batches launched
    every few tens of microseconds, at least two must coincide.  Every result
    is still checked against the oracle."""
    from test_gpu_batch import Q
    qs = [Q(50_000 + i, 2_000_000, 8, np.uint8, [B.PAC_COUNT, B.PAC_SUM], np.int64) for i in range(12)]
    srv = B.pac_serve_create(ctx, mem_budget=1 << 30, max_inflight=12, max_batch=1, n_streams=4)
    try:
        tickets = [B.pac_serve_submit(srv, q.query) for q in qs]
        for tk in tickets:
            _, st = B.pac_serve_wait(srv, tk)
            assert st == B.PAC_OK
        assert B.pac_serve_stats(srv, "batches") == len(qs)
        assert B.pac_serve_stats(srv, "max_device_overlap") >= 2
    finally:
        B.pac_serve_destroy(srv)
    for q in qs:
        q.check()


def test_memory_admission_in_rounds(ctx):
    """A budget that holds about two of these plans at once: every query still
    completes, the arena never exceeds the budget, and admission happens in
    many launches."""
    from test_gpu_batch import Q
    qs = [Q(30_000 + i, 60_000, 900, np.int32, [B.PAC_COUNT, B.PAC_SUM], np.int64) for i in range(10)]
    need = 2 * 900 * 64 * 8 + 900 * 8 + 4096      # atomic states + row counts + descriptors, roughly
    budget = 3 * need
    srv = B.pac_serve_create(ctx, mem_budget=budget, max_inflight=64, max_batch=64, n_streams=2)
    try:
        tickets = [B.pac_serve_submit(srv, q.query) for q in qs]
        for tk in tickets:
            _, st = B.pac_serve_wait(srv, tk)
            assert st == B.PAC_OK
        assert B.pac_serve_stats(srv, "arena_high_water") <= budget
        assert B.pac_serve_stats(srv, "batches") >= 4
    finally:
        B.pac_serve_destroy(srv)
    for q in qs:
        q.check()


def test_oversized_and_bad_queries_are_refused(ctx):
    from test_gpu_batch import Q
    q = Q(40_000, 1000, 5000, np.int32, [B.PAC_COUNT, B.PAC_SUM], np.int64)
    srv = B.pac_serve_create(ctx, mem_budget=64 * 1024, max_inflight=4, max_batch=4, n_streams=1)
    try:
        with pytest.raises(B.PacError) as e:
            B.pac_serve_submit(srv, q.query)
        assert e.value.status == B.PAC_E_NOMEM
        bad = B.make_query(q.query.in_, q.specs, 2, meta=0, fin_mode=B.PAC_FIN_ADAPTIVE)
        with pytest.raises(B.PacError) as e:
            B.pac_serve_submit(srv, bad)
        assert e.value.status == B.PAC_E_INVALID
        small = Q(40_001, 100, 1, None, [B.PAC_COUNT], np.int64)
        tk = B.pac_serve_submit(srv, small.query)
        for _ in range(2000):
            done, lat, st = B.pac_serve_poll(srv, tk)
            if done:
                break
            time.sleep(0.001)
        assert done and st == B.PAC_OK and lat > 0
    finally:
        B.pac_serve_destroy(srv)
    small.check()
