"""GPU parity of batched queries (pac_batch_plan / pac_batch_launch).

Every query of a mixed batch (row counts from 0 to 10^5, 1 to 5000 groups,
8/16/32-bit group ids, keys or masks, both hash modes, every exact kind over
int64/float32/float64 columns) is checked against the CPU oracle: integers,
MIN/MAX and meta bit-exact, float sums within 1e-6 of the FP64 oracle
relative to the world's sum of |v|.  Released cells are checked against the
oracle's finalize of the batch's own aggregates (NULL/flags bit-exact,
values within 1e-12 relative).  The autotuned plan, a plan captured in a CUDA
graph and replayed, and both state placements (warp-private shared memory
and global atomics) give the same results.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2603_15023_gb300 import binding as B
from paper_2603_15023_gb300 import inputs

pytestmark = pytest.mark.gpu

_VT = {np.dtype(np.int64): B.PAC_I64, np.dtype(np.float32): B.PAC_F32, np.dtype(np.float64): B.PAC_F64}


@pytest.fixture(scope="module")
def ctx():
    h = B.pac_create(0)
    yield h
    B.pac_destroy(h)


def _torch():
    import torch
    return torch


def _out_dtype(kind, vt):
    if kind == B.PAC_COUNT:
        return np.uint64
    if kind == B.PAC_AVG:
        return np.float64
    return np.int64 if vt == B.PAC_I64 else np.float64


class Q:
    """One query: host columns, device copies, specs and outputs."""

    def __init__(self, seed, n, G, gdt, specs_kinds, vdtype, *, masks_in=False, hash_mode=B.PAC_HASH_BALANCED,
                 fin_mode=-1):
        T = _torch()
        w = inputs.small(seed, n, G, max(n // 5, 1), vdtype=vdtype, vlo=-10**6, vhi=10**6)
        self.n, self.G = n, G
        self.gids = None if G == 1 else w.gids.astype(gdt)
        self.qk = orc.query_key(seed)
        self.hash_mode = hash_mode
        self.masks = orc.hash_keys(w.keys, self.qk, hash_mode)
        self.vals = w.values[0]
        first = self.masks.view(np.int64) if masks_in else w.keys
        self.d_first = T.from_numpy(np.ascontiguousarray(first)).cuda()
        self.d_g = T.from_numpy(self.gids).cuda() if self.gids is not None else None
        self.d_v = T.from_numpy(np.ascontiguousarray(self.vals)).cuda()
        vt = _VT[np.dtype(vdtype)]
        self.kinds = specs_kinds
        self.vt = vt
        self.outs = []
        spec_t = []
        for kind in specs_kinds:
            od = _out_dtype(kind, vt)
            t = T.full((G, 64), -7, dtype=T.float64 if od == np.float64 else T.int64, device="cuda")
            self.outs.append((t, od))
            spec_t.append((kind, B.PAC_EXACT, vt, 0 if kind == B.PAC_COUNT else self.d_v.data_ptr(), t.data_ptr()))
        self.specs = B.make_specs(spec_t)
        self.meta = T.full((G, 2), -1, dtype=T.int64, device="cuda")
        nc = G * len(specs_kinds)
        self.noised = T.zeros(nc, dtype=T.float64, device="cuda")
        self.is_null = T.zeros(nc, dtype=T.uint8, device="cuda")
        self.flags = T.zeros(nc, dtype=T.int32, device="cuda")
        self.fin_mode = fin_mode
        self.seed = 77 + seed
        inp = B.make_input(self.d_first.data_ptr(), n, in_flags=B.PAC_IN_MASKS if masks_in else B.PAC_IN_KEYS,
                           hash_mode=hash_mode, query_key=self.qk,
                           group_ids=self.d_g.data_ptr() if self.d_g is not None else 0,
                           gid_bytes=self.gids.dtype.itemsize if self.gids is not None else 0, n_groups=G)
        self.query = B.make_query(inp, self.specs, len(spec_t), meta=self.meta.data_ptr(), fin_mode=fin_mode,
                                  seed=self.seed, budget=1.0 / 64, noised=self.noised.data_ptr(),
                                  is_null=self.is_null.data_ptr(), flags=self.flags.data_ptr())

    def results(self):
        return [t.cpu().numpy().view(od) for t, od in self.outs], self.meta.cpu().numpy().view(np.uint64)

    def release(self):
        return (self.noised.cpu().numpy(), self.is_null.cpu().numpy(), self.flags.cpu().numpy().view(np.uint32))

    def abs_world(self, kind):
        """Per (group, world) sum of |v| (divided by the count for AVG): the
        scale of the float-sum tolerance."""
        absw, *_ = orc.aggregate(self.masks, np.abs(self.vals).astype(np.float64), self.gids, self.G, B.PAC_SUM)
        if kind == B.PAC_AVG:
            cnt, *_ = orc.aggregate(self.masks, None, self.gids, self.G, B.PAC_COUNT)
            absw = absw / np.maximum(cnt.astype(np.float64), 1)
        return absw

    def check(self):
        got, meta = self.results()
        for kind, g_out in zip(self.kinds, got):
            vals = None if kind == B.PAC_COUNT else self.vals
            ref, mn, mo, rst = orc.aggregate(self.masks, vals, self.gids, self.G, kind)
            assert rst == 0
            if vals is not None and vals.dtype != np.int64 and kind in (B.PAC_SUM, B.PAC_AVG):
                absw, *_ = orc.aggregate(self.masks, np.abs(vals).astype(np.float64), self.gids, self.G, B.PAC_SUM)
                if kind == B.PAC_AVG:
                    cnt, *_ = orc.aggregate(self.masks, None, self.gids, self.G, B.PAC_COUNT)
                    absw = absw / np.maximum(cnt.astype(np.float64), 1)
                err = np.abs(g_out - ref)
                assert np.all(err <= 1e-6 * absw + 1e-300), float(np.max(err / np.maximum(absw, 1e-300)))
            else:
                np.testing.assert_array_equal(g_out, ref)
            np.testing.assert_array_equal(meta[:, 0], mn)
            np.testing.assert_array_equal(meta[:, 1], mo)
        if self.fin_mode >= 0:
            y = np.stack([o.astype(np.float64) for o in got], axis=1)
            scales = [orc.release_scale(k) for k in self.kinds]
            ref = orc.finalize(y, scales, meta[:, 0], meta[:, 1], self.seed, 1.0 / 64, self.fin_mode)
            noised, is_null, flags = self.release()
            np.testing.assert_array_equal(is_null, ref["is_null"])
            np.testing.assert_array_equal(flags, ref["flags"])
            live = ref["is_null"] == 0
            np.testing.assert_allclose(noised[live], ref["noised"][live], rtol=1e-12, atol=0)


ALL = [B.PAC_COUNT, B.PAC_SUM, B.PAC_AVG, B.PAC_MIN, B.PAC_MAX]


def _mixed_batch():
    qs = []
    cases = [
        # n, G, gid dtype, kinds, value dtype, extra
        (0, 1, None, [B.PAC_COUNT, B.PAC_SUM], np.int64, {}),
        (1, 1, None, ALL, np.int64, {"fin_mode": B.PAC_FIN_ADAPTIVE}),
        (31, 3, np.uint8, ALL, np.float32, {}),
        (1000, 1, None, [B.PAC_COUNT, B.PAC_SUM], np.int64, {"fin_mode": B.PAC_FIN_ADAPTIVE}),
        (4097, 4, np.uint8, [B.PAC_COUNT, B.PAC_SUM, B.PAC_AVG], np.int64, {"masks_in": True}),
        (70_001, 2, np.uint16, ALL, np.float64, {"fin_mode": B.PAC_FIN_INDEPENDENT}),
        (100_003, 8, np.int32, [B.PAC_COUNT, B.PAC_SUM, B.PAC_SUM], np.float32, {}),
        (33_333, 20, np.uint16, ALL, np.int64, {"hash_mode": B.PAC_HASH_RAW}),
        (50_000, 300, np.int32, [B.PAC_COUNT, B.PAC_SUM, B.PAC_AVG], np.int64, {"fin_mode": B.PAC_FIN_ADAPTIVE}),
        (90_000, 5000, np.int32, ALL, np.float32, {}),
        (12_345, 700, np.int32, [B.PAC_MIN, B.PAC_MAX], np.float64, {}),
        (65_536, 16, np.uint8, [B.PAC_COUNT, B.PAC_SUM], np.float32, {"fin_mode": B.PAC_FIN_ADAPTIVE}),
        (40_000, 900, np.int32, [B.PAC_COUNT, B.PAC_SUM, B.PAC_AVG], np.int64,
         {"fin_mode": B.PAC_FIN_INDEPENDENT}),
    ]
    for i, (n, G, gdt, kinds, vdt, kw) in enumerate(cases):
        qs.append(Q(500 + i, n, G, gdt, kinds, vdt, **kw))
    return qs


def _run(ctx, qs, flags=0):
    T = _torch()
    arr = B.make_queries([q.query for q in qs])
    plan = B.pac_batch_plan(ctx, arr, len(qs), flags)
    try:
        s = T.cuda.current_stream().cuda_stream
        B.pac_batch_launch(ctx, plan, s)
        assert B.pac_sync_status(ctx, s) == B.PAC_OK
        info = {k: B.pac_batch_info(plan, k) for k in ("n_items", "item_rows", "smem_cap", "kernels",
                                                        "n_warp_private", "n_atomic")}
    finally:
        B.pac_batch_free(plan)
    return info


def test_mixed_batch_matches_oracle(ctx):
    qs = _mixed_batch()
    info = _run(ctx, qs)
    assert info["n_warp_private"] > 0 and info["n_atomic"] > 0, info
    assert info["kernels"] == 6   # partition (3) + aggregation + merge + release
    for q in qs:
        q.check()


def test_batch_equals_single_query_calls(ctx):
    """Integer results of a query are the same in a batch and alone."""
    T = _torch()
    qs = _mixed_batch()
    _run(ctx, qs)
    for q in qs:
        if q.vt != B.PAC_I64:
            continue
        got_b, meta_b = q.results()
        s = T.cuda.current_stream().cuda_stream
        B.pac_aggregate_multi(ctx, q.query.in_, q.specs, len(q.kinds), q.meta.data_ptr(), s)
        assert B.pac_sync_status(ctx, s) == B.PAC_OK
        got_s, meta_s = q.results()
        for a, b in zip(got_b, got_s):
            np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(meta_b, meta_s)


def test_autotuned_plan_matches(ctx):
    qs = _mixed_batch()
    info = _run(ctx, qs, flags=B.PAC_BATCH_AUTOTUNE)
    assert info["item_rows"] in (1 << 15, 1 << 17)
    for q in qs:
        q.check()


def test_batch_in_cuda_graph(ctx):
    """A plan's launch captured in a CUDA graph and replayed twice gives the
    results of the plain launch."""
    T = _torch()
    qs = _mixed_batch()
    arr = B.make_queries([q.query for q in qs])
    plan = B.pac_batch_plan(ctx, arr, len(qs), 0)
    try:
        s = T.cuda.Stream()
        with T.cuda.stream(s):
            B.pac_batch_launch(ctx, plan, s.cuda_stream)   # warm (lazy module loading, attributes)
        s.synchronize()
        ref = [q.results() for q in qs]
        rel = [q.release() for q in qs]
        for q in qs:
            for t, _ in q.outs:
                t.fill_(-3)
        g = T.cuda.CUDAGraph()
        with T.cuda.graph(g, stream=s):
            B.pac_batch_launch(ctx, plan, s.cuda_stream)
        for _ in range(2):
            g.replay()
            T.cuda.synchronize()
            assert B.pac_sync_status(ctx, 0) == B.PAC_OK
            for q, (r_out, r_meta), r_rel in zip(qs, ref, rel):
                got, meta = q.results()
                for kind, a, b in zip(q.kinds, got, r_out):
                    if q.vt == B.PAC_I64 or kind in (B.PAC_COUNT, B.PAC_MIN, B.PAC_MAX):
                        np.testing.assert_array_equal(a, b)
                    else:
                        # float sums: rows of a group are summed in scatter order,
                        # so replays agree within the bound, not bit for bit
                        bound = q.abs_world(kind)
                        assert np.all(np.abs(a - b) <= 2e-6 * bound + 1e-300)
                np.testing.assert_array_equal(meta, r_meta)
        for q in qs:
            q.check()
    finally:
        B.pac_batch_free(plan)


def test_many_small_queries(ctx):
    """512 tiny queries (1-300 rows, 1-9 groups): every one right."""
    r = np.random.default_rng(9)
    qs = []
    for i in range(512):
        n = int(r.integers(1, 300))
        G = int(r.integers(1, 10))
        qs.append(Q(10_000 + i, n, G, np.uint8, [B.PAC_COUNT, B.PAC_SUM, B.PAC_MAX], np.int64,
                    fin_mode=B.PAC_FIN_ADAPTIVE if i % 3 == 0 else -1))
    _run(ctx, qs)
    for q in qs[::7]:
        q.check()
    for q in qs:
        got, meta = q.results()
        assert np.all(got[0][:, :32].astype(np.int64) + got[0][:, 32:].astype(np.int64) ==
                      meta[:, 0].astype(np.int64)[:, None])


def test_batch_rejects_bad_queries(ctx):
    import ctypes
    q = Q(1, 100, 1, None, [B.PAC_COUNT], np.int64)
    bad = B.make_specs([(B.PAC_SUM, B.PAC_APPROX, B.PAC_I64, q.d_v.data_ptr(), q.outs[0][0].data_ptr())])
    qq = B.make_query(q.query.in_, bad, 1, meta=q.meta.data_ptr())
    arr = B.make_queries([qq])
    h = ctypes.c_void_p()
    assert B.lib().pac_batch_plan(ctx, arr, 1, 0, ctypes.byref(h)) == B.PAC_E_UNSUPPORTED
    q2 = B.make_query(q.query.in_, q.specs, 1, meta=0, fin_mode=B.PAC_FIN_ADAPTIVE)
    assert B.lib().pac_batch_plan(ctx, B.make_queries([q2]), 1, 0, ctypes.byref(h)) == B.PAC_E_INVALID
    assert B.lib().pac_batch_plan(ctx, arr, 0, 0, ctypes.byref(h)) == B.PAC_E_INVALID


def test_batch_4096_full_size_sampled(ctx):
    """The full batched workload (4096 queries, 4.26G rows generated in HBM)
    in the launch configuration the benchmark times (autotuned plan): sampled
    queries and worlds against the oracle on host-regenerated columns, every
    world of those queries against the balanced invariants."""
    T = _torch()
    from paper_2603_15023_gb300 import batch_inputs
    spec = inputs.batch_4096(seed=0)
    s = T.cuda.Stream()
    db = batch_inputs.DeviceBatch(spec, stream=s.cuda_stream)
    s.synchronize()
    plan = B.pac_batch_plan(ctx, db.queries, db.n_queries, B.PAC_BATCH_AUTOTUNE)
    try:
        B.pac_batch_launch(ctx, plan, s.cuda_stream)
        s.synchronize()
        assert B.pac_sync_status(ctx, s.cuda_stream) == B.PAC_OK
    finally:
        B.pac_batch_free(plan)
    order = np.argsort(spec.rows)
    picks = sorted({int(order[0]), int(order[1]), int(np.argmax(spec.groups)), int(np.argmax(spec.rows)),
                    int(order[len(order) // 2]), 7, 4095})
    for q in picks:
        keys, gids, v, f = spec.columns(q)
        G = int(spec.groups[q])
        masks = orc.hash_keys(keys, db.query_key(q), orc.BALANCED)
        cnt, sm, fs, meta = db.results(q)
        for j in (0, 17, 40, 63):
            c, _ = orc.aggregate_world(masks, None, gids, G, B.PAC_COUNT, j)
            np.testing.assert_array_equal(cnt[:, j], c)
            sj, _ = orc.aggregate_world(masks, v, gids, G, B.PAC_SUM, j)
            np.testing.assert_array_equal(sm[:, j], sj)
            fj, _ = orc.aggregate_world(masks, f, gids, G, B.PAC_SUM, j)
            # float32 values are non-negative: sum |v| of the world = its sum
            assert np.all(np.abs(fs[:, j] - fj) <= 1e-6 * np.abs(fj) + 1e-300)
        ng = np.bincount(gids, minlength=G).astype(np.uint64)
        np.testing.assert_array_equal(meta[:, 0], ng)
        assert np.all(cnt[:, :32].astype(np.int64) + cnt[:, 32:].astype(np.int64) == ng.astype(np.int64)[:, None])
        tot = np.bincount(gids, weights=v.astype(np.float64), minlength=G)
        assert np.all(sm[:, :32] + sm[:, 32:] == np.rint(tot).astype(np.int64)[:, None])
