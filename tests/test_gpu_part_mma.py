"""GPU parity of the many-group tensor-core path (agg_path 5): the rows are
partitioned into group order, then aggregated over the group-ordered rows --
groups of more than 32 rows by tcgen05 MMAs, groups of at most 32 rows by one
warp each (also across 32-row block and 512-row chunk edges), groups crossing
a range edge merged from partial records.  The ranges are cut at equal
shares of the rows' cost (a row costs 1, a group of more than 32 rows a fixed
amount more), inside heavy groups and at the starts of mid-size ones.

Bar: bit-exact against the oracle (COUNT, exact int64 SUM, AVG and the
metadata) and against the per-bit engine (agg_path 3), over group-size mixes
(one heavy group across many ranges, Zipf, groups of one to three rows, empty
groups), value magnitudes and signs, key or mask input, both hash modes,
dropped rows, ragged row counts and range edges.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2603_15023_gb300 import binding as B
from paper_2603_15023_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from pac_gpu_util import Ctx
    c = Ctx(0)
    yield c
    c.close()


def _specs(v, avg=True):
    s = [(B.PAC_COUNT, B.PAC_EXACT, None)]
    if v is not None:
        s.append((B.PAC_SUM, B.PAC_EXACT, v))
        if avg:
            s.append((B.PAC_AVG, B.PAC_EXACT, v))
    return s


def _check(ctx, first, gids, G, specs, masks, keep=None, engine=True, want=B.PAC_OK, **kw):
    got, meta, st = ctx.aggregate(first, gids, G, specs, path=5, **kw)
    assert st == want, B.status_name(st)
    assert ctx.last_path == 5
    m_ref = masks if keep is None else masks[keep]
    g_ref = gids if (keep is None or gids is None) else gids[keep]
    for (kind, _, v), g_out in zip(specs, got):
        v_ref = None if v is None else (v if keep is None else v[keep])
        ref, mn, mo, _ = orc.aggregate(m_ref, v_ref, g_ref, G, kind)
        np.testing.assert_array_equal(g_out, ref)
    np.testing.assert_array_equal(meta[:, 0], mn)
    np.testing.assert_array_equal(meta[:, 1], mo)
    if engine:
        got3, meta3, st3 = ctx.aggregate(first, gids, G, specs, path=3, **kw)
        assert st3 == want
        for (kind, _, _), a, b in zip(specs, got, got3):
            if want == B.PAC_OK or kind == B.PAC_COUNT:
                np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(meta, meta3)
    return got, meta


@pytest.mark.parametrize("G", [1, 3, 1000, 50_000])
@pytest.mark.parametrize("n", [1, 37, 511, 513, 4099, 200_003])
def test_part_shapes(ctx, G, n):
    r = np.random.default_rng(7 * G + n)
    keys = r.integers(0, max(n // 2, 1), n).astype(np.int64)
    gids = r.integers(0, G, n).astype(np.int32)
    v = r.integers(100, 10**7, n).astype(np.int64)
    qk = orc.query_key(G + n)
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    _check(ctx, keys, gids, G, _specs(v), masks, qkey=qk)


def test_part_zipf_heavy_groups_across_ranges(ctx):
    # 3M rows: one range per SM (~20K rows' cost each), the top group (~12 %
    # of the rows) spans many ranges, the next ones cross range edges, the
    # tail is tiny
    n = 3_000_017
    G = 100_000
    gids = inputs.zipf_groups(5, 0, n, G)
    r = np.random.default_rng(5)
    keys = r.integers(0, 1_000_000, n).astype(np.int64)
    v = inputs.lognormal_i64(5, 2, n, 8.0, 2.0, 1 << 40)
    qk = orc.query_key(5)
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    _check(ctx, keys, gids, G, _specs(v), masks, qkey=qk)


@pytest.mark.parametrize("mid", [33, 64, 200])
def test_part_cost_balanced_ranges(ctx, mid):
    # one group of 1.5M rows (cut into several ranges inside it), then groups
    # of `mid` rows (each adds a fixed cost: the ranges there hold fewer rows,
    # cut at group starts and inside groups), then 20K groups of 1 to 32 rows
    r = np.random.default_rng(mid)
    sizes = np.concatenate([[1_500_000], np.full(1_200_000 // mid, mid), r.integers(1, 33, 20_000)])
    G = sizes.size
    gids = np.repeat(np.arange(G, dtype=np.int32), sizes)
    r.shuffle(gids)  # the partition restores the group order
    n = gids.size
    keys = r.integers(0, n // 3, n).astype(np.int64)
    v = r.integers(-10**9, 10**9, n).astype(np.int64)
    qk = orc.query_key(mid)
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    _check(ctx, keys, gids, G, _specs(v), masks, qkey=qk)


@pytest.mark.parametrize("rows_per_group", [1, 2, 3, 7, 40])
def test_part_small_groups_and_empty_groups(ctx, rows_per_group):
    # groups of a few rows (one warp each, many across block and chunk
    # edges; 40 rows: tensor cores), every fifth group empty
    n = 100_003
    G = n // rows_per_group + 17
    r = np.random.default_rng(rows_per_group)
    gids = r.integers(0, G, n)
    gids = np.where(gids % 5 == 4, gids - 1, gids).astype(np.int32)
    keys = r.integers(0, 30_000, n).astype(np.int64)
    v = r.integers(-(10**9), 10**9, n).astype(np.int64)
    qk = orc.query_key(rows_per_group)
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    _check(ctx, keys, gids, G, _specs(v), masks, qkey=qk)


def _values(dist, r, n):
    if dist == "small":
        return r.integers(1, 100, n)
    if dist == "big":
        return r.integers(0, 2**40, n)
    if dist == "mixed":
        return r.integers(-(10**12), 10**12, n)
    if dist == "wide":   # all 16 digits, signed, sums still fit int64
        return r.integers(-(2**62), 2**62, n) // max(n, 1)
    if dist == "zeros":
        return np.zeros(n, dtype=np.int64)
    raise ValueError(dist)


@pytest.mark.parametrize("dist", ["small", "big", "mixed", "wide", "zeros"])
def test_part_value_ranges(ctx, dist):
    n = 150_001
    G = 3000
    r = np.random.default_rng(sum(map(ord, dist)))
    gids = np.where(r.random(n) < 0.3, 1, r.integers(0, G, n)).astype(np.int32)
    keys = r.integers(0, 40_000, n).astype(np.int64)
    v = _values(dist, r, n).astype(np.int64)
    qk = orc.query_key(9)
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    _check(ctx, keys, gids, G, _specs(v), masks, qkey=qk)


def test_part_sixteen_digit_values_in_few_runs(ctx):
    # a few values near +-2^60 among small ones: some MMA runs need 16 signed
    # digits while their neighbours need 12
    n = 40_000
    G = 500
    r = np.random.default_rng(21)
    v = r.integers(-50, 50, n).astype(np.int64)
    idx = r.choice(n, 12, replace=False)
    v[idx] = r.integers(-(2**60), 2**60, 12)
    gids = np.sort(r.integers(0, G, n)).astype(np.int32)
    keys = r.integers(0, 3000, n).astype(np.int64)
    qk = orc.query_key(21)
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    _check(ctx, keys, gids, G, _specs(v), masks, qkey=qk)


@pytest.mark.parametrize("in_flags", [B.PAC_IN_KEYS, B.PAC_IN_MASKS])
@pytest.mark.parametrize("mode", [B.PAC_HASH_BALANCED, B.PAC_HASH_RAW])
def test_part_masks_and_raw(ctx, in_flags, mode):
    n = 250_007
    G = 20_000
    r = np.random.default_rng(8)
    keys = r.integers(-(2**60), 2**60, n).astype(np.int64)
    gids = inputs.zipf_groups(8, 0, n, G)
    v = r.integers(-(10**6), 10**6, n).astype(np.int64)
    qk = orc.query_key(8)
    masks = orc.hash_keys(keys, qk, mode)
    first = masks if in_flags == B.PAC_IN_MASKS else keys
    _check(ctx, first, gids, G, _specs(v), masks, in_flags=in_flags, hash_mode=mode, qkey=qk)


def test_part_dropped_rows(ctx):
    # caller masks with PAC_IN_DROP_EMPTY: rows with mask 0 are in no group
    n = 120_001
    G = 7000
    r = np.random.default_rng(3)
    masks = r.integers(0, 2**63, n, dtype=np.int64).astype(np.uint64) * np.uint64(2) + r.integers(0, 2, n).astype(
        np.uint64)
    masks[r.random(n) < 0.05] = 0
    gids = r.integers(0, G, n).astype(np.int32)
    v = r.integers(-1000, 1000, n).astype(np.int64)
    _check(ctx, masks, gids, G, _specs(v), masks, keep=masks != 0,
           in_flags=B.PAC_IN_MASKS | B.PAC_IN_DROP_EMPTY)


def test_part_count_only(ctx):
    n = 90_001
    G = 4000
    r = np.random.default_rng(4)
    keys = r.integers(0, 20_000, n).astype(np.int64)
    gids = r.integers(0, G, n).astype(np.uint16)
    qk = orc.query_key(4)
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    _check(ctx, keys, gids, G, _specs(None), masks, qkey=qk)


def test_part_overflow_reported_avg_exact(ctx):
    """A world SUM beyond int64 is reported; the SUM is saturated and the AVG
    is the exact 128-bit total over the count (the oracle's reading), in
    groups summed by the tensor cores, by the warp and across ranges."""
    n = 200_000
    G = 800
    r = np.random.default_rng(12)
    gids = np.where(r.random(n) < 0.5, 0, r.integers(0, G, n)).astype(np.int32)
    keys = r.integers(0, 50_000, n).astype(np.int64)
    v = (2**62 + r.integers(0, 2**40, n)).astype(np.int64)
    qk = orc.query_key(12)
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    _check(ctx, keys, gids, G, _specs(v), masks, engine=True, want=B.PAC_E_OVERFLOW, qkey=qk)


def test_part_bad_group_ids_skipped_and_reported(ctx):
    n = 60_000
    G = 900
    r = np.random.default_rng(13)
    gids = r.integers(0, G, n).astype(np.int32)
    bad = r.choice(n, 25, replace=False)
    gids[bad] = G + 3
    keys = r.integers(0, 9000, n).astype(np.int64)
    v = r.integers(0, 10**6, n).astype(np.int64)
    qk = orc.query_key(13)
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    keep = gids < G
    got, meta, st = ctx.aggregate(keys, gids, G, _specs(v), qkey=qk, path=5)
    assert st == B.PAC_E_INVALID
    assert ctx.last_path == 5
    for (kind, _, vv), g_out in zip(_specs(v), got):
        ref, mn, mo, _ = orc.aggregate(masks[keep], None if vv is None else vv[keep], gids[keep], G, kind)
        np.testing.assert_array_equal(g_out, ref)
    np.testing.assert_array_equal(meta[:, 0], mn)


def test_part_auto_path(ctx):
    w = inputs.small(2, 50_000, 1000, 5000, vlo=0, vhi=1000)
    ctx.aggregate(w.keys, w.gids, 1000, _specs(w.values[0]))
    assert ctx.last_path == 5
    ctx.aggregate(w.keys, w.gids, 1000, [(B.PAC_MAX, 0, w.values[0])])
    assert ctx.last_path == 3   # MAX: the per-bit engine
    w2 = inputs.small(3, 50_000, 16, 5000, vlo=0, vhi=1000)
    ctx.aggregate(w2.keys, w2.gids, 16, _specs(w2.values[0]))
    assert ctx.last_path == 3   # few groups: the engine's per-warp states, no partition


def test_part_wait_give_up_reports_timeout_then_recovers(ctx):
    """The bounded waits of the many-group kernel on an ordinary launch: with
    the pipeline waits limited to 1 ns they run out before the first bulk
    copies land (nothing is left out; the copies are simply slower than
    that).  Every warp then stops, the loader waits for the copies it issued,
    the MMAs issued are drained, tensor memory is freed and the call reports
    PAC_E_TIMEOUT.  The next call on the same context is bit-exact."""
    n, G = 2_000_003, 50_000
    r = np.random.default_rng(4243)
    gids = inputs.zipf_groups(4243, 0, n, G)
    keys = r.integers(0, 200_000, n).astype(np.int64)
    v = r.integers(-(10**6), 10**6, n).astype(np.int64)
    qk = orc.query_key(4243)
    B.pac_set_option(ctx.h, "wait_limit_ns", 1)
    try:
        _, _, st = ctx.aggregate(keys, gids, G, _specs(v), path=5, qkey=qk)
    finally:
        B.pac_set_option(ctx.h, "wait_limit_ns", 0)
    assert st == B.PAC_E_TIMEOUT, B.status_name(st)
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    _check(ctx, keys, gids, G, _specs(v), masks, engine=False, qkey=qk)
