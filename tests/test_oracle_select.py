"""Pins of the oracle's PAC selection (Sec. 4.2 "PAC Selection"; Sec. 3.2
pac_select and the fused pac_select_<cmp>), each against something other
than the oracle's own compare loop:

- the selected worlds of every comparison recomputed from a sort of the 64
  operands and two binary searches (a different algorithm);
- partition identities (LT | GE = mask, LT & GE = 0, EQ = LE & GE, ...);
- IEEE NaN rules written out by hand;
- int64 operands that collide as doubles must still compare exactly;
- selecting and then aggregating equals, world by world, an ordinary
  filtered GROUP BY over the rows of that world (numpy), with rows whose
  selected mask is empty dropped from the group's row count.
"""
import numpy as np
import pytest

import oracle as orc

CMPS = [orc.LT, orc.LE, orc.EQ, orc.NE, orc.GT, orc.GE]
ALL = np.uint64(0xFFFFFFFFFFFFFFFF)


def _bits(worlds) -> int:
    b = 0
    for j in worlds:
        b |= 1 << int(j)
    return b


def _sorted_route(v, thr_row, cmp):
    """Worlds j with v <cmp> thr_row[j], from sorted operands: those below v
    are the first `lo` of the order, those not above v the first `hi`."""
    order = np.argsort(thr_row, kind="stable")
    srt = thr_row[order]
    lo = int(np.searchsorted(srt, v, side="left"))
    hi = int(np.searchsorted(srt, v, side="right"))
    sets = {orc.GT: order[:lo], orc.GE: order[:hi], orc.LT: order[hi:], orc.LE: order[lo:],
            orc.EQ: order[lo:hi]}
    if cmp == orc.NE:
        return ((1 << 64) - 1) ^ _bits(order[lo:hi])
    return _bits(sets[cmp])


@pytest.mark.parametrize("dtype", [np.int64, np.float32, np.float64])
@pytest.mark.parametrize("cmp", CMPS)
def test_select_matches_sorted_operands(dtype, cmp):
    r = np.random.default_rng(cmp * 7 + np.dtype(dtype).itemsize)
    n, n_thr = 600, 5
    # small domain: plenty of ties between the column and the operands
    col = r.integers(-20, 20, n).astype(dtype)
    thr = r.integers(-20, 20, (n_thr, 64)).astype(dtype)
    tid = r.integers(0, n_thr, n).astype(np.uint16)
    got, st = orc.select(np.full(n, ALL), col, cmp, thr, tid)
    assert st == 0
    for i in range(n):
        assert int(got[i]) == _sorted_route(col[i], thr[tid[i]], cmp), (i, cmp)


@pytest.mark.parametrize("dtype", [np.int64, np.float64])
def test_select_partitions_the_mask(dtype):
    r = np.random.default_rng(3)
    n = 2000
    masks = r.integers(0, 2**63, n, dtype=np.int64).astype(np.uint64) * np.uint64(2) + r.integers(0, 2, n).astype(np.uint64)
    col = (r.normal(0, 10, n)).astype(dtype) if dtype == np.float64 else r.integers(-50, 50, n)
    thr = (r.normal(0, 10, 64)).astype(dtype) if dtype == np.float64 else r.integers(-50, 50, 64)
    out = {c: orc.select(masks, col, c, thr)[0] for c in CMPS}
    for o in out.values():
        assert np.all(o & ~masks == 0)                                # only worlds of the row
    assert np.array_equal(out[orc.LT] | out[orc.GE], masks)
    assert np.all(out[orc.LT] & out[orc.GE] == 0)
    assert np.array_equal(out[orc.LE] | out[orc.GT], masks)
    assert np.all(out[orc.LE] & out[orc.GT] == 0)
    assert np.array_equal(out[orc.EQ] | out[orc.NE], masks)
    assert np.array_equal(out[orc.EQ], out[orc.LE] & out[orc.GE])


def test_select_nan_rules():
    """IEEE: every comparison with NaN is false except !=."""
    thr = np.arange(64, dtype=np.float64)
    thr[5] = np.nan
    col = np.array([np.nan, 10.0], dtype=np.float64)
    m = np.full(2, ALL)
    full = (1 << 64) - 1
    expect = {
        orc.LT: [0, _bits(range(11, 64)) & ~(1 << 5)],
        orc.LE: [0, _bits(range(10, 64)) & ~(1 << 5)],
        orc.EQ: [0, 1 << 10],
        orc.NE: [full, full ^ (1 << 10)],
        orc.GT: [0, _bits(range(0, 10)) & ~(1 << 5)],
        orc.GE: [0, _bits(range(0, 11)) & ~(1 << 5)],
    }
    for c, e in expect.items():
        got, st = orc.select(m, col, c, thr)
        assert st == 0 and [int(x) for x in got] == e, c


def test_select_int64_exact_where_doubles_collide():
    """2^62 + 1 and 2^62 are one double; as int64 they must stay apart."""
    big = np.int64(2**62)
    thr = np.full(64, big, dtype=np.int64)
    col = np.array([big + 1, big], dtype=np.int64)
    m = np.full(2, ALL)
    full = (1 << 64) - 1
    assert [int(x) for x in orc.select(m, col, orc.GT, thr)[0]] == [full, 0]
    assert [int(x) for x in orc.select(m, col, orc.EQ, thr)[0]] == [0, full]


def test_select_out_of_range_operand_row():
    thr = np.zeros((2, 64), dtype=np.int64)
    col = np.zeros(3, dtype=np.int64)
    tid = np.array([0, 2, 1], dtype=np.uint8)
    out, st = orc.select(np.full(3, ALL), col, orc.EQ, thr, tid)
    assert st == 1
    assert int(out[1]) == 0 and int(out[0]) == (1 << 64) - 1 and int(out[2]) == (1 << 64) - 1


@pytest.mark.parametrize("cmp", [orc.LT, orc.GE, orc.NE])
def test_select_then_aggregate_is_a_filtered_group_by_per_world(cmp):
    """Sec. 4.2 compiler step (3) then (2): for every world j the PAC SUM and
    COUNT equal an ordinary GROUP BY over the rows with pu[j] = 1 that pass
    the predicate against world j's operand; rows that pass in no world are
    dropped before the aggregate (they count in no group)."""
    r = np.random.default_rng(cmp)
    n, G, n_thr = 3000, 7, 4
    keys = r.integers(0, 800, n).astype(np.int64)
    gids = r.integers(0, G, n).astype(np.uint8)
    vals = r.integers(-1000, 1000, n).astype(np.int64)
    col = r.integers(0, 100, n).astype(np.int64)
    thr = r.integers(0, 100, (n_thr, 64)).astype(np.int64)
    tid = (gids % n_thr).astype(np.uint8)             # the operand vector of the row's part
    qk = orc.query_key(11)
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    sel, st = orc.select(masks, col, cmp, thr, tid)
    assert st == 0
    keep = sel != 0
    cnt, mn, mo, _ = orc.aggregate(sel[keep], None, gids[keep], G, orc.COUNT)
    sm, *_ = orc.aggregate(sel[keep], vals[keep], gids[keep], G, orc.SUM)
    ops = {orc.LT: np.less, orc.GE: np.greater_equal, orc.NE: np.not_equal}[cmp]
    for j in range(64):
        in_world = ((masks >> np.uint64(j)) & np.uint64(1)).astype(bool) & ops(col, thr[tid, j])
        ref_c = np.bincount(gids[in_world], minlength=G)
        ref_s = np.zeros(G, dtype=np.int64)
        np.add.at(ref_s, gids[in_world], vals[in_world])
        assert np.array_equal(cnt[:, j].astype(np.int64), ref_c), j
        assert np.array_equal(sm[:, j], ref_s), j
    assert np.array_equal(mn.astype(np.int64), np.bincount(gids[keep], minlength=G))
