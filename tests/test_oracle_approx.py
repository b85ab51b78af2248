"""Pins for the oracle's approximate SUM/AVG variants (Sec. 5 "Approximation").

Integer sums keep 25 levels of 16-bit counters per world that cascade every 4
bits: a value goes to level l(v) = floor((msb(|v|) - 8) / 4); on overflow a
level adds its counters shifted right by 4 into the next level; negatives go
to a second, negated state (two-sided SUM).  The hand-worked cases below
follow those rules step by step; the statistical checks follow Table 1
(%Err, variance ratio) on synthetic look-alikes of its distributions.
"""
import os

import numpy as np
import pytest

from paper_2603_15023_gb300 import inputs


def _masks(worlds_per_row):
    out = np.zeros(len(worlds_per_row), dtype=np.uint64)
    for i, ws in enumerate(worlds_per_row):
        for j in ws:
            out[i] |= np.uint64(1) << np.uint64(j)
    return out


def test_hand_worked_flush(orc):
    # 15 x 4095, then 4000, then 4095; all at level 0 (msb <= 11).
    # After 16 rows T = 65425; the 17th would make 69520 > 0xFFFF, so level 0
    # flushes first: C1 = C0 >> 4, i.e. 65425 -> 4089 (=65424), 4000 -> 250
    # (=4000), 61425 -> 3839 (=61424); then 4095 goes to level 0.
    vals = np.array([4095] * 15 + [4000, 4095], dtype=np.int64)
    worlds = [[0, 2]] * 15 + [[0, 1], [0, 3]]
    out, st = orc.approx_sum_i64(_masks(worlds), vals, None, 1)
    assert st == 0
    assert out[0, 0] == 65424 + 4095        # exact 69520, one unit lost
    assert out[0, 1] == 4000
    assert out[0, 2] == 61424               # exact 61425
    assert out[0, 3] == 4095
    assert np.all(out[0, 4:] == 0)


def test_hand_worked_routing(orc):
    # v = 2^20 + 2^16 + 5: msb 20 -> level 3, stored as v >> 12 = 272
    v = (1 << 20) + (1 << 16) + 5
    cases = [(v, 272 << 12), (-v, -(272 << 12)), (255, 255), (300, 300),
             (4095, 4095), (4096, 4096), (4097, 4096), (65535, 65520),
             (2**62 + 12345, (2**62 >> 52) << 52)]
    for val, expect in cases:
        out, st = orc.approx_sum_i64(_masks([[5]]), np.array([val], dtype=np.int64), None, 1)
        assert st == 0 and out[0, 5] == expect, (val, out[0, 5], expect)


def test_hand_worked_chunk_combine(orc):
    # chunk 0 (rows 0..4095) leaves 62001 at level 0; chunk 1 adds 4000.
    # Combining: 62001 + 4000 > 0xFFFF -> flush chunk 0's level 0 first:
    # 62001 >> 4 = 3875 (=62000) at level 1, then level 0 takes 4000.
    vals = np.zeros(4097, dtype=np.int64)
    vals[:15] = 4095
    vals[15] = 576
    vals[4096] = 4000
    masks = np.full(4097, np.uint64(1))
    out, st = orc.approx_sum_i64(masks, vals, None, 1)
    assert orc.APX_CHUNK == 4096
    assert st == 0 and out[0, 0] == 66000    # exact 66001


def test_small_values_without_flush_are_exact(orc):
    w = inputs.small(1, 4000, 3, 300, vlo=-15, vhi=15)
    masks = orc.hash_keys(w.keys, orc.query_key(1), orc.BALANCED)
    a, _ = orc.approx_sum_i64(masks, w.values[0], w.gids, 3)
    e, *_ = orc.aggregate(masks, w.values[0], w.gids, 3, orc.SUM)
    np.testing.assert_array_equal(a, e)


DISTS = {
    "uniform_int": lambda r, n: r.integers(-2**31, 2**31, n),
    "uniform_smallint": lambda r, n: r.integers(-2**15, 2**15, n),
    "uniform_bigint_pos": lambda r, n: r.integers(0, 2**40, n),
    "exponential": lambda r, n: np.rint(r.exponential(1e6, n)).astype(np.int64),
    "negative_mixed": lambda r, n: r.integers(-10**6, 10**6, n) - 10**5,
    "decimal_cents": lambda r, n: r.integers(100, 10**7 + 1, n),
}


@pytest.mark.parametrize("dist", sorted(DISTS))
def test_one_sided_error_bound(orc, dist):
    """Per side, 0 <= exact - approx <= 2^-8 * (world's |v|) + 2^-9 * (side's |v|).

    The first term is the truncation when a value is routed to its level
    (it loses less than 2^(4l) of a value >= 2^(8+4l)); the second bounds
    the low 4 bits lost per world at each flush, which needs a level mass of
    at least 0xFFFF - 0xFFF units, summed over cascaded levels and tree
    combines.  Checked on non-negative data (one side) and on the positive
    and negative parts of mixed-sign data separately."""
    r = np.random.default_rng(7)
    n, G = 200000, 2
    v = DISTS[dist](r, n).astype(np.int64)
    keys = r.integers(0, 20000, n).astype(np.int64)
    gids = r.integers(0, G, n).astype(np.uint8)
    masks = orc.hash_keys(keys, orc.query_key(7), orc.BALANCED)
    for sign in (1, -1):
        part = np.where(sign * v > 0, v, 0).astype(np.int64)
        if not np.any(part):
            continue
        a, st = orc.approx_sum_i64(masks, part, gids, G)
        e, *_ = orc.aggregate(masks, part, gids, G, orc.SUM)
        absw, *_ = orc.aggregate(masks, np.abs(part), gids, G, orc.SUM)
        side_tot = np.array([np.abs(part[gids == g]).sum() for g in range(G)], dtype=np.float64)
        err = sign * (e.astype(np.float64) - a.astype(np.float64))
        assert st == 0
        assert np.all(err >= 0)
        bound = absw.astype(np.float64) * 2.0**-8 + side_tot[:, None] * 2.0**-9
        assert np.all(err <= bound)


def _table1():
    rows = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "table1_two_sided.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, pct, z2, ratio = line.split()
                rows[name] = (float(pct), float(z2), float(ratio))
    return rows


# look-alikes of Table 1's named distributions (parameters are ours)
TABLE1_LOOKALIKES = {
    "uniform_int": lambda r, n: r.integers(0, 2**31, n),
    "uniform_smallint": lambda r, n: r.integers(0, 2**15, n),
    "uniform_tinyint": lambda r, n: r.integers(0, 2**7, n),
    "exponential": lambda r, n: np.rint(r.exponential(1e6, n)).astype(np.int64),
}


def _stats(orc, v):
    n = v.shape[0]
    masks = orc.hash_keys(np.arange(n, dtype=np.int64), orc.query_key(11), orc.BALANCED)
    a, _ = orc.approx_sum_i64(masks, v, None, 1)
    e, *_ = orc.aggregate(masks, v, None, 1, orc.SUM)
    a = a[0].astype(np.float64)
    e = e[0].astype(np.float64)
    pct = np.mean(np.abs(a - e) / np.abs(e)) * 100
    z2 = np.mean((a - e) ** 2) / np.var(a)
    return pct, z2, np.var(e) / np.var(a)


@pytest.mark.parametrize("dist", sorted(TABLE1_LOOKALIKES))
def test_table1_statistics(orc, dist):
    """Two-sided %Err within a factor 1.5 of Table 1's, variance ratio near 1."""
    r = np.random.default_rng(11)
    v = TABLE1_LOOKALIKES[dist](r, 1_000_000).astype(np.int64)
    pct, z2, ratio = _stats(orc, v)
    paper_pct = _table1()[dist][0]
    assert paper_pct / 1.5 < pct < paper_pct * 1.5, (pct, paper_pct)
    assert 0.9 < ratio < 1.1, ratio


def test_table1_negative_mixed_two_sided_is_stable(orc):
    # mixed signs: the two-sided state keeps the spread of the 64 sums
    # (variance ratio ~1) and the approximation noise small against it
    r = np.random.default_rng(11)
    v = (r.integers(-10**6, 10**6, 1_000_000) - 10**5).astype(np.int64)
    pct, z2, ratio = _stats(orc, v)
    assert 0.9 < ratio < 1.1 and z2 < 1.0


def test_approx_avg_uses_update_count(orc):
    # AVG = 2 * S_j / n_g with the exact update count n_g (Sec. 5 "Cascading"
    # and the two-sided result 2*(C_pos - C_neg))
    w = inputs.small(2, 30000, 3, 2000, vlo=-3000, vhi=3000)
    masks = orc.hash_keys(w.keys, orc.query_key(2), orc.BALANCED)
    s, _ = orc.approx_sum_i64(masks, w.values[0], w.gids, 3)
    avg, _ = orc.approx_avg_i64(masks, w.values[0], w.gids, 3)
    ng = np.bincount(w.gids, minlength=3).astype(np.float64)
    np.testing.assert_array_equal(avg, 2.0 * s.astype(np.float64) / ng[:, None])


def test_float_state_sum_within_fp32_bound(orc):
    # FLOAT state for DOUBLE sums: |err| <= gamma_n * sum|v|, gamma_n = n u/(1-n u)
    r = np.random.default_rng(3)
    n = 100000
    v = r.lognormal(0.0, 1.5, n)
    masks = orc.hash_keys(np.arange(n, dtype=np.int64), orc.query_key(3), orc.BALANCED)
    a, _ = orc.approx_sum_f32state(masks, v, None, 1)
    e, *_ = orc.aggregate(masks, v, None, 1, orc.SUM)
    u = 2.0**-24
    gam = (n + 1) * u / (1 - (n + 1) * u)
    absw, *_ = orc.aggregate(masks, np.abs(v), None, 1, orc.SUM)
    assert np.all(np.abs(a - e) <= gam * absw)
    assert np.max(np.abs(a - e) / np.abs(e)) > 1e-9   # it really is FP32
