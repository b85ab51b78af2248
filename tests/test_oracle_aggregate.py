"""Pins for the oracle's exact stochastic aggregates.

r_j = agg{ e(t) : t in T, pu[j] = 1 } (Sec. 4.2 "PAC Aggregation") is computed
two independent ways: row by row over the 64 bits (``aggregate``) and world
by world over 64 materialised subsamples joined back to the rows
(``aggregate_brute``, Sec. 4.1 steps (1)-(2) with the hash-coupled SamplePU of
Theorem 2).  Theorem 2 says both give the same answer; the tests also check
closed forms and invariants that hold whatever the code looks like.
"""
import numpy as np
import pytest

from paper_2603_15023_gb300 import inputs

KINDS = ["COUNT", "SUM", "AVG", "MIN", "MAX"]


def _kind(orc, name):
    return getattr(orc, name)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("vdtype", [np.int64, np.float32, np.float64])
@pytest.mark.parametrize("case", range(6))
def test_direct_equals_brute_tiny(orc, mode, vdtype, case):
    rng = np.random.default_rng(100 + case)
    n = int(rng.integers(0, 200))
    n_groups = int(rng.integers(1, 4))
    n_keys = int(rng.integers(1, 40))
    w = inputs.small(case, n, n_groups, n_keys, vdtype=vdtype, vlo=-500, vhi=500)
    if n_groups > 1:
        gids = w.gids.astype(np.uint8)
    else:
        gids = None
    qk = orc.query_key(case)
    masks = orc.hash_keys(w.keys, qk, mode)
    for kname in KINDS:
        kind = _kind(orc, kname)
        vals = None if kind == orc.COUNT else w.values[0]
        a, mn, mo, st1 = orc.aggregate(masks, vals, gids, n_groups, kind)
        b, st2 = orc.aggregate_brute(w.keys, qk, mode, vals, gids, n_groups, kind)
        assert st1 == 0 and st2 == 0
        # same rows in the same order per world: identical, floats included
        np.testing.assert_array_equal(a, b)


def test_direct_equals_brute_with_empty_and_single_key_groups(orc):
    n = 300
    keys = np.repeat(np.arange(10, dtype=np.int64), 30)
    gids = np.zeros(n, dtype=np.uint8)
    gids[:30] = 2            # group 2 holds exactly one PU (key 0)
    gids[30:] = 0            # group 1 is empty
    vals = np.arange(n, dtype=np.int64) - 100
    qk = orc.query_key(7)
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    for kname in KINDS:
        kind = _kind(orc, kname)
        v = None if kind == orc.COUNT else vals
        a, mn, mo, _ = orc.aggregate(masks, v, gids, 3, kind)
        b, _ = orc.aggregate_brute(keys, qk, orc.BALANCED, v, gids, 3, kind)
        np.testing.assert_array_equal(a, b)
        assert np.all(a[1] == 0)             # empty group -> zeros
    c, mn, mo, _ = orc.aggregate(masks, None, gids, 3, orc.COUNT)
    # one PU: its 32 worlds see all 30 rows, the other 32 see none
    assert sorted(set(c[2].tolist())) == [0, 30]
    assert int(mo[2]) == int(masks[0]) and int(mn[2]) == 30 and int(mn[1]) == 0


def test_direct_equals_brute_ungrouped_1m(orc):
    """Full size of the 1M-row ungrouped COUNT+SUM workload."""
    w = inputs.ungrouped_1m(seed=0)
    qk = orc.query_key(0)
    masks = orc.hash_keys(w.keys, qk, orc.BALANCED)
    for kind in (orc.COUNT, orc.SUM):
        v = None if kind == orc.COUNT else w.values[0]
        a, mn, mo, _ = orc.aggregate(masks, v, None, 1, kind)
        b, _ = orc.aggregate_brute(w.keys, qk, orc.BALANCED, v, None, 1, kind)
        np.testing.assert_array_equal(a, b)


def test_invariants_balanced(orc):
    w = inputs.small(3, 50000, 5, 3000, vlo=-10**6, vhi=10**6)
    masks = orc.hash_keys(w.keys, orc.query_key(3), orc.BALANCED)
    c, mn, mo, _ = orc.aggregate(masks, None, w.gids, 5, orc.COUNT)
    s, *_ = orc.aggregate(masks, w.values[0], w.gids, 5, orc.SUM)
    tot = np.array([w.values[0][w.gids == g].sum() for g in range(5)])
    ng = np.bincount(w.gids, minlength=5)
    c = c.astype(np.int64)
    assert np.array_equal(mn.astype(np.int64), ng)
    assert np.all(c.sum(1) == 32 * ng)                  # each row in 32 worlds
    assert np.all(c[:, :32] + c[:, 32:] == ng[:, None])  # complementary worlds
    assert np.all(s[:, :32] + s[:, 32:] == tot[:, None])
    assert np.all(s.sum(1) == 32 * tot)


def test_invariants_raw(orc):
    w = inputs.small(4, 20000, 3, 2000, vlo=0, vhi=10**5)
    masks = orc.hash_keys(w.keys, orc.query_key(4), orc.RAW)
    pc = np.unpackbits(masks.view(np.uint8)).reshape(-1, 64).sum(1).astype(np.int64)
    c, *_ = orc.aggregate(masks, None, w.gids, 3, orc.COUNT)
    s, *_ = orc.aggregate(masks, w.values[0], w.gids, 3, orc.SUM)
    for g in range(3):
        sel = w.gids == g
        assert int(c[g].astype(np.int64).sum()) == int(pc[sel].sum())
        assert int(s[g].sum()) == int((w.values[0][sel] * pc[sel]).sum())


@pytest.mark.parametrize("vdtype", [np.int64, np.float64])
def test_all_ones_mask_is_ordinary_group_by(orc, vdtype):
    # a PU present in every world: each world's result is the ordinary aggregate
    w = inputs.small(5, 5000, 4, 100, vdtype=vdtype, vlo=-1000, vhi=1000)
    masks = np.full(w.n, np.uint64(0xFFFFFFFFFFFFFFFF))
    v = w.values[0]
    for g in range(4):
        sel = w.gids == g
        ref = {
            "COUNT": sel.sum(),
            "SUM": v[sel].sum(),
            "AVG": v[sel].mean(),
            "MIN": v[sel].min(),
            "MAX": v[sel].max(),
        }
        for kname in KINDS:
            kind = _kind(orc, kname)
            out, *_ = orc.aggregate(masks, None if kind == orc.COUNT else v, w.gids, 4, kind)
            if vdtype == np.float64 and kname in ("SUM", "AVG"):
                np.testing.assert_allclose(out[g], ref[kname], rtol=1e-12)
            else:
                assert np.all(out[g] == ref[kname])


def test_single_world_mask(orc):
    # bit j alone: only world j sees the rows
    w = inputs.small(6, 1000, 1, 50, vlo=1, vhi=9)
    for j in (0, 17, 31, 32, 63):
        masks = np.full(w.n, np.uint64(1) << np.uint64(j))
        s, *_ = orc.aggregate(masks, w.values[0], None, 1, orc.SUM)
        exp = np.zeros(64, dtype=np.int64)
        exp[j] = w.values[0].sum()
        np.testing.assert_array_equal(s[0], exp)


def test_avg_min_max_consistency(orc):
    w = inputs.small(8, 20000, 3, 500, vlo=-5000, vhi=5000)
    masks = orc.hash_keys(w.keys, orc.query_key(8), orc.BALANCED)
    c, *_ = orc.aggregate(masks, None, w.gids, 3, orc.COUNT)
    s, *_ = orc.aggregate(masks, w.values[0], w.gids, 3, orc.SUM)
    a, *_ = orc.aggregate(masks, w.values[0], w.gids, 3, orc.AVG)
    lo, *_ = orc.aggregate(masks, w.values[0], w.gids, 3, orc.MIN)
    hi, *_ = orc.aggregate(masks, w.values[0], w.gids, 3, orc.MAX)
    assert np.array_equal(a, s / c.astype(np.float64))
    assert np.all(lo <= a) and np.all(a <= hi)


def test_sum_overflow_is_reported(orc):
    v = np.full(8, 2**62, dtype=np.int64)
    masks = np.full(8, np.uint64(1))
    s, _, _, st = orc.aggregate(masks, v, None, 1, orc.SUM)
    assert st == 4 and s[0, 0] == np.iinfo(np.int64).max


def test_avg_of_an_overflowing_sum_is_the_rounded_exact_quotient(orc):
    """AVG = s_j / c_j on the exact sum even when s_j leaves int64 (reading
    R4): the 128-bit sum rounded once to the nearest double (ties to even),
    then one IEEE division.  Python's integers give the exact sum and its
    int -> float conversion rounds to nearest, ties to even; a sum whose low
    bits sit exactly on a tie and one just past it check the rounding."""
    rng = np.random.default_rng(12)
    n = 40
    masks = rng.integers(0, 2**63, n, dtype=np.int64).astype(np.uint64) * np.uint64(2) + np.uint64(1)
    v = (2**62 + rng.integers(0, 2**20, n)).astype(np.int64)
    v[0] = 2**62 + 2**10          # with 2^62 x 39 others: sums whose 11 low bits decide the rounding
    a, _, _, st = orc.aggregate(masks, v, None, 1, orc.AVG)
    assert st == 0  # AVG itself fits; the SUM of the same worlds overflows
    s, _, _, st_s = orc.aggregate(masks, v, None, 1, orc.SUM)
    assert st_s == 4
    for j in range(64):
        rows = [i for i in range(n) if (int(masks[i]) >> j) & 1]
        if not rows:
            assert a[0, j] == 0.0
            continue
        exact = sum(int(v[i]) for i in rows)
        assert a[0, j] == float(exact) / float(len(rows)), j
    # the conversion itself: 2^63 + 1024 is a tie between 2^63 and 2^63 + 2048
    # (ties to even: 2^63); 2^63 + 1025 rounds up
    ties = np.array([2**62, 2**62 + 1024], dtype=np.int64)
    up = np.array([2**62, 2**62 + 1025], dtype=np.int64)
    one = np.array([np.uint64(1), np.uint64(1)])
    at, *_ = orc.aggregate(one, ties, None, 1, orc.AVG)
    au, *_ = orc.aggregate(one, up, None, 1, orc.AVG)
    assert at[0, 0] == float(2**63) / 2.0 and au[0, 0] == float(2**63 + 2048) / 2.0


def test_single_world_matches_all_worlds(orc):
    w = inputs.small(9, 30000, 4, 2000, vlo=-10**6, vhi=10**6)
    masks = orc.hash_keys(w.keys, orc.query_key(9), orc.RAW)
    for kname in KINDS:
        kind = _kind(orc, kname)
        v = None if kind == orc.COUNT else w.values[0]
        full, *_ = orc.aggregate(masks, v, w.gids, 4, kind)
        for j in (0, 31, 32, 63):
            one, st = orc.aggregate_world(masks, v, w.gids, 4, kind, j)
            assert st == 0
            np.testing.assert_array_equal(one, full[:, j])
