"""Pins of the oracle's vector-lifted expressions (Sec. 4.2 "Vector-lifted
Expression, and Lambda Functions") and probabilistic filter (Sec. 3.2
pac_filter), each against something other than the oracle's own stack
machine:

- programs against the same expressions written with numpy array operations
  (IEEE division by zero included);
- malformed programs (underflow, leftovers, missing specs, too deep);
- the Sec. 7 ratio of two SUMs, lifted, against the ratio of ordinary GROUP
  BY sums over each world's explicit subsample (materialised PU sets);
- pac_filter: a fraction of 0 never keeps, 1 always keeps, and over many
  groups the kept share matches the fraction.
"""
import numpy as np
import pytest

import oracle as orc


def _y(seed, G=7, S=3):
    r = np.random.default_rng(seed)
    y = r.integers(-50, 50, (G, S, 64)).astype(np.float64)
    y[0, 1, :5] = 0.0            # division by zero in some worlds
    return y


PROGRAMS = [
    # (program, numpy expression over scaled operands a, b, c)
    ([(orc.L_CONST, 0, 100.0), (orc.L_SPEC, 0, 0), (orc.L_MUL, 0, 0), (orc.L_SPEC, 1, 0), (orc.L_DIV, 0, 0)],
     lambda a, b, c: 100.0 * a / b),
    ([(orc.L_SPEC, 0, 0), (orc.L_SPEC, 1, 0), (orc.L_ADD, 0, 0), (orc.L_SPEC, 2, 0), (orc.L_MUL, 0, 0),
      (orc.L_CONST, 0, 3.5), (orc.L_SUB, 0, 0)],
     lambda a, b, c: (a + b) * c - 3.5),
    ([(orc.L_SPEC, 2, 0), (orc.L_NEG, 0, 0), (orc.L_ABS, 0, 0), (orc.L_SPEC, 0, 0), (orc.L_MIN, 0, 0)],
     lambda a, b, c: np.where(np.abs(c) < a, np.abs(c), a)),
    ([(orc.L_SPEC, 0, 0), (orc.L_SPEC, 1, 0), (orc.L_MAX, 0, 0)],
     lambda a, b, c: np.where(a > b, a, b)),
    ([(orc.L_SPEC, 0, 0), (orc.L_CONST, 0, 0.2), (orc.L_SPEC, 1, 0), (orc.L_MUL, 0, 0), (orc.L_LT, 0, 0)],
     lambda a, b, c: (a < 0.2 * b).astype(np.float64)),
    ([(orc.L_SPEC, 0, 0), (orc.L_SPEC, 1, 0), (orc.L_GE, 0, 0)], lambda a, b, c: (a >= b) * 1.0),
    ([(orc.L_SPEC, 0, 0), (orc.L_SPEC, 1, 0), (orc.L_EQ, 0, 0)], lambda a, b, c: (a == b) * 1.0),
    ([(orc.L_SPEC, 0, 0), (orc.L_SPEC, 1, 0), (orc.L_NE, 0, 0)], lambda a, b, c: (a != b) * 1.0),
    ([(orc.L_SPEC, 0, 0), (orc.L_SPEC, 1, 0), (orc.L_LE, 0, 0)], lambda a, b, c: (a <= b) * 1.0),
    ([(orc.L_SPEC, 0, 0), (orc.L_SPEC, 1, 0), (orc.L_GT, 0, 0)], lambda a, b, c: (a > b) * 1.0),
]


@pytest.mark.parametrize("k", range(len(PROGRAMS)))
def test_lift_matches_numpy(k):
    prog, fn = PROGRAMS[k]
    y = _y(k)
    scales = [2.0, 2.0, 1.0]
    out, st = orc.lift(y, scales, prog)
    assert st == 0
    with np.errstate(divide="ignore", invalid="ignore"):
        ref = fn(2.0 * y[:, 0], 2.0 * y[:, 1], 1.0 * y[:, 2])
    np.testing.assert_array_equal(out, ref)


@pytest.mark.parametrize("prog", [
    [(orc.L_ADD, 0, 0)],                                            # underflow
    [(orc.L_SPEC, 0, 0), (orc.L_SPEC, 1, 0)],                       # two values left
    [(orc.L_SPEC, 5, 0)],                                           # no such spec
    [(orc.L_CONST, 0, 1.0)] * 9 + [(orc.L_ADD, 0, 0)] * 8,          # deeper than 8
    [(99, 0, 0)],                                                   # no such operation
    [],
])
def test_lift_rejects_malformed_programs(prog):
    out, st = orc.lift(_y(1), [1.0, 1.0, 1.0], prog)
    assert st == 1


def test_lifted_ratio_is_the_per_world_ratio_of_subsample_sums():
    """Sec. 7 (TPC-H Q08): share = sum(sales if nation = X) / sum(sales), per
    world, from the 64 unnoised pac_sum vectors.  Each world's ratio equals
    the ratio of two ordinary GROUP BY sums over that world's materialised
    subsample (the release scale 2 cancels)."""
    r = np.random.default_rng(4)
    n, G = 4000, 5
    keys = r.integers(0, 700, n).astype(np.int64)
    gids = r.integers(0, G, n).astype(np.uint8)
    sales = r.integers(1, 10_000, n).astype(np.int64)
    brazil = np.where(r.random(n) < 0.3, sales, 0).astype(np.int64)
    qk = orc.query_key(8)
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    s_b, *_ = orc.aggregate(masks, brazil, gids, G, orc.SUM)
    s_a, *_ = orc.aggregate(masks, sales, gids, G, orc.SUM)
    y = np.stack([s_b, s_a], axis=1).astype(np.float64)
    prog = [(orc.L_SPEC, 0, 0), (orc.L_SPEC, 1, 0), (orc.L_DIV, 0, 0)]
    out, st = orc.lift(y, [orc.release_scale(orc.SUM)] * 2, prog)
    assert st == 0
    b_brute, _ = orc.aggregate_brute(keys, qk, orc.BALANCED, brazil, gids, G, orc.SUM)
    a_brute, _ = orc.aggregate_brute(keys, qk, orc.BALANCED, sales, gids, G, orc.SUM)
    np.testing.assert_array_equal(out, b_brute.astype(np.float64) / a_brute.astype(np.float64))


def test_filter_extremes_and_frequency():
    G = 40_000
    none = np.zeros((G, 64))
    assert orc.pac_filter(none, 1).sum() == 0
    everyone = np.ones((G, 64))
    assert orc.pac_filter(everyone, 1).sum() == G
    quarter = np.zeros((G, 64))
    quarter[:, ::4] = 1.0                                    # 16 of 64 worlds true
    k = orc.pac_filter(quarter, 3).astype(np.float64)
    sd = np.sqrt(0.25 * 0.75 / G)
    assert abs(k.mean() - 0.25) < 5 * sd
    # the same seed gives the same choices; the choice ignores which worlds are true
    shifted = np.roll(quarter, 1, axis=1)
    np.testing.assert_array_equal(orc.pac_filter(quarter, 3), orc.pac_filter(shifted, 3))
    assert orc.pac_filter(quarter, 4).tolist() != k.astype(np.uint8).tolist()
