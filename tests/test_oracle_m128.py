"""Pins for the oracle's m = 128 worlds (Sec. 2 says m = 128 is possible; the
paper runs 64).  Reading R7 of the oracle fixes the hash, the release and
their constants.  Each function is checked against something other than its
own code:

- the mask: exactly 64 of 128 worlds under balanced hashing, world j+64 the
  complement of world j, the two words independent, bit frequencies 1/2, and
  worlds 0..31 equal to those of the 64-world mask under the same key;
- aggregation: row by row against 128 materialised subsamples (Sec. 4.1
  steps (1)-(2), Theorem 2), the balanced invariants, an all-worlds mask
  against an ordinary GROUP BY;
- release: the secret world uniform over 128, the NULL rate
  (128 - popcount)/128, zero variance releasing the exact value, the noise
  of the first cell N(0, Var(y)/(2B)) with Var from numpy, and the first
  posterior update against a numpy softmax.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2603_15023_gb300 import inputs

KINDS = [orc.COUNT, orc.SUM, orc.AVG, orc.MIN, orc.MAX]


def _bits(m2):
    """[n, 2] words -> [n, 128] 0/1 matrix (world j: bit j % 64 of word j // 64)."""
    m2 = np.asarray(m2, dtype=np.uint64)
    j = np.arange(64, dtype=np.uint64)
    lo = (m2[:, :1] >> j) & np.uint64(1)
    hi = (m2[:, 1:2] >> j) & np.uint64(1)
    return np.concatenate([lo, hi], axis=1).astype(np.int64)


def test_keys_differ_and_masks_are_balanced():
    k1, k2 = orc.query_key(5), orc.query_key2(5)
    assert k1 != k2 and orc.query_key2(6) != k2
    keys = np.arange(-5000, 5000, dtype=np.int64) * 7919
    b = _bits(orc.hash_keys128(keys, k1, k2, orc.BALANCED))
    assert np.all(b.sum(axis=1) == 64)
    assert np.all(b[:, :64] + b[:, 64:] == 1)
    freq = b[:, :64].mean(axis=0)
    sd = np.sqrt(0.25 / len(keys))
    assert np.all(np.abs(freq - 0.5) < 5 * sd)
    # the two 32-world halves come from different keyed hashes: uncorrelated
    c = np.corrcoef(b[:, :32].sum(axis=1), b[:, 32:64].sum(axis=1))[0, 1]
    assert abs(c) < 5 / np.sqrt(len(keys))
    # worlds 0..31 are the 64-world mask's worlds 0..31 under the same key
    m64 = orc.hash_keys(keys, k1, orc.BALANCED)
    np.testing.assert_array_equal(b[:, :32], ((m64[:, None] >> np.arange(32, dtype=np.uint64)) & np.uint64(1)).astype(np.int64))


def test_raw_masks_are_two_independent_hashes():
    k1, k2 = orc.query_key(8), orc.query_key2(8)
    keys = np.arange(20000, dtype=np.int64)
    r = orc.hash_keys128(keys, k1, k2, orc.RAW)
    np.testing.assert_array_equal(r[:, 0], orc.hash_keys(keys, k1, orc.RAW))
    np.testing.assert_array_equal(r[:, 1], orc.hash_keys(keys, k2, orc.RAW))
    pop = _bits(r).sum(axis=1)
    assert abs(pop.mean() - 64) < 5 * np.sqrt(32 / len(keys))


@pytest.mark.parametrize("mode", [orc.BALANCED, orc.RAW])
@pytest.mark.parametrize("vdtype", [np.int64, np.float64])
@pytest.mark.parametrize("case", range(4))
def test_direct_equals_brute(mode, vdtype, case):
    rng = np.random.default_rng(300 + case)
    n = int(rng.integers(1, 150))
    G = int(rng.integers(1, 4))
    w = inputs.small(case + 50, n, G, int(rng.integers(1, 30)), vdtype=vdtype, vlo=-500, vhi=500)
    k1, k2 = orc.query_key(case), orc.query_key2(case)
    m2 = orc.hash_keys128(w.keys, k1, k2, mode)
    for kind in KINDS:
        v = None if kind == orc.COUNT else w.values[0]
        direct, mn, mo, st = orc.aggregate128(m2, v, w.gids, G, kind)
        brute, st2 = orc.aggregate_brute128(w.keys, k1, k2, mode, v, w.gids, G, kind)
        assert st == 0 and st2 == 0
        np.testing.assert_array_equal(direct, brute)
        gid = np.zeros(n, dtype=np.int64) if w.gids is None else w.gids.astype(np.int64)
        np.testing.assert_array_equal(mn, np.bincount(gid, minlength=G))


def test_balanced_invariants_and_all_worlds_mask():
    w = inputs.small(77, 20000, 5, 3000, vlo=-10**6, vhi=10**6)
    k1, k2 = orc.query_key(77), orc.query_key2(77)
    m2 = orc.hash_keys128(w.keys, k1, k2, orc.BALANCED)
    c, mn, mo, _ = orc.aggregate128(m2, None, w.gids, 5, orc.COUNT)
    s, *_ = orc.aggregate128(m2, w.values[0], w.gids, 5, orc.SUM)
    gid = w.gids.astype(np.int64)
    tot = np.array([w.values[0][gid == g].sum() for g in range(5)])
    assert np.all(c[:, :64].astype(np.int64) + c[:, 64:].astype(np.int64) == mn.astype(np.int64)[:, None])
    assert np.all(s[:, :64] + s[:, 64:] == tot[:, None])
    ones = np.full((w.n, 2), np.uint64(0xFFFFFFFFFFFFFFFF))
    for kind in KINDS:
        v = None if kind == orc.COUNT else w.values[0]
        a, *_ = orc.aggregate128(ones, v, w.gids, 5, kind)
        ref, *_ = orc.aggregate(np.full(w.n, np.uint64(0xFFFFFFFFFFFFFFFF)), v, w.gids, 5, kind)
        np.testing.assert_array_equal(a, np.concatenate([ref, ref], axis=1))


def test_secret_world_is_uniform_over_128():
    y = np.zeros((1, 1, 128))
    full = np.array([[np.uint64(0xFFFFFFFFFFFFFFFF)] * 2], dtype=np.uint64)
    js = np.array([orc.finalize128(y, [1.0], [1], full, seed, 0.01)["jstar"] for seed in range(6400)])
    counts = np.bincount(js, minlength=128)
    assert counts.shape == (128,) and counts.min() > 0
    chi2 = ((counts - 50.0) ** 2 / 50.0).sum()
    assert chi2 < 127 + 6 * np.sqrt(2 * 127)


def test_null_rate_follows_the_or_mask():
    # worlds 0..95 updated: NULL with probability 32/128
    orm = np.array([[np.uint64(0xFFFFFFFFFFFFFFFF), np.uint64(0xFFFFFFFF)]], dtype=np.uint64)
    y = np.ones((1, 1, 128))
    nulls = np.array([orc.finalize128(y, [1.0], [100], orm, seed, 0.01)["is_null"][0] for seed in range(4000)])
    sd = np.sqrt(0.25 * 0.75 / len(nulls))
    assert abs(nulls.mean() - 0.25) < 5 * sd
    full = np.array([[np.uint64(0xFFFFFFFFFFFFFFFF)] * 2], dtype=np.uint64)
    assert orc.finalize128(y, [1.0], [100], full, 3, 0.01)["is_null"][0] == 0


def test_zero_variance_releases_the_exact_value():
    y = np.full((2, 1, 128), 21.0)
    full = np.array([[np.uint64(0xFFFFFFFFFFFFFFFF)] * 2] * 2, dtype=np.uint64)
    out = orc.finalize128(y, [2.0], [10, 10], full, 9, 1.0 / 128)
    np.testing.assert_array_equal(out["noised"], [42.0, 42.0])
    assert np.all(out["flags"] & orc.F_ZEROVAR)
    np.testing.assert_allclose(out["posterior"], np.full(128, 1.0 / 128), rtol=1e-12)


def test_first_release_noise_and_posterior_update():
    rng = np.random.default_rng(1)
    yv = rng.normal(100.0, 5.0, 128)
    B = 1.0 / 64
    full = np.array([[np.uint64(0xFFFFFFFFFFFFFFFF)] * 2], dtype=np.uint64)
    delta = np.var(yv) / (2 * B)                       # uniform prior: population variance
    zs = []
    for seed in range(3000):
        out = orc.finalize128(yv.reshape(1, 1, 128), [1.0], [500], full, seed, B)
        zs.append((out["noised"][0] - yv[out["jstar"]]) / np.sqrt(delta))
        if seed < 5:
            yt = out["noised"][0]
            logw = -(yt - yv) ** 2 / (2 * delta)
            p = np.exp(logw - logw.max())
            np.testing.assert_allclose(out["posterior"], p / p.sum(), rtol=1e-9, atol=1e-300)
    zs = np.array(zs)
    assert abs(zs.mean()) < 5 / np.sqrt(len(zs))
    assert abs(zs.var() - 1.0) < 5 * np.sqrt(2.0 / len(zs))


def test_diversity_flag_at_five_eighths_of_the_worlds():
    y = np.ones((2, 1, 128))
    m80 = [np.uint64(0xFFFFFFFFFFFFFFFF), np.uint64(0xFFFF)]          # 80 worlds updated
    m81 = [np.uint64(0xFFFFFFFFFFFFFFFF), np.uint64(0x1FFFF)]         # 81 worlds
    orm = np.array([m80, m81], dtype=np.uint64)
    flags_seen = np.zeros(2, dtype=np.uint32)
    for seed in range(64):  # some cells are NULL; the flag is set either way
        flags_seen |= orc.finalize128(y, [1.0], [64, 64], orm, seed, 0.1)["flags"]
    assert flags_seen[0] & orc.F_DIVERSITY and not (flags_seen[1] & orc.F_DIVERSITY)
