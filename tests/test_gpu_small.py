"""GPU parity of the one-launch path (ungrouped COUNT / exact int64 SUM / AVG in
one kernel whose last CTA writes the outputs) against the oracle.

Bars: counts, sums, meta and the overflow / bad-group decisions bit-exact,
AVG as the oracle's IEEE quotient.  Cases: the batch and warp edges (0, 1, 31,
32, 33 rows, ragged tails), values that take the bit-sliced sums (non-negative
below 2^32) and values that do not (negative, beyond 2^32, mixed within a
batch), int128 intermediate sums, balanced and raw masks, masks given as
input, dropped zero-mask rows, a group-id column, up to four columns, repeated
calls (the kernel leaves its accumulators zero), the automatic choice up to
8M rows and the forced path beyond it.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2603_15023_gb300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from pac_gpu_util import Ctx
    c = Ctx(0)
    yield c
    c.close()


def _vals(kind, n, r):
    if kind == "small":
        return r.integers(0, 100_001, n)
    if kind == "neg":
        return r.integers(-10**6, 10**6, n)
    if kind == "wide":
        return r.integers(0, 2**40, n)
    # mixed: most batches bit-sliced, some with a negative or a wide value
    v = r.integers(0, 5000, n)
    v[r.random(n) < 0.002] = -7
    v[r.random(n) < 0.002] = 2**35
    return v


def _check(ctx, keys, vals_list, qk, *, hash_mode=B.PAC_HASH_BALANCED, in_flags=B.PAC_IN_KEYS, gids=None,
           path=0, expect_path=4, expect_st=B.PAC_OK, masks_ref=None, keep=None):
    specs = [(B.PAC_COUNT, B.PAC_EXACT, None)]
    for v in vals_list:
        specs += [(B.PAC_SUM, B.PAC_EXACT, v), (B.PAC_AVG, B.PAC_EXACT, v)]
    got, meta, st = ctx.aggregate(keys, gids, 1, specs, qkey=qk, hash_mode=hash_mode, in_flags=in_flags,
                                  path=path)
    assert st == expect_st
    assert ctx.last_path == expect_path
    masks = masks_ref if masks_ref is not None else orc.hash_keys(keys, qk, hash_mode)
    sel = np.ones(len(masks), dtype=bool) if keep is None else keep
    for (kind, _, v), g_out in zip(specs, got):
        ref, mn, mo, rst = orc.aggregate(masks[sel], None if v is None else v[sel], None, 1, kind)
        np.testing.assert_array_equal(g_out, ref)
        np.testing.assert_array_equal(meta[:, 0], mn)
        np.testing.assert_array_equal(meta[:, 1], mo)
    return got


@pytest.mark.parametrize("n", [0, 1, 31, 32, 33, 4095, 100_003, 1_000_000])
@pytest.mark.parametrize("vk", ["small", "neg", "wide", "mixed"])
def test_one_launch_matches_oracle(ctx, n, vk):
    r = np.random.default_rng(n * 7 + len(vk))
    keys = r.integers(0, 150_000, n).astype(np.int64)
    v = _vals(vk, n, r).astype(np.int64)
    _check(ctx, keys, [v], orc.query_key(n))


@pytest.mark.parametrize("C", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("hash_mode", [B.PAC_HASH_BALANCED, B.PAC_HASH_RAW])
def test_columns_and_hash_modes(ctx, C, hash_mode):
    n = 250_007
    r = np.random.default_rng(C + 10 * hash_mode)
    keys = r.integers(0, 40_000, n).astype(np.int64)
    cols = [_vals(k, n, r).astype(np.int64) for k in ["small", "neg", "wide", "mixed"][:C]]
    _check(ctx, keys, cols, orc.query_key(C), hash_mode=hash_mode)


def test_masks_input_with_dropped_rows(ctx):
    n = 70_001
    r = np.random.default_rng(3)
    masks = (r.integers(0, 2**63, n, dtype=np.int64).astype(np.uint64) << np.uint64(1)) | r.integers(0, 2, n).astype(np.uint64)
    masks[r.random(n) < 0.05] = 0
    v = r.integers(-1000, 1000, n).astype(np.int64)
    specs_v = [v]
    _check(ctx, masks, specs_v, 0, in_flags=B.PAC_IN_MASKS | B.PAC_IN_DROP_EMPTY, masks_ref=masks,
           keep=masks != 0)


def test_group_column_and_bad_ids(ctx):
    """One group given through a group-id column: ids other than 0 are out of
    range, skipped and reported."""
    n = 50_000
    r = np.random.default_rng(8)
    keys = r.integers(0, 9000, n).astype(np.int64)
    v = r.integers(1, 10**5, n).astype(np.int64)
    gids = np.zeros(n, dtype=np.uint8)
    _check(ctx, keys, [v], orc.query_key(8), gids=gids)
    gids[r.random(n) < 0.01] = 3
    _check(ctx, keys, [v], orc.query_key(8), gids=gids, expect_st=B.PAC_E_INVALID,
           masks_ref=orc.hash_keys(keys, orc.query_key(8), orc.BALANCED), keep=gids == 0)


def test_int128_sums_and_overflow(ctx):
    # running sums far beyond int64 (the first half's 2^62s) that the second
    # half cancels: the same PUs with -2^62, so every world ends near zero
    n = 200_000
    r = np.random.default_rng(11)
    keys = r.integers(0, 3000, n).astype(np.int64)
    keys[n // 2:] = keys[: n // 2]
    v = np.where(np.arange(n) < n // 2, 2**62, -(2**62)).astype(np.int64)
    v[-1] = 12345
    _check(ctx, keys, [v], orc.query_key(11))
    # totals that do not fit: reported, saturated like the oracle
    v2 = np.full(n, 2**62, dtype=np.int64)
    _check(ctx, keys, [v2], orc.query_key(12), expect_st=B.PAC_E_OVERFLOW)


def test_repeated_calls_start_from_zero(ctx):
    r = np.random.default_rng(21)
    for n in [1_000_000, 17, 333_333]:
        keys = r.integers(0, 150_000, n).astype(np.int64)
        v = r.integers(1, 100_000, n).astype(np.int64)
        first = _check(ctx, keys, [v], orc.query_key(21))
        again = _check(ctx, keys, [v], orc.query_key(21))
        for a, b in zip(first, again):
            np.testing.assert_array_equal(a, b)


def test_auto_choice_and_forced_path(ctx):
    r = np.random.default_rng(5)
    n = 8 * 2**20 + 1                       # past the automatic limit: tensor-core path
    keys = r.integers(0, 150_000, n).astype(np.int64)
    v = r.integers(1, 100_000, n).astype(np.int64)
    _check(ctx, keys, [v], orc.query_key(5), expect_path=2)
    _check(ctx, keys, [v], orc.query_key(5), path=4, expect_path=4)
    _check(ctx, keys[: 8 * 2**20], [v[: 8 * 2**20]], orc.query_key(5), expect_path=4)


def test_forced_path_rejects_grouped_and_float(ctx):
    n = 1000
    keys = np.arange(n, dtype=np.int64)
    gids = (np.arange(n) % 2).astype(np.uint8)
    with pytest.raises(B.PacError) as e:
        ctx.aggregate(keys, gids, 2, [(B.PAC_COUNT, 0, None)], path=4)
    assert e.value.status == B.PAC_E_UNSUPPORTED
    with pytest.raises(B.PacError) as e:
        ctx.aggregate(keys, None, 1, [(B.PAC_SUM, 0, np.ones(n, dtype=np.float64))], path=4)
    assert e.value.status == B.PAC_E_UNSUPPORTED
    B.pac_set_option(ctx.h, "agg_path", 0)
