"""GPU parity of the tensor-core (tcgen05) COUNT / exact int64 SUM / AVG path.

Bar: bit-exact against the oracle and against the per-bit CUDA-core path,
over group counts, column counts, tile and CTA boundaries, value magnitudes
(one to sixteen 4-bit digits), mixed signs, key or mask input and both hash
modes; int64 overflow of a world sum is detected exactly.
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


def _values(dist, r, n):
    if dist == "small":
        return r.integers(1, 100_001, n)
    if dist == "cents":
        return r.integers(100, 10**7 + 1, n)
    if dist == "big":
        return r.integers(0, 2**40, n)
    if dist == "mixed":
        return r.integers(-(10**9), 10**9, n)
    if dist == "wide":   # all 16 digits, signed, sums still fit int64
        return r.integers(-(2**62), 2**62, n) // max(n, 1)
    if dist == "zeros":
        return np.zeros(n, dtype=np.int64)
    raise ValueError(dist)


def _specs(vals):
    specs = [(B.PAC_COUNT, B.PAC_EXACT, None)]
    for v in vals:
        specs.append((B.PAC_SUM, B.PAC_EXACT, v))
    for v in vals[:1]:
        specs.append((B.PAC_AVG, B.PAC_EXACT, v))
    return specs


def _check(ctx, keys_or_masks, gids, G, specs, masks, **kw):
    got, meta, st = ctx.aggregate(keys_or_masks, gids, G, specs, path=2, **kw)
    assert st == B.PAC_OK, B.status_name(st)
    assert ctx.last_path == 2
    ref_meta = None
    for (kind, _, vals), g_out in zip(specs, got):
        ref, mn, mo, rst = orc.aggregate(masks, vals, gids, G, kind)
        assert rst == 0
        np.testing.assert_array_equal(g_out, ref)
        ref_meta = (mn, mo)
    np.testing.assert_array_equal(meta[:, 0], ref_meta[0])
    np.testing.assert_array_equal(meta[:, 1], ref_meta[1])
    # the per-bit path agrees bit for bit
    got1, meta1, st1 = ctx.aggregate(keys_or_masks, gids, G, specs, path=1, **kw)
    assert st1 == B.PAC_OK
    for a, b in zip(got, got1):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(meta, meta1)


@pytest.mark.parametrize("G", [1, 2, 4, 6])
@pytest.mark.parametrize("C", [0, 1, 2, 4])
@pytest.mark.parametrize("n", [1, 31, 513, 100_003])
def test_mma_shapes(ctx, G, C, n):
    r = np.random.default_rng(1000 * G + 10 * C + n % 97)
    keys = r.integers(0, max(n // 3, 1), n).astype(np.int64)
    gids = None if G == 1 else r.integers(0, G, n).astype(np.uint8)
    vals = [_values("cents", r, n).astype(np.int64) for _ in range(C)]
    qk = orc.query_key(n + G)
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    _check(ctx, keys, gids, G, _specs(vals), masks, qkey=qk)


@pytest.mark.parametrize("C", [0, 1])
def test_mma_eight_groups_skewed(ctx, C):
    # eight groups with a heavy head: uneven accumulator slots across MMA warps
    n = 250_003
    r = np.random.default_rng(77 + C)
    keys = r.integers(0, 20_000, n).astype(np.int64)
    gids = np.minimum(r.geometric(0.45, n) - 1, 7).astype(np.uint8)
    vals = [r.integers(0, 10**9, n).astype(np.int64) for _ in range(C)]
    qk = orc.query_key(77)
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    _check(ctx, keys, gids, 8, _specs(vals), masks, qkey=qk)


@pytest.mark.parametrize("dist", ["small", "cents", "big", "mixed", "wide", "zeros"])
@pytest.mark.parametrize("C", [1, 4])
def test_mma_value_ranges(ctx, dist, C):
    n = 70_001
    r = np.random.default_rng(sum(map(ord, dist)) + C)
    keys = r.integers(0, 5000, n).astype(np.int64)
    gids = r.integers(0, 3, n).astype(np.int32)
    vals = [_values(dist, r, n).astype(np.int64) for _ in range(C)]
    qk = orc.query_key(5)
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    _check(ctx, keys, gids, 3, _specs(vals), masks, qkey=qk)


@pytest.mark.parametrize("C", [1, 4])
def test_mma_sixteen_digit_values(ctx, C):
    # a few values near +-2^60 among small ones: 16 signed digits, sums fit int64
    n = 1500
    r = np.random.default_rng(21 + C)
    vals = []
    for _ in range(C):
        v = r.integers(-50, 50, n).astype(np.int64)
        idx = r.choice(n, 6, replace=False)
        v[idx] = r.integers(-(2**60), 2**60, 6)
        vals.append(v)
    keys = r.integers(0, 300, n).astype(np.int64)
    gids = r.integers(0, 2, n).astype(np.uint8)
    qk = orc.query_key(21)
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    _check(ctx, keys, gids, 2, _specs(vals), masks, qkey=qk)


def test_mma_mixed_digit_counts_across_tiles(ctx):
    # tiles alternate between 2-digit, 16-digit, signed and unsigned values,
    # so accumulator columns see several digit layouts
    n = 512 * 40 + 77
    r = np.random.default_rng(3)
    v = r.integers(0, 200, n).astype(np.int64)
    for t in range(0, n // 512, 3):
        v[t * 512:(t + 1) * 512] = r.integers(-(2**50), 2**50, 512)
    v[-77:] = -5
    keys = r.integers(0, 900, n).astype(np.int64)
    gids = r.integers(0, 4, n).astype(np.uint16)
    qk = orc.query_key(6)
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    _check(ctx, keys, gids, 4, _specs([v]), masks, qkey=qk)


@pytest.mark.parametrize("in_flags", [B.PAC_IN_KEYS, B.PAC_IN_MASKS])
@pytest.mark.parametrize("mode", [B.PAC_HASH_BALANCED, B.PAC_HASH_RAW])
def test_mma_masks_and_raw(ctx, in_flags, mode):
    n = 200_000
    r = np.random.default_rng(8)
    keys = r.integers(-(2**60), 2**60, n).astype(np.int64)
    gids = r.integers(0, 5, n).astype(np.uint8)
    vals = [r.integers(0, 10**6, n).astype(np.int64) for _ in range(2)]
    qk = orc.query_key(8)
    masks = orc.hash_keys(keys, qk, mode)
    first = masks if in_flags == B.PAC_IN_MASKS else keys
    _check(ctx, first, gids, 5, _specs(vals), masks, in_flags=in_flags, hash_mode=mode, qkey=qk)


def test_mma_many_ctas_and_cta_row_cap(ctx):
    # > 2^20 rows per CTA would break FP32 exactness: 3.2M rows on 152 SMs
    # stay under the cap; 2^21 + 5 rows of one group exercise several CTAs
    n = 3_200_017
    r = np.random.default_rng(11)
    keys = r.integers(0, 1_000_000, n).astype(np.int64)
    v = r.integers(0, 2**31, n).astype(np.int64)
    qk = orc.query_key(11)
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    _check(ctx, keys, None, 1, _specs([v]), masks, qkey=qk)


def test_mma_overflow_detected(ctx):
    n = 64
    v = np.full(n, 2**62, dtype=np.int64)
    keys = np.arange(n, dtype=np.int64)
    got, _, st = ctx.aggregate(keys, None, 1, [(B.PAC_SUM, B.PAC_EXACT, v)], qkey=1, path=2)
    assert st == B.PAC_E_OVERFLOW


@pytest.mark.parametrize("gdt", [np.uint8, np.uint32])
def test_mma_bad_group_id_is_reported(ctx, gdt):
    n = 1000
    keys = np.arange(n, dtype=np.int64)
    gids = np.zeros(n, dtype=gdt)
    gids[17] = 9        # >= n_groups
    if gdt == np.uint32:
        gids[500] = 0xFFFFFFFF   # all ones: out of range too, not a padding row
    v = np.ones(n, dtype=np.int64)
    for path in (1, 2, 3):
        g_in = gids.view(np.int32) if gdt == np.uint32 else gids
        got, meta, st = ctx.aggregate(keys, g_in, 3, [(B.PAC_COUNT, 0, None), (B.PAC_SUM, 0, v)], qkey=1, path=path)
        assert st == B.PAC_E_INVALID, path
        assert int(meta[0, 0]) == n - (2 if gdt == np.uint32 else 1), path


def test_auto_path_picks_tensor_cores(ctx):
    w = inputs.small(1, 10_000, 4, 100, vlo=0, vhi=1000)
    ctx.aggregate(w.keys, w.gids.astype(np.uint8), 4, [(B.PAC_COUNT, 0, None), (B.PAC_SUM, 0, w.values[0])])
    assert ctx.last_path == 2
    ctx.aggregate(w.keys, w.gids.astype(np.uint8), 4, [(B.PAC_MAX, 0, w.values[0])])
    assert ctx.last_path == 3   # MAX: the per-bit engine


def test_wait_give_up_reports_timeout_then_recovers(ctx):
    """The bounded-wait give-up path of the tensor-core kernel, on an ordinary
    launch: with the pipeline waits limited to 1 ns they run out while the
    producers are still filling the first tiles (nothing is left out; the
    producers are simply slower than that).  The kernel then stops its
    tensor-core work, drains, frees tensor memory and reports PAC_E_TIMEOUT.
    The next call on the same context, with the default limit, is bit-exact."""
    n, G = 4_000_003, 4
    w = inputs.small(4242, n, G, 200_000, vlo=-(10**6), vhi=10**6, gid_dtype=np.uint8)
    qk = orc.query_key(4242)
    specs = _specs(w.values)
    B.pac_set_option(ctx.h, "wait_limit_ns", 1)
    try:
        _, _, st = ctx.aggregate(w.keys, w.gids, G, specs, path=2, qkey=qk)
    finally:
        B.pac_set_option(ctx.h, "wait_limit_ns", 0)
    assert st == B.PAC_E_TIMEOUT, B.status_name(st)
    masks = orc.hash_keys(w.keys, qk, orc.BALANCED)
    _check(ctx, w.keys, w.gids, G, specs, masks, qkey=qk)
