"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Bars: masks, counts, integer sums, MIN/MAX, the approximate integer cascade
and the NULL/j*/flag decisions bit-exact; exact float sums within 1e-6 of the
FP64 oracle relative to the world's sum of |v|; the paper's FLOAT-state SUM
within the FP32 bound gamma_n * sum|v|; noised releases within 1e-12 relative.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2603_15023_gb300 import binding as B
from paper_2603_15023_gb300 import inputs

pytestmark = pytest.mark.gpu

KINDS = [B.PAC_COUNT, B.PAC_SUM, B.PAC_AVG, B.PAC_MIN, B.PAC_MAX]


@pytest.fixture(scope="module")
def ctx():
    from pac_gpu_util import Ctx
    c = Ctx(0)
    yield c
    c.close()


@pytest.mark.parametrize("mode", [B.PAC_HASH_BALANCED, B.PAC_HASH_RAW])
@pytest.mark.parametrize("n", [0, 1, 2, 31, 33, 4095, 100_003])
def test_hash_keys_bit_exact(ctx, mode, n):
    keys = inputs.uniform_i64(n, 0, n, -(2**62), 2**62)
    qk = B.pac_query_key(n)
    assert qk == orc.query_key(n)
    got = ctx.hash_keys(keys, qk, mode)
    np.testing.assert_array_equal(got, orc.hash_keys(keys, qk, mode))
    if n:
        np.testing.assert_array_equal(ctx.hash_keys(keys, qk, mode, inplace=True), got)


def _oracle_all(masks, gids, G, kind, vals):
    out, mn, mo, st = orc.aggregate(masks, vals, gids, G, kind)
    return out, mn, mo, st


def _check_exact(got, ref, kind, vals, masks, gids, G):
    if vals is not None and vals.dtype != np.int64 and kind in (B.PAC_SUM, B.PAC_AVG):
        absw, *_ = orc.aggregate(masks, np.abs(vals).astype(np.float64), gids, G, B.PAC_SUM)
        if kind == B.PAC_AVG:
            cnt, *_ = orc.aggregate(masks, None, gids, G, B.PAC_COUNT)
            absw = absw / np.maximum(cnt.astype(np.float64), 1)
        err = np.abs(got - ref)
        assert np.all(err <= 1e-6 * absw + 1e-300), float(np.max(err / np.maximum(absw, 1e-300)))
    else:
        np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("G,gdt", [(1, None), (3, np.uint8), (17, np.uint16), (5000, np.int32)])
@pytest.mark.parametrize("vdtype", [np.int64, np.float32, np.float64])
@pytest.mark.parametrize("n", [0, 1, 33, 10_000, 250_007])
def test_exact_aggregates(ctx, G, gdt, vdtype, n):
    w = inputs.small(n + G, n, G, max(n // 7, 1), vdtype=vdtype, vlo=-10**6, vhi=10**6)
    gids = None if G == 1 else w.gids.astype(gdt)
    qk = orc.query_key(n)
    masks = orc.hash_keys(w.keys, qk, orc.BALANCED)
    specs = [(k, B.PAC_EXACT, None if k == B.PAC_COUNT else w.values[0]) for k in KINDS]
    got, meta, st = ctx.aggregate(w.keys, gids, G, specs, qkey=qk)
    assert st == B.PAC_OK
    for (kind, _, vals), g_out in zip(specs, got):
        ref, mn, mo, rst = _oracle_all(masks, gids, G, kind, vals)
        assert rst == 0
        _check_exact(g_out, ref, kind, vals, masks, gids, G)
    np.testing.assert_array_equal(meta[:, 0], mn)
    np.testing.assert_array_equal(meta[:, 1], mo)


@pytest.mark.parametrize("in_flags", [B.PAC_IN_KEYS, B.PAC_IN_MASKS])
@pytest.mark.parametrize("hash_mode", [B.PAC_HASH_BALANCED, B.PAC_HASH_RAW])
def test_masks_input_and_raw_hash(ctx, in_flags, hash_mode):
    w = inputs.small(5, 70_001, 4, 9000, vlo=-(2**40), vhi=2**40)
    qk = orc.query_key(77)
    masks = orc.hash_keys(w.keys, qk, hash_mode)
    first = masks if in_flags == B.PAC_IN_MASKS else w.keys
    specs = [(B.PAC_COUNT, 0, None), (B.PAC_SUM, 0, w.values[0]), (B.PAC_MAX, 0, w.values[0])]
    got, meta, st = ctx.aggregate(first, w.gids.astype(np.uint8), 4, specs, in_flags=in_flags,
                                  hash_mode=hash_mode, qkey=qk)
    assert st == B.PAC_OK
    for (kind, _, vals), g_out in zip(specs, got):
        ref, *_ = orc.aggregate(masks, vals, w.gids.astype(np.uint8), 4, kind)
        np.testing.assert_array_equal(g_out, ref)


@pytest.mark.parametrize("G", [1, 4, 32])
@pytest.mark.parametrize("n", [0, 5, 4096, 4097, 100_000, 1_000_003])
def test_approx_int_cascade_bit_exact(ctx, G, n):
    w = inputs.small(n * 3 + G, n, G, max(n // 5, 1), vlo=-(10**9), vhi=10**9)
    gids = None if G == 1 else w.gids.astype(np.uint8)
    qk = orc.query_key(3)
    masks = orc.hash_keys(w.keys, qk, orc.BALANCED)
    specs = [(B.PAC_SUM, B.PAC_APPROX, w.values[0]), (B.PAC_AVG, B.PAC_APPROX, w.values[0])]
    got, meta, st = ctx.aggregate(w.keys, gids, G, specs, qkey=qk)
    assert st == B.PAC_OK
    rs, s1 = orc.approx_sum_i64(masks, w.values[0], gids, G)
    ra, s2 = orc.approx_avg_i64(masks, w.values[0], gids, G)
    np.testing.assert_array_equal(got[0], rs)
    np.testing.assert_array_equal(got[1], ra)


def test_approx_cascade_many_flushes(ctx):
    # large positive values in few groups: deep cascades inside chunks and in the tree
    n = 600_000
    r = np.random.default_rng(9)
    vals = r.integers(2**40, 2**41, n).astype(np.int64)
    keys = r.integers(0, 50, n).astype(np.int64)
    gids = r.integers(0, 2, n).astype(np.uint8)
    qk = orc.query_key(9)
    masks = orc.hash_keys(keys, qk, orc.RAW)
    got, _, st = ctx.aggregate(keys, gids, 2, [(B.PAC_SUM, B.PAC_APPROX, vals)], qkey=qk,
                               hash_mode=B.PAC_HASH_RAW)
    ref, _ = orc.approx_sum_i64(masks, vals, gids, 2)
    assert st == B.PAC_OK
    np.testing.assert_array_equal(got[0], ref)


@pytest.mark.parametrize("in_flags", [B.PAC_IN_KEYS, B.PAC_IN_MASKS])
@pytest.mark.parametrize("mode", [B.PAC_HASH_BALANCED, B.PAC_HASH_RAW])
def test_approx_cascade_headline_shape_bit_exact(ctx, in_flags, mode):
    """The headline's column shape (4 groups with probabilities .25/.25/.49/
    .01, cents uniform in [100, 10^7], so most rows land on level 3 and every
    level total flushes every few dozen rows) on 2M rows, keys or masks, both
    hash modes, with COUNT on its own path beside the cascades: bit-exact
    against the oracle's row-by-row cascade."""
    w = inputs.lowcard_60m(seed=5, n=2_000_000)
    qk = orc.query_key(5)
    masks = orc.hash_keys(w.keys, qk, mode)
    first = masks if in_flags == B.PAC_IN_MASKS else w.keys
    specs = [(B.PAC_COUNT, B.PAC_EXACT, None), (B.PAC_SUM, B.PAC_APPROX, w.values[0]),
             (B.PAC_AVG, B.PAC_APPROX, w.values[0]), (B.PAC_SUM, B.PAC_APPROX, w.values[1])]
    got, meta, st = ctx.aggregate(first, w.gids, 4, specs, in_flags=in_flags, hash_mode=mode, qkey=qk)
    assert st == B.PAC_OK
    cnt, mn, mo, _ = orc.aggregate(masks, None, w.gids, 4, orc.COUNT)
    np.testing.assert_array_equal(got[0], cnt)
    np.testing.assert_array_equal(meta[:, 0], mn)
    np.testing.assert_array_equal(meta[:, 1], mo)
    np.testing.assert_array_equal(got[1], orc.approx_sum_i64(masks, w.values[0], w.gids, 4)[0])
    np.testing.assert_array_equal(got[2], orc.approx_avg_i64(masks, w.values[0], w.gids, 4)[0])
    np.testing.assert_array_equal(got[3], orc.approx_sum_i64(masks, w.values[1], w.gids, 4)[0])


@pytest.mark.parametrize("vdtype", [np.float32, np.float64])
def test_approx_float_state_bound(ctx, vdtype):
    n = 300_000
    r = np.random.default_rng(4)
    vals = r.lognormal(0, 1.5, n).astype(vdtype)
    keys = r.integers(0, 30000, n).astype(np.int64)
    gids = r.integers(0, 3, n).astype(np.uint8)
    qk = orc.query_key(4)
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    got, _, st = ctx.aggregate(keys, gids, 3, [(B.PAC_SUM, B.PAC_APPROX, vals)], qkey=qk)
    ref, *_ = orc.aggregate(masks, vals, gids, 3, B.PAC_SUM)
    absw, *_ = orc.aggregate(masks, np.abs(vals).astype(np.float64), gids, 3, B.PAC_SUM)
    u = 2.0**-24
    gam = (n + 1) * u / (1 - (n + 1) * u)
    assert st == B.PAC_OK
    assert np.all(np.abs(got[0] - ref) <= gam * absw)


def test_int64_sum_overflow_reported(ctx):
    n = 64
    vals = np.full(n, 2**62, dtype=np.int64)
    keys = np.arange(n, dtype=np.int64)
    got, _, st = ctx.aggregate(keys, None, 1, [(B.PAC_SUM, B.PAC_EXACT, vals)], qkey=1)
    assert st == B.PAC_E_OVERFLOW


def test_argument_errors(ctx):
    import ctypes
    inp = B.make_input(0, 10, n_groups=1)
    sp = B.make_specs([(B.PAC_COUNT, 0, B.PAC_I64, 0, 1234)])
    with pytest.raises(B.PacError) as e:
        B.pac_aggregate_multi(ctx.h, inp, sp, 1, 0)
    assert e.value.status == B.PAC_E_INVALID
    inp = B.make_input(1234, 10, n_groups=3)  # ungrouped with 3 groups
    with pytest.raises(B.PacError):
        B.pac_aggregate_multi(ctx.h, inp, sp, 1, 0)
    bad = B.make_specs([(9, 0, B.PAC_I64, 0, 1234)])
    with pytest.raises(B.PacError):
        B.pac_aggregate_multi(ctx.h, B.make_input(1234, 10), bad, 1, 0)
    with pytest.raises(B.PacError):
        B.pac_set_option(ctx.h, "agg_path", 7)
    assert ctypes.c_int(B.lib().pac_hash_keys(ctx.h, None, None, 5, 0, 0, None)).value == B.PAC_E_INVALID


@pytest.mark.parametrize("mode", [B.PAC_FIN_ADAPTIVE, B.PAC_FIN_INDEPENDENT])
@pytest.mark.parametrize("G", [1, 7, 300])
def test_finalize_matches_oracle(ctx, mode, G):
    r = np.random.default_rng(G)
    kv = [(B.PAC_COUNT, 0, B.PAC_I64), (B.PAC_SUM, 0, B.PAC_I64), (B.PAC_AVG, 0, B.PAC_I64),
          (B.PAC_SUM, 0, B.PAC_F64), (B.PAC_MIN, 0, B.PAC_I64)]
    outs = [r.integers(0, 5000, (G, 64)).astype(np.uint64),
            r.integers(-10**9, 10**9, (G, 64)).astype(np.int64),
            r.normal(50, 9, (G, 64)),
            r.lognormal(3, 1, (G, 64)),
            r.integers(-100, 100, (G, 64)).astype(np.int64)]
    meta = np.zeros((G, 2), dtype=np.uint64)
    meta[:, 0] = r.integers(0, 200, G)
    meta[:, 1] = np.uint64(0xFFFFFFFFFFFFFFFF)
    meta[::3, 1] = np.uint64(0x0000FFFF0000FFFF)       # sparse groups: NULL draws
    meta[::5, 1] = np.uint64(0x00000000FFFFFFFF)       # single PU: diversity flag
    outs[0][2 % G, :] = 5                              # one constant cell (zero variance)
    seed, budget = 1234 + G, 1.0 / 128
    got = ctx.finalize(outs, kv, meta, seed, budget, mode)
    y = np.stack([o.astype(np.float64) for o in outs], axis=1)   # [G, S, 64]
    scales = [orc.release_scale(k) for k, _, _ in kv]
    ref = orc.finalize(y, scales, meta[:, 0], meta[:, 1], seed, budget, mode)
    np.testing.assert_array_equal(got["is_null"], ref["is_null"])
    np.testing.assert_array_equal(got["flags"], ref["flags"])
    live = ref["is_null"] == 0
    np.testing.assert_allclose(got["noised"][live], ref["noised"][live], rtol=1e-12, atol=0)
    np.testing.assert_allclose(got["posterior"], ref["posterior"], rtol=1e-10, atol=1e-15)


def _aggregate_like(G, seed):
    """World results shaped like real aggregates: each world holds about half
    of a group's rows, so the 64 results of a cell are close to one another
    and the adaptive posterior narrows over the cells until one world is left."""
    r = np.random.default_rng(seed)
    n = np.maximum(1, r.lognormal(6, 2, G)).astype(np.int64)
    cnt = r.binomial(n[:, None], 0.5, (G, 64)).astype(np.uint64)
    c = cnt.astype(np.float64)
    isum = (c * 500 + r.normal(0, 1, (G, 64)) * np.sqrt(c) * 290).astype(np.int64)
    fsum = c * 3.7 + r.normal(0, 1, (G, 64)) * np.sqrt(c) * 2.0
    avg = fsum / np.maximum(c, 1)
    meta = np.zeros((G, 2), dtype=np.uint64)
    meta[:, 0] = n
    meta[:, 1] = np.uint64(0xFFFFFFFFFFFFFFFF)
    meta[n < 40, 1] = np.uint64(0x00FF00FF00FF00FF)
    kv = [(B.PAC_COUNT, 0, B.PAC_I64), (B.PAC_SUM, 0, B.PAC_I64), (B.PAC_SUM, 0, B.PAC_F64),
          (B.PAC_AVG, 0, B.PAC_I64)]
    return [cnt, isum, fsum, avg], kv, meta


@pytest.mark.parametrize("mode", [B.PAC_FIN_ADAPTIVE, B.PAC_FIN_INDEPENDENT])
@pytest.mark.parametrize("case", ["long", "nonfinite", "bigint"])
def test_finalize_long_chain_matches_oracle(ctx, case, mode):
    """Thousands of releases on aggregate-like results.  Adaptive: the
    posterior collapses onto one world part-way, after which releases have
    variance 0.  Independent: every cell from the uniform prior, the
    posterior of the last release read back.
    'nonfinite' plants inf/NaN world values in float cells after the
    collapse (the variance sums turn them into NaN releases); 'bigint' puts
    int64 sums above 2^53, where distinct integers can meet as doubles."""
    G = 2500
    outs, kv, meta = _aggregate_like(G, 4242)
    r = np.random.default_rng(7)
    if case == "nonfinite":
        for g in r.choice(np.arange(G // 2, G), 40, replace=False):
            outs[2][g, r.integers(0, 64, 3)] = [np.inf, -np.inf, np.nan][int(r.integers(0, 3))]
        outs[3][G - 5, :] = np.nan
        outs[2][G - 7, :] = np.inf
        outs[2][G - 9, :] = 2.0 ** 1023          # doubled by the release scale: inf
    if case == "bigint":
        outs[1] = (np.int64(1) << 60) + r.integers(0, 100, (G, 64)).astype(np.int64)
        outs[1][::2] = r.integers(-2**62, 2**62, (G - G // 2, 64))
    seed, budget = 99, 1.0 / 128
    got = ctx.finalize(outs, kv, meta, seed, budget, mode)
    y = np.stack([o.astype(np.float64) for o in outs], axis=1)
    ref = orc.finalize(y, [orc.release_scale(k) for k, _, _ in kv], meta[:, 0], meta[:, 1], seed, budget, mode)
    if case == "long" and mode == B.PAC_FIN_ADAPTIVE:
        assert ((ref["flags"] & orc.F_ZEROVAR) != 0).sum() > G      # the chain did collapse
    np.testing.assert_array_equal(got["is_null"], ref["is_null"])
    np.testing.assert_array_equal(got["flags"], ref["flags"])
    live = ref["is_null"] == 0
    np.testing.assert_allclose(got["noised"][live], ref["noised"][live], rtol=1e-12, atol=0)
    np.testing.assert_allclose(got["posterior"], ref["posterior"], rtol=1e-10, atol=1e-15)


def test_lowcard_60m_full_size_sampled(ctx):
    """The 60M-row, 4-group, 4-column workload at full size, in the launch
    configuration the benchmark times: sampled worlds against the oracle,
    every world against the balanced invariants."""
    w = inputs.lowcard_60m(seed=0)
    qk = orc.query_key(0)
    specs = [(B.PAC_COUNT, 0, None)] + [(B.PAC_SUM, 0, v) for v in w.values] + \
            [(B.PAC_AVG, 0, v) for v in w.values]
    got, meta, st = ctx.aggregate(w.keys, w.gids, 4, specs, qkey=qk)
    assert st == B.PAC_OK
    masks = orc.hash_keys(w.keys, qk, orc.BALANCED)
    for j in (0, 21, 42, 63):
        c, _ = orc.aggregate_world(masks, None, w.gids, 4, B.PAC_COUNT, j)
        np.testing.assert_array_equal(got[0][:, j], c)
        for k, v in enumerate(w.values):
            s, _ = orc.aggregate_world(masks, v, w.gids, 4, B.PAC_SUM, j)
            np.testing.assert_array_equal(got[1 + k][:, j], s)
            a, _ = orc.aggregate_world(masks, v, w.gids, 4, B.PAC_AVG, j)
            np.testing.assert_array_equal(got[5 + k][:, j], a)
    ng = np.bincount(w.gids, minlength=4).astype(np.uint64)
    cnt = got[0].astype(np.int64)
    np.testing.assert_array_equal(meta[:, 0], ng)
    assert np.all(cnt[:, :32] + cnt[:, 32:] == ng.astype(np.int64)[:, None])
    for k, v in enumerate(w.values):
        tot = np.array([v[w.gids == g].sum() for g in range(4)])
        assert np.all(got[1 + k][:, :32] + got[1 + k][:, 32:] == tot[:, None])


@pytest.mark.parametrize("path", [1, 3])
@pytest.mark.parametrize("mode", [B.PAC_HASH_BALANCED, B.PAC_HASH_RAW])
@pytest.mark.parametrize("G,gdt", [(1, None), (17, np.uint16), (5000, np.int32)])
@pytest.mark.parametrize("vdtype", [np.int64, np.float32, np.float64])
def test_forced_per_bit_paths(ctx, path, mode, G, gdt, vdtype):
    """The plain per-bit kernels (path 1) and the per-bit engine (path 3) on
    every kind, both hash modes, few and many groups, against the oracle."""
    n = 100_003
    w = inputs.small(7 * G + n, n, G, 9_000, vdtype=vdtype, vlo=-10**6, vhi=10**6)
    gids = None if G == 1 else w.gids.astype(gdt)
    qk = orc.query_key(G)
    masks = orc.hash_keys(w.keys, qk, mode)
    specs = [(k, B.PAC_EXACT, None if k == B.PAC_COUNT else w.values[0]) for k in KINDS]
    got, meta, st = ctx.aggregate(w.keys, gids, G, specs, qkey=qk, hash_mode=mode, path=path)
    assert st == B.PAC_OK
    assert ctx.last_path == path
    for (kind, _, vals), g_out in zip(specs, got):
        ref, mn, mo, rst = _oracle_all(masks, gids, G, kind, vals)
        assert rst == 0
        _check_exact(g_out, ref, kind, vals, masks, gids, G)
    np.testing.assert_array_equal(meta[:, 0], mn)
    np.testing.assert_array_equal(meta[:, 1], mo)


@pytest.mark.parametrize("only_sum", [False, True, "two"])
@pytest.mark.parametrize("dist", ["narrow", "wide", "w45", "negative", "zeros", "short_runs"])
def test_engine_int_sums_bit_sliced_and_looped(ctx, dist, only_sum):
    """Int64 SUM on the engine: non-negative values in runs at least as long
    as their bit length take the bit-sliced form (planes of the low and high
    words), short runs and negative values the broadcast loop; all exact.
    only_sum: COUNT + SUM alone, "two": COUNT + two SUMs (both with
    compile-time slot operations)."""
    n, G = 200_000, 3
    r = np.random.default_rng(len(dist))
    keys = r.integers(0, 50_000, n).astype(np.int64)
    gids = r.integers(0, G, n).astype(np.uint8)
    if dist != "short_runs":
        gids = np.sort(gids)                                # long runs
    vals = {"narrow": r.integers(0, 2**31, n), "wide": r.integers(0, 2**40, n),
            "w45": r.integers(2**44, 2**45, n), "negative": r.integers(-10**9, 10**9, n),
            "zeros": np.zeros(n, dtype=np.int64), "short_runs": r.integers(0, 2**20, n)}[dist].astype(np.int64)
    qk = orc.query_key(99)
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    specs = [(B.PAC_COUNT, 0, None), (B.PAC_SUM, 0, vals)]
    if only_sum == "two":
        specs.append((B.PAC_SUM, 0, (vals // 3).astype(np.int64)))
    elif not only_sum:
        specs += [(B.PAC_AVG, 0, vals), (B.PAC_MIN, 0, vals)]
    got, meta, st = ctx.aggregate(keys, gids, G, specs, qkey=qk, path=3)
    assert st == B.PAC_OK and ctx.last_path == 3
    for (kind, _, v), g_out in zip(specs, got):
        ref, *_ = orc.aggregate(masks, v, gids, G, kind)
        np.testing.assert_array_equal(g_out, ref)


@pytest.mark.parametrize("G", [3, 3000])
def test_engine_bad_group_ids_skipped_and_reported(ctx, G):
    """Rows whose group id is >= n_groups are dropped (never written out of
    bounds) and reported as PAC_E_INVALID; the other rows aggregate exactly,
    on both state placements of the engine (few groups: shared memory; many
    groups: partitioned rows with atomics)."""
    n = 50_000
    r = np.random.default_rng(G)
    keys = r.integers(0, 9_000, n).astype(np.int64)
    gids = r.integers(0, G, n).astype(np.int32)
    bad = r.random(n) < 0.01
    gids_bad = gids.copy()
    gids_bad[bad] = G + 5
    gids_bad[np.flatnonzero(bad)[::2]] = -1     # 0xFFFFFFFF as an unsigned id
    vals = r.integers(-1000, 1000, n).astype(np.int64)
    qk = orc.query_key(5)
    specs = [(B.PAC_COUNT, 0, None), (B.PAC_SUM, 0, vals)]
    got, meta, st = ctx.aggregate(keys, gids_bad, G, specs, qkey=qk, path=3)
    assert st == B.PAC_E_INVALID
    keep = ~bad
    masks = orc.hash_keys(keys[keep], qk, orc.BALANCED)
    for (kind, _, v), g_out in zip(specs, got):
        ref, mn, mo, _ = orc.aggregate(masks, None if v is None else v[keep], gids[keep], G, kind)
        np.testing.assert_array_equal(g_out, ref)
    np.testing.assert_array_equal(meta[:, 0], mn)


@pytest.mark.parametrize("path", [1, 2, 3, 4])
def test_avg_exact_when_the_sum_overflows(ctx, path):
    """A world's int64 SUM that does not fit is reported (PAC_E_OVERFLOW) on
    every path.  The tensor-core and one-launch paths keep 128-bit totals:
    there the SUM is saturated and the AVG is still the exact sum over the
    count (the int128 total rounded to the nearest double, then divided: the
    oracle's reading).  The per-bit kernels keep 64-bit partial sums, so only
    the report and the counts are defined there."""
    n = 20_000
    r = np.random.default_rng(path)
    G = 1 if path == 4 else 3
    keys = r.integers(0, 5000, n).astype(np.int64)
    gids = None if G == 1 else r.integers(0, G, n).astype(np.uint8)
    vals = (2**62 + r.integers(0, 2**40, n)).astype(np.int64)
    specs = [(B.PAC_COUNT, 0, None), (B.PAC_SUM, 0, vals), (B.PAC_AVG, 0, vals)]
    qk = orc.query_key(path)
    got, _, st = ctx.aggregate(keys, gids, G, specs, qkey=qk, path=path)
    assert st == B.PAC_E_OVERFLOW
    assert ctx.last_path == path
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    checked = specs if path in (2, 4) else specs[:1]
    for (kind, _, v), g_out in zip(checked, got):
        ref, *_ = orc.aggregate(masks, v, gids, G, kind)
        np.testing.assert_array_equal(g_out, ref)


def test_highcard_100m_full_size_sampled(ctx):
    """The 100M-row, 1M-group Zipf workload at full size, in the launch
    configuration the benchmark times (automatic path: rows partitioned by
    group, then the many-group tensor-core kernel).  Sampled groups (the
    largest, a middle and a tail one) against the oracle on exactly their
    rows; every group against the balanced invariants (worlds j and j+32
    split the group's rows and its value total) and against the per-bit
    engine, bit for bit."""
    w = inputs.highcard_100m(seed=0)
    G = w.n_groups
    qk = orc.query_key(0)
    v = w.values[0]
    specs = [(B.PAC_COUNT, 0, None), (B.PAC_SUM, 0, v)]
    got, meta, st = ctx.aggregate(w.keys, w.gids, G, specs, qkey=qk)
    assert st == B.PAC_OK
    assert ctx.last_path == 5
    got3, meta3, st3 = ctx.aggregate(w.keys, w.gids, G, specs, qkey=qk, path=3)
    assert st3 == B.PAC_OK
    for a, b in zip(got, got3):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(meta, meta3)
    for g in (0, 4321, G - 1):
        rows = np.flatnonzero(w.gids == g)
        masks = orc.hash_keys(w.keys[rows], qk, orc.BALANCED)
        c, mn, mo, _ = orc.aggregate(masks, None, None, 1, B.PAC_COUNT)
        s, *_ = orc.aggregate(masks, v[rows], None, 1, B.PAC_SUM)
        np.testing.assert_array_equal(got[0][g], c[0])
        np.testing.assert_array_equal(got[1][g], s[0])
        assert int(meta[g, 0]) == int(mn[0]) and int(meta[g, 1]) == int(mo[0])
    ng = np.bincount(w.gids, minlength=G).astype(np.int64)
    tot = np.bincount(w.gids, weights=v.astype(np.float64), minlength=G)  # per-group sums < 2^53: exact
    np.testing.assert_array_equal(meta[:, 0].astype(np.int64), ng)
    cnt = got[0].astype(np.int64)
    assert np.all(cnt[:, :32] + cnt[:, 32:] == ng[:, None])
    assert np.all(got[1][:, :32] + got[1][:, 32:] == tot.astype(np.int64)[:, None])


def test_lowcard_60m_approx_full_size_bound(ctx):
    """The paper's approximate SUM / AVG on the 60M-row headline columns at
    full size, in the benchmark's launch configuration: for sampled worlds,
    each approximate SUM lies under the exact one (from the oracle) by at most
    the cascade's truncation bound, sum |v| (2^-8 + 25 * 2^-11.9) (values are
    positive, so only the positive side is used), and AVG is 2 S / n_g of the
    SUM the kernel wrote (bit-exact)."""
    w = inputs.lowcard_60m(seed=0)
    qk = orc.query_key(0)
    specs = [(B.PAC_COUNT, 0, None)] + [(B.PAC_SUM, B.PAC_APPROX, v) for v in w.values] + \
            [(B.PAC_AVG, B.PAC_APPROX, v) for v in w.values]
    got, meta, st = ctx.aggregate(w.keys, w.gids, 4, specs, qkey=qk)
    assert st == B.PAC_OK
    masks = orc.hash_keys(w.keys, qk, orc.BALANCED)
    ng = meta[:, 0].astype(np.float64)
    for k, v in enumerate(w.values):
        approx = got[1 + k]
        np.testing.assert_array_equal(got[5 + k], np.where(ng[:, None] > 0, 2.0 * approx / ng[:, None], 0.0))
        for j in (0, 17, 40, 63):
            exact, _ = orc.aggregate_world(masks, v, w.gids, 4, B.PAC_SUM, j)
            bound = exact.astype(np.float64) * (2.0**-8 + 25 * 2.0**-11.9)
            diff = exact - approx[:, j]
            assert np.all(diff >= 0) and np.all(diff <= bound), (k, j)


@pytest.mark.parametrize("G", [40_000, 150_001])
def test_many_groups_multi_block_scan(ctx, G):
    """Queries above 32K groups scan their group counts with several blocks:
    the partitioned engine path with Zipf-like skew (one hot group) and a
    uniform tail, every world against the oracle."""
    n = 400_003
    r = np.random.default_rng(G)
    gids = np.where(r.random(n) < 0.2, 0, r.integers(0, G, n)).astype(np.int32)
    keys = r.integers(0, 60_000, n).astype(np.int64)
    vals = r.integers(-(10**6), 10**6, n).astype(np.int64)
    qk = orc.query_key(G)
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    specs = [(B.PAC_COUNT, 0, None), (B.PAC_SUM, 0, vals), (B.PAC_MAX, 0, vals)]
    got, meta, st = ctx.aggregate(keys, gids, G, specs, qkey=qk)
    assert st == B.PAC_OK
    assert ctx.last_path == 3
    for (kind, _, v), g_out in zip(specs, got):
        ref, mn, mo, rst = orc.aggregate(masks, v, gids, G, kind)
        assert rst == 0
        np.testing.assert_array_equal(g_out, ref)
    np.testing.assert_array_equal(meta[:, 0], mn)
    np.testing.assert_array_equal(meta[:, 1], mo)
