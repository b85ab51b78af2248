"""GPU parity of m = 128 worlds (Sec. 2: m = 128 is possible with twice the
state) through the C ABI, against the oracle's 128-world functions.

Bars, as for m = 64: the two mask words, counts, integer sums, AVG of
integers, MIN/MAX, the per-group metadata and the release's NULL/flag
decisions bit-exact; exact float sums within 1e-6 of the FP64 oracle relative
to the world's sum of |v|; releases within 1e-12 relative, the posterior
within 1e-10.  Both hash modes, key and mask input, every kind and value
type, few and many groups; the tensor-core tile at M = 128 and the per-bit
engine on each 64-world half are both forced and checked.
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


def _check(got, ref, kind, vals, masks2, gids, G):
    if vals is not None and vals.dtype != np.int64 and kind in (B.PAC_SUM, B.PAC_AVG):
        absw, *_ = orc.aggregate128(masks2, np.abs(vals).astype(np.float64), gids, G, B.PAC_SUM)
        if kind == B.PAC_AVG:
            cnt, *_ = orc.aggregate128(masks2, None, gids, G, B.PAC_COUNT)
            absw = absw / np.maximum(cnt.astype(np.float64), 1)
        err = np.abs(got - ref)
        assert np.all(err <= 1e-6 * absw + 1e-300), float(np.max(err / np.maximum(absw, 1e-300)))
    else:
        np.testing.assert_array_equal(got, ref)


def _keys2(seed):
    k1, k2 = B.pac_query_key(seed), B.pac_query_key2(seed)
    assert (k1, k2) == (orc.query_key(seed), orc.query_key2(seed))
    return k1, k2


@pytest.mark.parametrize("mode", [B.PAC_HASH_BALANCED, B.PAC_HASH_RAW])
@pytest.mark.parametrize("n", [0, 1, 33, 100_003])
def test_hash128_bit_exact(ctx, mode, n):
    keys = inputs.uniform_i64(n + 11, 0, n, -(2**62), 2**62)
    k1, k2 = _keys2(n)
    got = ctx.hash_keys128(keys, k1, k2, mode)
    np.testing.assert_array_equal(got, orc.hash_keys128(keys, k1, k2, mode))
    if n and mode == B.PAC_HASH_BALANCED:
        assert np.all(got[:, 1] == ~got[:, 0])  # every PU in exactly 64 worlds


def _oracle_meta(masks2, gids, G):
    _, mn, mo, _ = orc.aggregate128(masks2, None, gids, G, B.PAC_COUNT)
    return mn, mo


@pytest.mark.parametrize("G,gdt", [(1, None), (5, np.uint8), (300, np.int32)])
@pytest.mark.parametrize("vdtype", [np.int64, np.float32, np.float64])
@pytest.mark.parametrize("mode", [B.PAC_HASH_BALANCED, B.PAC_HASH_RAW])
def test_aggregate128_every_kind(ctx, G, gdt, vdtype, mode):
    n = 60_007
    w = inputs.small(3 * G + 7, n, G, 7_000, vdtype=vdtype, vlo=-10**6, vhi=10**6)
    gids = None if G == 1 else w.gids.astype(gdt)
    k1, k2 = _keys2(G + 1000)
    masks2 = orc.hash_keys128(w.keys, k1, k2, mode)
    specs = [(k, B.PAC_EXACT, None if k == B.PAC_COUNT else w.values[0]) for k in KINDS]
    got, meta, st = ctx.aggregate128(w.keys, gids, G, specs, hash_mode=mode, qkey=k1, qkey2=k2)
    assert st == B.PAC_OK, B.status_name(st)
    for (kind, _, vals), g_out in zip(specs, got):
        ref, _, _, rst = orc.aggregate128(masks2, vals, gids, G, kind)
        assert rst == 0
        _check(g_out, ref, kind, vals, masks2, gids, G)
    mn, mo = _oracle_meta(masks2, gids, G)
    np.testing.assert_array_equal(meta[:, 0], mn)
    np.testing.assert_array_equal(meta[:, 1:], mo)


@pytest.mark.parametrize("path", [2, 3])
@pytest.mark.parametrize("in_flags", [B.PAC_IN_KEYS, B.PAC_IN_MASKS])
@pytest.mark.parametrize("mode", [B.PAC_HASH_BALANCED, B.PAC_HASH_RAW])
def test_aggregate128_paths_and_inputs(ctx, path, in_flags, mode):
    """COUNT / exact int64 SUM / AVG on the M = 128 tensor-core tile (path 2)
    and on the per-bit engine, one pass per 64-world half (path 3), from keys
    and from [n, 2] masks: both bit-exact against the oracle."""
    n, G = 250_003, 4
    w = inputs.small(91, n, G, 30_000, vlo=-(2**40), vhi=2**40, gid_dtype=np.uint8)
    k1, k2 = _keys2(91)
    masks2 = orc.hash_keys128(w.keys, k1, k2, mode)
    first = masks2 if in_flags == B.PAC_IN_MASKS else w.keys
    specs = [(B.PAC_COUNT, B.PAC_EXACT, None), (B.PAC_SUM, B.PAC_EXACT, w.values[0]),
             (B.PAC_AVG, B.PAC_EXACT, w.values[0])]
    got, meta, st = ctx.aggregate128(first, w.gids, G, specs, in_flags=in_flags, hash_mode=mode, qkey=k1,
                                     qkey2=k2, path=path)
    assert st == B.PAC_OK, B.status_name(st)
    if path == 2:
        assert ctx.last_path == 2
    for (kind, _, vals), g_out in zip(specs, got):
        ref, _, _, rst = orc.aggregate128(masks2, vals, w.gids, G, kind)
        assert rst == 0
        np.testing.assert_array_equal(g_out, ref)
    mn, mo = _oracle_meta(masks2, w.gids, G)
    np.testing.assert_array_equal(meta[:, 0], mn)
    np.testing.assert_array_equal(meta[:, 1:], mo)


def _values(dist, r, n):
    if dist == "cents":
        return r.integers(100, 10**7 + 1, n)
    if dist == "wide":   # all 16 digits, signed, sums still fit int64
        return r.integers(-(2**62), 2**62, n) // max(n, 1)
    return r.integers(-(10**9), 10**9, n)


@pytest.mark.parametrize("G", [1, 2, 6, 8])
@pytest.mark.parametrize("C", [0, 1, 4])
@pytest.mark.parametrize("n", [1, 257, 100_003])
def test_mma128_shapes(ctx, G, C, n):
    """Group counts up to the tensor-memory limit, 0/1/4 value columns, a
    single row, a ragged tile and many tiles, with signed 16-digit values."""
    if G * (32 if C <= 1 else 80) > 512:
        pytest.skip("more accumulator columns than tensor memory holds")
    r = np.random.default_rng(1000 * G + 10 * C + n % 97)
    keys = r.integers(0, max(n // 3, 1), n).astype(np.int64)
    gids = None if G == 1 else r.integers(0, G, n).astype(np.uint8)
    vals = [_values(["cents", "wide", "mixed", "cents"][c], r, n).astype(np.int64) for c in range(C)]
    k1, k2 = _keys2(n + G)
    masks2 = orc.hash_keys128(keys, k1, k2, orc.BALANCED)
    specs = [(B.PAC_COUNT, B.PAC_EXACT, None)] + [(B.PAC_SUM, B.PAC_EXACT, v) for v in vals] + \
            [(B.PAC_AVG, B.PAC_EXACT, v) for v in vals[:1]]
    got, meta, st = ctx.aggregate128(keys, gids, G, specs, qkey=k1, qkey2=k2, path=2)
    assert st == B.PAC_OK, B.status_name(st)
    assert ctx.last_path == 2
    for (kind, _, v), g_out in zip(specs, got):
        ref, _, _, rst = orc.aggregate128(masks2, v, gids, G, kind)
        assert rst == 0
        np.testing.assert_array_equal(g_out, ref)
    mn, mo = _oracle_meta(masks2, gids, G)
    np.testing.assert_array_equal(meta[:, 0], mn)
    np.testing.assert_array_equal(meta[:, 1:], mo)


@pytest.mark.parametrize("mode", [B.PAC_FIN_ADAPTIVE, B.PAC_FIN_INDEPENDENT])
@pytest.mark.parametrize("G", [1, 7, 300])
def test_finalize128_matches_oracle(ctx, mode, G):
    r = np.random.default_rng(128 + G)
    kv = [(B.PAC_COUNT, 0, B.PAC_I64), (B.PAC_SUM, 0, B.PAC_I64), (B.PAC_AVG, 0, B.PAC_I64),
          (B.PAC_SUM, 0, B.PAC_F64), (B.PAC_MIN, 0, B.PAC_I64)]
    outs = [r.integers(0, 5000, (G, 128)).astype(np.uint64),
            r.integers(-10**9, 10**9, (G, 128)).astype(np.int64),
            r.normal(50, 9, (G, 128)),
            r.lognormal(3, 1, (G, 128)),
            r.integers(-100, 100, (G, 128)).astype(np.int64)]
    meta = np.zeros((G, 3), dtype=np.uint64)
    meta[:, 0] = r.integers(0, 200, G)
    meta[:, 1:] = np.uint64(0xFFFFFFFFFFFFFFFF)
    meta[::3, 2] = np.uint64(0x0000FFFF0000FFFF)       # sparse groups: NULL draws
    meta[::5, 1] = np.uint64(0x00000000FFFFFFFF)       # few worlds: diversity flag
    meta[::5, 2] = np.uint64(0x000000000000FFFF)
    outs[0][2 % G, :] = 5                              # one constant cell (zero variance)
    seed, budget = 4321 + G, 1.0 / 128
    got = ctx.finalize128(outs, kv, meta, seed, budget, mode)
    y = np.stack([o.astype(np.float64) for o in outs], axis=1)   # [G, S, 128]
    ref = orc.finalize128(y, [orc.release_scale(k) for k, _, _ in kv], meta[:, 0], meta[:, 1:], seed, budget,
                          mode)
    np.testing.assert_array_equal(got["is_null"], ref["is_null"])
    np.testing.assert_array_equal(got["flags"], ref["flags"])
    live = ref["is_null"] == 0
    np.testing.assert_allclose(got["noised"][live], ref["noised"][live], rtol=1e-12, atol=0)
    np.testing.assert_allclose(got["posterior"], ref["posterior"], rtol=1e-10, atol=1e-15)


@pytest.mark.parametrize("mode", [B.PAC_FIN_ADAPTIVE, B.PAC_FIN_INDEPENDENT])
def test_finalize128_long_chain(ctx, mode):
    """2,500 groups of aggregate-like cells: the adaptive posterior over 128
    worlds collapses part-way, after which releases have variance 0."""
    G = 2500
    r = np.random.default_rng(1281)
    n = np.maximum(1, r.lognormal(6, 2, G)).astype(np.int64)
    cnt = r.binomial(n[:, None], 0.5, (G, 128)).astype(np.uint64)
    c = cnt.astype(np.float64)
    isum = (c * 500 + r.normal(0, 1, (G, 128)) * np.sqrt(c) * 290).astype(np.int64)
    fsum = c * 3.7 + r.normal(0, 1, (G, 128)) * np.sqrt(c) * 2.0
    meta = np.zeros((G, 3), dtype=np.uint64)
    meta[:, 0] = n
    meta[:, 1:] = np.uint64(0xFFFFFFFFFFFFFFFF)
    meta[n < 40, 2] = np.uint64(0x00FF00FF00FF00FF)
    kv = [(B.PAC_COUNT, 0, B.PAC_I64), (B.PAC_SUM, 0, B.PAC_I64), (B.PAC_SUM, 0, B.PAC_F64)]
    outs = [cnt, isum, fsum]
    got = ctx.finalize128(outs, kv, meta, 99, 1.0 / 128, mode)
    y = np.stack([o.astype(np.float64) for o in outs], axis=1)
    ref = orc.finalize128(y, [orc.release_scale(k) for k, _, _ in kv], meta[:, 0], meta[:, 1:], 99, 1.0 / 128,
                          mode)
    if mode == B.PAC_FIN_ADAPTIVE:
        assert ((ref["flags"] & orc.F_ZEROVAR) != 0).sum() > G      # the chain did collapse
    np.testing.assert_array_equal(got["is_null"], ref["is_null"])
    np.testing.assert_array_equal(got["flags"], ref["flags"])
    live = ref["is_null"] == 0
    np.testing.assert_allclose(got["noised"][live], ref["noised"][live], rtol=1e-12, atol=0)
    np.testing.assert_allclose(got["posterior"], ref["posterior"], rtol=1e-10, atol=1e-15)


def test_lowcard_60m_m128_full_size_sampled(ctx):
    """The 60M-row, 4-group, 4-column workload over 128 worlds, in the launch
    configuration the benchmark times (M = 128 tensor-core tiles): sampled
    worlds of both mask words against the oracle, every world against the
    balanced invariant (world 64 + j is the complement of world j)."""
    w = inputs.lowcard_60m(seed=0)
    k1, k2 = _keys2(0)
    specs = [(B.PAC_COUNT, 0, None)] + [(B.PAC_SUM, 0, v) for v in w.values]
    got, meta, st = ctx.aggregate128(w.keys, w.gids, 4, specs, qkey=k1, qkey2=k2)
    assert st == B.PAC_OK
    assert ctx.last_path == 2
    masks2 = orc.hash_keys128(w.keys, k1, k2, orc.BALANCED)
    for j in (0, 45, 64, 127):
        word = np.ascontiguousarray(masks2[:, j // 64])
        c, _ = orc.aggregate_world(word, None, w.gids, 4, B.PAC_COUNT, j % 64)
        np.testing.assert_array_equal(got[0][:, j], c)
        for k, v in enumerate(w.values):
            s, _ = orc.aggregate_world(word, v, w.gids, 4, B.PAC_SUM, j % 64)
            np.testing.assert_array_equal(got[1 + k][:, j], s)
    ng = np.bincount(w.gids, minlength=4).astype(np.uint64)
    np.testing.assert_array_equal(meta[:, 0], ng)
    cnt = got[0].astype(np.int64)
    assert np.all(cnt[:, :64] + cnt[:, 64:] == ng.astype(np.int64)[:, None])
    for k, v in enumerate(w.values):
        tot = np.array([v[w.gids == g].sum() for g in range(4)])
        assert np.all(got[1 + k][:, :64] + got[1 + k][:, 64:] == tot[:, None])
