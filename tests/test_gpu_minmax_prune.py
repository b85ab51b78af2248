"""GPU parity of the MIN/MAX bound pruning (Sec. 5 "Pruning") on the per-bit
engine.

With pruning on (the default) and off, MIN and MAX of every world equal the
oracle's on random data (most rows pruned), on the adversarial monotone
orders (no row pruned), on heavy ties, and on floats with signed zeros,
infinities and NaN.  Few groups keep warp-private states; many groups
partition the rows by group and carry runs across batches.  Queries whose
loop also holds a SUM take the unpruned loop.  Values compare as numbers: -0
equals +0, because which zero a world keeps depends on the order in which
rows arrive.

On the 1G-row MAX workloads the bench times, the result is checked against
the oracle on the rows that decide it. With increasing values those are the
last rows of the column. With random values they are the rows of largest
value. Every world must hold at least one of those rows.
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
    B.pac_set_option(c.h, "minmax_prune", 1)
    c.close()


def _values(dist, n, vdtype, r):
    if dist == "random":
        v = r.integers(-10**12, 10**12, n) if vdtype == np.int64 else r.normal(0.0, 1e6, n)
    elif dist == "increasing":
        v = np.arange(n) - n // 2
    elif dist == "decreasing":
        v = n // 2 - np.arange(n)
    elif dist == "ties":
        v = r.integers(-3, 4, n)
    else:  # "specials": floats with signed zeros, NaN and infinities
        v = r.normal(0.0, 10.0, n)
        pick = r.integers(0, 40, n)
        v[pick == 0] = 0.0
        v[pick == 1] = -0.0
        v[pick == 2] = np.nan
        v[pick == 3] = np.inf
        v[pick == 4] = -np.inf
    return np.asarray(v).astype(vdtype)


CASES = [("random", np.int64), ("increasing", np.int64), ("decreasing", np.int64), ("ties", np.int64),
         ("random", np.float64), ("decreasing", np.float64), ("specials", np.float64)]


def _run(ctx, prune, keys, gids, G, specs, qk):
    B.pac_set_option(ctx.h, "minmax_prune", prune)
    try:
        return ctx.aggregate(keys, gids, G, specs, qkey=qk, path=3)
    finally:
        B.pac_set_option(ctx.h, "minmax_prune", 1)


@pytest.mark.parametrize("prune", [1, 0])
@pytest.mark.parametrize("G", [1, 4, 3000])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_minmax_matches_oracle(ctx, prune, G, case):
    dist, vdtype = CASES[case]
    n = 150_001
    r = np.random.default_rng(1000 * case + G)
    keys = r.integers(0, 20_000, n).astype(np.int64)
    gids = None if G == 1 else r.integers(0, G, n).astype(np.int32 if G > 255 else np.uint8)
    vals = _values(dist, n, vdtype, r)
    qk = orc.query_key(case)
    specs = [(B.PAC_COUNT, 0, None), (B.PAC_MIN, 0, vals), (B.PAC_MAX, 0, vals)]
    got, meta, st = _run(ctx, prune, keys, gids, G, specs, qk)
    assert st == B.PAC_OK
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    for (kind, _, v), g_out in zip(specs, got):
        ref, mn, mo, rst = orc.aggregate(masks, v, gids, G, kind)
        assert rst == 0
        np.testing.assert_array_equal(g_out, ref)
    np.testing.assert_array_equal(meta[:, 0], mn)


@pytest.mark.parametrize("extra", ["int_sum_looped", "float_sum"])
def test_minmax_beside_looped_sums(ctx, extra):
    """A SUM that the broadcast loop serves (negative int64 values are not
    bit-sliced; float sums always loop) keeps every row in the loop."""
    n, G = 120_007, 3
    r = np.random.default_rng(5)
    keys = r.integers(0, 9000, n).astype(np.int64)
    gids = r.integers(0, G, n).astype(np.uint8)
    iv = r.integers(-10**9, 10**9, n).astype(np.int64)
    fv = r.normal(0, 100.0, n).astype(np.float64)
    sv = iv if extra == "int_sum_looped" else fv
    specs = [(B.PAC_COUNT, 0, None), (B.PAC_SUM, 0, sv), (B.PAC_MAX, 0, iv), (B.PAC_MIN, 0, fv)]
    qk = orc.query_key(55)
    got, _, st = _run(ctx, 1, keys, gids, G, specs, qk)
    assert st == B.PAC_OK
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    for (kind, _, v), g_out in zip(specs, got):
        ref, *_ = orc.aggregate(masks, v, gids, G, kind)
        if kind == B.PAC_SUM and v.dtype == np.float64:
            absw, *_ = orc.aggregate(masks, np.abs(v), gids, G, B.PAC_SUM)
            assert np.all(np.abs(g_out - ref) <= 1e-6 * absw)
        else:
            np.testing.assert_array_equal(g_out, ref)


@pytest.mark.parametrize("workload", ["max_1g_increasing", "max_1g"])
def test_max_1g_full_size(ctx, workload):
    """The bench's 1G-row MAX workloads (rank 0's inputs and query key), in the
    bench's launch configuration (automatic path, pruning on)."""
    w = inputs.WORKLOADS[workload](seed=0)
    n, v = w.n, w.values[0]
    qk = orc.query_key(0)
    specs = [(B.PAC_COUNT, 0, None), (B.PAC_MAX, 0, v)]
    got, meta, st = ctx.aggregate(w.keys, None, 1, specs, qkey=qk)
    assert st == B.PAC_OK
    K = 4096
    idx = np.arange(n - K, n) if workload == "max_1g_increasing" else np.argpartition(v, n - K)[n - K:]
    sub = orc.hash_keys(w.keys[idx], qk, orc.BALANCED)
    cnt, *_ = orc.aggregate(sub, None, None, 1, orc.COUNT)
    assert np.all(cnt > 0)  # every world holds one of the deciding rows
    ref, *_ = orc.aggregate(sub, v[idx], None, 1, orc.MAX)
    np.testing.assert_array_equal(got[1], ref)
    c = got[0][0].astype(np.int64)
    assert np.all(c[:32] + c[32:] == n)  # balanced masks: worlds j and j+32 split every row
    assert int(meta[0, 0]) == n
