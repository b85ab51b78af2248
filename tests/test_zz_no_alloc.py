"""pac_aggregate_noalloc: the aggregation for callers that cannot allocate.

Some callers cannot call cudaMalloc: code running under a memory pool that
owns all device memory (a database engine's buffer manager, a framework's
caching allocator) or under a device-memory budget fixed in advance, where an
allocation may fail or stall the device at the wrong time.  For them the
library offers pac_aggregate_noalloc, whose scratch is a fixed array compiled
into the library instead of memory it allocates.

These tests call it through the C ABI and check it against the CPU oracle's
exact definition (counts, int64 sums, the AVG doubles and the per-group
metadata, bit for bit) and against the ordinary entry point
pac_aggregate_multi.  The small queries run one after another with different
shapes (grouped with 1-, 2- and 4-byte group ids, ungrouped, COUNT only), so
whatever one call leaves in the shared scratch cannot leak into the next; one
query is large enough that the aggregation runs more blocks than the GPU has
SMs.  The file sorts last so that a run that stops at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2603_15023_gb300 import binding as B
from paper_2603_15023_gb300 import inputs

pytestmark = pytest.mark.gpu


def _case(seed, n, G, n_cols, gid_dtype, vlo=-(10**9), vhi=10**9):
    keys = inputs.uniform_i64(seed, 0, n, 0, max(n // 4, 1) - 1)
    gids = None
    if gid_dtype is not None:
        gids = inputs.uniform_i64(seed, 1, n, 0, G - 1).astype(gid_dtype)
    vals = [inputs.uniform_i64(seed, 2 + c, n, vlo, vhi) for c in range(n_cols)]
    return keys, gids, vals


def _specs(vals):
    """COUNT, a SUM per value column and the AVG of the first column."""
    kinds = [(B.PAC_COUNT, None)] + [(B.PAC_SUM, c) for c in range(len(vals))]
    if vals:
        kinds.append((B.PAC_AVG, 0))
    return kinds


def _run(keys, gids, G, vals, qkey, use_noalloc, ctx=None):
    import torch
    n = keys.shape[0]
    dk = torch.from_numpy(keys).cuda()
    dg = torch.from_numpy(gids).cuda() if gids is not None else None
    dv = [torch.from_numpy(v).cuda() for v in vals]
    outs, specs = [], []
    for kind, c in _specs(vals):
        dt = torch.float64 if kind == B.PAC_AVG else torch.int64
        o = torch.full((G, 64), -3, dtype=dt, device="cuda")
        outs.append(o)
        specs.append((kind, B.PAC_EXACT, B.PAC_I64, 0 if c is None else dv[c].data_ptr(), o.data_ptr()))
    meta = torch.full((G, 2), -3, dtype=torch.int64, device="cuda")
    inp = B.make_input(dk.data_ptr() if n else 0, n, query_key=qkey,
                       group_ids=dg.data_ptr() if dg is not None and n else 0,
                       gid_bytes=gids.dtype.itemsize if gids is not None else 0, n_groups=G)
    sp = B.make_specs(specs)
    stream = torch.cuda.current_stream().cuda_stream
    if use_noalloc:
        B.pac_aggregate_noalloc(inp, sp, len(specs), meta.data_ptr(), stream)
    else:
        B.pac_aggregate_multi(ctx, inp, sp, len(specs), meta.data_ptr(), stream)
        assert B.pac_sync_status(ctx, stream) == B.PAC_OK
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs], meta.cpu().numpy().view(np.uint64)


def _oracle(keys, gids, G, vals, qkey):
    masks = orc.hash_keys(keys, qkey, orc.BALANCED)
    exp = []
    mn = mo = None
    for kind, c in _specs(vals):
        out, n_g, or_g, st = orc.aggregate(masks, None if c is None else vals[c], gids, G, kind)
        assert st == 0
        exp.append(out.view(np.int64) if out.dtype == np.uint64 else out)
        mn, mo = n_g, or_g
    return exp, np.stack([mn, mo], axis=1)


# (seed, rows, groups, value columns, group-id type): grouped with 1-, 2- and
# 4-byte ids, COUNT only (the unused column slots read the key column), and
# ungrouped
SMALL_CASES = [(1, 300_007, 4, 4, np.uint8), (2, 77_777, 3, 1, np.uint16), (3, 50_001, 8, 0, np.uint32),
               (4, 120_000, 1, 2, None)]


def test_noalloc_matches_the_oracle_on_calls_in_a_row():
    ctx = B.pac_create(0)
    try:
        for seed, n, G, n_cols, gdt in SMALL_CASES:
            keys, gids, vals = _case(seed, n, G, n_cols, gdt)
            qk = B.pac_query_key(seed)
            got, gmeta = _run(keys, gids, G, vals, qk, use_noalloc=True)
            exp, emeta = _oracle(keys, gids, G, vals, qk)
            for a, b in zip(got, exp):
                np.testing.assert_array_equal(a, b)
            np.testing.assert_array_equal(gmeta, emeta)
            # and the allocating entry point gives the same, bit for bit
            ref, rmeta = _run(keys, gids, G, vals, qk, use_noalloc=False, ctx=ctx)
            for a, b in zip(got, ref):
                np.testing.assert_array_equal(a, b)
            np.testing.assert_array_equal(gmeta, rmeta)
    finally:
        B.pac_destroy(ctx)


def test_noalloc_more_blocks_than_sms():
    """A block aggregates at most 2^20 rows, so more than SMs x 2^20 rows
    run more blocks than there are SMs and every block adds into the one
    static scratch.  Sampled worlds against the oracle, every world against
    the balanced invariants (world j + 32 is the complement of world j)."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = sms * (1 << 20) + 100_003
    keys, _, vals = _case(5, n, 1, 1, None, vlo=1, vhi=100_000)
    qk = B.pac_query_key(5)
    got, gmeta = _run(keys, None, 1, vals, qk, use_noalloc=True)
    cnt, sm, avg = got
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    for j in (0, 17, 40, 63):
        c, _ = orc.aggregate_world(masks, None, None, 1, B.PAC_COUNT, j)
        s, _ = orc.aggregate_world(masks, vals[0], None, 1, B.PAC_SUM, j)
        a, _ = orc.aggregate_world(masks, vals[0], None, 1, B.PAC_AVG, j)
        assert cnt[0, j] == int(c[0]) and sm[0, j] == int(s[0]) and avg[0, j] == a[0]
    assert gmeta[0, 0] == n
    assert np.all(cnt[0, :32] + cnt[0, 32:] == n)
    assert np.all(sm[0, :32] + sm[0, 32:] == int(vals[0].sum()))


def test_noalloc_empty_input_and_what_it_cannot_serve():
    import torch
    # n = 0: every output and the metadata are zero
    got, gmeta = _run(np.zeros(0, np.int64), np.zeros(0, np.uint8), 3, [np.zeros(0, np.int64)], 1,
                      use_noalloc=True)
    for a in got:
        assert not a.any()
    assert not gmeta.any()

    keys, gids, vals = _case(6, 1000, 8, 4, np.uint8)
    dk = torch.from_numpy(keys).cuda()
    dg = torch.from_numpy(gids).cuda()
    dv = [torch.from_numpy(v).cuda() for v in vals]
    out = torch.full((8, 64), -3, dtype=torch.int64, device="cuda")
    # eight groups x four value columns exceed the fixed accumulator budget
    specs = B.make_specs([(B.PAC_SUM, B.PAC_EXACT, B.PAC_I64, v.data_ptr(), out.data_ptr()) for v in dv])
    inp = B.make_input(dk.data_ptr(), 1000, query_key=1, group_ids=dg.data_ptr(), gid_bytes=1, n_groups=8)
    with pytest.raises(B.PacError) as e:
        B.pac_aggregate_noalloc(inp, specs, 4, 0)
    assert e.value.status == B.PAC_E_UNSUPPORTED
    # kinds other than COUNT / exact int64 SUM / AVG are not served, and the
    # answer does not depend on the row count
    specs = B.make_specs([(B.PAC_MAX, B.PAC_EXACT, B.PAC_I64, dv[0].data_ptr(), out.data_ptr())])
    for n in (1000, 0):
        inp = B.make_input(dk.data_ptr(), n, query_key=1, group_ids=dg.data_ptr(), gid_bytes=1, n_groups=8)
        with pytest.raises(B.PacError) as e:
            B.pac_aggregate_noalloc(inp, specs, 1, 0)
        assert e.value.status == B.PAC_E_UNSUPPORTED
    torch.cuda.synchronize()
    assert bool((out == -3).all())
