"""pac_aggregate_noalloc: the aggregation for callers that cannot allocate.

Some callers cannot call cudaMalloc: code running under a memory pool that
owns all device memory (a database engine's buffer manager, a framework's
caching allocator) or under a device-memory budget fixed in advance, where an
allocation may fail or stall the device at the wrong time.  For them the
library offers pac_aggregate_noalloc, whose scratch is a fixed array compiled
into the library instead of memory it allocates.

These tests call it through the C ABI and check that it gives exactly what
the ordinary entry point pac_aggregate_multi gives (bit for bit: counts,
int64 sums, the AVG doubles and the per-group metadata), on two calls in a
row with different inputs, so that whatever the first call left in the shared
scratch cannot leak into the second.  The file sorts last so that a run that
stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2603_15023_gb300 import binding as B
from paper_2603_15023_gb300 import inputs

pytestmark = pytest.mark.gpu


def _case(seed, n, G, n_cols):
    r = np.random.default_rng(seed)
    keys = r.integers(0, max(n // 4, 1), n).astype(np.int64)
    gids = r.integers(0, G, n).astype(np.uint8) if G > 1 else None
    vals = [r.integers(-(10**9), 10**9, n).astype(np.int64) for _ in range(n_cols)]
    return keys, gids, vals


def _run(keys, gids, G, vals, qkey, use_noalloc, ctx=None):
    import torch
    n = keys.shape[0]
    dk = torch.from_numpy(keys).cuda()
    dg = torch.from_numpy(gids).cuda() if gids is not None else None
    dv = [torch.from_numpy(v).cuda() for v in vals]
    outs = [torch.full((G, 64), -3, dtype=torch.int64, device="cuda")]
    specs = [(B.PAC_COUNT, B.PAC_EXACT, B.PAC_I64, 0, outs[0].data_ptr())]
    for v in dv:
        o = torch.full((G, 64), -3, dtype=torch.int64, device="cuda")
        outs.append(o)
        specs.append((B.PAC_SUM, B.PAC_EXACT, B.PAC_I64, v.data_ptr(), o.data_ptr()))
    if dv:
        o = torch.full((G, 64), -3.0, dtype=torch.float64, device="cuda")
        outs.append(o)
        specs.append((B.PAC_AVG, B.PAC_EXACT, B.PAC_I64, dv[0].data_ptr(), o.data_ptr()))
    meta = torch.full((G, 2), -3, dtype=torch.int64, device="cuda")
    inp = B.make_input(dk.data_ptr(), n, query_key=qkey, group_ids=dg.data_ptr() if dg is not None else 0,
                       gid_bytes=1 if dg is not None else 0, n_groups=G)
    sp = B.make_specs(specs)
    stream = torch.cuda.current_stream().cuda_stream
    if use_noalloc:
        B.pac_aggregate_noalloc(inp, sp, len(specs), meta.data_ptr(), stream)
    else:
        B.pac_aggregate_multi(ctx, inp, sp, len(specs), meta.data_ptr(), stream)
        assert B.pac_sync_status(ctx, stream) == B.PAC_OK
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs], meta.cpu().numpy()


def test_noalloc_matches_the_allocating_entry_point_twice_in_a_row():
    ctx = B.pac_create(0)
    try:
        cases = [(1, 300_007, 4, 4), (2, 77_777, 3, 1)]   # second call: other sizes and groups
        for seed, n, G, n_cols in cases:
            keys, gids, vals = _case(seed, n, G, n_cols)
            qk = B.pac_query_key(seed)
            got, gmeta = _run(keys, gids, G, vals, qk, use_noalloc=True)
            ref, rmeta = _run(keys, gids, G, vals, qk, use_noalloc=False, ctx=ctx)
            for a, b in zip(got, ref):
                np.testing.assert_array_equal(a, b)
            np.testing.assert_array_equal(gmeta, rmeta)
    finally:
        B.pac_destroy(ctx)


def test_noalloc_rejects_what_it_cannot_serve():
    import torch
    keys, gids, vals = _case(3, 1000, 8, 4)
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
    torch.cuda.synchronize()
    assert bool((out == -3).all())
    # kinds other than COUNT / exact int64 SUM / AVG are not served either
    specs = B.make_specs([(B.PAC_MAX, B.PAC_EXACT, B.PAC_I64, dv[0].data_ptr(), out.data_ptr())])
    with pytest.raises(B.PacError) as e:
        B.pac_aggregate_noalloc(inp, specs, 1, 0)
    assert e.value.status == B.PAC_E_UNSUPPORTED
