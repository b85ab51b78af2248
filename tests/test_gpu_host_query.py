"""GPU parity of the end-to-end entry point pac_query_host (host columns in,
released cells out) against the oracle's aggregate followed by its release.

Below 16M rows the columns are copied and then aggregated; from 16M rows on
a query the tensor-core path serves alone is pipelined (row chunks copied on
a second stream, each aggregated once it has arrived).  Both forms must
release exactly what the oracle releases: NULL decisions and flags
bit-exact, values within 1e-12 relative.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2603_15023_gb300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    h = B.pac_create(0)
    yield h
    B.pac_destroy(h)


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("n,with_avg,pinned", [(100_003, True, False), (100_003, True, True),
                                               (17_000_001, False, False), (17_000_001, True, True)])
def test_query_host_matches_oracle(ctx, n, with_avg, pinned):
    """Pageable host columns are copied in; pinned ones are read where they
    are by the tensor-core aggregation."""
    r = np.random.default_rng(n)
    G = 4
    keys = r.integers(0, 1_500_000, n).astype(np.int64)
    gids = r.choice(G, n, p=[0.25, 0.25, 0.49, 0.01]).astype(np.uint8)
    v = r.integers(100, 10_000_000, n).astype(np.int64)
    keep = []
    if pinned:
        import torch
        hk, hg, hv = (torch.from_numpy(a).pin_memory() for a in (keys, gids, v))
        keep = [hk, hg, hv]
        kp, gp, vp = hk.data_ptr(), hg.data_ptr(), hv.data_ptr()
    else:
        kp, gp, vp = keys.ctypes.data, gids.ctypes.data, v.ctypes.data
    kinds = [B.PAC_COUNT, B.PAC_SUM] + ([B.PAC_AVG] if with_avg else [])
    specs = B.make_specs([(k, B.PAC_EXACT, B.PAC_I64, 0 if k == B.PAC_COUNT else vp, 1) for k in kinds])
    qk = orc.query_key(4)
    inp = B.make_input(kp, n, query_key=qk, group_ids=gp, gid_bytes=1, n_groups=G)
    cells = G * len(kinds)
    noised = np.zeros(cells, dtype=np.float64)
    is_null = np.zeros(cells, dtype=np.uint8)
    flags = np.zeros(cells, dtype=np.uint32)
    seed, budget = 321, 1.0 / 128
    B.pac_query_host(ctx, inp, specs, len(kinds), seed, budget, B.PAC_FIN_ADAPTIVE, noised.ctypes.data,
                     is_null.ctypes.data, flags.ctypes.data, _stream())
    assert B.pac_get_info(ctx, "last_path") == 2
    del keep
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    ys, mn, mo = [], None, None
    for k in kinds:
        out, mn, mo, st = orc.aggregate(masks, None if k == B.PAC_COUNT else v, gids, G, k)
        assert st == 0
        ys.append(out.astype(np.float64))
    ref = orc.finalize(np.stack(ys, axis=1), [orc.release_scale(k) for k in kinds], mn, mo, seed, budget,
                       orc.ADAPTIVE)
    np.testing.assert_array_equal(is_null, ref["is_null"])
    np.testing.assert_array_equal(flags, ref["flags"])
    live = ref["is_null"] == 0
    np.testing.assert_allclose(noised[live], ref["noised"][live], rtol=1e-12, atol=0)
