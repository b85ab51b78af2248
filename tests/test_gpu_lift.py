"""GPU parity of vector-lifted expressions (pac_lift, Sec. 4.2), their single
release (pac_finalize with PAC_LIFTED) and pac_filter (Sec. 3.2) against the
oracle.

- pac_lift bit-exact against the oracle's program evaluation on the same
  stored world vectors (uint64 counts, int64 sums, double averages, earlier
  lifted vectors), IEEE division by zero included; malformed programs are
  refused before launch.
- A lifted vector released with pac_finalize (scale 1) matches the oracle's
  release of the same vector.
- pac_filter's keep decisions bit-exact.
- The Sec. 7 ratio query end to end on the GPU (aggregate -> lift ->
  release) against the same chain computed by the oracle alone.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2603_15023_gb300 import binding as B

pytestmark = pytest.mark.gpu


def _t():
    import torch
    return torch


def dev(a):
    return _t().from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def ctx():
    h = B.pac_create(0)
    yield h
    B.pac_destroy(h)


def _stream():
    return _t().cuda.current_stream().cuda_stream


def _vectors(G, seed):
    """Stored world vectors of four specs: COUNT (uint64), int64 SUM, AVG
    (double), float SUM (double)."""
    r = np.random.default_rng(seed)
    cnt = r.integers(0, 5000, (G, 64)).astype(np.uint64)
    cnt[0, :3] = 0
    sm = r.integers(-10**12, 10**12, (G, 64)).astype(np.int64)
    avg = r.normal(0, 50, (G, 64))
    fs = r.lognormal(2, 2, (G, 64))
    kinds = [(B.PAC_COUNT, B.PAC_I64), (B.PAC_SUM, B.PAC_I64), (B.PAC_AVG, B.PAC_I64), (B.PAC_SUM, B.PAC_F64)]
    return [cnt, sm, avg, fs], kinds


PROGRAMS = [
    [(B.PAC_LIFT_CONST, 0, 100.0), (B.PAC_LIFT_SPEC, 1, 0), (B.PAC_LIFT_MUL, 0, 0), (B.PAC_LIFT_SPEC, 0, 0),
     (B.PAC_LIFT_DIV, 0, 0)],
    [(B.PAC_LIFT_SPEC, 2, 0), (B.PAC_LIFT_SPEC, 3, 0), (B.PAC_LIFT_ADD, 0, 0), (B.PAC_LIFT_SPEC, 0, 0),
     (B.PAC_LIFT_SUB, 0, 0), (B.PAC_LIFT_NEG, 0, 0), (B.PAC_LIFT_ABS, 0, 0)],
    [(B.PAC_LIFT_SPEC, 2, 0), (B.PAC_LIFT_CONST, 0, 0.5), (B.PAC_LIFT_MIN, 0, 0), (B.PAC_LIFT_SPEC, 1, 0),
     (B.PAC_LIFT_MAX, 0, 0)],
    [(B.PAC_LIFT_SPEC, 1, 0), (B.PAC_LIFT_CONST, 0, 0.2), (B.PAC_LIFT_SPEC, 3, 0), (B.PAC_LIFT_MUL, 0, 0),
     (B.PAC_LIFT_LT, 0, 0)],
] + [[(B.PAC_LIFT_SPEC, 0, 0), (B.PAC_LIFT_SPEC, 2, 0), (op, 0, 0)]
     for op in (B.PAC_LIFT_LE, B.PAC_LIFT_EQ, B.PAC_LIFT_NE, B.PAC_LIFT_GT, B.PAC_LIFT_GE)]


def _gpu_lift(ctx, vecs, kinds, prog, G):
    T = _t()
    dv = [dev(v.view(np.int64) if v.dtype == np.uint64 else v) for v in vecs]
    specs = B.make_specs([(k, 0, vt, 0, d.data_ptr()) for (k, vt), d in zip(kinds, dv)])
    out = T.full((G, 64), -7.0, dtype=T.float64, device="cuda")
    lp = B.make_lift(prog)
    B.pac_lift(ctx, specs, len(kinds), G, lp, len(prog), out.data_ptr(), _stream())
    T.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("k", range(len(PROGRAMS)))
@pytest.mark.parametrize("G", [1, 333, 20_000])
def test_lift_matches_oracle(ctx, k, G):
    vecs, kinds = _vectors(G, k + G)
    got = _gpu_lift(ctx, vecs, kinds, PROGRAMS[k], G)
    y = np.stack([v.astype(np.float64) for v in vecs], axis=1)
    ref, st = orc.lift(y, [orc.release_scale(kd) for kd, _ in kinds], PROGRAMS[k])
    assert st == 0
    np.testing.assert_array_equal(got, ref)


def test_lift_of_a_lifted_vector(ctx):
    G = 500
    vecs, kinds = _vectors(G, 9)
    first = _gpu_lift(ctx, vecs, kinds, PROGRAMS[0], G)
    r = np.random.default_rng(1)
    lifted_in = r.normal(0, 10, (G, 64))                    # a stored lifted vector (host-made)
    got = _gpu_lift(ctx, [lifted_in, vecs[0]], [(B.PAC_LIFTED, B.PAC_F64), kinds[0]],
                    [(B.PAC_LIFT_SPEC, 0, 0), (B.PAC_LIFT_SPEC, 1, 0), (B.PAC_LIFT_DIV, 0, 0)], G)
    y = np.stack([lifted_in, vecs[0].astype(np.float64)], axis=1)
    ref, _ = orc.lift(y, [orc.release_scale(orc.LIFTED), orc.release_scale(orc.COUNT)],
                      [(orc.L_SPEC, 0, 0), (orc.L_SPEC, 1, 0), (orc.L_DIV, 0, 0)])
    np.testing.assert_array_equal(got, ref)
    assert np.isfinite(first).any()


@pytest.mark.parametrize("prog", [
    [(B.PAC_LIFT_ADD, 0, 0)],
    [(B.PAC_LIFT_SPEC, 0, 0), (B.PAC_LIFT_SPEC, 1, 0)],
    [(B.PAC_LIFT_SPEC, 9, 0)],
    [(B.PAC_LIFT_CONST, 0, 1.0)] * 9 + [(B.PAC_LIFT_ADD, 0, 0)] * 8,
    [(77, 0, 0)],
])
def test_lift_refuses_malformed_programs(ctx, prog):
    vecs, kinds = _vectors(3, 1)
    with pytest.raises(B.PacError) as e:
        _gpu_lift(ctx, vecs, kinds, prog, 3)
    assert e.value.status == B.PAC_E_INVALID


@pytest.mark.parametrize("mode", [B.PAC_FIN_ADAPTIVE, B.PAC_FIN_INDEPENDENT])
def test_lifted_release_matches_oracle(ctx, mode):
    T = _t()
    G = 300
    r = np.random.default_rng(mode)
    lifted = r.normal(0.3, 0.02, (G, 64))                    # market shares of 64 worlds
    meta = np.zeros((G, 2), dtype=np.uint64)
    meta[:, 0] = r.integers(0, 500, G)
    meta[:, 1] = np.uint64(0xFFFFFFFFFFFFFFFF)
    meta[::7, 1] = np.uint64(0x0F0F0F0F0F0F0F0F)
    dl, dm = dev(lifted), dev(meta.view(np.int64))
    specs = B.make_specs([(B.PAC_LIFTED, 0, B.PAC_F64, 0, dl.data_ptr())])
    noised = T.zeros(G, dtype=T.float64, device="cuda")
    is_null = T.zeros(G, dtype=T.uint8, device="cuda")
    flags = T.zeros(G, dtype=T.int32, device="cuda")
    post = T.zeros(64, dtype=T.float64, device="cuda")
    B.pac_finalize(ctx, specs, 1, G, dm.data_ptr(), 55, 1.0 / 128, mode, noised.data_ptr(), is_null.data_ptr(),
                   flags.data_ptr(), post.data_ptr(), _stream())
    T.cuda.synchronize()
    ref = orc.finalize(lifted[:, None, :], [orc.release_scale(orc.LIFTED)], meta[:, 0], meta[:, 1], 55,
                       1.0 / 128, mode)
    np.testing.assert_array_equal(is_null.cpu().numpy(), ref["is_null"])
    np.testing.assert_array_equal(flags.cpu().numpy().view(np.uint32), ref["flags"])
    live = ref["is_null"] == 0
    np.testing.assert_allclose(noised.cpu().numpy()[live], ref["noised"][live], rtol=1e-12, atol=0)
    np.testing.assert_allclose(post.cpu().numpy(), ref["posterior"], rtol=1e-10, atol=1e-15)


@pytest.mark.parametrize("G", [1, 1000, 100_003])
def test_filter_matches_oracle(ctx, G):
    T = _t()
    r = np.random.default_rng(G)
    b = (r.random((G, 64)) < r.random((G, 1))).astype(np.float64)
    b[0] = 0.0
    if G > 1:
        b[1] = 1.0
    keep = T.zeros(G, dtype=T.uint8, device="cuda")
    B.pac_filter(ctx, dev(b).data_ptr(), G, 42, keep.data_ptr(), _stream())
    T.cuda.synchronize()
    np.testing.assert_array_equal(keep.cpu().numpy(), orc.pac_filter(b, 42))


def test_ratio_query_end_to_end(ctx):
    """Sec. 7 (TPC-H Q08 shape): share = sum(sales if nation = X) / sum(sales)
    per group, lifted world by world and released once, on the GPU
    (pac_aggregate_multi -> pac_lift -> pac_finalize) and in the oracle."""
    T = _t()
    r = np.random.default_rng(3)
    n, G = 300_000, 7
    keys = r.integers(0, 40_000, n).astype(np.int64)
    gids = r.integers(0, G, n).astype(np.uint8)
    sales = r.integers(1, 100_000, n).astype(np.int64)
    brazil = np.where(r.random(n) < 0.25, sales, 0).astype(np.int64)
    qk = orc.query_key(12)
    dk, dg, ds, db = dev(keys), dev(gids), dev(sales), dev(brazil)
    o_b = T.zeros((G, 64), dtype=T.int64, device="cuda")
    o_a = T.zeros((G, 64), dtype=T.int64, device="cuda")
    meta = T.zeros((G, 2), dtype=T.int64, device="cuda")
    inp = B.make_input(dk.data_ptr(), n, query_key=qk, group_ids=dg.data_ptr(), gid_bytes=1, n_groups=G)
    agg = B.make_specs([(B.PAC_SUM, 0, B.PAC_I64, db.data_ptr(), o_b.data_ptr()),
                        (B.PAC_SUM, 0, B.PAC_I64, ds.data_ptr(), o_a.data_ptr())])
    B.pac_aggregate_multi(ctx, inp, agg, 2, meta.data_ptr(), _stream())
    share = T.zeros((G, 64), dtype=T.float64, device="cuda")
    prog = [(B.PAC_LIFT_SPEC, 0, 0), (B.PAC_LIFT_SPEC, 1, 0), (B.PAC_LIFT_DIV, 0, 0)]
    B.pac_lift(ctx, agg, 2, G, B.make_lift(prog), 3, share.data_ptr(), _stream())
    rel = B.make_specs([(B.PAC_LIFTED, 0, B.PAC_F64, 0, share.data_ptr())])
    noised = T.zeros(G, dtype=T.float64, device="cuda")
    is_null = T.zeros(G, dtype=T.uint8, device="cuda")
    flags = T.zeros(G, dtype=T.int32, device="cuda")
    B.pac_finalize(ctx, rel, 1, G, meta.data_ptr(), 77, 1.0 / 128, B.PAC_FIN_ADAPTIVE, noised.data_ptr(),
                   is_null.data_ptr(), flags.data_ptr(), 0, _stream())
    assert B.pac_sync_status(ctx, _stream()) == B.PAC_OK
    masks = orc.hash_keys(keys, qk, orc.BALANCED)
    rb, mn, mo, _ = orc.aggregate(masks, brazil, gids, G, orc.SUM)
    ra, *_ = orc.aggregate(masks, sales, gids, G, orc.SUM)
    y = np.stack([rb, ra], axis=1).astype(np.float64)
    sh, _ = orc.lift(y, [orc.release_scale(orc.SUM)] * 2, [(orc.L_SPEC, 0, 0), (orc.L_SPEC, 1, 0), (orc.L_DIV, 0, 0)])
    np.testing.assert_array_equal(share.cpu().numpy(), sh)
    ref = orc.finalize(sh[:, None, :], [1.0], mn, mo, 77, 1.0 / 128, orc.ADAPTIVE)
    np.testing.assert_array_equal(is_null.cpu().numpy(), ref["is_null"])
    np.testing.assert_array_equal(flags.cpu().numpy().view(np.uint32), ref["flags"])
    live = ref["is_null"] == 0
    np.testing.assert_allclose(noised.cpu().numpy()[live], ref["noised"][live], rtol=1e-12, atol=0)
