"""GPU parity of PAC selection (Sec. 4.2 "PAC Selection"; Sec. 3.2
pac_select_<cmp>) against the oracle.

- pac_select: the selected masks bit-exact for every comparison, column type
  (int64 / float / double, with ties, NaN and signed zeros), one or many
  operand vectors (8-, 16- and 32-bit ids), keys or masks in, balanced or raw
  hash, ragged sizes; out-of-range operand ids keep no world and are
  reported.
- pac_aggregate_select: every aggregate over the selected rows equals the
  oracle's aggregate over the rows whose selected mask is non-zero (meta n_g
  counts only those), on the tensor-core path, the plain per-bit path, the
  per-bit engine (few and many groups) and the approximate cascade.
- PAC_IN_DROP_EMPTY on caller masks: rows with mask 0 belong to no group.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2603_15023_gb300 import binding as B

pytestmark = pytest.mark.gpu

VT = {np.dtype(np.int64): B.PAC_I64, np.dtype(np.float32): B.PAC_F32, np.dtype(np.float64): B.PAC_F64}
CMPS = [B.PAC_CMP_LT, B.PAC_CMP_LE, B.PAC_CMP_EQ, B.PAC_CMP_NE, B.PAC_CMP_GT, B.PAC_CMP_GE]


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


def _columns(seed, n, dtype, n_thr):
    """A compared column and operand vectors on one small domain, so that
    equal values are common; floats carry NaN and signed zeros."""
    r = np.random.default_rng(seed)
    col = r.integers(-30, 30, n).astype(dtype)
    thr = r.integers(-30, 30, (n_thr, 64)).astype(dtype)
    if np.dtype(dtype).kind == "f":
        col[r.random(n) < 0.01] = np.nan
        col[r.random(n) < 0.02] = -0.0
        thr[r.random(thr.shape) < 0.03] = np.nan
        thr[r.random(thr.shape) < 0.03] = -0.0
    return col, thr


class Sel:
    """Device copies of one selection's columns and its binding spec."""

    def __init__(self, col, cmp, thr, ids):
        self.dcol, self.dthr = dev(col), dev(thr)
        self.dids = dev(ids.view({1: np.uint8, 2: np.int16, 4: np.int32}[ids.dtype.itemsize])) \
            if ids is not None else None
        self.spec = B.make_select(self.dcol.data_ptr(), VT[col.dtype], cmp, self.dthr.data_ptr(), thr.shape[0],
                                  self.dids.data_ptr() if ids is not None else 0,
                                  ids.dtype.itemsize if ids is not None else 0)


def _gpu_select(ctx, first, in_flags, qk, sel, hash_mode=B.PAC_HASH_BALANCED):
    T = _t()
    n = first.shape[0]
    dk = dev(first.view(np.int64))
    out = T.zeros(max(n, 1), dtype=T.int64, device="cuda")
    inp = B.make_input(dk.data_ptr(), n, in_flags=in_flags, query_key=qk, hash_mode=hash_mode)
    B.pac_select(ctx, inp, sel.spec, out.data_ptr(), _stream())
    st = B.pac_sync_status(ctx, _stream())
    return out.cpu().numpy().view(np.uint64)[:n], st


@pytest.mark.parametrize("cmp", CMPS)
@pytest.mark.parametrize("dtype", [np.int64, np.float32, np.float64])
@pytest.mark.parametrize("n_thr,id_dtype", [(1, None), (3, np.uint8), (300, np.uint16), (70_000, np.uint32)])
def test_select_matches_oracle(ctx, cmp, dtype, n_thr, id_dtype):
    n = 70_001
    r = np.random.default_rng(n_thr)
    keys = r.integers(0, 9000, n).astype(np.int64)
    col, thr = _columns(cmp * 31 + n_thr, n, dtype, n_thr)
    ids = r.integers(0, n_thr, n).astype(id_dtype) if id_dtype is not None else None
    qk = orc.query_key(3)
    sel = Sel(col, cmp, thr, ids)
    got, st = _gpu_select(ctx, keys, B.PAC_IN_KEYS, qk, sel)
    assert st == B.PAC_OK
    ref, rst = orc.select(orc.hash_keys(keys, qk, orc.BALANCED), col, cmp, thr, ids)
    assert rst == 0
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("form", ["masks", "raw_hash"])
def test_select_masks_in_and_raw_hash(ctx, form):
    n = 33_333
    r = np.random.default_rng(7)
    col, thr = _columns(11, n, np.int64, 1)
    sel = Sel(col, B.PAC_CMP_GE, thr, None)
    if form == "masks":
        first = r.integers(0, 2**63, n, dtype=np.int64).astype(np.uint64) << np.uint64(1)
        got, st = _gpu_select(ctx, first, B.PAC_IN_MASKS, 0, sel)
        masks = first
    else:
        first = r.integers(0, 10**6, n).astype(np.int64)
        qk = orc.query_key(9)
        got, st = _gpu_select(ctx, first, B.PAC_IN_KEYS, qk, sel, hash_mode=B.PAC_HASH_RAW)
        masks = orc.hash_keys(first, qk, orc.RAW)
    assert st == B.PAC_OK
    np.testing.assert_array_equal(got, orc.select(masks, col, orc.GE, thr)[0])


def test_select_out_of_range_operand_ids(ctx):
    n = 5000
    r = np.random.default_rng(5)
    keys = r.integers(0, 900, n).astype(np.int64)
    col, thr = _columns(5, n, np.float64, 4)
    ids = r.integers(0, 4, n).astype(np.uint8)
    ids[::97] = 200
    sel = Sel(col, B.PAC_CMP_LT, thr, ids)
    got, st = _gpu_select(ctx, keys, B.PAC_IN_KEYS, 1, sel)
    assert st == B.PAC_E_INVALID
    ref, rst = orc.select(orc.hash_keys(keys, 1, orc.BALANCED), col, orc.LT, thr, ids)
    assert rst == 1
    np.testing.assert_array_equal(got, ref)
    assert np.all(got[::97] == 0)


def test_select_empty_and_bad_arguments(ctx):
    col, thr = _columns(1, 10, np.int64, 2)
    sel = Sel(col, B.PAC_CMP_EQ, thr, None)   # two vectors but no ids
    with pytest.raises(B.PacError) as e:
        _gpu_select(ctx, np.zeros(10, dtype=np.int64), B.PAC_IN_KEYS, 0, sel)
    assert e.value.status == B.PAC_E_INVALID
    ok = Sel(col, B.PAC_CMP_EQ, thr[:1], None)
    got, st = _gpu_select(ctx, np.zeros(0, dtype=np.int64), B.PAC_IN_KEYS, 0, ok)
    assert st == B.PAC_OK and got.shape == (0,)


def _out_np(kind, vtype):
    if kind == B.PAC_COUNT:
        return np.uint64
    if kind == B.PAC_AVG or vtype != B.PAC_I64:
        return np.float64
    return np.int64


def _aggregate_select(ctx, keys, gids, G, qk, sel, specs, path):
    """specs: (kind, variant, values ndarray or None).  Returns (outs, meta, status)."""
    T = _t()
    B.pac_set_option(ctx, "agg_path", path)
    n = keys.shape[0]
    dk, dg = dev(keys), dev(gids)
    keep, spec_t, outs = [dk, dg], [], []
    for kind, variant, vals in specs:
        vt = B.PAC_I64 if vals is None else VT[vals.dtype]
        dv = dev(vals) if vals is not None else None
        keep.append(dv)
        od = _out_np(kind, vt)
        o = T.full((G, 64), -7, dtype=T.int64 if od != np.float64 else T.float64, device="cuda")
        outs.append((o, od))
        spec_t.append((kind, variant, vt, dv.data_ptr() if dv is not None else 0, o.data_ptr()))
    meta = T.full((G, 2), -1, dtype=T.int64, device="cuda")
    inp = B.make_input(dk.data_ptr(), n, query_key=qk, group_ids=dg.data_ptr(), gid_bytes=gids.dtype.itemsize,
                       n_groups=G)
    sp = B.make_specs(spec_t)
    B.pac_aggregate_select(ctx, inp, sel.spec, sp, len(spec_t), meta.data_ptr(), _stream())
    st = B.pac_sync_status(ctx, _stream())
    path_used = B.pac_get_info(ctx, "last_path")
    B.pac_set_option(ctx, "agg_path", 0)
    return [o.cpu().numpy().view(od) for o, od in outs], meta.cpu().numpy().view(np.uint64), st, path_used


def _ref_aggregate(masks_sel, gids, G, specs):
    keep = masks_sel != 0
    res = []
    for kind, variant, vals in specs:
        v = None if vals is None else vals[keep]
        if variant == orc.APPROX:
            # dropped rows update nothing; the chunk schedule stays over row positions
            out, st = orc.approx_sum_i64(masks_sel, vals, gids, G, drop_empty=True)
            res.append(out)
            continue
        out, mn, mo, st = orc.aggregate(masks_sel[keep], v, gids[keep], G, kind)
        res.append(out)
    _, mn, mo, _ = orc.aggregate(masks_sel[keep], None, gids[keep], G, orc.COUNT)
    return res, mn, mo


@pytest.mark.parametrize("path,G,kinds", [
    (2, 5, "int"),        # tensor cores (<= 8 groups, COUNT / exact SUM / AVG)
    (1, 5, "all"),        # plain per-bit kernels
    (3, 5, "all"),        # per-bit engine, warp-private states
    (3, 3000, "all"),     # per-bit engine, partitioned rows
    (0, 20, "approx"),    # approximate integer SUM (cascade, <= 32 groups)
])
def test_aggregate_select_matches_oracle(ctx, path, G, kinds):
    n = 90_001
    r = np.random.default_rng(G + path)
    keys = r.integers(0, 20_000, n).astype(np.int64)
    gids = r.integers(0, G, n).astype(np.uint8 if G <= 255 else np.int32)
    v = r.integers(-10**6, 10**6, n).astype(np.int64)
    f = r.normal(0, 100, n)
    col = r.integers(0, 100, n).astype(np.int64)
    n_thr = 6
    thr = r.integers(0, 100, (n_thr, 64)).astype(np.int64)
    ids = (gids.astype(np.int64) % n_thr).astype(np.uint8)   # the row's correlation key
    sel = Sel(col, B.PAC_CMP_LT, thr, ids)
    specs = [(B.PAC_COUNT, 0, None), (B.PAC_SUM, 0, v), (B.PAC_AVG, 0, v)]
    if kinds == "all":
        specs += [(B.PAC_MIN, 0, v), (B.PAC_MAX, 0, f)]
    if kinds == "approx":
        specs = [(B.PAC_COUNT, 0, None), (B.PAC_SUM, B.PAC_APPROX, v)]
    qk = orc.query_key(21)
    got, meta, st, used = _aggregate_select(ctx, keys, gids, G, qk, sel, specs, path)
    assert st == B.PAC_OK
    if path:
        assert used == path
    masks_sel, _ = orc.select(orc.hash_keys(keys, qk, orc.BALANCED), col, orc.LT, thr, ids)
    assert 0 < int((masks_sel == 0).sum()) < n          # some rows are dropped, some kept
    ref, mn, mo = _ref_aggregate(masks_sel, gids, G, specs)
    for (kind, _, _), g_out, r_out in zip(specs, got, ref):
        np.testing.assert_array_equal(g_out, r_out, err_msg=f"kind {kind}")
    np.testing.assert_array_equal(meta[:, 0], mn)
    np.testing.assert_array_equal(meta[:, 1], mo)


@pytest.mark.parametrize("path", [1, 2, 3])
def test_drop_empty_on_caller_masks(ctx, path):
    """PAC_IN_MASKS | PAC_IN_DROP_EMPTY: rows with mask 0 count in no group;
    without the flag they still count in n_g."""
    T = _t()
    n, G = 50_003, 4
    r = np.random.default_rng(path)
    masks = r.integers(0, 2**63, n, dtype=np.int64).astype(np.uint64) << np.uint64(1)
    masks[r.random(n) < 0.3] = 0
    gids = r.integers(0, G, n).astype(np.uint8)
    v = r.integers(0, 1000, n).astype(np.int64)
    dm, dg, dv = dev(masks.view(np.int64)), dev(gids), dev(v)
    for flags in (B.PAC_IN_MASKS, B.PAC_IN_MASKS | B.PAC_IN_DROP_EMPTY):
        B.pac_set_option(ctx, "agg_path", path)
        oc = T.zeros((G, 64), dtype=T.int64, device="cuda")
        osum = T.zeros((G, 64), dtype=T.int64, device="cuda")
        meta = T.zeros((G, 2), dtype=T.int64, device="cuda")
        inp = B.make_input(dm.data_ptr(), n, in_flags=flags, group_ids=dg.data_ptr(), gid_bytes=1, n_groups=G)
        sp = B.make_specs([(B.PAC_COUNT, 0, B.PAC_I64, 0, oc.data_ptr()),
                           (B.PAC_SUM, 0, B.PAC_I64, dv.data_ptr(), osum.data_ptr())])
        B.pac_aggregate_multi(ctx, inp, sp, 2, meta.data_ptr(), _stream())
        assert B.pac_sync_status(ctx, _stream()) == B.PAC_OK
        B.pac_set_option(ctx, "agg_path", 0)
        keep = masks != 0 if flags & B.PAC_IN_DROP_EMPTY else np.ones(n, dtype=bool)
        rc, mn, mo, _ = orc.aggregate(masks[keep], None, gids[keep], G, orc.COUNT)
        rs, *_ = orc.aggregate(masks[keep], v[keep], gids[keep], G, orc.SUM)
        np.testing.assert_array_equal(oc.cpu().numpy().view(np.uint64), rc)
        np.testing.assert_array_equal(osum.cpu().numpy(), rs)
        np.testing.assert_array_equal(meta.cpu().numpy().view(np.uint64)[:, 0], mn)


def test_select_60m_full_size_sampled(ctx):
    """The 60M-row select workload at full size, as the benchmark runs it:
    operands = world j's exact AVG of column 0 per group (from the oracle, on
    the first 1M rows, which keeps it to seconds), pac_aggregate_select on the
    auto path (tensor cores); worlds 0, 21, 42 and 63 of COUNT and SUM
    against the oracle's aggregate of the selected rows, meta n_g for every
    group."""
    from paper_2603_15023_gb300 import inputs
    T = _t()
    w = inputs.lowcard_60m(seed=0)
    n, G = w.n, w.n_groups
    qk = orc.query_key(0)
    masks = orc.hash_keys(w.keys, qk, orc.BALANCED)
    m1 = 1_000_000
    avg, *_ = orc.aggregate(masks[:m1], w.values[0][:m1], w.gids[:m1], G, orc.AVG)
    thr = np.trunc(avg).astype(np.int64)
    sel_masks, st = orc.select(masks, w.values[0], orc.LT, thr, w.gids)
    assert st == 0
    keep = sel_masks != 0
    dk, dg = dev(w.keys), dev(w.gids)
    dv = [dev(v) for v in w.values]
    dthr = dev(thr)
    sel = B.make_select(dv[0].data_ptr(), B.PAC_I64, B.PAC_CMP_LT, dthr.data_ptr(), G, dg.data_ptr(), 1)
    outs = [T.zeros((G, 64), dtype=T.int64, device="cuda") for _ in range(5)]
    meta = T.zeros((G, 2), dtype=T.int64, device="cuda")
    specs = [(B.PAC_COUNT, 0, B.PAC_I64, 0, outs[0].data_ptr())]
    specs += [(B.PAC_SUM, 0, B.PAC_I64, dv[c].data_ptr(), outs[1 + c].data_ptr()) for c in range(4)]
    inp = B.make_input(dk.data_ptr(), n, query_key=qk, group_ids=dg.data_ptr(), gid_bytes=1, n_groups=G)
    B.pac_aggregate_select(ctx, inp, sel, B.make_specs(specs), 5, meta.data_ptr(), _stream())
    assert B.pac_sync_status(ctx, _stream()) == B.PAC_OK
    assert B.pac_get_info(ctx, "last_path") == 2
    got = [o.cpu().numpy() for o in outs]
    sm, sg = sel_masks[keep], w.gids[keep]
    for j in (0, 21, 42, 63):
        rc, st = orc.aggregate_world(sm, None, sg, G, orc.COUNT, j)
        np.testing.assert_array_equal(got[0][:, j].view(np.uint64), rc)
        for c in range(4):
            rs, st = orc.aggregate_world(sm, w.values[c][keep], sg, G, orc.SUM, j)
            np.testing.assert_array_equal(got[1 + c][:, j], rs)
    np.testing.assert_array_equal(meta.cpu().numpy()[:, 0], np.bincount(sg, minlength=G))
