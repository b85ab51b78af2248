"""Helpers for the GPU parity tests: move numpy columns to the device, call
the C ABI through the binding, bring results back as numpy arrays."""
from __future__ import annotations

import numpy as np

from paper_2603_15023_gb300 import binding as B

_VT = {np.dtype(np.int64): B.PAC_I64, np.dtype(np.float32): B.PAC_F32, np.dtype(np.float64): B.PAC_F64}


def torch():
    import torch as T
    return T


def dev(a: np.ndarray):
    T = torch()
    return T.from_numpy(np.ascontiguousarray(a)).cuda()


def out_dtype(kind: int, vtype: int):
    if kind == B.PAC_COUNT:
        return np.uint64
    if kind == B.PAC_AVG:
        return np.float64
    return np.int64 if vtype == B.PAC_I64 else np.float64


def _torch_dtype(npdt):
    T = torch()
    return {np.dtype(np.uint64): T.int64, np.dtype(np.int64): T.int64, np.dtype(np.float64): T.float64}[np.dtype(npdt)]


class Ctx:
    def __init__(self, device: int = 0):
        self.h = B.pac_create(device)

    def close(self):
        if self.h:
            B.pac_destroy(self.h)
            self.h = 0

    def stream(self) -> int:
        return torch().cuda.current_stream().cuda_stream

    def hash_keys(self, keys: np.ndarray, qkey: int, mode: int, inplace: bool = False) -> np.ndarray:
        T = torch()
        dk = dev(keys.astype(np.int64))
        dm = dk if inplace else T.empty_like(dk)
        B.pac_hash_keys(self.h, dk.data_ptr(), dm.data_ptr(), keys.shape[0], qkey, mode, self.stream())
        return dm.cpu().numpy().view(np.uint64)

    def aggregate(self, first: np.ndarray, gids, n_groups: int, specs, *, in_flags=B.PAC_IN_KEYS,
                  hash_mode=B.PAC_HASH_BALANCED, qkey=0, want_meta=True, keep=None, path=0):
        """specs: list of (kind, variant, values ndarray or None).  path: 0 auto,
        1 per-bit, 2 tensor core.  Returns (outs list of ndarrays [G,64],
        meta [G,2] uint64 or None, status)."""
        T = torch()
        B.pac_set_option(self.h, "agg_path", path)
        n = first.shape[0]
        dfirst = dev(first.view(np.int64) if first.dtype == np.uint64 else first.astype(np.int64))
        dg = dev(gids) if gids is not None else None
        tensors = [dfirst, dg]
        cols = {}
        spec_t = []
        outs = []
        for kind, variant, vals in specs:
            if vals is None:
                vt, vp = B.PAC_I64, 0
            else:
                key = id(vals)
                if key not in cols:
                    cols[key] = dev(vals)
                vt = _VT[np.dtype(vals.dtype)]
                vp = cols[key].data_ptr()
            od = out_dtype(kind, vt)
            o = T.full((n_groups, 64), -7, dtype=_torch_dtype(od), device="cuda")
            outs.append((o, od))
            spec_t.append((kind, variant, vt, vp, o.data_ptr()))
        meta = T.full((n_groups, 2), -1, dtype=T.int64, device="cuda") if want_meta else None
        inp = B.make_input(dfirst.data_ptr(), n, in_flags=in_flags, hash_mode=hash_mode, query_key=qkey,
                           group_ids=dg.data_ptr() if dg is not None else 0,
                           gid_bytes=gids.dtype.itemsize if gids is not None else 0, n_groups=n_groups)
        sp = B.make_specs(spec_t)
        B.pac_aggregate_multi(self.h, inp, sp, len(spec_t), meta.data_ptr() if meta is not None else 0,
                              self.stream())
        st = B.pac_sync_status(self.h, self.stream())
        self.last_path = B.pac_get_info(self.h, "last_path")
        B.pac_set_option(self.h, "agg_path", 0)
        res = [o.cpu().numpy().view(od) for o, od in outs]
        m = meta.cpu().numpy().view(np.uint64) if meta is not None else None
        if keep is not None:
            keep.extend([tensors, cols, outs, meta, sp])
        return res, m, st

    def finalize(self, outs_np, kinds_variants_vtypes, meta_np, seed, budget, mode):
        """outs_np: list of [G,64] arrays (as the aggregate wrote them)."""
        T = torch()
        G = meta_np.shape[0]
        douts = []
        spec_t = []
        for arr, (kind, variant, vt) in zip(outs_np, kinds_variants_vtypes):
            d = dev(arr.view(np.int64) if arr.dtype == np.uint64 else arr)
            douts.append(d)
            spec_t.append((kind, variant, vt, 0, d.data_ptr()))
        sp = B.make_specs(spec_t)
        dmeta = dev(meta_np.view(np.int64))
        nc = G * len(spec_t)
        noised = T.zeros(nc, dtype=T.float64, device="cuda")
        is_null = T.zeros(nc, dtype=T.uint8, device="cuda")
        flags = T.zeros(nc, dtype=T.int32, device="cuda")
        post = T.zeros(64, dtype=T.float64, device="cuda")
        B.pac_finalize(self.h, sp, len(spec_t), G, dmeta.data_ptr(), seed, budget, mode, noised.data_ptr(),
                       is_null.data_ptr(), flags.data_ptr(), post.data_ptr(), self.stream())
        T.cuda.synchronize()
        return {"noised": noised.cpu().numpy(), "is_null": is_null.cpu().numpy(),
                "flags": flags.cpu().numpy().view(np.uint32), "posterior": post.cpu().numpy()}

    # ---- m = 128 worlds --------------------------------------------------
    def hash_keys128(self, keys: np.ndarray, k1: int, k2: int, mode: int) -> np.ndarray:
        T = torch()
        dk = dev(keys.astype(np.int64))
        dm = T.empty((keys.shape[0], 2), dtype=T.int64, device="cuda")
        B.pac_hash_keys128(self.h, dk.data_ptr(), dm.data_ptr(), keys.shape[0], k1, k2, mode, self.stream())
        return dm.cpu().numpy().view(np.uint64)

    def aggregate128(self, first: np.ndarray, gids, n_groups: int, specs, *, in_flags=B.PAC_IN_KEYS,
                     hash_mode=B.PAC_HASH_BALANCED, qkey=0, qkey2=0, path=0):
        """As aggregate(), over 128 worlds: first is [n] keys or [n, 2] masks.
        Returns (outs [G,128], meta [G,3] uint64, status)."""
        T = torch()
        B.pac_set_option(self.h, "agg_path", path)
        n = first.shape[0]
        dfirst = dev(first.view(np.int64) if first.dtype == np.uint64 else first.astype(np.int64))
        dg = dev(gids) if gids is not None else None
        cols, spec_t, outs = {}, [], []
        for kind, variant, vals in specs:
            if vals is None:
                vt, vp = B.PAC_I64, 0
            else:
                if id(vals) not in cols:
                    cols[id(vals)] = dev(vals)
                vt = _VT[np.dtype(vals.dtype)]
                vp = cols[id(vals)].data_ptr()
            od = out_dtype(kind, vt)
            o = T.full((n_groups, 128), -7, dtype=_torch_dtype(od), device="cuda")
            outs.append((o, od))
            spec_t.append((kind, variant, vt, vp, o.data_ptr()))
        meta = T.full((n_groups, 3), -1, dtype=T.int64, device="cuda")
        inp = B.make_input(dfirst.data_ptr() if n else 0, n, in_flags=in_flags, hash_mode=hash_mode,
                           query_key=qkey, group_ids=dg.data_ptr() if dg is not None and n else 0,
                           gid_bytes=gids.dtype.itemsize if gids is not None else 0, n_groups=n_groups)
        sp = B.make_specs(spec_t)
        try:
            B.pac_aggregate128(self.h, inp, qkey2, sp, len(spec_t), meta.data_ptr(), self.stream())
        finally:
            B.pac_set_option(self.h, "agg_path", 0)
        st = B.pac_sync_status(self.h, self.stream())
        self.last_path = B.pac_get_info(self.h, "last_path")
        res = [o.cpu().numpy().view(od) for o, od in outs]
        return res, meta.cpu().numpy().view(np.uint64), st

    def finalize128(self, outs_np, kinds_variants_vtypes, meta_np, seed, budget, mode):
        """outs_np: list of [G,128] arrays; meta_np [G,3] uint64."""
        T = torch()
        G = meta_np.shape[0]
        douts, spec_t = [], []
        for arr, (kind, variant, vt) in zip(outs_np, kinds_variants_vtypes):
            d = dev(arr.view(np.int64) if arr.dtype == np.uint64 else arr)
            douts.append(d)
            spec_t.append((kind, variant, vt, 0, d.data_ptr()))
        sp = B.make_specs(spec_t)
        dmeta = dev(np.ascontiguousarray(meta_np).view(np.int64))
        nc = G * len(spec_t)
        noised = T.zeros(nc, dtype=T.float64, device="cuda")
        is_null = T.zeros(nc, dtype=T.uint8, device="cuda")
        flags = T.zeros(nc, dtype=T.int32, device="cuda")
        post = T.zeros(128, dtype=T.float64, device="cuda")
        B.pac_finalize128(self.h, sp, len(spec_t), G, dmeta.data_ptr(), seed, budget, mode, noised.data_ptr(),
                          is_null.data_ptr(), flags.data_ptr(), post.data_ptr(), self.stream())
        T.cuda.synchronize()
        return {"noised": noised.cpu().numpy(), "is_null": is_null.cpu().numpy(),
                "flags": flags.cpu().numpy().view(np.uint32), "posterior": post.cpu().numpy()}
