"""Plain scalar CPU oracle for PAC stochastic aggregation (SIMD-PAC-DB).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product path (``paper_2603_15023_gb300``) never imports it, and the two share
no code: this wrapper marshals numpy arrays into the C oracle in
``pac_oracle.c`` and nothing else.

Every function cites the passage of the paper it follows; the readings taken
where the paper is silent are listed at the top of ``pac_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pac_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

COUNT, SUM, AVG, MIN, MAX, LIFTED = 0, 1, 2, 3, 4, 5
I64, F32, F64 = 0, 1, 2
EXACT, APPROX = 0, 1
BALANCED, RAW = 0, 1
ADAPTIVE, INDEPENDENT = 0, 1
F_NULL, F_DIVERSITY, F_ZEROVAR = 1, 2, 4
APX_CHUNK = 4096

_lib: Optional[ctypes.CDLL] = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc into ``oracle/liboracle.so``."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "pac_oracle.h"))
    ):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        u64, i64, u32, i32, sz, vp, dbl = (
            ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int,
            ctypes.c_size_t, ctypes.c_void_p, ctypes.c_double,
        )
        sig = {
            "orc_fmix64": (u64, [u64]),
            "orc_fmix64_inverse": (u64, [u64]),
            "orc_query_key": (u64, [u64]),
            "orc_pac_hash": (u64, [i64, u64, i32]),
            "orc_hash_keys": (None, [vp, sz, u64, i32, vp]),
            "orc_rng_u64": (u64, [u64, u64, u64]),
            "orc_u01": (dbl, [u64]),
            "orc_u01_open0": (dbl, [u64]),
            "orc_box_muller": (dbl, [u64, u64]),
            "orc_aggregate_direct": (i32, [vp, vp, i32, vp, i32, sz, u32, i32, vp, vp, vp]),
            "orc_aggregate_world": (i32, [vp, vp, i32, vp, i32, sz, u32, i32, i32, vp]),
            "orc_aggregate_brute": (i32, [vp, u64, i32, vp, i32, vp, i32, sz, u32, i32, vp]),
            "orc_approx_sum_i64": (i32, [vp, vp, vp, i32, sz, u32, vp]),
            "orc_approx_avg_i64": (i32, [vp, vp, vp, i32, sz, u32, vp]),
            "orc_approx_sum_i64_ex": (i32, [vp, vp, vp, i32, sz, u32, vp, i32]),
            "orc_approx_avg_i64_ex": (i32, [vp, vp, vp, i32, sz, u32, vp, i32]),
            "orc_approx_sum_f32state": (i32, [vp, vp, i32, vp, i32, sz, u32, vp]),
            "orc_release_scale": (dbl, [i32, i32]),
            "orc_finalize": (None, [vp, vp, u32, u32, vp, vp, u64, dbl, i32, vp, vp, vp, vp, vp]),
            "orc_select": (i32, [vp, vp, i32, i32, vp, u32, vp, i32, sz, vp]),
            "orc_lift": (i32, [vp, vp, u32, u32, vp, i32, vp]),
            "orc_filter": (None, [vp, u32, u64, vp]),
            "orc_query_key2": (u64, [u64]),
            "orc_hash_keys128": (None, [vp, sz, u64, u64, i32, vp]),
            "orc_aggregate128": (i32, [vp, vp, i32, vp, i32, sz, u32, i32, vp, vp, vp]),
            "orc_aggregate_brute128": (i32, [vp, u64, u64, i32, vp, i32, vp, i32, sz, u32, i32, vp]),
            "orc_finalize128": (None, [vp, vp, u32, u32, vp, vp, u64, dbl, i32, vp, vp, vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _vtype(values: Optional[np.ndarray]) -> int:
    if values is None or values.dtype == np.int64:
        return I64
    if values.dtype == np.float32:
        return F32
    if values.dtype == np.float64:
        return F64
    raise TypeError(values.dtype)


def _out_dtype(kind: int, vtype: int):
    if kind == COUNT:
        return np.uint64
    if kind == AVG:
        return np.float64
    return np.int64 if vtype == I64 else np.float64


# -- PAC selection (Sec. 4.2 "PAC Selection"; Sec. 3.2 pac_select_<cmp>) ------
LT, LE, EQ, NE, GT, GE = 0, 1, 2, 3, 4, 5


def select(masks: np.ndarray, col: np.ndarray, cmp: int, thr: np.ndarray,
           thr_ids: Optional[np.ndarray] = None):
    """masks AND {world j : col[i] <cmp> thr[t_i][j]}.  thr: [n_thr, 64] of
    col's dtype; thr_ids: [n] uint8/uint16/uint32 row -> t_i (None when
    n_thr == 1).  Returns (selected masks uint64 [n], status)."""
    masks = np.ascontiguousarray(masks, dtype=np.uint64)
    col = np.ascontiguousarray(col)
    thr = np.ascontiguousarray(thr, dtype=col.dtype).reshape(-1, 64)
    tb = 0 if thr_ids is None else thr_ids.dtype.itemsize
    t = None if thr_ids is None else np.ascontiguousarray(thr_ids)
    out = np.zeros(masks.shape[0], dtype=np.uint64)
    st = lib().orc_select(_p(masks), _p(col), _vtype(col), cmp, _p(thr), thr.shape[0], _p(t), tb,
                          masks.shape[0], _p(out))
    return out, st


# -- vector-lifted expressions and pac_filter (Sec. 4.2; Sec. 3.2) -------------
(L_SPEC, L_CONST, L_ADD, L_SUB, L_MUL, L_DIV, L_NEG, L_ABS, L_MIN, L_MAX,
 L_LT, L_LE, L_EQ, L_NE, L_GT, L_GE) = range(16)
_LIFT_OP = np.dtype([("op", np.int32), ("arg", np.int32), ("c", np.float64)])


def lift(y: np.ndarray, scales, prog):
    """y: [n_groups, n_specs, 64] stored world results; scales: release scale
    per spec; prog: (op, arg, c) tuples, postfix.  Returns (out [n_groups, 64],
    status 0, or 1 for a malformed program)."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    G, S = y.shape[0], y.shape[1]
    sc = np.ascontiguousarray(np.asarray(scales, dtype=np.float64))
    p = np.array([tuple(t) for t in prog], dtype=_LIFT_OP)
    out = np.zeros((G, 64), dtype=np.float64)
    st = lib().orc_lift(_p(y), _p(sc), S, G, _p(p), len(prog), _p(out))
    return out, st


def pac_filter(b: np.ndarray, seed: int) -> np.ndarray:
    """b: [n_groups, 64] lifted booleans (true = non-zero).  Returns keep uint8 [n_groups]."""
    b = np.ascontiguousarray(b, dtype=np.float64)
    keep = np.zeros(b.shape[0], dtype=np.uint8)
    lib().orc_filter(_p(b), b.shape[0], seed, _p(keep))
    return keep


# -- hashing (Sec. 2 "SIMD-PAC-DB", Sec. 4.2 "PAC Hash") -----------------------

def fmix64(k: int) -> int:
    return lib().orc_fmix64(k)


def fmix64_inverse(h: int) -> int:
    return lib().orc_fmix64_inverse(h)


def query_key(seed: int) -> int:
    return lib().orc_query_key(seed)


def pac_hash(key: int, qkey: int, mode: int = BALANCED) -> int:
    return lib().orc_pac_hash(key, qkey, mode)


def hash_keys(keys: np.ndarray, qkey: int, mode: int = BALANCED) -> np.ndarray:
    keys = np.ascontiguousarray(keys, dtype=np.int64)
    out = np.empty(keys.shape[0], dtype=np.uint64)
    lib().orc_hash_keys(_p(keys), keys.shape[0], qkey, mode, _p(out))
    return out


def rng_u64(seed: int, stream: int, counter: int) -> int:
    return lib().orc_rng_u64(seed, stream, counter)


# -- aggregation (Sec. 4.2 "PAC Aggregation") -------------------------------

def _gid_args(gids: Optional[np.ndarray]):
    if gids is None:
        return None, 0
    gids = np.ascontiguousarray(gids)
    return gids, gids.dtype.itemsize


def aggregate(masks: np.ndarray, values: Optional[np.ndarray], gids: Optional[np.ndarray],
              n_groups: int, kind: int):
    """Exact definition, row by row.  Returns (out[n_groups,64], n_g, or_g, status)."""
    masks = np.ascontiguousarray(masks, dtype=np.uint64)
    values = None if values is None else np.ascontiguousarray(values)
    vt = _vtype(values)
    g, gb = _gid_args(gids)
    out = np.zeros((n_groups, 64), dtype=_out_dtype(kind, vt))
    mn = np.zeros(n_groups, dtype=np.uint64)
    mo = np.zeros(n_groups, dtype=np.uint64)
    st = lib().orc_aggregate_direct(_p(masks), _p(values), vt, _p(g), gb, masks.shape[0],
                                    n_groups, kind, _p(out), _p(mn), _p(mo))
    return out, mn, mo, st


def aggregate_world(masks: np.ndarray, values: Optional[np.ndarray], gids: Optional[np.ndarray],
                    n_groups: int, kind: int, world: int):
    """r_j of one world for every group.  Returns (out[n_groups], status)."""
    masks = np.ascontiguousarray(masks, dtype=np.uint64)
    values = None if values is None else np.ascontiguousarray(values)
    vt = _vtype(values)
    g, gb = _gid_args(gids)
    out = np.zeros(n_groups, dtype=_out_dtype(kind, vt))
    st = lib().orc_aggregate_world(_p(masks), _p(values), vt, _p(g), gb, masks.shape[0], n_groups,
                                   kind, world, _p(out))
    return out, st


def aggregate_brute(keys: np.ndarray, qkey: int, mode: int, values: Optional[np.ndarray],
                    gids: Optional[np.ndarray], n_groups: int, kind: int):
    """Same definition over 64 materialised subsamples.  Returns (out, status)."""
    keys = np.ascontiguousarray(keys, dtype=np.int64)
    values = None if values is None else np.ascontiguousarray(values)
    vt = _vtype(values)
    g, gb = _gid_args(gids)
    out = np.zeros((n_groups, 64), dtype=_out_dtype(kind, vt))
    st = lib().orc_aggregate_brute(_p(keys), qkey, mode, _p(values), vt, _p(g), gb,
                                   keys.shape[0], n_groups, kind, _p(out))
    return out, st


def approx_sum_i64(masks, values, gids, n_groups, drop_empty: bool = False):
    """Two-sided 25-level approximate integer SUM (Sec. 5 "Approximation").
    drop_empty: rows whose mask is 0 update nothing (filtered by a selection)."""
    masks = np.ascontiguousarray(masks, dtype=np.uint64)
    values = np.ascontiguousarray(values, dtype=np.int64)
    g, gb = _gid_args(gids)
    out = np.zeros((n_groups, 64), dtype=np.int64)
    st = lib().orc_approx_sum_i64_ex(_p(masks), _p(values), _p(g), gb, masks.shape[0], n_groups, _p(out),
                                     int(drop_empty))
    return out, st


def approx_avg_i64(masks, values, gids, n_groups, drop_empty: bool = False):
    masks = np.ascontiguousarray(masks, dtype=np.uint64)
    values = np.ascontiguousarray(values, dtype=np.int64)
    g, gb = _gid_args(gids)
    out = np.zeros((n_groups, 64), dtype=np.float64)
    st = lib().orc_approx_avg_i64_ex(_p(masks), _p(values), _p(g), gb, masks.shape[0], n_groups, _p(out),
                                     int(drop_empty))
    return out, st


def approx_sum_f32state(masks, values, gids, n_groups):
    masks = np.ascontiguousarray(masks, dtype=np.uint64)
    values = np.ascontiguousarray(values)
    vt = _vtype(values)
    g, gb = _gid_args(gids)
    out = np.zeros((n_groups, 64), dtype=np.float64)
    st = lib().orc_approx_sum_f32state(_p(masks), _p(values), vt, _p(g), gb, masks.shape[0],
                                       n_groups, _p(out))
    return out, st


# -- finalize (Sec. 4.1 noise function; Sec. 2; Sec. 3.2 "NULLs") --------------

def release_scale(kind: int, variant: int = EXACT) -> float:
    return lib().orc_release_scale(kind, variant)


def finalize(y: np.ndarray, scales, meta_n: np.ndarray, meta_or: np.ndarray, seed: int,
             budget: float, mode: int = ADAPTIVE):
    """y: [n_groups, n_specs, 64] unscaled results.  Returns dict of outputs."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    n_groups, n_specs = y.shape[0], y.shape[1]
    scales = np.ascontiguousarray(np.asarray(scales, dtype=np.float64))
    assert scales.shape == (n_specs,)
    meta_n = np.ascontiguousarray(meta_n, dtype=np.uint64)
    meta_or = np.ascontiguousarray(meta_or, dtype=np.uint64)
    nc = n_groups * n_specs
    noised = np.zeros(nc, dtype=np.float64)
    is_null = np.zeros(nc, dtype=np.uint8)
    flags = np.zeros(nc, dtype=np.uint32)
    post = np.zeros(64, dtype=np.float64)
    js = ctypes.c_int32(0)
    lib().orc_finalize(_p(y), _p(scales), n_specs, n_groups, _p(meta_n), _p(meta_or), seed,
                       budget, mode, _p(noised), _p(is_null), _p(flags), _p(post),
                       ctypes.byref(js))
    return {"noised": noised, "is_null": is_null, "flags": flags, "posterior": post,
            "jstar": js.value}


# -- m = 128 worlds (reading R7 of pac_oracle.c; Sec. 2 says m = 128 is possible) --

def query_key2(seed: int) -> int:
    """The second per-query key: the SplitMix64 output after K."""
    return lib().orc_query_key2(seed)


def hash_keys128(keys: np.ndarray, k1: int, k2: int, mode: int = BALANCED) -> np.ndarray:
    """[n, 2] uint64 world masks over 128 worlds (world j: bit j % 64 of word j // 64)."""
    keys = np.ascontiguousarray(keys, dtype=np.int64)
    out = np.empty((keys.shape[0], 2), dtype=np.uint64)
    lib().orc_hash_keys128(_p(keys), keys.shape[0], k1, k2, mode, _p(out))
    return out


def aggregate128(masks2: np.ndarray, values: Optional[np.ndarray], gids: Optional[np.ndarray],
                 n_groups: int, kind: int):
    """Exact definition over 128 worlds, row by row.  Returns (out[n_groups,128],
    n_g, or_g[n_groups,2], status)."""
    masks2 = np.ascontiguousarray(masks2, dtype=np.uint64).reshape(-1, 2)
    values = None if values is None else np.ascontiguousarray(values)
    vt = _vtype(values)
    g, gb = _gid_args(gids)
    out = np.zeros((n_groups, 128), dtype=_out_dtype(kind, vt))
    mn = np.zeros(n_groups, dtype=np.uint64)
    mo = np.zeros((n_groups, 2), dtype=np.uint64)
    st = lib().orc_aggregate128(_p(masks2), _p(values), vt, _p(g), gb, masks2.shape[0], n_groups, kind,
                                _p(out), _p(mn), _p(mo))
    return out, mn, mo, st


def aggregate_brute128(keys: np.ndarray, k1: int, k2: int, mode: int, values: Optional[np.ndarray],
                       gids: Optional[np.ndarray], n_groups: int, kind: int):
    """Same definition over 128 materialised subsamples.  Returns (out, status)."""
    keys = np.ascontiguousarray(keys, dtype=np.int64)
    values = None if values is None else np.ascontiguousarray(values)
    vt = _vtype(values)
    g, gb = _gid_args(gids)
    out = np.zeros((n_groups, 128), dtype=_out_dtype(kind, vt))
    st = lib().orc_aggregate_brute128(_p(keys), k1, k2, mode, _p(values), vt, _p(g), gb, keys.shape[0],
                                      n_groups, kind, _p(out))
    return out, st


def finalize128(y: np.ndarray, scales, meta_n: np.ndarray, meta_or2: np.ndarray, seed: int,
                budget: float, mode: int = ADAPTIVE):
    """y: [n_groups, n_specs, 128] unscaled results; meta_or2 [n_groups, 2]."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    n_groups, n_specs = y.shape[0], y.shape[1]
    scales = np.ascontiguousarray(np.asarray(scales, dtype=np.float64))
    assert scales.shape == (n_specs,) and y.shape[2] == 128
    meta_n = np.ascontiguousarray(meta_n, dtype=np.uint64)
    meta_or2 = np.ascontiguousarray(meta_or2, dtype=np.uint64).reshape(n_groups, 2)
    nc = n_groups * n_specs
    noised = np.zeros(nc, dtype=np.float64)
    is_null = np.zeros(nc, dtype=np.uint8)
    flags = np.zeros(nc, dtype=np.uint32)
    post = np.zeros(128, dtype=np.float64)
    js = ctypes.c_int32(0)
    lib().orc_finalize128(_p(y), _p(scales), n_specs, n_groups, _p(meta_n), _p(meta_or2), seed, budget, mode,
                          _p(noised), _p(is_null), _p(flags), _p(post), ctypes.byref(js))
    return {"noised": noised, "is_null": is_null, "flags": flags, "posterior": post, "jstar": js.value}
