"""Thin ctypes binding of the C ABI in ``include/pac.h`` (``libpac.so``).

Function names are the C names; arguments are marshalled, nothing is
computed here.  Device buffers are passed as integer addresses (for example
``tensor.data_ptr()`` of a CUDA tensor) and streams as ``cudaStream_t``
handles (``torch.cuda.current_stream().cuda_stream``).  Loading fails loudly
when the library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpac.so")

PAC_OK, PAC_E_INVALID, PAC_E_NOMEM, PAC_E_CUDA, PAC_E_OVERFLOW, PAC_E_TIMEOUT, PAC_E_UNSUPPORTED = range(7)
PAC_COUNT, PAC_SUM, PAC_AVG, PAC_MIN, PAC_MAX, PAC_LIFTED = range(6)
(PAC_LIFT_SPEC, PAC_LIFT_CONST, PAC_LIFT_ADD, PAC_LIFT_SUB, PAC_LIFT_MUL, PAC_LIFT_DIV, PAC_LIFT_NEG,
 PAC_LIFT_ABS, PAC_LIFT_MIN, PAC_LIFT_MAX, PAC_LIFT_LT, PAC_LIFT_LE, PAC_LIFT_EQ, PAC_LIFT_NE, PAC_LIFT_GT,
 PAC_LIFT_GE) = range(16)
PAC_I64, PAC_F32, PAC_F64 = range(3)
PAC_EXACT, PAC_APPROX = 0, 1
PAC_HASH_BALANCED, PAC_HASH_RAW = 0, 1
PAC_FIN_ADAPTIVE, PAC_FIN_INDEPENDENT = 0, 1
PAC_IN_KEYS, PAC_IN_MASKS, PAC_IN_DROP_EMPTY = 0, 1, 2
PAC_CMP_LT, PAC_CMP_LE, PAC_CMP_EQ, PAC_CMP_NE, PAC_CMP_GT, PAC_CMP_GE = range(6)
PAC_F_NULL, PAC_F_DIVERSITY, PAC_F_ZEROVAR = 1, 2, 4
PAC_MAX_SPECS = 16

# every symbol the header declares
EXPORTED = (
    "pac_create", "pac_destroy", "pac_last_error", "pac_status_string", "pac_sync_status",
    "pac_query_key", "pac_hash_keys", "pac_aggregate", "pac_aggregate_multi", "pac_select",
    "pac_aggregate_select", "pac_finalize", "pac_lift", "pac_filter",
    "pac_query_host", "pac_set_option", "pac_get_info", "pac_aggregate_noalloc",
    "pac_batch_plan", "pac_batch_launch", "pac_batch_free", "pac_batch_info", "pac_batch_run",
    "pac_serve_create", "pac_serve_submit", "pac_serve_poll", "pac_serve_wait", "pac_serve_stats",
    "pac_serve_destroy", "pac_query_key2", "pac_hash_keys128", "pac_aggregate128", "pac_finalize128",
)
PAC_BATCH_AUTOTUNE = 1


class PacInput(ctypes.Structure):
    _fields_ = [
        ("keys_or_masks", ctypes.c_void_p),
        ("in_flags", ctypes.c_uint32),
        ("hash_mode", ctypes.c_int32),
        ("query_key", ctypes.c_uint64),
        ("group_ids", ctypes.c_void_p),
        ("gid_bytes", ctypes.c_int32),
        ("n_groups", ctypes.c_uint32),
        ("n", ctypes.c_size_t),
    ]


class PacSelectSpec(ctypes.Structure):
    _fields_ = [
        ("col", ctypes.c_void_p),
        ("vtype", ctypes.c_int32),
        ("cmp", ctypes.c_int32),
        ("thr", ctypes.c_void_p),
        ("n_thr", ctypes.c_uint32),
        ("thr_id_bytes", ctypes.c_int32),
        ("thr_ids", ctypes.c_void_p),
    ]


class PacLiftOp(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("arg", ctypes.c_int32), ("c", ctypes.c_double)]


class PacAggSpec(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("variant", ctypes.c_int32),
        ("vtype", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("values", ctypes.c_void_p),
        ("out", ctypes.c_void_p),
    ]


class PacQuery(ctypes.Structure):
    _fields_ = [
        ("in_", PacInput),
        ("specs", ctypes.POINTER(PacAggSpec)),
        ("n_specs", ctypes.c_int32),
        ("fin_mode", ctypes.c_int32),
        ("meta", ctypes.c_void_p),
        ("seed", ctypes.c_uint64),
        ("budget", ctypes.c_double),
        ("noised", ctypes.c_void_p),
        ("is_null", ctypes.c_void_p),
        ("flags", ctypes.c_void_p),
    ]


class PacServeConfig(ctypes.Structure):
    _fields_ = [
        ("mem_budget", ctypes.c_size_t),
        ("max_inflight", ctypes.c_int32),
        ("max_batch", ctypes.c_int32),
        ("n_streams", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class PacError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_name(status)}: {msg}")
        self.status = status


_lib: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    """Loads libpac.so (raises if it is missing: no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, u32, i32, u64, i64, sz, dbl = (ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int32, ctypes.c_uint64,
                                       ctypes.c_int64, ctypes.c_size_t, ctypes.c_double)
    sigs = {
        "pac_create": (i32, [ctypes.POINTER(vp), ctypes.c_int]),
        "pac_destroy": (None, [vp]),
        "pac_last_error": (ctypes.c_char_p, [vp]),
        "pac_status_string": (ctypes.c_char_p, [i32]),
        "pac_sync_status": (i32, [vp, vp]),
        "pac_query_key": (u64, [u64]),
        "pac_hash_keys": (i32, [vp, vp, vp, sz, u64, i32, vp]),
        "pac_aggregate": (i32, [vp, vp, u32, u64, i32, vp, i32, vp, i32, sz, u32, i32, i32, vp, vp, vp]),
        "pac_aggregate_multi": (i32, [vp, ctypes.POINTER(PacInput), ctypes.POINTER(PacAggSpec), i32, vp, vp]),
        "pac_select": (i32, [vp, ctypes.POINTER(PacInput), ctypes.POINTER(PacSelectSpec), vp, vp]),
        "pac_lift": (i32, [vp, ctypes.POINTER(PacAggSpec), i32, u32, ctypes.POINTER(PacLiftOp), i32, vp, vp]),
        "pac_filter": (i32, [vp, vp, u32, u64, vp, vp]),
        "pac_aggregate_select": (i32, [vp, ctypes.POINTER(PacInput), ctypes.POINTER(PacSelectSpec),
                                       ctypes.POINTER(PacAggSpec), i32, vp, vp]),
        "pac_finalize": (i32, [vp, ctypes.POINTER(PacAggSpec), i32, u32, vp, u64, dbl, i32, vp, vp, vp, vp, vp]),
        "pac_query_host": (i32, [vp, ctypes.POINTER(PacInput), ctypes.POINTER(PacAggSpec), i32, u64, dbl, i32,
                                 vp, vp, vp, vp]),
        "pac_set_option": (i32, [vp, ctypes.c_char_p, i64]),
        "pac_get_info": (i32, [vp, ctypes.c_char_p, ctypes.POINTER(i64)]),
        "pac_aggregate_noalloc": (i32, [ctypes.POINTER(PacInput), ctypes.POINTER(PacAggSpec), i32, vp, vp,
                                        ctypes.c_char_p, sz]),
        "pac_batch_plan": (i32, [vp, ctypes.POINTER(PacQuery), i32, u32, ctypes.POINTER(vp)]),
        "pac_batch_launch": (i32, [vp, vp, vp]),
        "pac_batch_free": (None, [vp]),
        "pac_batch_info": (i32, [vp, ctypes.c_char_p, ctypes.POINTER(i64)]),
        "pac_batch_run": (i32, [vp, ctypes.POINTER(PacQuery), i32, vp]),
        "pac_serve_create": (i32, [vp, ctypes.POINTER(PacServeConfig), ctypes.POINTER(vp)]),
        "pac_serve_submit": (i32, [vp, ctypes.POINTER(PacQuery), ctypes.POINTER(u64)]),
        "pac_serve_poll": (i32, [vp, u64, ctypes.POINTER(i32), ctypes.POINTER(dbl)]),
        "pac_serve_wait": (i32, [vp, u64, ctypes.POINTER(dbl)]),
        "pac_serve_stats": (i32, [vp, ctypes.c_char_p, ctypes.POINTER(dbl)]),
        "pac_serve_destroy": (None, [vp]),
        "pac_query_key2": (u64, [u64]),
        "pac_hash_keys128": (i32, [vp, vp, vp, sz, u64, u64, i32, vp]),
        "pac_aggregate128": (i32, [vp, ctypes.POINTER(PacInput), u64, ctypes.POINTER(PacAggSpec), i32, vp, vp]),
        "pac_finalize128": (i32, [vp, ctypes.POINTER(PacAggSpec), i32, u32, vp, u64, dbl, i32, vp, vp, vp, vp,
                                  vp]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def status_name(st: int) -> str:
    return lib().pac_status_string(st).decode()


def _check(ctx, st: int):
    if st != PAC_OK:
        msg = lib().pac_last_error(ctx).decode() if ctx else ""
        raise PacError(st, msg)


# ---- the C entry points, same names ---------------------------------------

def pac_create(device: int = 0) -> int:
    h = ctypes.c_void_p()
    st = lib().pac_create(ctypes.byref(h), device)
    if st != PAC_OK:
        raise PacError(st, f"pac_create(device={device})")
    return h.value


def pac_destroy(ctx: int) -> None:
    lib().pac_destroy(ctx)


def pac_last_error(ctx: int) -> str:
    return lib().pac_last_error(ctx).decode()


def pac_status_string(st: int) -> str:
    return status_name(st)


def pac_sync_status(ctx: int, stream: int = 0) -> int:
    """Returns the status code (does not raise on OVERFLOW/TIMEOUT)."""
    return lib().pac_sync_status(ctx, stream)


def pac_query_key(seed: int) -> int:
    return lib().pac_query_key(seed)


def pac_hash_keys(ctx: int, keys: int, masks: int, n: int, query_key: int, hash_mode: int,
                  stream: int = 0) -> None:
    _check(ctx, lib().pac_hash_keys(ctx, keys, masks, n, query_key, hash_mode, stream))


def pac_aggregate(ctx: int, keys_or_masks: int, in_flags: int, query_key: int, hash_mode: int,
                  values: int, vtype: int, group_ids: int, gid_bytes: int, n: int, n_groups: int,
                  kind: int, variant: int, out: int, meta: int, stream: int = 0) -> None:
    _check(ctx, lib().pac_aggregate(ctx, keys_or_masks, in_flags, query_key, hash_mode, values, vtype,
                                    group_ids, gid_bytes, n, n_groups, kind, variant, out, meta, stream))


def make_input(keys_or_masks: int, n: int, *, in_flags: int = PAC_IN_KEYS, hash_mode: int = PAC_HASH_BALANCED,
               query_key: int = 0, group_ids: int = 0, gid_bytes: int = 0, n_groups: int = 1) -> PacInput:
    return PacInput(keys_or_masks, in_flags, hash_mode, query_key, group_ids or None, gid_bytes, n_groups, n)


def make_specs(specs: Sequence[tuple]) -> ctypes.Array:
    """specs: (kind, variant, vtype, values_ptr, out_ptr) tuples."""
    arr = (PacAggSpec * max(len(specs), 1))()
    for i, (kind, variant, vtype, values, out) in enumerate(specs):
        arr[i] = PacAggSpec(kind, variant, vtype, 0, values or None, out)
    return arr


def pac_aggregate_multi(ctx: int, inp: PacInput, specs: ctypes.Array, n_specs: int, meta: int,
                        stream: int = 0) -> None:
    _check(ctx, lib().pac_aggregate_multi(ctx, ctypes.byref(inp), specs, n_specs, meta or None, stream))


def make_select(col: int, vtype: int, cmp: int, thr: int, n_thr: int = 1, thr_ids: int = 0,
                thr_id_bytes: int = 0) -> PacSelectSpec:
    return PacSelectSpec(col or None, vtype, cmp, thr or None, n_thr, thr_id_bytes, thr_ids or None)


def pac_select(ctx: int, inp: PacInput, sel: PacSelectSpec, masks_out: int, stream: int = 0) -> None:
    _check(ctx, lib().pac_select(ctx, ctypes.byref(inp), ctypes.byref(sel), masks_out or None, stream))


def pac_aggregate_select(ctx: int, inp: PacInput, sel: PacSelectSpec, specs: ctypes.Array, n_specs: int,
                         meta: int, stream: int = 0) -> None:
    _check(ctx, lib().pac_aggregate_select(ctx, ctypes.byref(inp), ctypes.byref(sel), specs, n_specs,
                                           meta or None, stream))


def make_lift(prog: Sequence[tuple]) -> ctypes.Array:
    """prog: (op, arg, c) tuples, postfix."""
    arr = (PacLiftOp * max(len(prog), 1))()
    for i, (op, arg, c) in enumerate(prog):
        arr[i] = PacLiftOp(op, arg, c)
    return arr


def pac_lift(ctx: int, specs: ctypes.Array, n_specs: int, n_groups: int, prog: ctypes.Array, n_ops: int,
             out: int, stream: int = 0) -> None:
    _check(ctx, lib().pac_lift(ctx, specs, n_specs, n_groups, prog, n_ops, out or None, stream))


def pac_filter(ctx: int, b: int, n_groups: int, seed: int, keep: int, stream: int = 0) -> None:
    _check(ctx, lib().pac_filter(ctx, b or None, n_groups, seed, keep or None, stream))


def pac_finalize(ctx: int, specs: ctypes.Array, n_specs: int, n_groups: int, meta: int, seed: int,
                 budget: float, mode: int, noised: int, is_null: int, flags: int, posterior: int,
                 stream: int = 0) -> None:
    _check(ctx, lib().pac_finalize(ctx, specs, n_specs, n_groups, meta, seed, budget, mode, noised, is_null,
                                   flags, posterior or None, stream))


def pac_query_key2(seed: int) -> int:
    return lib().pac_query_key2(seed)


def pac_hash_keys128(ctx: int, keys: int, masks: int, n: int, query_key: int, query_key2: int, hash_mode: int,
                     stream: int = 0) -> None:
    _check(ctx, lib().pac_hash_keys128(ctx, keys, masks, n, query_key, query_key2, hash_mode, stream))


def pac_aggregate128(ctx: int, inp: PacInput, query_key2: int, specs: ctypes.Array, n_specs: int, meta: int,
                     stream: int = 0) -> None:
    _check(ctx, lib().pac_aggregate128(ctx, ctypes.byref(inp), query_key2, specs, n_specs, meta or None, stream))


def pac_finalize128(ctx: int, specs: ctypes.Array, n_specs: int, n_groups: int, meta: int, seed: int,
                    budget: float, mode: int, noised: int, is_null: int, flags: int, posterior: int,
                    stream: int = 0) -> None:
    _check(ctx, lib().pac_finalize128(ctx, specs, n_specs, n_groups, meta, seed, budget, mode, noised, is_null,
                                      flags, posterior or None, stream))


def pac_query_host(ctx: int, inp: PacInput, specs: ctypes.Array, n_specs: int, seed: int, budget: float,
                   mode: int, noised: int, is_null: int, flags: int, stream: int = 0) -> None:
    _check(ctx, lib().pac_query_host(ctx, ctypes.byref(inp), specs, n_specs, seed, budget, mode, noised,
                                     is_null, flags, stream))


def pac_set_option(ctx: int, name: str, value: int) -> None:
    _check(ctx, lib().pac_set_option(ctx, name.encode(), value))


def pac_get_info(ctx: int, name: str) -> int:
    v = ctypes.c_int64(0)
    _check(ctx, lib().pac_get_info(ctx, name.encode(), ctypes.byref(v)))
    return v.value


def pac_aggregate_noalloc(inp: PacInput, specs: ctypes.Array, n_specs: int, meta: int, stream: int = 0) -> None:
    """The allocation-free aggregation (see include/pac.h); raises PacError."""
    buf = ctypes.create_string_buffer(512)
    st = lib().pac_aggregate_noalloc(ctypes.byref(inp), specs, n_specs, meta or None, stream, buf, len(buf))
    if st != PAC_OK:
        raise PacError(st, buf.value.decode())


def make_query(inp: PacInput, specs: ctypes.Array, n_specs: int, *, meta: int = 0, fin_mode: int = -1,
               seed: int = 0, budget: float = 1.0 / 128, noised: int = 0, is_null: int = 0,
               flags: int = 0) -> PacQuery:
    """One query of a batch; `specs` must outlive the plan call (it is copied there)."""
    return PacQuery(inp, ctypes.cast(specs, ctypes.POINTER(PacAggSpec)), n_specs, fin_mode, meta or None, seed,
                    budget, noised or None, is_null or None, flags or None)


def make_queries(qs: Sequence[PacQuery]) -> ctypes.Array:
    arr = (PacQuery * max(len(qs), 1))()
    for i, q in enumerate(qs):
        arr[i] = q
    return arr


def pac_batch_plan(ctx: int, queries: ctypes.Array, n_queries: int, flags: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(ctx, lib().pac_batch_plan(ctx, queries, n_queries, flags, ctypes.byref(h)))
    return h.value


def pac_batch_launch(ctx: int, plan: int, stream: int = 0) -> None:
    _check(ctx, lib().pac_batch_launch(ctx, plan, stream))


def pac_batch_free(plan: int) -> None:
    lib().pac_batch_free(plan)


def pac_batch_info(plan: int, name: str) -> int:
    v = ctypes.c_int64(0)
    st = lib().pac_batch_info(plan, name.encode(), ctypes.byref(v))
    if st != PAC_OK:
        raise PacError(st, f"pac_batch_info({name})")
    return v.value


def pac_batch_run(ctx: int, queries: ctypes.Array, n_queries: int, stream: int = 0) -> int:
    """Returns the status (device conditions included) instead of raising on them."""
    return lib().pac_batch_run(ctx, queries, n_queries, stream)


# ---- serving -------------------------------------------------------------

def pac_serve_create(ctx: int, mem_budget: int, max_inflight: int = 256, max_batch: int = 64,
                     n_streams: int = 2) -> int:
    h = ctypes.c_void_p()
    cfg = PacServeConfig(mem_budget, max_inflight, max_batch, n_streams, 0)
    _check(ctx, lib().pac_serve_create(ctx, ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def pac_serve_submit(srv: int, query: PacQuery) -> int:
    """Returns the ticket; raises PacError for a rejected query."""
    t = ctypes.c_uint64(0)
    st = lib().pac_serve_submit(srv, ctypes.byref(query), ctypes.byref(t))
    if st != PAC_OK:
        raise PacError(st, "pac_serve_submit")
    return t.value


def pac_serve_poll(srv: int, ticket: int):
    """(done, latency_ms, status) without blocking."""
    d, lat = ctypes.c_int32(0), ctypes.c_double(0.0)
    st = lib().pac_serve_poll(srv, ticket, ctypes.byref(d), ctypes.byref(lat))
    return bool(d.value), lat.value, st


def pac_serve_wait(srv: int, ticket: int):
    """(latency_ms, status); blocks until the ticket is done."""
    lat = ctypes.c_double(0.0)
    st = lib().pac_serve_wait(srv, ticket, ctypes.byref(lat))
    return lat.value, st


def pac_serve_stats(srv: int, name: str) -> float:
    v = ctypes.c_double(0.0)
    st = lib().pac_serve_stats(srv, name.encode(), ctypes.byref(v))
    if st != PAC_OK:
        raise PacError(st, f"pac_serve_stats({name})")
    return v.value


def pac_serve_destroy(srv: int) -> None:
    lib().pac_serve_destroy(srv)
