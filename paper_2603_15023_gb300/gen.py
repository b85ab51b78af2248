"""ctypes binding of ``libpacgen.so`` (include/pac_gen.h): seeded synthetic
columns generated on the GPU for benchmarks and tests.  Not part of the PAC
method; the host twin of every mapping is in ``inputs.py``."""
from __future__ import annotations

import ctypes
import os
from typing import Optional

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpacgen.so")
_lib: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is not built; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, sz, u64, i64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64, ctypes.c_int64
        L.pacgen_fill_i64.argtypes = [vp, sz, u64, u64, u64, i64, u64, vp]
        L.pacgen_fill_u32.argtypes = [vp, sz, u64, u64, u64, u64, vp]
        L.pacgen_fill_f32_1000.argtypes = [vp, sz, u64, u64, u64, vp]
        for f in (L.pacgen_fill_i64, L.pacgen_fill_u32, L.pacgen_fill_f32_1000):
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def _ok(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"{what}: CUDA error {rc}")


def fill_i64(dst: int, n: int, seed: int, column: int, lo: int, span: int, row0: int = 0, stream: int = 0):
    _ok(lib().pacgen_fill_i64(dst, n, seed, column, row0, lo, span, stream), "pacgen_fill_i64")


def fill_u32(dst: int, n: int, seed: int, column: int, span: int, row0: int = 0, stream: int = 0):
    _ok(lib().pacgen_fill_u32(dst, n, seed, column, row0, span, stream), "pacgen_fill_u32")


def fill_f32_1000(dst: int, n: int, seed: int, column: int, row0: int = 0, stream: int = 0):
    _ok(lib().pacgen_fill_f32_1000(dst, n, seed, column, row0, stream), "pacgen_fill_f32_1000")
