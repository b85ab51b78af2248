"""Seeded synthetic input columns shaped like the paper's workloads.

This module holds no part of the method: it only draws random columns (PU
keys, group ids, values) with numpy's PCG64, one independent stream per
column, so that the CUDA path and the CPU oracle can be fed the same inputs.
The method's own random numbers (the query key, the secret world, the noise)
are not drawn here.

Shapes follow the paper's micro-benchmarks (Sec. 6.1: N rows, uniform value
domains, K scattered GROUP BY keys) at the sizes of the three single-query
workloads:

* ``ungrouped_1m``: 1,000,000 rows, int64 PU key uniform over [0, 150000),
  int64 value uniform in [1, 100000], no GROUP BY.
* ``lowcard_60m``: 60,000,000 rows, uint8 group id over 4 groups with
  probabilities 0.25/0.25/0.49/0.01, PU key uniform over [0, 1.5M), four
  int64 decimal(12,2) columns in cents uniform in [100, 10^7].
* ``highcard_100m``: 100,000,000 rows, int32 group id = rank-1 of a
  Zipf(s=1.1) law over 10^6 groups, PU key uniform over [0, 10^7), int64
  value round(exp(8 + 2 z)) clipped to 2^40 (lognormal, mu=8, sigma=2).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np


def _rng(seed: int, column: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([int(seed), int(column)]))


@dataclass
class Workload:
    name: str
    n: int
    n_groups: int
    keys: np.ndarray                      # int64 [n]
    gids: Optional[np.ndarray]            # uint8/int32 [n] or None (ungrouped)
    values: List[np.ndarray] = field(default_factory=list)  # value columns
    meta: Dict[str, object] = field(default_factory=dict)


def uniform_i64(seed: int, column: int, n: int, lo: int, hi_inclusive: int) -> np.ndarray:
    return _rng(seed, column).integers(lo, hi_inclusive + 1, size=n, dtype=np.int64)


def ungrouped_1m(seed: int = 0, n: int = 1_000_000, n_keys: int = 150_000) -> Workload:
    keys = uniform_i64(seed, 0, n, 0, n_keys - 1)
    vals = uniform_i64(seed, 1, n, 1, 100_000)
    return Workload("ungrouped_1m", n, 1, keys, None, [vals],
                    {"n_keys": n_keys, "value_range": [1, 100_000]})


LOWCARD_PROBS = (0.25, 0.25, 0.49, 0.01)


def lowcard_groups(seed: int, column: int, n: int, probs=LOWCARD_PROBS) -> np.ndarray:
    u = _rng(seed, column).random(n)
    edges = np.cumsum(np.asarray(probs, dtype=np.float64))
    edges[-1] = 1.0
    return np.searchsorted(edges, u, side="right").astype(np.uint8)


def lowcard_60m(seed: int = 0, n: int = 60_000_000, n_keys: int = 1_500_000,
                n_value_cols: int = 4) -> Workload:
    gids = lowcard_groups(seed, 0, n)
    keys = uniform_i64(seed, 1, n, 0, n_keys - 1)
    vals = [uniform_i64(seed, 2 + c, n, 100, 10_000_000) for c in range(n_value_cols)]
    return Workload("lowcard_60m", n, len(LOWCARD_PROBS), keys, gids, vals,
                    {"n_keys": n_keys, "probs": list(LOWCARD_PROBS),
                     "value_range": [100, 10_000_000]})


def zipf_groups(seed: int, column: int, n: int, n_groups: int, s: float = 1.1) -> np.ndarray:
    ranks = np.arange(1, n_groups + 1, dtype=np.float64)
    w = ranks ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = _rng(seed, column).random(n)
    g = np.searchsorted(cdf, u, side="right")
    np.minimum(g, n_groups - 1, out=g)
    return g.astype(np.int32)


def lognormal_i64(seed: int, column: int, n: int, mu: float, sigma: float,
                  clip: int) -> np.ndarray:
    z = _rng(seed, column).standard_normal(n)
    v = np.exp(mu + sigma * z)
    np.minimum(v, float(clip), out=v)
    return np.rint(v).astype(np.int64)


def highcard_100m(seed: int = 0, n: int = 100_000_000, n_groups: int = 1_000_000,
                  n_keys: int = 10_000_000) -> Workload:
    gids = zipf_groups(seed, 0, n, n_groups)
    keys = uniform_i64(seed, 1, n, 0, n_keys - 1)
    vals = lognormal_i64(seed, 2, n, 8.0, 2.0, 1 << 40)
    return Workload("highcard_100m", n, n_groups, keys, gids, [vals],
                    {"n_keys": n_keys, "zipf_s": 1.1})


def small(seed: int, n: int, n_groups: int, n_keys: int, vdtype=np.int64,
          vlo: int = -1000, vhi: int = 1000, gid_dtype=np.int32) -> Workload:
    """Generic small case for the tests: uniform keys, uniform groups, values
    uniform in [vlo, vhi] (integers) or [vlo, vhi) (floats)."""
    keys = uniform_i64(seed, 0, n, 0, max(n_keys, 1) - 1)
    gids = None
    if n_groups > 1:
        gids = _rng(seed, 1).integers(0, n_groups, size=n).astype(gid_dtype)
    if np.dtype(vdtype).kind == "f":
        vals = (_rng(seed, 2).random(n) * (vhi - vlo) + vlo).astype(vdtype)
    else:
        vals = uniform_i64(seed, 2, n, vlo, vhi)
    return Workload("small", n, n_groups, keys, gids, [vals], {"n_keys": n_keys})


WORKLOADS = {
    "ungrouped_1m": ungrouped_1m,
    "lowcard_60m": lowcard_60m,
    "highcard_100m": highcard_100m,
}
