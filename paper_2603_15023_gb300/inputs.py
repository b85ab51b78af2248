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


def ratio_100m(seed: int = 0, n: int = 100_000_000, n_groups: int = 1_000_000,
               n_keys: int = 10_000_000) -> Workload:
    """The highcard shape with the two sums of a market-share ratio (the
    Sec. 7 TPC-H Q08 form): v0 = sales where the row's nation is the chosen
    one (a quarter of the rows) else 0, v1 = sales."""
    w = highcard_100m(seed=seed, n=n, n_groups=n_groups, n_keys=n_keys)
    sales = w.values[0]
    chosen = _rng(seed, 3).random(n) < 0.25
    share_num = np.where(chosen, sales, 0).astype(np.int64)
    return Workload("ratio_100m", n, n_groups, w.keys, w.gids, [share_num, sales],
                    {"n_keys": n_keys, "zipf_s": 1.1, "chosen_fraction": 0.25})


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


def max_1g(seed: int = 0, n: int = 1_000_000_000, n_keys: int = 10_000_000,
           order: str = "random") -> Workload:
    """Sec. 6 MAX experiment shape: 1G rows, ungrouped, one int64 value column.
    order "random": values uniform in [0, 1e12]; "increasing": value = row
    index, the adversarial input of bound pruning for MAX (every row raises
    every world it belongs to)."""
    keys = uniform_i64(seed, 0, n, 0, n_keys - 1)
    if order == "increasing":
        vals = np.arange(n, dtype=np.int64)
    else:
        vals = uniform_i64(seed, 1, n, 0, 10**12)
    return Workload("max_1g" if order == "random" else "max_1g_" + order, n, 1, keys, None, [vals],
                    {"n_keys": n_keys, "order": order})


def max_1g_increasing(seed: int = 0, n: int = 1_000_000_000) -> Workload:
    return max_1g(seed, n, order="increasing")


def hash_100m(seed: int = 0, n: int = 100_000_000, n_keys: int = 10_000_000) -> Workload:
    """The key column of the high-cardinality shape alone: PU keys uniform over
    10M keys, for the standalone key-to-mask hash."""
    keys = uniform_i64(seed, 0, n, 0, n_keys - 1)
    return Workload("hash_100m", n, 1, keys, None, [], {"n_keys": n_keys})


WORKLOADS = {
    "hash_100m": hash_100m,
    "lowcard_60m_m128": lowcard_60m,  # the same columns over 128 worlds
    "ungrouped_1m": ungrouped_1m,
    "max_1g": max_1g,
    "max_1g_increasing": max_1g_increasing,
    "lowcard_60m": lowcard_60m,
    "select_60m": lowcard_60m,   # the same columns, read under a PAC selection
    "lowcard_60m_approx": lowcard_60m,  # the same columns, approximate SUM / AVG
    "ratio_100m": ratio_100m,
    "highcard_100m": highcard_100m,
}


# ---------------------------------------------------------------------------
# Counter-based columns (the host twin of the GPU generator in libpacgen.so):
# draw `row` of `column` under `seed` is mix(mix(seed + (column+1) G) + (row+1) G)
# with SplitMix64's output function `mix` and G its golden gamma.  Used for the
# batched workload, whose 4.45G rows are generated on the device; any sampled
# query can be regenerated here, bit for bit, for the oracle.
# ---------------------------------------------------------------------------
_G = np.uint64(0x9E3779B97F4A7C15)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def counter_u64(seed: int, column: int, rows: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        start = _mix(np.asarray([np.uint64(seed) + (np.uint64(column) + np.uint64(1)) * _G], dtype=np.uint64))[0]
        r = np.asarray(rows, dtype=np.uint64)
        return _mix(start + (r + np.uint64(1)) * _G)


def counter_i64(seed: int, column: int, n: int, lo: int, span: int, row0: int = 0) -> np.ndarray:
    u = counter_u64(seed, column, np.arange(row0, row0 + n, dtype=np.uint64))
    return (np.int64(lo) + (u % np.uint64(span)).astype(np.int64)).astype(np.int64)


def counter_u32(seed: int, column: int, n: int, span: int, row0: int = 0) -> np.ndarray:
    u = counter_u64(seed, column, np.arange(row0, row0 + n, dtype=np.uint64))
    return (u % np.uint64(span)).astype(np.uint32)


def counter_f32_1000(seed: int, column: int, n: int, row0: int = 0) -> np.ndarray:
    u = counter_u64(seed, column, np.arange(row0, row0 + n, dtype=np.uint64))
    return ((u >> np.uint64(40)).astype(np.float64) * (1000.0 / 16777216.0)).astype(np.float32)


@dataclass
class BatchSpec:
    """Shapes of the batched workload: per query rows, groups and PU-key
    domain; its columns come from the counter-based generator with column
    ids 4*q + {0: key, 1: group id, 2: int64 value, 3: float32 value}."""
    seed: int
    rows: np.ndarray     # int64 [Q]
    groups: np.ndarray   # int64 [Q]
    keys: np.ndarray     # int64 [Q]

    @property
    def n_queries(self) -> int:
        return int(self.rows.shape[0])

    def columns(self, q: int):
        """Host copy of query q's columns: keys int64, gids uint32, v int64, f float32."""
        n, G, K = int(self.rows[q]), int(self.groups[q]), int(self.keys[q])
        return (counter_i64(self.seed, 4 * q, n, 0, K), counter_u32(self.seed, 4 * q + 1, n, G),
                counter_i64(self.seed, 4 * q + 2, n, 1, 100_000), counter_f32_1000(self.seed, 4 * q + 3, n))


def _log_uniform(r: np.random.Generator, lo: float, hi: float, n: int) -> np.ndarray:
    return np.exp(r.uniform(np.log(lo), np.log(hi), n))


def batch_4096(seed: int = 0, n_queries: int = 4096, rows_lo: float = 1e3, rows_hi: float = 1e7,
               groups_hi: float = 1e4, keys_lo: float = 1e3, keys_hi: float = 1e6) -> BatchSpec:
    """4096 independent queries: rows log-uniform in [1e3, 1e7], groups
    log-uniform integers in [1, 1e4], PU keys uniform over a domain whose size
    is log-uniform in [1e3, 1e6]; int64 values uniform in [1, 1e5] and
    float32 values uniform in [0, 1000)."""
    r = _rng(seed, 1000)
    rows = np.rint(_log_uniform(r, rows_lo, rows_hi, n_queries)).astype(np.int64)
    groups = np.clip(np.rint(_log_uniform(r, 1.0, groups_hi, n_queries)), 1, groups_hi).astype(np.int64)
    keys = np.rint(_log_uniform(r, keys_lo, keys_hi, n_queries)).astype(np.int64)
    return BatchSpec(seed, rows, groups, keys)
