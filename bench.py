"""Benchmark of the PAC stochastic-aggregation hot path on GB300.

One step = one PAC query over a synthetic workload resident in HBM: the hash
of the PU keys (fused into the aggregation), the per-group per-world
aggregates over the m = 64 worlds, and the release of every cell (variance
under the posterior + PAC noise).  Workloads (``--workload``):

* ``lowcard_60m`` (default, the headline): 60M rows, 4 groups (uint8),
  COUNT + 4 exact SUMs + 4 exact AVGs of int64 cents, adaptive finalize of
  the 36 cells.  Inputs 2.46 GB > L2, no flush needed.
* ``ungrouped_1m``: 1M rows, no GROUP BY, COUNT + exact SUM, adaptive
  finalize of 2 cells.  The 16 MB input fits in L2, so L2 is flushed
  (a 512 MB write) before every step, outside the step's events.
* ``highcard_100m``: 100M rows, Zipf(1.1) over 1M groups (int32), COUNT +
  exact SUM.  The adaptive release of 2M cells is one sequential posterior
  chain, so the step is the aggregation alone and the release of all cells in
  the independent mode is timed once beside it (``finalize_ms``).
* ``batch_4096``: 4096 independent queries (4.26G rows, 102 GB generated in
  HBM), COUNT + exact int64 SUM + exact float32 SUM each; a step is one
  replay of the CUDA graph holding the autotuned plan's launch.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "PAC-aggregated rows/s at m=64 worlds, % of HBM roofline; p99 query latency"
L2_BYTES = 129 * 1024 * 1024

# per workload: group-id width, value columns used, specs, release mode,
# algorithmic bytes per row (inputs read once), per-group output bytes
WORKLOADS = {
    "lowcard_60m": {"gid_bytes": 1, "n_cols": 4, "aggs": "count+sum+avg", "finalize": "adaptive",
                    "in_bytes_per_row": 8 + 1 + 4 * 8, "flush_l2": False,
                    "describe": "count + 4 sum + 4 avg, exact; adaptive finalize of 36 cells"},
    "ungrouped_1m": {"gid_bytes": 0, "n_cols": 1, "aggs": "count+sum", "finalize": "adaptive",
                     "in_bytes_per_row": 8 + 8, "flush_l2": True,
                     "describe": "count + sum, exact; adaptive finalize of 2 cells"},
    "max_1g": {"gid_bytes": 0, "n_cols": 1, "aggs": "count+max", "finalize": "adaptive",
               "in_bytes_per_row": 8 + 8, "flush_l2": False,
               "describe": "ungrouped count + MAX of int64 values uniform in [0, 1e12] (Sec. 5 bound pruning "
                           "applies); adaptive finalize of 2 cells"},
    "max_1g_increasing": {"gid_bytes": 0, "n_cols": 1, "aggs": "count+max", "finalize": "adaptive",
                          "in_bytes_per_row": 8 + 8, "flush_l2": False,
                          "describe": "ungrouped count + MAX of value = row index, the adversarial order for "
                                      "bound pruning (every row raises its worlds); adaptive finalize of 2 cells"},
    "highcard_100m": {"gid_bytes": 4, "n_cols": 1, "aggs": "count+sum", "finalize": "separate",
                      "in_bytes_per_row": 8 + 4 + 8, "flush_l2": False,
                      "describe": "count + sum, exact; release of the 2M cells timed separately"},
    "lowcard_60m_approx": {"gid_bytes": 1, "n_cols": 4, "aggs": "count+sum+avg", "finalize": "adaptive",
                           "in_bytes_per_row": 8 + 1 + 4 * 8, "flush_l2": False, "approx": True,
                           "describe": "lowcard_60m with the paper's approximate SUM and AVG (Sec. 5: 25 levels "
                                       "of 16-bit counters cascading every 4 bits, two-sided); count + 4 sum + 4 "
                                       "avg, adaptive finalize of 36 cells"},
    "hash_100m": {"gid_bytes": 0, "n_cols": 0, "aggs": "hash", "finalize": "none", "hash_only": True,
                  "in_bytes_per_row": 8 + 8, "flush_l2": False,
                  "describe": "pac_hash_keys alone: 100M int64 PU keys (uniform over 10M) to balanced 64-bit "
                              "world masks (Sec. 2, Sec. 4.2), 8 bytes in and 8 out per row"},
    "lowcard_60m_m128": {"gid_bytes": 1, "n_cols": 4, "aggs": "count+sum+avg", "finalize": "adaptive",
                         "in_bytes_per_row": 8 + 1 + 4 * 8, "flush_l2": False, "worlds": 128,
                         "describe": "lowcard_60m over m = 128 worlds (two keyed re-hashes, Sec. 2): count + 4 "
                                     "sum + 4 avg, exact; adaptive finalize of 36 cells over 128 worlds"},
    "select_60m": {"gid_bytes": 1, "n_cols": 4, "aggs": "count+sum+avg", "finalize": "adaptive",
                   "in_bytes_per_row": 8 + 1 + 4 * 8, "flush_l2": False, "select": True,
                   "describe": "lowcard_60m under a correlated PAC selection (Sec. 4.2): world j of a row kept "
                               "iff value column 0 < world j's exact AVG of column 0 in the row's group; then "
                               "count + 4 sum + 4 avg over the selected rows and adaptive release of 36 cells"},
    "ratio_100m": {"gid_bytes": 4, "n_cols": 2, "aggs": "count+sum", "finalize": "separate", "lift": True,
                   "in_bytes_per_row": 8 + 4 + 2 * 8, "flush_l2": False,
                   "describe": "highcard shape, count + exact sum of the chosen nation's sales and of all "
                               "sales, market share lifted world by world (Sec. 4.2, Sec. 7: 100 * s1 / s2 over "
                               "1M groups x 64 worlds); the single release of the 1M shares timed separately"},
    "serving": {"gid_bytes": 4, "n_cols": 3, "aggs": "count+sum+fsum+dsum", "finalize": "adaptive",
                "in_bytes_per_row": 8 + 4 + 8 + 4 + 8, "flush_l2": False,
                "describe": "Poisson arrivals, shapes of batch_4096, count + exact int64 sum + exact "
                            "float32 sum + exact float64 lognormal(0,1.5) sum, adaptive release of every cell"},
    "batch_4096": {"gid_bytes": 4, "n_cols": 2, "aggs": "count+sum+fsum", "finalize": "none",
                   "in_bytes_per_row": 8 + 4 + 8 + 4, "flush_l2": False,
                   "describe": "4096 independent queries (rows log-uniform 1e3..1e7, groups 1..1e4): count + "
                               "exact int64 sum + exact float32 sum, one plan launch in a CUDA graph"},
}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


E2E_TIMING = ("median of the timed steps, each timed on the host around one synchronous step "
              "(host-to-device copies of its inputs, the GPU work, device-to-host copies of its results)")


def _median(xs):
    ys = sorted(xs)
    k = len(ys)
    return ys[k // 2] if k % 2 else 0.5 * (ys[k // 2 - 1] + ys[k // 2])


def _source_sha(path: str) -> str:
    with open(os.path.join(ROOT, path), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:12]


def _traffic(workload: str, n: int, path: int):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summaries (a `bench-traffic:` line for the workload and aggregation path,
    path 2 when the line names none), scaled to n rows; None when no capture
    exists or the kernel source changed since it was taken."""
    return _traffic_kernel(workload, n, path)[0]


def _traffic_kernel(workload: str, n: int, path: int):
    """(bytes, kernel) of the `bench-traffic:` line (kernel: the line's
    `kernel=` field, None when it names none); (None, None) when none applies."""
    pat = re.compile(r"bench-traffic:\s*workload=(\S+)\s+(?:path=(\d+)\s+)?(?:kernel=(\S+)\s+)?kernel_source=(\S+)"
                     r"\s+sha=(\S+)\s+bytes_per_row=([0-9.]+)")
    for f in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(f) as fh:
            for line in fh:
                m = pat.search(line)
                if m and m.group(1) == workload and int(m.group(2) or 2) == path:
                    try:
                        if _source_sha(m.group(4)) != m.group(5):
                            return None, None
                    except OSError:
                        return None, None
                    return float(m.group(6)) * n, m.group(3)
    return None, None


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                self.samples.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for name, v in zip(names, s[4:8]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(vals, world: int):
    """Each entry's maximum over the ranks: the job takes as long as its
    slowest rank (NCCL on GPUs, gloo on CPU)."""
    import torch
    t = torch.tensor(list(vals), dtype=torch.float64)
    if world > 1:
        import torch.distributed as dist
        if dist.get_backend() == "nccl":
            t = t.cuda()
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def job_throughput(units_per_rank: float, world: int, ms: float) -> float:
    """Whole-job units per second: every rank processes its own units (weak
    scaling, no data-path collective) in at most `ms`."""
    return units_per_rank * world / (ms / 1e3)


def _gen(workload: str, seed: int, rows):
    from paper_2603_15023_gb300 import inputs
    fn = inputs.WORKLOADS[workload]
    return fn(seed=seed) if rows is None else fn(seed=seed, n=rows)


def _spec_list(B, wcfg, vals, outs):
    """(kind, variant, vtype, values, out) per spec: COUNT, then SUM (or MAX)
    per column, then AVG per column where the workload has it."""
    C = wcfg["n_cols"]
    var = B.PAC_APPROX if wcfg.get("approx") else B.PAC_EXACT
    specs = [(B.PAC_COUNT, B.PAC_EXACT, B.PAC_I64, 0, outs[0])]
    if "max" in wcfg["aggs"]:
        return specs + [(B.PAC_MAX, B.PAC_EXACT, B.PAC_I64, vals[k], outs[1 + k]) for k in range(C)]
    for k in range(C):
        specs.append((B.PAC_SUM, var, B.PAC_I64, vals[k], outs[1 + k]))
    if "avg" in wcfg["aggs"]:
        for k in range(C):
            specs.append((B.PAC_AVG, var, B.PAC_I64, vals[k], outs[1 + C + k]))
    return specs


def _n_specs(wcfg):
    C = wcfg["n_cols"]
    return 1 + C + (C if "avg" in wcfg["aggs"] else 0)


def cpu_oracle_sample(workload: str, rows: int, reps: int = 1, seed: int = 0):
    """Times the oracle (as it stands) on the first `rows` rows of the
    workload, `reps` times over: hash, every aggregate of the step, and the
    release."""
    import oracle as orc
    wcfg = WORKLOADS[workload]
    wl = _gen(workload, seed, rows)
    G = wl.n_groups
    qk = orc.query_key(seed)
    thr = _select_operands(orc, wl, G, qk) if wcfg.get("select") else None
    t0 = time.perf_counter()
    for _ in range(reps):
        _oracle_step(orc, wcfg, wl, G, qk, thr)
    dt = time.perf_counter() - t0
    return rows * reps / dt, dt


def RATIO_PROG_ORC(orc):
    """100 * spec 0 / spec 1, the market share of the ratio workload."""
    return [(orc.L_CONST, 0, 100.0), (orc.L_SPEC, 0, 0), (orc.L_MUL, 0, 0), (orc.L_SPEC, 1, 0), (orc.L_DIV, 0, 0)]


def _select_operands(orc, wl, G, qk):
    """Per-world operands of the select workloads: world j's exact AVG of
    value column 0 in each group, truncated to int64 (computed once, outside
    the timed step, like the subquery result a correlated selection reads)."""
    masks = orc.hash_keys(wl.keys, qk, orc.BALANCED)
    avg, *_ = orc.aggregate(masks, wl.values[0], wl.gids, G, orc.AVG)
    return np.trunc(avg).astype(np.int64)


def _oracle_step(orc, wcfg, wl, G, qk, thr=None):
    masks = orc.hash_keys(wl.keys, qk, orc.BALANCED)
    if wcfg.get("hash_only"):
        return
    gids, vals = wl.gids, wl.values[:wcfg["n_cols"]]
    if thr is not None:
        masks, _ = orc.select(masks, wl.values[0], orc.LT, thr, wl.gids)
        keep = masks != 0
        masks, gids, vals = masks[keep], gids[keep], [v[keep] for v in vals]
    res = [orc.aggregate(masks, None, gids, G, orc.COUNT)]
    if "max" in wcfg["aggs"]:
        for v in vals:
            res.append(orc.aggregate(masks, v, gids, G, orc.MAX))
    elif wcfg.get("approx"):
        for v in vals:
            res.append(orc.approx_sum_i64(masks, v, gids, G))
        for v in vals:
            res.append(orc.approx_avg_i64(masks, v, gids, G))
    else:
        for v in vals:
            res.append(orc.aggregate(masks, v, gids, G, orc.SUM))
        if "avg" in wcfg["aggs"]:
            for v in vals:
                res.append(orc.aggregate(masks, v, gids, G, orc.AVG))
    if wcfg.get("lift"):
        y = np.stack([r[0].astype(np.float64) for r in res[1:3]], axis=1)
        orc.lift(y, [2.0, 2.0], RATIO_PROG_ORC(orc))
    if wcfg["finalize"] != "separate":
        y = np.stack([r[0].astype(np.float64) for r in res], axis=1)
        per_col = 1.0 if "max" in wcfg["aggs"] else 2.0  # COUNT and SUM scale by 2, MAX and AVG by 1
        scales = [2.0] + [per_col] * wcfg["n_cols"] + [1.0] * (len(res) - 1 - wcfg["n_cols"])
        orc.finalize(y, scales, res[0][1], res[0][2], 99, 1.0 / 128, orc.ADAPTIVE)


def host_cpu():
    """Host cores this process may use and the CPU model (lscpu's model
    name, else /proc/cpuinfo), recorded beside every CPU baseline."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"nproc": cores, "cpu_model": model or "unknown", "machine": os.uname().machine}


def _gen_groups(workload: str) -> int:
    """Group count of a workload's generator (its default size)."""
    from paper_2603_15023_gb300 import inputs
    import inspect
    sig = inspect.signature(inputs.WORKLOADS[workload])
    p = sig.parameters.get("n_groups")
    if p is not None:
        return int(p.default)
    return 4 if WORKLOADS[workload]["gid_bytes"] == 1 else 1


def _chunked_ok(wcfg) -> bool:
    """Workloads whose per-thread states merge by addition: COUNT, exact SUM
    (and AVG, derived from the merged COUNT and SUM states)."""
    return not (wcfg.get("approx") or wcfg.get("select") or wcfg.get("lift") or "max" in wcfg["aggs"])


def cpu_oracle_chunked(workload: str, rows: int, threads: int, chunk: int = 1 << 18, seed: int = 0, wl=None):
    """The oracle on all host cores: rows cut into consecutive chunks, each
    thread hashing its chunks and aggregating them with the oracle's COUNT and
    SUM (per-thread chunk states), the states merged in chunk order
    (COUNT, SUM, n_g by addition, or_g by OR), AVG = SUM / COUNT of the merged
    states, then the release of every cell.  The oracle's C functions release
    the GIL, so the threads run in parallel."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle as orc
    wcfg = WORKLOADS[workload]
    wl = _gen(workload, seed, rows) if wl is None else wl
    G, C = wl.n_groups, wcfg["n_cols"]
    qk = orc.query_key(seed)
    bounds = [(a, min(a + chunk, rows)) for a in range(0, rows, chunk)]

    def one(b):
        a, e = b
        masks = orc.hash_keys(wl.keys[a:e], qk, orc.BALANCED)
        if wcfg.get("hash_only"):
            return None
        gids = None if wl.gids is None else wl.gids[a:e]
        cnt, n_g, or_g, _ = orc.aggregate(masks, None, gids, G, orc.COUNT)
        sums = [orc.aggregate(masks, v[a:e], gids, G, orc.SUM)[0] for v in wl.values[:C]]
        return cnt, sums, n_g, or_g

    if G > 4096:
        # many groups: a row chunk's state would hold every group, so each
        # thread takes a range of groups instead (all of their rows, in row
        # order) and the disjoint states are placed side by side
        return _cpu_oracle_group_ranges(orc, wcfg, wl, rows, threads, qk)
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(one, bounds))
    if wcfg.get("hash_only"):
        dt = time.perf_counter() - t0
        return rows / dt, dt
    cnt = np.zeros((G, 64), np.uint64)
    sums = [np.zeros((G, 64), np.int64) for _ in range(C)]
    n_g = np.zeros(G, np.uint64)
    or_g = np.zeros(G, np.uint64)
    for c, sm, ng, og in parts:              # chunk order
        cnt += c
        for k in range(C):
            sums[k] += sm[k]
        n_g += ng
        or_g |= og
    res = [cnt.astype(np.float64)] + [x.astype(np.float64) for x in sums]
    scales = [2.0] * (1 + C)
    if "avg" in wcfg["aggs"]:
        cf = cnt.astype(np.float64)
        res += [np.where(cnt > 0, x / np.maximum(cf, 1.0), 0.0) for x in res[1:1 + C]]
        scales += [1.0] * C
    if wcfg["finalize"] != "separate":
        orc.finalize(np.stack(res, axis=1), scales, n_g, or_g, 99, 1.0 / 128, orc.ADAPTIVE)
    dt = time.perf_counter() - t0
    return rows / dt, dt


def _cpu_oracle_group_ranges(orc, wcfg, wl, rows, threads, qk):
    """All-cores leg for many groups: thread t aggregates the rows of groups
    [t*G/T, (t+1)*G/T) with the oracle (hash, COUNT, SUM per column), then
    the release.  Timed from the row selection on."""
    from concurrent.futures import ThreadPoolExecutor
    G, C = wl.n_groups, wcfg["n_cols"]
    gids = wl.gids[:rows]
    edges = [G * t // threads for t in range(threads + 1)]

    def one(t):
        lo, hi = edges[t], edges[t + 1]
        sel = np.flatnonzero((gids >= lo) & (gids < hi))
        masks = orc.hash_keys(wl.keys[sel], qk, orc.BALANCED)
        g = (gids[sel] - lo).astype(np.uint32)
        Gt = max(hi - lo, 1)
        cnt, n_g, or_g, _ = orc.aggregate(masks, None, g, Gt, orc.COUNT)
        sums = [orc.aggregate(masks, v[sel], g, Gt, orc.SUM)[0] for v in wl.values[:C]]
        return cnt, sums, n_g, or_g

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(one, range(threads)))
    cnt = np.concatenate([p[0] for p in parts])
    sums = [np.concatenate([p[1][k] for p in parts]) for k in range(C)]
    n_g = np.concatenate([p[2] for p in parts])
    or_g = np.concatenate([p[3] for p in parts])
    if wcfg["finalize"] != "separate":
        res = [cnt.astype(np.float64)] + [x.astype(np.float64) for x in sums]
        orc.finalize(np.stack(res, axis=1), [2.0] * (1 + C), n_g, or_g, 99, 1.0 / 128, orc.ADAPTIVE)
    dt = time.perf_counter() - t0
    return rows / dt, dt


def cpu_baseline(workload: str, n: int, one_rows: int, all_rows: int):
    """Both legs of the CPU baseline: (i) the oracle's step as it stands on
    one thread, (ii) all host cores with per-thread chunk states merged in
    order.  The line's value is the all-cores leg where the workload's states
    merge by addition, else the one-thread leg."""
    host = host_cpu()
    wcfg = WORKLOADS[workload]
    srows = min(one_rows, n)
    reps = max(1, one_rows // srows)
    v1, dt1 = cpu_oracle_sample(workload, srows, reps)
    what = f"first {srows} rows of {workload}" if srows < n else f"the whole {workload} workload ({n} rows), {reps}x"
    legs = {"one_thread": {"value": v1, "cores": 1, "seconds": dt1,
                           "sample": f"{what} ({wcfg['describe']}), the oracle's step as it stands"}}
    out = {"value": v1, "unit": "rows/s", "cores": 1, "kind": "oracle",
           "sample": f"{what} ({wcfg['describe']}), one thread, {dt1:.1f} s", **host, "legs": legs}
    if _chunked_ok(wcfg) and host["nproc"] > 1:
        arows = min(all_rows, n)
        areps = max(1, all_rows // arows)
        vals = [cpu_oracle_chunked(workload, arows, host["nproc"]) for _ in range(areps)]
        va = arows * areps / sum(dt for _, dt in vals)
        dta = sum(dt for _, dt in vals)
        awhat = f"first {arows} rows of {workload}" if arows < n else f"the whole {workload} workload, {areps}x"
        how = ("one range of groups per thread (all of its rows, in row order), the disjoint states side by side"
               if _gen_groups(workload) > 4096 else
               "256K-row chunks over the threads, chunk states (COUNT, SUM, n_g, or_g) merged in order, AVG from "
               "the merged states")
        legs["all_cores"] = {"value": va, "cores": host["nproc"], "seconds": dta,
                             "sample": f"{awhat}, {host['nproc']} threads: {how}, then the release"}
        out.update({"value": va, "cores": host["nproc"],
                    "sample": f"{awhat}, {host['nproc']} threads ({how}), {dta:.1f} s; one-thread leg "
                              f"{v1 / 1e6:.2f} M rows/s"})
    return out


def cpu_oracle_batch_sample(rows_budget: int, seed: int = 0, threads: int = 1):
    """Times the oracle on the first queries of the batched workload (whole
    queries, in order, until `rows_budget` rows): hash, COUNT, SUM, float SUM."""
    import oracle as orc
    from paper_2603_15023_gb300 import inputs
    spec = inputs.batch_4096(seed=seed)
    cols, rows = [], 0
    for q in range(spec.n_queries):
        if rows + int(spec.rows[q]) > rows_budget and cols:
            break
        cols.append((q, spec.columns(q)))
        rows += int(spec.rows[q])

    def one(item):
        q, (keys, gids, v, f) = item
        G = int(spec.groups[q])
        masks = orc.hash_keys(keys, orc.query_key(1_000_000 + q), orc.BALANCED)
        orc.aggregate(masks, None, gids, G, orc.COUNT)
        orc.aggregate(masks, v, gids, G, orc.SUM)
        orc.aggregate(masks, f, gids, G, orc.SUM)

    t0 = time.perf_counter()
    if threads <= 1:
        for item in cols:
            one(item)
    else:  # independent queries: whole queries per thread
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(one, cols))
    dt = time.perf_counter() - t0
    return rows / dt, dt, len(cols), rows


def cpu_baseline_batch(one_rows: int, all_rows: int, what: str = "batch_4096"):
    """Both legs on the batched workload's queries: one thread, then all host
    cores with whole queries per thread."""
    host = host_cpu()
    v1, dt1, nq1, r1 = cpu_oracle_batch_sample(one_rows)
    legs = {"one_thread": {"value": v1, "cores": 1, "seconds": dt1,
                           "sample": f"the first {nq1} queries of batch_4096 ({r1} rows; hash, count, sum, "
                                     f"float sum)"}}
    out = {"value": v1, "unit": "rows/s", "cores": 1, "kind": "oracle",
           "sample": f"the first {nq1} queries of batch_4096 ({r1} rows), one thread, {dt1:.1f} s", **host,
           "legs": legs}
    if host["nproc"] > 1:
        va, dta, nqa, ra = cpu_oracle_batch_sample(all_rows, threads=host["nproc"])
        legs["all_cores"] = {"value": va, "cores": host["nproc"], "seconds": dta,
                             "sample": f"the first {nqa} queries of batch_4096 ({ra} rows), whole queries per "
                                       f"thread over {host['nproc']} threads"}
        out.update({"value": va, "cores": host["nproc"],
                    "sample": f"the first {nqa} queries of batch_4096 ({ra} rows), {host['nproc']} threads "
                              f"(whole queries per thread), {dta:.1f} s; one-thread leg {v1 / 1e6:.2f} M rows/s"
                              + ("" if what == "batch_4096" else f"; {what} draws its queries from these shapes")})
    return out


def run_reference(args):
    """The reference arm: the oracle, as it stands, on the host cores (rank 0
    only).  Workloads whose states merge by addition run on every core with
    per-thread chunk states merged in order, a bounded sample of --ref-rows
    rows per step; the others on one thread."""
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    workload = args.workload or "lowcard_60m"
    wcfg = WORKLOADS[workload]
    host = host_cpu()
    rows = args.ref_rows
    vals = []
    if workload in ("batch_4096", "serving"):
        # serving draws its queries from the batched workload's shapes
        for i in range(args.warmup + args.steps):
            v, dt, _, rows = cpu_oracle_batch_sample(args.ref_rows, threads=host["nproc"])
            if i >= args.warmup:
                vals.append((v, dt))
        cores = host["nproc"]
        sample = f"the first queries of batch_4096 ({rows} rows) per step, whole queries per thread"
    elif _chunked_ok(wcfg):
        wl = _gen(workload, 0, rows)
        rows = wl.n
        for i in range(args.warmup + args.steps):
            v, dt = cpu_oracle_chunked(workload, rows, host["nproc"], wl=wl)
            if i >= args.warmup:
                vals.append((v, dt))
        cores = host["nproc"]
        sample = (f"first {rows} rows of {workload} per step, 256K-row chunks over {cores} threads, chunk states "
                  "merged in order, then the release")
    else:
        rows = min(rows, 1_000_000)
        for i in range(args.warmup + args.steps):
            v, dt = cpu_oracle_sample(workload, rows)
            if i >= args.warmup:
                vals.append((v, dt))
        cores = 1
        sample = f"first {rows} rows of {workload} per step, one thread"
    value = statistics.median(v for v, _ in vals)
    ms = statistics.median(dt for _, dt in vals) * 1e3
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": workload, "rows": rows, "aggregates": wcfg["describe"], "worlds": 64},
        "cpu_baseline": {"value": value, "unit": "rows/s", "cores": cores, "kind": "oracle", "sample": sample,
                         **host},
        "e2e": {"value": value, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def measure_batch(args, suite=False):
    """The batched workload: every query's columns generated in HBM, one
    autotuned plan, its launch captured in a CUDA graph; a step is one replay
    (the aggregation of all queries).  Returns the JSON dict (rank 0)."""
    import torch
    from paper_2603_15023_gb300 import batch_inputs, inputs
    from paper_2603_15023_gb300 import binding as B

    world, rank, local = _dist()
    ctx = B.pac_create(local)
    spec = inputs.batch_4096(seed=rank, n_queries=4096 if suite else args.queries)
    s = torch.cuda.Stream()
    db = batch_inputs.DeviceBatch(spec, stream=s.cuda_stream)
    s.synchronize()
    t0 = time.perf_counter()
    plan = B.pac_batch_plan(ctx, db.queries, db.n_queries, 0 if args.no_autotune else B.PAC_BATCH_AUTOTUNE)
    plan_s = time.perf_counter() - t0
    info = {k: B.pac_batch_info(plan, k) for k in ("n_items", "item_rows", "smem_cap", "kernels",
                                                    "n_warp_private", "n_atomic")}
    with torch.cuda.stream(s):
        B.pac_batch_launch(ctx, plan, s.cuda_stream)
    s.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        B.pac_batch_launch(ctx, plan, s.cuda_stream)
    with torch.cuda.stream(s):
        for _ in range(args.warmup):
            graph.replay()
    s.synchronize()
    st = B.pac_sync_status(ctx, s.cuda_stream)
    if st != B.PAC_OK:
        raise RuntimeError(B.status_name(st))
    clocks = ClockSampler(local)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    with torch.cuda.stream(s):
        start.record(s)
        for i in range(args.steps):
            evs[i][0].record(s)
            graph.replay()
            evs[i][1].record(s)
        end.record(s)
    torch.cuda.synchronize()
    clocks.stop()
    st = B.pac_sync_status(ctx, s.cuda_stream)
    if st != B.PAC_OK:
        raise RuntimeError(B.status_name(st))
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms_step = max_over_ranks([statistics.median(step_ms)], world)[0]
    value = job_throughput(db.total_rows, world, ms_step)
    peak, peak_src = _peaks()
    algo = db.algorithmic_bytes()
    achieved = algo / (ms_step / 1e3) / 1e9
    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            cpu = cpu_baseline_batch(args.cpu_rows, args.cpu_rows_all)
        wcfg = WORKLOADS["batch_4096"]
        line = {
            "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64+f32", "data": "synthetic (generated in HBM)",
            "config": {"workload": "batch_4096", "queries": db.n_queries, "rows": db.total_rows,
                       "groups_total": db.total_groups, "worlds": 64, "aggregates": wcfg["describe"],
                       "l2": f"inputs {db.total_rows * wcfg['in_bytes_per_row'] / 1e9:.1f} GB > 129 MB L2",
                       "plan": info, "plan_seconds_incl_autotune": plan_s,
                       "timing": f"median of {args.steps} CUDA-graph replays, CUDA events on the launching stream"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": _traffic("batch_4096", db.total_rows, 3),
                         "traffic_kernel": _traffic_kernel("batch_4096", db.total_rows, 3)[1],
                         "kernel": "k_batch_agg + k_batch_merge (one graph replay)",
                         "algorithmic_bytes": algo, "peak_source": peak_src},
            "cpu_baseline": cpu,
            "e2e": None,
            "e2e_note": "the 102 GB of columns are generated in HBM (larger than the host memory of the build "
                        "machine); no host-to-device leg is timed for this workload",
            "gpu_launches": info["kernels"] * args.steps,
            "clocks": clocks.summary(),
        }
    B.pac_batch_free(plan)
    B.pac_destroy(ctx)
    del db, graph
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return line


def measure_serving(args):
    """Continuous batching under Poisson arrivals: a pool of query shapes drawn
    from the batched workload's distribution lives in HBM (columns generated
    on the device, plus a float64 lognormal(0, 1.5) column); every arrival
    takes a pool shape, a seed and a slot of an output ring, and is submitted
    to the server at its scheduled arrival time (or as soon as its ring slot
    is free).  Latency = completion stamp - scheduled arrival."""
    import torch
    from paper_2603_15023_gb300 import binding as B
    from paper_2603_15023_gb300 import gen, inputs

    world, rank, local = _dist()
    ctx = B.pac_create(local)
    spec = inputs.batch_4096(seed=100 + rank, n_queries=args.pool)
    P = spec.n_queries
    s = torch.cuda.Stream()
    cols = []
    r = inputs._rng(100 + rank, 2000)
    for q in range(P):
        n, G, K = int(spec.rows[q]), int(spec.groups[q]), int(spec.keys[q])
        k = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
        g = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
        v = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
        f = torch.empty(max(n, 1), dtype=torch.float32, device="cuda")
        gen.fill_i64(k.data_ptr(), n, spec.seed, 4 * q, 0, K, stream=s.cuda_stream)
        gen.fill_u32(g.data_ptr(), n, spec.seed, 4 * q + 1, G, stream=s.cuda_stream)
        gen.fill_i64(v.data_ptr(), n, spec.seed, 4 * q + 2, 1, 100_000, stream=s.cuda_stream)
        gen.fill_f32_1000(f.data_ptr(), n, spec.seed, 4 * q + 3, stream=s.cuda_stream)
        d = torch.from_numpy(r.lognormal(0.0, 1.5, max(n, 1))).to("cuda")
        cols.append((n, G, k, g, v, f, d))
    s.synchronize()
    max_g = int(spec.groups.max())
    R = args.ring
    ring = []
    for _ in range(R):
        outs = [torch.empty((max_g, 64), dtype=dt, device="cuda")
                for dt in (torch.int64, torch.int64, torch.float64, torch.float64)]
        meta = torch.empty((max_g, 2), dtype=torch.int64, device="cuda")
        nz = torch.empty(max_g * 4, dtype=torch.float64, device="cuda")
        nl = torch.empty(max_g * 4, dtype=torch.uint8, device="cuda")
        fl = torch.empty(max_g * 4, dtype=torch.int32, device="cuda")
        ring.append((outs, meta, nz, nl, fl))
    srv = B.pac_serve_create(ctx, mem_budget=args.serve_mem_gb << 30, max_inflight=args.ring,
                             max_batch=256, n_streams=8)
    lam = args.rate
    n_req = int(lam * args.serve_seconds)
    rr = inputs._rng(100 + rank, 3000)
    arrivals = np.cumsum(rr.exponential(1.0 / lam, n_req))
    shapes = rr.integers(0, P, n_req)
    keep = []
    tickets = [None] * n_req
    t_sub = np.zeros(n_req)
    busy = [None] * R
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    t0 = time.perf_counter()
    for i in range(n_req):
        slot = i % R
        if busy[slot] is not None:
            j = busy[slot]
            lat, st = B.pac_serve_wait(srv, tickets[j])
            if st != B.PAC_OK:
                raise RuntimeError(B.status_name(st))
            tickets[j] = (t_sub[j] - arrivals[j] + lat / 1e3)
        now = time.perf_counter() - t0
        if now < arrivals[i]:
            time.sleep(arrivals[i] - now)
        n, G, k, g, v, f, d = cols[int(shapes[i])]
        outs, meta, nz, nl, fl = ring[slot]
        specs = B.make_specs([(B.PAC_COUNT, B.PAC_EXACT, B.PAC_I64, 0, outs[0].data_ptr()),
                              (B.PAC_SUM, B.PAC_EXACT, B.PAC_I64, v.data_ptr(), outs[1].data_ptr()),
                              (B.PAC_SUM, B.PAC_EXACT, B.PAC_F32, f.data_ptr(), outs[2].data_ptr()),
                              (B.PAC_SUM, B.PAC_EXACT, B.PAC_F64, d.data_ptr(), outs[3].data_ptr())])
        inp = B.make_input(k.data_ptr(), n, query_key=B.pac_query_key(7_000_000 + i), group_ids=g.data_ptr(),
                           gid_bytes=4, n_groups=G)
        qd = B.make_query(inp, specs, 4, meta=meta.data_ptr(), fin_mode=B.PAC_FIN_ADAPTIVE, seed=9_000 + i,
                          budget=1.0 / 128, noised=nz.data_ptr(), is_null=nl.data_ptr(), flags=fl.data_ptr())
        keep.append(specs)
        t_sub[i] = time.perf_counter() - t0
        tickets[i] = B.pac_serve_submit(srv, qd)
        busy[slot] = i
    for i in range(n_req):
        if not isinstance(tickets[i], float):
            lat, st = B.pac_serve_wait(srv, tickets[i])
            if st != B.PAC_OK:
                raise RuntimeError(B.status_name(st))
            tickets[i] = (t_sub[i] - arrivals[i] + lat / 1e3)
    wall = time.perf_counter() - t0
    clocks.stop()
    lat_ms = np.array(tickets, dtype=np.float64) * 1e3
    rows = int(sum(cols[int(q)][0] for q in shapes))
    stats = {k: B.pac_serve_stats(srv, k) for k in ("batches", "mean_batch", "max_inflight_seen",
                                                     "arena_high_water", "max_device_overlap")}
    B.pac_serve_destroy(srv)
    value = rows / wall
    line = {
        "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": world, "steps": n_req, "warmup": 0,
        "ms_per_step": wall * 1e3 / n_req, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64+f32+f64", "data": "synthetic (generated in HBM)",
        "config": {"workload": "serving", "arrival_rate_qps": lam, "requests": n_req, "pool_shapes": P,
                   "offered_rows_per_s": rows / float(arrivals[-1]) if n_req else 0.0,
                   "aggregates": WORKLOADS["serving"]["describe"], "server": stats,
                   "output_ring_slots": R},
        "latency": {"p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
                    "max_ms": float(lat_ms.max()), "definition": "completion stamp - scheduled Poisson arrival"},
        "roofline": None,
        "roofline_note": "latency-bound by design: the offered load is about 1% of HBM bandwidth",
        "cpu_baseline": None if args.no_cpu_baseline else cpu_baseline_batch(args.cpu_rows, args.cpu_rows_all,
                                                                              "serving"),
        "e2e": None,
        "e2e_note": "queries are submitted through the public serving API (pac_serve_submit / pac_serve_wait) "
                    "with their columns resident in HBM; latency is measured from the scheduled arrival",
        "gpu_launches": int(stats["batches"]) * 3,
        "clocks": clocks.summary(),
    }
    B.pac_destroy(ctx)
    del cols, ring
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return line if rank == 0 else None


def measure_single(args, workload: str, rows=None, steps=None, warmup=None, suite=False):
    """One workload of single queries: returns its JSON dict (rank 0) or None."""
    import torch
    from paper_2603_15023_gb300 import binding as B

    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    world, rank, local = _dist()
    ctx = B.pac_create(local)
    if args.path and not suite:
        B.pac_set_option(ctx, "agg_path", {"auto": 0, "bitloop": 1, "mma": 2, "engine": 3, "small": 4, "part": 5}[args.path])
    B.pac_set_option(ctx, "minmax_prune", args.minmax_prune)

    wcfg = WORKLOADS[workload]
    wl = _gen(workload, rank, rows)
    n, G = wl.n, wl.n_groups
    C = wcfg["n_cols"]
    n_specs = _n_specs(wcfg)
    stream = torch.cuda.Stream()
    sptr = stream.cuda_stream
    d_keys = torch.from_numpy(wl.keys).cuda()
    d_gids = torch.from_numpy(wl.gids).cuda() if wl.gids is not None else None
    d_vals = [torch.from_numpy(v).cuda() for v in wl.values[:C]]
    W = wcfg.get("worlds", 64)
    outs = [torch.empty((G, W), dtype=torch.int64 if i < 1 + C else torch.float64, device="cuda")
            for i in range(n_specs)]
    meta = torch.empty((G, 2 if W == 64 else 3), dtype=torch.int64, device="cuda")
    n_cells = G * n_specs
    noised = torch.empty(n_cells, dtype=torch.float64, device="cuda")
    is_null = torch.empty(n_cells, dtype=torch.uint8, device="cuda")
    flags = torch.empty(n_cells, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    qk = B.pac_query_key(rank)
    inp = B.make_input(d_keys.data_ptr(), n, query_key=qk,
                       group_ids=d_gids.data_ptr() if d_gids is not None else 0,
                       gid_bytes=wcfg["gid_bytes"], n_groups=G)
    specs = B.make_specs(_spec_list(B, wcfg, [v.data_ptr() for v in d_vals], [o.data_ptr() for o in outs]))
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda") if wcfg["flush_l2"] else None
    in_step_finalize = wcfg["finalize"] == "adaptive"
    sel = None
    if wcfg.get("select"):
        # the correlated operands: world j's AVG of column 0 per group (a PAC
        # aggregate, computed once outside the timed step), truncated to int64
        d_avg = torch.empty((G, 64), dtype=torch.float64, device="cuda")
        B.pac_aggregate_multi(ctx, inp, B.make_specs([(B.PAC_AVG, B.PAC_EXACT, B.PAC_I64, d_vals[0].data_ptr(),
                                                         d_avg.data_ptr())]), 1, 0, sptr)
        stream.synchronize()
        d_thr = torch.trunc(d_avg).to(torch.int64).contiguous()
        sel = B.make_select(d_vals[0].data_ptr(), B.PAC_I64, B.PAC_CMP_LT, d_thr.data_ptr(), G,
                            d_gids.data_ptr(), 1)

    lift = None
    lift_ms = []
    if wcfg.get("lift"):
        # the market share 100 * s1 / s2, world by world, from the two SUM outputs
        share = torch.empty((G, 64), dtype=torch.float64, device="cuda")
        lift_specs = B.make_specs(_spec_list(B, wcfg, [v.data_ptr() for v in d_vals],
                                             [o.data_ptr() for o in outs])[1:3])
        prog = [(B.PAC_LIFT_CONST, 0, 100.0), (B.PAC_LIFT_SPEC, 0, 0), (B.PAC_LIFT_MUL, 0, 0),
                (B.PAC_LIFT_SPEC, 1, 0), (B.PAC_LIFT_DIV, 0, 0)]
        lift = (lift_specs, B.make_lift(prog), len(prog), share)

    qk2 = B.pac_query_key2(rank)

    d_masks = torch.empty(n if wcfg.get("hash_only") else 0, dtype=torch.int64, device="cuda")

    def aggregate(sp_ptr):
        if wcfg.get("hash_only"):
            B.pac_hash_keys(ctx, d_keys.data_ptr(), d_masks.data_ptr(), n, qk, B.PAC_HASH_BALANCED, sp_ptr)
        elif W == 128:
            B.pac_aggregate128(ctx, inp, qk2, specs, n_specs, meta.data_ptr(), sp_ptr)
        elif sel is not None:
            B.pac_aggregate_select(ctx, inp, sel, specs, n_specs, meta.data_ptr(), sp_ptr)
        else:
            B.pac_aggregate_multi(ctx, inp, specs, n_specs, meta.data_ptr(), sp_ptr)
        return B.pac_get_info(ctx, "last_launches")

    def release(i, sp_ptr, lift_ev=None):
        k = 0
        if lift is not None:
            le = None
            if lift_ev is not None:
                le = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                le[0].record(torch.cuda.current_stream())
            B.pac_lift(ctx, lift[0], 2, G, lift[1], lift[2], lift[3].data_ptr(), sp_ptr)
            if le is not None:
                le[1].record(torch.cuda.current_stream())
                lift_ev.append(le)
            k += B.pac_get_info(ctx, "last_launches")
        if in_step_finalize:
            fin = B.pac_finalize128 if W == 128 else B.pac_finalize
            fin(ctx, specs, n_specs, G, meta.data_ptr(), 1000 + i, 1.0 / 128, B.PAC_FIN_ADAPTIVE,
                noised.data_ptr(), is_null.data_ptr(), flags.data_ptr(), 0, sp_ptr)
            k += B.pac_get_info(ctx, "last_launches")
        return k

    with torch.cuda.stream(stream):
        for i in range(warmup):
            if flush is not None:
                flush.fill_(i)
            aggregate(sptr)
            release(i, sptr)
    torch.cuda.synchronize()
    st = B.pac_sync_status(ctx, sptr)
    if st != B.PAC_OK:
        raise RuntimeError(B.status_name(st))
    path = B.pac_get_info(ctx, "last_path")

    # The tensor-core and one-launch paths enqueue only kernels and memsets
    # once warm, so a step is captured as CUDA graphs (aggregation; release)
    # and replayed; the other paths plan on the host per call and are timed
    # as stream work.  Either way the reported time is the median step.
    graphs = None
    if (path in (2, 4) or wcfg.get("hash_only")) and sel is None and lift is None and not wcfg.get("approx"):
        try:
            g_agg, g_rel = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
            launches_agg = launches_rel = 0
            with torch.cuda.graph(g_agg, stream=stream):
                launches_agg = aggregate(stream.cuda_stream)
            with torch.cuda.graph(g_rel, stream=stream):
                launches_rel = release(warmup, stream.cuda_stream)
            with torch.cuda.stream(stream):
                for _ in range(3):
                    g_agg.replay()
                    g_rel.replay()
            torch.cuda.synchronize()
            graphs = (g_agg, g_rel, launches_agg, launches_rel)
        except Exception as e:  # fall back to stream-timed steps
            print(f"graph capture unavailable ({e}); timing stream steps", file=sys.stderr)
            torch.cuda.synchronize()
            graphs = None

    clocks = ClockSampler(local)
    evs = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    launches = 0
    with torch.cuda.stream(stream):
        for i in range(steps):
            if flush is not None:
                flush.fill_(i)  # L2 flush between steps, outside the step's events
            ev = evs[i]
            ev[0].record(stream)
            if graphs is not None:
                graphs[0].replay()
                launches += graphs[2]
            else:
                launches += aggregate(sptr)
            ev[1].record(stream)
            if graphs is not None:
                graphs[1].replay()
                launches += graphs[3]
            else:
                launches += release(warmup + i, sptr, lift_ms)
            ev[2].record(stream)
    torch.cuda.synchronize()
    clocks.stop()
    st = B.pac_sync_status(ctx, sptr)
    if st != B.PAC_OK:
        raise RuntimeError(B.status_name(st))
    agg_ms = [a.elapsed_time(b) for a, b, _ in evs]
    step_ms = [a.elapsed_time(c) for a, _, c in evs]
    ms_step, agg_med = max_over_ranks([statistics.median(step_ms), statistics.median(agg_ms)], world)
    value = job_throughput(n, world, ms_step)
    timing = (f"median of {steps} CUDA-graph replays (aggregation graph + release graph), CUDA events on the "
              "launching stream" if graphs is not None else
              f"median of {steps} steps enqueued on one stream, CUDA events on that stream")

    # m = 128: the same columns aggregated over 64 worlds, timed the same way,
    # for the cost ratio of the second mask word
    m128 = None
    if W == 128:
        o64 = [torch.empty((G, 64), dtype=torch.int64 if i < 1 + C else torch.float64, device="cuda")
               for i in range(n_specs)]
        meta64 = torch.empty((G, 2), dtype=torch.int64, device="cuda")
        specs64 = B.make_specs(_spec_list(B, wcfg, [v.data_ptr() for v in d_vals], [o.data_ptr() for o in o64]))
        g64 = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            for _ in range(3):
                B.pac_aggregate_multi(ctx, inp, specs64, n_specs, meta64.data_ptr(), sptr)
        torch.cuda.synchronize()
        with torch.cuda.graph(g64, stream=stream):
            B.pac_aggregate_multi(ctx, inp, specs64, n_specs, meta64.data_ptr(), stream.cuda_stream)
        ev64 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        with torch.cuda.stream(stream):
            for a, b in ev64:
                a.record(stream)
                g64.replay()
                b.record(stream)
        torch.cuda.synchronize()
        ms64 = statistics.median(a.elapsed_time(b) for a, b in ev64)
        m128 = {"agg_ms_m128": agg_med, "agg_ms_m64": ms64, "cost_ratio": agg_med / ms64,
                "note": "the paper expects at most twice the cost for m = 128 (Sec. 2)"}

    # the release of every cell, timed once beside the step when it is not in it
    fin_ms = fin_adaptive_ms = None
    if not in_step_finalize:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if lift is not None:
            rel = B.make_specs([(B.PAC_LIFTED, B.PAC_EXACT, B.PAC_F64, 0, lift[3].data_ptr())])
            B.pac_finalize(ctx, rel, 1, G, meta.data_ptr(), 5, 1.0 / 128, B.PAC_FIN_INDEPENDENT,
                           noised.data_ptr(), is_null.data_ptr(), flags.data_ptr(), 0, sptr)
        else:
            B.pac_finalize(ctx, specs, n_specs, G, meta.data_ptr(), 5, 1.0 / 128, B.PAC_FIN_INDEPENDENT,
                           noised.data_ptr(), is_null.data_ptr(), flags.data_ptr(), 0, sptr)
        e1.record(stream)
        torch.cuda.synchronize()
        fin_ms = e0.elapsed_time(e1)
        if lift is None:
            # the paper's composition as well: one adaptive chain over every cell
            # (sequential until the posterior collapses onto one world)
            e0.record(stream)
            B.pac_finalize(ctx, specs, n_specs, G, meta.data_ptr(), 5, 1.0 / 128, B.PAC_FIN_ADAPTIVE,
                           noised.data_ptr(), is_null.data_ptr(), flags.data_ptr(), 0, sptr)
            e1.record(stream)
            torch.cuda.synchronize()
            fin_adaptive_ms = e0.elapsed_time(e1)

    # end to end through the C ABI from pinned host memory
    e2e = None
    if args.e2e_steps > 0 and wcfg.get("hash_only"):
        # keys from pinned host memory, the hash, the masks back to pinned host memory
        h_keys = torch.from_numpy(wl.keys).pin_memory()
        h_masks = torch.empty(n, dtype=torch.int64).pin_memory()

        def e2e_hash():
            with torch.cuda.stream(stream):
                d_keys.copy_(h_keys, non_blocking=True)
                B.pac_hash_keys(ctx, d_keys.data_ptr(), d_masks.data_ptr(), n, qk, B.PAC_HASH_BALANCED, sptr)
                h_masks.copy_(d_masks, non_blocking=True)
            torch.cuda.synchronize()

        for _ in range(2):
            e2e_hash()
        dts = []
        for _ in range(args.e2e_steps):
            t0 = time.perf_counter()
            e2e_hash()
            dts.append(time.perf_counter() - t0)
        dt = _median(dts)
        e2e = {"value": n * world / dt, "unit": "rows/s", "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8,
               "ms_per_step": dt * 1e3, "timing": E2E_TIMING}
    elif args.e2e_steps > 0 and (sel is not None or lift is not None or W == 128):
        # host columns -> device (pinned, on the step's stream), selection /
        # aggregation / lifting and the release through the C ABI, released
        # cells -> host
        h_keys = torch.from_numpy(wl.keys).pin_memory()
        h_gids = torch.from_numpy(wl.gids).pin_memory()
        h_vals = [torch.from_numpy(v).pin_memory() for v in wl.values[:C]]
        rel_specs, rel_n = specs, n_specs
        if lift is not None:
            rel_specs = B.make_specs([(B.PAC_LIFTED, B.PAC_EXACT, B.PAC_F64, 0, lift[3].data_ptr())])
            rel_n = 1
        rel_cells = G * rel_n
        h_noised = torch.empty(rel_cells, dtype=torch.float64).pin_memory()
        h_null = torch.empty(rel_cells, dtype=torch.uint8).pin_memory()
        h_flags = torch.empty(rel_cells, dtype=torch.int32).pin_memory()
        rel_mode = B.PAC_FIN_ADAPTIVE if in_step_finalize else B.PAC_FIN_INDEPENDENT

        def e2e_step(i):
            with torch.cuda.stream(stream):
                d_keys.copy_(h_keys, non_blocking=True)
                d_gids.copy_(h_gids, non_blocking=True)
                for d, h in zip(d_vals, h_vals):
                    d.copy_(h, non_blocking=True)
                aggregate(sptr)
                if lift is not None:
                    B.pac_lift(ctx, lift[0], 2, G, lift[1], lift[2], lift[3].data_ptr(), sptr)
                (B.pac_finalize128 if W == 128 else B.pac_finalize)(
                    ctx, rel_specs, rel_n, G, meta.data_ptr(), 100 + i, 1.0 / 128, rel_mode, noised.data_ptr(),
                    is_null.data_ptr(), flags.data_ptr(), 0, sptr)
                h_noised.copy_(noised[:rel_cells], non_blocking=True)
                h_null.copy_(is_null[:rel_cells], non_blocking=True)
                h_flags.copy_(flags[:rel_cells], non_blocking=True)
            torch.cuda.synchronize()

        for i in range(2):
            e2e_step(i)
        dts = []
        for i in range(args.e2e_steps):
            t0 = time.perf_counter()
            e2e_step(2 + i)
            dts.append(time.perf_counter() - t0)
        dt = _median(dts)
        e2e = {"value": n * world / dt, "unit": "rows/s", "h2d_bytes_per_step": n * wcfg["in_bytes_per_row"],
               "d2h_bytes_per_step": rel_cells * (8 + 1 + 4), "ms_per_step": dt * 1e3, "timing": E2E_TIMING}
    elif args.e2e_steps > 0:
        h_keys = torch.from_numpy(wl.keys).pin_memory()
        h_gids = torch.from_numpy(wl.gids).pin_memory() if wl.gids is not None else None
        h_vals = [torch.from_numpy(v).pin_memory() for v in wl.values[:C]]
        h_noised = torch.empty(n_cells, dtype=torch.float64).pin_memory()
        h_null = torch.empty(n_cells, dtype=torch.uint8).pin_memory()
        h_flags = torch.empty(n_cells, dtype=torch.int32).pin_memory()
        hin = B.make_input(h_keys.data_ptr(), n, query_key=qk,
                           group_ids=h_gids.data_ptr() if h_gids is not None else 0,
                           gid_bytes=wcfg["gid_bytes"], n_groups=G)
        hspecs = B.make_specs(_spec_list(B, wcfg, [v.data_ptr() for v in h_vals], [1] * n_specs))
        mode = B.PAC_FIN_ADAPTIVE if in_step_finalize else B.PAC_FIN_INDEPENDENT
        for i in range(2):
            B.pac_query_host(ctx, hin, hspecs, n_specs, 7 + i, 1.0 / 128, mode, h_noised.data_ptr(),
                             h_null.data_ptr(), h_flags.data_ptr(), sptr)
        dts = []
        for i in range(args.e2e_steps):
            t0 = time.perf_counter()
            B.pac_query_host(ctx, hin, hspecs, n_specs, 100 + i, 1.0 / 128, mode, h_noised.data_ptr(),
                             h_null.data_ptr(), h_flags.data_ptr(), sptr)
            dts.append(time.perf_counter() - t0)
        dt = _median(dts)
        h2d = n * wcfg["in_bytes_per_row"]
        d2h = n_cells * (8 + 1 + 4)
        e2e = {"value": n * world / dt, "unit": "rows/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": dt * 1e3, "timing": E2E_TIMING}

    peak, peak_src = _peaks()
    out_bytes = 0 if wcfg.get("hash_only") else G * W * 8 * n_specs + G * (16 if W == 64 else 24)
    algo_bytes = n * wcfg["in_bytes_per_row"] + out_bytes
    achieved = algo_bytes / (agg_med / 1e3) / 1e9
    path_name = {1: "per-bit CUDA cores", 2: "tcgen05 tensor cores",
                 3: "per-bit engine (rows partitioned by group first when the groups' states exceed "
                    "shared memory)",
                 4: "one launch on CUDA cores (warp bit-transpose, int128 sums, last CTA writes the outputs)",
                 5: "rows partitioned by group, then tcgen05 tensor cores over the group-ordered rows "
                    "(bulk-copy staged; groups of at most 32 rows summed by one warp each)"
                 }.get(path, str(path))
    if wcfg.get("hash_only"):
        path_name = "k_hash_keys (16-byte vector loads and stores, grid = SMs x 8)"
    kernel = {1: "per-bit CUDA-core aggregation (all launches of pac_aggregate_multi)",
              2: ("k_select_prep + k_select + k_agg_mma + k_mma_finish (all launches of pac_aggregate_select)"
                  if sel is not None else "k_agg_mma + k_mma_finish (all launches of pac_aggregate_multi)"),
              3: "k_batch_agg + k_batch_merge, after k_part_hist + k_part_scan + k_part_scatter when the "
                 "rows are partitioned by group (all launches of pac_aggregate_multi)",
              4: "k_small_agg (the only launch of pac_aggregate_multi)",
              5: "k_part_hist + k_part_scan + k_part_scatter + k_range_tiles + k_range_plan + k_range_cuts + "
                 "k_part_mma + k_part_merge + k_part_small (all launches of pac_aggregate_multi)"}.get(path, str(path))
    if wcfg.get("hash_only"):
        kernel = "k_hash_keys (the only launch of pac_hash_keys)"
    if wcfg.get("approx"):
        # the exact specs (COUNT and the row counts) take `path`; each distinct
        # value column of an approximate spec runs one cascade
        kernel = ("k_apx_chunks + k_apx_combine_level + k_apx_emit per approximate value column, plus "
                  f"{path_name} for the exact specs (all launches of pac_aggregate_multi)")
        path_name = f"approximate cascades + {path_name} (exact specs)"
    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            cpu = cpu_baseline(workload, n, args.cpu_rows, args.cpu_rows_all)
        l2 = ("L2 flushed before every step (512 MB write), inputs 16 MB" if flush is not None else
              f"inputs {n * wcfg['in_bytes_per_row'] / 1e9:.2f} GB > 129 MB L2 (no flush needed)")
        line = {
            "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": workload, "rows": n, "groups": G, "value_columns": C, "worlds": 64,
                       "aggregates": wcfg["describe"], "l2": l2, "agg_path": path_name, "timing": timing,
                       **({"minmax_prune": bool(args.minmax_prune)} if "max" in wcfg["aggs"] else {})},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": _traffic(workload, n, path),
                         "traffic_kernel": _traffic_kernel(workload, n, path)[1] or kernel.split(" ")[0],
                         "kernel": kernel, "algorithmic_bytes": algo_bytes, "peak_source": peak_src,
                         "agg_ms": agg_med, "agg_ms_min": min(agg_ms)},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks.summary(),
        }
        if fin_ms is not None:
            line["finalize_ms"] = fin_ms
        if fin_adaptive_ms is not None:
            line["finalize_adaptive_ms"] = fin_adaptive_ms
        if m128 is not None:
            line["m128"] = m128
        if lift is not None and lift_ms:
            lms = statistics.median(a.elapsed_time(b) for a, b in lift_ms)
            lb = G * 64 * (8 + 8 + 8)   # two operand vectors in, the lifted vector out
            line["lift"] = {"kernel": "k_lift", "ms": lms, "bytes": lb, "achieved_gbs": lb / (lms / 1e3) / 1e9,
                            "frac": lb / (lms / 1e3) / 1e9 / peak, "cells": G * 64}
    B.pac_destroy(ctx)
    del d_keys, d_gids, d_vals, outs, flush
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return line


# The default run: the headline workload, then (one GPU) one entry per other
# configuration of the benchmark suite inside the same JSON line.
SUITE = ("ungrouped_1m", "highcard_100m", "batch_4096", "serving")


def run_ours(args):
    import torch
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    line = measure(args, args.workload or "lowcard_60m")
    if args.workload is None and world == 1 and not args.no_suite:
        line["workloads"] = {w: measure(args, w, suite=True) for w in SUITE}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def measure(args, workload: str, suite: bool = False):
    if workload == "batch_4096":
        return measure_batch(args, suite=suite)
    if workload == "serving":
        return measure_serving(args)
    return measure_single(args, workload, rows=None if suite else args.rows, suite=suite)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=None, choices=sorted(WORKLOADS),
                    help="one workload; default: lowcard_60m as the headline plus (one GPU) an entry per "
                         "configuration of the suite in `workloads`")
    ap.add_argument("--no-suite", action="store_true", help="default run: the headline workload only")
    ap.add_argument("--rows", type=int, default=None, help="override the workload's row count")
    ap.add_argument("--path", default=None, choices=[None, "auto", "bitloop", "mma", "engine", "small", "part"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--minmax-prune", type=int, default=1, choices=[0, 1],
                    help="MIN/MAX bound pruning on the per-bit engine (results are identical either way)")
    ap.add_argument("--cpu-rows", type=int, default=4_000_000, help="CPU baseline: rows of the one-thread leg")
    ap.add_argument("--cpu-rows-all", type=int, default=16_000_000,
                    help="CPU baseline: rows of the all-cores leg")
    ap.add_argument("--ref-rows", type=int, default=8_000_000,
                    help="--impl reference: rows per step (all host cores)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--queries", type=int, default=4096, help="batch_4096: number of queries")
    ap.add_argument("--no-autotune", action="store_true", help="batch_4096: default plan configuration")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: Poisson arrival rate (queries/s)")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="serving: seconds of arrivals")
    ap.add_argument("--pool", type=int, default=64, help="serving: resident query shapes")
    ap.add_argument("--ring", type=int, default=512, help="serving: output slots (outstanding requests)")
    ap.add_argument("--serve-mem-gb", type=int, default=32, help="serving: server arena (GiB)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
