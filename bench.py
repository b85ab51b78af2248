"""Benchmark of the PAC stochastic-aggregation hot path on GB300.

One step = one PAC query over the 60M-row, 4-group, 4-column low-cardinality
workload: hash of the PU keys, per-group per-world COUNT + 4 exact SUMs + 4
exact AVGs over the m = 64 worlds, and the adaptive finalize (variance under
the posterior + PAC noise) of all 36 cells.  Inputs are resident in HBM and
larger than L2 (2.46 GB), so no flush is needed between steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
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
WORKLOAD = "lowcard_60m"
BYTES_PER_ROW = 8 + 1 + 4 * 8   # int64 PU key + uint8 group id + four int64 value columns


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


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


def _specs_for(w, B, outs):
    specs = [(B.PAC_COUNT, B.PAC_EXACT, B.PAC_I64, 0, outs[0])]
    for k in range(4):
        specs.append((B.PAC_SUM, B.PAC_EXACT, B.PAC_I64, w["vals"][k], outs[1 + k]))
    for k in range(4):
        specs.append((B.PAC_AVG, B.PAC_EXACT, B.PAC_I64, w["vals"][k], outs[5 + k]))
    return specs


def cpu_oracle_sample(rows: int, seed: int = 0):
    """Times the oracle (as it stands) on the first `rows` rows of the workload."""
    import oracle as orc
    from paper_2603_15023_gb300 import inputs
    wl = inputs.lowcard_60m(seed=seed, n=rows)
    qk = orc.query_key(seed)
    t0 = time.perf_counter()
    masks = orc.hash_keys(wl.keys, qk, orc.BALANCED)
    res = [orc.aggregate(masks, None, wl.gids, 4, orc.COUNT)]
    for v in wl.values:
        res.append(orc.aggregate(masks, v, wl.gids, 4, orc.SUM))
    for v in wl.values:
        res.append(orc.aggregate(masks, v, wl.gids, 4, orc.AVG))
    y = np.stack([r[0].astype(np.float64) for r in res], axis=1)
    scales = [2.0] * 5 + [1.0] * 4
    orc.finalize(y, scales, res[0][1], res[0][2], 99, 1.0 / 128, orc.ADAPTIVE)
    dt = time.perf_counter() - t0
    return rows / dt, dt


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    rows = args.ref_rows
    vals = []
    for i in range(args.warmup + args.steps):
        v, dt = cpu_oracle_sample(rows)
        if i >= args.warmup:
            vals.append((v, dt))
    value = statistics.median(v for v, _ in vals)
    ms = statistics.median(dt for _, dt in vals) * 1e3
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "rows": rows, "groups": 4, "value_columns": 4,
                   "aggregates": "count + 4 sum + 4 avg, exact", "worlds": 64},
        "cpu_baseline": {"value": value, "unit": "rows/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {rows} rows of {WORKLOAD}, one thread"},
        "e2e": {"value": value, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch
    from paper_2603_15023_gb300 import binding as B
    from paper_2603_15023_gb300 import inputs

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    ctx = B.pac_create(local)
    if args.path:
        B.pac_set_option(ctx, "agg_path", {"auto": 0, "bitloop": 1, "mma": 2}[args.path])

    wl = inputs.lowcard_60m(seed=rank, n=args.rows)
    n, G = wl.n, wl.n_groups
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    d_keys = torch.from_numpy(wl.keys).cuda()
    d_gids = torch.from_numpy(wl.gids).cuda()
    d_vals = [torch.from_numpy(v).cuda() for v in wl.values]
    outs = [torch.empty((G, 64), dtype=torch.int64 if i < 5 else torch.float64, device="cuda") for i in range(9)]
    meta = torch.empty((G, 2), dtype=torch.int64, device="cuda")
    n_cells = G * 9
    noised = torch.empty(n_cells, dtype=torch.float64, device="cuda")
    is_null = torch.empty(n_cells, dtype=torch.uint8, device="cuda")
    flags = torch.empty(n_cells, dtype=torch.int32, device="cuda")
    qk = B.pac_query_key(rank)
    inp = B.make_input(d_keys.data_ptr(), n, query_key=qk, group_ids=d_gids.data_ptr(), gid_bytes=1, n_groups=G)
    w = {"vals": [v.data_ptr() for v in d_vals]}
    specs = B.make_specs(_specs_for(w, B, [o.data_ptr() for o in outs]))

    def step(i, ev=None):
        if ev is not None:
            ev[0].record(stream)
        B.pac_aggregate_multi(ctx, inp, specs, 9, meta.data_ptr(), sptr)
        if ev is not None:
            ev[1].record(stream)
        B.pac_finalize(ctx, specs, 9, G, meta.data_ptr(), 1000 + i, 1.0 / 128, B.PAC_FIN_ADAPTIVE,
                       noised.data_ptr(), is_null.data_ptr(), flags.data_ptr(), 0, sptr)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    st = B.pac_sync_status(ctx, sptr)
    if st != B.PAC_OK:
        raise RuntimeError(B.status_name(st))
    agg_launches = B.pac_get_info(ctx, "last_path")
    path = B.pac_get_info(ctx, "last_path")

    clocks = ClockSampler(local)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    start.record(stream)
    launches = 0
    for i in range(args.steps):
        step(args.warmup + i, evs[i])
        launches += B.pac_get_info(ctx, "last_launches")  # finalize's launch
    end.record(stream)
    torch.cuda.synchronize()
    clocks.stop()
    # aggregation launches per step (the finalize call overwrote last_launches)
    B.pac_aggregate_multi(ctx, inp, specs, 9, meta.data_ptr(), sptr)
    torch.cuda.synchronize()
    agg_launches = B.pac_get_info(ctx, "last_launches")
    launches += agg_launches * args.steps
    total_ms = start.elapsed_time(end)
    agg_ms = [a.elapsed_time(b) for a, b in evs]
    ms_step = total_ms / args.steps
    t = torch.tensor([ms_step, statistics.mean(agg_ms)], dtype=torch.float64)
    if world > 1:
        import torch.distributed as dist
        t = t.cuda()
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t = t.cpu()
    ms_step, agg_mean = float(t[0]), float(t[1])
    value = n * world / (ms_step / 1e3)

    # end to end through the C ABI from pinned host memory
    e2e = None
    if args.e2e_steps > 0:
        h_keys = torch.from_numpy(wl.keys).pin_memory()
        h_gids = torch.from_numpy(wl.gids).pin_memory()
        h_vals = [torch.from_numpy(v).pin_memory() for v in wl.values]
        h_noised = torch.empty(n_cells, dtype=torch.float64).pin_memory()
        h_null = torch.empty(n_cells, dtype=torch.uint8).pin_memory()
        h_flags = torch.empty(n_cells, dtype=torch.int32).pin_memory()
        hin = B.make_input(h_keys.data_ptr(), n, query_key=qk, group_ids=h_gids.data_ptr(), gid_bytes=1,
                           n_groups=G)
        hw = {"vals": [v.data_ptr() for v in h_vals]}
        hspecs = B.make_specs(_specs_for(hw, B, [1] * 9))
        for i in range(2):
            B.pac_query_host(ctx, hin, hspecs, 9, 7 + i, 1.0 / 128, B.PAC_FIN_ADAPTIVE, h_noised.data_ptr(),
                             h_null.data_ptr(), h_flags.data_ptr(), sptr)
        t0 = time.perf_counter()
        for i in range(args.e2e_steps):
            B.pac_query_host(ctx, hin, hspecs, 9, 100 + i, 1.0 / 128, B.PAC_FIN_ADAPTIVE, h_noised.data_ptr(),
                             h_null.data_ptr(), h_flags.data_ptr(), sptr)
        dt = (time.perf_counter() - t0) / args.e2e_steps
        h2d = n * BYTES_PER_ROW
        d2h = n_cells * (8 + 1 + 4)
        e2e = {"value": n * world / dt, "unit": "rows/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": dt * 1e3}

    peak, peak_src = _peaks()
    algo_bytes = n * BYTES_PER_ROW
    achieved = algo_bytes / (agg_mean / 1e3) / 1e9
    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            v, dt = cpu_oracle_sample(args.cpu_rows)
            cpu = {"value": v, "unit": "rows/s", "cores": 1, "kind": "oracle",
                   "sample": f"first {args.cpu_rows} rows of {WORKLOAD} (COUNT + 4 SUM + 4 AVG + finalize), "
                             f"one thread, {dt:.1f} s"}
        line = {
            "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "rows": n, "groups": G, "value_columns": 4, "worlds": 64,
                       "aggregates": "count + 4 sum + 4 avg, exact; adaptive finalize of 36 cells",
                       "l2": "inputs 2.46 GB > 129 MB L2 (no flush needed)",
                       "agg_path": {1: "per-bit CUDA cores", 2: "tcgen05 tensor cores"}.get(path, str(path))},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "aggregation (main + merge)",
                         "peak_source": peak_src, "agg_ms": agg_mean},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks.summary(),
        }
        print(json.dumps(line))
    B.pac_destroy(ctx)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--rows", type=int, default=60_000_000)
    ap.add_argument("--path", default=None, choices=[None, "auto", "bitloop", "mma"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-rows", type=int, default=4_000_000)
    ap.add_argument("--ref-rows", type=int, default=1_000_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
