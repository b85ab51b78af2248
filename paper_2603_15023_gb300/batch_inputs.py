"""Device-resident columns and query descriptors of the batched workload.

Generates every query's columns of an ``inputs.BatchSpec`` directly in HBM
with the counter-based generator of ``libpacgen.so`` (one arena for all
columns), allocates every query's outputs and builds the ``pac_query`` array
for ``pac_batch_plan``.  Memory plumbing only: nothing of the method is
computed here.
"""
from __future__ import annotations

from typing import List

import numpy as np

from . import binding as B
from . import gen
from .inputs import BatchSpec

# specs of every batched query: COUNT, exact SUM of the int64 column, exact
# SUM of the float32 column
SPEC_KINDS = ((B.PAC_COUNT, B.PAC_I64), (B.PAC_SUM, B.PAC_I64), (B.PAC_SUM, B.PAC_F32))
BYTES_PER_ROW = 8 + 4 + 8 + 4


class DeviceBatch:
    def __init__(self, spec: BatchSpec, queries=None, fin_mode: int = -1, stream: int = 0):
        import torch
        self.spec = spec
        idx = list(range(spec.n_queries)) if queries is None else list(queries)
        self.idx = idx
        rows = [int(spec.rows[q]) for q in idx]
        groups = [int(spec.groups[q]) for q in idx]
        self.total_rows = int(sum(rows))
        self.total_groups = int(sum(groups))
        # one arena per column type, 256-byte aligned query slices
        def offsets(sizes, align):
            off, out = 0, []
            for s in sizes:
                out.append(off)
                off += (s + align - 1) // align * align
            return out, off
        o8, n8 = offsets(rows, 32)
        o4, n4 = offsets(rows, 64)
        self.keys = torch.empty(max(n8, 1), dtype=torch.int64, device="cuda")
        self.vals = torch.empty(max(n8, 1), dtype=torch.int64, device="cuda")
        self.gids = torch.empty(max(n4, 1), dtype=torch.int32, device="cuda")
        self.fvals = torch.empty(max(n4, 1), dtype=torch.float32, device="cuda")
        og, ng = offsets([g * 64 for g in groups], 32)
        self.out_cnt = torch.empty(max(ng, 1), dtype=torch.int64, device="cuda")
        self.out_sum = torch.empty(max(ng, 1), dtype=torch.int64, device="cuda")
        self.out_fsum = torch.empty(max(ng, 1), dtype=torch.float64, device="cuda")
        om, nm = offsets([g * 2 for g in groups], 32)
        self.meta = torch.empty(max(nm, 1), dtype=torch.int64, device="cuda")
        oc, nc = offsets([g * 3 for g in groups], 32)
        self.noised = torch.empty(max(nc, 1), dtype=torch.float64, device="cuda")
        self.is_null = torch.empty(max(nc, 1), dtype=torch.uint8, device="cuda")
        self.flags = torch.empty(max(nc, 1), dtype=torch.int32, device="cuda")
        self.layout = []
        self._specs: List = []
        qlist = []
        for i, q in enumerate(idx):
            n, G, K = rows[i], groups[i], int(spec.keys[q])
            kp = self.keys.data_ptr() + 8 * o8[i]
            vp = self.vals.data_ptr() + 8 * o8[i]
            gp = self.gids.data_ptr() + 4 * o4[i]
            fp = self.fvals.data_ptr() + 4 * o4[i]
            gen.fill_i64(kp, n, spec.seed, 4 * q, 0, K, stream=stream)
            gen.fill_u32(gp, n, spec.seed, 4 * q + 1, G, stream=stream)
            gen.fill_i64(vp, n, spec.seed, 4 * q + 2, 1, 100_000, stream=stream)
            gen.fill_f32_1000(fp, n, spec.seed, 4 * q + 3, stream=stream)
            outs = (self.out_cnt.data_ptr() + 8 * og[i], self.out_sum.data_ptr() + 8 * og[i],
                    self.out_fsum.data_ptr() + 8 * og[i])
            specs = B.make_specs([(B.PAC_COUNT, B.PAC_EXACT, B.PAC_I64, 0, outs[0]),
                                  (B.PAC_SUM, B.PAC_EXACT, B.PAC_I64, vp, outs[1]),
                                  (B.PAC_SUM, B.PAC_EXACT, B.PAC_F32, fp, outs[2])])
            self._specs.append(specs)
            inp = B.make_input(kp, n, query_key=B.pac_query_key(1_000_000 + q), group_ids=gp, gid_bytes=4,
                               n_groups=G)
            qlist.append(B.make_query(inp, specs, 3, meta=self.meta.data_ptr() + 8 * om[i], fin_mode=fin_mode,
                                      seed=5_000 + q, budget=1.0 / 128,
                                      noised=self.noised.data_ptr() + 8 * oc[i],
                                      is_null=self.is_null.data_ptr() + oc[i],
                                      flags=self.flags.data_ptr() + 4 * oc[i]))
            self.layout.append((n, G, og[i], om[i], oc[i]))
        self.queries = B.make_queries(qlist)
        self.n_queries = len(qlist)

    def algorithmic_bytes(self) -> int:
        """Inputs read once plus every output and meta written once."""
        return self.total_rows * BYTES_PER_ROW + self.total_groups * (64 * 8 * len(SPEC_KINDS) + 16)

    def results(self, i: int):
        """Query i's (count uint64 [G,64], sum int64 [G,64], fsum float64 [G,64], meta uint64 [G,2])."""
        n, G, og, om, _ = self.layout[i]
        cnt = self.out_cnt[og:og + 64 * G].cpu().numpy().view(np.uint64).reshape(G, 64)
        sm = self.out_sum[og:og + 64 * G].cpu().numpy().reshape(G, 64)
        fs = self.out_fsum[og:og + 64 * G].cpu().numpy().reshape(G, 64)
        meta = self.meta[om:om + 2 * G].cpu().numpy().view(np.uint64).reshape(G, 2)
        return cnt, sm, fs, meta

    def query_key(self, i: int) -> int:
        return B.pac_query_key(1_000_000 + self.idx[i])
