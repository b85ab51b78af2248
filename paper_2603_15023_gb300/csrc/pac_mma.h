// pac_mma.h -- the tensor-core (tcgen05) aggregation path.
#pragma once

#include "pac_ctx.h"

namespace pacgpu {

// True when every spec is COUNT or an exact int64 SUM/AVG and the group
// count fits the tensor-memory accumulators.
bool mma_supported(const pac_input *in, const pac_agg_spec *specs, int n_specs);

// The same test on the specs and the group count alone, whatever the row
// count (mma_supported also needs n > 0).
bool mma_specs_served(uint32_t n_groups, const pac_agg_spec *specs, int n_specs);

// Largest scratch mma_scratch_bytes returns for a query the path serves:
// 512 tensor-memory columns x 64 worlds of 8-byte digit totals, 256 bytes of
// alignment and the row counts of at most 8 groups.
constexpr size_t kMmaMaxScratchBytes = 512 * 64 * 8 + 256 + 8 * 8;

pac_status run_mma(pac_ctx *ctx, const pac_input *in, const pac_agg_spec *specs, int n_specs,
                   uint64_t *meta, cudaStream_t stream, int *launches);

// Scratch (accumulators and row counts) the tensor-core path needs.
size_t mma_scratch_bytes(const pac_input *in, const pac_agg_spec *specs, int n_specs, int worlds = 64);

// Enqueues the tensor-core path with caller-provided scratch and status word.
// wait_ns: limit of the kernel's pipeline waits (0: the default of 2 s).
// worlds: 64, or 128 (masks [n][2], or keys hashed with query_key and
// qkey2; meta [G][3]).  PAC_E_UNSUPPORTED when the tile does not fit shared
// memory.
pac_status mma_launch(const pac_input *in, const pac_agg_spec *specs, int n_specs, uint64_t *meta,
                      cudaStream_t stream, void *scratch, uint32_t *status, int n_sms, int *launches,
                      const char **why, uint64_t wait_ns = 0, int worlds = 64, uint64_t qkey2 = 0);

}  // namespace pacgpu
