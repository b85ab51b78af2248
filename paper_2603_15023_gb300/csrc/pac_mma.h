// pac_mma.h -- the tensor-core (tcgen05) aggregation path.
#pragma once

#include "pac_ctx.h"

namespace pacgpu {

// True when every spec is COUNT or an exact int64 SUM/AVG and the group
// count fits the tensor-memory accumulators.
bool mma_supported(const pac_input *in, const pac_agg_spec *specs, int n_specs);

pac_status run_mma(pac_ctx *ctx, const pac_input *in, const pac_agg_spec *specs, int n_specs,
                   uint64_t *meta, cudaStream_t stream, int *launches);

// Scratch (accumulators and row counts) the tensor-core path needs.
size_t mma_scratch_bytes(const pac_input *in, const pac_agg_spec *specs, int n_specs);

// Enqueues the tensor-core path with caller-provided scratch and status word.
pac_status mma_launch(const pac_input *in, const pac_agg_spec *specs, int n_specs, uint64_t *meta,
                      cudaStream_t stream, void *scratch, uint32_t *status, int n_sms, int *launches,
                      const char **why);

}  // namespace pacgpu
