// pac_mma.h -- the tensor-core (tcgen05) aggregation path.
#pragma once

#include "pac_ctx.h"

namespace pacgpu {

// True when every spec is COUNT or an exact int64 SUM/AVG and the group
// count fits the tensor-memory accumulators.
bool mma_supported(const pac_input *in, const pac_agg_spec *specs, int n_specs);

pac_status run_mma(pac_ctx *ctx, const pac_input *in, const pac_agg_spec *specs, int n_specs,
                   uint64_t *meta, cudaStream_t stream, int *launches);

}  // namespace pacgpu
