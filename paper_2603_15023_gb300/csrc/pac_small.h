// pac_small.h -- the one-launch path for small ungrouped queries.
#pragma once

#include "pac_ctx.h"

namespace pacgpu {

// Rows up to which the automatic choice takes the one-launch path.
constexpr uint64_t kSmallAutoRows = 8ull << 20;

// True when the query has one group and every spec is COUNT or an exact
// int64 SUM / AVG over at most 4 distinct value columns.
bool small_supported(const pac_input *in, const pac_agg_spec *specs, int n_specs);

// One kernel: aggregation, then (its last CTA) COUNT / SUM / AVG and meta.
pac_status run_small(pac_ctx *ctx, const pac_input *in, const pac_agg_spec *specs, int n_specs,
                     uint64_t *meta, cudaStream_t stream, int *launches);

}  // namespace pacgpu
