// pac_mma.cu -- the tensor-core (tcgen05) aggregation path.
#include "pac_mma.h"

namespace pacgpu {

bool mma_supported(const pac_input *, const pac_agg_spec *, int) { return false; }

pac_status run_mma(pac_ctx *ctx, const pac_input *, const pac_agg_spec *, int, uint64_t *, cudaStream_t,
                   int *) {
    return fail(ctx, PAC_E_UNSUPPORTED, "tensor-core path not built");
}

}  // namespace pacgpu
