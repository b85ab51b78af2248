// pac_batch.h -- batched-query plans: device descriptors shared by the batch
// kernels, and the host-side plan object used by pac_batch_* and the server.
#pragma once

#include <vector>

#include "pac_ctx.h"
#include "pac_kernels.h"

namespace pacgpu {

constexpr int kBatchWarps = 8;

struct BatchQueryDev {
    InputDev in;
    int32_t n_slots, n_out;
    int32_t mode;  // 0: warp-private shared-memory states, 1: global atomics
    int32_t pad;
    SlotDev slot[kMaxSpecs];
    OutDev outs[kMaxSpecs];
    uint64_t *meta;
    uint64_t *state;  // mode 0: [n_items][1+n_slots][G][64] partials; mode 1: [1+n_slots][G][64]
    uint64_t *ng;     // mode 0: [n_items][G]; mode 1: [G]
    unsigned long long *abs;  // mode 1: [n_slots] running sums of |v| (zeroed)
    uint32_t first_item, n_items;
};

struct BatchItem {
    uint32_t q, k;     // query, item index within the query
    uint64_t row0;
    uint32_t rows, pad;
};

struct BatchConfig {
    uint32_t item_rows;  // rows per work item
    size_t smem_cap;     // warp-private states only when they fit this many bytes
};
constexpr BatchConfig kBatchDefault = {1u << 16, 100 * 1024};

}  // namespace pacgpu

// A plan: host image of the device descriptors plus the device layout.
// Device memory (one block, plan-owned or placed by the server):
//   [zeroed scratch: item counter, atomic states | item partials | image]
// image = [BatchQueryDev x n_queries | BatchItem x n_items |
//          uint64 cell prefix x (n_queries+1) | FinParams x n_rel].
struct pac_batch {
    int device = 0;
    int n_queries = 0;
    uint32_t n_items = 0;
    int n_rel = 0;
    int ns = 1;
    size_t smem = 0;
    int n_ctas = 0;
    int n_warp_private = 0, n_atomic = 0;
    pacgpu::BatchConfig cfg{};
    uint64_t total_cells = 0;
    std::vector<unsigned char> image;
    size_t img_q = 0, img_items = 0, img_prefix = 0, img_fin = 0;
    std::vector<size_t> rel_state, rel_ng, rel_abs;  // per query, relative to the device block
    size_t zero_bytes = 0, image_off = 0, device_bytes = 0;
    void *dbuf = nullptr;
    bool owns_dbuf = false;
    uint32_t *d_status = nullptr;
};

namespace pacgpu {

// Host-side layout of a batch (no CUDA call).  *out owns no device memory.
pac_status plan_build(pac_ctx *ctx, const pac_query *qs, int n_queries, const BatchConfig &cfg, pac_batch **out);
// Places the plan at `dbuf` (plan->device_bytes bytes): patches every
// device pointer of the image.
void plan_bind(pac_batch *b, void *dbuf);
// Work-item grid and dynamic shared memory for the plan on this device.
pac_status plan_setup_kernel(pac_ctx *ctx, pac_batch *b);
// Enqueues: the image copy from `image_src` (host; pinned for an
// asynchronous copy) when non-null, the scratch memset and the kernels.
pac_status plan_enqueue(pac_ctx *ctx, pac_batch *b, cudaStream_t s, const void *image_src);
// Frees the plan (and its device block when the plan owns it).
void plan_destroy(pac_batch *b);
// Argument checks of one batched query (PAC_E_INVALID / PAC_E_UNSUPPORTED).
pac_status check_query(pac_ctx *ctx, const pac_query *q);

}  // namespace pacgpu
