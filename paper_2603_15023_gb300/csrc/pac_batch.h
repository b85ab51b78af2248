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
    int32_t bal;   // balanced keyed masks: worlds 32..63 are the complements of 0..31
    int32_t prune; // MIN/MAX bound pruning (rows that improve no world skip the update)
    int32_t pack;  // balanced keys: partition records {low mask word | group id << 32, slot 0
                   // value} (the high word is the complement of the low one), no sgid
    SlotDev slot[kMaxSpecs];
    OutDev outs[kMaxSpecs];
    uint64_t *meta;
    // per-world states [quantity][G][64], quantity 0 = COUNT, 1+s = slot s.
    // With bal, COUNT and SUM states hold worlds 0..31 in entries 0..31 and
    // the group's total in entry 32 (worlds 32..63 = total - world j-32);
    // MIN/MAX states always hold all 64 worlds.
    uint64_t *state;  // mode 0: [n_items][1+n_slots][G][64] partials; mode 1: [1+n_slots][G][64]
    uint64_t *ng;     // mode 0: [n_items][G]; mode 1: [G]
    unsigned long long *abs;  // mode 1: [n_slots] running sums of |v| (zeroed)
    uint32_t first_item, n_items;
    // mode 1: the rows partitioned by group before aggregation, so that runs
    // of one group are long and atomics are paid once per run
    uint32_t *pcnt;   // [G+2] rows per group (zeroed); [G] = rows kept, [G+1] = hot flag (after the scan)
    uint32_t *pcur;   // [G] scatter cursors
    uint64_t *smask;  // [n] 16-byte records {world mask, slot 0 value} in group order
    uint32_t *sgid;   // [n] group ids in group order
    uint64_t *sval;   // [n_slots-1][n] values of slots 1.. (64-bit patterns) in group order
};

struct BatchItem {
    uint32_t q, k;     // query, item index within the query
    uint64_t row0;
    uint32_t rows, pad;
};

struct BatchConfig {
    uint32_t item_rows;  // rows per work item
    size_t smem_cap;     // warp-private states only when they fit this many bytes
    // every query partitioned, no aggregation states and no aggregation
    // launches: the plan ends with the group-ordered copies (read by the
    // many-group tensor-core kernel)
    bool partition_only = false;
};
constexpr BatchConfig kBatchDefault = {1u << 16, 100 * 1024};

// The zeroed head of a plan's device block (256 bytes): the work-item
// counter at 0, the server's status word at 8, and at kPlanSpanOffset two
// uint64 words that the aggregation kernel fills with the device-time span
// it ran in (~earliest block start, latest block end; %globaltimer ns).
constexpr size_t kPlanSpanOffset = 16;

// A partitioned query with more groups than this scans its group counts with
// a multi-block scan of up to kWideScanBlocks blocks (16K groups or more per
// block) instead of one block per query.  Its block sums and maxima follow
// the query's pcnt[G+2] counters (2 * kWideScanBlocks more words, zeroed).
constexpr uint32_t kWideScanGroups = 32768;
constexpr uint32_t kWideScanBlocks = 64;
inline uint32_t wide_scan_blocks(uint32_t G) {
    const uint32_t nb = (G + 16383) / 16384;
    return nb < kWideScanBlocks ? nb : kWideScanBlocks;
}

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
    int sig = 0;  // shared slot signature (0: operations read at run time)
    size_t smem = 0;
    int n_ctas = 0;
    int n_warp_private = 0, n_atomic = 0;
    int n_wide = 0;  // partitioned queries with the multi-block scan
    pacgpu::BatchConfig cfg{};
    uint64_t total_cells = 0;
    std::vector<unsigned char> image;
    size_t img_q = 0, img_items = 0, img_prefix = 0, img_fin = 0;
    std::vector<size_t> rel_state, rel_ng, rel_abs;  // per query, relative to the device block
    std::vector<size_t> rel_pcnt, rel_pcur, rel_smask, rel_sgid, rel_sval;  // mode-1 partition buffers
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
