// pac_part_mma.h -- the many-group tensor-core aggregation over the
// group-ordered rows of the partition (pac_part_mma.cu).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "pac.h"
#include "pac_internal.cuh"

namespace pacgpu {

// The automatic path choice takes the many-group tensor-core path above this
// many groups (fewer groups: the few-group tensor-core path or the per-bit
// engine's per-warp states, which need no partition).
constexpr uint32_t kPartMmaAutoGroups = 64;

struct PartMmaArgs {
    InputDev in;                 // the query (n, n_groups, flags, hash mode)
    const void *rec;             // [n] group-ordered 16-byte records {mask, value}
    const uint32_t *sgid;        // [n] group-ordered group ids, 16 bytes readable past the end (unpacked)
    int packed;                  // records {low mask word | group id << 32, value}: balanced keys, no sgid
    const uint32_t *pcnt;        // [G + 2]: rows per group, [G] = rows kept
    const uint32_t *pend;        // [G]: end of each group's rows (the scatter's cursors)
    const pac_agg_spec *specs;   // COUNT and exact int64 SUM/AVG of one column
    int n_specs;
    uint64_t *meta;              // [G][2] or null
    void *scratch;               // part_mma_scratch_bytes
    uint32_t *status;
    int n_sms;
    uint64_t wait_ns;            // 0: 2 s
};

bool part_mma_specs_served(const pac_agg_spec *specs, int n_specs);
size_t part_mma_scratch_bytes(uint64_t n, uint32_t n_groups, int n_sms);
pac_status part_mma_launch(const PartMmaArgs &a, cudaStream_t stream, int *launches, const char **why);

}  // namespace pacgpu
