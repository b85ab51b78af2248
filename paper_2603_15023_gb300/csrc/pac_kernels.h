// pac_kernels.h -- launch parameters and launchers of the PAC kernels.
#pragma once

#include "pac_internal.cuh"

namespace pacgpu {

// Per-world state operations of the per-bit path.
enum SlotOp : int32_t {
    OP_ISUM = 0,       // exact int64 sum (wrapping partials, int128 merge)
    OP_FSUM_COMP = 1,  // FP32 sum + compensation (two-sum), exact variant
    OP_FSUM_PLAIN = 2, // FP32 state only (the paper's approximate float SUM)
    OP_IMIN = 3,
    OP_IMAX = 4,
    OP_FMIN = 5,
    OP_FMAX = 6,
};

struct SlotDev {
    int32_t op, vtype;
    const void *values;
};

struct OutDev {
    int32_t kind, slot;  // slot: index into SlotDev[] (unused for COUNT)
    void *out;
};

struct BitloopParams {
    InputDev in;
    int32_t n_slots, n_out;
    SlotDev slot[kMaxSpecs];
    OutDev outs[kMaxSpecs];
    uint64_t rows_per_cta;
    void *partials;         // lowcard: [ctas][1+n_slots][G][64]; atomic: [1+n_slots][G][64]
    uint64_t *ng_partials;  // lowcard: [ctas][G]; atomic: [G]
    uint64_t *meta;         // [G][2] or nullptr
    uint32_t *status;
    unsigned long long *abs_total;  // atomic path: running sum of |v| (zeroed)
};

int bitloop_pick_ns(int n_slots);
size_t bitloop_smem_bytes(int n_warps, int n_slots, uint32_t G, int ns);
cudaError_t launch_bitloop_lowcard(const BitloopParams &p, int n_ctas, int n_warps, cudaStream_t s);
cudaError_t launch_bitloop_atomic(const BitloopParams &p, int n_ctas, cudaStream_t s);
cudaError_t launch_bitloop_merge(const BitloopParams &p, int n_parts, bool atomic, cudaStream_t s);

// ---- hash --------------------------------------------------------------
cudaError_t launch_hash(const int64_t *keys, uint64_t *masks, size_t n, uint64_t qkey, int mode,
                        int n_sms, cudaStream_t s);

// ---- path dispatch of pac_aggregate_multi (checked arguments) -----------
pac_status aggregate_dispatch(pac_ctx *ctx, const pac_input *in, const pac_agg_spec *specs, int32_t n_specs,
                              uint64_t *meta, cudaStream_t stream);

// ---- PAC selection (Sec. 4.2 "PAC Selection") ---------------------------
struct SelectDev {
    const void *col;      // [n] of vtype
    const void *thr;      // [n_thr][64] of vtype
    const void *thr_ids;  // [n] or nullptr
    int32_t vtype, cmp, thr_id_bytes;
    uint32_t n_thr;
};
// One operand vector, sorted: key[0..n_valid) are the order-preserving keys
// of its non-NaN operands, ascending; pm[k] = the worlds of the k smallest.
struct SelTable {
    unsigned long long key[64];
    unsigned long long pm[65];
    uint32_t n_valid;
    uint32_t pad;
};
cudaError_t launch_select_prep(const SelectDev &sel, SelTable *tabs, cudaStream_t s);
// out[i] = mask_i & {j : col[i] <cmp> thr[t_i][j]}; an out-of-range t_i keeps
// no world and raises kStatusBadGroup.
cudaError_t launch_select(const InputDev &in, const SelectDev &sel, const SelTable *tabs, uint64_t *out,
                          uint32_t *status, int n_sms, cudaStream_t s);

// ---- approximate integer SUM / AVG (Sec. 5 "Approximation") -------------
constexpr int kApxLevels = 25;
constexpr int kApxChunk = 4096;
constexpr int kApxBlockChunks = 16;  // chunks per CTA of the cascade kernel (first tree levels)
// One (chunk-block, group) state: per side 25 levels x 32 packed words
// (world l in the low 16 bits, world l+32 in the high 16 bits) and 25
// level totals.
struct ApxSide {
    uint32_t w[kApxLevels][32];
    uint32_t t[kApxLevels];
};
struct ApxState {
    ApxSide side[2];
};

struct ApxParams {
    InputDev in;
    const int64_t *values;
    ApxState *states;   // [n_blocks][G]
    uint64_t *ng;       // [G] row counts (zeroed by the launcher)
    uint32_t *status;
    uint64_t n_chunks;
    uint32_t chunks_per_block;
    // COUNT and meta of the query from the same pass (or nullptr): cnt [G][64]
    // accumulators (zeroed by the launcher), count_out [G][64] uint64, meta
    // [G][2] {n_g, or_g}
    unsigned long long *cnt;
    unsigned long long *count_out;
    uint64_t *meta;
};

int apx_max_groups();
size_t apx_scratch_bytes(uint64_t n, uint32_t G);
// Fills out ([G][64] int64 for SUM, double for AVG).
cudaError_t launch_approx(const ApxParams &p, void *out_sum, void *out_avg, cudaStream_t s,
                          int *launches);

// ---- finalize -------------------------------------------------------------
struct FinSpec {
    int32_t kind, vtype, variant, pad;
    const void *out;
};
struct FinParams {
    FinSpec spec[kMaxSpecs];
    int32_t n_specs;
    uint32_t n_groups;
    const uint64_t *meta;
    uint64_t seed;
    double budget;
    int32_t mode;
    double *noised;
    uint8_t *is_null;
    uint32_t *flags;
    double *posterior;
};
// ---- vector-lifted expressions and pac_filter (Sec. 4.2; Sec. 3.2) -------
struct LiftOp {
    int32_t op, arg;
    double c;
};
struct LiftParams {
    const void *in[kMaxSpecs];  // operand vectors [n_groups*64]
    int32_t code[kMaxSpecs];    // bits 0-1: 0 uint64, 1 int64, 2 double; bit 2: scale 2
    LiftOp prog[32];
    int32_t n_ops;
    uint32_t n_groups;
    double *out;
};
cudaError_t launch_lift(const LiftParams &p, int n_sms, cudaStream_t s);
cudaError_t launch_filter(const double *b, uint32_t n_groups, uint64_t seed, uint8_t *keep, int n_sms,
                          cudaStream_t s);
cudaError_t launch_finalize(const FinParams &p, cudaStream_t s);
// The same release over 128 worlds (meta [G][3], results [G][128]).
cudaError_t launch_finalize128(const FinParams &p, cudaStream_t s);
// One warp per query: d_params[n] device array of per-query parameters.
cudaError_t launch_finalize_batch(const FinParams *d_params, int n, cudaStream_t s);

}  // namespace pacgpu
