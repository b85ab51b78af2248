// pac_part_mma.cu -- tensor-core COUNT and exact int64 SUM/AVG over many
// groups (Sec. 4.2 "PAC Aggregation" on a high-cardinality GROUP BY).
//
// Input: the query's rows in group order, as the partition (histogram, scan,
// scatter of pac_batch.cu) writes them: one 16-byte record per row, packed
// {low mask word | group id << 32, value} under balanced keys (the high mask
// word is the complement of the low one), else {world mask, value} with the
// group ids beside the records.  A group's rows are consecutive, so the
// per-group contraction D_g = Bits_g^T * Digits_g of the tensor-core path
// (E4M3 world bytes times E4M3 value digits, FP32 in tensor memory, exact:
// see pac_mma.cu) needs no sort.
//
// Work split: three small kernels cut the kept rows into R ranges of equal
// cost (a row costs 1, a group of more than 32 rows kGroupCost more), at most
// 2^16 rows each; k_part_mma runs one persistent CTA per SM, which takes the
// ranges one at a time from an atomic counter, the last range of the group
// order first (many small groups, the most output per row).  A range's rows
// arrive in 512-row chunks through bulk asynchronous copies (cp.async.bulk,
// one elected thread) into a ring in shared memory.  Each group is
// aggregated one of two ways:
//   - a group of at most 32 rows by k_part_small (one warp per 32 groups;
//     k_part_mma's classifier marks its rows to be skipped);
//   - a larger group, or one of more than 32 rows that crosses a range edge,
//     by the tensor cores: one 32-row MMA per 32-row block it touches, with
//     the block's world bytes as A and a B copy that holds the group's digits
//     and zeros in the block's other rows (at most two per block: such a
//     group always holds the block's first or last row).
// The MMAs of one group accumulate into one of sixteen tensor-memory slots (a
// ring over the range's tensor-core groups in order; the group's first MMA
// overwrites the slot, so a slot is never zeroed); the slot of a new group is
// taken once the epilogue has read it out.  When a group's last MMA is done,
// an epilogue warp set reads its slot and writes the group's COUNT/SUM/AVG
// and metadata; two sets drain alternate groups, since one group's drain is a
// chain of dependent latencies (tensor-memory load, conversion, the total's
// hand-over, stores) far longer than its issue time.  A group that crosses a
// range edge writes its digit totals as a partial record instead;
// k_part_merge adds the partials of each such group in range order.
// No result is written with an atomic operation.
//
// Warps: 0-15 producers (block w of every chunk), 16-19 and 20-23 the two
// epilogue sets (tensor-memory lane quadrant = warp % 4), 24 bulk-copy
// loader, 25 MMA issuer, 26 classifier (each chunk's group starts and edge
// classes, ahead of the producers, which then share no barrier).
// Every wait is bounded (%globaltimer); a wait that gives up stops its warp's
// work, the CTA drains what it has in flight, takes no further range and
// reports PAC_E_TIMEOUT.
#include <algorithm>
#include <climits>

#include "pac_internal.cuh"
#include "pac_kernels.h"
#include "pac_part_mma.h"
#include "pac_tc.cuh"

namespace pacgpu {

namespace {

using namespace tc;

constexpr int kChunk = 512;                // rows per bulk-copied chunk
constexpr int kBlocks = kChunk / 32;       // 32-row blocks per chunk
constexpr int kPairs = 2 * kBlocks;        // MMAs per chunk at most (two runs per block)
constexpr int kRawStages = 4;              // chunks in flight
constexpr int kOpStages = 2;               // operand stages
constexpr int kProdWarps = 16;             // one 32-row block each per chunk
constexpr int kBlocksPerWarp = kBlocks / kProdWarps;
constexpr int kEpiSets = 2;                // epilogue warp sets (set e drains the groups k = e mod kEpiSets)
constexpr int kEpiWarp0 = kProdWarps;      // set e: warps kEpiWarp0 + 4 e + q, lane quadrant q
constexpr int kLoadWarp = kEpiWarp0 + 4 * kEpiSets;
constexpr int kMmaWarp = kLoadWarp + 1;    // one issuing thread (more issuing warps did not pay)
constexpr int kClsWarp = kMmaWarp + 1;     // classifies each chunk's groups ahead of the producers
constexpr int kThreadsP = (kClsWarp + 1) * 32;
constexpr int kAlloc = 32;                 // tensor-memory columns per accumulator (a slot)
constexpr int kSlots = 512 / kAlloc;       // slots in the ring
constexpr int kFeat = 20;                  // COUNT, three pad features, 16 digits
constexpr int kInfo = 256;                 // per-group records of the ring (see the MMA warp)
constexpr int kNMax = 32;                  // B bytes per row: N for 16 digits
// rows per range at most (digit totals below 2^20: FP32 accumulation stays exact)
constexpr uint32_t kMaxRowsPerRange = 1u << 16;
// Range planning.  A range's time on one SM is close to (its rows) +
// kGroupCost x (its groups of more than 32 rows) row times: each such group
// is drained once by the epilogue, about 300 rows' worth (1.3 us against
// 4.2 ns a row, measured).  The rows are cut into ranges of equal cost, at
// most kRangeCost each (every row costs at least 1, so no range exceeds
// kMaxRowsPerRange rows once its ends are rounded down to chunk boundaries).
constexpr uint32_t kGroupCost = 300;
constexpr uint32_t kRangeCost = kMaxRowsPerRange - kChunk;
constexpr uint32_t kMinRangeCost = 8 * kChunk;  // fewer ranges than SMs rather than ranges below this
constexpr uint32_t kTileGroups = 4096;           // groups per planning tile
constexpr int kPlanThreads = 256;
constexpr uint32_t kNone = 0xFFFFFFFFu;

// one raw chunk: records, then group ids
constexpr uint32_t kRawRecBytes = kChunk * 16;
constexpr uint32_t kRawBytes = kRawRecBytes + kChunk * 4;
// one operand stage: A (512 rows x 64 world bytes) then B (kPairs copies of
// 32 rows x kNMax feature bytes)
constexpr uint32_t kABytes = kChunk * 64;
constexpr uint32_t kPairBytes = 32 * kNMax;
constexpr uint32_t kBBytes = kPairs * kPairBytes;
constexpr uint32_t kOpBytes = kABytes + kBBytes;
constexpr size_t kSmemP = static_cast<size_t>(kRawStages) * kRawBytes + kOpStages * kOpBytes;

static_assert(kSlots >= 2, "the slot ring needs two slots");
static_assert(kBlocks % kProdWarps == 0 && kProdWarps <= 32, "producer warps split the chunk's blocks evenly");
static_assert(kPairs == 32, "the MMA warp holds one pair per lane");
static_assert(kEpiWarp0 % 4 == 0, "epilogue warp q must own tensor-memory lane quadrant q");
static_assert(kSlots % kEpiSets == 0, "a slot's groups must all fall to one epilogue set");
static_assert(kAlloc >= kNMax, "a slot holds one accumulator of N = kNMax columns");
static_assert(kInfo >= kSlots + 3 * kPairs, "the group records must outlive the ring");

// One MMA of a chunk: a run of group `gid` in block (pair index / 2).
struct PairRec {
    uint32_t gid;
    uint16_t n;      // rows of the run that count (dropped rows excluded)
    uint8_t valid;
    uint8_t pad;
};

// A tensor-core group of the range in MMA order (ordinal k at k % kInfo).
struct OrdInfo {
    uint32_t gid;
    uint32_t n;
    uint32_t end;    // 1: no more groups (the epilogue stops)
    uint32_t pad;
};

struct PartShared {
    uint64_t raw_full[kRawStages];
    uint64_t raw_empty[kRawStages];
    uint64_t full[kOpStages];
    uint64_t empty[kOpStages];
    uint64_t done[kSlots];   // MMA warp (a commit + an arrive) -> epilogue: the slot's group is complete
    uint64_t freeb[kSlots];  // epilogue (the set's 3 or 4 warps) -> MMA warp: the slot has been read out
    uint64_t drain;
    uint32_t tmem_slot;
    int abort_flag;
    uint32_t range;          // the range in work (kNone: none left)
    uint32_t lo, hi;         // its rows [lo, hi)
    uint32_t split_lo;       // group crossing the range's left edge, or kNone
    uint32_t split_hi;       // group crossing its right edge, or kNone
    uint64_t cls_full[kRawStages];   // classifier -> producers: the chunk in raw slot r is classified
    uint8_t ccls[kRawStages][kBlocks];  // per raw slot and block: first-row class | last-row class << 2
    uint8_t pvalid[kOpStages][kProdWarps];  // valid pairs of warp w: bits 2bb, 2bb + 1 = block w + 16 bb
    uint32_t prev_gid0;              // chunk 0: the group crossing the left edge (or kNone) ...
    int prev_cls0;                   // ... and its class
    PairRec pairs[kOpStages][kPairs];
    OrdInfo info[kInfo];
    uint64_t tot_ready[kSlots];         // quadrant-2 epilogue warp -> quadrants 0, 1: the slot's total row
    long long tot[kSlots][kFeat];       // balanced keys: accumulator row 32 (the group total) per slot
    unsigned long long meta_or[kInfo];  // per group record: worlds with a nonzero count, ...
    uint32_t meta_cnt[kInfo];           // ... and the epilogue warps that have added theirs
};

}  // namespace

struct PartRec {
    uint32_t gid, used;
    unsigned long long n;
    long long d[kWorlds][kFeat];   // digit totals per accumulator row (units of 2^-18 folded out)
};

namespace {

// The ranges of k_part_mma (written by k_range_plan).
struct RangePlan {
    unsigned long long total;  // the kept rows' cost
    unsigned long long share;  // cost per range (at most kRangeCost)
    uint32_t n_ranges;         // R
    uint32_t next;             // ranges handed out so far (k_part_mma's counter)
};

struct PartMmaParams {
    InputDev in;
    const ulonglong2 *rec;     // [n] group-ordered {mask, value}
    const uint32_t *sgid;      // [n] group-ordered group ids (unpacked records)
    int32_t packed;            // records {low mask word | group id << 32, value} (balanced keys)
    const uint32_t *pcnt;      // [G + 2]: rows per group, [G] = rows kept
    const uint32_t *pend;      // [G]: end of each group's rows in the group order
    RangePlan *plan;
    uint32_t *range_lo;        // [R + 1]: range r = rows [range_lo[r], range_lo[r + 1])
    unsigned long long *tile;  // [ceil(G / kTileGroups)]: tile costs, then their exclusive sums
    uint32_t r_max;            // R at most (the partial records' capacity)
    int32_t bal;               // balanced keys: accumulator row 32 is the run total
    int32_t has_col;           // 0: COUNT only (the records carry no value)
    int32_t n_out;
    int32_t out_kind[kMaxSpecs];
    void *out[kMaxSpecs];
    uint64_t *meta;            // [G][2] {n_g, worlds with a nonzero count} or null
    PartRec *part;             // [R][2]: range r's records (used = 0 unless written)
    uint32_t *status;
    uint64_t wait_ns;
};

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// A record's world mask and group id.  Packed records (balanced keys) hold
// the low mask word and the group id in their first 8 bytes; the high mask
// word is the complement of the low one.
__device__ __forceinline__ uint64_t rec_mask(uint64_t x, bool packed) {
    if (!packed) return x;
    const uint64_t lo = x & 0xFFFFFFFFull;
    return lo | ((lo ^ 0xFFFFFFFFull) << 32);
}

struct GidView {
    const ulonglong2 *rec;
    const uint32_t *gid;
    bool packed;
    __device__ __forceinline__ uint32_t operator[](int i) const {
        return packed ? static_cast<uint32_t>(rec[i].x >> 32) : gid[i];
    }
};

__device__ __forceinline__ bool fits_i64(__int128 v) {
    return v >= static_cast<__int128>(LLONG_MIN) && v <= static_cast<__int128>(LLONG_MAX);
}

// The results of world w of group g: every output spec, overflow reported.
__device__ __forceinline__ void emit_world(const PartMmaParams &p, uint32_t g, int w, unsigned long long cnt,
                                           __int128 sum) {
    const size_t cell = static_cast<size_t>(g) * kWorlds + w;
    const bool fits = fits_i64(sum);
    bool used = false;
    for (int s = 0; s < p.n_out; s++) {
        const int k = p.out_kind[s];
        if (k == PAC_COUNT) {
            static_cast<unsigned long long *>(p.out[s])[cell] = cnt;
        } else if (k == PAC_SUM) {
            used = true;
            static_cast<long long *>(p.out[s])[cell] =
                fits ? static_cast<long long>(sum) : (sum < 0 ? LLONG_MIN : LLONG_MAX);
        } else {
            used = true;
            static_cast<double *>(p.out[s])[cell] = cnt ? i128_to_double(sum) / static_cast<double>(cnt) : 0.0;
        }
    }
    if (used && !fits) raise_status(p.status, kStatusOverflow);
}

// A group's SUM from its digit totals d[4 + q] (digit q, weight 16^q).  A
// digit total is below 2^24 in magnitude (at most 2^20 rows of digits below
// 16), so each half, sum_{q<8} d_q 16^q and sum_{q>=8} d_q 16^(q-8), stays
// below 2^53: two 64-bit Horner chains, joined once in 128 bits.
__device__ __forceinline__ __int128 digits_to_sum(const long long (&d)[kFeat]) {
    long long lo = 0, hi = 0;
#pragma unroll
    for (int q = 7; q >= 0; q--) {
        lo = lo * 16 + d[4 + q];
        hi = hi * 16 + d[12 + q];
    }
    return static_cast<__int128>(lo) + (static_cast<__int128>(hi) << 32);
}

// The same for digit totals added over several ranges (no bound on their size
// beyond int64): one 128-bit Horner chain.
__device__ __forceinline__ __int128 digits_to_sum_wide(const long long (&d)[kFeat]) {
    __int128 t = 0;
#pragma unroll
    for (int q = 15; q >= 0; q--) t = t * 16 + d[4 + q];
    return t;
}


// 32 x 32 bit transpose across a warp: lane r holds row r's 32 world bits;
// afterwards lane j holds world j's bits of the 32 rows (bit r = row r).
__device__ __forceinline__ uint32_t warp_transpose(uint32_t x, int lane) {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const uint32_t m = s == 16 ? 0x0000FFFFu : s == 8 ? 0x00FF00FFu : s == 4 ? 0x0F0F0F0Fu
                                  : s == 2 ? 0x33333333u : 0x55555555u;
        const uint32_t o = __shfl_xor_sync(kFull, x, s);
        x = (lane & s) ? ((x & ~m) | ((o >> s) & m)) : ((x & m) | ((o << s) & ~m));
    }
    return x;
}

// The features of one row in B copy `pair` (a 32-row region, rows by lane):
// the row's digits when it counts in the copy's run, else zeros.
template <int L>
__device__ __forceinline__ void pair_features(uint32_t b_pair, int lane, bool member, long long v, bool sgn) {
    using F = Features<1, L>;
    uint32_t w[F::kWords];
    F::build(v, 0, 0, 0, sgn, w);
    const uint32_t base = b_pair + (lane >> 3) * ((F::kN / 16) * 128) + (lane & 7) * 16;
#pragma unroll
    for (int h = 0; h < F::kN / 16; h++) {
        if (member) sts128_unordered(base + h * 128, w[4 * h], w[4 * h + 1], w[4 * h + 2], w[4 * h + 3]);
        else sts128_unordered(base + h * 128, 0u, 0u, 0u, 0u);
    }
}

// A group's results from its rows in the warp's lanes: lane j = world j (and
// j + 32); T, T2: the rows' world bits, transposed (bit i = lane i's row);
// Rl: the lanes whose rows count; v: this lane's row value.
__device__ __forceinline__ void group_results(const PartMmaParams &p, uint32_t g, uint32_t T, uint32_t T2,
                                              uint32_t Rl, long long v) {
    const int lane = threadIdx.x & 31;
    const uint32_t c_lo = __popc(T & Rl);
    const uint32_t c_hi = p.bal ? __popc(Rl) - c_lo : __popc(T2 & Rl);
    __int128 s_lo = 0, s_hi = 0, tot = 0;
    // at most 32 values below 2^58 in magnitude: every sum fits int64
    const bool wide = __any_sync(kFull, ((Rl >> lane) & 1u) &&
                                            (static_cast<unsigned long long>(v ^ (v >> 63)) >> 58) != 0);
    if (!wide) {
        long long a_lo = 0, a_hi = 0, at = 0;
        for (uint32_t rr = Rl; rr; rr &= rr - 1) {
            const int i = __ffs(rr) - 1;
            const long long vi = __shfl_sync(kFull, v, i);
            at += vi;
            a_lo += ((T >> i) & 1u) ? vi : 0ll;
            a_hi += ((T2 >> i) & 1u) ? vi : 0ll;
        }
        s_lo = a_lo;
        s_hi = a_hi;
        tot = at;
    } else {
        for (uint32_t rr = Rl; rr; rr &= rr - 1) {
            const int i = __ffs(rr) - 1;
            const long long vi = __shfl_sync(kFull, v, i);
            tot += vi;
            if ((T >> i) & 1u) s_lo += vi;
            if ((T2 >> i) & 1u) s_hi += vi;
        }
    }
    if (p.bal) s_hi = tot - s_lo;
    emit_world(p, g, lane, c_lo, s_lo);
    emit_world(p, g, lane + 32, c_hi, s_hi);
    if (p.meta) {
        const uint32_t o_lo = __ballot_sync(kFull, c_lo > 0), o_hi = __ballot_sync(kFull, c_hi > 0);
        if (lane == 0) {
            p.meta[2 * static_cast<size_t>(g)] = __popc(Rl);
            p.meta[2 * static_cast<size_t>(g) + 1] = o_lo | (static_cast<uint64_t>(o_hi) << 32);
        }
    }
}

// How the tensor-core kernel treats a group of its range.  MMA: more than 32
// rows (tensor cores); SMALL: at most 32 rows, left to k_part_small; SKIP: a
// SMALL group that began in the previous chunk (or range).
enum : int { kClsMma = 0, kClsSmall = 1, kClsSkip = 2 };

// Inclusive prefix maximum over lanes (up) and suffix minimum (down).
__device__ __forceinline__ int scan_max_up(int x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x = max(x, y);
    }
    return x;
}

__device__ __forceinline__ int scan_min_down(int x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_down_sync(kFull, x, o);
        if (lane + o < 32) x = min(x, y);
    }
    return x;
}

// The classes of every block's edge groups in one pass over the chunk's
// start bits (lane b < 16 = block b; bit i of word b: row 32b + i is the first
// row of a group): the group holding the block's first row and the one
// holding its last valid row (distinct when the block holds a start after
// its first row).  chunk_scans: per lane the last start before word b and
// the first start after it, and (uniform) the first row of the chunk's last
// group (-1: it began in an earlier chunk).
struct ChunkScan {
    int pmax_ex, smin_ex, ls, last_s;
};

__device__ __forceinline__ ChunkScan chunk_scans(uint32_t Sk, int lane) {
    ChunkScan c;
    c.ls = Sk ? 32 * lane + 31 - __clz(static_cast<int>(Sk)) : -1;
    const int fs = Sk ? 32 * lane + __ffs(static_cast<int>(Sk)) - 1 : INT_MAX;
    const int pmax = scan_max_up(c.ls, lane);
    const int smin = scan_min_down(fs, lane);
    c.pmax_ex = __shfl_up_sync(kFull, pmax, 1);
    if (lane == 0) c.pmax_ex = -1;
    c.smin_ex = __shfl_down_sync(kFull, smin, 1);
    if (lane == 31) c.smin_ex = INT_MAX;
    c.last_s = __shfl_sync(kFull, pmax, 31);
    return c;
}

__device__ __forceinline__ void block_classes(uint32_t Sk, int lane, int nv, const ChunkScan &c, int last_cls,
                                              int prev_cls, int &cls_f, int &cls_l) {
    const uint32_t after0 = Sk & ~1u;
    const int sF = (Sk & 1u) ? 32 * lane : c.pmax_ex;
    const int eF = after0 ? 32 * lane + __ffs(static_cast<int>(after0)) - 1 : min(c.smin_ex, nv);
    const int sL = after0 ? c.ls : sF;
    const int eL = min(c.smin_ex, nv);
    auto cls = [&](int s0, int e0) {
        if (e0 >= nv) return last_cls;
        if (s0 < 0) return prev_cls;
        return e0 - s0 <= 32 ? static_cast<int>(kClsSmall) : static_cast<int>(kClsMma);
    };
    cls_f = cls(sF, eF);
    cls_l = cls(sL, eL);
}

// One 32-row block of a chunk on its producer warp: operands and pair records
// of its MMA runs (the block's first and last run, when their groups are
// MMA-class; a group of more than 32 rows always holds one of them).
// Returns the valid pairs: bit 0 = pair 2b, bit 1 = pair 2b + 1.
__device__ __forceinline__ uint32_t produce_block(const PartMmaParams &p, const ulonglong2 *rec_s,
                                                  const GidView gid_s, int nv, int b, int cls_f, int cls_l,
                                                  uint32_t a_stage, uint32_t b_stage, PairRec *pairs) {
    const int lane = threadIdx.x & 31;
    const int ri = 32 * b + lane;  // row within the chunk
    const bool valid = ri < nv;
    const uint32_t VB = __ballot_sync(kFull, valid);
    if (VB == 0) return 0u;
    const uint32_t gid = valid ? gid_s[ri] : kNone;
    const int last = 31 - __clz(static_cast<int>(VB));
    const uint32_t g_first = __shfl_sync(kFull, gid, 0), g_lastb = __shfl_sync(kFull, gid, last);
    const bool two = g_first != g_lastb;
    const uint32_t mmaF = cls_f == kClsMma ? __ballot_sync(kFull, valid && gid == g_first) : 0u;
    const uint32_t mmaL = (two && cls_l == kClsMma) ? __ballot_sync(kFull, valid && gid == g_lastb) : 0u;
    if (!(mmaF | mmaL)) return 0u;
    const uint32_t me = 1u << lane;
    const ulonglong2 rc = rec_s[ri];
    const uint64_t mask = valid ? rec_mask(rc.x, p.packed) : 0ull;
    const long long v = (valid && p.has_col) ? static_cast<long long>(rc.y) : 0ll;
    const bool live = valid && !drop_row(p.in, mask);
    const uint32_t LB = __ballot_sync(kFull, live);
    // A: world bytes of the MMA rows
    if ((mmaF | mmaL) & me) {
        const uint32_t a_row = a_stage + (static_cast<uint32_t>(ri) >> 3) * 512 + (ri & 7) * 16;
        const uint32_t x = static_cast<uint32_t>(mask);
        sts128_unordered(a_row, world_bytes(x, 0), world_bytes(x, 1), world_bytes(x, 2), world_bytes(x, 3));
        sts128_unordered(a_row + 128, world_bytes(x, 4), world_bytes(x, 5), world_bytes(x, 6), world_bytes(x, 7));
        if (!p.bal) {
            const uint32_t y = static_cast<uint32_t>(mask >> 32);
            sts128_unordered(a_row + 256, world_bytes(y, 0), world_bytes(y, 1), world_bytes(y, 2), world_bytes(y, 3));
            sts128_unordered(a_row + 384, world_bytes(y, 4), world_bytes(y, 5), world_bytes(y, 6), world_bytes(y, 7));
        }
    }
    // B: one copy per MMA run, digits chosen per run
    uint32_t out = 0;
#pragma unroll
    for (int e = 0; e < 2; e++) {
        const uint32_t R = e == 0 ? mmaF : mmaL;
        if (!R) continue;
        const bool member = (R & me) && live;
        // 16 digits, the top one signed: every int64 value, no per-run digit count
        const uint32_t b_pair = b_stage + static_cast<uint32_t>(2 * b + e) * kPairBytes;
        pair_features<16>(b_pair, lane, member, v, true);
        static_assert(Features<1, 16>::kN == kNMax, "every B copy has N = kNMax columns");
        if (lane == 0) {
            PairRec &pr = pairs[2 * b + e];
            pr.gid = e == 0 ? g_first : g_lastb;
            pr.n = static_cast<uint16_t>(__popc(R & LB));
            pr.valid = 1;
        }
        out |= 1u << e;
    }
    return out;
}

// One tensor-memory slot's accumulator rows of this warp's lane quadrant as
// integer digit totals (units of 2^-18: exact below 2^24).
__device__ __forceinline__ void read_slot(uint32_t taddr, long long (&d)[kFeat]) {
    static_assert(kFeat == 20, "columns 0-15 and 16-19");
    uint32_t r[kFeat];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19])
                 : "r"(taddr + 16));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int f = 0; f < kFeat; f++) d[f] = __float2ll_rn(__uint_as_float(r[f]) * 262144.0f);
}

// ---------------- range planning ----------------
// k_part_mma's ranges cut the kept rows at equal shares of their cost: a row
// costs 1 and a group of more than 32 rows kGroupCost more, at its first row,
// so that a range of many mid-size groups holds fewer rows than one inside a
// heavy group.  Three launches: the cost of every tile of kTileGroups groups;
// their exclusive sums, the total and the plan (one block); the cuts.

__device__ __forceinline__ unsigned long long group_cost(uint32_t n) {
    return static_cast<unsigned long long>(n) + (n > 32 ? kGroupCost : 0u);
}

// Exclusive sum over the block of one value per thread (kPlanThreads or
// 1024 threads); *total = the block's sum.  Every thread of the block calls it.
template <int T>
__device__ __forceinline__ unsigned long long block_exclusive(unsigned long long v, unsigned long long *total) {
    __shared__ unsigned long long wsum[T / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned long long s = lane < T / 32 ? wsum[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += y;
        }
        if (lane < T / 32) wsum[lane] = s;
    }
    __syncthreads();
    const unsigned long long before = (w ? wsum[w - 1] : 0ull) + x - v;
    *total = wsum[T / 32 - 1];
    __syncthreads();  // wsum is reused by the next call
    return before;
}

// block b: the cost of groups [b kTileGroups, (b + 1) kTileGroups)
__global__ void __launch_bounds__(kPlanThreads) k_range_tiles(const __grid_constant__ PartMmaParams p) {
    const uint64_t G = p.in.n_groups;
    const uint64_t g0 = static_cast<uint64_t>(blockIdx.x) * kTileGroups, g1 = min(g0 + kTileGroups, G);
    unsigned long long c = 0;
    for (uint64_t g = g0 + threadIdx.x; g < g1; g += kPlanThreads) c += group_cost(p.pcnt[g]);
    unsigned long long tot;
    block_exclusive<kPlanThreads>(c, &tot);
    if (threadIdx.x == 0) p.tile[blockIdx.x] = tot;
}

// One block: the tiles' exclusive sums (in place), the total cost, the plan:
// R = a multiple of the SM count with shares of at most kRangeCost (fewer
// when the rows are few), share = ceil(total / R); cuts at or past the total
// are the end of the kept rows.
__global__ void __launch_bounds__(1024) k_range_plan(const __grid_constant__ PartMmaParams p, uint32_t n_tiles,
                                                     uint32_t n_sms) {
    __shared__ unsigned long long s_total, s_share;
    __shared__ uint32_t s_r;
    unsigned long long running = 0;
    for (uint32_t base = 0; base < n_tiles; base += 1024) {
        const uint32_t t = base + threadIdx.x;
        const unsigned long long v = t < n_tiles ? p.tile[t] : 0ull;
        unsigned long long tot;
        const unsigned long long before = block_exclusive<1024>(v, &tot);
        if (t < n_tiles) p.tile[t] = running + before;
        running += tot;
    }
    if (threadIdx.x == 0) {
        const unsigned long long total = running;
        const unsigned long long per_wave = static_cast<unsigned long long>(n_sms) * kRangeCost;
        unsigned long long r = static_cast<unsigned long long>(n_sms) * max(1ull, (total + per_wave - 1) / per_wave);
        r = min(r, max(1ull, (total + kMinRangeCost - 1) / kMinRangeCost));
        r = min(r, static_cast<unsigned long long>(p.r_max));
        const unsigned long long share = max(1ull, (total + r - 1) / r);
        p.plan->total = total;
        p.plan->share = share;
        p.plan->n_ranges = static_cast<uint32_t>(r);
        p.plan->next = 0;
        p.range_lo[0] = 0;
        s_total = total;
        s_share = share;
        s_r = static_cast<uint32_t>(r);
    }
    __syncthreads();
    const uint32_t kept = p.pcnt[p.in.n_groups];
    for (uint32_t j = 1 + threadIdx.x; j <= s_r; j += 1024)
        if (static_cast<unsigned long long>(j) * s_share >= s_total) p.range_lo[j] = kept;
}

// block b: the cuts that fall in tile b's groups.  Cut j (0 < j < R) sits at
// cost j share; inside group g (cost interval [c0, c1)) it is the group's
// first row while in the group's extra cost, else the row that many units
// further, rounded down to a chunk boundary.
__global__ void __launch_bounds__(kPlanThreads) k_range_cuts(const __grid_constant__ PartMmaParams p) {
    constexpr int kPer = kTileGroups / kPlanThreads;
    __shared__ uint32_t cnt_s[kTileGroups];
    const uint64_t G = p.in.n_groups;
    const uint64_t g0 = static_cast<uint64_t>(blockIdx.x) * kTileGroups;
    for (uint32_t i = threadIdx.x; i < kTileGroups; i += kPlanThreads)
        cnt_s[i] = g0 + i < G ? p.pcnt[g0 + i] : 0u;
    __syncthreads();
    unsigned long long c = 0;
#pragma unroll
    for (int k = 0; k < kPer; k++) c += group_cost(cnt_s[kPer * threadIdx.x + k]);
    unsigned long long tot;
    unsigned long long c0 = p.tile[blockIdx.x] + block_exclusive<kPlanThreads>(c, &tot);
    const unsigned long long share = p.plan->share;
    const uint32_t R = p.plan->n_ranges;
    for (int k = 0; k < kPer; k++) {
        const uint64_t g = g0 + kPer * threadIdx.x + k;
        if (g >= G) break;
        const uint32_t n = cnt_s[kPer * threadIdx.x + k];
        const unsigned long long c1 = c0 + group_cost(n);
        if (n) {
            const uint32_t extra = n > 32 ? kGroupCost : 0u;
            const uint32_t start = p.pend[g] - n;
            for (unsigned long long j = max(1ull, (c0 + share - 1) / share); j < R && j * share < c1; j++) {
                const unsigned long long o = j * share - c0;
                const uint32_t r = o < extra ? 0u : static_cast<uint32_t>(o - extra);
                p.range_lo[j] = (start + r) / kChunk * kChunk;
            }
        }
        c0 = c1;
    }
}

// Re-arms the barriers and reads range sh.range's ends and edge groups (one
// thread).  Every barrier is idle here: each wait of the previous range has
// returned, and every copy and MMA that range issued is complete (the loader
// and the issuer wait for their last completions before the range ends).
__device__ __forceinline__ void begin_range(const PartMmaParams &p, PartShared &sh, bool rearm) {
    auto arm = [&](uint64_t *bar, uint32_t count) {
        if (rearm) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
        mbar_init(bar, count);
    };
    for (int r = 0; r < kRawStages; r++) {
        arm(&sh.raw_full[r], 1);
        arm(&sh.raw_empty[r], kProdWarps + 1);  // the producers and the classifier
        arm(&sh.cls_full[r], 1);
    }
    for (int s = 0; s < kOpStages; s++) {
        arm(&sh.full[s], kProdWarps);
        arm(&sh.empty[s], 1);
    }
    for (int k = 0; k < kSlots; k++) {
        arm(&sh.done[k], 2);                // the issuer's commit and its arrive with the group's record
        arm(&sh.freeb[k], p.bal ? 3 : 4);   // the epilogue set's warps that read the slot
        arm(&sh.tot_ready[k], 1);
    }
    arm(&sh.drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
    const uint32_t rng = sh.range;
    const uint32_t G = p.in.n_groups;
    const uint32_t kept = p.pcnt[G];
    const uint32_t lo = min(p.range_lo[rng], kept);
    const uint32_t hi = max(lo, min(p.range_lo[rng + 1], kept));
    sh.lo = lo;
    sh.hi = hi;
    // groups crossing the range's edges: partial records when they are
    // tensor-core groups (more than 32 rows in all); chunk 0 sees the one
    // crossing the left edge as a group begun earlier
    const GidView pg{p.rec, p.sgid, p.packed != 0};
    const uint32_t g_lo = lo < hi ? pg[lo] : kNone;
    const bool cont_lo = lo < hi && lo > 0 && pg[lo - 1] == g_lo;
    const bool big_lo = cont_lo && p.pcnt[g_lo] > 32;
    sh.split_lo = big_lo ? g_lo : kNone;
    sh.prev_gid0 = cont_lo ? g_lo : kNone;
    sh.prev_cls0 = (cont_lo && !big_lo) ? kClsSkip : kClsMma;
    const uint32_t g_hi = lo < hi ? pg[hi - 1] : kNone;
    const bool cont_hi = lo < hi && hi < kept && pg[hi] == g_hi;
    sh.split_hi = (cont_hi && p.pcnt[g_hi] > 32) ? g_hi : kNone;
    p.part[2 * static_cast<size_t>(rng)].used = 0;
    p.part[2 * static_cast<size_t>(rng) + 1].used = 0;
}

// One range [sh.lo, sh.hi) of the group order on the whole CTA: the warp roles.
__device__ __forceinline__ void part_range(const PartMmaParams &p, PartShared &sh, unsigned char *smem,
                                           uint32_t raw_base, uint32_t op_base, uint32_t tmem, uint32_t rng) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lo = sh.lo, hi = sh.hi;
    const uint32_t n_chunks = (hi - lo + kChunk - 1) / kChunk;
    volatile int *abort_v = &sh.abort_flag;

    if (warp < kProdWarps) {
        // ---------------- producers: block warp (+ 16 bb) of every chunk ----------------
        // Per chunk: wait for its classes and the operand stage, lay out the
        // block's tensor-core runs, arrive.  No barrier among the producers.
        for (uint32_t i = 0; i < n_chunks; i++) {
            const int r = static_cast<int>(i % kRawStages), s = static_cast<int>(i % kOpStages);
            const uint32_t c0 = lo + i * kChunk;
            const int nv = static_cast<int>(min(static_cast<uint32_t>(kChunk), hi - c0));
            int ok = 1;
            if (lane == 0) {
                ok = !*abort_v && mbar_wait(&sh.cls_full[r], (i / kRawStages) & 1, p.wait_ns);
                // the bulk copy's own completion as well (already complete: one try)
                if (ok) ok = !*abort_v && mbar_wait(&sh.raw_full[r], (i / kRawStages) & 1, p.wait_ns);
                if (ok && i >= kOpStages)
                    ok = !*abort_v && mbar_wait(&sh.empty[s], ((i / kOpStages) - 1) & 1, p.wait_ns);
                if (!ok) *abort_v = 1;
            }
            ok = __shfl_sync(kFull, ok, 0);
            if (!ok) break;
            const unsigned char *raw = smem + r * kRawBytes;
            const ulonglong2 *rec_s = reinterpret_cast<const ulonglong2 *>(raw);
            const GidView gid_s{rec_s, reinterpret_cast<const uint32_t *>(raw + kRawRecBytes), p.packed != 0};
            const uint32_t a_stage = op_base + s * kOpBytes, b_stage = a_stage + kABytes;
            uint32_t pv = 0;
#pragma unroll
            for (int bb = 0; bb < kBlocksPerWarp; bb++) {
                const int b = warp + kProdWarps * bb;
                const uint32_t cc = sh.ccls[r][b];
                pv |= produce_block(p, rec_s, gid_s, nv, b, static_cast<int>(cc & 3u), static_cast<int>(cc >> 2),
                                    a_stage, b_stage, sh.pairs[s])
                      << (2 * bb);
            }
            if (lane == 0) sh.pvalid[s][warp] = static_cast<uint8_t>(pv);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&sh.full[s]);
                mbar_arrive(&sh.raw_empty[r]);
            }
        }
    } else if (warp == kClsWarp) {
        // ---------------- classifier: the chunk's groups, one chunk ahead ----------------
        // Group start bits of the chunk's rows (lane b ends with block b's
        // word), then every block's edge classes in one pass; the chunk's last
        // group is measured into the next chunk (already landed) when more
        // rows follow.  The previous chunk's last group and its class stay in
        // registers.
        uint32_t prev_gid = sh.prev_gid0;
        int prev_cls = sh.prev_cls0;
        for (uint32_t i = 0; i < n_chunks; i++) {
            const int r = static_cast<int>(i % kRawStages);
            const uint32_t rn = (i + 1) % kRawStages;
            const uint32_t c0 = lo + i * kChunk;
            const int nv = static_cast<int>(min(static_cast<uint32_t>(kChunk), hi - c0));
            const bool more = c0 + kChunk < hi;
            int ok = 1;
            if (lane == 0) {
                ok = !*abort_v && mbar_wait(&sh.raw_full[r], (i / kRawStages) & 1, p.wait_ns);
                if (ok && more) ok = !*abort_v && mbar_wait(&sh.raw_full[rn], ((i + 1) / kRawStages) & 1, p.wait_ns);
                if (!ok) *abort_v = 1;
            }
            ok = __shfl_sync(kFull, ok, 0);
            if (!ok) break;
            const GidView gid_s{reinterpret_cast<const ulonglong2 *>(smem + r * kRawBytes),
                                reinterpret_cast<const uint32_t *>(smem + r * kRawBytes + kRawRecBytes), p.packed != 0};
            const uint32_t g_last = gid_s[nv - 1];
            if (gid_s[0] == prev_gid && g_last == prev_gid) {
                // the whole chunk continues the previous chunk's group (rows are
                // in group order): every block's class is that group's
                if (lane < kBlocks) sh.ccls[r][lane] = static_cast<uint8_t>(prev_cls | (prev_cls << 2));
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&sh.cls_full[r]);
                    mbar_arrive(&sh.raw_empty[r]);
                }
                continue;
            }
            uint32_t Sk = 0;
#pragma unroll 4
            for (int b = 0; b < kBlocks; b++) {
                const int ri = 32 * b + lane;
                const bool valid = ri < nv;
                const uint32_t g = valid ? gid_s[ri] : kNone;
                const uint32_t gp = ri == 0 ? prev_gid : (valid ? gid_s[ri - 1] : kNone);
                const uint32_t w = __ballot_sync(kFull, valid && g != gp);
                if (lane == b) Sk = w;
            }
            const ChunkScan cs = chunk_scans(Sk, lane);
            int last_cls;
            if (cs.last_s < 0) {
                last_cls = prev_cls;
            } else {
                int tot = nv - cs.last_s;
                if (!more) {
                    last_cls = (g_last == sh.split_hi || tot > 32) ? kClsMma : kClsSmall;
                } else if (tot > 32) {
                    last_cls = kClsMma;
                } else {
                    const GidView gid_n{reinterpret_cast<const ulonglong2 *>(smem + rn * kRawBytes),
                                        reinterpret_cast<const uint32_t *>(smem + rn * kRawBytes + kRawRecBytes),
                                        p.packed != 0};
                    const uint32_t rows_n = min(static_cast<uint32_t>(kChunk), hi - (c0 + kChunk));
                    const uint32_t gn = static_cast<uint32_t>(lane) < rows_n ? gid_n[lane] : kNone;
                    const uint32_t eq = __ballot_sync(kFull, gn == g_last);
                    const int ext = ~eq ? __ffs(static_cast<int>(~eq)) - 1 : 32;
                    tot += ext;
                    last_cls = (tot > 32 || (g_last == sh.split_hi && c0 + kChunk + ext == hi)) ? kClsMma : kClsSmall;
                }
            }
            int cls_f, cls_l;
            block_classes(Sk, lane, nv, cs, last_cls, prev_cls, cls_f, cls_l);
            if (lane < kBlocks) sh.ccls[r][lane] = static_cast<uint8_t>(cls_f | (cls_l << 2));
            prev_gid = g_last;
            prev_cls = last_cls == kClsSmall ? kClsSkip : last_cls;
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&sh.cls_full[r]);
                mbar_arrive(&sh.raw_empty[r]);
            }
        }
    } else if (warp == kLoadWarp) {
        // ---------------- bulk-copy loader ----------------
        if (lane == 0) {
            uint32_t issued = 0;
            for (uint32_t i = 0; i < n_chunks; i++) {
                const int r = static_cast<int>(i % kRawStages);
                if (i >= kRawStages &&
                    (*abort_v || !mbar_wait(&sh.raw_empty[r], ((i / kRawStages) - 1) & 1, p.wait_ns))) {
                    *abort_v = 1;
                    break;
                }
                const uint32_t c0 = lo + i * kChunk;
                const uint32_t rows = min(static_cast<uint32_t>(kChunk), hi - c0);
                const uint32_t rows4 = (rows + 3) & ~3u;  // the group-id array has 16 bytes of slack
                mbar_expect_tx(&sh.raw_full[r], rows * 16 + (p.packed ? 0u : rows4 * 4));
                bulk_g2s(raw_base + r * kRawBytes, p.rec + c0, rows * 16, &sh.raw_full[r]);
                if (!p.packed)
                    bulk_g2s(raw_base + r * kRawBytes + kRawRecBytes, p.sgid + c0, rows4 * 4, &sh.raw_full[r]);
                issued = i + 1;
            }
            // every issued copy has landed before the range ends
            for (uint32_t i = issued > kRawStages ? issued - kRawStages : 0; i < issued; i++)
                if (!mbar_wait(&sh.raw_full[i % kRawStages], (i / kRawStages) & 1, kWaitNs)) *abort_v = 1;
        }
        __syncwarp();
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issuer ----------------
        // Completion: a commit per chunk (its operand stage), per group (its
        // slot; with an arrive that publishes the group's record) and a final
        // drain.  The chunk's pair records are read lane-parallel (lane p:
        // pair p); lane 0 alone issues, each MMA's operand descriptors
        // computed from its pair index: no shuffle or shared-memory load sits
        // between two MMAs (a tcgen05.mma from one thread costs about 100
        // cycles of issue; a dependent load or shuffle per MMA more than
        // doubled that).
        {
            int k = -1;  // ordinal of the current group
            uint32_t cur = kNone, n_acc = 0, n_mma = 0;
            uint32_t n_committed = 0;  // chunks whose stage commit is issued
            int gave_up = 0;
            auto close = [&](int kk) {
                if (lane == 0) {
                    OrdInfo &oi = sh.info[kk % kInfo];
                    oi.gid = cur;
                    oi.n = n_acc;
                    oi.end = 0;
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_u32(&sh.done[kk % kSlots])));
                    mbar_arrive(&sh.done[kk % kSlots]);
                }
            };
            // the slot of ordinal kk is free once the epilogue has read out ordinal kk - kSlots
            auto take_slot = [&](int kk) -> bool {
                if (kk < kSlots) return true;
                int ok = 1;
                if (lane == 0) {
                    ok = !*abort_v && mbar_wait(&sh.freeb[kk % kSlots], ((kk / kSlots) - 1) & 1, p.wait_ns);
                    asm volatile("tcgen05.fence::after_thread_sync;");
                }
                return __shfl_sync(kFull, ok, 0) != 0;
            };
            // pair p's A block is p / 2 (2048 bytes each) and its B copy p
            // (kPairBytes each): the descriptors' address fields (16-byte
            // units, below 2^14 for any shared-memory address) advance by
            // 128 and kPairBytes / 16 per step
            static_assert((32 * 64) / 16 == (1 << 7) && kPairBytes / 16 == (1 << 6), "descriptor steps");
            const uint32_t idesc = instr_desc<64>(kNMax);
            for (uint32_t i = 0; i < n_chunks && !gave_up; i++) {
                const int s = static_cast<int>(i % kOpStages);
                int ok = 1;
                if (lane == 0) ok = !*abort_v && mbar_wait(&sh.full[s], (i / kOpStages) & 1, p.wait_ns);
                if (!__shfl_sync(kFull, ok, 0)) {
                    gave_up = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t a_stage = op_base + s * kOpBytes, b_stage = a_stage + kABytes;
                const uint64_t da0 = smem_desc(a_stage, 512, 128);
                const uint64_t db0 = smem_desc(b_stage, (kNMax / 16) * 128, 128);
                // lane p: pair p's validity and record
                const int wq = lane >> 1, bq = wq % kProdWarps, bbq = wq / kProdWarps;
                const uint32_t nib = sh.pvalid[s][bq];
                const bool pvld = (nib >> (2 * bbq + (lane & 1))) & 1u;
                const PairRec prl = sh.pairs[s][lane];
                const uint32_t pm = __ballot_sync(kFull, pvld);
                const uint32_t gid_l = pvld ? prl.gid : kNone;
                const uint32_t n_l = pvld ? prl.n : 0u;
                // Inside a heavy group every valid pair continues the current
                // group: one vote, then the pairs' MMAs, with no group-start
                // scan or segment walk (a chunk of single-run blocks, pairs 0,
                // 2, .., 30, fully unrolled)
                const bool cont = k >= 0 && __all_sync(kFull, !pvld || gid_l == cur);
                if (cont) {
                    n_acc += __reduce_add_sync(kFull, n_l);
                    const uint32_t dacc = tmem + static_cast<uint32_t>(k % kSlots) * kAlloc;
                    if (lane == 0 && pm) {
                        uint32_t acc = n_mma != 0 ? 1u : 0u;
                        if (pm == 0x55555555u) {
#pragma unroll
                            for (uint32_t b = 0; b < kBlocks; b++) {  // pair 2b: A block b, B copy 2b
                                mma_f8_acc(dacc, da0 + (b << 7), db0 + (b << 7), idesc, acc);
                                acc = 1u;
                            }
                        } else {
                            for (uint32_t q = pm; q; q &= q - 1) {
                                const uint32_t pi = static_cast<uint32_t>(__ffs(static_cast<int>(q)) - 1);
                                mma_f8_acc(dacc, da0 + ((pi >> 1) << 7), db0 + (pi << 6), idesc, acc);
                                acc = 1u;
                            }
                        }
                    }
                    n_mma += static_cast<uint32_t>(__popc(pm));
                } else {
                    // group starts: a valid pair whose group differs from the previous valid pair's
                    int pv_idx = pvld ? lane : -1;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(kFull, pv_idx, o);
                        if (lane >= o) pv_idx = max(pv_idx, y);
                    }
                    int prev_valid = __shfl_up_sync(kFull, pv_idx, 1);
                    if (lane == 0) prev_valid = -1;
                    const uint32_t gprev = __shfl_sync(kFull, gid_l, prev_valid < 0 ? 0 : prev_valid);
                    const uint32_t ng = __ballot_sync(kFull, pvld && gid_l != (prev_valid < 0 ? cur : gprev));
                    // segments of one group, issued back to back
                    for (uint32_t rest = pm; rest;) {
                        const int p0 = __ffs(static_cast<int>(rest)) - 1;
                        if ((ng >> p0) & 1u) {
                            if (k >= 0) close(k);
                            k++;
                            if (!take_slot(k)) {
                                gave_up = 1;
                                break;
                            }
                            cur = __shfl_sync(kFull, gid_l, p0);
                            n_acc = 0;
                            n_mma = 0;
                        }
                        // the segment: valid pairs from p0 up to the next group start
                        const uint32_t after = ng & ~((2u << p0) - 1u) & ~(p0 == 31 ? 0xFFFFFFFFu : 0u);
                        const uint32_t seg = after ? (rest & ((1u << (__ffs(static_cast<int>(after)) - 1)) - 1u)) : rest;
                        rest &= ~seg;
                        n_acc += __reduce_add_sync(kFull, ((seg >> lane) & 1u) ? n_l : 0u);
                        const uint32_t dacc = tmem + static_cast<uint32_t>(k % kSlots) * kAlloc;
                        if (lane == 0) {
                            uint32_t acc = n_mma != 0 ? 1u : 0u;  // the group's first MMA overwrites its slot
                            for (uint32_t q = seg; q; q &= q - 1) {
                                const uint32_t pi = static_cast<uint32_t>(__ffs(static_cast<int>(q)) - 1);
                                mma_f8_acc(dacc, da0 + ((pi >> 1) << 7), db0 + (pi << 6), idesc, acc);
                                acc = 1u;
                            }
                        }
                        n_mma += static_cast<uint32_t>(__popc(seg));
                    }
                }
                if (gave_up) break;
                if (lane == 0)
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_u32(&sh.empty[s])));
                n_committed = i + 1;
            }
            if (gave_up) {
                if (lane == 0) *abort_v = 1;
            } else {
                if (k >= 0) close(k);
                // end markers: ordinals k + 1 .. k + kEpiSets, one for each
                // epilogue set (each slot's previous group read out first)
                for (int ke = k + 1; ke <= k + kEpiSets; ke++) {
                    if (!take_slot(ke)) {
                        if (lane == 0) *abort_v = 1;
                        break;
                    }
                    if (lane == 0) {
                        OrdInfo &oi = sh.info[ke % kInfo];
                        oi.gid = kNone;
                        oi.n = 0;
                        oi.end = 1;
                        mbar_arrive(&sh.done[ke % kSlots]);
                        mbar_arrive(&sh.done[ke % kSlots]);
                    }
                }
            }
            // every MMA issued is complete before tensor memory is read or
            // freed, and the last stage commits have arrived before the
            // barriers are re-armed for the next range
            if (lane == 0) {
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&sh.drain)));
                if (!mbar_wait(&sh.drain, 0, kWaitNs)) *abort_v = 1;
                for (uint32_t i = n_committed > kOpStages ? n_committed - kOpStages : 0; i < n_committed; i++)
                    if (!mbar_wait(&sh.empty[i % kOpStages], (i / kOpStages) & 1, kWaitNs)) *abort_v = 1;
            }
        }
        __syncwarp();
    } else if (warp >= kEpiWarp0 && warp < kLoadWarp && (warp & 3) < (p.bal ? 3 : 4)) {
        // ------- epilogue set (warp - kEpiWarp0) / 4: lane quadrant q holds accumulator rows 16q .. 16q + 15 -------
        // Each warp drains its set's groups (ordinals e, e + kEpiSets, ...) in
        // order on its own (no named barrier): wait for the group's slot, read
        // its quadrant, free it, write its worlds.  Under balanced keys
        // quadrants 0 and 1 hold worlds 0..31 and quadrant 2 the group's total
        // (row 32), which it hands to them through the slot's total buffer and
        // an mbarrier; worlds j + 32 are total - world j.  Quadrants 0 and 1
        // free the slot only after reading the total, so the buffer is not
        // written again before.  The metadata's world bits meet in shared
        // memory; the last warp writes them.
        const int q = warp & 3;
        const int eset = (warp - kEpiWarp0) >> 2;
        const int n_meta = p.bal ? 2 : 4;  // warps that hold worlds
        const uint32_t lane_base = static_cast<uint32_t>(32 * q) << 16;
        const int m = 16 * q + lane;  // accumulator row of this lane (lane < 16)
        for (int k = eset;; k += kEpiSets) {
            const int slot = k % kSlots;
            const uint32_t ph = (k / kSlots) & 1;
            int ok = 1;
            if (lane == 0) {
                ok = !*abort_v && mbar_wait(&sh.done[slot], ph, p.wait_ns);
                if (!ok) *abort_v = 1;
            }
            if (!__shfl_sync(kFull, ok, 0)) break;
            const OrdInfo oi = sh.info[k % kInfo];
            if (oi.end) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            long long d[kFeat];
            read_slot(tmem + lane_base + static_cast<uint32_t>(slot) * kAlloc, d);
            asm volatile("tcgen05.fence::before_thread_sync;");
            const bool split = (k == 0 && oi.gid == sh.split_lo) || oi.gid == sh.split_hi;
            long long tot_cnt = 0;
            __int128 tot_sum = 0;
            if (p.bal && q == 2) {
                if (lane == 0) {
#pragma unroll
                    for (int f = 0; f < kFeat; f++) sh.tot[slot][f] = d[f];
                }
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&sh.tot_ready[slot]);
                    mbar_arrive(&sh.freeb[slot]);
                }
            } else if (p.bal) {
                int tok = 1;
                if (lane == 0) {
                    tok = !*abort_v && mbar_wait(&sh.tot_ready[slot], ph, p.wait_ns);
                    if (!tok) *abort_v = 1;
                }
                if (!__shfl_sync(kFull, tok, 0)) break;
                {
                    long long td[kFeat];
#pragma unroll
                    for (int f = 0; f < kFeat; f++) td[f] = sh.tot[slot][f];
                    tot_cnt = td[0];
                    tot_sum = digits_to_sum(td);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh.freeb[slot]);
            } else {
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh.freeb[slot]);
            }
            if (split) {
                const int side = (k == 0 && oi.gid == sh.split_lo) ? 0 : 1;
                PartRec &pr = p.part[2 * static_cast<size_t>(rng) + side];
                if (lane < 16) {
#pragma unroll
                    for (int f = 0; f < kFeat; f++) pr.d[m][f] = d[f];
                }
                if (q == 0 && lane == 0) {
                    pr.gid = oi.gid;
                    pr.n = oi.n;
                    pr.used = 1;
                }
                continue;
            }
            if (p.bal && q == 2) continue;
            unsigned long long bits = 0;
            if (lane < 16) {
                const int w = world_of_row(m);
                const __int128 sw = digits_to_sum(d);
                emit_world(p, oi.gid, w, static_cast<unsigned long long>(d[0]), sw);
                bits = (d[0] > 0 ? 1ull : 0ull) << w;
                if (p.bal) {
                    const long long c2 = tot_cnt - d[0];
                    emit_world(p, oi.gid, w + 32, static_cast<unsigned long long>(c2), tot_sum - sw);
                    bits |= (c2 > 0 ? 1ull : 0ull) << (w + 32);
                }
            }
            const uint32_t o_lo = __reduce_or_sync(kFull, static_cast<uint32_t>(bits));
            const uint32_t o_hi = __reduce_or_sync(kFull, static_cast<uint32_t>(bits >> 32));
            if (lane == 0 && p.meta) {
                const int ix = k % kInfo;
                atomicOr(&sh.meta_or[ix], o_lo | (static_cast<unsigned long long>(o_hi) << 32));
                __threadfence_block();
                if (atomicAdd(&sh.meta_cnt[ix], 1u) == static_cast<uint32_t>(n_meta - 1)) {
                    __threadfence_block();
                    const unsigned long long orw = atomicOr(&sh.meta_or[ix], 0ull);
                    p.meta[2 * static_cast<size_t>(oi.gid)] = oi.n;
                    p.meta[2 * static_cast<size_t>(oi.gid) + 1] = orw;
                    sh.meta_or[ix] = 0;
                    sh.meta_cnt[ix] = 0;
                }
            }
        }
    }
}

// One CTA per SM, persistent: the CTAs take the ranges one at a time, the
// last range of the group order first (many small groups, the most output
// per row), until none is left.
__global__ void __launch_bounds__(kThreadsP, 1) k_part_mma(const __grid_constant__ PartMmaParams p) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ PartShared sh;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t smem_base = smem_u32(smem);
    const uint32_t raw_base = smem_base;
    const uint32_t op_base = smem_base + kRawStages * kRawBytes;
    if (tid == 0) sh.abort_flag = 0;
    if (warp == kEpiWarp0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem_slot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // A rows start as zeros, with the constant world byte of balanced keys:
    // accumulator row 32 (upper half, first byte) counts every row, so it
    // becomes the group's total (worlds 32..63 are total - worlds 0..31)
    for (uint32_t i = static_cast<uint32_t>(tid); i < kOpStages * kChunk; i += blockDim.x) {
        const uint32_t st = i / kChunk, r = i % kChunk;
        const uint32_t a_row = op_base + st * kOpBytes + (r >> 3) * 512 + (r & 7) * 16;
#pragma unroll
        for (int k = 0; k < 4; k++) sts128(a_row + 128 * k, (p.bal && k == 2) ? 1u : 0u, 0u, 0u, 0u);
    }
    for (int i = tid; i < kInfo; i += blockDim.x) {
        sh.meta_or[i] = 0;
        sh.meta_cnt[i] = 0;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = sh.tmem_slot;
    for (bool rearm = false;; rearm = true) {
        if (tid == 0) {
            const uint32_t n_r = p.plan->n_ranges;
            const uint32_t j = sh.abort_flag ? n_r : atomicAdd(&p.plan->next, 1u);
            sh.range = j < n_r ? n_r - 1 - j : kNone;
            if (sh.range != kNone) begin_range(p, sh, rearm);
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t rng = sh.range;
        if (rng == kNone) break;
        part_range(p, sh, smem, raw_base, op_base, tmem, rng);
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
    }
    if (tid == 0 && sh.abort_flag) raise_status(p.status, kStatusTimeout);
    if (warp == kEpiWarp0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// Groups that cross a range edge: the first record of a group (in range
// order) adds up the group's records and writes the results.  A block takes
// the records blockIdx.x, blockIdx.x + gridDim.x, ...; thread t is accumulator
// row t % 64 of slice t / 64, and the slices sum every kMergeSlices-th record
// of the group (a heavy group spans hundreds of ranges: one thread walking
// them in turn would wait out one memory latency per record).
constexpr int kMergeSlices = 4;

__global__ void __launch_bounds__(64 * kMergeSlices) k_part_merge(const __grid_constant__ PartMmaParams p) {
    __shared__ long long part_s[kMergeSlices - 1][64][kFeat];
    __shared__ unsigned long long n_s[kMergeSlices - 1];
    __shared__ long long tot[kFeat];
    __shared__ unsigned long long orw[2];
    __shared__ uint32_t end_s;
    const uint32_t n_recs = 2 * p.plan->n_ranges;
    const int m = threadIdx.x & 63, sl = threadIdx.x >> 6;
    for (uint32_t r0 = blockIdx.x; r0 < n_recs; r0 += gridDim.x) {
        const PartRec &first = p.part[r0];
        if (!first.used) continue;
        const uint32_t g = first.gid;
        bool is_first = true;
        for (uint32_t j = r0; j-- > 0;) {
            if (!p.part[j].used) continue;
            is_first = p.part[j].gid != g;
            break;
        }
        if (!is_first) continue;
        // the group's records end at the first used record of another group
        if (threadIdx.x == 0) end_s = n_recs;
        __syncthreads();
        for (uint32_t base = r0 + 1; base < n_recs; base += blockDim.x) {
            const uint32_t j = base + threadIdx.x;
            if (j < n_recs && p.part[j].used && p.part[j].gid != g) atomicMin(&end_s, j);
            __syncthreads();
            const uint32_t e = end_s;
            __syncthreads();
            if (e < base + blockDim.x) break;
        }
        const uint32_t end = end_s;
        long long d[kFeat];
#pragma unroll
        for (int f = 0; f < kFeat; f++) d[f] = 0;
        unsigned long long n = 0;
        for (uint32_t j = r0 + sl; j < end; j += kMergeSlices) {
            const PartRec &pr = p.part[j];
            if (!pr.used) continue;  // a used record before `end` is of group g
#pragma unroll
            for (int f = 0; f < kFeat; f++) d[f] += pr.d[m][f];
            n += pr.n;
        }
        if (sl > 0) {
#pragma unroll
            for (int f = 0; f < kFeat; f++) part_s[sl - 1][m][f] = d[f];
            if (m == 0) n_s[sl - 1] = n;
        }
        __syncthreads();
        if (sl == 0) {
#pragma unroll
            for (int t = 0; t < kMergeSlices - 1; t++) {
#pragma unroll
                for (int f = 0; f < kFeat; f++) d[f] += part_s[t][m][f];
                n += n_s[t];
            }
            // balanced keys: row 32 is the group total
            if (m == 32) {
#pragma unroll
                for (int f = 0; f < kFeat; f++) tot[f] = d[f];
            }
        }
        __syncthreads();
        if (sl == 0) {  // warps 0 and 1
            unsigned long long bits = 0;
            if (!p.bal || m < 32) {
                const int w = world_of_row(m);
                const __int128 sw = digits_to_sum_wide(d);
                emit_world(p, g, w, static_cast<unsigned long long>(d[0]), sw);
                bits = (d[0] > 0 ? 1ull : 0ull) << w;
                if (p.bal) {
                    long long dc[kFeat];
#pragma unroll
                    for (int f = 0; f < kFeat; f++) dc[f] = tot[f] - d[f];
                    emit_world(p, g, w + 32, static_cast<unsigned long long>(dc[0]), digits_to_sum_wide(dc));
                    bits |= (dc[0] > 0 ? 1ull : 0ull) << (w + 32);
                }
            }
            const uint32_t o_lo = __reduce_or_sync(kFull, static_cast<uint32_t>(bits));
            const uint32_t o_hi = __reduce_or_sync(kFull, static_cast<uint32_t>(bits >> 32));
            if ((m & 31) == 0) orw[m >> 5] = o_lo | (static_cast<unsigned long long>(o_hi) << 32);
        }
        __syncthreads();
        if (threadIdx.x == 0 && p.meta) {
            p.meta[2 * static_cast<size_t>(g)] = n;
            p.meta[2 * static_cast<size_t>(g) + 1] = orw[0] | orw[1];
        }
        __syncthreads();  // the shared buffers are reused for the next record
    }
}

// Groups of at most 32 rows (and groups without rows): warp w takes the 32
// groups [32w, 32w + 32).  Lane l loads group 32w + l's row count and end in
// the group order (one coalesced load each); the warp then walks its small
// groups in order, the rows [end - n, end) of the next one loaded while the
// current one is summed.  Lane j = world j (and j + 32).
__global__ void __launch_bounds__(256) k_part_small(const __grid_constant__ PartMmaParams p) {
    const int lane = threadIdx.x & 31;
    const uint64_t g0 = ((static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * 32;
    const uint32_t G = p.in.n_groups;
    if (g0 >= G) return;
    const uint64_t gl = g0 + lane;
    const bool in_g = gl < G;
    const uint32_t cnt = in_g ? p.pcnt[gl] : 0xFFFFFFFFu;
    const uint32_t end = in_g ? p.pend[gl] : 0u;
    uint32_t todo = __ballot_sync(kFull, in_g && cnt <= 32);
    auto fetch = [&](int j, ulonglong2 &rc, uint32_t &n) {
        n = __shfl_sync(kFull, cnt, j);
        const uint32_t e = __shfl_sync(kFull, end, j);
        rc = make_ulonglong2(0ull, 0ull);
        if (static_cast<uint32_t>(lane) < n) rc = p.rec[static_cast<uint64_t>(e) - n + lane];
    };
    if (!todo) return;
    int j = __ffs(static_cast<int>(todo)) - 1;
    todo &= todo - 1;
    ulonglong2 rc;
    uint32_t n;
    fetch(j, rc, n);
    for (;;) {
        ulonglong2 rc_next = make_ulonglong2(0ull, 0ull);
        uint32_t n_next = 0;
        const int j_next = todo ? __ffs(static_cast<int>(todo)) - 1 : -1;
        if (j_next >= 0) {
            todo &= todo - 1;
            fetch(j_next, rc_next, n_next);
        }
        const bool in = static_cast<uint32_t>(lane) < n;
        const uint64_t mask = rec_mask(rc.x, p.packed);
        const long long v = (in && p.has_col) ? static_cast<long long>(rc.y) : 0ll;
        const bool live = in && !drop_row(p.in, mask);
        const uint32_t T = warp_transpose(live ? static_cast<uint32_t>(mask) : 0u, lane);
        const uint32_t T2 = p.bal ? 0u : warp_transpose(live ? static_cast<uint32_t>(mask >> 32) : 0u, lane);
        group_results(p, static_cast<uint32_t>(g0) + j, T, T2, __ballot_sync(kFull, live), v);
        if (j_next < 0) break;
        j = j_next;
        rc = rc_next;
        n = n_next;
    }
}

// R at most: the kept rows' cost is at most n + kGroupCost x min(G, n / 33)
// (a group of more than 32 rows holds at least 33 of them), and the plan
// takes the fewest whole waves of SM-count ranges with shares of at most
// kRangeCost.
uint32_t part_r_max(uint64_t n, uint64_t G, int n_sms) {
    const uint64_t cmax = n + kGroupCost * std::min<uint64_t>(G, n / 33);
    const uint64_t per_wave = static_cast<uint64_t>(n_sms) * kRangeCost;
    return static_cast<uint32_t>(static_cast<uint64_t>(n_sms) * std::max<uint64_t>(1, (cmax + per_wave - 1) / per_wave));
}

uint32_t part_n_tiles(uint64_t G) { return static_cast<uint32_t>(std::max<uint64_t>(1, (G + kTileGroups - 1) / kTileGroups)); }

// The scratch: partial records [r_max][2], the plan, the cuts [r_max + 1],
// the tile sums.
struct PartScratch {
    size_t plan, cuts, tiles, bytes;
};

PartScratch part_scratch_layout(uint64_t n, uint64_t G, int n_sms) {
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    const uint64_t r_max = part_r_max(n, G, n_sms);
    PartScratch l;
    l.plan = up(static_cast<size_t>(2 * r_max) * sizeof(PartRec));
    l.cuts = up(l.plan + sizeof(RangePlan));
    l.tiles = up(l.cuts + static_cast<size_t>(r_max + 1) * sizeof(uint32_t));
    l.bytes = l.tiles + static_cast<size_t>(part_n_tiles(G)) * sizeof(unsigned long long);
    return l;
}

}  // namespace
}  // namespace pacgpu

namespace pacgpu {

bool part_mma_specs_served(const pac_agg_spec *specs, int n_specs) {
    const void *col = nullptr;
    for (int i = 0; i < n_specs; i++) {
        const pac_agg_spec &s = specs[i];
        if (s.kind == PAC_COUNT) continue;
        if (!((s.kind == PAC_SUM || s.kind == PAC_AVG) && s.vtype == PAC_I64 && s.variant == PAC_EXACT)) return false;
        if (col && col != s.values) return false;  // one value column
        col = s.values;
    }
    return true;
}

size_t part_mma_scratch_bytes(uint64_t n, uint32_t n_groups, int n_sms) {
    return part_scratch_layout(n, n_groups, n_sms).bytes;
}

pac_status part_mma_launch(const PartMmaArgs &a, cudaStream_t stream, int *launches, const char **why) {
    PartMmaParams p{};
    p.in = a.in;
    p.rec = static_cast<const ulonglong2 *>(a.rec);
    p.sgid = a.sgid;
    p.packed = a.packed;
    p.pcnt = a.pcnt;
    p.pend = a.pend;
    p.bal = !(a.in.in_flags & PAC_IN_MASKS) && a.in.hash_mode == PAC_HASH_BALANCED;
    p.has_col = 0;
    for (int i = 0; i < a.n_specs; i++) {
        p.out_kind[i] = a.specs[i].kind;
        p.out[i] = a.specs[i].out;
        if (a.specs[i].kind != PAC_COUNT) p.has_col = 1;
    }
    p.n_out = a.n_specs;
    p.meta = a.meta;
    const PartScratch l = part_scratch_layout(a.in.n, a.in.n_groups, a.n_sms);
    char *scratch = static_cast<char *>(a.scratch);
    p.part = reinterpret_cast<PartRec *>(scratch);
    p.plan = reinterpret_cast<RangePlan *>(scratch + l.plan);
    p.range_lo = reinterpret_cast<uint32_t *>(scratch + l.cuts);
    p.tile = reinterpret_cast<unsigned long long *>(scratch + l.tiles);
    p.r_max = part_r_max(a.in.n, a.in.n_groups, a.n_sms);
    p.status = a.status;
    p.wait_ns = a.wait_ns ? a.wait_ns : kWaitNs;
    const uint32_t n_tiles = part_n_tiles(a.in.n_groups);
    cudaError_t e = cudaFuncSetAttribute(k_part_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kSmemP));
    if (e == cudaSuccess) {
        k_range_tiles<<<n_tiles, kPlanThreads, 0, stream>>>(p);
        k_range_plan<<<1, 1024, 0, stream>>>(p, n_tiles, static_cast<uint32_t>(a.n_sms));
        k_range_cuts<<<n_tiles, kPlanThreads, 0, stream>>>(p);
        // one persistent CTA per SM (tensor memory and shared memory admit one)
        k_part_mma<<<static_cast<unsigned>(std::min<uint32_t>(static_cast<uint32_t>(a.n_sms), p.r_max)), kThreadsP,
                     kSmemP, stream>>>(p);
        k_part_merge<<<std::min<uint32_t>(2 * p.r_max, 4u * static_cast<uint32_t>(a.n_sms)), 64 * kMergeSlices, 0,
                       stream>>>(p);
        // one warp per 32 groups, 8 warps per block
        k_part_small<<<static_cast<unsigned>((static_cast<uint64_t>(a.in.n_groups) + 255) / 256), 256, 0,
                       stream>>>(p);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        *why = cudaGetErrorString(e);
        return PAC_E_CUDA;
    }
    *launches += 6;
    return PAC_OK;
}

}  // namespace pacgpu
