// pac_part_mma.cu -- tensor-core COUNT and exact int64 SUM/AVG over many
// groups (Sec. 4.2 "PAC Aggregation" on a high-cardinality GROUP BY).
//
// Input: the query's rows in group order, as the partition (histogram, scan,
// scatter of pac_batch.cu) writes them: one 16-byte record {world mask,
// value} and the group id of every row.  A group's rows are consecutive, so
// the per-group contraction D_g = Bits_g^T * Digits_g of the tensor-core path
// (E4M3 world bytes times E4M3 value digits, FP32 in tensor memory, exact:
// see pac_mma.cu) needs no sort.
//
// Work split: CTA c takes the group-ordered rows [c R, (c+1) R), R a multiple
// of 512 and at most 2^16 (many more CTAs than SMs, launched last range
// first, so that ranges of many small groups -- the most output per row --
// spread over the SMs).  Its rows arrive in 512-row chunks through bulk
// asynchronous copies (cp.async.bulk, one elected thread) into a ring in
// shared memory.  Each group is aggregated one of two ways:
//   - a group of at most 32 rows (inside the CTA's range) by one warp:
//     lane j holds world j's bits of the group's rows after a warp bit
//     transpose; counts by popcount, sums exact in 128 bits.  Groups wholly
//     inside a 32-row block share the block's transpose; a group that
//     crosses a block or chunk edge is gathered into one warp (the chunk's
//     last group is looked up in the next chunk, already in the ring);
//   - a larger group, or one that crosses an edge of the CTA's range, by the
//     tensor cores: one 32-row MMA per 32-row block it touches, with the
//     block's world bytes as A and a B copy that holds the group's digits
//     and zeros in the block's other rows (at most two per block: such a
//     group always holds the block's first or last row).
// The MMAs of one group accumulate into one of 16 tensor-memory slots, a ring
// over the CTA's tensor-core groups in order; the slot of a new group is
// taken once the epilogue has emptied it.  When a group's last MMA is done,
// the epilogue warps read its slot, zero it, and write the group's
// COUNT/SUM/AVG and metadata.  A group that crosses an edge of the CTA's
// range writes its digit totals as a partial record instead; k_part_merge
// adds the partials of each such group in CTA order.  No result is written
// with an atomic operation.
//
// Warps: 0-7 producers (blocks w and w + 8 of every chunk), 8-11 epilogue
// (tensor-memory lane quadrants 0-3), 12 bulk-copy loader, 13 MMA issuer.
// Every wait is bounded (%globaltimer); a wait that gives up stops its warp's
// work, the CTA drains what it has in flight and reports PAC_E_TIMEOUT.
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
constexpr int kProdWarps = 8;
constexpr int kEpiWarp0 = 8;               // warps 8..11: epilogue, quadrant = warp % 4
constexpr int kLoadWarp = 12;
constexpr int kMmaWarp = 13;
constexpr int kThreadsP = 14 * 32;
constexpr int kAlloc = 32;                 // tensor-memory columns per slot
constexpr int kSlots = 512 / kAlloc;       // accumulator slots
constexpr int kFeat = 20;                  // COUNT, three pad features, 16 digits
constexpr int kInfo = 256;                 // per-group records of the ring (see the MMA warp)
constexpr int kNMax = 32;                  // B bytes per row: N for 16 digits
// rows per CTA at most: many more CTAs than SMs, so that ranges of many small
// groups (more output per row) spread over the SMs (below 2^20: FP32 digit
// totals stay exact)
constexpr uint32_t kMaxRowsPerCtaP = 1u << 16;
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
static_assert(kInfo >= kSlots + 3 * kPairs, "the group records must outlive the ring");

// One MMA of a chunk: a run of group `gid` in block (pair index / 2).
struct PairRec {
    uint32_t gid;
    uint16_t n;      // rows of the run that count (dropped rows excluded)
    uint8_t valid;
    uint8_t nfeat;   // N of the run's B copy (16 or 32)
};

// A group of the CTA in MMA order (ordinal k at k % kInfo).
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
    uint64_t done[kSlots];   // MMA warp (commit + arrive) -> epilogue: the slot's group is complete
    uint64_t freeb[kSlots];  // epilogue (4 warps) -> MMA warp: the slot is zero and free
    uint64_t drain;
    uint32_t tmem_slot;
    int abort_flag;
    uint32_t lo, hi;         // the CTA's rows [lo, hi)
    uint32_t split_lo;       // group crossing the CTA's left edge, or kNone
    uint32_t split_hi;       // group crossing its right edge, or kNone
    int epi_go;
    int prod_go;             // producers: the chunk (and the next one, when needed) has landed
    uint32_t sbits[2][kBlocks];      // per chunk parity: group start bits of the chunk's rows
    uint32_t prev_gid[2];            // per chunk parity: the chunk's last group ...
    int prev_cls[2];                 // ... and its class as the next chunk sees it
    PairRec pairs[kOpStages][kPairs];
    OrdInfo info[kInfo];
    long long tot[kFeat];            // balanced keys: the total row of the group being emitted
    unsigned long long orw[4];       // per quadrant: worlds with a nonzero count
};

}  // namespace

struct PartRec {
    uint32_t gid, used;
    unsigned long long n;
    long long d[kWorlds][kFeat];   // digit totals per accumulator row (units of 2^-18 folded out)
};

namespace {

struct PartMmaParams {
    InputDev in;
    const ulonglong2 *rec;     // [n] group-ordered {mask, value}
    const uint32_t *sgid;      // [n] group-ordered group ids
    const uint32_t *pcnt;      // [G + 2]: rows per group, [G] = rows kept
    uint32_t rows_per_cta;
    int32_t bal;               // balanced keys: accumulator row 32 is the run total
    int32_t has_col;           // 0: COUNT only (the records carry no value)
    int32_t n_out;
    int32_t out_kind[kMaxSpecs];
    void *out[kMaxSpecs];
    uint64_t *meta;            // [G][2] {n_g, worlds with a nonzero count} or null
    PartRec *part;             // [grid][2] (zeroed)
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

__device__ __forceinline__ void producers_sync() {
    asm volatile("bar.sync 1, 256;" ::: "memory");
}

__device__ __forceinline__ void epi_sync() {
    asm volatile("bar.sync 3, 128;" ::: "memory");
}

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

// A group's SUM from its digit totals d[4 + q] (digit q, weight 16^q).
__device__ __forceinline__ __int128 digits_to_sum(const long long (&d)[kFeat]) {
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
        if (member) sts128(base + h * 128, w[4 * h], w[4 * h + 1], w[4 * h + 2], w[4 * h + 3]);
        else sts128(base + h * 128, 0u, 0u, 0u, 0u);
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
    for (uint32_t rr = Rl; rr; rr &= rr - 1) {
        const int i = __ffs(rr) - 1;
        const long long vi = __shfl_sync(kFull, v, i);
        tot += vi;
        if ((T >> i) & 1u) s_lo += vi;
        if ((T2 >> i) & 1u) s_hi += vi;
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

// How a group is aggregated.  MMA: tensor cores (more than 32 rows, or the
// group crosses an edge of the CTA's range); DIRECT: by one warp, all its
// rows at once (at most 32 rows); SKIP: a group that began in the previous
// chunk and was finished there.
enum : int { kClsMma = 0, kClsDirect = 1, kClsSkip = 2 };

// Start-bit searches over a chunk (lane k < 16 holds word k; bit i of word k:
// row 32k + i is the first row of a group in the chunk).  Warp-uniform.
__device__ __forceinline__ int prev_start(uint32_t Sk, int lane, int r) {
    const int w = r >> 5;
    const uint32_t upto = (r & 31) == 31 ? 0xFFFFFFFFu : ((2u << (r & 31)) - 1u);
    const uint32_t m = lane < w ? Sk : (lane == w ? (Sk & upto) : 0u);
    const uint32_t bl = __ballot_sync(kFull, m != 0);
    if (!bl) return -1;
    const int k = 31 - __clz(static_cast<int>(bl));
    const uint32_t mk = __shfl_sync(kFull, m, k);
    return 32 * k + 31 - __clz(static_cast<int>(mk));
}

__device__ __forceinline__ int next_start(uint32_t Sk, int lane, int r, int nv) {
    const int w = r >> 5;
    const uint32_t above = (r & 31) == 31 ? 0u : ~((2u << (r & 31)) - 1u);
    const uint32_t m = (lane > w && lane < kBlocks) ? Sk : (lane == w ? (Sk & above) : 0u);
    const uint32_t bl = __ballot_sync(kFull, m != 0);
    if (!bl) return nv;
    const int k = __ffs(bl) - 1;
    const uint32_t mk = __shfl_sync(kFull, m, k);
    return 32 * k + __ffs(mk) - 1;
}

// What every producer warp knows of the chunk after its start bits are in.
struct ChunkView {
    const ulonglong2 *rec_s;   // this chunk's records
    const ulonglong2 *rec_n;   // the next chunk's (when the last group was looked up in it)
    const uint32_t *gid_s;
    uint32_t Sk;               // this lane's start-bit word (lanes < 16)
    int nv;                    // valid rows of the chunk
    int last_s, last_tot, last_cls;  // the chunk's last group: first row (-1: began earlier), rows, class
    int prev_cls;              // class of a group that began in an earlier chunk
};

// Extent and class of the group that holds chunk row r.
__device__ __forceinline__ void group_at(const ChunkView &cv, int lane, int r, int &s, int &tot, int &cls) {
    s = prev_start(cv.Sk, lane, r);
    const int e = next_start(cv.Sk, lane, r, cv.nv);
    if (e >= cv.nv) {
        s = cv.last_s;
        tot = cv.last_tot;
        cls = cv.last_cls;
        return;
    }
    if (s < 0) {  // began in an earlier chunk, ends in this one
        tot = 0;
        cls = cv.prev_cls;
        return;
    }
    tot = e - s;
    cls = tot <= 32 ? kClsDirect : kClsMma;
}

// A DIRECT group that reaches past its first block: its rows [s, s + tot)
// of the chunk (rows from 512 on are the next chunk's first rows).
__device__ __forceinline__ void direct_group(const PartMmaParams &p, const ChunkView &cv, uint32_t g, int s,
                                             int tot) {
    const int lane = threadIdx.x & 31;
    const int r = s + lane;
    const bool in = lane < tot;
    ulonglong2 rc = make_ulonglong2(0ull, 0ull);
    if (in) rc = r < kChunk ? cv.rec_s[r] : cv.rec_n[r - kChunk];
    const uint64_t mask = rc.x;
    const long long v = (in && p.has_col) ? static_cast<long long>(rc.y) : 0ll;
    const bool live = in && !drop_row(p.in, mask);
    const uint32_t T = warp_transpose(live ? static_cast<uint32_t>(mask) : 0u, lane);
    const uint32_t T2 = p.bal ? 0u : warp_transpose(live ? static_cast<uint32_t>(mask >> 32) : 0u, lane);
    group_results(p, g, T, T2, __ballot_sync(kFull, live), v);
}

// One 32-row block of a chunk on its producer warp: operands and pair records
// of its MMA runs (the block's first and last run, when their groups are
// MMA-class), the DIRECT groups that begin in it.
__device__ __forceinline__ void produce_block(const PartMmaParams &p, const ChunkView &cv, int b, uint32_t a_stage,
                                              uint32_t b_stage, PairRec *pairs) {
    const int lane = threadIdx.x & 31;
    const int ri = 32 * b + lane;  // row within the chunk
    const bool valid = ri < cv.nv;
    const uint32_t gid = valid ? cv.gid_s[ri] : kNone;
    const ulonglong2 rc = cv.rec_s[ri];
    const uint64_t mask = valid ? rc.x : 0ull;
    const long long v = (valid && p.has_col) ? static_cast<long long>(rc.y) : 0ll;
    const bool live = valid && !drop_row(p.in, mask);
    const uint32_t VB = __ballot_sync(kFull, valid);
    PairRec &p0 = pairs[2 * b], &p1 = pairs[2 * b + 1];
    if (VB == 0) {
        if (lane == 0) {
            p0.valid = 0;
            p1.valid = 0;
        }
        return;
    }
    const int last = 31 - __clz(static_cast<int>(VB));
    const uint32_t g_first = __shfl_sync(kFull, gid, 0), g_lastb = __shfl_sync(kFull, gid, last);
    const uint32_t F = __ballot_sync(kFull, valid && gid == g_first);
    const uint32_t Lr = __ballot_sync(kFull, valid && gid == g_lastb);
    const uint32_t LB = __ballot_sync(kFull, live);
    const uint32_t me = 1u << lane;
    int sF, tF, cF, sL, tL, cL;
    group_at(cv, lane, 32 * b, sF, tF, cF);
    if (Lr == F) {
        sL = sF;
        tL = tF;
        cL = cF;
    } else {
        group_at(cv, lane, 32 * b + last, sL, tL, cL);
    }
    const int b0 = 32 * b, b1 = b0 + 32;
    const bool two = Lr != F;
    // DIRECT groups wholly inside the block share one transpose
    const bool f_inside = cF == kClsDirect && sF >= b0 && sF + tF <= b1;
    const bool l_inside = two && cL == kClsDirect && sL >= b0 && sL + tL <= b1;
    uint32_t I = VB & ~(F | Lr);
    if (f_inside) I |= F;
    if (l_inside) I |= Lr;
    // MMA runs: A world bytes of their rows, one B copy each
    const uint32_t mmaF = cF == kClsMma ? F : 0u;
    const uint32_t mmaL = (two && cL == kClsMma) ? Lr : 0u;
    if ((mmaF | mmaL) & me) {
        const uint32_t a_row = a_stage + (static_cast<uint32_t>(ri) >> 3) * 512 + (ri & 7) * 16;
        const uint32_t x = static_cast<uint32_t>(mask);
        sts128(a_row, world_bytes(x, 0), world_bytes(x, 1), world_bytes(x, 2), world_bytes(x, 3));
        sts128(a_row + 128, world_bytes(x, 4), world_bytes(x, 5), world_bytes(x, 6), world_bytes(x, 7));
        if (!p.bal) {
            const uint32_t y = static_cast<uint32_t>(mask >> 32);
            sts128(a_row + 256, world_bytes(y, 0), world_bytes(y, 1), world_bytes(y, 2), world_bytes(y, 3));
            sts128(a_row + 384, world_bytes(y, 4), world_bytes(y, 5), world_bytes(y, 6), world_bytes(y, 7));
        }
    }
#pragma unroll
    for (int e = 0; e < 2; e++) {
        const uint32_t R = e == 0 ? mmaF : mmaL;
        PairRec &pr = e == 0 ? p0 : p1;
        if (!R) {
            if (lane == 0) pr.valid = 0;
            continue;
        }
        const bool member = (R & me) && live;
        const unsigned long long mg = member ? static_cast<unsigned long long>(v ^ (v >> 63)) : 0ull;
        const uint32_t mh = __reduce_or_sync(kFull, static_cast<uint32_t>(mg >> 32));
        const uint32_t ml = __reduce_or_sync(kFull, static_cast<uint32_t>(mg));
        const bool neg = __any_sync(kFull, member && v < 0);
        const int bits = mh ? 64 - __clz(static_cast<int>(mh)) : (ml ? 32 - __clz(static_cast<int>(ml)) : 0);
        const int need = neg ? (bits + 4) / 4 : (bits + 3) / 4;
        const uint32_t b_pair = b_stage + static_cast<uint32_t>(2 * b + e) * kPairBytes;
        int nfeat;
        if (need <= 12) {
            pair_features<12>(b_pair, lane, member, v, neg);
            nfeat = Features<1, 12>::kN;
        } else {
            pair_features<16>(b_pair, lane, member, v, neg);
            nfeat = Features<1, 16>::kN;
        }
        if (lane == 0) {
            pr.gid = e == 0 ? g_first : g_lastb;
            pr.n = static_cast<uint16_t>(__popc(R & LB));
            pr.valid = 1;
            pr.nfeat = static_cast<uint8_t>(nfeat);
        }
    }
    // DIRECT groups that begin in this block and reach past it
    if (cF == kClsDirect && sF >= b0 && !f_inside) direct_group(p, cv, g_first, sF, tF);
    if (two && cL == kClsDirect && sL >= b0 && !l_inside) direct_group(p, cv, g_lastb, sL, tL);
    // DIRECT groups inside the block: lane j = world j (and j + 32)
    if (!I) return;
    const uint32_t T = warp_transpose(live ? static_cast<uint32_t>(mask) : 0u, lane);
    const uint32_t T2 = p.bal ? 0u : warp_transpose(live ? static_cast<uint32_t>(mask >> 32) : 0u, lane);
    while (I) {
        const uint32_t g = __shfl_sync(kFull, gid, __ffs(I) - 1);
        const uint32_t R = __ballot_sync(kFull, gid == g) & I;
        I &= ~R;
        group_results(p, g, T, T2, R & LB, v);
    }
}

// One tensor-memory slot's accumulator rows of this warp's lane quadrant as
// integer digit totals (units of 2^-18: exact below 2^24).
__device__ __forceinline__ void read_slot(uint32_t taddr, long long (&d)[kFeat]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
          "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
          "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int f = 0; f < kFeat; f++) d[f] = __float2ll_rn(__uint_as_float(r[f]) * 262144.0f);
}

__device__ __forceinline__ void zero_slot(uint32_t taddr) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,"
        "%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
        "r"(0u));
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(kThreadsP, 1) k_part_mma(const __grid_constant__ PartMmaParams p) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ PartShared sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // row ranges in reverse launch order: the last ranges of the group order
    // (many small groups, the most output per row) start first
    const uint32_t cta = gridDim.x - 1 - blockIdx.x;
    const uint32_t smem_base = smem_u32(smem);
    const uint32_t raw_base = smem_base;
    const uint32_t op_base = smem_base + kRawStages * kRawBytes;

    if (tid == 0) {
        for (int r = 0; r < kRawStages; r++) {
            mbar_init(&sh.raw_full[r], 1);
            mbar_init(&sh.raw_empty[r], kProdWarps);
        }
        for (int s = 0; s < kOpStages; s++) {
            mbar_init(&sh.full[s], kProdWarps);
            mbar_init(&sh.empty[s], 1);
        }
        for (int k = 0; k < kSlots; k++) {
            mbar_init(&sh.done[k], 2);
            mbar_init(&sh.freeb[k], 4);
        }
        mbar_init(&sh.drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
        sh.abort_flag = 0;
        const uint32_t G = p.in.n_groups;
        const uint64_t kept = p.pcnt[G];
        const uint64_t lo = min(static_cast<uint64_t>(cta) * p.rows_per_cta, kept);
        const uint64_t hi = min(lo + p.rows_per_cta, kept);
        sh.lo = static_cast<uint32_t>(lo);
        sh.hi = static_cast<uint32_t>(hi);
        sh.split_lo = (lo < hi && lo > 0 && p.sgid[lo - 1] == p.sgid[lo]) ? p.sgid[lo] : kNone;
        sh.split_hi = (lo < hi && hi < kept && p.sgid[hi - 1] == p.sgid[hi]) ? p.sgid[hi - 1] : kNone;
        // chunk 0 sees the group crossing the left edge as an MMA group begun earlier
        sh.prev_gid[1] = sh.split_lo;
        sh.prev_cls[1] = kClsMma;
    }
    if (warp == kEpiWarp0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem_slot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = sh.tmem_slot;
    if (warp >= kEpiWarp0 && warp < kEpiWarp0 + 4) {  // zero every slot (lane quadrant warp % 4)
        const uint32_t lane_base = static_cast<uint32_t>(32 * (warp & 3)) << 16;
        for (uint32_t c0 = 0; c0 < 512; c0 += 32) zero_slot(tmem + lane_base + c0);
    }
    // A rows start as zeros, with the constant world byte of balanced keys:
    // accumulator row 32 (upper half, first byte) counts every row, so it
    // becomes the run's total
    for (uint32_t i = static_cast<uint32_t>(tid); i < kOpStages * kChunk; i += blockDim.x) {
        const uint32_t st = i / kChunk, r = i % kChunk;
        const uint32_t a_row = op_base + st * kOpBytes + (r >> 3) * 512 + (r & 7) * 16;
#pragma unroll
        for (int k = 0; k < 4; k++) sts128(a_row + 128 * k, (p.bal && k == 2) ? 1u : 0u, 0u, 0u, 0u);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");

    const uint32_t lo = sh.lo, hi = sh.hi;
    const uint32_t n_chunks = (hi - lo + kChunk - 1) / kChunk;
    volatile int *abort_v = &sh.abort_flag;

    if (warp < kProdWarps) {
        // ---------------- producers: blocks warp and warp + 8 ----------------
        // Per chunk: one thread waits for the chunk (and the operand stage),
        // every warp writes its blocks' start bits, one thread waits for the
        // next chunk when more rows follow (the chunk's last group may end
        // there), then every warp lays out its blocks.  Both go/no-go
        // decisions are read by all producer warps after a barrier.
        for (uint32_t i = 0; i < n_chunks; i++) {
            const int r = static_cast<int>(i % kRawStages), s = static_cast<int>(i & 1), par = s;
            const uint32_t c0 = lo + i * kChunk;
            const int nv = static_cast<int>(min(static_cast<uint32_t>(kChunk), hi - c0));
            const bool more = c0 + kChunk < hi;
            if (tid == 0) {
                bool ok = !*abort_v && mbar_wait(&sh.raw_full[r], (i / kRawStages) & 1, p.wait_ns);
                if (ok && i >= kOpStages) ok = !*abort_v && mbar_wait(&sh.empty[s], ((i >> 1) - 1) & 1, p.wait_ns);
                if (!ok) *abort_v = 1;
                sh.prod_go = ok;
            }
            producers_sync();
            if (!*reinterpret_cast<volatile int *>(&sh.prod_go)) break;
            const unsigned char *raw = smem + r * kRawBytes;
            const uint32_t *gid_s = reinterpret_cast<const uint32_t *>(raw + kRawRecBytes);
#pragma unroll
            for (int bb = 0; bb < 2; bb++) {
                const int b = warp + kProdWarps * bb;
                const int ri = 32 * b + lane;
                const bool valid = ri < nv;
                const bool st = valid && (ri == 0 || gid_s[ri] != gid_s[ri - 1]);
                const uint32_t bits = __ballot_sync(kFull, st);
                if (lane == 0) sh.sbits[par][b] = bits;
            }
            if (tid == 0) {
                const uint32_t rn = (i + 1) % kRawStages;
                bool ok = !more || (!*abort_v && mbar_wait(&sh.raw_full[rn], ((i + 1) / kRawStages) & 1, p.wait_ns));
                if (!ok) *abort_v = 1;
                sh.prod_go = ok;
            }
            producers_sync();
            if (!*reinterpret_cast<volatile int *>(&sh.prod_go)) break;
            ChunkView cv;
            cv.rec_s = reinterpret_cast<const ulonglong2 *>(raw);
            const unsigned char *raw_n = smem + ((i + 1) % kRawStages) * kRawBytes;
            cv.rec_n = reinterpret_cast<const ulonglong2 *>(raw_n);
            cv.gid_s = gid_s;
            cv.nv = nv;
            const uint32_t pg = sh.prev_gid[par ^ 1];
            cv.prev_cls = sh.prev_cls[par ^ 1];
            // row 0 begins a group unless it continues the previous chunk's last one
            uint32_t Sk = lane < kBlocks ? sh.sbits[par][lane] : 0u;
            if (lane == 0 && gid_s[0] == pg) Sk &= ~1u;
            cv.Sk = Sk;
            // the chunk's last group, looked up in the next chunk when it reaches the end
            const uint32_t g_last = gid_s[nv - 1];
            cv.last_s = prev_start(Sk, lane, nv - 1);
            if (cv.last_s < 0) {
                cv.last_tot = 0;
                cv.last_cls = cv.prev_cls;
            } else {
                cv.last_tot = nv - cv.last_s;
                if (!more) {
                    cv.last_cls = (g_last == sh.split_hi || cv.last_tot > 32) ? kClsMma : kClsDirect;
                } else if (cv.last_tot > 32) {
                    cv.last_cls = kClsMma;
                } else {
                    const uint32_t *gid_n = reinterpret_cast<const uint32_t *>(raw_n + kRawRecBytes);
                    const uint32_t rows_n = min(static_cast<uint32_t>(kChunk), hi - (c0 + kChunk));
                    const uint32_t gn = static_cast<uint32_t>(lane) < rows_n ? gid_n[lane] : kNone;
                    const uint32_t eq = __ballot_sync(kFull, gn == g_last);
                    const int ext = ~eq ? __ffs(~eq) - 1 : 32;
                    cv.last_tot += ext;
                    cv.last_cls = (cv.last_tot > 32 || (g_last == sh.split_hi && c0 + kChunk + ext == hi))
                                      ? kClsMma
                                      : kClsDirect;
                }
            }
            if (tid == 0) {
                sh.prev_gid[par] = g_last;
                sh.prev_cls[par] = cv.last_cls == kClsDirect ? kClsSkip : cv.last_cls;
            }
            const uint32_t a_stage = op_base + s * kOpBytes, b_stage = a_stage + kABytes;
            produce_block(p, cv, warp, a_stage, b_stage, sh.pairs[s]);
            produce_block(p, cv, warp + kProdWarps, a_stage, b_stage, sh.pairs[s]);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&sh.full[s]);
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
                mbar_expect_tx(&sh.raw_full[r], rows * 16 + rows4 * 4);
                bulk_g2s(raw_base + r * kRawBytes, p.rec + c0, rows * 16, &sh.raw_full[r]);
                bulk_g2s(raw_base + r * kRawBytes + kRawRecBytes, p.sgid + c0, rows4 * 4, &sh.raw_full[r]);
                issued = i + 1;
            }
            // every issued copy has landed before the CTA ends
            for (uint32_t i = issued > kRawStages ? issued - kRawStages : 0; i < issued; i++)
                if (!mbar_wait(&sh.raw_full[i % kRawStages], (i / kRawStages) & 1, kWaitNs)) *abort_v = 1;
        }
        __syncwarp();
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            int k = -1;  // ordinal of the current group
            uint32_t cur = kNone, n_acc = 0;
            bool gave_up = false;
            auto close = [&](int kk) {
                OrdInfo &oi = sh.info[kk % kInfo];
                oi.gid = cur;
                oi.n = n_acc;
                oi.end = 0;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&sh.done[kk % kSlots])));
                mbar_arrive(&sh.done[kk % kSlots]);
            };
            // the slot of ordinal kk is free once the epilogue has emptied ordinal kk - kSlots
            auto take_slot = [&](int kk) -> bool {
                if (kk < kSlots) return true;
                if (*abort_v || !mbar_wait(&sh.freeb[kk % kSlots], ((kk / kSlots) - 1) & 1, p.wait_ns)) return false;
                asm volatile("tcgen05.fence::after_thread_sync;");
                return true;
            };
            for (uint32_t i = 0; i < n_chunks && !gave_up; i++) {
                const int s = static_cast<int>(i & 1);
                if (*abort_v || !mbar_wait(&sh.full[s], (i >> 1) & 1, p.wait_ns)) {
                    gave_up = true;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t a_stage = op_base + s * kOpBytes, b_stage = a_stage + kABytes;
                for (int pi = 0; pi < kPairs; pi++) {
                    const PairRec pr = sh.pairs[s][pi];
                    if (!pr.valid) continue;
                    if (pr.gid != cur) {
                        if (k >= 0) close(k);
                        k++;
                        if (!take_slot(k)) {
                            gave_up = true;
                            break;
                        }
                        cur = pr.gid;
                        n_acc = 0;
                    }
                    n_acc += pr.n;
                    const uint64_t da = smem_desc(a_stage + static_cast<uint32_t>(pi >> 1) * 2048, 512, 128);
                    const uint64_t db = smem_desc(b_stage + static_cast<uint32_t>(pi) * kPairBytes,
                                                  (static_cast<uint32_t>(pr.nfeat) / 16) * 128, 128);
                    mma_f8(tmem + static_cast<uint32_t>(k % kSlots) * kAlloc, da, db, instr_desc<64>(pr.nfeat));
                }
                if (gave_up) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&sh.empty[s])));
            }
            if (gave_up) {
                *abort_v = 1;
            } else {
                if (k >= 0) close(k);
                // end marker: ordinal k + 1 (its slot's previous group emptied first)
                const int ke = k + 1;
                if (take_slot(ke)) {
                    OrdInfo &oi = sh.info[ke % kInfo];
                    oi.gid = kNone;
                    oi.n = 0;
                    oi.end = 1;
                    mbar_arrive(&sh.done[ke % kSlots]);
                    mbar_arrive(&sh.done[ke % kSlots]);
                } else {
                    *abort_v = 1;
                }
            }
            // every MMA issued is complete before tensor memory is read or freed
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&sh.drain)));
            if (!mbar_wait(&sh.drain, 0, kWaitNs)) *abort_v = 1;
        }
        __syncwarp();
    } else if (warp >= kEpiWarp0 && warp < kEpiWarp0 + 4) {
        // ---------------- epilogue: lane quadrant q holds accumulator rows 16q .. 16q + 15 ----------------
        const int q = warp & 3;
        const uint32_t lane_base = static_cast<uint32_t>(32 * q) << 16;
        const int m = 16 * q + lane;  // accumulator row of this lane (lane < 16)
        for (int k = 0;; k++) {
            const int slot = k % kSlots;
            if (warp == kEpiWarp0 && lane == 0) {
                const bool ok = !*abort_v && mbar_wait(&sh.done[slot], (k / kSlots) & 1, p.wait_ns);
                if (!ok) *abort_v = 1;
                sh.epi_go = ok ? (sh.info[k % kInfo].end ? 2 : 1) : 0;
            }
            epi_sync();
            const int go = *reinterpret_cast<volatile int *>(&sh.epi_go);
            if (go != 1) break;
            const OrdInfo oi = sh.info[k % kInfo];
            asm volatile("tcgen05.fence::after_thread_sync;");
            long long d[kFeat];
            const uint32_t taddr = tmem + lane_base + static_cast<uint32_t>(slot) * kAlloc;
            read_slot(taddr, d);
            zero_slot(taddr);
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh.freeb[slot]);
            const bool split = (k == 0 && oi.gid == sh.split_lo) || oi.gid == sh.split_hi;
            if (p.bal && q == 2 && lane == 0) {
#pragma unroll
                for (int f = 0; f < kFeat; f++) sh.tot[f] = d[f];
            }
            epi_sync();
            unsigned long long bits = 0;
            if (split) {
                const int side = (k == 0 && oi.gid == sh.split_lo) ? 0 : 1;
                PartRec &pr = p.part[2 * static_cast<size_t>(cta) + side];
                if (lane < 16) {
#pragma unroll
                    for (int f = 0; f < kFeat; f++) pr.d[m][f] = d[f];
                }
                if (q == 0 && lane == 0) {
                    pr.gid = oi.gid;
                    pr.n = oi.n;
                    pr.used = 1;
                }
            } else if (lane < 16 && (!p.bal || q < 2)) {
                const int w = world_of_row(m);
                emit_world(p, oi.gid, w, static_cast<unsigned long long>(d[0]), digits_to_sum(d));
                bits = (d[0] > 0 ? 1ull : 0ull) << w;
                if (p.bal) {
                    long long dc[kFeat];
#pragma unroll
                    for (int f = 0; f < kFeat; f++) dc[f] = sh.tot[f] - d[f];
                    emit_world(p, oi.gid, w + 32, static_cast<unsigned long long>(dc[0]), digits_to_sum(dc));
                    bits |= (dc[0] > 0 ? 1ull : 0ull) << (w + 32);
                }
            }
            const uint32_t o_lo = __reduce_or_sync(kFull, static_cast<uint32_t>(bits));
            const uint32_t o_hi = __reduce_or_sync(kFull, static_cast<uint32_t>(bits >> 32));
            if (lane == 0) sh.orw[q] = o_lo | (static_cast<unsigned long long>(o_hi) << 32);
            epi_sync();
            if (!split && p.meta && warp == kEpiWarp0 && lane == 0) {
                p.meta[2 * static_cast<size_t>(oi.gid)] = oi.n;
                p.meta[2 * static_cast<size_t>(oi.gid) + 1] = sh.orw[0] | sh.orw[1] | sh.orw[2] | sh.orw[3];
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0 && sh.abort_flag) raise_status(p.status, kStatusTimeout);
    if (warp == kEpiWarp0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// Groups that cross a CTA edge: one CTA per partial record; the first record
// of a group (in CTA order) adds up its group's records and writes the
// results.  Thread m (of 64) = accumulator row m.
__global__ void __launch_bounds__(64) k_part_merge(const __grid_constant__ PartMmaParams p, uint32_t n_recs) {
    __shared__ long long tot[kFeat];
    __shared__ unsigned long long orw[2];
    const uint32_t r0 = blockIdx.x;
    const PartRec &first = p.part[r0];
    if (!first.used) return;
    const uint32_t g = first.gid;
    for (uint32_t j = r0; j-- > 0;) {
        if (!p.part[j].used) continue;
        if (p.part[j].gid == g) return;  // not the group's first record
        break;
    }
    const int m = threadIdx.x;
    long long d[kFeat];
#pragma unroll
    for (int f = 0; f < kFeat; f++) d[f] = 0;
    unsigned long long n = 0;
    for (uint32_t j = r0; j < n_recs; j++) {
        const PartRec &pr = p.part[j];
        if (!pr.used) continue;
        if (pr.gid != g) break;
#pragma unroll
        for (int f = 0; f < kFeat; f++) d[f] += pr.d[m][f];
        n += pr.n;
    }
    if (m == 32) {
#pragma unroll
        for (int f = 0; f < kFeat; f++) tot[f] = d[f];
    }
    __syncthreads();
    unsigned long long bits = 0;
    if (!p.bal || m < 32) {
        const int w = world_of_row(m);
        emit_world(p, g, w, static_cast<unsigned long long>(d[0]), digits_to_sum(d));
        bits = (d[0] > 0 ? 1ull : 0ull) << w;
        if (p.bal) {
            long long dc[kFeat];
#pragma unroll
            for (int f = 0; f < kFeat; f++) dc[f] = tot[f] - d[f];
            emit_world(p, g, w + 32, static_cast<unsigned long long>(dc[0]), digits_to_sum(dc));
            bits |= (dc[0] > 0 ? 1ull : 0ull) << (w + 32);
        }
    }
    const uint32_t o_lo = __reduce_or_sync(kFull, static_cast<uint32_t>(bits));
    const uint32_t o_hi = __reduce_or_sync(kFull, static_cast<uint32_t>(bits >> 32));
    if ((m & 31) == 0) orw[m >> 5] = o_lo | (static_cast<unsigned long long>(o_hi) << 32);
    __syncthreads();
    if (m == 0 && p.meta) {
        p.meta[2 * static_cast<size_t>(g)] = n;
        p.meta[2 * static_cast<size_t>(g) + 1] = orw[0] | orw[1];
    }
}

// Groups without rows: zero results and metadata.
__global__ void k_part_empty(const __grid_constant__ PartMmaParams p) {
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= p.in.n_groups || p.pcnt[g] != 0) return;
    for (int w = 0; w < kWorlds; w++) emit_world(p, g, w, 0ull, 0);
    if (p.meta) {
        p.meta[2 * static_cast<size_t>(g)] = 0;
        p.meta[2 * static_cast<size_t>(g) + 1] = 0;
    }
}

uint32_t part_rows_per_cta(uint64_t n, int n_sms) {
    uint64_t per = (n + n_sms - 1) / n_sms;
    per = (per + kChunk - 1) / kChunk * kChunk;
    if (per > kMaxRowsPerCtaP) per = kMaxRowsPerCtaP;
    if (per == 0) per = kChunk;
    return static_cast<uint32_t>(per);
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

size_t part_mma_scratch_bytes(uint64_t n, int n_sms) {
    const uint64_t per = part_rows_per_cta(n, n_sms);
    const uint64_t grid = n == 0 ? 1 : (n + per - 1) / per;
    return static_cast<size_t>(grid) * 2 * sizeof(PartRec);
}

pac_status part_mma_launch(const PartMmaArgs &a, cudaStream_t stream, int *launches, const char **why) {
    PartMmaParams p{};
    p.in = a.in;
    p.rec = static_cast<const ulonglong2 *>(a.rec);
    p.sgid = a.sgid;
    p.pcnt = a.pcnt;
    p.rows_per_cta = part_rows_per_cta(a.in.n, a.n_sms);
    p.bal = !(a.in.in_flags & PAC_IN_MASKS) && a.in.hash_mode == PAC_HASH_BALANCED;
    p.has_col = 0;
    for (int i = 0; i < a.n_specs; i++) {
        p.out_kind[i] = a.specs[i].kind;
        p.out[i] = a.specs[i].out;
        if (a.specs[i].kind != PAC_COUNT) p.has_col = 1;
    }
    p.n_out = a.n_specs;
    p.meta = a.meta;
    p.part = static_cast<PartRec *>(a.scratch);
    p.status = a.status;
    p.wait_ns = a.wait_ns ? a.wait_ns : kWaitNs;
    const uint64_t grid = a.in.n == 0 ? 1 : (a.in.n + p.rows_per_cta - 1) / p.rows_per_cta;
    const size_t part_bytes = static_cast<size_t>(grid) * 2 * sizeof(PartRec);
    cudaError_t e = cudaMemsetAsync(a.scratch, 0, part_bytes, stream);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_part_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kSmemP));
    if (e == cudaSuccess) {
        k_part_mma<<<static_cast<unsigned>(grid), kThreadsP, kSmemP, stream>>>(p);
        k_part_merge<<<static_cast<unsigned>(2 * grid), 64, 0, stream>>>(p, static_cast<uint32_t>(2 * grid));
        k_part_empty<<<(a.in.n_groups + 255) / 256, 256, 0, stream>>>(p);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        *why = cudaGetErrorString(e);
        return PAC_E_CUDA;
    }
    *launches += 3;
    return PAC_OK;
}

}  // namespace pacgpu
