// pac_mma.cu -- tensor-core (tcgen05) stochastic COUNT and exact int64
// SUM/AVG (Sec. 4.2 "PAC Aggregation").
//
// For one group g the 64 world sums of a value column are a contraction over
// rows:  S[j] = sum_i v_i * bit_j(mask_i).  Splitting every value into 4-bit
// digits, S[j] = sum_q 16^q * sum_i d_q(v_i) * bit_j(mask_i), so the per-group
// state is the small matrix product  D_g = Bits_g^T * Digits_g  (64 worlds x
// features) accumulated on the tensor cores:
//   A operand  (M = 64 worlds x K rows): bit j of row i as an E4M3 byte,
//              0x00 or 0x01 (worlds in an interleaved row order that takes
//              two operations per four bytes to lay out);
//   B operand  (N features x K rows): a constant 1 (COUNT) and the digits of
//              each value column as E4M3 bytes 0x00..0x0F;
//   D          FP32 in tensor memory.
// E4M3 bytes 0..15 encode exactly n * 2^-9 (subnormal and first binade share
// the scale), so every product is an integer times 2^-18 and the FP32
// accumulation stays exact while a column's digit total is below 2^24: a CTA
// handles at most 2^20 rows.  Digit totals are recombined with exact 128-bit
// integer arithmetic, so SUM is bit-exact and overflow is detected exactly.
//
// A value column's digits are chosen per 512-row tile: L = the number of
// digits the tile's largest magnitude needs (rounded up to 2, 4, 6, 8, 12
// or 16).  Tiles without negative values use unsigned digits; tiles with
// negatives use two's-complement digits whose top digit is signed (-8..7,
// sign-magnitude E4M3).  Features are ordered digit-major, so a tile with
// fewer digits touches a prefix of the accumulator columns.
//
// Rows of a tile are sorted by group in shared memory (each group's run is
// padded with zero rows to the 32-row MMA step) and each group's run is
// multiplied into its own accumulator.  Operands use the MN-major,
// no-swizzle canonical layout: a 128-byte core matrix is 8 rows (K) x 16
// bytes (M or N); LBO is the stride between 8-row blocks, SBO = 128 the
// stride between 16-byte column blocks.
#include <climits>

#include "pac_internal.cuh"
#include "pac_kernels.h"
#include "pac_mma.h"
#include "pac_tc.cuh"

namespace pacgpu {

namespace {

using namespace tc;

constexpr int kThreads = 512;        // producer threads: two groups of 8 warps
constexpr int kGroupThreads = 256;   // one producer group
constexpr int kMmaWarps = 4;         // warps issuing tcgen05.mma
constexpr int kMaxSlots = 16;        // accumulator slots (one group each)
// M = accumulator rows = worlds (64, or 128 for m = 128).  An M = 128
// operand row is twice as wide, so its tiles hold half the rows.
template <int M>
__host__ __device__ constexpr int rows_per_thread() { return M == 64 ? 2 : 1; }
template <int M>
__host__ __device__ constexpr int tile_rows() { return kGroupThreads * rows_per_thread<M>(); }
constexpr int kStages = 2;                        // one per producer group
constexpr int kMmaK = 32;               // rows per tcgen05.mma of 8-bit operands
constexpr int kMaxGroups = 8;
constexpr int kMaxCols = 4;
constexpr uint32_t kMaxRowsPerCta = 1u << 20;  // keeps FP32 digit totals below 2^24
constexpr uint32_t kTmemCols = 512;

// Accumulator / feature columns per group for C value columns.
__host__ __device__ constexpr int feat_alloc(int C) { return C == 1 ? 32 : 80; }

struct MmaParams {
    InputDev in;
    uint64_t qkey2;          // K2 of the second mask word (m = 128 from keys)
    const long long *col[kMaxCols];
    int32_t n_cols;
    int32_t n_alloc;
    uint32_t rows_per_cta;
    uint32_t k_cap;          // row slots per stage (multiple of 32)
    uint32_t a_bytes;        // per stage
    uint32_t b_bytes;        // per stage
    unsigned long long *acc; // [G][64][n_alloc] int64 digit totals (zeroed)
    unsigned long long *ng;  // [G] rows per group (zeroed)
    uint32_t *status;
    uint64_t wait_ns;        // limit of the pipeline waits (the final drain keeps kWaitNs)
};

template <int C4, int L>
__device__ __forceinline__ void write_features(uint32_t b_stage, uint32_t slot, long long v0, long long v1,
                                               long long v2, long long v3, bool sgn) {
    using F = Features<C4, L>;
    uint32_t w[F::kWords];
    F::build(v0, v1, v2, v3, sgn, w);
    const uint32_t lbo = (F::kN / 16) * 128;
    const uint32_t base = b_stage + (slot >> 3) * lbo + (slot & 7) * 16;
#pragma unroll
    for (int h = 0; h < F::kN / 16; h++) sts128(base + h * 128, w[4 * h], w[4 * h + 1], w[4 * h + 2], w[4 * h + 3]);
}

// Digit classes: C4 = 4 uses 4, 6, 8 or 16 digits; C4 = 1 uses 12 or 16.
template <int C4>
__device__ __forceinline__ void write_features_l(int L, uint32_t b_stage, uint32_t slot, long long v0, long long v1,
                                                 long long v2, long long v3, bool sgn) {
    if (C4 == 1) {
        if (L <= 12) write_features<C4, 12>(b_stage, slot, v0, v1, v2, v3, sgn);
        else write_features<C4, 16>(b_stage, slot, v0, v1, v2, v3, sgn);
    } else {
        if (L <= 4) write_features<C4, 4>(b_stage, slot, v0, v1, v2, v3, sgn);
        else if (L <= 6) write_features<C4, 6>(b_stage, slot, v0, v1, v2, v3, sgn);
        else if (L <= 8) write_features<C4, 8>(b_stage, slot, v0, v1, v2, v3, sgn);
        else write_features<C4, 16>(b_stage, slot, v0, v1, v2, v3, sgn);
    }
}

template <int C4>
__device__ __forceinline__ int digit_class(int need) {
    if (C4 == 1) return need <= 12 ? 12 : 16;
    if (need <= 4) return 4;
    if (need <= 6) return 6;
    if (need <= 8) return 8;
    return 16;
}

// Raw columns of one row, loaded two tiles ahead of their use.  km2: the
// second mask word of an m = 128 mask input.
struct RawRow {
    unsigned long long km, km2;
    uint32_t gid;
    long long v0, v1, v2, v3;
};

template <int GB>
__device__ __forceinline__ uint32_t gid_load(const void *gids, uint64_t row) {
    if (GB == 1) return __ldg(static_cast<const unsigned char *>(gids) + row);
    if (GB == 2) return __ldg(static_cast<const unsigned short *>(gids) + row);
    if (GB == 4) return __ldg(static_cast<const unsigned int *>(gids) + row);
    return 0;
}

// Loads row `off` of the CTA's range.  Rows past the end load the last row
// instead (always in bounds) and come back with the invalid group id; value
// columns beyond n_cols load column 0 and are zeroed.  No branches.
template <int C4, int GB, int M>
__device__ __forceinline__ void load_raw(const MmaParams &p, uint64_t cta_begin, uint32_t off, uint32_t n_rows,
                                         RawRow &r) {
    const bool ok = off < n_rows;
    const uint64_t row = cta_begin + (ok ? off : n_rows - 1);
    if (M == 128 && (p.in.in_flags & PAC_IN_MASKS)) {  // [n][2] mask words
        r.km = __ldg(static_cast<const unsigned long long *>(p.in.km) + 2 * row);
        r.km2 = __ldg(static_cast<const unsigned long long *>(p.in.km) + 2 * row + 1);
    } else {
        r.km = __ldg(static_cast<const unsigned long long *>(p.in.km) + row);
        r.km2 = 0;
    }
    const uint32_t g = gid_load<GB>(p.in.gids, row);
    // all-ones marks a row past the end: a stored all-ones id (out of range
    // too) becomes all-ones minus one, so it is still skipped and reported
    r.gid = ok ? (g == 0xFFFFFFFFu ? 0xFFFFFFFEu : g) : 0xFFFFFFFFu;
    const long long x0 = __ldg(p.col[0] + row);
    r.v0 = p.n_cols > 0 ? x0 : 0;
    if (C4 == 4) {
        const long long x1 = __ldg(p.col[1] + row);
        const long long x2 = __ldg(p.col[2] + row);
        const long long x3 = __ldg(p.col[3] + row);
        r.v1 = p.n_cols > 1 ? x1 : 0;
        r.v2 = p.n_cols > 2 ? x2 : 0;
        r.v3 = p.n_cols > 3 ? x3 : 0;
    } else {
        r.v1 = r.v2 = r.v3 = 0;
    }
}

// The rows of a thread under one dispatch on the tile's digit class.
template <int C4, int R>
__device__ __forceinline__ void write_features_rows(int L, uint32_t b_stage, const uint32_t (&sl)[R],
                                                    const RawRow (&rr)[R], bool sgn) {
#define PAC_FEATR(LL)                                                                         \
    do {                                                                                      \
        _Pragma("unroll") for (int r = 0; r < R; r++)                                         \
            write_features<C4, LL>(b_stage, sl[r], rr[r].v0, rr[r].v1, rr[r].v2, rr[r].v3, sgn); \
    } while (0)
    if (C4 == 1) {
        if (L <= 12) PAC_FEATR(12);
        else PAC_FEATR(16);
    } else {
        if (L <= 4) PAC_FEATR(4);
        else if (L <= 6) PAC_FEATR(6);
        else if (L <= 8) PAC_FEATR(8);
        else PAC_FEATR(16);
    }
#undef PAC_FEATR
}

// Named barrier among the warps of one producer group (ids 1 and 2).
__device__ __forceinline__ void producers_sync(int pg) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + pg), "n"(kGroupThreads) : "memory");
}


// Shared state of one CTA of the tensor-core aggregation.  Producer group g
// (warps 8g..8g+7) fills stage g with the tiles it = g, g+2, g+4, ...
struct MmaShared {
    uint64_t full_bar[kStages];   // producers -> MMA warps: the stage holds a tile
    uint64_t empty_bar[kStages];  // MMA warps (tcgen05.commit) -> producers: the stage is free
    uint64_t drain_bar;           // one tcgen05.commit per MMA warp at the end: every MMA done
    uint32_t tmem_slot;
    int abort_flag;
    uint32_t st_cnt[kStages][2][kGroupThreads / 32][kMaxGroups];  // per group, tile parity, warp
    uint32_t st_mag[kStages][2][kGroupThreads / 32][2];
    uint32_t meta_lo[kStages][kMaxGroups], meta_len[kStages][kMaxGroups];
    int meta_n[kStages];
    unsigned long long ng_acc[kStages][kMaxGroups];
    // accumulator slots: slot s holds group sl_group[s], is fed by MMA warp
    // sl_warp[s] and takes the group's 32-row blocks with index = sl_idx[s]
    // modulo grp_nslot[g]
    int n_slots;
    uint8_t sl_group[kMaxSlots], sl_warp[kMaxSlots], sl_idx[kMaxSlots], grp_nslot[kMaxGroups];
};

// Slot plan from the first tile's group counts: one slot per group, spare
// slots to the groups with most rows per slot, slots dealt to the MMA warps
// heaviest first.  One thread.
__device__ void plan_slots(MmaShared &sh, uint32_t G, uint32_t max_slots, const uint32_t *cnt) {
    uint32_t ns[kMaxGroups];
    for (uint32_t g = 0; g < kMaxGroups; g++) ns[g] = g < G ? 1u : 0u;
    for (uint32_t e = G; e < max_slots; e++) {
        uint32_t best = 0;
        for (uint32_t g = 1; g < G; g++)
            if (static_cast<unsigned long long>(cnt[g] + 1) * ns[best] >
                static_cast<unsigned long long>(cnt[best] + 1) * ns[g])
                best = g;
        ns[best]++;
    }
    int sl = 0;
    for (uint32_t g = 0; g < G; g++) {
        sh.grp_nslot[g] = static_cast<uint8_t>(ns[g]);
        for (uint32_t k = 0; k < ns[g]; k++, sl++) {
            sh.sl_group[sl] = static_cast<uint8_t>(g);
            sh.sl_idx[sl] = static_cast<uint8_t>(k);
        }
    }
    sh.n_slots = sl;
    uint32_t load[kMmaWarps] = {0, 0, 0, 0};
    int held[kMmaWarps] = {0, 0, 0, 0};
    bool dealt[kMaxSlots] = {};
    for (int r = 0; r < sl; r++) {
        int pick = -1;
        uint32_t wmax = 0;
        for (int t = 0; t < sl; t++) {
            const uint32_t w = (cnt[sh.sl_group[t]] + 1) / ns[sh.sl_group[t]];
            if (!dealt[t] && (pick < 0 || w > wmax)) {
                pick = t;
                wmax = w;
            }
        }
        // lightest warp that still has room (a warp keeps at most
        // kMaxSlots / kMmaWarps slots in registers)
        int lw = -1;
        for (int q = 0; q < kMmaWarps; q++)
            if (held[q] < kMaxSlots / kMmaWarps && (lw < 0 || load[q] < load[lw])) lw = q;
        dealt[pick] = true;
        sh.sl_warp[pick] = static_cast<uint8_t>(lw);
        load[lw] += wmax;
        held[lw]++;
    }
}

// One tile of the producer warps: statistics, layout, operands.  Each
// thread holds R = rows_per_thread<M>() rows; a row's M world bits are kept
// as M/32 words (word k: worlds 32k .. 32k+31).
template <int C4, int M>
__device__ __forceinline__ void produce_tile(const MmaParams &p, MmaShared &sh, uint32_t it, uint32_t max_slots,
                                             const RawRow (&rr)[rows_per_thread<M>()], uint32_t a_stage,
                                             uint32_t b_stage, bool keys_in, bool balanced_keys) {
    constexpr int R = rows_per_thread<M>();
    constexpr int kWords = M / 32;
    const int lane = threadIdx.x & 31;
    constexpr int kWarps = kGroupThreads / 32;
    const int pg = static_cast<int>(it & 1);                 // producer group = stage
    const int warp = (threadIdx.x >> 5) - pg * kWarps;       // warp within the group
    const uint32_t G = p.in.n_groups;
    const uint32_t lt = (1u << lane) - 1u;
    const int pb = (it >> 1) & 1;                            // the group's tile parity

    // (1) group, world mask, magnitude and sign statistics of the rows
    uint32_t gid[R], wd[R][kWords];
    bool valid[R];
    bool any_bad = false;
    const bool raw_hash = p.in.hash_mode == PAC_HASH_RAW;
    unsigned long long mag = 0, sgnbits = 0;
#pragma unroll
    for (int r = 0; r < R; r++) {
        const RawRow &c = rr[r];
        gid[r] = c.gid;
        const bool bad = gid[r] != 0xFFFFFFFFu && gid[r] >= G;  // out-of-range group id: skip, report
        any_bad |= bad;
        gid[r] = bad ? 0xFFFFFFFFu : gid[r];
        valid[r] = gid[r] != 0xFFFFFFFFu;
        if (M == 64) {
            const uint64_t h = mm3_fmix64(mm3_fmix64(c.km) ^ p.in.qkey);
            const uint32_t hl = static_cast<uint32_t>(h);
            const uint32_t hh = raw_hash ? static_cast<uint32_t>(h >> 32) : ~hl;  // balanced: complement
            wd[r][0] = keys_in ? hl : static_cast<uint32_t>(c.km);
            wd[r][1] = keys_in ? hh : static_cast<uint32_t>(c.km >> 32);
            if (valid[r] && drop_row(p.in, (static_cast<uint64_t>(wd[r][1]) << 32) | wd[r][0])) {
                gid[r] = 0xFFFFFFFFu;  // a row of no group: into the trash slot like a padding row
                valid[r] = false;
            }
        } else {
            uint64_t w0 = c.km, w1 = c.km2;
            if (keys_in) keyed_world_mask128(static_cast<int64_t>(c.km), p.in.qkey, p.qkey2, p.in.hash_mode, w0, w1);
            wd[r][0] = static_cast<uint32_t>(w0);
            wd[r][1] = static_cast<uint32_t>(w0 >> 32);
            wd[r][kWords > 2 ? 2 : 0] = static_cast<uint32_t>(w1);
            wd[r][kWords > 3 ? 3 : 0] = static_cast<uint32_t>(w1 >> 32);
        }
        // OR of |v| in one's complement (v, or ~v for v < 0) bounds every
        // value's bit length; the sign bits say whether any is negative
        mag |= static_cast<unsigned long long>(c.v0 ^ (c.v0 >> 63));
        sgnbits |= static_cast<unsigned long long>(c.v0);
        if (C4 == 4) {
            mag |= static_cast<unsigned long long>(c.v1 ^ (c.v1 >> 63));
            mag |= static_cast<unsigned long long>(c.v2 ^ (c.v2 >> 63));
            mag |= static_cast<unsigned long long>(c.v3 ^ (c.v3 >> 63));
            sgnbits |= static_cast<unsigned long long>(c.v1 | c.v2 | c.v3);
        }
    }
    // (2) ranks inside the warp: rows of one group get consecutive ranks,
    // row 0 of every thread first; leaders publish the warp's count per group
    if (__any_sync(kFull, any_bad) && lane == 0) raise_status(p.status, kStatusBadGroup);
    uint32_t rank[R];
    {
        uint32_t *cnt_row = sh.st_cnt[pg][pb][warp];
        if (lane < kMaxGroups) cnt_row[lane] = 0;
        __syncwarp();
#pragma unroll
        for (int r = 0; r < R; r++) {
            const uint32_t peers = __match_any_sync(kFull, gid[r]);
            const uint32_t rk = __popc(peers & lt);
            const uint32_t before = (r > 0 && valid[r]) ? cnt_row[gid[r]] : 0u;
            rank[r] = before + rk;
            if (r > 0) __syncwarp();
            if (valid[r] && rk == 0) cnt_row[gid[r]] = before + __popc(peers);
            __syncwarp();
        }
    }
    const uint32_t mag_hi = __reduce_or_sync(kFull, static_cast<uint32_t>(mag >> 32));
    const uint32_t mag_lo = __reduce_or_sync(kFull, static_cast<uint32_t>(mag));
    const uint32_t any_neg = __reduce_or_sync(kFull, static_cast<uint32_t>(sgnbits >> 63));
    if (lane == 0) {
        sh.st_mag[pg][pb][warp][0] = mag_hi | (any_neg << 31);  // bit 63 of a magnitude is never set
        sh.st_mag[pg][pb][warp][1] = mag_lo;
    }
    producers_sync(pg);
    // (3) every warp derives the tile layout: group runs, its own offsets, digits
    uint32_t cnt = 0, before = 0;
    if (lane < kMaxGroups) {
        uint32_t c[kWarps];
#pragma unroll
        for (int w = 0; w < kWarps; w++) c[w] = sh.st_cnt[pg][pb][w][lane];
#pragma unroll
        for (int w = 0; w < kWarps; w++) {
            cnt += c[w];
            before += w < warp ? c[w] : 0u;
        }
    }
    uint32_t oh = lane < kWarps ? sh.st_mag[pg][pb][lane][0] : 0u;
    uint32_t ol = lane < kWarps ? sh.st_mag[pg][pb][lane][1] : 0u;
    oh = __reduce_or_sync(kFull, oh);
    ol = __reduce_or_sync(kFull, ol);
    const uint32_t len = (cnt + kMmaK - 1) & ~static_cast<uint32_t>(kMmaK - 1);
    uint32_t incl = len;
#pragma unroll
    for (int o = 1; o < kMaxGroups; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    const uint32_t glo = incl - len;
    const bool neg = (oh >> 31) != 0;
    const uint32_t mh = oh & 0x7FFFFFFFu;
    const int bits = mh ? 64 - __clz(static_cast<int>(mh)) : (ol ? 32 - __clz(static_cast<int>(ol)) : 0);
    const int L = digit_class<C4>(neg ? (bits + 4) / 4 : (bits + 3) / 4);
    const int N = C4 == 1 ? round16(4 + L) : round16(4 + L * 4);
    const uint32_t base = glo + before;  // lane g: this warp's first slot in group g
    // invalid rows (past the end of the range) go to a trash slot past k_cap
    uint32_t slot[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
        const uint32_t sv = __shfl_sync(kFull, base, valid[r] ? static_cast<int>(gid[r]) : 0) + rank[r];
        slot[r] = valid[r] ? sv : p.k_cap;
    }
    // (4) the stage must be free: the MMAs of the group's previous tile are done.
    // After a give-up the MMA warps issue nothing more, so nothing is awaited.
    if (it >= kStages) {
        if (lane == 0 && !*reinterpret_cast<volatile int *>(&sh.abort_flag) &&
            !mbar_wait(&sh.empty_bar[pg], ((it >> 1) - 1) & 1, p.wait_ns))
            sh.abort_flag = 1;
        __syncwarp();
    }
    if (warp == 0) {
        if (lane < static_cast<int>(G)) {
            sh.meta_lo[pg][lane] = glo;
            sh.meta_len[pg][lane] = len;
            sh.ng_acc[pg][lane] += cnt;
        }
        if (lane == 0) sh.meta_n[pg] = N;
        if (it == 0) {
            uint32_t cg[kMaxGroups];
#pragma unroll
            for (int g = 0; g < kMaxGroups; g++) cg[g] = __shfl_sync(kFull, cnt, g);
            if (lane == 0) plan_slots(sh, G, max_slots, cg);
        }
    }
    // (5) operands into the stage, rows sorted by group.  An A row is M world
    // bytes in M/16 column blocks of 16 (one core matrix row each); under
    // balanced keys the upper half is the constant written at launch.
#pragma unroll
    for (int r = 0; r < R; r++) {
        const uint32_t a_row = a_stage + (slot[r] >> 3) * (M * 8) + (slot[r] & 7) * 16;
#pragma unroll
        for (int k = 0; k < kWords; k++) {
            if (k >= kWords / 2 && balanced_keys) continue;
            const uint32_t x = wd[r][k];
            sts128(a_row + 256 * k, world_bytes(x, 0), world_bytes(x, 1), world_bytes(x, 2), world_bytes(x, 3));
            sts128(a_row + 256 * k + 128, world_bytes(x, 4), world_bytes(x, 5), world_bytes(x, 6),
                   world_bytes(x, 7));
        }
    }
    write_features_rows<C4, R>(L, b_stage, slot, rr, neg);
    // zero the rows that pad each group's run to the MMA step (warp g: group g)
    if (warp < static_cast<int>(G)) {
        const uint32_t gcnt = __shfl_sync(kFull, cnt, warp), glen = __shfl_sync(kFull, len, warp);
        const uint32_t gl = __shfl_sync(kFull, glo, warp);
        if (static_cast<uint32_t>(lane) < glen - gcnt) {
            // zero features make a padding row add nothing, whatever its world
            // bytes (finite E4M3 0/1 values: the stage was cleared at launch)
            const uint32_t ps = gl + gcnt + lane;
            const uint32_t b_row = b_stage + (ps >> 3) * ((N / 16) * 128) + (ps & 7) * 16;
            for (int h = 0; h < N / 16; h++) sts128(b_row + h * 128, 0, 0, 0, 0);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane == 0) mbar_arrive(&sh.full_bar[pg]);
}

// Warp-specialised CTA: warps 0..15 produce operands (rows_per_thread<M>()
// rows per thread per tile), warps 16..19 issue the tensor-core MMAs, each
// into its own accumulator slots.  Producers agree on a tile's layout through
// a producer-only named barrier; the single operand stage is handed over with
// two mbarriers (full: 16 producer-warp arrivals; empty: one tcgen05.commit
// per MMA warp).  M = 64 or 128 accumulator rows (worlds).
template <int C4, int GB, int M>
__global__ void __launch_bounds__(kThreads + 32 * kMmaWarps, 1) k_agg_mma(const __grid_constant__ MmaParams p) {
    constexpr int R = rows_per_thread<M>();
    constexpr int kTile = tile_rows<M>();
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ MmaShared sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int kWarps = kThreads / 32;
    const uint32_t G = p.in.n_groups;

    if (tid == 0) {
        for (int s = 0; s < kStages; s++) {
            mbar_init(&sh.full_bar[s], kGroupThreads / 32);
            mbar_init(&sh.empty_bar[s], kMmaWarps);
        }
        mbar_init(&sh.drain_bar, kMmaWarps);
        asm volatile("fence.mbarrier_init.release.cluster;");
        sh.abort_flag = 0;
    }
    if (tid < kStages * kMaxGroups) (&sh.ng_acc[0][0])[tid] = 0;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem_slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = sh.tmem_slot;
    const uint32_t max_slots = min(static_cast<uint32_t>(kMaxSlots), kTmemCols / static_cast<uint32_t>(p.n_alloc));
    const uint32_t used_cols = max_slots * static_cast<uint32_t>(p.n_alloc);
    if (warp < 4) {  // zero the accumulators (warps 0-3 own TMEM lane quadrants 0-3)
        const uint32_t lane_base = static_cast<uint32_t>(32 * warp) << 16;
        for (uint32_t c0 = 0; c0 < used_cols; c0 += 16) {
            asm volatile(
                "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(
                    tmem + lane_base + c0),
                "r"(0u));
        }
        asm volatile("tcgen05.wait::st.sync.aligned;");
    }
    // Balanced keys: worlds M/2..M-1 are the complements of worlds 0..M/2-1,
    // so the upper half of A is one constant for every row -- world M/2 set,
    // the rest clear -- and accumulator row M/2 becomes the run's total (world
    // M/2 + j = total - world j, derived by the finish kernel).  Written once
    // per stage; the producers then write only the lower half.
    // The world bytes of every slot start at 0, so that the rows padding a
    // group's run (their features zeroed per tile) multiply finite values.
    {
        const bool bal = !(p.in.in_flags & PAC_IN_MASKS) && p.in.hash_mode == PAC_HASH_BALANCED;
        const uint32_t slots = p.k_cap + 8;
        for (uint32_t i = static_cast<uint32_t>(tid); i < kStages * slots; i += blockDim.x) {
            const uint32_t stage = i / slots, sl = i % slots;
            const uint32_t a_row =
                smem_u32(smem) + stage * (p.a_bytes + p.b_bytes) + (sl >> 3) * (M * 8) + (sl & 7) * 16;
#pragma unroll
            for (int k = 0; k < M / 16; k++) sts128(a_row + 128 * k, (bal && k == M / 32) ? 1u : 0u, 0u, 0u, 0u);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");

    const uint64_t begin = static_cast<uint64_t>(blockIdx.x) * p.rows_per_cta;
    const uint64_t end = min(p.in.n, begin + p.rows_per_cta);
    const uint32_t n_rows = static_cast<uint32_t>(end - begin);
    const uint32_t n_tiles = (n_rows + kTile - 1) / kTile;
    const uint32_t smem_base = smem_u32(smem);

    if (warp >= kWarps) {
        // ---------------- MMA warps ----------------
        const int mw = warp - kWarps;
        // this warp's slots (known after the first tile): up to 4 cached in registers
        int my_n = 0;
        uint32_t my_sl[kMaxSlots / kMmaWarps], my_g[kMaxSlots / kMmaWarps], my_idx[kMaxSlots / kMmaWarps],
            my_share[kMaxSlots / kMmaWarps];
        // Once a wait has given up, this warp reads no stage and issues no MMA
        // (a stage's layout may not be written yet) and commits nothing more;
        // the results are then discarded with PAC_E_TIMEOUT.
        bool gave_up = false;
        for (uint32_t it = 0; it < n_tiles; it++) {
            if (lane == 0 && !gave_up) {
                if (!mbar_wait(&sh.full_bar[it & 1], (it >> 1) & 1, p.wait_ns)) {
                    sh.abort_flag = 1;
                    gave_up = true;
                }
            }
            if (lane == 0 && !gave_up) {
                const int s = static_cast<int>(it & 1);
                const uint32_t a_stage = smem_base + s * (p.a_bytes + p.b_bytes);
                const uint32_t b_stage = a_stage + p.a_bytes;
                asm volatile("tcgen05.fence::after_thread_sync;");
                if (it == 0) {
                    // the k-th slot dealt to this warp goes to register set k
                    // (compile-time indices keep the sets in registers)
#pragma unroll
                    for (int k = 0; k < kMaxSlots / kMmaWarps; k++) my_sl[k] = my_g[k] = my_idx[k] = my_share[k] = 0;
                    int found = 0;
#pragma unroll
                    for (int sl = 0; sl < kMaxSlots; sl++) {
                        const bool mine = sl < sh.n_slots && sh.sl_warp[sl] == mw;
#pragma unroll
                        for (int k = 0; k < kMaxSlots / kMmaWarps; k++) {
                            if (mine && found == k) {
                                my_sl[k] = static_cast<uint32_t>(sl);
                                my_g[k] = sh.sl_group[sl];
                                my_idx[k] = sh.sl_idx[sl];
                                my_share[k] = sh.grp_nslot[sh.sl_group[sl]];
                            }
                        }
                        found += mine ? 1 : 0;
                    }
                    my_n = found < kMaxSlots / kMmaWarps ? found : kMaxSlots / kMmaWarps;
                }
                const int N = sh.meta_n[s];
                const uint32_t idesc = instr_desc<M>(N);
                const uint32_t lbo_b = (N / 16) * 128;
                // descriptors of slot 0; one 32-row block moves the start address
                // (in 16-byte units) by 4*(8M)/16 for A and 4*lbo_b/16 for B
                const uint64_t da0 = smem_desc(a_stage, M * 8, 128);
                const uint64_t db0 = smem_desc(b_stage, lbo_b, 128);
                const uint32_t step_b = lbo_b >> 2;
                uint32_t lo[kMaxSlots / kMmaWarps], nb[kMaxSlots / kMmaWarps];
#pragma unroll
                for (int k = 0; k < kMaxSlots / kMmaWarps; k++) {
                    if (k < my_n) {
                        lo[k] = sh.meta_lo[s][my_g[k]];
                        nb[k] = sh.meta_len[s][my_g[k]] / kMmaK;
                    }
                }
#pragma unroll
                for (int k = 0; k < kMaxSlots / kMmaWarps; k++) {
                    if (k >= my_n) continue;
                    const uint32_t d = tmem + my_sl[k] * static_cast<uint32_t>(p.n_alloc);
                    const uint32_t blk0 = (lo[k] >> 5) + my_idx[k];
                    const uint32_t blk_end = (lo[k] >> 5) + nb[k];
                    uint64_t da = da0 + blk0 * (2u * M);
                    uint64_t db = db0 + blk0 * step_b;
                    const uint64_t sa = 2ull * M * my_share[k], sb = static_cast<uint64_t>(step_b) * my_share[k];
                    for (uint32_t blk = blk0; blk < blk_end; blk += my_share[k]) {
                        mma_f8(d, da, db, idesc);
                        da += sa;
                        db += sb;
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&sh.empty_bar[s])));
            }
            __syncwarp();
        }
        // drain: a last commit of each MMA warp covers every MMA it issued; the
        // wait keeps the default limit even when the pipeline waits are short,
        // so no MMA is still in flight when TMEM is read and freed
        if (lane == 0) {
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&sh.drain_bar)));
            if (!mbar_wait(&sh.drain_bar, 0, kWaitNs)) sh.abort_flag = 1;
        }
        __syncwarp();
    } else {
        // ---------------- producer warps ----------------
        // group pg produces the tiles it = pg, pg+2, ...; two register sets of
        // raw rows, each reloaded right after its tile is produced, so a load
        // has a whole tile of work to arrive in
        const int pg = warp / (kGroupThreads / 32);
        const uint32_t gt = static_cast<uint32_t>(tid - pg * kGroupThreads);  // thread within the group
        const uint32_t a_stage = smem_base + pg * (p.a_bytes + p.b_bytes);
        const uint32_t b_stage = a_stage + p.a_bytes;
        const bool keys_in = !(p.in.in_flags & PAC_IN_MASKS);
        const bool balanced_keys = keys_in && p.in.hash_mode == PAC_HASH_BALANCED;
        // thread gt holds rows gt + r * kGroupThreads (r < R) of a tile
        RawRow ra[R], rb[R];
#pragma unroll
        for (int r = 0; r < R; r++) {
            load_raw<C4, GB, M>(p, begin, pg * kTile + gt + r * kGroupThreads, n_rows, ra[r]);
            load_raw<C4, GB, M>(p, begin, (pg + 2) * kTile + gt + r * kGroupThreads, n_rows, rb[r]);
        }
        for (uint32_t it = pg; it < n_tiles; it += 4) {
            produce_tile<C4, M>(p, sh, it, max_slots, ra, a_stage, b_stage, keys_in, balanced_keys);
#pragma unroll
            for (int r = 0; r < R; r++) load_raw<C4, GB, M>(p, begin, (it + 4) * kTile + gt + r * kGroupThreads, n_rows, ra[r]);
            if (it + 2 < n_tiles) {
                produce_tile<C4, M>(p, sh, it + 2, max_slots, rb, a_stage, b_stage, keys_in, balanced_keys);
#pragma unroll
                for (int r = 0; r < R; r++)
                    load_raw<C4, GB, M>(p, begin, (it + 6) * kTile + gt + r * kGroupThreads, n_rows, rb[r]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (sh.abort_flag) {
        if (tid == 0) raise_status(p.status, kStatusTimeout);
    } else if (warp < 4) {
        // read back: for M = 64, TMEM lane 32w + l (l < 16) holds accumulator
        // row 16w + l; for M = 128, lane 32w + l holds row 32w + l.  Row r
        // holds world world_of_row(r) (under balanced keys row M/2, the run
        // total, maps to itself).  The slots of a group add into the same totals.
        const uint32_t lane_base = static_cast<uint32_t>(32 * warp) << 16;
        const int world = world_of_row((M / 4) * warp + lane);
        for (int sl = 0; sl < sh.n_slots; sl++) {
            const uint32_t g = sh.sl_group[sl];
            for (int c0 = 0; c0 < p.n_alloc; c0 += 16) {
                uint32_t r[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15])
                    : "r"(tmem + lane_base + static_cast<uint32_t>(sl) * static_cast<uint32_t>(p.n_alloc) + c0));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                if (lane < M / 4) {
                    unsigned long long *dst = p.acc + (static_cast<size_t>(g) * M + world) * p.n_alloc + c0;
#pragma unroll
                    for (int k = 0; k < 16; k++) {
                        const int x = __float2int_rn(__uint_as_float(r[k]) * 262144.0f);  // units of 2^-18
                        if (x) atomicAdd(dst + k, static_cast<unsigned long long>(static_cast<long long>(x)));
                    }
                }
            }
        }
    }
    if (tid < static_cast<int>(G)) {
        const unsigned long long rows_g = sh.ng_acc[0][tid] + sh.ng_acc[1][tid];
        if (rows_g) atomicAdd(p.ng + tid, rows_g);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

struct FinishParams {
    const unsigned long long *acc;
    const unsigned long long *ng;
    uint32_t G;
    int32_t worlds;    // M: 64 (meta {n_g, or}) or 128 (meta {n_g, or word 0, or word 1})
    int32_t balanced;  // accumulator row M/2 holds the run totals; worlds M/2+j = total - world j
    int32_t n_cols, c4, n_alloc;
    int32_t n_out;
    int32_t out_kind[kMaxSpecs];
    int32_t out_col[kMaxSpecs];
    void *out[kMaxSpecs];
    uint64_t *meta;
    uint32_t *status;
};

// Digit totals -> COUNT / SUM / AVG per (group, world), metadata per group.
// One thread per (value column, cell), cells fastest: a column's 16 digit
// totals are read once and serve its SUM and AVG specs; the column-0 threads
// also write COUNT and the metadata.
__global__ void k_mma_finish(const __grid_constant__ FinishParams f) {
    const int W = f.worlds, half = W / 2;
    const size_t cells = static_cast<size_t>(f.G) * W;
    const int cp = f.n_cols > 0 ? f.n_cols : 1;
    const size_t t = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
    const bool live = t < cells * cp;
    const int c = live ? static_cast<int>(t / cells) : 0;
    const size_t cell = live ? t % cells : 0;
    const uint32_t g = static_cast<uint32_t>(cell / W);
    const int j = static_cast<int>(cell % W);
    // digit total k of this cell; under balanced keys world W/2 + j is the
    // group total (row W/2) minus world j, exactly (wrapping 64-bit integers)
    const bool derive = f.balanced && j >= half;
    const unsigned long long *a = f.acc + cell * f.n_alloc;
    const unsigned long long *tot_row = f.acc + (static_cast<size_t>(g) * W + half) * f.n_alloc;
    const unsigned long long *low_row = f.acc + (static_cast<size_t>(g) * W + (j & (half - 1))) * f.n_alloc;
    auto digit = [&](int k) -> long long {
        return static_cast<long long>(derive ? tot_row[k] - low_row[k] : a[k]);
    };
    const unsigned long long cnt = live ? static_cast<unsigned long long>(digit(0)) : 0ull;
    // a warp holds 32 consecutive cells of one column (cells is a multiple of 64)
    const unsigned bal = __ballot_sync(kFull, live && cnt > 0);
    if (!live) return;
    if (c == 0) {
        if (f.meta) {
            // meta per group: {n_g, OR word 0[, OR word 1]}; a warp's 32 cells
            // are one 32-bit half of an OR word
            const size_t stride = W == 64 ? 2 : 3;
            if ((threadIdx.x & 31) == 0)
                reinterpret_cast<uint32_t *>(f.meta + stride * g + 1 + (j >> 6))[(j >> 5) & 1] = bal;
            if (j == 0) f.meta[stride * g] = f.ng[g];
        }
        for (int s = 0; s < f.n_out; s++)
            if (f.out_kind[s] == PAC_COUNT) static_cast<unsigned long long *>(f.out[s])[cell] = cnt;
    }
    if (f.n_cols == 0) return;
    long long dq[16];
#pragma unroll
    for (int q = 0; q < 16; q++) {
        const int feat = f.c4 == 1 ? 4 + q : 4 + q * f.c4 + c;
        dq[q] = feat < f.n_alloc ? digit(feat) : 0;
    }
    __int128 tot = 0;
#pragma unroll
    for (int q = 15; q >= 0; q--) tot = tot * 16 + dq[q];
    const bool fits = tot >= static_cast<__int128>(LLONG_MIN) && tot <= static_cast<__int128>(LLONG_MAX);
    const long long val = fits ? static_cast<long long>(tot) : (tot < 0 ? LLONG_MIN : LLONG_MAX);
    bool used = false;
    for (int s = 0; s < f.n_out; s++) {
        if (f.out_kind[s] == PAC_COUNT || f.out_col[s] != c) continue;
        used = true;
        if (f.out_kind[s] == PAC_SUM) static_cast<long long *>(f.out[s])[cell] = val;
        else static_cast<double *>(f.out[s])[cell] = cnt ? i128_to_double(tot) / static_cast<double>(cnt) : 0.0;
    }
    if (used && !fits) raise_status(f.status, kStatusOverflow);
}

int mma_c4(int C) { return C == 1 ? 1 : 4; }

// Distinct value columns of the specs (or -1 when a spec is not served).
int mma_columns(const pac_agg_spec *specs, int n_specs, const void **cols) {
    int C = 0;
    for (int i = 0; i < n_specs; i++) {
        const pac_agg_spec &s = specs[i];
        if (s.kind == PAC_COUNT) continue;
        if (!((s.kind == PAC_SUM || s.kind == PAC_AVG) && s.vtype == PAC_I64 && s.variant == PAC_EXACT)) return -1;
        int k = 0;
        while (k < C && cols[k] != s.values) k++;
        if (k == C) {
            if (C == kMaxCols) return -1;
            cols[C++] = s.values;
        }
    }
    return C;
}

}  // namespace

static_assert(world_of_row(kWorlds / 2) == kWorlds / 2 && world_of_row(1) == 8 && world_of_row(4) == 1 &&
                  world_of_row(127) == 127,
              "accumulator rows must map onto the worlds as the operand words lay them out");
static_assert(kMmaMaxScratchBytes == static_cast<size_t>(kTmemCols) * kWorlds * 8 + 256 + kMaxGroups * 8,
              "kMmaMaxScratchBytes must follow the tensor-memory and group limits");

bool mma_specs_served(uint32_t n_groups, const pac_agg_spec *specs, int n_specs) {
    const void *cols[kMaxCols];
    const int C = mma_columns(specs, n_specs, cols);
    if (C < 0) return false;
    if (n_groups > static_cast<uint32_t>(kMaxGroups)) return false;
    const int n_alloc = feat_alloc(C == 0 ? 1 : C);
    return n_groups * static_cast<uint32_t>(n_alloc) <= kTmemCols;
}

bool mma_supported(const pac_input *in, const pac_agg_spec *specs, int n_specs) {
    return in->n > 0 && mma_specs_served(in->n_groups, specs, n_specs);
}

// Builds the launch of the tensor-core path.  scratch: the accumulators
// (mma_scratch_bytes bytes, cleared here); status: the device status word.
static pac_status mma_plan(const pac_input *in, const pac_agg_spec *specs, int n_specs, int n_sms, int worlds,
                           MmaParams &p, size_t &smem, int &c4, const void **cols, int &C, const char **why) {
    p = MmaParams{};
    C = mma_columns(specs, n_specs, cols);
    if (C < 0) {
        *why = "tensor-core path: unsupported spec";
        return PAC_E_UNSUPPORTED;
    }
    const int Ceff = C == 0 ? 1 : C;  // COUNT only: one zero column
    c4 = mma_c4(Ceff);
    p.in.km = in->keys_or_masks;
    p.in.gids = in->group_ids;
    p.in.qkey = in->query_key;
    p.in.n = in->n;
    p.in.in_flags = in->in_flags;
    p.in.hash_mode = in->hash_mode;
    p.in.gid_bytes = in->group_ids ? in->gid_bytes : 0;
    p.in.n_groups = in->n_groups;
    for (int c = 0; c < C; c++) p.col[c] = static_cast<const long long *>(cols[c]);
    // The producers load every column slot without a branch: unused slots
    // point at a live n-row 8-byte column (column 0, or the key/mask column
    // of a COUNT-only query) and their values are zeroed after the load.
    for (int c = C; c < kMaxCols; c++)
        p.col[c] = C > 0 ? p.col[0] : static_cast<const long long *>(in->keys_or_masks);
    p.n_cols = C;
    p.n_alloc = feat_alloc(Ceff);
    const uint32_t G = in->n_groups;
    const uint32_t tile = worlds == 64 ? tile_rows<64>() : tile_rows<128>();
    uint64_t per = (in->n + n_sms - 1) / n_sms;
    per = (per + tile - 1) / tile * tile;
    if (per > kMaxRowsPerCta) per = kMaxRowsPerCta;
    if (per == 0) per = tile;
    p.rows_per_cta = static_cast<uint32_t>(per);
    p.k_cap = (tile + (kMmaK - 1) * G + kMmaK - 1) / kMmaK * kMmaK;
    // one more 8-row block past k_cap takes the writes of invalid rows
    p.a_bytes = (p.k_cap + 8) * static_cast<uint32_t>(worlds);
    p.b_bytes = (p.k_cap + 8) * p.n_alloc;
    smem = static_cast<size_t>(kStages) * (p.a_bytes + p.b_bytes);
    if (smem > 220 * 1024) {
        *why = "tensor-core path: tile does not fit shared memory";
        return PAC_E_UNSUPPORTED;
    }
    // one CTA per SM: the CTA owns all 512 tensor-memory columns
    if (smem < 120 * 1024) smem = 120 * 1024;
    return PAC_OK;
}

size_t mma_scratch_bytes(const pac_input *in, const pac_agg_spec *specs, int n_specs, int worlds) {
    const void *cols[kMaxCols];
    const int C = mma_columns(specs, n_specs, cols);
    const int Ceff = C <= 0 ? 1 : C;
    return static_cast<size_t>(in->n_groups) * worlds * feat_alloc(Ceff) * 8 + 256 + in->n_groups * 8;
}

pac_status mma_launch(const pac_input *in, const pac_agg_spec *specs, int n_specs, uint64_t *meta,
                      cudaStream_t stream, void *scratch, uint32_t *status, int n_sms, int *launches,
                      const char **why, uint64_t wait_ns, int worlds, uint64_t qkey2) {
    MmaParams p;
    size_t smem;
    int c4, C;
    const void *cols[kMaxCols];
    if (worlds != 64 && worlds != 128) {
        *why = "tensor-core path: 64 or 128 worlds";
        return PAC_E_INVALID;
    }
    pac_status st = mma_plan(in, specs, n_specs, n_sms, worlds, p, smem, c4, cols, C, why);
    if (st != PAC_OK) return st;
    p.qkey2 = qkey2;
    const uint32_t G = in->n_groups;
    const uint64_t n_ctas = (in->n + p.rows_per_cta - 1) / p.rows_per_cta;
    const size_t acc_bytes = static_cast<size_t>(G) * worlds * p.n_alloc * 8;
    p.acc = static_cast<unsigned long long *>(scratch);
    p.ng = reinterpret_cast<unsigned long long *>(static_cast<char *>(scratch) + ((acc_bytes + 255) / 256) * 256);
    p.status = status;
    p.wait_ns = wait_ns ? wait_ns : kWaitNs;
    cudaError_t e = cudaMemsetAsync(scratch, 0, ((acc_bytes + 255) / 256) * 256 + G * 8, stream);
    if (e != cudaSuccess) {
        *why = cudaGetErrorString(e);
        return PAC_E_CUDA;
    }
    const int gb = in->group_ids ? in->gid_bytes : 0;
#define PAC_MMA_LAUNCH1(C4_, GB_, M_)                                                                           \
    do {                                                                                                        \
        e = cudaFuncSetAttribute(k_agg_mma<C4_, GB_, M_>, cudaFuncAttributeMaxDynamicSharedMemorySize,         \
                                 static_cast<int>(smem));                                                      \
        if (e == cudaSuccess)                                                                                   \
            k_agg_mma<C4_, GB_, M_><<<static_cast<unsigned>(n_ctas), kThreads + 32 * kMmaWarps, smem, stream>>>(p); \
    } while (0)
#define PAC_MMA_LAUNCH(C4_, GB_)                              \
    do {                                                      \
        if (worlds == 64) PAC_MMA_LAUNCH1(C4_, GB_, 64);      \
        else PAC_MMA_LAUNCH1(C4_, GB_, 128);                  \
    } while (0)
    if (c4 == 1) {
        switch (gb) {
        case 1: PAC_MMA_LAUNCH(1, 1); break;
        case 2: PAC_MMA_LAUNCH(1, 2); break;
        case 4: PAC_MMA_LAUNCH(1, 4); break;
        default: PAC_MMA_LAUNCH(1, 0); break;
        }
    } else {
        switch (gb) {
        case 1: PAC_MMA_LAUNCH(4, 1); break;
        case 2: PAC_MMA_LAUNCH(4, 2); break;
        case 4: PAC_MMA_LAUNCH(4, 4); break;
        default: PAC_MMA_LAUNCH(4, 0); break;
        }
    }
#undef PAC_MMA_LAUNCH
#undef PAC_MMA_LAUNCH1
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        *why = cudaGetErrorString(e);
        return PAC_E_CUDA;
    }
    FinishParams f{};
    f.acc = p.acc;
    f.ng = p.ng;
    f.G = G;
    f.worlds = worlds;
    f.balanced = !(in->in_flags & PAC_IN_MASKS) && in->hash_mode == PAC_HASH_BALANCED;
    f.n_cols = C;
    f.c4 = c4;
    f.n_alloc = p.n_alloc;
    f.meta = meta;
    f.status = status;
    for (int i = 0; i < n_specs; i++) {
        f.out_kind[f.n_out] = specs[i].kind;
        int c = 0;
        while (c < C && cols[c] != specs[i].values) c++;
        f.out_col[f.n_out] = c;
        f.out[f.n_out] = specs[i].out;
        f.n_out++;
    }
    const size_t threads = static_cast<size_t>(G) * worlds * (C > 0 ? C : 1);
    k_mma_finish<<<static_cast<unsigned>((threads + 255) / 256), 256, 0, stream>>>(f);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        *why = cudaGetErrorString(e);
        return PAC_E_CUDA;
    }
    *launches += 2;  // aggregation + finish kernels (the clearing memset is not a kernel)
    return PAC_OK;
}

pac_status run_mma(pac_ctx *ctx, const pac_input *in, const pac_agg_spec *specs, int n_specs, uint64_t *meta,
                   cudaStream_t stream, int *launches) {
    pac_status st = ensure_buffer(ctx, &ctx->ws, &ctx->ws_bytes, mma_scratch_bytes(in, specs, n_specs) + 1024);
    if (st != PAC_OK) return st;
    const char *why = "";
    st = mma_launch(in, specs, n_specs, meta, stream, ctx->ws, ctx->d_status, ctx->n_sms, launches, &why,
                    static_cast<uint64_t>(ctx->opt_wait_ns));
    if (st != PAC_OK) return fail(ctx, st, "%s", why);
    return PAC_OK;
}

}  // namespace pacgpu
