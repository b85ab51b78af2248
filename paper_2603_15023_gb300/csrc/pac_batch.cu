// pac_batch.cu -- many independent PAC queries in one persistent launch
// (Sec. 4.2 "PAC Aggregation" per query; the release of Sec. 2 / Sec. 4.1
// per query through the batched finalize kernel).
//
// A plan cuts every query into work items of consecutive rows and uploads
// one descriptor per query and one record per item.  A launch is:
//   memset of the plan's zeroed scratch (atomic states, item counter);
//   k_batch_agg   persistent CTAs (occupancy x SMs) take items from a global
//                 counter.  A query whose per-world states fit shared memory
//                 keeps them warp-private (lane l owns worlds l and l+32, the
//                 rows of one group inside a 32-row batch are folded in
//                 registers first) and writes one partial state per item; a
//                 query with many groups folds the same way and adds the
//                 folded values into its global state with atomics;
//   k_batch_merge one thread per (query, group, world) cell: item partials
//                 merged in item order (deterministic float results) or the
//                 atomic state decoded, typed outputs and meta written;
//   k_finalize_batch (optional) one warp per releasing query.
// Atomic MIN/MAX states use an order-preserving unsigned encoding whose
// identity is 0, so one memset initialises every atomic state.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "pac_ctx.h"
#include "pac_kernels.h"
#include "pac_ops.cuh"
#include "pac_validate.h"
#include "pac_batch.h"

namespace pacgpu {

namespace {

constexpr unsigned kFull = 0xffffffffu;
using namespace ops;

// Order-preserving map of a MIN/MAX state value to an unsigned key whose
// identity (the value no row can beat) is 0.
__device__ __forceinline__ unsigned long long minmax_key(int op, uint64_t bits) {
    const unsigned long long sign = 1ull << 63;
    long long ord = static_cast<long long>(bits);
    if (op == OP_FMIN || op == OP_FMAX) ord = ord >= 0 ? ord : (ord ^ 0x7fffffffffffffffll);
    const unsigned long long u = static_cast<unsigned long long>(ord) ^ sign;
    return (op == OP_IMIN || op == OP_FMIN) ? ~u : u;
}

__device__ __forceinline__ uint64_t minmax_value(int op, unsigned long long key) {
    const unsigned long long sign = 1ull << 63;
    const unsigned long long u = (op == OP_IMIN || op == OP_FMIN) ? ~key : key;
    long long ord = static_cast<long long>(u ^ sign);
    if (op == OP_FMIN || op == OP_FMAX) ord = ord >= 0 ? ord : (ord ^ 0x7fffffffffffffffll);
    return static_cast<uint64_t>(ord);
}

// Adds one lane's folded state of one world into the global atomic state.
__device__ __forceinline__ void atomic_fold(int op, uint64_t *cell, uint64_t acc) {
    switch (op) {
    case OP_ISUM: atomicAdd(reinterpret_cast<unsigned long long *>(cell), static_cast<unsigned long long>(acc)); break;
    case OP_FSUM_COMP: {
        const double v = static_cast<double>(__int_as_float(static_cast<int>(acc))) +
                         static_cast<double>(__int_as_float(static_cast<int>(acc >> 32)));
        atomicAdd(reinterpret_cast<double *>(cell), v);
        break;
    }
    case OP_FSUM_PLAIN: atomicAdd(reinterpret_cast<float *>(cell), __int_as_float(static_cast<int>(acc))); break;
    default: atomicMax(reinterpret_cast<unsigned long long *>(cell), minmax_key(op, acc)); break;
    }
}

// Per-item copy of the query's descriptor fields the row loop reads.
struct ItemShared {
    InputDev in;
    SlotDev slot[kMaxSpecs];
    int32_t n_slots, mode, bal, prune, pack;
    uint64_t *state, *ng;
    unsigned long long *abs;
    uint64_t row0, row_end;
    uint32_t k;
    uint32_t item;
    // mode 1: rows read from the group-ordered copies
    const uint64_t *smask;
    const uint32_t *sgid;
    const uint64_t *sval;
    uint64_t n;
};

// ---------------------------------------------------------------------------
// The per-bit engine on one 32-row batch of a warp.
//
// Lane r loads row r; the 32x32 bit matrix of world bits (row r, world j) is
// transposed across the warp so that lane j holds T_j, the set of this
// batch's rows in world j (a 32-bit row mask).  For every run R of rows of
// one group, lane j then gets:
//   count      popc(T_j & R);
//   int64 SUM  sum_b 2^b popc(T_j & R & V_b), V_b = rows whose value has
//              bit b (non-negative values of at most 32 bits, long runs), or
//              a broadcast loop over the rows of R;
//   float SUM  a broadcast loop over R in FP32, 8-row blocks folded into a
//              compensated (two-sum) accumulator;
//   MIN/MAX    a broadcast loop over R.
// With balanced masks (world j+32 = complement of world j) COUNT and int64
// SUM are kept for worlds 0..31 plus the run's total (exact integers, so
// world j+32 = total - world j); float SUM and MIN/MAX keep both worlds,
// since a float complement would cancel.  Without balance lane j also
// holds T'_j for world j+32.  The run's contributions go to a sink: the warp's
// private shared-memory state or the query's global state (atomics).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const uint32_t m = s == 16 ? 0x0000FFFFu : s == 8 ? 0x00FF00FFu : s == 4 ? 0x0F0F0F0Fu : s == 2 ? 0x33333333u : 0x55555555u;
        const uint32_t o = __shfl_xor_sync(kFull, x, s);
        x = (lane & s) ? ((x & ~m) | ((o >> s) & m)) : ((x & m) | ((o << s) & ~m));
    }
    return x;
}

// Slot operations of a batch whose queries share one spec signature are
// compile-time constants (no per-row dispatch on the operation); SIG 0 reads
// them from the query at run time.
//   SIG 1: {int64 SUM}                     (COUNT + SUM)
//   SIG 2: {int64 SUM, float SUM}
//   SIG 3: {int64 SUM, float SUM, float SUM}
//   SIG 4: {float SUM}
//   SIG 5: {int64 SUM, int64 SUM}          (two sums, e.g. a lifted ratio)
template <int SIG>
__device__ __forceinline__ int op_of(const ItemShared &is, int s) {
    if (SIG == 1 || SIG == 5) return OP_ISUM;
    if (SIG == 2 || SIG == 3) return s == 0 ? OP_ISUM : OP_FSUM_COMP;
    if (SIG == 4) return OP_FSUM_COMP;
    return is.slot[s].op;
}
template <int SIG>
__device__ __forceinline__ int nslots_of(const ItemShared &is) {
    return SIG == 1 ? 1 : SIG == 2 ? 2 : SIG == 3 ? 3 : SIG == 4 ? 1 : SIG == 5 ? 2 : is.n_slots;
}

// Loads row `row`'s group, mask and slot values; invalid rows get valid=false.
template <int NS, int SIG>
__device__ __forceinline__ void load_row(const ItemShared &is, uint64_t row, bool &valid, uint32_t &gid,
                                         uint64_t &mask, uint64_t (&vals)[NS], uint64_t (&my_abs)[NS],
                                         uint32_t *status) {
    const uint32_t G = is.in.n_groups;
    gid = 0;
    mask = 0;
    if (is.smask) {  // group-ordered copy: ids already checked, masks already hashed
        // records of 16 bytes: {mask, first slot value}; further slots in sval
        unsigned long long v0 = 0;
        if (valid) {
            const ulonglong2 rec = __ldg(reinterpret_cast<const ulonglong2 *>(is.smask) + row);
            if (is.pack) {  // {low mask word | group id << 32, value}: the high word is the complement
                gid = static_cast<uint32_t>(rec.x >> 32);
                const uint64_t lo = rec.x & 0xFFFFFFFFull;
                mask = lo | ((lo ^ 0xFFFFFFFFull) << 32);
            } else {
                gid = __ldg(is.sgid + row);
                mask = rec.x;
            }
            v0 = rec.y;
            if (drop_row(is.in, mask)) {
                valid = false;
                gid = 0;
            }
        }
#pragma unroll
        for (int s = 0; s < NS; s++) {
            vals[s] = 0;
            if (s < nslots_of<SIG>(is) && valid) {
                vals[s] = s == 0 ? v0 : __ldg(reinterpret_cast<const unsigned long long *>(is.sval) + (s - 1) * is.n + row);
                if (op_of<SIG>(is, s) == OP_ISUM) {
                    const long long v = static_cast<long long>(vals[s]);
                    const uint64_t a = v < 0 ? 0ull - static_cast<uint64_t>(v) : static_cast<uint64_t>(v);
                    const uint64_t t = my_abs[s] + a;
                    my_abs[s] = t < a ? ~0ull : t;
                }
            }
        }
        return;
    }
    if (valid) {
        gid = row_gid(is.in, row);
        if (gid >= G) {  // out-of-range group id: skip the row, report it
            raise_status(status, kStatusBadGroup);
            valid = false;
            gid = 0;
        } else {
            mask = row_mask(is.in, row);
            if (drop_row(is.in, mask)) {
                valid = false;
                gid = 0;
            }
        }
    }
#pragma unroll
    for (int s = 0; s < NS; s++) {
        vals[s] = 0;
        if (s < nslots_of<SIG>(is) && valid) {
            vals[s] = load_slot_value(is.slot[s], row);
            if (op_of<SIG>(is, s) == OP_ISUM) {
                const long long v = static_cast<long long>(vals[s]);
                const uint64_t a = v < 0 ? 0ull - static_cast<uint64_t>(v) : static_cast<uint64_t>(v);
                const uint64_t t = my_abs[s] + a;
                my_abs[s] = t < a ? ~0ull : t;
            }
        }
    }
}

// One lane's row as loaded from HBM, before the group check and the hash.
// The warp-private item loop of the run-time signature fetches the next
// 32-row batch into one of these while it folds the current one, so the
// loads' latency overlaps the work (the compile-time signatures keep
// load_row: their register budget has no room for a second batch).
template <int NS>
struct RawLane {
    uint32_t gid;
    uint64_t km;        // key, or world mask with PAC_IN_MASKS
    uint64_t vals[NS];  // slot value patterns
};

template <int NS, int SIG>
__device__ __forceinline__ void fetch_lane(const ItemShared &is, uint64_t row, uint64_t end, RawLane<NS> &r) {
    r.gid = 0;
    r.km = 0;
#pragma unroll
    for (int s = 0; s < NS; s++) r.vals[s] = 0;
    if (row >= end) return;
    r.gid = row_gid(is.in, row);
    r.km = __ldg(static_cast<const unsigned long long *>(is.in.km) + row);
#pragma unroll
    for (int s = 0; s < NS; s++)
        if (s < nslots_of<SIG>(is)) r.vals[s] = load_slot_value(is.slot[s], row);
}

// load_row's checks on a fetched lane: group range, world mask, dropped rows,
// running sums of |v|.
template <int NS, int SIG>
__device__ __forceinline__ void finish_lane(const ItemShared &is, const RawLane<NS> &r, bool &valid, uint32_t &gid,
                                            uint64_t &mask, uint64_t (&vals)[NS], uint64_t (&my_abs)[NS],
                                            uint32_t *status) {
    gid = 0;
    mask = 0;
    if (valid) {
        if (r.gid >= is.in.n_groups) {
            raise_status(status, kStatusBadGroup);
            valid = false;
        } else {
            mask = (is.in.in_flags & PAC_IN_MASKS) ? r.km
                                                    : keyed_world_mask(static_cast<long long>(r.km), is.in.qkey,
                                                                       is.in.hash_mode);
            if (drop_row(is.in, mask)) valid = false;
            else gid = r.gid;
        }
    }
#pragma unroll
    for (int s = 0; s < NS; s++) {
        vals[s] = 0;
        if (s < nslots_of<SIG>(is) && valid) {
            vals[s] = r.vals[s];
            if (op_of<SIG>(is, s) == OP_ISUM) {
                const long long v = static_cast<long long>(vals[s]);
                const uint64_t a = v < 0 ? 0ull - static_cast<uint64_t>(v) : static_cast<uint64_t>(v);
                const uint64_t t = my_abs[s] + a;
                my_abs[s] = t < a ? ~0ull : t;
            }
        }
    }
    if (!valid) mask = 0;
}

// One run's contributions for this lane: worlds j (index 0) and j+32 (1).
template <int NS>
struct RunAcc {
    uint32_t c0, c1;         // counts (c1 unused with bal)
    uint32_t n;              // rows in the run (uniform)
    uint32_t loop;           // rows the broadcast loop visited (uniform; 0: MIN/MAX states are identities)
    uint64_t a0[NS], a1[NS]; // slot states of worlds j and j+32 (a1 unused for int64 SUM with bal)
    uint64_t tot[NS];        // int64 SUM totals over the run (uniform)
};

__device__ __forceinline__ uint64_t pack_pair(float s, float c) {
    return static_cast<uint32_t>(__float_as_int(s)) | (static_cast<uint64_t>(static_cast<uint32_t>(__float_as_int(c))) << 32);
}

// Folds one 8-row block sum into a compensated (sum, comp) pair.
__device__ __forceinline__ void comp_add(float &s, float &c, float blk) {
    float ns, e;
    two_sum(s, blk, ns, e);
    s = ns;
    c += e;
}

// One row r of the broadcast loop: every loop-type slot takes row r's value.
template <int NS, int SIG>
__device__ __forceinline__ void loop_row(const ItemShared &is, int r, uint32_t M0, uint32_t M1, bool bal,
                                         const uint64_t (&vals)[NS], const bool (&sliced)[NS],
                                         RunAcc<NS> &ra, float (&fb0)[NS], float (&fb1)[NS]) {
    const bool b0 = (M0 >> r) & 1u, b1 = (M1 >> r) & 1u;
#pragma unroll
    for (int s = 0; s < NS; s++) {
        if (s >= nslots_of<SIG>(is)) continue;
        const int op = op_of<SIG>(is, s);
        if (op == OP_ISUM) {
            if (sliced[s]) continue;
            const uint64_t x = __shfl_sync(kFull, vals[s], r);
            ra.a0[s] += b0 ? x : 0ull;
            if (!bal) ra.a1[s] += b1 ? x : 0ull;  // with bal world j+32 = total - world j
            ra.tot[s] += x;
        } else if (op == OP_FSUM_COMP || op == OP_FSUM_PLAIN) {
            const float x = __int_as_float(__shfl_sync(kFull, static_cast<int>(vals[s]), r));
            fb0[s] += b0 ? x : 0.0f;
            fb1[s] += b1 ? x : 0.0f;
        } else {
            const uint64_t x = __shfl_sync(kFull, vals[s], r);
            op_update(op, ra.a0[s], x, b0 ? 1u : 0u);
            op_update(op, ra.a1[s], x, b1 ? 1u : 0u);
        }
    }
}

// Fills `ra` for run R of this batch.  T0/T1: transposed world sets of
// worlds j and j+32 (T1 ignored with bal).  slice[s]: bit count when slot s
// may be bit-sliced (0: loop).  L (a subset of R): the rows the broadcast
// loop visits; rows of R outside L change no loop-type state (bound
// pruning).  With compile-time slot operations a run of all 32 rows (the
// common case of group-ordered rows) takes a fully unrolled loop.
template <int NS, int SIG>
__device__ __forceinline__ void run_fold(const ItemShared &is, uint32_t R, uint32_t L, uint32_t T0, uint32_t T1,
                                         bool bal, const uint64_t (&vals)[NS], const int (&slice)[NS], int lane,
                                         RunAcc<NS> &ra) {
    const uint32_t M0 = T0 & R;
    const uint32_t M1 = bal ? (R & ~T0) : (T1 & R);
    ra.n = __popc(R);
    ra.loop = L;
    ra.c0 = __popc(M0);
    ra.c1 = __popc(M1);
    bool any_loop = false;
    // bit-slicing costs a fixed amount per value bit, the broadcast loop a
    // fixed amount per row: slice runs with at least as many rows as bits
    bool sliced[NS];
#pragma unroll
    for (int s = 0; s < NS; s++) {
        sliced[s] = false;
        if (s >= nslots_of<SIG>(is)) continue;
        const int op = op_of<SIG>(is, s);
        ra.a0[s] = ra.a1[s] = op_identity(op);
        ra.tot[s] = 0;
        sliced[s] = op == OP_ISUM && slice[s] > 0 && ra.n >= static_cast<uint32_t>(slice[s]);
        if (sliced[s]) {
            // bits below 26 add up in 32 bits (at most 32 rows * 2^26 < 2^31)
            uint32_t p0 = 0, p1 = 0, pt = 0;
            uint64_t acc0 = 0, acc1 = 0, tot = 0;
            for (int b = 0; b < slice[s]; b++) {
                const uint32_t vb = __ballot_sync(kFull, (vals[s] >> b) & 1ull) & R;
                const uint32_t c0 = __popc(M0 & vb), ct = __popc(vb);
                const uint32_t c1 = bal ? 0u : __popc(M1 & vb);
                if (b < 26) {
                    p0 += c0 << b;
                    p1 += c1 << b;
                    pt += ct << b;
                } else {
                    acc0 += static_cast<uint64_t>(c0) << b;
                    acc1 += static_cast<uint64_t>(c1) << b;
                    tot += static_cast<uint64_t>(ct) << b;
                }
            }
            ra.a0[s] = acc0 + p0;
            ra.a1[s] = acc1 + p1;  // unused with bal (world j+32 = total - world j)
            ra.tot[s] = tot + pt;
        } else {
            any_loop = true;
        }
    }
    // fixed signatures hold no MIN/MAX slot, so their loop covers R (kept
    // literal: a separate mask there doubles the kernels' register count)
    if (!any_loop || (SIG == 0 && L == 0)) return;
    // broadcast loop over the rows of L for the remaining slots; float sums
    // fold 8-row blocks into a compensated pair
    float fs0[NS], fc0[NS], fb0[NS], fs1[NS], fc1[NS], fb1[NS];
#pragma unroll
    for (int s = 0; s < NS; s++) fs0[s] = fc0[s] = fb0[s] = fs1[s] = fc1[s] = fb1[s] = 0.0f;
    auto flush_blocks = [&]() {
#pragma unroll
        for (int s = 0; s < NS; s++) {
            comp_add(fs0[s], fc0[s], fb0[s]);
            comp_add(fs1[s], fc1[s], fb1[s]);
            fb0[s] = fb1[s] = 0.0f;
        }
    };
    if (SIG != 0 && R == kFull) {
#pragma unroll
        for (int r = 0; r < 32; r++) {
            loop_row<NS, SIG>(is, r, M0, M1, bal, vals, sliced, ra, fb0, fb1);
            if ((r & 7) == 7) flush_blocks();
        }
    } else {
        int blk = 0;
        for (uint32_t rr = SIG != 0 ? R : L; rr; rr &= rr - 1) {
            loop_row<NS, SIG>(is, __ffs(rr) - 1, M0, M1, bal, vals, sliced, ra, fb0, fb1);
            if (++blk == 8) {
                blk = 0;
                flush_blocks();
            }
        }
        flush_blocks();
    }
#pragma unroll
    for (int s = 0; s < NS; s++) {
        if (s >= nslots_of<SIG>(is)) continue;
        const int op = op_of<SIG>(is, s);
        if (op == OP_FSUM_COMP) {
            ra.a0[s] = pack_pair(fs0[s], fc0[s]);
            ra.a1[s] = pack_pair(fs1[s], fc1[s]);
        } else if (op == OP_FSUM_PLAIN) {
            ra.a0[s] = pack_pair(fs0[s] + fc0[s], 0.0f);
            ra.a1[s] = pack_pair(fs1[s] + fc1[s], 0.0f);
        }
    }
}

// States kept as worlds 0..31 + total with balanced masks (exact integers).
__device__ __forceinline__ bool by_complement(int op, bool bal) { return bal && op == OP_ISUM; }

__device__ __forceinline__ bool is_minmax(int op) {
    return op == OP_IMIN || op == OP_IMAX || op == OP_FMIN || op == OP_FMAX;
}

// True when one row's value v would replace a MIN/MAX state st (the test of
// op_update): MAX takes strictly greater values, MIN strictly smaller ones,
// floats by IEEE comparison (a NaN value replaces nothing).
__device__ __forceinline__ bool mm_improves(int op, uint64_t v, uint64_t st) {
    switch (op) {
    case OP_IMAX: return static_cast<long long>(v) > static_cast<long long>(st);
    case OP_IMIN: return static_cast<long long>(v) < static_cast<long long>(st);
    case OP_FMAX: return __longlong_as_double(static_cast<long long>(v)) > __longlong_as_double(static_cast<long long>(st));
    default: return __longlong_as_double(static_cast<long long>(v)) < __longlong_as_double(static_cast<long long>(st));
    }
}

constexpr uint32_t kPruneMinRun = 8;  // shorter runs visit every row

// The bounds of one group, kept by a warp across the runs of an item.
template <int NS>
struct PruneCache {
    uint32_t g = 0xFFFFFFFFu;  // group the bounds belong to; none when all ones
    uint64_t b[NS];            // per slot, this lane's copy of the bound
};

// MIN/MAX bound pruning (Sec. 5 "Pruning"): the bound is the weakest of the
// 64 world states of the run's group (the smallest maximum for MAX, the
// largest minimum for MIN).  A value that does not improve the bound
// improves no world, so its row is left out of the broadcast loop.  The
// bound is read from the sink's state (a warp reduction over the 64 worlds)
// when the cache holds none for the group, and dropped after a run in which
// some row survived, since the state may have moved (the paper refreshes it
// every 2048 updates).  A stale bound is weaker, never wrong: states only
// move towards the extreme.  Returns the rows the loop must visit: R itself
// unless every loop-type slot is MIN/MAX.
template <int NS, int SIG, typename Sink>
__device__ __forceinline__ uint32_t prune_rows(const ItemShared &is, uint32_t R, uint32_t g,
                                               const uint64_t (&vals)[NS], const int (&slice)[NS],
                                               Sink &sink, PruneCache<NS> &pc, int lane) {
    if (SIG != 0 || !is.prune) return R;  // compile-time signatures hold no MIN/MAX slot
    const uint32_t n = __popc(R);
    if (n < kPruneMinRun) return R;
    bool any_mm = false;
#pragma unroll
    for (int s = 0; s < NS; s++) {
        if (s >= is.n_slots) continue;
        const int op = is.slot[s].op;
        if (op == OP_ISUM) {
            if (slice[s] > 0 && n >= static_cast<uint32_t>(slice[s])) continue;  // bit-sliced, not looped
            return R;
        }
        if (op == OP_FSUM_COMP || op == OP_FSUM_PLAIN) return R;
        any_mm = true;
    }
    if (!any_mm) return R;
    if (pc.g != g) {
#pragma unroll
        for (int s = 0; s < NS; s++) {
            if (s >= is.n_slots) continue;
            const int op = is.slot[s].op;
            if (!is_minmax(op)) continue;
            uint64_t b0, b1;
            if (!sink.bound(g, s, lane, b0, b1)) return R;
            uint64_t b = mm_improves(op, b0, b1) ? b1 : b0;  // the weaker of this lane's two worlds
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                const uint64_t other = __shfl_xor_sync(kFull, b, o);
                b = mm_improves(op, b, other) ? other : b;
            }
            pc.b[s] = b;
        }
        pc.g = g;
    }
    uint32_t keep = 0;
#pragma unroll
    for (int s = 0; s < NS; s++) {
        if (s >= is.n_slots) continue;
        const int op = is.slot[s].op;
        if (is_minmax(op)) keep |= __ballot_sync(kFull, ((R >> lane) & 1u) && mm_improves(op, vals[s], pc.b[s]));
    }
    if (keep) pc.g = 0xFFFFFFFFu;  // the state moves: read the bound again next time
    return keep;
}

// Processes rows [base, base+32) of the item: transposes, finds the runs and
// hands every run to `sink(g, ra)`.  With `pre` the rows were fetched
// already; otherwise they are loaded here.
template <int NS, int SIG, typename Sink>
__device__ __forceinline__ void batch32w(const ItemShared &is, uint64_t base, uint64_t end, uint64_t (&my_abs)[NS],
                                         uint32_t *status, Sink &sink, PruneCache<NS> &pc,
                                         const RawLane<NS> *pre = nullptr) {
    const int lane = threadIdx.x & 31;
    const uint64_t row = base + lane;
    bool valid = row < end;
    uint32_t gid;
    uint64_t mask, vals[NS];
    if (pre) finish_lane<NS, SIG>(is, *pre, valid, gid, mask, vals, my_abs, status);
    else load_row<NS, SIG>(is, row, valid, gid, mask, vals, my_abs, status);
    const bool bal = is.bal != 0;
    const uint32_t T0 = warp_transpose32(valid ? static_cast<uint32_t>(mask) : 0u, lane);
    const uint32_t T1 = bal ? 0u : warp_transpose32(valid ? static_cast<uint32_t>(mask >> 32) : 0u, lane);
    // bit-slicing is used for non-negative int64 values of at most 32 bits
    int slice[NS];
#pragma unroll
    for (int s = 0; s < NS; s++) {
        slice[s] = 0;
        if (s < nslots_of<SIG>(is) && op_of<SIG>(is, s) == OP_ISUM) {
            const uint32_t hi = __reduce_or_sync(kFull, static_cast<uint32_t>(vals[s] >> 32));
            const uint32_t lo = __reduce_or_sync(kFull, static_cast<uint32_t>(vals[s]));
            slice[s] = hi ? 0 : 32 - __clz(static_cast<int>(lo));
        }
    }
    uint32_t pending = __ballot_sync(kFull, valid);
    while (pending) {
        const int leader = __ffs(pending) - 1;
        const uint32_t g = __shfl_sync(kFull, gid, leader);
        const uint32_t R = __ballot_sync(kFull, valid && gid == g);
        pending &= ~R;
        RunAcc<NS> ra;
        const uint32_t L = prune_rows<NS, SIG>(is, R, g, vals, slice, sink, pc, lane);
        run_fold<NS, SIG>(is, R, L, T0, T1, bal, vals, slice, lane, ra);
        sink(g, ra, lane, bal);
    }
}

// Sink into the warp's private shared-memory state.
template <int NS, int SIG>
struct SmemSink {
    const ItemShared &is;
    uint64_t *st;    // this warp's [1+n_slots][G][64]
    uint64_t *ng;    // this warp's [G]
    uint32_t G;
    __device__ __forceinline__ void operator()(uint32_t g, const RunAcc<NS> &ra, int lane, bool bal) {
        uint64_t *cst = st + static_cast<size_t>(g) * kWorlds;
        cst[lane] += ra.c0;
        if (!bal) cst[lane + 32] += ra.c1;
        else if (lane == 0) cst[32] += ra.n;
#pragma unroll
        for (int s = 0; s < NS; s++) {
            if (s >= nslots_of<SIG>(is)) continue;
            const int op = op_of<SIG>(is, s);
            if (is_minmax(op) && !ra.loop) continue;  // identities: nothing to merge
            uint64_t *sst = st + (static_cast<size_t>(s + 1) * G + g) * kWorlds;
            op_merge(op, sst[lane], ra.a0[s]);
            if (!by_complement(op, bal)) op_merge(op, sst[lane + 32], ra.a1[s]);
            else if (lane == 0) op_merge(op, sst[32], ra.tot[s]);
        }
        if (lane == 0) ng[g] += ra.n;
    }
    // this lane's current MIN/MAX states of worlds j and j+32 for slot s
    __device__ __forceinline__ bool bound(uint32_t g, int s, int lane, uint64_t &b0, uint64_t &b1) const {
        const uint64_t *sst = st + (static_cast<size_t>(s + 1) * G + g) * kWorlds;
        b0 = sst[lane];
        b1 = sst[lane + 32];
        return true;
    }
};

// Sink into the query's global state with atomics.
template <int NS, int SIG>
struct AtomicSink {
    const ItemShared &is;
    uint32_t G;
    __device__ __forceinline__ void operator()(uint32_t g, const RunAcc<NS> &ra, int lane, bool bal) {
        uint64_t *cst = is.state + static_cast<size_t>(g) * kWorlds;
        if (ra.c0) atomicAdd(reinterpret_cast<unsigned long long *>(cst + lane), static_cast<unsigned long long>(ra.c0));
        if (!bal) {
            if (ra.c1) atomicAdd(reinterpret_cast<unsigned long long *>(cst + lane + 32), static_cast<unsigned long long>(ra.c1));
        } else if (lane == 0) {
            atomicAdd(reinterpret_cast<unsigned long long *>(cst + 32), static_cast<unsigned long long>(ra.n));
        }
#pragma unroll
        for (int s = 0; s < NS; s++) {
            if (s >= nslots_of<SIG>(is)) continue;
            const int op = op_of<SIG>(is, s);
            uint64_t *sst = is.state + (static_cast<size_t>(s + 1) * G + g) * kWorlds;
            if (ra.c0) atomic_fold(op, sst + lane, ra.a0[s]);
            if (!by_complement(op, bal)) {
                if (ra.c1) atomic_fold(op, sst + lane + 32, ra.a1[s]);
            } else if (lane == 0) {
                atomic_fold(op, sst + 32, ra.tot[s]);
            }
        }
        if (lane == 0) atomicAdd(reinterpret_cast<unsigned long long *>(is.ng + g), static_cast<unsigned long long>(ra.n));
    }
};

// Adds run `b` into run accumulator `a` (same group).
template <int NS, int SIG>
__device__ __forceinline__ void run_merge(const ItemShared &is, RunAcc<NS> &a, const RunAcc<NS> &b) {
    a.c0 += b.c0;
    a.c1 += b.c1;
    a.n += b.n;
    a.loop |= b.loop;
#pragma unroll
    for (int s = 0; s < NS; s++) {
        if (s >= nslots_of<SIG>(is)) continue;
        const int op = op_of<SIG>(is, s);
        if (op == OP_ISUM) {
            a.a0[s] += b.a0[s];
            a.a1[s] += b.a1[s];
            a.tot[s] += b.tot[s];
        } else if (!is_minmax(op) || b.loop) {
            op_merge(op, a.a0[s], b.a0[s]);
            op_merge(op, a.a1[s], b.a1[s]);
        }
    }
}

// Carries the current group's run across 32-row batches (rows in group
// order) and flushes it to the global state with atomics when the group
// changes and at the end of the item.
template <int NS, int SIG>
struct CarrySink {
    AtomicSink<NS, SIG> out;
    const ItemShared &is;
    RunAcc<NS> acc;
    uint32_t g_cur = 0xFFFFFFFFu;
    __device__ __forceinline__ void operator()(uint32_t g, const RunAcc<NS> &ra, int lane, bool bal) {
        if (g == g_cur) {
            run_merge<NS, SIG>(is, acc, ra);
            return;
        }
        if (g_cur != 0xFFFFFFFFu) out(g_cur, acc, lane, bal);
        acc = ra;
        g_cur = g;
    }
    __device__ __forceinline__ void flush(int lane, bool bal) {
        if (g_cur != 0xFFFFFFFFu) out(g_cur, acc, lane, bal);
        g_cur = 0xFFFFFFFFu;
    }
    // the carried run of group g is part of its final state: a bound for it
    // (other groups' states live in global memory and are not read)
    __device__ __forceinline__ bool bound(uint32_t g, int s, int lane, uint64_t &b0, uint64_t &b1) const {
        if (g != g_cur) return false;
        b0 = acc.a0[s];
        b1 = acc.a1[s];
        return true;
    }
};

// One item of a query with warp-private shared-memory states.
template <int NS, int SIG>
__device__ void item_warp_private(const ItemShared &is, unsigned char *smem_raw, uint32_t *status) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
    const uint32_t G = is.in.n_groups;
    const int nq = 1 + is.n_slots;
    const size_t per_warp = static_cast<size_t>(nq) * G * kWorlds;
    uint64_t *st = reinterpret_cast<uint64_t *>(smem_raw) + warp * per_warp;
    uint64_t *ng_all = reinterpret_cast<uint64_t *>(smem_raw) + n_warps * per_warp;  // [warps][G]
    uint64_t *ng = ng_all + warp * G;
    unsigned long long *abssum = reinterpret_cast<unsigned long long *>(ng_all + n_warps * G);  // [warps][NS]

    for (size_t k = lane; k < per_warp; k += 32) {
        const int qn = static_cast<int>(k / (static_cast<size_t>(G) * kWorlds));
        st[k] = qn == 0 ? 0ull : op_identity(is.slot[qn - 1].op);
    }
    for (uint32_t g = lane; g < G; g += 32) ng[g] = 0;
    __syncwarp();

    uint64_t my_abs[NS];
#pragma unroll
    for (int s = 0; s < NS; s++) my_abs[s] = 0;
    SmemSink<NS, SIG> sink{is, st, ng, G};
    PruneCache<NS> pc;
    const uint64_t stride = static_cast<uint64_t>(n_warps) * 32;
    uint64_t base = is.row0 + static_cast<uint64_t>(warp) * 32;
    if (SIG == 0 && NS <= 4) {
        // the next batch is fetched before the current one is folded
        RawLane<NS> cur;
        fetch_lane<NS, SIG>(is, base + lane, is.row_end, cur);
        for (; base < is.row_end; base += stride) {
            RawLane<NS> nxt;
            fetch_lane<NS, SIG>(is, base + stride + lane, is.row_end, nxt);
            batch32w<NS, SIG>(is, base, is.row_end, my_abs, status, sink, pc, &cur);
            cur = nxt;
        }
    } else {
        for (; base < is.row_end; base += stride) batch32w<NS, SIG>(is, base, is.row_end, my_abs, status, sink, pc);
    }
#pragma unroll
    for (int s = 0; s < NS; s++) {
        uint64_t m = my_abs[s];
        for (int o = 16; o; o >>= 1) {
            const uint64_t t = __shfl_xor_sync(kFull, m, o);
            const uint64_t u = m + t;
            m = u < t ? ~0ull : u;
        }
        if (lane == 0) abssum[warp * NS + s] = m;
    }
    __syncthreads();

    // the item's partial: warps merged in warp order
    uint64_t *out = is.state + static_cast<size_t>(is.k) * per_warp;
    const uint64_t *st0 = reinterpret_cast<const uint64_t *>(smem_raw);
    for (size_t k = threadIdx.x; k < per_warp; k += blockDim.x) {
        const int qn = static_cast<int>(k / (static_cast<size_t>(G) * kWorlds));
        uint64_t a = st0[k];
        for (int w = 1; w < n_warps; w++) {
            const uint64_t b = st0[static_cast<size_t>(w) * per_warp + k];
            if (qn == 0) a += b;
            else op_merge(is.slot[qn - 1].op, a, b);
        }
        out[k] = a;
    }
    uint64_t *ng_out = is.ng + static_cast<size_t>(is.k) * G;
    for (uint32_t g = threadIdx.x; g < G; g += blockDim.x) {
        uint64_t a = 0;
        for (int w = 0; w < n_warps; w++) a += ng_all[w * G + g];
        ng_out[g] = a;
    }
    // an exact int64 SUM needs every item partial to fit: sum |v| < 2^63
    if (threadIdx.x < NS && static_cast<int>(threadIdx.x) < is.n_slots && is.slot[threadIdx.x].op == OP_ISUM) {
        uint64_t tot = 0;
        for (int w = 0; w < n_warps; w++) {
            const uint64_t t = tot + abssum[w * NS + threadIdx.x];
            tot = t < tot ? ~0ull : t;
        }
        if (tot >= (1ull << 63)) raise_status(status, kStatusOverflow);
    }
    __syncthreads();  // shared memory is reused by the next item
}

// One item of a query with global-atomic states.
template <int NS, int SIG>
__device__ void item_atomic(const ItemShared &is, uint32_t *status) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
    const uint32_t G = is.in.n_groups;
    uint64_t my_abs[NS];
#pragma unroll
    for (int s = 0; s < NS; s++) my_abs[s] = 0;
    CarrySink<NS, SIG> sink{AtomicSink<NS, SIG>{is, G}, is};
    PruneCache<NS> pc;
    // each warp takes one contiguous stretch of the item, so group runs of
    // the group-ordered rows stay long within a warp
    const uint64_t span = is.row_end > is.row0 ? is.row_end - is.row0 : 0;
    const uint64_t per_warp = ((span + n_warps - 1) / n_warps + 31) / 32 * 32;
    const uint64_t w0 = is.row0 + static_cast<uint64_t>(warp) * per_warp;
    const uint64_t w1 = min(is.row_end, w0 + per_warp);
    ItemShared const &isr = is;
    for (uint64_t base = w0; base < w1; base += 32) batch32w<NS, SIG>(isr, base, w1, my_abs, status, sink, pc);
    sink.flush(lane, is.bal != 0);
    // int64 SUM guard: the wrapping atomics are exact while the query's total
    // of |v| stays below 2^63, which bounds every world's sum
#pragma unroll
    for (int s = 0; s < NS; s++) {
        if (s >= nslots_of<SIG>(is) || op_of<SIG>(is, s) != OP_ISUM) continue;
        unsigned long long m = my_abs[s];
        for (int o = 16; o; o >>= 1) {
            const unsigned long long t = __shfl_xor_sync(kFull, m, o);
            const unsigned long long u = m + t;
            m = u < t ? ~0ull : u;
        }
        if (lane == 0 && m) {
            const unsigned long long prev = atomicAdd(is.abs + s, m);
            if (prev + m < prev || prev + m >= (1ull << 63)) raise_status(status, kStatusOverflow);
        }
    }
}

// span[0] = ~(earliest block start), span[1] = latest block end, in
// %globaltimer nanoseconds (both zeroed before the launch): the device-time
// interval the kernel ran in, read back by the server to show that batches
// overlap on the device.
__device__ __forceinline__ unsigned long long device_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int NS, int SIG>
__global__ void __launch_bounds__(kBatchWarps * 32) k_batch_agg(const BatchQueryDev *__restrict__ qs,
                                                                const BatchItem *__restrict__ items,
                                                                uint32_t n_items, unsigned int *counter,
                                                                uint32_t *status, unsigned long long *span) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ ItemShared is;
    if (threadIdx.x == 0) atomicMax(span, ~device_ns());
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t it = atomicAdd(counter, 1u);
            is.item = it;
            if (it < n_items) {
                const BatchItem item = items[it];
                const BatchQueryDev &q = qs[item.q];
                is.in = q.in;
                is.n_slots = q.n_slots;
                is.mode = q.mode;
                is.bal = q.bal;
                is.prune = q.prune;
                is.state = q.state;
                is.ng = q.ng;
                is.abs = q.abs;
                is.row0 = item.row0;
                is.row_end = item.row0 + item.rows;
                is.k = item.k;
                is.smask = q.mode == 1 ? q.smask : nullptr;
                is.sgid = q.sgid;
                is.pack = q.pack;
                is.sval = q.sval;
                is.n = q.in.n;
                if (q.mode == 1) {
                    const uint64_t kept = q.pcnt[q.in.n_groups];  // rows that survived the group-id check
                    if (is.row_end > kept) is.row_end = kept;
                }
            }
        }
        __syncthreads();
        if (is.item >= n_items) break;
        if (threadIdx.x < kMaxSpecs && static_cast<int>(threadIdx.x) < is.n_slots)
            is.slot[threadIdx.x] = qs[items[is.item].q].slot[threadIdx.x];
        __syncthreads();
        if (is.mode == 0) item_warp_private<NS, SIG>(is, smem_raw, status);
        else item_atomic<NS, SIG>(is, status);
        __syncthreads();  // every thread is done with `is` before thread 0 refills it
    }
    if (threadIdx.x == 0) atomicMax(span + 1, device_ns());
}

// ---------------------------------------------------------------------------
// Partition of the many-group (mode 1) queries by group: a histogram of the
// group ids, an exclusive scan per query, and a scatter of (mask, group id,
// slot values) into group order.  Every row takes its own atomic: a warp
// aggregation per distinct group (match_any) cost more than the atomics it
// saved (highcard 100M: 7.91 -> 7.20 ms for the whole step, batch of 4096
// queries 293 -> 280 ms).
// ---------------------------------------------------------------------------
// Group ids below kPartSmem are counted per work item in shared memory and
// flushed with one global atomic per group and item; larger ids take a
// global atomic per row.
constexpr uint32_t kPartSmem = 2048;

__global__ void __launch_bounds__(256) k_part_hist(const BatchQueryDev *__restrict__ qs,
                                                   const BatchItem *__restrict__ items, uint32_t n_items,
                                                   uint32_t *status) {
    __shared__ uint32_t cnt_s[kPartSmem];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
    for (uint32_t it = blockIdx.x; it < n_items; it += gridDim.x) {
        const BatchItem item = items[it];
        const BatchQueryDev &q = qs[item.q];
        if (q.mode != 1) continue;
        const uint32_t G = q.in.n_groups;
        const uint32_t S = G < kPartSmem ? G : kPartSmem;
        for (uint32_t g = threadIdx.x; g < S; g += blockDim.x) cnt_s[g] = 0;
        __syncthreads();
        const uint64_t end = item.row0 + item.rows;
        constexpr int kC = 4;  // batches whose group ids are in flight together
        for (uint64_t base = item.row0 + static_cast<uint64_t>(warp) * 32 * kC; base < end;
             base += static_cast<uint64_t>(n_warps) * 32 * kC) {
            uint32_t gc[kC];
#pragma unroll
            for (int u = 0; u < kC; u++) {
                const uint64_t r = base + 32 * u + lane;
                gc[u] = r < end ? row_gid(q.in, r) : 0xFFFFFFFFu;
            }
#pragma unroll
            for (int u = 0; u < kC; u++) {
                uint32_t g = gc[u];
                bool valid = base + 32 * u + lane < end;
                if (valid && g >= G) {  // out-of-range group id: the row is dropped, and reported
                    raise_status(status, kStatusBadGroup);
                    valid = false;
                    g = 0xFFFFFFFFu;
                }
                if (valid) {
                    if (g < S) atomicAdd(cnt_s + g, 1u);
                    else atomicAdd(q.pcnt + g, 1u);
                }
            }
        }
        __syncthreads();
        for (uint32_t g = threadIdx.x; g < S; g += blockDim.x)
            if (cnt_s[g]) atomicAdd(q.pcnt + g, cnt_s[g]);
        __syncthreads();
    }
}

// One CTA (1024 threads) per query: pcur = exclusive prefix of pcnt,
// pcnt[G] = the number of rows kept, pcnt[G+1] = 1 when one group holds more
// than 1/64 of them.  Queries above kWideScanGroups take the multi-block scan
// below instead.
__global__ void __launch_bounds__(1024) k_part_scan(const BatchQueryDev *__restrict__ qs) {
    __shared__ uint32_t wsum[32];
    const BatchQueryDev &q = qs[blockIdx.x];
    if (q.mode != 1 || q.in.n_groups > kWideScanGroups) return;
    const uint32_t G = q.in.n_groups;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t chunk = (G + blockDim.x - 1) / blockDim.x;
    const uint32_t g0 = min(G, t * chunk), g1 = min(G, g0 + chunk);
    uint32_t local = 0, mx = 0;
    for (uint32_t g = g0; g < g1; g++) {
        local += q.pcnt[g];
        mx = max(mx, q.pcnt[g]);
    }
    __shared__ uint32_t s_mx;
    if (t == 0) s_mx = 0;
    uint32_t incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < static_cast<int>(blockDim.x >> 5) ? wsum[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += v;
        }
        wsum[lane] = w;  // inclusive prefix over warps
    }
    __syncthreads();
    uint32_t run = incl - local + (warp > 0 ? wsum[warp - 1] : 0u);
    for (uint32_t g = g0; g < g1; g++) {
        const uint32_t c = q.pcnt[g];
        q.pcur[g] = run;
        run += c;
    }
    atomicMax(&s_mx, mx);
    __syncthreads();
    if (t == static_cast<int>(blockDim.x) - 1) {
        const uint32_t kept = wsum[(blockDim.x >> 5) - 1];
        q.pcnt[G] = kept;
        // a group holding more than 1/64 of the rows makes the query "hot":
        // its scatter then reserves ranges per item instead of per warp
        q.pcnt[G + 1] = static_cast<uint64_t>(s_mx) * 64 > kept ? 1u : 0u;
    }
}

// Multi-block scan of one query with many groups: block b of nb takes the
// groups [G b / nb, G (b+1) / nb).  Pass 1 writes each range's sum and
// maximum to part[b] and part[nb + b]; pass 2 scans each range in 1024-group
// tiles (coalesced) from the sum of the ranges before it, and the last block
// writes pcnt[G] (rows kept) and pcnt[G+1] (the hot flag).
__device__ __forceinline__ uint32_t block_incl_scan(uint32_t v, uint32_t *wsum, uint32_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) wsum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    total = wsum[nw - 1];
    const uint32_t r = v + (warp > 0 ? wsum[warp - 1] : 0u);
    __syncthreads();  // wsum is reused by the next call
    return r;
}

__global__ void __launch_bounds__(1024) k_scan_wide_sum(const uint32_t *__restrict__ pcnt, uint32_t G, uint32_t nb,
                                                        uint32_t *__restrict__ part) {
    __shared__ uint32_t red[2][32];
    const uint32_t b = blockIdx.x;
    const uint32_t g0 = static_cast<uint32_t>(static_cast<uint64_t>(G) * b / nb);
    const uint32_t g1 = static_cast<uint32_t>(static_cast<uint64_t>(G) * (b + 1) / nb);
    uint32_t sum = 0, mx = 0;
    for (uint32_t g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
        const uint32_t c = pcnt[g];
        sum += c;
        mx = max(mx, c);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    sum = __reduce_add_sync(kFull, sum);
    mx = __reduce_max_sync(kFull, mx);
    if (lane == 0) {
        red[0][warp] = sum;
        red[1][warp] = mx;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        sum = __reduce_add_sync(kFull, lane < nw ? red[0][lane] : 0u);
        mx = __reduce_max_sync(kFull, lane < nw ? red[1][lane] : 0u);
        if (lane == 0) {
            part[b] = sum;
            part[nb + b] = mx;
        }
    }
}

__global__ void __launch_bounds__(1024) k_scan_wide_apply(uint32_t *__restrict__ pcnt, uint32_t *__restrict__ pcur,
                                                          uint32_t G, uint32_t nb, const uint32_t *__restrict__ part) {
    __shared__ uint32_t wsum[32];
    const uint32_t b = blockIdx.x;
    const uint32_t g0 = static_cast<uint32_t>(static_cast<uint64_t>(G) * b / nb);
    const uint32_t g1 = static_cast<uint32_t>(static_cast<uint64_t>(G) * (b + 1) / nb);
    uint32_t run = 0;
    for (uint32_t k = 0; k < b; k++) run += part[k];
    for (uint32_t base = g0; base < g1; base += blockDim.x) {
        const uint32_t g = base + threadIdx.x;
        const uint32_t c = g < g1 ? pcnt[g] : 0u;
        uint32_t total;
        const uint32_t incl = block_incl_scan(c, wsum, total);
        if (g < g1) pcur[g] = run + incl - c;
        run += total;
    }
    if (b == nb - 1 && threadIdx.x == 0) {
        uint32_t mx = 0;
        for (uint32_t k = 0; k < nb; k++) mx = max(mx, part[nb + k]);
        pcnt[G] = run;  // every range's rows: the rows kept
        pcnt[G + 1] = static_cast<uint64_t>(mx) * 64 > run ? 1u : 0u;
    }
}

// Scatter of one work item.  In a hot query (one group above 1/64 of the
// rows) the item's rows of groups below kPartSmem are counted in shared
// memory, each such group reserves one range of the query's cursor, and the
// rows take places of that range through shared cursors; every other row
// takes a place from the query's global cursor.  The order of a group's rows
// is not fixed (rows of different warps and CTAs never had a fixed order):
// the aggregations over them are exact integer sums, or float sums that
// combine in any order.
__global__ void __launch_bounds__(256) k_part_scatter(const BatchQueryDev *__restrict__ qs,
                                                      const BatchItem *__restrict__ items, uint32_t n_items) {
    __shared__ uint32_t cur_s[kPartSmem];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
    for (uint32_t it = blockIdx.x; it < n_items; it += gridDim.x) {
        const BatchItem item = items[it];
        const BatchQueryDev &q = qs[item.q];
        if (q.mode != 1) continue;
        const uint32_t G = q.in.n_groups;
        const bool hot = q.pcnt[G + 1] != 0;
        const uint32_t S = hot ? (G < kPartSmem ? G : kPartSmem) : 0u;  // no shared cursors for a cool query
        const uint64_t end = item.row0 + item.rows;
        // (1) the item's rows per small group
        for (uint32_t g = threadIdx.x; g < S; g += blockDim.x) cur_s[g] = 0;
        __syncthreads();
        constexpr int kC = 4;  // batches whose group ids are in flight together
        for (uint64_t base = item.row0 + static_cast<uint64_t>(warp) * 32 * kC; hot && base < end;
             base += static_cast<uint64_t>(n_warps) * 32 * kC) {
            uint32_t gc[kC];
#pragma unroll
            for (int u = 0; u < kC; u++) {
                const uint64_t r = base + 32 * u + lane;
                gc[u] = r < end ? row_gid(q.in, r) : 0xFFFFFFFFu;
            }
#pragma unroll
            for (int u = 0; u < kC; u++)
                if (gc[u] < S) atomicAdd(cur_s + gc[u], 1u);
        }
        __syncthreads();
        // (2) one range of the query's cursor per small group
        for (uint32_t g = threadIdx.x; g < S; g += blockDim.x) {
            const uint32_t c = cur_s[g];
            if (c) cur_s[g] = atomicAdd(q.pcur + g, c);
        }
        __syncthreads();
        // (3) rows into group order, four 32-row batches per warp at a time:
        // the group ids, keys and first values of all four are loaded before
        // the cursor atomics and the hashing, so their latencies overlap (two
        // at a time: batch of 4096 queries 281.8 -> 268.7 ms with four,
        // highcard 100M 7.20 -> 7.23 ms)
        constexpr int kU = 4, kHoist = 2;
        const uint64_t stride = static_cast<uint64_t>(n_warps) * 32 * kU;
        const bool masks_in = (q.in.in_flags & PAC_IN_MASKS) != 0;
        for (uint64_t base = item.row0 + static_cast<uint64_t>(warp) * 32 * kU; base < end; base += stride) {
            uint64_t r[kU], raw[kU], v[kU][kHoist];
            uint32_t g[kU];
            bool valid[kU];
#pragma unroll
            for (int u = 0; u < kU; u++) {
                r[u] = base + 32 * u + lane;
                valid[u] = r[u] < end;
                g[u] = valid[u] ? row_gid(q.in, r[u]) : 0xFFFFFFFFu;
                raw[u] = valid[u] ? static_cast<uint64_t>(__ldg(static_cast<const long long *>(q.in.km) + r[u])) : 0ull;
#pragma unroll
                for (int s2 = 0; s2 < kHoist; s2++)
                    v[u][s2] = (valid[u] && s2 < q.n_slots) ? load_slot_value(q.slot[s2], r[u]) : 0ull;
            }
            uint64_t d[kU];
#pragma unroll
            for (int u = 0; u < kU; u++) {
                if (valid[u] && g[u] >= G) {
                    valid[u] = false;
                    g[u] = 0xFFFFFFFFu;
                }
                d[u] = 0;
                if (valid[u]) d[u] = g[u] < S ? atomicAdd(cur_s + g[u], 1u) : atomicAdd(q.pcur + g[u], 1u);
            }
#pragma unroll
            for (int u = 0; u < kU; u++) {
                if (!valid[u]) continue;
                const uint64_t m = masks_in ? raw[u] : keyed_world_mask(static_cast<long long>(raw[u]), q.in.qkey,
                                                                        q.in.hash_mode);
                // one 16-byte record per row: the mask and the first slot value
                // (a scattered row then touches two sectors, not three); packed:
                // the low mask word and the group id share the first 8 bytes
                // (one sector per row)
                if (q.pack) {
                    reinterpret_cast<ulonglong2 *>(q.smask)[d[u]] =
                        make_ulonglong2((m & 0xFFFFFFFFull) | (static_cast<uint64_t>(g[u]) << 32),
                                        q.n_slots > 0 ? v[u][0] : 0ull);
                } else {
                    if (q.n_slots > 0)
                        reinterpret_cast<ulonglong2 *>(q.smask)[d[u]] = make_ulonglong2(m, v[u][0]);
                    else
                        q.smask[2 * static_cast<uint64_t>(d[u])] = m;
                    q.sgid[d[u]] = g[u];
                }
#pragma unroll
                for (int s2 = 1; s2 < kHoist; s2++)
                    if (s2 < q.n_slots) q.sval[static_cast<uint64_t>(s2 - 1) * q.in.n + d[u]] = v[u][s2];
                for (int s2 = kHoist; s2 < q.n_slots; s2++)
                    q.sval[static_cast<uint64_t>(s2 - 1) * q.in.n + d[u]] = load_slot_value(q.slot[s2], r[u]);
            }
        }
        __syncthreads();
    }
}

// One thread per (query, group, world) cell of the whole batch.
__global__ void __launch_bounds__(256) k_batch_merge(const BatchQueryDev *__restrict__ qs,
                                                     const uint64_t *__restrict__ cell_prefix, int n_queries,
                                                     uint64_t total_cells, uint32_t *status) {
    const uint64_t cell = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
    const bool live = cell < total_cells;
    // query of this cell: the last q with cell_prefix[q] <= cell (prefixes are multiples of 64)
    int lo = 0, hi = n_queries - 1;
    const uint64_t c = live ? cell : 0;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cell_prefix[mid] <= c) lo = mid;
        else hi = mid - 1;
    }
    const BatchQueryDev &q = qs[lo];
    const uint64_t local = c - cell_prefix[lo];
    const uint32_t G = q.in.n_groups;
    const uint32_t g = static_cast<uint32_t>(local / kWorlds);
    const int j = static_cast<int>(local % kWorlds);
    const size_t per_q = static_cast<size_t>(G) * kWorlds;
    const size_t per_part = per_q * (1 + q.n_slots);
    const bool atomic = q.mode == 1;
    const uint32_t parts = atomic ? 1u : q.n_items;
    // balanced masks: COUNT / int64 SUM of world j >= 32 = group total - world j-32
    const bool comp = q.bal != 0 && j >= 32;
    const size_t src = comp ? local - 32 : local;        // world j-32
    const size_t tot_at = local - j + 32;                 // the group's total

    uint64_t cnt = 0;
    if (live) {
        for (uint32_t k = 0; k < parts; k++) cnt += q.state[k * per_part + src];
        if (comp) {
            uint64_t tot = 0;
            for (uint32_t k = 0; k < parts; k++) tot += q.state[k * per_part + tot_at];
            cnt = tot - cnt;
        }
    }
    // meta: rows and OR of masks (bit j set iff world j saw a row); a warp
    // covers 32 worlds of one group because query prefixes are multiples of 64
    const unsigned bal = __ballot_sync(kFull, live && cnt > 0);
    if (!live) return;
    if (q.meta) {
        if ((threadIdx.x & 31) == 0) reinterpret_cast<uint32_t *>(q.meta + 2 * g + 1)[j >= 32 ? 1 : 0] = bal;
        if (j == 0) {
            uint64_t ng = 0;
            for (uint32_t k = 0; k < parts; k++) ng += q.ng[static_cast<size_t>(k) * G + g];
            q.meta[2 * g] = ng;
        }
    }
    for (int s = 0; s < q.n_out; s++) {
        const OutDev o = q.outs[s];
        if (o.kind == PAC_COUNT) {
            static_cast<uint64_t *>(o.out)[local] = cnt;
            continue;
        }
        const int op = q.slot[o.slot].op;
        const uint64_t *sp = q.state + static_cast<size_t>(o.slot + 1) * per_q + local;
        if (op == OP_ISUM) {
            const uint64_t *sq = q.state + static_cast<size_t>(o.slot + 1) * per_q;
            __int128 tot = 0;
            for (uint32_t k = 0; k < parts; k++) tot += static_cast<long long>(sq[k * per_part + src]);
            if (comp) {
                __int128 all = 0;
                for (uint32_t k = 0; k < parts; k++) all += static_cast<long long>(sq[k * per_part + tot_at]);
                tot = all - tot;
            }
            const bool fits = tot >= static_cast<__int128>(LLONG_MIN) && tot <= static_cast<__int128>(LLONG_MAX);
            if (!fits) raise_status(status, kStatusOverflow);
            const long long v = fits ? static_cast<long long>(tot) : (tot < 0 ? LLONG_MIN : LLONG_MAX);
            if (o.kind == PAC_SUM) static_cast<long long *>(o.out)[local] = v;
            else static_cast<double *>(o.out)[local] = cnt ? i128_to_double(tot) / static_cast<double>(cnt) : 0.0;
        } else if (op == OP_FSUM_COMP || op == OP_FSUM_PLAIN) {
            double total;
            if (atomic) {
                total = op == OP_FSUM_COMP ? __longlong_as_double(static_cast<long long>(sp[0]))
                                           : static_cast<double>(__int_as_float(static_cast<int>(sp[0])));
            } else {
                uint64_t a = sp[0];
                for (uint32_t k = 1; k < parts; k++) op_merge(op, a, sp[k * per_part]);
                total = static_cast<double>(__int_as_float(static_cast<int>(a)));
                if (op == OP_FSUM_COMP) total += static_cast<double>(__int_as_float(static_cast<int>(a >> 32)));
            }
            if (o.kind == PAC_SUM) static_cast<double *>(o.out)[local] = total;
            else static_cast<double *>(o.out)[local] = cnt ? total / static_cast<double>(cnt) : 0.0;
        } else {
            uint64_t a;
            if (atomic) {
                a = minmax_value(op, sp[0]);
            } else {
                a = sp[0];
                for (uint32_t k = 1; k < parts; k++) op_merge(op, a, sp[k * per_part]);
            }
            if (op == OP_IMIN || op == OP_IMAX)
                static_cast<long long *>(o.out)[local] = cnt ? static_cast<long long>(a) : 0ll;
            else
                static_cast<double *>(o.out)[local] = cnt ? __longlong_as_double(static_cast<long long>(a)) : 0.0;
        }
    }
}

}  // namespace


// ===========================================================================
// host side: plans
// ===========================================================================
namespace {

template <int NS, int SIG>
cudaError_t batch_kernel_setup(size_t smem, int *blocks_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_batch_agg<NS, SIG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batch_agg<NS, SIG>, kBatchWarps * 32, smem);
}

// The kernel variant of a plan: (NS, SIG) pairs instantiated below.
#define PAC_BATCH_VARIANTS(X) X(1, 0) X(2, 0) X(4, 0) X(kMaxSpecs, 0) X(1, 1) X(2, 2) X(4, 3) X(1, 4) X(2, 5)

template <typename T>
T *img_at(pac_batch *b, size_t off) {
    return reinterpret_cast<T *>(b->image.data() + off);
}

}  // namespace

pac_status plan_build(pac_ctx *ctx, const pac_query *qs, int n_queries, const BatchConfig &cfg, pac_batch **out) {
    pac_batch *b = new (std::nothrow) pac_batch();
    if (!b) return fail(ctx, PAC_E_NOMEM, "plan allocation");
    b->device = ctx->device;
    b->n_queries = n_queries;
    b->cfg = cfg;
    std::vector<BatchQueryDev> hq(n_queries);
    std::vector<BatchItem> hitems;
    std::vector<uint64_t> prefix(n_queries + 1, 0);
    std::vector<FinParams> hfin;
    b->rel_state.assign(n_queries, 0);
    b->rel_ng.assign(n_queries, 0);
    b->rel_abs.assign(n_queries, 0);
    b->rel_pcnt.assign(n_queries, SIZE_MAX);
    b->rel_pcur.assign(n_queries, SIZE_MAX);
    b->rel_smask.assign(n_queries, SIZE_MAX);
    b->rel_sgid.assign(n_queries, SIZE_MAX);
    b->rel_sval.assign(n_queries, SIZE_MAX);
    // the largest distinct-slot count decides the kernel's register arrays
    int max_slots = 0;
    for (int i = 0; i < n_queries; i++) {
        BatchQueryDev &d = hq[i];
        std::memset(&d, 0, sizeof(d));
        const pac_query &q = qs[i];
        int slot_of[kMaxSpecs];
        for (int s = 0; s < q.n_specs; s++) {
            slot_of[s] = -1;
            const int op = spec_op(q.specs[s]);
            if (op < 0) continue;
            for (int k = 0; k < d.n_slots; k++)
                if (d.slot[k].op == op && d.slot[k].values == q.specs[s].values && d.slot[k].vtype == q.specs[s].vtype)
                    slot_of[s] = k;
            if (slot_of[s] < 0) {
                d.slot[d.n_slots].op = op;
                d.slot[d.n_slots].vtype = q.specs[s].vtype;
                d.slot[d.n_slots].values = q.specs[s].values;
                slot_of[s] = d.n_slots++;
            }
        }
        for (int s = 0; s < q.n_specs; s++) {
            d.outs[d.n_out].kind = q.specs[s].kind;
            d.outs[d.n_out].slot = slot_of[s];
            d.outs[d.n_out].out = q.specs[s].out;
            d.n_out++;
        }
        max_slots = std::max(max_slots, static_cast<int>(d.n_slots));
    }
    b->ns = max_slots <= 1 ? 1 : max_slots <= 2 ? 2 : max_slots <= 4 ? 4 : kMaxSpecs;
    // one shared slot signature -> a kernel with compile-time slot operations
    auto sig_of = [](const BatchQueryDev &d) {
        auto op = [&](int k) { return d.slot[k].op; };
        if (d.n_slots == 1 && op(0) == OP_ISUM) return 1;
        if (d.n_slots == 2 && op(0) == OP_ISUM && op(1) == OP_FSUM_COMP) return 2;
        if (d.n_slots == 3 && op(0) == OP_ISUM && op(1) == OP_FSUM_COMP && op(2) == OP_FSUM_COMP) return 3;
        if (d.n_slots == 1 && op(0) == OP_FSUM_COMP) return 4;
        if (d.n_slots == 2 && op(0) == OP_ISUM && op(1) == OP_ISUM) return 5;
        return 0;
    };
    b->sig = n_queries > 0 ? sig_of(hq[0]) : 0;
    for (int i = 1; i < n_queries && b->sig; i++)
        if (sig_of(hq[i]) != b->sig) b->sig = 0;
    if (b->sig == 1 || b->sig == 4) b->ns = 1;
    if (b->sig == 2 || b->sig == 5) b->ns = 2;
    if (b->sig == 3) b->ns = 4;
    // device block: [zeroed scratch | partials | image]; offsets relative to it
    size_t zero_off = 256;  // the item counter lives at offset 0
    size_t part_off = 0;    // relative to the start of the partials region
    std::vector<size_t> p_state(n_queries, 0), p_ng(n_queries, 0);
    std::vector<size_t> p_pcur(n_queries, 0), p_smask(n_queries, 0), p_sgid(n_queries, 0), p_sval(n_queries, 0);
    size_t smem_max = 1024;
    for (int i = 0; i < n_queries; i++) {
        const pac_query &q = qs[i];
        BatchQueryDev &d = hq[i];
        d.in = make_input(&q.in);
        d.meta = q.meta;
        d.bal = ((q.in.in_flags & PAC_IN_MASKS) == 0 && q.in.hash_mode == PAC_HASH_BALANCED) ? 1 : 0;
        d.prune = ctx->opt_minmax_prune ? 1 : 0;
        d.pack = d.bal;  // partitioned queries with balanced keys write packed records
        const uint32_t G = q.in.n_groups;
        const size_t per_part = static_cast<size_t>(1 + d.n_slots) * G * kWorlds * 8;
        const size_t smem_need = bitloop_smem_bytes(kBatchWarps, d.n_slots, G, b->ns);
        d.mode = (smem_need <= cfg.smem_cap && !cfg.partition_only) ? 0 : 1;
        const uint64_t n = q.in.n;
        const uint32_t n_items = n == 0 ? 1u : static_cast<uint32_t>((n + cfg.item_rows - 1) / cfg.item_rows);
        d.first_item = static_cast<uint32_t>(hitems.size());
        d.n_items = n_items;
        for (uint32_t k = 0; k < n_items; k++) {
            BatchItem it{};
            it.q = static_cast<uint32_t>(i);
            it.k = k;
            it.row0 = static_cast<uint64_t>(k) * cfg.item_rows;
            const uint64_t rem = n - std::min<uint64_t>(n, it.row0);
            it.rows = static_cast<uint32_t>(std::min<uint64_t>(rem, cfg.item_rows));
            hitems.push_back(it);
        }
        if (d.mode == 0) {
            smem_max = std::max(smem_max, smem_need);
            p_state[i] = align_up(part_off, 256);
            part_off = p_state[i] + per_part * n_items;
            p_ng[i] = align_up(part_off, 256);
            part_off = p_ng[i] + static_cast<size_t>(G) * 8 * n_items;
            b->n_warp_private++;
        } else {
            if (!cfg.partition_only) {
                b->rel_state[i] = align_up(zero_off, 256);
                zero_off = b->rel_state[i] + per_part;
                b->rel_ng[i] = align_up(zero_off, 256);
                zero_off = b->rel_ng[i] + static_cast<size_t>(G) * 8;
                b->rel_abs[i] = align_up(zero_off, 256);
                zero_off = b->rel_abs[i] + kMaxSpecs * 8;
            }
            b->rel_pcnt[i] = align_up(zero_off, 256);
            zero_off = b->rel_pcnt[i] + (static_cast<size_t>(G) + 2 + 2 * kWideScanBlocks) * 4;
            if (G > kWideScanGroups) b->n_wide++;
            // group-ordered copies (fully overwritten by the scatter)
            p_pcur[i] = align_up(part_off, 256);
            part_off = p_pcur[i] + static_cast<size_t>(G) * 4;
            p_smask[i] = align_up(part_off, 256);  // 16-byte records {mask, slot 0}
            part_off = p_smask[i] + n * 16;
            p_sgid[i] = align_up(part_off, 256);
            // 16 bytes readable past the end (bulk copies of whole 16-byte units);
            // packed records carry the group ids themselves
            part_off = p_sgid[i] + (d.pack ? 0 : n * 4) + 16;
            p_sval[i] = align_up(part_off, 256);  // slots 1 .. n_slots-1
            part_off = p_sval[i] + n * 8 * static_cast<size_t>(d.n_slots > 0 ? d.n_slots - 1 : 0);
            b->n_atomic++;
        }
        prefix[i + 1] = prefix[i] + static_cast<uint64_t>(G) * kWorlds;
        if (q.fin_mode >= 0) {
            FinParams f{};
            for (int s = 0; s < q.n_specs; s++) {
                f.spec[s].kind = q.specs[s].kind;
                f.spec[s].vtype = q.specs[s].kind == PAC_COUNT ? PAC_I64 : q.specs[s].vtype;
                f.spec[s].variant = q.specs[s].variant;
                f.spec[s].out = q.specs[s].out;
            }
            f.n_specs = q.n_specs;
            f.n_groups = G;
            f.meta = q.meta;
            f.seed = q.seed;
            f.budget = q.budget;
            f.mode = q.fin_mode;
            f.noised = q.noised;
            f.is_null = q.is_null;
            f.flags = q.flags;
            f.posterior = nullptr;
            hfin.push_back(f);
        }
    }
    b->n_items = static_cast<uint32_t>(hitems.size());
    b->n_rel = static_cast<int>(hfin.size());
    b->total_cells = prefix[n_queries];
    b->smem = smem_max;
    b->zero_bytes = align_up(zero_off, 256);
    const size_t parts_base = b->zero_bytes;
    for (int i = 0; i < n_queries; i++) {
        if (hq[i].mode == 0) {
            b->rel_state[i] = parts_base + p_state[i];
            b->rel_ng[i] = parts_base + p_ng[i];
            b->rel_abs[i] = SIZE_MAX;
        } else {
            b->rel_pcur[i] = parts_base + p_pcur[i];
            b->rel_smask[i] = parts_base + p_smask[i];
            b->rel_sgid[i] = parts_base + p_sgid[i];
            b->rel_sval[i] = parts_base + p_sval[i];
        }
    }
    b->image_off = align_up(parts_base + part_off, 256);
    // the image
    size_t off = 0;
    b->img_q = off;
    off = align_up(off + sizeof(BatchQueryDev) * n_queries, 256);
    b->img_items = off;
    off = align_up(off + sizeof(BatchItem) * hitems.size(), 256);
    b->img_prefix = off;
    off = align_up(off + sizeof(uint64_t) * prefix.size(), 256);
    b->img_fin = off;
    off = align_up(off + sizeof(FinParams) * hfin.size(), 256);
    b->image.assign(off, 0);
    std::memcpy(b->image.data() + b->img_q, hq.data(), sizeof(BatchQueryDev) * n_queries);
    if (!hitems.empty()) std::memcpy(b->image.data() + b->img_items, hitems.data(), sizeof(BatchItem) * hitems.size());
    std::memcpy(b->image.data() + b->img_prefix, prefix.data(), sizeof(uint64_t) * prefix.size());
    if (!hfin.empty()) std::memcpy(b->image.data() + b->img_fin, hfin.data(), sizeof(FinParams) * hfin.size());
    b->device_bytes = b->image_off + b->image.size();
    *out = b;
    return PAC_OK;
}

void plan_bind(pac_batch *b, void *dbuf) {
    b->dbuf = dbuf;
    char *base = static_cast<char *>(dbuf);
    BatchQueryDev *q = img_at<BatchQueryDev>(b, b->img_q);
    for (int i = 0; i < b->n_queries; i++) {
        q[i].state = reinterpret_cast<uint64_t *>(base + b->rel_state[i]);
        q[i].ng = reinterpret_cast<uint64_t *>(base + b->rel_ng[i]);
        q[i].abs = b->rel_abs[i] == SIZE_MAX ? nullptr : reinterpret_cast<unsigned long long *>(base + b->rel_abs[i]);
        auto at = [&](size_t rel) { return rel == SIZE_MAX ? nullptr : base + rel; };
        q[i].pcnt = reinterpret_cast<uint32_t *>(at(b->rel_pcnt[i]));
        q[i].pcur = reinterpret_cast<uint32_t *>(at(b->rel_pcur[i]));
        q[i].smask = reinterpret_cast<uint64_t *>(at(b->rel_smask[i]));
        q[i].sgid = reinterpret_cast<uint32_t *>(at(b->rel_sgid[i]));
        q[i].sval = reinterpret_cast<uint64_t *>(at(b->rel_sval[i]));
    }
}

pac_status plan_setup_kernel(pac_ctx *ctx, pac_batch *b) {
    int per_sm = 0;
    cudaError_t e = cudaErrorInvalidValue;
#define PAC_SETUP(NS_, SIG_) \
    if (b->ns == NS_ && b->sig == SIG_) e = batch_kernel_setup<NS_, SIG_>(b->smem, &per_sm);
    PAC_BATCH_VARIANTS(PAC_SETUP)
#undef PAC_SETUP
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch kernel setup");
    b->n_ctas = ctx->n_sms * std::max(per_sm, 1);
    return PAC_OK;
}

pac_status plan_enqueue(pac_ctx *ctx, pac_batch *b, cudaStream_t s, const void *image_src) {
    char *base = static_cast<char *>(b->dbuf);
    if (image_src)
        PAC_CUDA(ctx, cudaMemcpyAsync(base + b->image_off, image_src, b->image.size(), cudaMemcpyHostToDevice, s));
    PAC_CUDA(ctx, cudaMemsetAsync(base, 0, b->zero_bytes, s));
    const BatchQueryDev *d_q = reinterpret_cast<const BatchQueryDev *>(base + b->image_off + b->img_q);
    const BatchItem *d_items = reinterpret_cast<const BatchItem *>(base + b->image_off + b->img_items);
    const uint64_t *d_prefix = reinterpret_cast<const uint64_t *>(base + b->image_off + b->img_prefix);
    const FinParams *d_fin = reinterpret_cast<const FinParams *>(base + b->image_off + b->img_fin);
    unsigned int *counter = reinterpret_cast<unsigned int *>(base);
    unsigned long long *span = reinterpret_cast<unsigned long long *>(base + kPlanSpanOffset);
    const unsigned grid = static_cast<unsigned>(std::min<uint64_t>(b->n_ctas, std::max<uint32_t>(b->n_items, 1)));
    if (b->n_atomic > 0) {
        const unsigned pgrid = static_cast<unsigned>(std::min<uint64_t>(static_cast<uint64_t>(ctx->n_sms) * 8,
                                                                        std::max<uint32_t>(b->n_items, 1)));
        k_part_hist<<<pgrid, 256, 0, s>>>(d_q, d_items, b->n_items, b->d_status);
        k_part_scan<<<static_cast<unsigned>(b->n_queries), 1024, 0, s>>>(d_q);
        if (b->n_wide > 0) {
            const BatchQueryDev *hq = reinterpret_cast<const BatchQueryDev *>(b->image.data() + b->img_q);
            for (int i = 0; i < b->n_queries; i++) {
                const uint32_t G = hq[i].in.n_groups;
                if (hq[i].mode != 1 || G <= kWideScanGroups) continue;
                uint32_t *pcnt = reinterpret_cast<uint32_t *>(base + b->rel_pcnt[i]);
                uint32_t *pcur = reinterpret_cast<uint32_t *>(base + b->rel_pcur[i]);
                const uint32_t nb = wide_scan_blocks(G);
                k_scan_wide_sum<<<nb, 1024, 0, s>>>(pcnt, G, nb, pcnt + G + 2);
                k_scan_wide_apply<<<nb, 1024, 0, s>>>(pcnt, pcur, G, nb, pcnt + G + 2);
            }
        }
        k_part_scatter<<<pgrid, 256, 0, s>>>(d_q, d_items, b->n_items);
        PAC_CUDA(ctx, cudaGetLastError());
    }
    if (b->cfg.partition_only) return PAC_OK;
#define PAC_LAUNCH(NS_, SIG_)                                                                              \
    if (b->ns == NS_ && b->sig == SIG_)                                                                    \
        k_batch_agg<NS_, SIG_><<<grid, kBatchWarps * 32, b->smem, s>>>(d_q, d_items, b->n_items, counter,  \
                                                                       b->d_status, span);
    PAC_BATCH_VARIANTS(PAC_LAUNCH)
#undef PAC_LAUNCH
    PAC_CUDA(ctx, cudaGetLastError());
    if (b->total_cells > 0) {
        const uint64_t blocks = (b->total_cells + 255) / 256;
        k_batch_merge<<<static_cast<unsigned>(blocks), 256, 0, s>>>(d_q, d_prefix, b->n_queries, b->total_cells,
                                                                    b->d_status);
        PAC_CUDA(ctx, cudaGetLastError());
    }
    if (b->n_rel > 0) PAC_CUDA(ctx, launch_finalize_batch(d_fin, b->n_rel, s));
    return PAC_OK;
}

void plan_destroy(pac_batch *b) {
    if (!b) return;
    if (b->owns_dbuf && b->dbuf) {
        cudaSetDevice(b->device);
        cudaDeviceSynchronize();
        cudaFree(b->dbuf);
    }
    delete b;
}

namespace {

// A plan with its own device block, image uploaded synchronously.
pac_status build_owned_plan(pac_ctx *ctx, const pac_query *qs, int n, const BatchConfig &cfg, pac_batch **out) {
    pac_batch *b = nullptr;
    pac_status st = plan_build(ctx, qs, n, cfg, &b);
    if (st != PAC_OK) return st;
    void *dbuf = nullptr;
    cudaError_t e = cudaMalloc(&dbuf, b->device_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return fail(ctx, PAC_E_NOMEM, "batch plan: cudaMalloc(%zu): %s", b->device_bytes, cudaGetErrorString(e));
    }
    b->owns_dbuf = true;
    plan_bind(b, dbuf);
    b->d_status = ctx->d_status;
    e = cudaMemcpy(static_cast<char *>(dbuf) + b->image_off, b->image.data(), b->image.size(), cudaMemcpyHostToDevice);
    // a copy from pageable memory may still be in flight on the legacy
    // stream when cudaMemcpy returns; the plan may be launched on a
    // non-blocking stream, which is not ordered after it
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) {
        plan_destroy(b);
        return cuda_fail(ctx, e, "batch plan upload");
    }
    st = plan_setup_kernel(ctx, b);
    if (st != PAC_OK) {
        plan_destroy(b);
        return st;
    }
    *out = b;
    return PAC_OK;
}

pac_status check_batch(pac_ctx *ctx, const pac_query *qs, int32_t n) {
    if (n < 1) return fail(ctx, PAC_E_INVALID, "n_queries %d", n);
    if (!qs) return fail(ctx, PAC_E_INVALID, "queries is NULL");
    for (int i = 0; i < n; i++) {
        pac_status st = check_query(ctx, &qs[i]);
        if (st != PAC_OK) return fail(ctx, st, "query %d: %s", i, ctx->last_error.c_str());
    }
    return PAC_OK;
}

// Configurations the autotuner tries: work-item size x shared-memory cap.
const BatchConfig kCandidates[] = {
    {1u << 15, 48 * 1024}, {1u << 15, 100 * 1024}, {1u << 15, 200 * 1024},
    {1u << 17, 48 * 1024}, {1u << 17, 100 * 1024}, {1u << 17, 200 * 1024},
};

uint64_t batch_signature(const pac_query *qs, int n) {
    uint64_t rows = 0, cells = 0;
    for (int i = 0; i < n; i++) {
        rows += qs[i].in.n;
        cells += qs[i].in.n_groups;
    }
    auto lg = [](uint64_t x) {
        uint64_t l = 0;
        while (x > 1) {
            x >>= 1;
            l++;
        }
        return l;
    };
    return (static_cast<uint64_t>(n) << 32) ^ (lg(rows) << 16) ^ lg(cells + 1);
}

// Autotune cache per process: batch signature -> configuration.
std::map<uint64_t, BatchConfig> &tune_cache() {
    static std::map<uint64_t, BatchConfig> m;
    return m;
}

}  // namespace

pac_status check_query(pac_ctx *ctx, const pac_query *q) {
    pac_status st = check_input(ctx, &q->in);
    if (st == PAC_OK) st = check_specs(ctx, &q->in, q->specs, q->n_specs);
    if (st == PAC_OK && q->n_specs < 1) st = fail(ctx, PAC_E_INVALID, "n_specs %d", q->n_specs);
    if (st != PAC_OK) return st;
    for (int s = 0; s < q->n_specs; s++)
        if (q->specs[s].variant != PAC_EXACT)
            return fail(ctx, PAC_E_UNSUPPORTED, "spec %d: batches serve PAC_EXACT specs only", s);
    if (q->in.n > 0xFFFFFFFFull * 1024ull) return fail(ctx, PAC_E_INVALID, "too many rows");
    if (q->fin_mode != -1) {
        if (q->fin_mode != PAC_FIN_ADAPTIVE && q->fin_mode != PAC_FIN_INDEPENDENT)
            return fail(ctx, PAC_E_INVALID, "fin_mode %d", q->fin_mode);
        if (!q->meta || !q->noised || !q->is_null || !q->flags)
            return fail(ctx, PAC_E_INVALID, "a release needs meta and its outputs");
        if (!(q->budget > 0.0)) return fail(ctx, PAC_E_INVALID, "budget must be > 0");
    }
    return PAC_OK;
}

}  // namespace pacgpu

using namespace pacgpu;

extern "C" {

pac_status pac_batch_plan(pac_ctx *ctx, const pac_query *queries, int32_t n_queries, uint32_t flags,
                          pac_batch **plan) {
    if (!ctx || !plan) return PAC_E_INVALID;
    *plan = nullptr;
    pac_status st = check_batch(ctx, queries, n_queries);
    if (st != PAC_OK) return st;
    st = bind_device(ctx);
    if (st != PAC_OK) return st;
    BatchConfig cfg = kBatchDefault;
    const uint64_t sig = batch_signature(queries, n_queries);
    auto hit = tune_cache().find(sig);
    if (hit != tune_cache().end()) {
        cfg = hit->second;
    } else if (flags & PAC_BATCH_AUTOTUNE) {
        cudaStream_t s = nullptr;
        PAC_CUDA(ctx, cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = 1e30f;
        for (const BatchConfig &c : kCandidates) {
            pac_batch *b = nullptr;
            if (build_owned_plan(ctx, queries, n_queries, c, &b) != PAC_OK) continue;
            float ms = 1e30f;
            if (plan_enqueue(ctx, b, s, nullptr) == PAC_OK && cudaStreamSynchronize(s) == cudaSuccess) {
                cudaEventRecord(e0, s);
                plan_enqueue(ctx, b, s, nullptr);
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
            }
            plan_destroy(b);
            if (ms < best) {
                best = ms;
                cfg = c;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaStreamDestroy(s);
        cudaGetLastError();
        tune_cache()[sig] = cfg;
    }
    return build_owned_plan(ctx, queries, n_queries, cfg, plan);
}

pac_status pac_batch_launch(pac_ctx *ctx, pac_batch *plan, pac_stream stream) {
    if (!ctx || !plan) return PAC_E_INVALID;
    if (plan->device != ctx->device) return fail(ctx, PAC_E_INVALID, "plan belongs to device %d", plan->device);
    pac_status st = bind_device(ctx);
    if (st != PAC_OK) return st;
    plan->d_status = ctx->d_status;
    st = plan_enqueue(ctx, plan, stream, nullptr);
    if (st != PAC_OK) return st;
    ctx->last_launches = 2 + (plan->n_rel > 0 ? 1 : 0) + (plan->n_atomic > 0 ? 3 : 0);
    return PAC_OK;
}

void pac_batch_free(pac_batch *plan) { plan_destroy(plan); }

pac_status pac_batch_info(const pac_batch *plan, const char *name, int64_t *value) {
    if (!plan || !name || !value) return PAC_E_INVALID;
    if (!strcmp(name, "n_items")) *value = plan->n_items;
    else if (!strcmp(name, "item_rows")) *value = plan->cfg.item_rows;
    else if (!strcmp(name, "smem_cap")) *value = static_cast<int64_t>(plan->cfg.smem_cap);
    else if (!strcmp(name, "kernels"))
        *value = 2 + (plan->n_rel > 0 ? 1 : 0) + (plan->n_atomic > 0 ? 3 : 0) + 2 * plan->n_wide;
    else if (!strcmp(name, "n_warp_private")) *value = plan->n_warp_private;
    else if (!strcmp(name, "n_atomic")) *value = plan->n_atomic;
    else if (!strcmp(name, "device_bytes")) *value = static_cast<int64_t>(plan->device_bytes);
    else return PAC_E_INVALID;
    return PAC_OK;
}

pac_status pac_batch_run(pac_ctx *ctx, const pac_query *queries, int32_t n_queries, pac_stream stream) {
    pac_batch *plan = nullptr;
    pac_status st = pac_batch_plan(ctx, queries, n_queries, 0, &plan);
    if (st != PAC_OK) return st;
    st = pac_batch_launch(ctx, plan, stream);
    if (st == PAC_OK) st = pac_sync_status(ctx, stream);
    else cudaStreamSynchronize(stream);
    pac_batch_free(plan);
    return st;
}

}  // extern "C"
