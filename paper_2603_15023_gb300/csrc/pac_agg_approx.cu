// pac_agg_approx.cu -- the paper's approximate integer SUM/AVG (Sec. 5
// "Approximation", "Two-sided SUM").
//
// Per world, 25 levels of 16-bit counters that cascade every 4 bits: a value
// v goes to level l = floor((msb(|v|) - 8) / 4) (0 below 2^8) as |v| >> 4l;
// every level keeps the exact total of what it received, and a level whose
// total would pass 0xFFFF is first flushed: its counters, shifted right by 4,
// are added to the next level (which is flushed first if it would overflow
// in turn).  Negative values go to a second, negated state; the result is
// S_pos - S_neg with S = sum_l C_l << 4l.
//
// The cascade depends on update order, so the schedule is fixed: rows are cut
// into chunks of 4096 consecutive rows, each chunk fills a fresh state per
// group in row order, and chunk states are merged level by level (flush on
// overflow, then add) in a pairwise tree over the chunk index.
//
// GPU mapping: one warp per (chunk, group); lane l owns worlds l and l+32,
// packed as the low and high halves of one 32-bit word per level (a half can
// never carry into the other: each half is bounded by the level total, which
// stays <= 0xFFFF); lane k < 25 holds the level-k totals of both sides in
// registers.  A CTA holds an aligned block of 16 chunks of one group (so a
// group with few rows frees its SM early) and does the first tree levels in
// shared memory; the remaining levels run one launch per level
// over the block states in global memory.
//
// Row loop: between two flushes of a level, its 64 counters only grow by
// sum_i x_i * bit_j(mask_i); the sequential part of the cascade is the scalar
// level totals alone.  The warp queues its group's rows of the chunk (in row
// order) and takes them 32 at a time: lane r computes row r's side, level and
// units x_r, the 32 masks are bit-transposed (lane j: world j's bits of the
// batch), and the batch is cut at the first row whose update would overflow
// its level's total (found from per-level prefix sums of x against the
// totals).  The rows before the cut are added level by level as bit-plane
// popcount sums (12 planes of x); the cut row's level is flushed with its
// cascade and the walk resumes at that row.  Every flush decision reads exact
// totals, so the state equals the row-by-row definition.
#include "pac_internal.cuh"
#include "pac_kernels.h"

namespace pacgpu {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kCap = 0xFFFFu;

__device__ __forceinline__ uint32_t lvl_total(uint32_t t, int level) {
    return __shfl_sync(kFull, t, level);
}

// level k -> k+1 (k+1 known to have room)
__device__ __forceinline__ void apx_move(ApxSide *s, uint32_t &t, int k, int lane) {
    const uint32_t tk = lvl_total(t, k);
    const uint32_t w = s->w[k][lane];
    const uint32_t add = ((w & 0xFFFFu) >> 4) | (((w >> 16) >> 4) << 16);
    s->w[k + 1][lane] += add;
    s->w[k][lane] = 0;
    if (lane == k + 1) t += tk >> 4;
    if (lane == k) t = 0;
    __syncwarp();
}

// Flush level l: the chain of levels that must move first is found on the
// totals, then the moves run from the top down.
__device__ __forceinline__ void apx_flush(ApxSide *s, uint32_t &t, int l, int lane, bool &ovf) {
    if (l == kApxLevels - 1) {
        ovf = true;
        return;
    }
    int h = l;
    while (h < kApxLevels - 2 && lvl_total(t, h + 1) + (lvl_total(t, h) >> 4) > kCap) h++;
    if (h == kApxLevels - 2 && lvl_total(t, h + 1) + (lvl_total(t, h) >> 4) > kCap) ovf = true;
    for (int k = h; k >= l; k--) apx_move(s, t, k, lane);
}

// dst (+)= src for one side; dst totals in registers, src totals in memory.
__device__ __forceinline__ void apx_combine_side(ApxSide *dst, uint32_t &t, const ApxSide *src,
                                                 int lane, bool &ovf) {
    for (int l = 0; l < kApxLevels; l++) {
        const uint32_t ts = src->t[l];
        if (ts == 0) continue;  // an empty level adds nothing and cannot trigger a flush
        if (lvl_total(t, l) + ts > kCap) apx_flush(dst, t, l, lane, ovf);
        dst->w[l][lane] += src->w[l][lane];
        if (lane == l) t += ts;
        __syncwarp();
    }
}

__device__ __forceinline__ void apx_zero(ApxState *st, int lane) {
    uint32_t *w = reinterpret_cast<uint32_t *>(st);
    for (int k = lane; k < static_cast<int>(sizeof(ApxState) / 4); k += 32) w[k] = 0;
    __syncwarp();
}

__device__ __forceinline__ void apx_store_totals(ApxState *st, uint32_t t0, uint32_t t1, int lane) {
    if (lane < kApxLevels) {
        st->side[0].t[lane] = t0;
        st->side[1].t[lane] = t1;
    }
    __syncwarp();
}

__device__ __forceinline__ void apx_combine(ApxState *dst, const ApxState *src, int lane, bool &ovf) {
    uint32_t t0 = lane < kApxLevels ? dst->side[0].t[lane] : 0;
    uint32_t t1 = lane < kApxLevels ? dst->side[1].t[lane] : 0;
    apx_combine_side(&dst->side[0], t0, &src->side[0], lane, ovf);
    apx_combine_side(&dst->side[1], t1, &src->side[1], lane, ovf);
    apx_store_totals(dst, t0, t1, lane);
}

// 32 x 32 bit transpose across a warp: lane r holds row r's 32 world bits;
// afterwards lane j holds world j's bits of the 32 rows (bit r = row r).
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        const uint32_t m = s == 16 ? 0x0000FFFFu : s == 8 ? 0x00FF00FFu : s == 4 ? 0x0F0F0F0Fu
                                  : s == 2 ? 0x33333333u : 0x55555555u;
        const uint32_t y = __shfl_xor_sync(kFull, x, s);
        x = (lane & s) ? ((x & ~m) | ((y >> s) & m)) : ((x & m) | ((y << s) & ~m));
    }
    return x;
}

// sum over rows r in the set TS (a lane's world bits of the batch, already
// restricted to the rows that count) of x_r, from the bit planes V[b] of the
// rows' units (x < 2^12): a Horner sum of popcounts.
__device__ __forceinline__ uint32_t plane_sum(uint32_t TS, const uint32_t (&V)[12]) {
    // three independent 4-plane Horner chains (more instruction-level
    // parallelism than one 12-long chain), joined at the end
    uint32_t a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
    for (int b = 3; b >= 0; b--) {
        a0 = 2 * a0 + __popc(TS & V[b]);
        a1 = 2 * a1 + __popc(TS & V[b + 4]);
        a2 = 2 * a2 + __popc(TS & V[b + 8]);
    }
    return a0 + (a1 << 4) + (a2 << 8);
}

// One side of a dense batch (rows R of the warp's batch, lane r = row r in
// row order; lane r's level lv and units x).  Between two flushes a level's
// 64 counters only grow by sum x_r * bit_j(mask_r), so the batch is cut at
// the first row whose update would overflow its level total: the rows before
// it are added level by level as plane sums, the level of that row is
// flushed (with its cascade), and the walk resumes at that row.  The flush
// decisions read exact totals, so the state equals the row-by-row
// definition.  bal: world j + 32 is the complement of world j, so its sum is
// the segment total minus world j's.
__device__ __forceinline__ void apx_side_batch(ApxSide *s, uint32_t &t, uint32_t R, int lv, uint32_t x,
                                               uint32_t Tlo, uint32_t Thi, bool bal, const uint32_t (&V)[12],
                                               int lane, bool &ovf) {
    const uint32_t me = 1u << lane;
    // inclusive prefix of x over this lane's level's rows in R; after each cut
    // the rows already added are taken out of it (so it counts from the
    // first row not yet added)
    uint32_t P = 0;
    for (uint32_t todo = R; todo;) {
        const int l = __shfl_sync(kFull, lv, __ffs(todo) - 1);
        const uint32_t Ml = __ballot_sync(kFull, lv == l) & R;
        uint32_t xv = (Ml & me) ? x : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, xv, o);
            if (lane >= o) xv += y;
        }
        if (Ml & me) P = xv;
        todo &= ~Ml;
    }
    for (;;) {
        const uint32_t tl = __shfl_sync(kFull, t, lv & 31);
        const uint32_t over = __ballot_sync(kFull, (R & me) && tl + P > kCap);
        const uint32_t pre = over ? (R & ((1u << (__ffs(over) - 1)) - 1u)) : R;
        for (uint32_t todo = pre; todo;) {
            const int l = __shfl_sync(kFull, lv, __ffs(todo) - 1);
            const uint32_t S = __ballot_sync(kFull, lv == l) & todo;
            const uint32_t tot = __shfl_sync(kFull, P, 31 - __clz(static_cast<int>(S)));
            uint32_t lo, hi;
            if (__popc(S) <= 4) {  // a few rows: broadcast them
                lo = 0;
                hi = 0;
                for (uint32_t rr = S; rr; rr &= rr - 1) {
                    const int r = __ffs(rr) - 1;
                    const uint32_t xr = __shfl_sync(kFull, x, r);
                    lo += ((Tlo >> r) & 1u) * xr;
                    hi += ((Thi >> r) & 1u) * xr;
                }
                if (bal) hi = tot - lo;
            } else {
                lo = plane_sum(Tlo & S, V);
                hi = bal ? tot - lo : plane_sum(Thi & S, V);
            }
            s->w[l][lane] += lo | (hi << 16);
            if (lane == l) t += tot;
            if (lv == l && !(pre & me)) P -= tot;  // later rows of level l count from here
            todo &= ~S;
        }
        __syncwarp();
        if (!over) break;
        apx_flush(s, t, __shfl_sync(kFull, lv, __ffs(over) - 1), lane, ovf);
        R &= ~pre;  // the overflowing row stays: its level is empty now
    }
}

// Rows of the warp's group waiting in its ring (offsets in the chunk).
constexpr int kRing = 64;

// One warp per (chunk, group).  The warp scans the chunk's group ids 32 rows
// at a time and queues the offsets of its group's rows in a ring, in row
// order; every 32 queued rows form a dense batch: lane r hashes row r, the
// masks are bit-transposed, and each side is walked with apx_side_batch.
__global__ void __launch_bounds__(32 * kApxBlockChunks, 2) k_apx_chunks(const __grid_constant__ ApxParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint16_t ring_all[kApxBlockChunks][kRing];
    ApxState *sm = reinterpret_cast<ApxState *>(smem_raw);
    const int lane = threadIdx.x & 31, ci = threadIdx.x >> 5;
    const uint32_t G = p.in.n_groups;
    // consecutive CTAs: the groups of one block of chunks (its group ids are
    // read once from HBM, then from L2)
    const uint32_t g = blockIdx.x % G;
    const uint64_t blk = blockIdx.x / G;
    const uint64_t chunk = blk * kApxBlockChunks + ci;
    ApxState *st = sm + ci;
    uint16_t *ring = ring_all[ci];
    apx_zero(st, lane);
    uint32_t t0 = 0, t1 = 0;
    bool ovf = false;
    uint64_t rows_g = 0;
    uint32_t c_lo = 0, c_hi = 0;  // this lane's COUNT of worlds lane and lane + 32 (when p.cnt)
    const bool keys_in = (p.in.in_flags & PAC_IN_MASKS) == 0;
    const bool bal = keys_in && p.in.hash_mode == PAC_HASH_BALANCED;
    const uint32_t lt = (1u << lane) - 1u;
    if (chunk < p.n_chunks) {
        const uint64_t lo = chunk * kApxChunk;
        const uint64_t hi = min(p.in.n, lo + kApxChunk);
        uint32_t head = 0, qn = 0;  // ring: rows queued at head .. head+qn-1 (mod kRing)
        // a dense batch of k queued rows (k <= 32), lane r = the r-th
        auto batch = [&](uint32_t k) {
            const bool act = static_cast<uint32_t>(lane) < k;
            const uint64_t row = lo + (act ? ring[(head + lane) & (kRing - 1)] : 0u);
            long long v = act ? row_i64(p.values, row) : 0;
            const uint64_t km = act ? __ldg(static_cast<const unsigned long long *>(p.in.km) + row) : 0ull;
            const uint64_t mask =
                keys_in ? keyed_world_mask(static_cast<long long>(km), p.in.qkey, p.in.hash_mode) : km;
            const bool valid = act && !drop_row(p.in, mask);
            rows_g += __popc(__ballot_sync(kFull, valid));
            if (!valid) v = 0;
            // (side, level, units): a = |v| goes to level l = floor((msb(a) - 8) / 4)
            // (0 below 2^8) as x = a >> 4l < 2^12
            const uint64_t a = v < 0 ? 0ull - static_cast<uint64_t>(v) : static_cast<uint64_t>(v);
            const int msb = a ? 63 - __clzll(static_cast<long long>(a)) : 0;
            const int lv = msb < 8 ? 0 : (msb - 8) >> 2;
            const uint32_t x = static_cast<uint32_t>(a >> (4 * lv));
            uint32_t V[12];
#pragma unroll
            for (int b = 0; b < 12; b++) V[b] = __ballot_sync(kFull, (x >> b) & 1u);
            const uint32_t Tlo = transpose32(valid ? static_cast<uint32_t>(mask) : 0u, lane);
            const uint32_t Thi = bal ? 0u : transpose32(valid ? static_cast<uint32_t>(mask >> 32) : 0u, lane);
            c_lo += __popc(Tlo);
            c_hi += __popc(Thi);
            const uint32_t Rp = __ballot_sync(kFull, v > 0), Rn = __ballot_sync(kFull, v < 0);
            if (Rp) apx_side_batch(&st->side[0], t0, Rp, lv, x, Tlo, Thi, bal, V, lane, ovf);
            if (Rn) apx_side_batch(&st->side[1], t1, Rn, lv, x, Tlo, Thi, bal, V, lane, ovf);
            head = (head + k) & (kRing - 1);
            qn -= k;
            __syncwarp();  // every lane has read its ring slot before the next writes
        };
        uint32_t gid_n = lo + lane < hi ? row_gid(p.in, lo + lane) : 0xFFFFFFFFu;
        for (uint64_t base = lo; base < hi; base += 32) {
            const uint32_t gid = gid_n;
            gid_n = base + 32 + lane < hi ? row_gid(p.in, base + 32 + lane) : 0xFFFFFFFFu;
            const bool in_range = base + lane < hi;
            if (in_range && gid >= G && g == 0) raise_status(p.status, kStatusBadGroup);
            const uint32_t mine = __ballot_sync(kFull, in_range && gid == g);
            if (mine & (1u << lane))
                ring[(head + qn + __popc(mine & lt)) & (kRing - 1)] = static_cast<uint16_t>(base + lane - lo);
            qn += __popc(mine);
            __syncwarp();
            if (qn >= 32) batch(32);
        }
        if (qn) batch(qn);
    }
    apx_store_totals(st, t0, t1, lane);
    if (lane == 0 && rows_g) atomicAdd(reinterpret_cast<unsigned long long *>(p.ng + g), rows_g);
    if (p.cnt) {
        if (c_lo) atomicAdd(p.cnt + static_cast<size_t>(g) * kWorlds + lane, static_cast<unsigned long long>(c_lo));
        if (c_hi) atomicAdd(p.cnt + static_cast<size_t>(g) * kWorlds + 32 + lane, static_cast<unsigned long long>(c_hi));
    }
    __syncthreads();
    // first tree levels inside the block of chunks
    for (uint32_t width = 1; width < kApxBlockChunks; width *= 2) {
        if ((ci % (2 * width)) == 0 && ci + width < kApxBlockChunks && chunk + width < p.n_chunks)
            apx_combine(st, sm + ci + width, lane, ovf);
        __syncthreads();
    }
    if (ci == 0) {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(st);
        uint32_t *dst = reinterpret_cast<uint32_t *>(p.states + static_cast<size_t>(blk) * G + g);
        for (int k = lane; k < static_cast<int>(sizeof(ApxState) / 4); k += 32) dst[k] = src[k];
    }
    if (ovf && lane == 0) raise_status(p.status, kStatusOverflow);
}

// one tree level over block states: dst = b, src = b + width, b % (2 width) == 0
__global__ void k_apx_combine_level(const __grid_constant__ ApxParams p, uint64_t n_blocks,
                                    uint64_t width) {
    const int lane = threadIdx.x & 31;
    const uint64_t wid = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint32_t G = p.in.n_groups;
    const uint64_t pair = wid / G;
    const uint32_t g = wid % G;
    const uint64_t b = pair * 2 * width;
    if (b + width >= n_blocks) return;
    bool ovf = false;
    apx_combine(p.states + b * G + g, p.states + (b + width) * G + g, lane, ovf);
    if (ovf && lane == 0) raise_status(p.status, kStatusOverflow);
}

__global__ void k_apx_emit(const __grid_constant__ ApxParams p, long long *out_sum, double *out_avg) {
    const size_t cell = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
    const uint32_t G = p.in.n_groups;
    const bool live = cell < static_cast<size_t>(G) * kWorlds;
    const uint32_t g = live ? static_cast<uint32_t>(cell / kWorlds) : 0u;
    const int j = static_cast<int>(cell % kWorlds);
    if (p.cnt) {
        // COUNT of the cascade's pass; under balanced keys world 32 + j is the
        // group's rows minus world j
        const bool bal = (p.in.in_flags & PAC_IN_MASKS) == 0 && p.in.hash_mode == PAC_HASH_BALANCED;
        const unsigned long long c =
            !live ? 0ull : (bal && j >= 32 ? p.ng[g] - p.cnt[static_cast<size_t>(g) * kWorlds + j - 32] : p.cnt[cell]);
        const unsigned orm = __ballot_sync(0xffffffffu, live && c > 0);  // 32 cells of one group per warp
        if (live) {
            if (p.count_out) p.count_out[cell] = c;
            if (p.meta && (threadIdx.x & 31) == 0) reinterpret_cast<uint32_t *>(p.meta + 2 * g + 1)[j >= 32 ? 1 : 0] = orm;
            if (p.meta && j == 0) p.meta[2 * g] = p.ng[g];
        }
    }
    if (!live) return;
    const ApxState *st = p.states + g;  // block 0 holds the tree root
    __int128 side[2] = {0, 0};
    for (int s = 0; s < 2; s++)
        for (int l = 0; l < kApxLevels; l++) {
            const uint32_t w = st->side[s].w[l][j & 31];
            const uint32_t c = j < 32 ? (w & 0xFFFFu) : (w >> 16);
            side[s] += static_cast<__int128>(c) << (4 * l);
        }
    const __int128 v = side[0] - side[1];
    const bool fits = v >= -static_cast<__int128>(0x7fffffffffffffffll) - 1 && v <= static_cast<__int128>(0x7fffffffffffffffll);
    if (!fits) raise_status(p.status, kStatusOverflow);
    if (out_sum) out_sum[cell] = fits ? static_cast<long long>(v) : (v < 0 ? (-0x7fffffffffffffffll - 1) : 0x7fffffffffffffffll);
    if (out_avg) {
        const uint64_t ng = p.ng[g];
        const double dv = i128_to_double(v);
        out_avg[cell] = ng ? 2.0 * dv / static_cast<double>(ng) : 0.0;
    }
}

}  // namespace

int apx_max_groups() { return 32; }

size_t apx_scratch_bytes(uint64_t n, uint32_t G) {
    const uint64_t n_chunks = (n + kApxChunk - 1) / kApxChunk;
    const uint64_t n_blocks = (n_chunks + kApxBlockChunks - 1) / kApxBlockChunks;
    return static_cast<size_t>(n_blocks ? n_blocks : 1) * G * sizeof(ApxState) + G * sizeof(uint64_t) +
           static_cast<size_t>(G) * kWorlds * 8 + 512;
}

cudaError_t launch_approx(const ApxParams &pin, void *out_sum, void *out_avg, cudaStream_t s,
                          int *launches) {
    ApxParams p = pin;
    const uint32_t G = p.in.n_groups;
    p.n_chunks = (p.in.n + kApxChunk - 1) / kApxChunk;
    p.chunks_per_block = kApxBlockChunks;
    const uint64_t n_blocks = (p.n_chunks + kApxBlockChunks - 1) / kApxBlockChunks;
    cudaError_t e = cudaMemsetAsync(p.ng, 0, G * sizeof(uint64_t), s);
    if (e == cudaSuccess && p.cnt) e = cudaMemsetAsync(p.cnt, 0, static_cast<size_t>(G) * kWorlds * 8, s);
    if (e != cudaSuccess) return e;
    if (n_blocks == 0) {
        // no rows: one zero state so that the emit kernel writes zeros
        e = cudaMemsetAsync(p.states, 0, G * sizeof(ApxState), s);
        if (e != cudaSuccess) return e;
    } else {
        const size_t smem = static_cast<size_t>(kApxBlockChunks) * sizeof(ApxState);
        e = cudaFuncSetAttribute(k_apx_chunks, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        k_apx_chunks<<<static_cast<unsigned>(n_blocks * G), 32 * kApxBlockChunks, smem, s>>>(p);
        (*launches)++;
        for (uint64_t width = 1; width < n_blocks; width *= 2) {
            const uint64_t pairs = (n_blocks + 2 * width - 1) / (2 * width);
            const uint64_t warps = pairs * G;
            const unsigned blocks = static_cast<unsigned>((warps * 32 + 255) / 256);
            k_apx_combine_level<<<blocks, 256, 0, s>>>(p, n_blocks, width);
            (*launches)++;
        }
    }
    const size_t cells = static_cast<size_t>(G) * kWorlds;
    k_apx_emit<<<static_cast<unsigned>((cells + 255) / 256), 256, 0, s>>>(
        p, static_cast<long long *>(out_sum), static_cast<double *>(out_avg));
    (*launches)++;
    return cudaGetLastError();
}

}  // namespace pacgpu
