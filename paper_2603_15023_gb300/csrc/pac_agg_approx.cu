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
// Row loop: the lanes of a 32-row batch compute their rows' side, level and
// level units in parallel; the warp then walks the group's rows in order.
// Per side, the levels of the two latest slow updates are "open": their
// counters since the last commit sit in registers (acc) and their exact
// totals in uniform registers (ct).  A row of an open level whose units still
// fit under the cap only adds to those registers; any other row commits both
// to the level state and takes the full update with its flush chain.  Every
// flush decision reads exact totals, so the state equals the row-by-row
// definition.
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

// One open level of one side (see the row loop above).
struct ApxOpen {
    uint32_t acc;  // this lane's packed counters added since the last commit
    uint32_t ct;   // the level's exact total (uniform)
    int cl;        // the level, -1 when none (uniform)
};

// Writes an open level back: counters into the level state, total into the
// lane that holds it.
__device__ __forceinline__ void apx_commit(ApxSide *s, uint32_t &t, ApxOpen &o, int lane) {
    if (o.cl >= 0) {
        s->w[o.cl][lane] += o.acc;
        if (lane == o.cl) t = o.ct;
        __syncwarp();
    }
    o.acc = 0;
    o.cl = -1;
}

// One nonzero value of one side: x units at level l, this lane's world bits.
// oa holds the latest slow update's level, ob the one before.
__device__ __forceinline__ void apx_row(ApxSide *s, uint32_t &t, ApxOpen &oa, ApxOpen &ob, int l, uint32_t x,
                                        uint32_t b0, uint32_t b1, int lane, bool &ovf) {
    const uint32_t add = x * b0 + ((x * b1) << 16);
    if (l == oa.cl && oa.ct + x <= kCap) {  // no flush: the update stays in registers
        oa.acc += add;
        oa.ct += x;
        return;
    }
    if (l == ob.cl && ob.ct + x <= kCap) {
        ob.acc += add;
        ob.ct += x;
        return;
    }
    const int keep = l == oa.cl ? ob.cl : oa.cl;  // the other recent level stays open
    apx_commit(s, t, oa, lane);
    apx_commit(s, t, ob, lane);
    if (lvl_total(t, l) + x > kCap) apx_flush(s, t, l, lane, ovf);
    oa.cl = l;
    oa.ct = lvl_total(t, l) + x;
    oa.acc = add;
    const int kb = keep != l ? keep : -1;
    const uint32_t tb = lvl_total(t, kb < 0 ? 0 : kb);
    ob.cl = kb;
    ob.ct = tb;
}

__global__ void __launch_bounds__(32 * kApxBlockChunks, 2) k_apx_chunks(const __grid_constant__ ApxParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ApxState *sm = reinterpret_cast<ApxState *>(smem_raw);
    const int lane = threadIdx.x & 31, ci = threadIdx.x >> 5;
    const uint32_t G = p.in.n_groups;
    // consecutive CTAs: the groups of one block of chunks (its group ids are
    // read once from HBM, then from L2)
    const uint32_t g = blockIdx.x % G;
    const uint64_t blk = blockIdx.x / G;
    const uint64_t chunk = blk * kApxBlockChunks + ci;
    ApxState *st = sm + ci;
    apx_zero(st, lane);
    uint32_t t0 = 0, t1 = 0;
    ApxOpen o0{0, 0, -1}, p0{0, 0, -1}, o1{0, 0, -1}, p1{0, 0, -1};
    bool ovf = false;
    uint64_t rows_g = 0;
    if (chunk < p.n_chunks) {
        const uint64_t lo = chunk * kApxChunk;
        const uint64_t hi = min(p.in.n, lo + kApxChunk);
        // loads run ahead of the row walk: group ids two batches ahead, keys
        // and values of this group's rows one batch ahead
        const bool keys_in = (p.in.in_flags & PAC_IN_MASKS) == 0;
        uint32_t gid_n1 = lo + lane < hi ? row_gid(p.in, lo + lane) : 0u;
        uint32_t gid_n2 = lo + 32 + lane < hi ? row_gid(p.in, lo + 32 + lane) : 0u;
        long long v_n1 = 0;
        uint64_t km_n1 = 0;
        if (lo + lane < hi && gid_n1 == g) {
            v_n1 = row_i64(p.values, lo + lane);
            km_n1 = __ldg(static_cast<const unsigned long long *>(p.in.km) + lo + lane);
        }
        for (uint64_t base = lo; base < hi; base += 32) {
            const uint64_t row = base + lane;
            bool valid = row < hi;
            const uint32_t gid = gid_n1;
            long long v = v_n1;
            const uint64_t km = km_n1;
            gid_n1 = gid_n2;
            v_n1 = 0;
            km_n1 = 0;
            if (row + 32 < hi && gid_n1 == g) {
                v_n1 = row_i64(p.values, row + 32);
                km_n1 = __ldg(static_cast<const unsigned long long *>(p.in.km) + row + 32);
            }
            gid_n2 = row + 64 < hi ? row_gid(p.in, row + 64) : 0u;
            uint64_t mask = 0;
            if (valid) {
                if (gid >= G && g == 0) raise_status(p.status, kStatusBadGroup);
                if (gid == g) {
                    mask = keys_in ? keyed_world_mask(static_cast<long long>(km), p.in.qkey, p.in.hash_mode) : km;
                    if (drop_row(p.in, mask)) valid = false;
                }
            }
            if (!valid || gid != g) v = 0;
            const uint32_t mine = __ballot_sync(kFull, valid && gid == g);
            rows_g += __popc(mine);
            const uint32_t todo = __ballot_sync(kFull, valid && gid == g && v != 0);
            // this lane's row as (side, level, units): a = |v| goes to level
            // l = floor((msb(a) - 8) / 4) (0 below 2^8) as a >> 4l < 2^12
            const uint64_t a = v < 0 ? 0ull - static_cast<uint64_t>(v) : static_cast<uint64_t>(v);
            const int msb = a ? 63 - __clzll(static_cast<long long>(a)) : 0;
            const int lv = msb < 8 ? 0 : (msb - 8) >> 2;
            const uint32_t pk = static_cast<uint32_t>(a >> (4 * lv)) | (static_cast<uint32_t>(lv) << 12) |
                                (v < 0 ? 1u << 17 : 0u);
            const uint32_t mlo = static_cast<uint32_t>(mask), mhi = static_cast<uint32_t>(mask >> 32);
            for (uint32_t rr = todo; rr; rr &= rr - 1) {
                const int r = __ffs(rr) - 1;
                const uint32_t q = __shfl_sync(kFull, pk, r);
                const uint32_t b0 = (__shfl_sync(kFull, mlo, r) >> lane) & 1u;
                const uint32_t b1 = (__shfl_sync(kFull, mhi, r) >> lane) & 1u;
                const uint32_t x = q & 0xFFFu;
                const int l = static_cast<int>((q >> 12) & 31u);
                if (q >> 17) apx_row(&st->side[1], t1, o1, p1, l, x, b0, b1, lane, ovf);
                else apx_row(&st->side[0], t0, o0, p0, l, x, b0, b1, lane, ovf);
            }
        }
    }
    apx_commit(&st->side[0], t0, o0, lane);
    apx_commit(&st->side[0], t0, p0, lane);
    apx_commit(&st->side[1], t1, o1, lane);
    apx_commit(&st->side[1], t1, p1, lane);
    apx_store_totals(st, t0, t1, lane);
    if (lane == 0 && rows_g) atomicAdd(reinterpret_cast<unsigned long long *>(p.ng + g), rows_g);
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
    if (cell >= static_cast<size_t>(G) * kWorlds) return;
    const uint32_t g = cell / kWorlds;
    const int j = cell % kWorlds;
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
    return static_cast<size_t>(n_blocks ? n_blocks : 1) * G * sizeof(ApxState) + G * sizeof(uint64_t);
}

cudaError_t launch_approx(const ApxParams &pin, void *out_sum, void *out_avg, cudaStream_t s,
                          int *launches) {
    ApxParams p = pin;
    const uint32_t G = p.in.n_groups;
    p.n_chunks = (p.in.n + kApxChunk - 1) / kApxChunk;
    p.chunks_per_block = kApxBlockChunks;
    const uint64_t n_blocks = (p.n_chunks + kApxBlockChunks - 1) / kApxBlockChunks;
    cudaError_t e = cudaMemsetAsync(p.ng, 0, G * sizeof(uint64_t), s);
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
