// pac_small.cu -- COUNT and exact int64 SUM / AVG of an ungrouped query in
// one launch (Sec. 4.2 "PAC Aggregation": r_j = agg{v_i : bit j of the row's
// world mask}).  For inputs too small to fill the tensor-core pipeline, whose
// cost there is per-tile latency, not bandwidth.
//
// A warp takes `batches` consecutive 32-row batches, the next batch's loads
// in flight while the current one is folded.  Per batch, lane r hashes row
// r's key, and a five-stage shuffle butterfly transposes the 32 x 32 world
// bits so that lane j holds T_j, the batch's rows in world j.  Lane j then
// adds popc(T_j) to its count and, per value column,
//   sum_b 2^b popc(T_j & V_b)    (V_b = the rows whose value has bit b)
// when the batch's values are non-negative and below 2^32, else the values
// of T_j's rows one by one.  Under balanced masks lane j keeps world j and
// the batch totals (world j+32 = total - world j); otherwise it keeps j and
// j+32.  Sums are exact: int128 in registers, int128 accumulators in shared
// and global memory (a 64-bit atomic add on the low word, its carry added to
// the high word).  A CTA folds its warps with shared-memory atomics and adds
// its fold to the global accumulators once; the last CTA to finish (a ticket
// counter) writes COUNT, SUM, AVG and meta, then clears the accumulators and
// the ticket for the next call.
#include <climits>

#include "pac_internal.cuh"
#include "pac_kernels.h"
#include "pac_small.h"
#include "pac_validate.h"

namespace pacgpu {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSmallCols = 4;
constexpr int kSmallWarps = 8;
constexpr uint32_t kMinBatches = 4;

// Global accumulators; all zero between calls.
struct SmallAcc {
    unsigned long long ticket;
    unsigned long long rows;
    unsigned long long cnt[kWorlds];
    unsigned long long sum[kSmallCols][kWorlds + 1][2];  // [64] = total over the rows; (low, high)
};

struct SmallParams {
    InputDev in;
    const long long *col[kSmallCols];
    uint32_t batches;  // 32-row batches per warp
    int32_t bal;       // balanced keyed masks: world j+32 = complement of world j (selects the kernel)
    SmallAcc *acc;
    unsigned long long *meta;  // [n_g, or mask] or null
    void *out[PAC_MAX_SPECS];
    int32_t out_kind[PAC_MAX_SPECS];
    int32_t out_col[PAC_MAX_SPECS];
    int32_t n_out;
    uint32_t *status;
};

__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const uint32_t m = s == 16 ? 0x0000FFFFu : s == 8 ? 0x00FF00FFu : s == 4 ? 0x0F0F0F0Fu : s == 2 ? 0x33333333u : 0x55555555u;
        const uint32_t o = __shfl_xor_sync(kFull, x, s);
        x = (lane & s) ? ((x & ~m) | ((o >> s) & m)) : ((x & m) | ((o << s) & ~m));
    }
    return x;
}

// (low, high) += x, exactly modulo 2^128, with two 64-bit atomics.
__device__ __forceinline__ void atomic_add_i128(unsigned long long *p, __int128 x) {
    if (x == 0) return;
    const unsigned long long lo = static_cast<unsigned long long>(x);
    const unsigned long long hi = static_cast<unsigned long long>(static_cast<unsigned __int128>(x) >> 64);
    const unsigned long long old = atomicAdd(p, lo);
    const unsigned long long carry = old + lo < old ? 1ull : 0ull;
    if (hi + carry) atomicAdd(p + 1, hi + carry);
}

__device__ __forceinline__ __int128 load_i128(const unsigned long long *p) {
    const unsigned long long lo = __ldcg(p), hi = __ldcg(p + 1);
    return static_cast<__int128>((static_cast<unsigned __int128>(hi) << 64) | lo);
}

template <int C>
struct RowLoad {
    uint32_t gid;
    unsigned long long km;
    long long v[C > 0 ? C : 1];
};

template <int C>
__device__ __forceinline__ void load_rows(const SmallParams &p, uint64_t row, RowLoad<C> &r) {
    r.gid = 0;
    r.km = 0;
#pragma unroll
    for (int c = 0; c < (C > 0 ? C : 1); c++) r.v[c] = 0;
    if (row >= p.in.n) return;
    r.gid = row_gid(p.in, row);
    r.km = __ldg(static_cast<const unsigned long long *>(p.in.km) + row);
#pragma unroll
    for (int c = 0; c < C; c++) r.v[c] = __ldg(p.col[c] + row);
}

template <int C, bool BAL>
__global__ void __launch_bounds__(kSmallWarps * 32) k_small_agg(const __grid_constant__ SmallParams p) {
    constexpr int CC = C > 0 ? C : 1;
    __shared__ unsigned long long s_cnt[kWorlds];
    __shared__ unsigned long long s_rows;
    __shared__ unsigned long long s_sum[CC][kWorlds + 1][2];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr bool bal = BAL;
    for (int k = threadIdx.x; k < kWorlds; k += blockDim.x) s_cnt[k] = 0;
    for (int k = threadIdx.x; k < CC * (kWorlds + 1) * 2; k += blockDim.x) (&s_sum[0][0][0])[k] = 0;
    if (threadIdx.x == 0) s_rows = 0;
    __syncthreads();

    uint32_t c0 = 0, c1 = 0, rows = 0;  // at most 32 per batch, batches < 2^26
    // sums of world j and of world j+32 (or, under balanced masks, of all the
    // rows): u from the bit-sliced batches (each below 2^37, so 64 bits hold
    // 2^26 batches), s from the others
    unsigned long long u0[CC], u1[CC];
    __int128 s0[CC], s1[CC];
#pragma unroll
    for (int c = 0; c < CC; c++) {
        u0[c] = u1[c] = 0;
        s0[c] = s1[c] = 0;
    }
    bool bad = false;

    const uint64_t first = (static_cast<uint64_t>(blockIdx.x) * kSmallWarps + warp) * p.batches * 32;
    RowLoad<C> nxt;
    load_rows<C>(p, first + lane, nxt);
    for (uint32_t b = 0; b < p.batches; b++) {
        const uint64_t row = first + static_cast<uint64_t>(b) * 32 + lane;
        if (row - lane >= p.in.n) break;  // warp-uniform: the batch starts past the end
        const RowLoad<C> cur = nxt;
        load_rows<C>(p, row + 32, nxt);
        bool valid = row < p.in.n;
        if (valid && cur.gid != 0) {  // one group: any other id is out of range
            bad = true;
            valid = false;
        }
        uint64_t mask = 0;
        if (valid) {
            mask = (p.in.in_flags & PAC_IN_MASKS) ? cur.km
                                                   : keyed_world_mask(static_cast<long long>(cur.km), p.in.qkey,
                                                                      p.in.hash_mode);
            if (drop_row(p.in, mask)) valid = false;
        }
        if (!valid) mask = 0;
        const uint32_t vmask = __ballot_sync(kFull, valid);
        const uint32_t T0 = transpose32(static_cast<uint32_t>(mask), lane);
        const uint32_t T1 = bal ? 0u : transpose32(static_cast<uint32_t>(mask >> 32), lane);
        c0 += __popc(T0);
        c1 += __popc(T1);
        rows += __popc(vmask);
#pragma unroll
        for (int c = 0; c < C; c++) {
            const long long v = valid ? cur.v[c] : 0;
            const uint32_t vlo = static_cast<uint32_t>(v);
            if (!__any_sync(kFull, (static_cast<unsigned long long>(v) >> 32) != 0)) {
                // non-negative values below 2^32: bit-sliced.  Horner from the
                // top bit plane down (the plane's bit is the sign of x, which
                // shifts left), in 32 bits while the planes fit (32 rows x
                // 2^26 < 2^31), above that in 64
                const uint32_t orv = __reduce_or_sync(kFull, vlo);
                const int bits = orv ? 32 - __clz(static_cast<int>(orv)) : 0;
                uint32_t x = bits ? vlo << (32 - bits) : 0u;
                unsigned long long h0 = 0, h1 = 0;
                int k = bits;
                for (; k > 26; k--) {
                    const uint32_t vb = __ballot_sync(kFull, static_cast<int>(x) < 0);
                    x <<= 1;
                    h0 = 2 * h0 + __popc(T0 & vb);
                    h1 = 2 * h1 + __popc(T1 & vb);
                }
                uint32_t p0 = 0, p1 = 0;
#pragma unroll 4
                for (; k > 0; k--) {
                    const uint32_t vb = __ballot_sync(kFull, static_cast<int>(x) < 0);
                    x <<= 1;
                    p0 = 2 * p0 + __popc(T0 & vb);
                    p1 = 2 * p1 + __popc(T1 & vb);
                }
                const int low = bits < 26 ? bits : 26;
                u0[c] += (h0 << low) + p0;
                if (bal) {
                    // the batch's total: 16-bit halves summed over the warp (each below 2^21)
                    const uint32_t t_lo = __reduce_add_sync(kFull, vlo & 0xFFFFu);
                    const uint32_t t_hi = __reduce_add_sync(kFull, vlo >> 16);
                    u1[c] += t_lo + (static_cast<unsigned long long>(t_hi) << 16);
                } else {
                    u1[c] += (h1 << low) + p1;
                }
            } else {
                for (uint32_t rr = vmask; rr; rr &= rr - 1) {
                    const int r = __ffs(rr) - 1;
                    const long long x = __shfl_sync(kFull, v, r);
                    if ((T0 >> r) & 1u) s0[c] += x;
                    if (bal || ((T1 >> r) & 1u)) s1[c] += x;
                }
            }
        }
    }
    if (__any_sync(kFull, bad) && lane == 0) raise_status(p.status, kStatusBadGroup);
#pragma unroll
    for (int c = 0; c < C; c++) {
        s0[c] += static_cast<__int128>(u0[c]);
        s1[c] += static_cast<__int128>(u1[c]);
    }

    // fold the CTA in shared memory, then add it to the global accumulators once
    atomicAdd(&s_cnt[lane], static_cast<unsigned long long>(c0));
    if (!bal) atomicAdd(&s_cnt[lane + 32], static_cast<unsigned long long>(c1));
    if (lane == 0) atomicAdd(&s_rows, static_cast<unsigned long long>(rows));
#pragma unroll
    for (int c = 0; c < C; c++) {
        atomic_add_i128(s_sum[c][lane], s0[c]);
        if (!bal) atomic_add_i128(s_sum[c][lane + 32], s1[c]);
        else if (lane == 0) atomic_add_i128(s_sum[c][kWorlds], s1[c]);
    }
    __syncthreads();
    for (int k = threadIdx.x; k <= kWorlds; k += blockDim.x) {
        if (k < kWorlds) {
            if (s_cnt[k]) atomicAdd(&p.acc->cnt[k], s_cnt[k]);
        } else if (s_rows) {
            atomicAdd(&p.acc->rows, s_rows);
        }
#pragma unroll
        for (int c = 0; c < C; c++) {
            const __int128 x = static_cast<__int128>((static_cast<unsigned __int128>(s_sum[c][k][1]) << 64) | s_sum[c][k][0]);
            atomic_add_i128(p.acc->sum[c][k], x);
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&p.acc->ticket, 1ull) == gridDim.x - 1 ? 1 : 0;
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // the last CTA: outputs of the 64 worlds (threads 0..63), then a clean slate
    if (threadIdx.x < kWorlds) {
        const int j = threadIdx.x;
        const bool derive = bal && j >= 32;
        const unsigned long long n_rows = __ldcg(&p.acc->rows);
        const unsigned long long cnt = derive ? n_rows - __ldcg(&p.acc->cnt[j - 32]) : __ldcg(&p.acc->cnt[j]);
        const unsigned ormask = __ballot_sync(kFull, cnt > 0);
        if (p.meta) {
            if (lane == 0) reinterpret_cast<uint32_t *>(p.meta + 1)[j >= 32 ? 1 : 0] = ormask;
            if (j == 0) p.meta[0] = n_rows;
        }
        for (int s = 0; s < p.n_out; s++) {
            if (p.out_kind[s] == PAC_COUNT) {
                static_cast<unsigned long long *>(p.out[s])[j] = cnt;
                continue;
            }
            const int c = p.out_col[s];
            const __int128 tot = derive ? load_i128(p.acc->sum[c][kWorlds]) - load_i128(p.acc->sum[c][j - 32])
                                        : load_i128(p.acc->sum[c][j]);
            const bool fits = tot >= static_cast<__int128>(LLONG_MIN) && tot <= static_cast<__int128>(LLONG_MAX);
            if (!fits) raise_status(p.status, kStatusOverflow);
            const long long val = fits ? static_cast<long long>(tot) : (tot < 0 ? LLONG_MIN : LLONG_MAX);
            if (p.out_kind[s] == PAC_SUM) static_cast<long long *>(p.out[s])[j] = val;
            else static_cast<double *>(p.out[s])[j] = cnt ? i128_to_double(tot) / static_cast<double>(cnt) : 0.0;
        }
    }
    __syncthreads();
    unsigned long long *w = reinterpret_cast<unsigned long long *>(p.acc);
    for (int k = threadIdx.x; k < static_cast<int>(sizeof(SmallAcc) / 8); k += blockDim.x) w[k] = 0;
}

// Distinct value columns of the specs, or -1 when a spec is not COUNT or an
// exact int64 SUM / AVG.
int small_columns(const pac_agg_spec *specs, int n_specs, const void **cols) {
    int C = 0;
    for (int i = 0; i < n_specs; i++) {
        const pac_agg_spec &s = specs[i];
        if (s.kind == PAC_COUNT) continue;
        if (!((s.kind == PAC_SUM || s.kind == PAC_AVG) && s.vtype == PAC_I64 && s.variant == PAC_EXACT)) return -1;
        int k = 0;
        while (k < C && cols[k] != s.values) k++;
        if (k == C) {
            if (C == kSmallCols) return -1;
            cols[C++] = s.values;
        }
    }
    return C;
}

}  // namespace

bool small_supported(const pac_input *in, const pac_agg_spec *specs, int n_specs) {
    const void *cols[kSmallCols];
    return in->n_groups == 1 && n_specs <= PAC_MAX_SPECS && small_columns(specs, n_specs, cols) >= 0;
}

pac_status run_small(pac_ctx *ctx, const pac_input *in, const pac_agg_spec *specs, int n_specs, uint64_t *meta,
                     cudaStream_t stream, int *launches) {
    if (!ctx->small_acc) {
        if (cudaMalloc(&ctx->small_acc, sizeof(SmallAcc)) != cudaSuccess) {
            cudaGetLastError();
            ctx->small_acc = nullptr;
            return fail(ctx, PAC_E_NOMEM, "one-launch path: %zu bytes of accumulators", sizeof(SmallAcc));
        }
        // cleared on the caller's stream, ahead of the first kernel (every
        // kernel leaves the accumulators zero again)
        PAC_CUDA(ctx, cudaMemsetAsync(ctx->small_acc, 0, sizeof(SmallAcc), stream));
    }
    SmallParams p{};
    const void *cols[kSmallCols];
    const int C = small_columns(specs, n_specs, cols);
    if (C < 0 || in->n_groups != 1) return fail(ctx, PAC_E_UNSUPPORTED, "one-launch path: unsupported query");
    p.in = make_input(in);
    for (int c = 0; c < C; c++) p.col[c] = static_cast<const long long *>(cols[c]);
    p.bal = ((in->in_flags & PAC_IN_MASKS) == 0 && in->hash_mode == PAC_HASH_BALANCED) ? 1 : 0;
    p.acc = static_cast<SmallAcc *>(ctx->small_acc);
    p.meta = reinterpret_cast<unsigned long long *>(meta);
    p.status = ctx->d_status;
    p.n_out = n_specs;
    for (int s = 0; s < n_specs; s++) {
        p.out[s] = specs[s].out;
        p.out_kind[s] = specs[s].kind;
        int k = 0;
        while (k < C && cols[k] != specs[s].values) k++;
        p.out_col[s] = specs[s].kind == PAC_COUNT ? 0 : k;
    }
    // batches per warp: enough that all warps are resident at once (32 per SM)
    const uint64_t resident = static_cast<uint64_t>(ctx->n_sms) * 32;
    const uint64_t batches_all = (in->n + 31) / 32;
    uint64_t per_warp = (batches_all + resident - 1) / resident;
    if (per_warp < kMinBatches) per_warp = kMinBatches;
    const uint64_t warps = batches_all ? (batches_all + per_warp - 1) / per_warp : 1;
    const uint64_t blocks = (warps + kSmallWarps - 1) / kSmallWarps;
    if (per_warp >= (1ull << 26) || blocks > 0x7FFFFFFFull)
        return fail(ctx, PAC_E_UNSUPPORTED, "one-launch path: %llu rows", static_cast<unsigned long long>(in->n));
    p.batches = static_cast<uint32_t>(per_warp);
    const dim3 grid(static_cast<unsigned>(blocks)), block(kSmallWarps * 32);
    const bool bal = p.bal != 0;
    switch (C) {
    case 0: bal ? k_small_agg<0, true><<<grid, block, 0, stream>>>(p) : k_small_agg<0, false><<<grid, block, 0, stream>>>(p); break;
    case 1: bal ? k_small_agg<1, true><<<grid, block, 0, stream>>>(p) : k_small_agg<1, false><<<grid, block, 0, stream>>>(p); break;
    case 2: bal ? k_small_agg<2, true><<<grid, block, 0, stream>>>(p) : k_small_agg<2, false><<<grid, block, 0, stream>>>(p); break;
    case 3: bal ? k_small_agg<3, true><<<grid, block, 0, stream>>>(p) : k_small_agg<3, false><<<grid, block, 0, stream>>>(p); break;
    default: bal ? k_small_agg<4, true><<<grid, block, 0, stream>>>(p) : k_small_agg<4, false><<<grid, block, 0, stream>>>(p); break;
    }
    PAC_CUDA(ctx, cudaGetLastError());
    (*launches)++;
    ctx->last_path = 4;
    return PAC_OK;
}

}  // namespace pacgpu
