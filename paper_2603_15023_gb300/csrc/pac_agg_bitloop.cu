// pac_agg_bitloop.cu -- per-bit CUDA-core stochastic aggregation.
//
// r_j = agg{ e(t) : t in T, pu[j] = 1 } for agg in {count, sum, avg, min, max}
// (Sec. 4.2 "PAC Aggregation"), computed the way the predicated update of
// Sec. 5 ("Naive"/predication) is written: every row updates the 64 world
// states it belongs to.  On the GPU a warp owns a batch of 32 rows; lane l
// owns worlds l and l+32, and the rows of one group inside the batch are
// folded in registers before one update of the warp's private shared-memory
// state.  Each CTA writes its partial state; a merge kernel combines the CTA
// partials in CTA order (so float results are deterministic) and writes the
// typed outputs and the per-group {rows, OR-of-masks} metadata (Sec. 3.2
// "NULLs").
//
// Two variants:
//   k_bitloop_lowcard  warp-private states in shared memory (few groups);
//   k_bitloop_atomic   global-memory atomics into a [G][64] scratch (many
//                      groups; float SUM then accumulates in FP64 atomics).
#include <cfloat>
#include <climits>

#include "pac_internal.cuh"
#include "pac_kernels.h"
#include "pac_ops.cuh"

namespace pacgpu {

namespace {

constexpr unsigned kFull = 0xffffffffu;
using namespace ops;

template <int NS>
__global__ void __launch_bounds__(256) k_bitloop_lowcard(const __grid_constant__ BitloopParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
    const uint32_t G = p.in.n_groups;
    const int nq = 1 + p.n_slots;  // quantity 0 = count
    const size_t per_warp = static_cast<size_t>(nq) * G * kWorlds;
    uint64_t *st = reinterpret_cast<uint64_t *>(smem_raw) + warp * per_warp;
    uint64_t *ng_all = reinterpret_cast<uint64_t *>(smem_raw) + n_warps * per_warp;  // [warps][G]
    uint64_t *ng = ng_all + warp * G;
    // per warp, per slot: saturating sum of |v| (an exact int64 SUM needs every
    // CTA partial to fit; |partial| <= sum |v| < 2^63 guarantees it)
    unsigned long long *abssum = reinterpret_cast<unsigned long long *>(ng_all + n_warps * G);  // [warps][NS]

    for (size_t k = lane; k < per_warp; k += 32) {
        const int q = static_cast<int>(k / (static_cast<size_t>(G) * kWorlds));
        st[k] = q == 0 ? 0ull : op_identity(p.slot[q - 1].op);
    }
    for (uint32_t g = lane; g < G; g += 32) ng[g] = 0;
    __syncthreads();

    const uint64_t begin = static_cast<uint64_t>(blockIdx.x) * p.rows_per_cta;
    const uint64_t end = min(p.in.n, begin + p.rows_per_cta);
    uint64_t my_abs[NS];
#pragma unroll
    for (int s = 0; s < NS; s++) my_abs[s] = 0;

    for (uint64_t base = begin + static_cast<uint64_t>(warp) * 32; base < end;
         base += static_cast<uint64_t>(n_warps) * 32) {
        const uint64_t row = base + lane;
        bool valid = row < end;
        uint64_t mask = 0, vals[NS];
        uint32_t gid = 0;
        if (valid) {
            gid = row_gid(p.in, row);
            if (gid >= G) {  // out-of-range group id: skip the row, report it
                raise_status(p.status, kStatusBadGroup);
                valid = false;
                gid = 0;
            } else {
                mask = row_mask(p.in, row);
                if (drop_row(p.in, mask)) {
                    valid = false;
                    gid = 0;
                }
            }
        }
#pragma unroll
        for (int s = 0; s < NS; s++) {
            vals[s] = 0;
            if (s < p.n_slots && valid) {
                vals[s] = load_slot_value(p.slot[s], row);
                if (p.slot[s].op == OP_ISUM) {
                    const long long v = static_cast<long long>(vals[s]);
                    const uint64_t a = v < 0 ? 0ull - static_cast<uint64_t>(v) : static_cast<uint64_t>(v);
                    const uint64_t t = my_abs[s] + a;
                    my_abs[s] = t < a ? ~0ull : t;
                }
            }
        }
        const uint32_t mlo = static_cast<uint32_t>(mask), mhi = static_cast<uint32_t>(mask >> 32);
        uint32_t pending = __ballot_sync(kFull, valid);
        while (pending) {
            const int leader = __ffs(pending) - 1;
            const uint32_t g = __shfl_sync(kFull, gid, leader);
            const uint32_t run = __ballot_sync(kFull, valid && gid == g);
            pending &= ~run;
            uint32_t c0 = 0, c1 = 0;
            uint64_t acc[NS][2];
#pragma unroll
            for (int s = 0; s < NS; s++) {
                const uint64_t id = s < p.n_slots ? op_identity(p.slot[s].op) : 0ull;
                acc[s][0] = id;
                acc[s][1] = id;
            }
            for (uint32_t rr = run; rr; rr &= rr - 1) {
                const int r = __ffs(rr) - 1;
                const uint32_t b0 = (__shfl_sync(kFull, mlo, r) >> lane) & 1u;
                const uint32_t b1 = (__shfl_sync(kFull, mhi, r) >> lane) & 1u;
                c0 += b0;
                c1 += b1;
#pragma unroll
                for (int s = 0; s < NS; s++) {
                    if (s < p.n_slots) {
                        const uint64_t v = __shfl_sync(kFull, vals[s], r);
                        op_update(p.slot[s].op, acc[s][0], v, b0);
                        op_update(p.slot[s].op, acc[s][1], v, b1);
                    }
                }
            }
            uint64_t *cst = st + static_cast<size_t>(g) * kWorlds;
            cst[lane] += c0;
            cst[lane + 32] += c1;
#pragma unroll
            for (int s = 0; s < NS; s++) {
                if (s < p.n_slots) {
                    uint64_t *sst = st + (static_cast<size_t>(s + 1) * G + g) * kWorlds;
                    op_merge(p.slot[s].op, sst[lane], acc[s][0]);
                    op_merge(p.slot[s].op, sst[lane + 32], acc[s][1]);
                }
            }
            if (lane == 0) ng[g] += __popc(run);
        }
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

    // CTA partial: warps merged in warp order.
    uint64_t *out = static_cast<uint64_t *>(p.partials) + static_cast<size_t>(blockIdx.x) * per_warp;
    const uint64_t *st0 = reinterpret_cast<const uint64_t *>(smem_raw);
    for (size_t k = threadIdx.x; k < per_warp; k += blockDim.x) {
        const int q = static_cast<int>(k / (static_cast<size_t>(G) * kWorlds));
        uint64_t a = st0[k];
        for (int w = 1; w < n_warps; w++) {
            const uint64_t b = st0[static_cast<size_t>(w) * per_warp + k];
            if (q == 0) a += b;
            else op_merge(p.slot[q - 1].op, a, b);
        }
        out[k] = a;
    }
    uint64_t *ng_out = p.ng_partials + static_cast<size_t>(blockIdx.x) * G;
    for (uint32_t g = threadIdx.x; g < G; g += blockDim.x) {
        uint64_t a = 0;
        for (int w = 0; w < n_warps; w++) a += ng_all[w * G + g];
        ng_out[g] = a;
    }
    if (threadIdx.x < NS && threadIdx.x < p.n_slots && p.slot[threadIdx.x].op == OP_ISUM) {
        uint64_t tot = 0;
        for (int w = 0; w < n_warps; w++) {
            const uint64_t t = tot + abssum[w * NS + threadIdx.x];
            tot = t < tot ? ~0ull : t;
        }
        if (tot >= (1ull << 63)) raise_status(p.status, kStatusOverflow);
    }
}

// Global-atomic variant for many groups: one warp per 32-row batch, every
// member world updated with an atomic.
__device__ __forceinline__ long long fkey(double d) {
    long long b = __double_as_longlong(d);
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffll);
}
__device__ __forceinline__ double fkey_inv(long long k) {
    return __longlong_as_double(k >= 0 ? k : (k ^ 0x7fffffffffffffffll));
}

__device__ __forceinline__ void atomic_update(int op, uint64_t *cell, uint64_t vbits) {
    switch (op) {
    case OP_ISUM: atomicAdd(reinterpret_cast<unsigned long long *>(cell), static_cast<unsigned long long>(vbits)); break;
    case OP_FSUM_COMP: atomicAdd(reinterpret_cast<double *>(cell), static_cast<double>(__int_as_float(static_cast<int>(vbits)))); break;
    case OP_FSUM_PLAIN: atomicAdd(reinterpret_cast<float *>(cell), __int_as_float(static_cast<int>(vbits))); break;
    case OP_IMIN: atomicMin(reinterpret_cast<long long *>(cell), static_cast<long long>(vbits)); break;
    case OP_IMAX: atomicMax(reinterpret_cast<long long *>(cell), static_cast<long long>(vbits)); break;
    case OP_FMIN: atomicMin(reinterpret_cast<long long *>(cell), fkey(__longlong_as_double(static_cast<long long>(vbits)))); break;
    case OP_FMAX: atomicMax(reinterpret_cast<long long *>(cell), fkey(__longlong_as_double(static_cast<long long>(vbits)))); break;
    }
}

__device__ __forceinline__ uint64_t atomic_identity(int op) {
    switch (op) {
    case OP_IMIN: return static_cast<uint64_t>(LLONG_MAX);
    case OP_IMAX: return static_cast<uint64_t>(LLONG_MIN);
    case OP_FMIN: return static_cast<uint64_t>(LLONG_MAX);
    case OP_FMAX: return static_cast<uint64_t>(LLONG_MIN);
    default: return 0ull;
    }
}

__global__ void k_atomic_init(const __grid_constant__ BitloopParams p) {
    const uint32_t G = p.in.n_groups;
    const size_t per_q = static_cast<size_t>(G) * kWorlds;
    const size_t total = per_q * (1 + p.n_slots);
    uint64_t *st = static_cast<uint64_t *>(p.partials);
    for (size_t k = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; k < total;
         k += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const int q = static_cast<int>(k / per_q);
        st[k] = q == 0 ? 0ull : atomic_identity(p.slot[q - 1].op);
    }
    for (size_t g = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; g < G;
         g += static_cast<size_t>(gridDim.x) * blockDim.x)
        p.ng_partials[g] = 0;
}

__global__ void __launch_bounds__(256) k_bitloop_atomic(const __grid_constant__ BitloopParams p) {
    const int lane = threadIdx.x & 31;
    const uint32_t G = p.in.n_groups;
    const size_t per_q = static_cast<size_t>(G) * kWorlds;
    uint64_t *st = static_cast<uint64_t *>(p.partials);
    const uint64_t warp_global = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps_total = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
    unsigned long long my_abs = 0;
    for (uint64_t base = warp_global * 32; base < p.in.n; base += n_warps_total * 32) {
        const uint64_t row = base + lane;
        bool valid = row < p.in.n;
        uint64_t mask = 0;
        uint32_t gid = 0;
        uint64_t vals[kMaxSpecs];
        if (valid) {
            gid = row_gid(p.in, row);
            if (gid >= G) {  // out-of-range group id: skip the row, report it
                raise_status(p.status, kStatusBadGroup);
                valid = false;
                gid = 0;
            } else {
                mask = row_mask(p.in, row);
                if (drop_row(p.in, mask)) {
                    valid = false;
                    gid = 0;
                }
            }
        }
        for (int s = 0; s < p.n_slots; s++) {
            vals[s] = valid ? load_slot_value(p.slot[s], row) : 0ull;
            if (p.slot[s].op == OP_ISUM) {
                const long long v = static_cast<long long>(vals[s]);
                const unsigned long long a = v < 0 ? 0ull - static_cast<unsigned long long>(v) : static_cast<unsigned long long>(v);
                const unsigned long long t = my_abs + a;
                my_abs = t < a ? ~0ull : t;
            }
        }
        const uint32_t mlo = static_cast<uint32_t>(mask), mhi = static_cast<uint32_t>(mask >> 32);
        const uint32_t live = __ballot_sync(kFull, valid);
        for (uint32_t rr = live; rr; rr &= rr - 1) {
            const int r = __ffs(rr) - 1;
            const uint32_t g = __shfl_sync(kFull, gid, r);
            const uint32_t b0 = (__shfl_sync(kFull, mlo, r) >> lane) & 1u;
            const uint32_t b1 = (__shfl_sync(kFull, mhi, r) >> lane) & 1u;
            uint64_t *cst = st + static_cast<size_t>(g) * kWorlds;
            if (b0) atomicAdd(reinterpret_cast<unsigned long long *>(cst + lane), 1ull);
            if (b1) atomicAdd(reinterpret_cast<unsigned long long *>(cst + lane + 32), 1ull);
            for (int s = 0; s < p.n_slots; s++) {
                const uint64_t v = __shfl_sync(kFull, vals[s], r);
                uint64_t *sst = st + (static_cast<size_t>(s + 1) * G + g) * kWorlds;
                if (b0) atomic_update(p.slot[s].op, sst + lane, v);
                if (b1) atomic_update(p.slot[s].op, sst + lane + 32, v);
            }
            if (lane == 0) atomicAdd(reinterpret_cast<unsigned long long *>(p.ng_partials + g), 1ull);
        }
    }
    // int64 SUM guard: the wrapping atomics are exact while every world's sum
    // fits; the total of |v| over all rows bounds every world's sum
    for (int o = 16; o; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(kFull, my_abs, o);
        const unsigned long long u = my_abs + t;
        my_abs = u < t ? ~0ull : u;
    }
    if (lane == 0 && my_abs) {
        const unsigned long long prev = atomicAdd(p.abs_total, my_abs);
        if (prev + my_abs < prev || prev + my_abs >= (1ull << 63)) raise_status(p.status, kStatusOverflow);
    }
}

}  // namespace

// Merge of the CTA partials (lowcard) or conversion of the atomic scratch
// (n_parts = 1, atomic = true) into the typed outputs and the metadata.
__global__ void k_bitloop_merge(const __grid_constant__ BitloopParams p, int n_parts, int atomic) {
    const uint32_t G = p.in.n_groups;
    const size_t per_q = static_cast<size_t>(G) * kWorlds;
    const size_t per_part = per_q * (1 + p.n_slots);
    const uint64_t *part = static_cast<const uint64_t *>(p.partials);
    const size_t cell = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;  // (g, j)
    const bool live = cell < per_q;
    const uint32_t g = live ? static_cast<uint32_t>(cell / kWorlds) : 0;
    const int j = static_cast<int>(cell % kWorlds);

    uint64_t cnt = 0;
    if (live)
        for (int c = 0; c < n_parts; c++) cnt += part[c * per_part + cell];

    // metadata: rows and OR of masks (bit j set iff world j saw a row)
    const unsigned bal = __ballot_sync(kFull, live && cnt > 0);
    if (p.meta && live) {
        if ((threadIdx.x & 31) == 0)
            reinterpret_cast<uint32_t *>(p.meta + 2 * g + 1)[j >= 32 ? 1 : 0] = bal;
        if (j == 0) {
            uint64_t ng = 0;
            for (int c = 0; c < n_parts; c++) ng += p.ng_partials[static_cast<size_t>(c) * G + g];
            p.meta[2 * g] = ng;
        }
    }
    if (!live) return;

    for (int s = 0; s < p.n_out; s++) {
        const OutDev &o = p.outs[s];
        if (o.kind == PAC_COUNT) {
            static_cast<uint64_t *>(o.out)[cell] = cnt;
            continue;
        }
        const int op = p.slot[o.slot].op;
        const uint64_t *sp = part + static_cast<size_t>(o.slot + 1) * per_q + cell;
        if (op == OP_ISUM) {
            __int128 tot = 0;
            if (atomic) tot = static_cast<long long>(sp[0]);
            else
                for (int c = 0; c < n_parts; c++) tot += static_cast<long long>(sp[c * per_part]);
            const bool fits = tot >= static_cast<__int128>(LLONG_MIN) && tot <= static_cast<__int128>(LLONG_MAX);
            if (!fits) raise_status(p.status, kStatusOverflow);
            const long long v = fits ? static_cast<long long>(tot) : (tot < 0 ? LLONG_MIN : LLONG_MAX);
            if (o.kind == PAC_SUM) static_cast<long long *>(o.out)[cell] = v;
            else static_cast<double *>(o.out)[cell] = cnt ? i128_to_double(tot) / static_cast<double>(cnt) : 0.0;
        } else if (op == OP_FSUM_COMP || op == OP_FSUM_PLAIN) {
            double total;
            if (atomic) {
                total = op == OP_FSUM_COMP ? __longlong_as_double(static_cast<long long>(sp[0]))
                                           : static_cast<double>(__int_as_float(static_cast<int>(sp[0])));
            } else {
                uint64_t a = sp[0];
                for (int c = 1; c < n_parts; c++) op_merge(op, a, sp[c * per_part]);
                total = static_cast<double>(__int_as_float(static_cast<int>(a)));
                if (op == OP_FSUM_COMP) total += static_cast<double>(__int_as_float(static_cast<int>(a >> 32)));
            }
            if (o.kind == PAC_SUM) static_cast<double *>(o.out)[cell] = total;
            else static_cast<double *>(o.out)[cell] = cnt ? total / static_cast<double>(cnt) : 0.0;
        } else {
            uint64_t a = sp[0];
            if (!atomic)
                for (int c = 1; c < n_parts; c++) op_merge(op, a, sp[c * per_part]);
            if (op == OP_IMIN || op == OP_IMAX) {
                static_cast<long long *>(o.out)[cell] = cnt ? static_cast<long long>(a) : 0ll;
            } else {
                const double d = atomic ? fkey_inv(static_cast<long long>(a)) : __longlong_as_double(static_cast<long long>(a));
                static_cast<double *>(o.out)[cell] = cnt ? d : 0.0;
            }
        }
    }
}

int bitloop_pick_ns(int n_slots) { return n_slots <= 1 ? 1 : (n_slots <= 4 ? 4 : kMaxSpecs); }

size_t bitloop_smem_bytes(int n_warps, int n_slots, uint32_t G, int ns) {
    return static_cast<size_t>(n_warps) * (1 + n_slots) * G * kWorlds * 8 +
           static_cast<size_t>(n_warps) * G * 8 + static_cast<size_t>(n_warps) * ns * 8;
}

cudaError_t launch_bitloop_lowcard(const BitloopParams &p, int n_ctas, int n_warps, cudaStream_t s) {
    const int ns = bitloop_pick_ns(p.n_slots);
    const size_t smem = bitloop_smem_bytes(n_warps, p.n_slots, p.in.n_groups, ns);
    cudaError_t e = cudaSuccess;
    switch (ns) {
    case 1:
        e = cudaFuncSetAttribute(k_bitloop_lowcard<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e == cudaSuccess) k_bitloop_lowcard<1><<<n_ctas, n_warps * 32, smem, s>>>(p);
        break;
    case 4:
        e = cudaFuncSetAttribute(k_bitloop_lowcard<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e == cudaSuccess) k_bitloop_lowcard<4><<<n_ctas, n_warps * 32, smem, s>>>(p);
        break;
    default:
        e = cudaFuncSetAttribute(k_bitloop_lowcard<kMaxSpecs>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e == cudaSuccess) k_bitloop_lowcard<kMaxSpecs><<<n_ctas, n_warps * 32, smem, s>>>(p);
        break;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_bitloop_atomic(const BitloopParams &p, int n_ctas, cudaStream_t s) {
    k_atomic_init<<<n_ctas, 256, 0, s>>>(p);
    k_bitloop_atomic<<<n_ctas, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_bitloop_merge(const BitloopParams &p, int n_parts, bool atomic, cudaStream_t s) {
    const size_t cells = static_cast<size_t>(p.in.n_groups) * kWorlds;
    const int threads = 256;
    const unsigned blocks = static_cast<unsigned>((cells + threads - 1) / threads);
    k_bitloop_merge<<<blocks, threads, 0, s>>>(p, n_parts, atomic ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace pacgpu
