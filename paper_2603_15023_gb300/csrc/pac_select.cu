// pac_select.cu -- PAC selection (Sec. 4.2 "PAC Selection" and compiler step
// (3); Sec. 3.2 "Categorical Rewrites": pac_select and the fused
// pac_select_<cmp>).  World j of a row survives iff it was set and the row's
// column compares true with world j's operand.
//
// Each operand vector is sorted once (k_select_prep), with prefix masks over
// the sorted order: pm[k] = the worlds of the k smallest operands.  A row
// then needs two binary searches over its vector's sorted keys (lo = the
// operands below the value, hi = those not above it), and the worlds of
// every comparison are unions and differences of pm[lo], pm[hi] and pm[n]:
//   GT pm[lo]   GE pm[hi]   LT pm[n] & ~pm[hi]   LE pm[n] & ~pm[lo]
//   EQ pm[hi] & ~pm[lo]     NE ~EQ (over all 64 worlds)
// NaN operands are left out of the sorted keys (n < 64), so they satisfy
// only NE, through the complement; a NaN value satisfies only NE.  Values
// compare through an order-preserving map to uint64: int64 with the sign
// bit flipped; doubles (floats widened exactly) with -0 folded onto +0,
// negatives bit-inverted and positives with the sign bit set.
#include "pac_internal.cuh"
#include "pac_kernels.h"

namespace pacgpu {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned long long ord_i64(long long v) {
    return static_cast<unsigned long long>(v) ^ 0x8000000000000000ull;
}

__device__ __forceinline__ unsigned long long ord_f64(double v) {
    unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
    if ((b << 1) == 0) b = 0;  // -0 compares equal to +0
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// Order key of element i of a vtype column; nan is set for a NaN float.
__device__ __forceinline__ unsigned long long ord_at(const void *p, int vtype, uint64_t i, bool &nan) {
    if (vtype == PAC_I64) {
        nan = false;
        return ord_i64(__ldg(static_cast<const long long *>(p) + i));
    }
    const double v = vtype == PAC_F32 ? static_cast<double>(__ldg(static_cast<const float *>(p) + i))
                                      : __ldg(static_cast<const double *>(p) + i);
    nan = v != v;
    return ord_f64(v);
}

__device__ __forceinline__ uint32_t thr_id_at(const SelectDev &sel, uint64_t i) {
    if (!sel.thr_ids) return 0;
    switch (sel.thr_id_bytes) {
    case 1: return __ldg(static_cast<const unsigned char *>(sel.thr_ids) + i);
    case 2: return __ldg(static_cast<const unsigned short *>(sel.thr_ids) + i);
    default: return __ldg(static_cast<const unsigned int *>(sel.thr_ids) + i);
    }
}

// One warp per operand vector: lane l holds worlds l and l + 32; the rank of
// an operand is the number of non-NaN operands with a smaller key, ties
// broken by world.
__global__ void __launch_bounds__(256) k_select_prep(const SelectDev sel, SelTable *__restrict__ tabs) {
    const int lane = threadIdx.x & 31;
    const uint32_t wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t n_w = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t t = wid; t < sel.n_thr; t += n_w) {
        bool nan0, nan1;
        const unsigned long long k0 = ord_at(sel.thr, sel.vtype, static_cast<uint64_t>(t) * 64 + lane, nan0);
        const unsigned long long k1 = ord_at(sel.thr, sel.vtype, static_cast<uint64_t>(t) * 64 + lane + 32, nan1);
        const uint32_t nb0 = __ballot_sync(kFull, nan0), nb1 = __ballot_sync(kFull, nan1);
        uint32_t r0 = 0, r1 = 0;
        for (int m = 0; m < 64; m++) {
            const unsigned long long km = __shfl_sync(kFull, m < 32 ? k0 : k1, m & 31);
            const bool nm = ((m < 32 ? nb0 : nb1) >> (m & 31)) & 1u;
            if (!nm) {
                r0 += (km < k0 || (km == k0 && m < lane)) ? 1u : 0u;
                r1 += (km < k1 || (km == k1 && m < lane + 32)) ? 1u : 0u;
            }
        }
        SelTable &tab = tabs[t];
        if (!nan0) tab.key[r0] = k0;
        if (!nan1) tab.key[r1] = k1;
        // pm[k] for k = lane, lane + 32 (and 64 on lane 0): worlds of rank < k
        unsigned long long pa = 0, pb = 0, pc = 0;
        for (int m = 0; m < 64; m++) {
            const uint32_t rm = __shfl_sync(kFull, m < 32 ? r0 : r1, m & 31);
            const bool nm = ((m < 32 ? nb0 : nb1) >> (m & 31)) & 1u;
            if (nm) continue;
            const unsigned long long bit = 1ull << m;
            if (rm < static_cast<uint32_t>(lane)) pa |= bit;
            if (rm < static_cast<uint32_t>(lane + 32)) pb |= bit;
            pc |= bit;
        }
        tab.pm[lane] = pa;
        tab.pm[lane + 32] = pb;
        if (lane == 0) {
            tab.pm[64] = pc;
            tab.n_valid = 64u - __popc(nb0) - __popc(nb1);
            tab.pad = 0;
        }
    }
}

// Worlds of {j : value <cmp> operand_j} from the value's key.
__device__ __forceinline__ unsigned long long select_worlds(const SelTable &tab, int cmp, unsigned long long kv,
                                                            bool nan) {
    if (nan) return cmp == PAC_CMP_NE ? ~0ull : 0ull;
    const int n = static_cast<int>(__ldg(&tab.n_valid));
    int lo = 0, hi = 0;  // keys < kv, keys <= kv
#pragma unroll
    for (int step = 64; step; step >>= 1) {
        const int cl = lo + step, ch = hi + step;
        if (cl <= n && __ldg(&tab.key[cl - 1]) < kv) lo = cl;
        if (ch <= n && __ldg(&tab.key[ch - 1]) <= kv) hi = ch;
    }
    const unsigned long long plo = __ldg(&tab.pm[lo]), phi = __ldg(&tab.pm[hi]);
    switch (cmp) {
    case PAC_CMP_GT: return plo;
    case PAC_CMP_GE: return phi;
    case PAC_CMP_LT: return __ldg(&tab.pm[n]) & ~phi;
    case PAC_CMP_LE: return __ldg(&tab.pm[n]) & ~plo;
    case PAC_CMP_EQ: return phi & ~plo;
    default: return ~(phi & ~plo);
    }
}

__global__ void __launch_bounds__(256) k_select(const InputDev in, const SelectDev sel,
                                                const SelTable *__restrict__ tabs, unsigned long long *__restrict__ out,
                                                uint32_t *status) {
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; i < in.n; i += stride) {
        const unsigned long long km = __ldg(static_cast<const unsigned long long *>(in.km) + i);
        const uint32_t t = thr_id_at(sel, i);
        bool nan;
        const unsigned long long kv = ord_at(sel.col, sel.vtype, i, nan);
        unsigned long long keep = 0;
        if (t < sel.n_thr) {
            keep = select_worlds(tabs[t], sel.cmp, kv, nan);
        } else {
            raise_status(status, kStatusBadGroup);
        }
        const unsigned long long mask =
            (in.in_flags & PAC_IN_MASKS) ? km : keyed_world_mask(static_cast<long long>(km), in.qkey, in.hash_mode);
        out[i] = mask & keep;
    }
}

}  // namespace

cudaError_t launch_select_prep(const SelectDev &sel, SelTable *tabs, cudaStream_t s) {
    const unsigned blocks = (sel.n_thr + 7) / 8 < 1024 ? (sel.n_thr + 7) / 8 : 1024;
    k_select_prep<<<blocks, 256, 0, s>>>(sel, tabs);
    return cudaGetLastError();
}

cudaError_t launch_select(const InputDev &in, const SelectDev &sel, const SelTable *tabs, uint64_t *out,
                          uint32_t *status, int n_sms, cudaStream_t s) {
    if (in.n == 0) return cudaSuccess;
    uint64_t blocks = (in.n + 255) / 256;
    const uint64_t cap = static_cast<uint64_t>(n_sms) * 8;
    if (blocks > cap) blocks = cap;
    k_select<<<static_cast<unsigned>(blocks), 256, 0, s>>>(in, sel, tabs, reinterpret_cast<unsigned long long *>(out),
                                                           status);
    return cudaGetLastError();
}

}  // namespace pacgpu
