// pac_tc.cuh -- tcgen05 / mbarrier building blocks shared by the tensor-core
// aggregation kernels: shared-memory matrix descriptors, the E4M3 MMA, the
// digit features of the value columns and bounded mbarrier waits.
//
// Operands use the MN-major, no-swizzle canonical layout: a 128-byte core
// matrix is 8 rows (K) x 16 bytes (M or N); LBO is the stride between 8-row
// blocks, SBO = 128 the stride between 16-byte column blocks.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pacgpu {
namespace tc {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint64_t kWaitNs = 2000000000ull;  // default: a wait gives up after 2 s of wall time
constexpr uint32_t kSuspendHintNs = 20000;    // longest park of one try_wait

__host__ __device__ constexpr int round16(int x) { return (x + 15) & ~15; }

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on an mbarrier phase; false once limit_ns of wall time have
// passed.  Each try_wait may park the warp until the phase completes
// (suspend-time hint, never longer than the limit) and polls back off with
// __nanosleep, so a waiting warp takes few issue slots from the warps it is
// waiting for.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    uint32_t done = 0;
    uint32_t ns = 16;
    const uint32_t hint = limit_ns < kSuspendHintNs ? static_cast<uint32_t>(limit_ns) : kSuspendHintNs;
    uint64_t t0 = 0;  // the clock is read only once the first try has failed
    for (uint32_t it = 0;; ++it) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity), "r"(hint)
            : "memory");
        if (done) return true;
        if (it == 0) {
            t0 = global_ns();
            continue;
        }
        if (global_ns() - t0 > limit_ns) return false;
        if (it >= 8) {
            __nanosleep(ns);
            if (ns < 128) ns <<= 1;
        }
    }
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return static_cast<uint64_t>((addr >> 4) & 0x3FFFu) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
           (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// kind::f8f6f4, A = B = E4M3, D = F32, A and B MN-major, M = 64 or 128.
template <int M>
__device__ __forceinline__ uint32_t instr_desc(int n) {
    return (1u << 4) | (1u << 15) | (1u << 16) | (static_cast<uint32_t>(n >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f8(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, 1, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc));
}

// The same MMA with D's input enabled only when acc != 0: acc = 0 makes
// D = A B, overwriting what the accumulator held.
__device__ __forceinline__ void mma_f8_acc(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

// The same store with no compiler memory barrier: ordinary loads may be
// scheduled across it.  For operand stores to shared memory that nothing in
// the thread reads back; they keep their order relative to every other asm
// volatile statement (the proxy fence that publishes them among them).
__device__ __forceinline__ void sts128_unordered(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d));
}

// Operand word q (q < 8) of a 32-world block: bytes b = 0..3 are world bits
// q + 8b, each 0x00 or 0x01.  So accumulator row 4q + b of the block holds
// world q + 8b (world_of_row undoes this at read-back); two operations per
// operand word instead of a nibble-to-byte multiply.
__device__ __forceinline__ uint32_t world_bytes(uint32_t x, int q) { return (x >> q) & 0x01010101u; }
__host__ __device__ constexpr int world_of_row(int r) { return 32 * (r >> 5) + ((r & 31) >> 2) + 8 * (r & 3); }

// Digit bytes of one row.  C4 = 1: one column, feature 4+q = digit q.
// C4 = 4: up to four columns, feature 4 + 4q + c = digit q of column c.
// Word 0 holds the COUNT feature (byte 1) and three zero pad features.
template <int C4, int L>
struct Features {
    static constexpr int kN = round16(4 + L * C4);
    static constexpr int kWords = kN / 4;
    __device__ __forceinline__ static uint32_t sm_byte(long long d) {
        return d < 0 ? (0x80u | static_cast<uint32_t>(-d)) : static_cast<uint32_t>(d);
    }
    __device__ __forceinline__ static void build(long long v0, long long v1, long long v2, long long v3, bool sgn,
                                                 uint32_t *w) {
        w[0] = 1u;
#pragma unroll
        for (int k = 1; k < kWords; k++) w[k] = 0u;
        if (C4 == 1) {
            const unsigned long long u = static_cast<unsigned long long>(v0);
#pragma unroll
            for (int k = 0; k < (L + 3) / 4; k++) {
                uint32_t x = static_cast<uint32_t>(u >> (16 * k)) & 0xFFFFu;
                x = (x | (x << 8)) & 0x00FF00FFu;
                x = (x | (x << 4)) & 0x0F0F0F0Fu;
                w[1 + k] = x;
            }
            if (L % 4) w[1 + (L - 1) / 4] &= (1u << (8 * (L % 4))) - 1u;  // digits < L only
            if (sgn) {
                const int wi = 1 + (L - 1) / 4, sh = 8 * ((L - 1) % 4);
                w[wi] = (w[wi] & ~(0xFFu << sh)) | (sm_byte(v0 >> (4 * (L - 1))) << sh);
            }
        } else {
            // byte p of the four values holds digits 2p and 2p+1
#pragma unroll
            for (int p = 0; p < L / 2; p++) {
                const int h = p / 4, b = p % 4;
                const uint32_t a0 = static_cast<uint32_t>(static_cast<unsigned long long>(v0) >> (32 * h));
                const uint32_t a1 = static_cast<uint32_t>(static_cast<unsigned long long>(v1) >> (32 * h));
                const uint32_t a2 = static_cast<uint32_t>(static_cast<unsigned long long>(v2) >> (32 * h));
                const uint32_t a3 = static_cast<uint32_t>(static_cast<unsigned long long>(v3) >> (32 * h));
                const uint32_t sel = static_cast<uint32_t>(b | ((4 + b) << 4));
                const uint32_t word = __byte_perm(__byte_perm(a0, a1, sel), __byte_perm(a2, a3, sel), 0x5410);
                w[1 + 2 * p] = word & 0x0F0F0F0Fu;
                w[2 + 2 * p] = (word >> 4) & 0x0F0F0F0Fu;
            }
            if (sgn) {
                const int sh = 4 * (L - 1);
                w[L] = sm_byte(v0 >> sh) | (sm_byte(v1 >> sh) << 8) | (sm_byte(v2 >> sh) << 16) |
                       (sm_byte(v3 >> sh) << 24);
            }
        }
    }
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(bar)) : "memory");
}

}  // namespace tc
}  // namespace pacgpu
