// pac_internal.cuh -- device-side building blocks of the PAC aggregation
// library: the keyed world-mask hash, the finalizer's counter-based
// generator, column accessors and the launch-parameter structs shared by the
// kernels and the C ABI layer.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "pac.h"

namespace pacgpu {

// Device status word bits (read back by pac_sync_status).
constexpr uint32_t kStatusOverflow = 1u;
constexpr uint32_t kStatusTimeout = 2u;
constexpr uint32_t kStatusBadGroup = 4u;  // a row's group id was >= n_groups (row skipped)

constexpr int kWorlds = 64;   // m = 64 possible worlds (Sec. 2 "SIMD-PAC-DB")
constexpr int kMaxSpecs = PAC_MAX_SPECS;

// ---------------------------------------------------------------------------
// Keyed world-mask hash (Sec. 2 "SIMD-PAC-DB", Sec. 4.2 "PAC Hash").
// fmix64 is MurmurHash3's 64-bit finalizer.  The PU key's engine hash is
// fmix64(key); the per-query re-hash is fmix64(engine_hash ^ K).  Balanced
// mode keeps the low 32 bits and stores their complement in the high 32, so
// every PU is in exactly 32 worlds and world j+32 is the complement of j.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t mm3_fmix64(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdull;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ull;
    x ^= x >> 33;
    return x;
}

// An int128 integer as the nearest double (ties to even), as the IEEE
// conversion defines it: within int64 the hardware conversion; beyond, the
// top 53 bits of the magnitude rounded on the bits below them, then scaled
// by a power of two (exact).
__device__ __forceinline__ double i128_to_double(__int128 x) {
    if (x >= -static_cast<__int128>(0x7fffffffffffffffll) - 1 && x <= static_cast<__int128>(0x7fffffffffffffffll))
        return static_cast<double>(static_cast<long long>(x));
    const bool neg = x < 0;
    const unsigned __int128 m = neg ? static_cast<unsigned __int128>(0) - static_cast<unsigned __int128>(x)
                                    : static_cast<unsigned __int128>(x);
    const unsigned long long hi = static_cast<unsigned long long>(m >> 64), lo = static_cast<unsigned long long>(m);
    const int msb = hi ? 127 - __clzll(static_cast<long long>(hi)) : 63 - __clzll(static_cast<long long>(lo));
    const int sh = msb - 52;  // >= 11: |x| >= 2^63
    unsigned long long mant = static_cast<unsigned long long>(m >> sh);
    const unsigned __int128 rem = m - (static_cast<unsigned __int128>(mant) << sh);
    const unsigned __int128 half = static_cast<unsigned __int128>(1) << (sh - 1);
    if (rem > half || (rem == half && (mant & 1ull))) mant++;  // mant <= 2^53: still exact
    const double d = ldexp(static_cast<double>(mant), sh);
    return neg ? -d : d;
}

__host__ __device__ __forceinline__ uint64_t keyed_world_mask(int64_t key, uint64_t qkey,
                                                              int mode) {
    const uint64_t h = mm3_fmix64(mm3_fmix64(static_cast<uint64_t>(key)) ^ qkey);
    if (mode == PAC_HASH_RAW) return h;
    const uint64_t lo = h & 0xffffffffull;
    return lo | ((lo ^ 0xffffffffull) << 32);
}

// m = 128 worlds (Sec. 2: m = 128 is possible with twice the state): two
// keyed re-hashes of one engine hash, h_a with K and h_b with K2.  Word 0
// holds worlds 0..63, word 1 worlds 64..127.  Balanced: word 0 = low 32 bits
// of h_a | low 32 bits of h_b << 32, word 1 its complement (every PU in
// exactly 64 worlds); raw: h_a and h_b.
constexpr int kWorlds128 = 128;

__host__ __device__ __forceinline__ void keyed_world_mask128(int64_t key, uint64_t k1, uint64_t k2, int mode,
                                                             uint64_t &w0, uint64_t &w1) {
    const uint64_t inner = mm3_fmix64(static_cast<uint64_t>(key));
    const uint64_t ha = mm3_fmix64(inner ^ k1), hb = mm3_fmix64(inner ^ k2);
    if (mode == PAC_HASH_RAW) {
        w0 = ha;
        w1 = hb;
        return;
    }
    w0 = (ha & 0xffffffffull) | (hb << 32);
    w1 = ~w0;
}

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea & Flood 2014) used as a counter-based generator:
// output i of the sequence started at state s is mix(s + (i+1) * gamma).
// Draw `ctr` of stream `st` = output ctr of the sequence whose start state is
// output st of SplitMix64(seed).
// ---------------------------------------------------------------------------
constexpr uint64_t kGolden = 0x9e3779b97f4a7c15ull;

__host__ __device__ __forceinline__ uint64_t splitmix_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t counter_draw(uint64_t seed, uint64_t st,
                                                          uint64_t ctr) {
    const uint64_t start = splitmix_mix(seed + (st + 1) * kGolden);
    return splitmix_mix(start + (ctr + 1) * kGolden);
}

// ---------------------------------------------------------------------------
// Launch parameters.
// ---------------------------------------------------------------------------
struct InputDev {
    const void *km;        // int64 keys or uint64 masks
    const void *gids;      // group ids or nullptr
    uint64_t qkey;
    uint64_t n;
    uint32_t in_flags;
    int32_t hash_mode;
    int32_t gid_bytes;
    uint32_t n_groups;
};

struct SpecDev {
    int32_t kind, variant, vtype, slot;  // slot: index of this spec's state
    const void *values;
    void *out;
};

__device__ __forceinline__ uint64_t row_mask(const InputDev &in, uint64_t i) {
    if (in.in_flags & PAC_IN_MASKS) return __ldg(static_cast<const unsigned long long *>(in.km) + i);
    const long long k = __ldg(static_cast<const long long *>(in.km) + i);
    return keyed_world_mask(k, in.qkey, in.hash_mode);
}

// PAC_IN_DROP_EMPTY: a row whose world mask is 0 belongs to no group.
__device__ __forceinline__ bool drop_row(const InputDev &in, uint64_t mask) {
    return (in.in_flags & PAC_IN_DROP_EMPTY) != 0 && mask == 0;
}

__device__ __forceinline__ uint32_t row_gid(const InputDev &in, uint64_t i) {
    if (!in.gids) return 0;
    switch (in.gid_bytes) {
    case 1: return __ldg(static_cast<const unsigned char *>(in.gids) + i);
    case 2: return __ldg(static_cast<const unsigned short *>(in.gids) + i);
    default: return __ldg(static_cast<const unsigned int *>(in.gids) + i);
    }
}

__device__ __forceinline__ int64_t row_i64(const void *p, uint64_t i) {
    return __ldg(static_cast<const long long *>(p) + i);
}

__device__ __forceinline__ double row_f(const void *p, int vtype, uint64_t i) {
    if (vtype == PAC_F32) return static_cast<double>(__ldg(static_cast<const float *>(p) + i));
    return __ldg(static_cast<const double *>(p) + i);
}

__device__ __forceinline__ void raise_status(uint32_t *status, uint32_t bit) {
    if (status) atomicOr(status, bit);
}

}  // namespace pacgpu
