// pac_hash.cu -- PU key -> 64-bit world mask (Sec. 2 "SIMD-PAC-DB", Sec. 4.2
// "PAC Hash").  Pure streaming: 8 bytes in, 8 bytes out per row.  Each thread
// moves 16-byte vectors (two keys) with a grid sized to the SM count; the
// last odd element is done by one thread.
#include "pac_internal.cuh"
#include "pac_kernels.h"

namespace pacgpu {

namespace {

__global__ void __launch_bounds__(256) k_hash_keys(const longlong2 *keys2,
                                                   ulonglong2 *masks2, size_t n2,
                                                   const long long *keys,
                                                   unsigned long long *masks, size_t n,
                                                   uint64_t qkey, int mode) {
    const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n2; i += stride) {
        const longlong2 k = __ldcs(keys2 + i);
        ulonglong2 m;
        m.x = keyed_world_mask(k.x, qkey, mode);
        m.y = keyed_world_mask(k.y, qkey, mode);
        __stcs(masks2 + i, m);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && (n & 1))
        masks[n - 1] = keyed_world_mask(keys[n - 1], qkey, mode);
}

__global__ void __launch_bounds__(256) k_hash_keys_scalar(const long long *keys,
                                                          unsigned long long *masks,
                                                          size_t n, uint64_t qkey, int mode) {
    const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n; i += stride)
        masks[i] = keyed_world_mask(keys[i], qkey, mode);
}

}  // namespace

cudaError_t launch_hash(const int64_t *keys, uint64_t *masks, size_t n, uint64_t qkey, int mode,
                        int n_sms, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int threads = 256;
    const bool aligned = (reinterpret_cast<uintptr_t>(keys) % 16 == 0) &&
                         (reinterpret_cast<uintptr_t>(masks) % 16 == 0);
    if (aligned) {
        const size_t n2 = n / 2;
        size_t blocks = (n2 + threads - 1) / threads;
        const size_t cap = static_cast<size_t>(n_sms) * 8;
        if (blocks > cap) blocks = cap;
        if (blocks == 0) blocks = 1;
        k_hash_keys<<<static_cast<unsigned>(blocks), threads, 0, s>>>(
            reinterpret_cast<const longlong2 *>(keys), reinterpret_cast<ulonglong2 *>(masks), n2,
            reinterpret_cast<const long long *>(keys), reinterpret_cast<unsigned long long *>(masks), n,
            qkey, mode);
    } else {
        size_t blocks = (n + threads - 1) / threads;
        const size_t cap = static_cast<size_t>(n_sms) * 8;
        if (blocks > cap) blocks = cap;
        k_hash_keys_scalar<<<static_cast<unsigned>(blocks), threads, 0, s>>>(
            reinterpret_cast<const long long *>(keys), reinterpret_cast<unsigned long long *>(masks), n,
            qkey, mode);
    }
    return cudaGetLastError();
}

}  // namespace pacgpu
