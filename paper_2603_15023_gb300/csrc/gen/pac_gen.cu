// pac_gen.cu -- seeded synthetic input columns on the GPU (libpacgen.so).
// Not part of the PAC method; see include/pac_gen.h for the definition the
// host-side generator in inputs.py reproduces.
#include <cuda_runtime.h>

#include "pac_gen.h"

namespace {

constexpr unsigned long long kGamma = 0x9e3779b97f4a7c15ull;

__device__ __forceinline__ unsigned long long mix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned long long draw(unsigned long long start, unsigned long long row) {
    return mix(start + (row + 1) * kGamma);
}

__global__ void k_fill_i64(long long *dst, size_t n, unsigned long long start, unsigned long long row0, long long lo,
                           unsigned long long span) {
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x)
        dst[i] = lo + static_cast<long long>(draw(start, row0 + i) % span);
}

__global__ void k_fill_u32(unsigned *dst, size_t n, unsigned long long start, unsigned long long row0,
                           unsigned long long span) {
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x)
        dst[i] = static_cast<unsigned>(draw(start, row0 + i) % span);
}

__global__ void k_fill_f32_1000(float *dst, size_t n, unsigned long long start, unsigned long long row0) {
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<size_t>(gridDim.x) * blockDim.x) {
        const double k = static_cast<double>(draw(start, row0 + i) >> 40);
        dst[i] = static_cast<float>(k * (1000.0 / 16777216.0));
    }
}

unsigned grid_for(size_t n) {
    size_t b = (n + 255) / 256;
    if (b > 152 * 32) b = 152 * 32;
    return static_cast<unsigned>(b ? b : 1);
}

unsigned long long column_start(uint64_t seed, uint64_t column) {
    unsigned long long z = seed + (column + 1) * kGamma;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

}  // namespace

extern "C" {

int pacgen_fill_i64(int64_t *dst, size_t n, uint64_t seed, uint64_t column, uint64_t row0, int64_t lo,
                    uint64_t span, void *stream) {
    if (n == 0) return 0;
    if (!dst || span == 0) return static_cast<int>(cudaErrorInvalidValue);
    k_fill_i64<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<long long *>(dst), n, column_start(seed, column), row0, lo, span);
    return static_cast<int>(cudaGetLastError());
}

int pacgen_fill_u32(uint32_t *dst, size_t n, uint64_t seed, uint64_t column, uint64_t row0, uint64_t span,
                    void *stream) {
    if (n == 0) return 0;
    if (!dst || span == 0 || span > (1ull << 32)) return static_cast<int>(cudaErrorInvalidValue);
    k_fill_u32<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(dst, n, column_start(seed, column), row0,
                                                                           span);
    return static_cast<int>(cudaGetLastError());
}

int pacgen_fill_f32_1000(float *dst, size_t n, uint64_t seed, uint64_t column, uint64_t row0, void *stream) {
    if (n == 0) return 0;
    if (!dst) return static_cast<int>(cudaErrorInvalidValue);
    k_fill_f32_1000<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(dst, n, column_start(seed, column),
                                                                                row0);
    return static_cast<int>(cudaGetLastError());
}

}  // extern "C"
