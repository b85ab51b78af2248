/*
 * pac_gen.h -- seeded synthetic input columns generated on the GPU
 * (libpacgen.so).  Not part of the PAC method: these fill benchmark and test
 * columns too large to draw on the host.  The same columns are reproduced
 * on the host by paper_2603_15023_gb300/inputs.py (counter_u64 and the
 * mappings below), so the CPU oracle can check any sampled query.
 *
 * Draw `row` of column `column` under `seed` (a counter-based generator,
 * SplitMix64 of Steele, Lea & Flood 2014 used with explicit counters):
 *   start = mix(seed + (column + 1) * G),  u = mix(start + (row + 1) * G),
 *   G = 0x9e3779b97f4a7c15, mix = SplitMix64's output function.
 * Mappings (row0 + i is the row of element i):
 *   pacgen_fill_i64:   dst[i] = lo + (int64)(u % span)          (span >= 1)
 *   pacgen_fill_u32:   dst[i] = (uint32)(u % span)              (1 <= span <= 2^32)
 *   pacgen_fill_f32_1000: dst[i] = (float)((u >> 40) * 1000 / 2^24), uniform
 *                      on [0, 1000) with 24-bit resolution (the product is
 *                      exact in double, rounded once to float).
 * dst is a DEVICE pointer; work is enqueued on `stream` (a cudaStream_t).
 * Returns 0, or a CUDA error code (no error is raised for n = 0).
 */
#ifndef PAC_GEN_H
#define PAC_GEN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

int pacgen_fill_i64(int64_t *dst, size_t n, uint64_t seed, uint64_t column, uint64_t row0, int64_t lo,
                    uint64_t span, void *stream);
int pacgen_fill_u32(uint32_t *dst, size_t n, uint64_t seed, uint64_t column, uint64_t row0, uint64_t span,
                    void *stream);
int pacgen_fill_f32_1000(float *dst, size_t n, uint64_t seed, uint64_t column, uint64_t row0, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PAC_GEN_H */
