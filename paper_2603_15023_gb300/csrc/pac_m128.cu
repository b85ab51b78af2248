// pac_m128.cu -- m = 128 possible worlds (Sec. 2 "SIMD-PAC-DB": 64 worlds
// are the paper's choice; 128 are possible with twice the state, at most
// twice the cost).
//
// A PU's 128-bit membership is two 64-bit words from two keyed re-hashes of
// one engine hash (keyed_world_mask128).  The worlds of word 0 and word 1 are
// independent sets of 64 worlds, so every aggregate over 128 worlds is the
// 64-world aggregate of word 0 next to the 64-world aggregate of word 1:
//   - COUNT and exact int64 SUM/AVG over at most 8 groups run once on the
//     tensor cores with 128-row accumulator tiles (k_agg_mma<.., 128>);
//   - every other query runs the 64-world paths twice, once per mask word
//     (written planar by k_hash_split128 / k_split_words), and the two halves
//     are interleaved into the [n_groups][128] outputs.
// The release (pac_finalize128) is the chain of pac_finalize with 128
// threads.
#include <cstring>

#include "pac_ctx.h"
#include "pac_internal.cuh"
#include "pac_kernels.h"
#include "pac_mma.h"
#include "pac_validate.h"

namespace pacgpu {

namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_hash_keys128(const long long *keys, unsigned long long *masks2,
                                                            size_t n, uint64_t k1, uint64_t k2, int mode) {
    const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
        uint64_t w0, w1;
        keyed_world_mask128(__ldg(keys + i), k1, k2, mode, w0, w1);
        masks2[2 * i] = w0;
        masks2[2 * i + 1] = w1;
    }
}

// Keys -> the two mask words, planar (w0[n], w1[n]).
__global__ void __launch_bounds__(kThreads) k_hash_split128(const long long *keys, unsigned long long *w0,
                                                             unsigned long long *w1, size_t n, uint64_t k1,
                                                             uint64_t k2, int mode) {
    const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
        uint64_t a, b;
        keyed_world_mask128(__ldg(keys + i), k1, k2, mode, a, b);
        w0[i] = a;
        w1[i] = b;
    }
}

// [n][2] mask words -> planar.
__global__ void __launch_bounds__(kThreads) k_split_words(const unsigned long long *masks2, unsigned long long *w0,
                                                           unsigned long long *w1, size_t n) {
    const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
    for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n; i += stride) {
        w0[i] = __ldg(masks2 + 2 * i);
        w1[i] = __ldg(masks2 + 2 * i + 1);
    }
}

// Two [G][64] halves (8-byte results) -> [G][128]: worlds 0..63 from lo,
// 64..127 from hi.
__global__ void __launch_bounds__(kThreads) k_interleave128(const unsigned long long *lo,
                                                             const unsigned long long *hi,
                                                             unsigned long long *out, size_t G) {
    const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
    for (size_t t = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; t < G * 128; t += stride) {
        const size_t g = t >> 7, j = t & 127;
        out[t] = j < 64 ? lo[g * 64 + j] : hi[g * 64 + (j - 64)];
    }
}

// Two [G][2] {n_g, or} halves -> [G][3] {n_g, or word 0, or word 1}.
__global__ void __launch_bounds__(kThreads) k_meta128(const unsigned long long *m0, const unsigned long long *m1,
                                                       unsigned long long *meta, size_t G) {
    const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
    for (size_t g = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; g < G; g += stride) {
        meta[3 * g] = m0[2 * g];
        meta[3 * g + 1] = m0[2 * g + 1];
        meta[3 * g + 2] = m1[2 * g + 1];
    }
}

unsigned grid_for(size_t work, int n_sms) {
    size_t blocks = (work + kThreads - 1) / kThreads;
    const size_t cap = static_cast<size_t>(n_sms > 0 ? n_sms : 1) * 8;
    if (blocks > cap) blocks = cap;
    return static_cast<unsigned>(blocks ? blocks : 1);
}

bool mma128_ok(const pac_input *in, const pac_agg_spec *specs, int n_specs) {
    return in->n > 0 && !(in->in_flags & PAC_IN_DROP_EMPTY) && mma_specs_served(in->n_groups, specs, n_specs);
}

}  // namespace

}  // namespace pacgpu

using namespace pacgpu;

namespace {

// The 64-world paths once per mask word.  Workspace (ctx->m128): the planar
// mask words, then per spec two [G][64] halves, then two [G][2] metas.
pac_status aggregate128_halves(pac_ctx *ctx, const pac_input *in, uint64_t k2, const pac_agg_spec *specs,
                               int32_t n_specs, uint64_t *meta, cudaStream_t stream, int *launches) {
    const size_t n = in->n, G = in->n_groups;
    const size_t words = align_up(n * 8, 256), half = align_up(G * 64 * 8, 256), mh = align_up(G * 16, 256);
    const size_t need = 2 * words + 2 * static_cast<size_t>(n_specs) * half + 2 * mh;
    pac_status st = ensure_buffer(ctx, &ctx->m128, &ctx->m128_bytes, need);
    if (st != PAC_OK) return st;
    Carver cv(ctx->m128);
    auto *w0 = static_cast<unsigned long long *>(cv.take(n * 8));
    auto *w1 = static_cast<unsigned long long *>(cv.take(n * 8));
    unsigned long long *tmp[2][PAC_MAX_SPECS];
    for (int h = 0; h < 2; h++)
        for (int i = 0; i < n_specs; i++) tmp[h][i] = static_cast<unsigned long long *>(cv.take(G * 64 * 8));
    unsigned long long *tmeta[2];
    for (int h = 0; h < 2; h++) tmeta[h] = static_cast<unsigned long long *>(cv.take(G * 16));
    if (n > 0) {
        if (in->in_flags & PAC_IN_MASKS)
            k_split_words<<<grid_for(n, ctx->n_sms), kThreads, 0, stream>>>(
                static_cast<const unsigned long long *>(in->keys_or_masks), w0, w1, n);
        else
            k_hash_split128<<<grid_for(n, ctx->n_sms), kThreads, 0, stream>>>(
                static_cast<const long long *>(in->keys_or_masks), w0, w1, n, in->query_key, k2, in->hash_mode);
        PAC_CUDA(ctx, cudaGetLastError());
        (*launches)++;
    }
    for (int h = 0; h < 2; h++) {
        pac_input ih = *in;
        ih.keys_or_masks = h == 0 ? w0 : w1;
        ih.in_flags = PAC_IN_MASKS;
        pac_agg_spec sh[PAC_MAX_SPECS];
        for (int i = 0; i < n_specs; i++) {
            sh[i] = specs[i];
            sh[i].out = tmp[h][i];
        }
        st = aggregate_dispatch(ctx, &ih, sh, n_specs, meta ? reinterpret_cast<uint64_t *>(tmeta[h]) : nullptr, stream);
        if (st != PAC_OK) return st;
        *launches += static_cast<int>(ctx->last_launches);
    }
    for (int i = 0; i < n_specs; i++) {
        k_interleave128<<<grid_for(G * 128, ctx->n_sms), kThreads, 0, stream>>>(
            tmp[0][i], tmp[1][i], static_cast<unsigned long long *>(specs[i].out), G);
        (*launches)++;
    }
    if (meta) {
        k_meta128<<<grid_for(G, ctx->n_sms), kThreads, 0, stream>>>(tmeta[0], tmeta[1],
                                                                      reinterpret_cast<unsigned long long *>(meta), G);
        (*launches)++;
    }
    PAC_CUDA(ctx, cudaGetLastError());
    return PAC_OK;
}

}  // namespace

extern "C" {

uint64_t pac_query_key2(uint64_t seed) { return splitmix_mix((seed ^ 0x5041435f4b455921ull) + 2 * kGolden); }

pac_status pac_hash_keys128(pac_ctx *ctx, const int64_t *keys, uint64_t *masks, size_t n, uint64_t query_key,
                            uint64_t query_key2, int32_t hash_mode, pac_stream stream) {
    if (!ctx) return PAC_E_INVALID;
    if (n > 0 && (!keys || !masks)) return fail(ctx, PAC_E_INVALID, "keys/masks is NULL");
    if (hash_mode != PAC_HASH_BALANCED && hash_mode != PAC_HASH_RAW)
        return fail(ctx, PAC_E_INVALID, "hash_mode %d", hash_mode);
    if (n == 0) return PAC_OK;
    const char *k = reinterpret_cast<const char *>(keys), *m = reinterpret_cast<const char *>(masks);
    if (k < m + 16 * n && m < k + 8 * n) return fail(ctx, PAC_E_INVALID, "keys and masks overlap");
    pac_status st = bind_device(ctx);
    if (st != PAC_OK) return st;
    k_hash_keys128<<<grid_for(n, ctx->n_sms), kThreads, 0, stream>>>(
        reinterpret_cast<const long long *>(keys), reinterpret_cast<unsigned long long *>(masks), n, query_key,
        query_key2, hash_mode);
    PAC_CUDA(ctx, cudaGetLastError());
    ctx->last_launches = 1;
    return PAC_OK;
}

pac_status pac_aggregate128(pac_ctx *ctx, const pac_input *in, uint64_t query_key2, const pac_agg_spec *specs,
                            int32_t n_specs, uint64_t *meta, pac_stream stream) {
    if (!ctx) return PAC_E_INVALID;
    pac_status st = check_input(ctx, in);
    if (st != PAC_OK) return st;
    st = check_specs(ctx, in, specs, n_specs);
    if (st != PAC_OK) return st;
    if (n_specs == 0 && !meta) return fail(ctx, PAC_E_INVALID, "nothing to compute");
    if (in->in_flags & PAC_IN_DROP_EMPTY) return fail(ctx, PAC_E_UNSUPPORTED, "m = 128: PAC_IN_DROP_EMPTY");
    for (int i = 0; i < n_specs; i++)
        if (specs[i].variant != PAC_EXACT)
            return fail(ctx, PAC_E_UNSUPPORTED, "m = 128: spec %d: only exact aggregates", i);
    st = bind_device(ctx);
    if (st != PAC_OK) return st;
    const cudaStream_t s = stream;
    const size_t G = in->n_groups;
    ctx->last_launches = 0;
    if (in->n == 0) {  // every output and the metadata are zero
        for (int i = 0; i < n_specs; i++) PAC_CUDA(ctx, cudaMemsetAsync(specs[i].out, 0, G * 128 * 8, s));
        if (meta) PAC_CUDA(ctx, cudaMemsetAsync(meta, 0, G * 24, s));
        return PAC_OK;
    }
    int launches = 0;
    const int64_t want = ctx->opt_agg_path;
    if ((want == 0 || want == 2) && mma128_ok(in, specs, n_specs)) {
        st = ensure_buffer(ctx, &ctx->ws, &ctx->ws_bytes, mma_scratch_bytes(in, specs, n_specs, 128) + 1024);
        if (st != PAC_OK) return st;
        const char *why = "";
        st = mma_launch(in, specs, n_specs, meta, s, ctx->ws, ctx->d_status, ctx->n_sms, &launches, &why,
                        static_cast<uint64_t>(ctx->opt_wait_ns), 128, query_key2);
        if (st != PAC_OK) return fail(ctx, st, "%s", why);
        ctx->last_path = 2;
        ctx->last_launches = launches;
        return PAC_OK;
    }
    if (want == 2) return fail(ctx, PAC_E_UNSUPPORTED, "tensor-core path cannot serve this query");
    st = aggregate128_halves(ctx, in, query_key2, specs, n_specs, meta, s, &launches);
    ctx->last_launches = launches;
    return st;
}

pac_status pac_finalize128(pac_ctx *ctx, const pac_agg_spec *specs, int32_t n_specs, uint32_t n_groups,
                           const uint64_t *meta, uint64_t seed, double budget, int32_t mode, double *noised,
                           uint8_t *is_null, uint32_t *flags, double *posterior, pac_stream stream) {
    if (!ctx) return PAC_E_INVALID;
    FinParams p{};
    pac_status st = build_fin_params(ctx, specs, n_specs, n_groups, meta, seed, budget, mode, noised, is_null,
                                     flags, posterior, p);
    if (st != PAC_OK) return st;
    st = bind_device(ctx);
    if (st != PAC_OK) return st;
    PAC_CUDA(ctx, launch_finalize128(p, stream));
    ctx->last_launches = 1;
    return PAC_OK;
}

}  // extern "C"
