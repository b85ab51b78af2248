// pac_ctx.h -- the context object behind the C ABI and the helpers the
// entry points share (error recording, workspace growth, buffer carving).
#pragma once

#include <cstdarg>
#include <cstdio>
#include <string>

#include "pac_internal.cuh"

struct pac_ctx {
    int device = 0;
    int n_sms = 0;
    void *ws = nullptr;  // aggregation scratch
    size_t ws_bytes = 0;
    void *qws = nullptr;  // pac_query_host staging (inputs and outputs)
    size_t qws_bytes = 0;
    void *sws = nullptr;  // selection: sorted operand tables, selected masks
    size_t sws_bytes = 0;
    void *small_acc = nullptr;  // one-launch path: accumulators, zero between calls
    void *m128 = nullptr;  // m = 128: mask words and the two 64-world halves
    size_t m128_bytes = 0;
    uint32_t *d_status = nullptr;
    void *pin = nullptr;  // pinned staging of per-bit engine descriptors
    size_t pin_bytes = 0;
    cudaEvent_t pin_ev = nullptr;  // the last copy out of `pin`
    int64_t opt_agg_path = 0;
    int64_t opt_minmax_prune = 1;
    int64_t opt_wait_ns = 0;  // tensor-core pipeline wait limit (0: default 2 s)
    int64_t last_path = 0;
    int64_t last_launches = 0;
    std::string last_error;
};

inline pac_status fail(pac_ctx *ctx, pac_status st, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->last_error = buf;
    }
    return st;
}

inline pac_status cuda_fail(pac_ctx *ctx, cudaError_t e, const char *where) {
    return fail(ctx, PAC_E_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define PAC_CUDA(ctx, call)                                   \
    do {                                                      \
        cudaError_t e__ = (call);                             \
        if (e__ != cudaSuccess) return cuda_fail(ctx, e__, #call); \
    } while (0)

inline pac_status bind_device(pac_ctx *ctx) {
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    return PAC_OK;
}

// Grows a device buffer; freeing the old one synchronises the device, so no
// kernel still reads it.
inline pac_status ensure_buffer(pac_ctx *ctx, void **buf, size_t *have, size_t need) {
    if (need <= *have) return PAC_OK;
    if (*buf) {
        cudaFree(*buf);
        *buf = nullptr;
        *have = 0;
    }
    size_t want = need + need / 4 + (1u << 20);
    cudaError_t e = cudaMalloc(buf, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *buf = nullptr;
        return fail(ctx, PAC_E_NOMEM, "cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
    }
    *have = want;
    return PAC_OK;
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base(static_cast<char *>(b)) {}
    void *take(size_t bytes) {
        off = align_up(off, 256);
        void *p = base + off;
        off += bytes;
        return p;
    }
};

