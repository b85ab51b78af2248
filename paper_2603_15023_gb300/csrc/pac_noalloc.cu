// pac_noalloc.cu -- pac_aggregate_noalloc: the tensor-core COUNT / exact
// int64 SUM / AVG aggregation without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs under a memory pool
// which owns all device memory (a database engine's buffer manager, a
// framework's caching allocator), and code whose memory budget is fixed
// before it starts, where an allocation can fail or stall the device at the
// wrong moment.  This entry point serves them: its scratch (the tensor-core
// accumulators' digit totals and the per-group row counts) and its status
// word are file-scope __device__ arrays of fixed size, resident on every GPU
// that loads the library until the process exits.  The caller still owns and
// passes every input and output buffer.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "pac_ctx.h"
#include "pac_internal.cuh"
#include "pac_mma.h"

// Largest scratch the tensor-core path can ask for: 512 accumulator columns
// (n_groups x features per group) x 64 worlds x 8-byte totals, the per-group
// row counts and alignment: 263,168 bytes.
static constexpr size_t kNoallocScratchBytes = 512 * 64 * 8 + 1024;
static_assert(kNoallocScratchBytes >= pacgpu::kMmaMaxScratchBytes,
              "the static scratch must hold the largest query the tensor-core path serves");

// The scratch and the status word every call shares (one copy per GPU).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];
static __device__ __align__(256) unsigned int g_noalloc_status;

namespace {

constexpr int kMaxDevices = 64;

struct DeviceSlots {
    void *scratch = nullptr;
    uint32_t *status = nullptr;
    int n_sms = 0;
};
DeviceSlots g_dev[kMaxDevices];
std::mutex g_setup_mutex;

void put_err(char *err, size_t err_len, const char *fmt, ...) {
    if (!err || err_len == 0) return;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(err, err_len, fmt, ap);
    va_end(ap);
}

// Device addresses of the static arrays on the current device.  In host code
// the arrays' names are host-side stand-ins, so the addresses come from
// cudaGetSymbolAddress, once per device, with that device current.  The
// addresses are kept for the life of the process: after cudaDeviceReset the
// module is loaded again and the arrays may move, so the entry point must not
// be used across a device reset.
pac_status device_setup(int dev, DeviceSlots &out, char *err, size_t err_len) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSlots &d = g_dev[dev];
    if (!d.scratch) {
        void *scratch = nullptr, *status = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&scratch, g_noalloc_scratch);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&status, g_noalloc_status);
        int sms = 0;
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) {
            put_err(err, err_len, "device set-up failed: %s", cudaGetErrorString(e));
            return PAC_E_CUDA;
        }
        d.scratch = scratch;
        d.status = static_cast<uint32_t *>(status);
        d.n_sms = sms;
    }
    out = d;
    return PAC_OK;
}

pac_status cuda_fail(char *err, size_t err_len) {
    put_err(err, err_len, "%s", cudaGetErrorString(cudaGetLastError()));
    return PAC_E_CUDA;
}

}  // namespace

extern "C" pac_status pac_aggregate_noalloc(const pac_input *in, const pac_agg_spec *specs, int32_t n_specs,
                                            uint64_t *meta, pac_stream stream, char *err, size_t err_len) {
    if (err && err_len) err[0] = '\0';
    if (!in || !specs || n_specs < 1 || n_specs > PAC_MAX_SPECS) {
        put_err(err, err_len, "invalid input, specs or n_specs");
        return PAC_E_INVALID;
    }
    if (in->n > 0 && !in->keys_or_masks) {
        put_err(err, err_len, "keys_or_masks is NULL");
        return PAC_E_INVALID;
    }
    if ((in->in_flags != PAC_IN_KEYS && in->in_flags != PAC_IN_MASKS) ||
        (in->hash_mode != PAC_HASH_BALANCED && in->hash_mode != PAC_HASH_RAW) || in->n_groups == 0 ||
        (!in->group_ids && in->n_groups != 1 && in->n > 0) ||
        (in->group_ids && in->gid_bytes != 1 && in->gid_bytes != 2 && in->gid_bytes != 4)) {
        put_err(err, err_len, "invalid pac_input field");
        return PAC_E_INVALID;
    }
    for (int i = 0; i < n_specs; i++) {
        const pac_agg_spec &s = specs[i];
        if (!s.out || s.reserved != 0 || (s.kind != PAC_COUNT && in->n > 0 && !s.values)) {
            put_err(err, err_len, "spec %d: invalid", i);
            return PAC_E_INVALID;
        }
    }
    // the same specs and group counts are served whatever the row count
    if (!pacgpu::mma_specs_served(in->n_groups, specs, n_specs)) {
        put_err(err, err_len,
                "only COUNT and exact int64 SUM/AVG over at most 4 value columns and 8 groups are served here");
        return PAC_E_UNSUPPORTED;
    }
    const cudaStream_t st = stream;
    if (in->n == 0) {  // every output is zero
        for (int i = 0; i < n_specs; i++)
            if (cudaMemsetAsync(specs[i].out, 0, static_cast<size_t>(in->n_groups) * 64 * 8, st) != cudaSuccess)
                return cuda_fail(err, err_len);
        if (meta && cudaMemsetAsync(meta, 0, static_cast<size_t>(in->n_groups) * 16, st) != cudaSuccess)
            return cuda_fail(err, err_len);
        return cudaStreamSynchronize(st) == cudaSuccess ? PAC_OK : cuda_fail(err, err_len);
    }
    // cannot trigger with the limits above (see the static_assert); kept so
    // that a later change of those limits cannot overrun the array
    const size_t need = pacgpu::mma_scratch_bytes(in, specs, n_specs);
    if (need > kNoallocScratchBytes) {
        put_err(err, err_len, "query needs %zu bytes of scratch; the static limit is %zu", need,
                kNoallocScratchBytes);
        return PAC_E_INVALID;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        put_err(err, err_len, "no usable current device");
        return PAC_E_CUDA;
    }
    DeviceSlots d;
    pac_status ps = device_setup(dev, d, err, err_len);
    if (ps != PAC_OK) return ps;
    if (cudaMemsetAsync(d.status, 0, sizeof(uint32_t), st) != cudaSuccess) return cuda_fail(err, err_len);
    int launches = 0;
    const char *why = "";
    ps = pacgpu::mma_launch(in, specs, n_specs, meta, st, d.scratch, d.status, d.n_sms, &launches, &why);
    if (ps != PAC_OK) {
        put_err(err, err_len, "%s", why);
        return ps;
    }
    uint32_t h = 0;
    if (cudaMemcpyAsync(&h, d.status, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        put_err(err, err_len, "%s", cudaGetErrorString(cudaGetLastError()));
        return PAC_E_CUDA;
    }
    if (h & pacgpu::kStatusTimeout) {
        put_err(err, err_len, "a bounded device wait gave up; the outputs are incomplete");
        return PAC_E_TIMEOUT;
    }
    if (h & pacgpu::kStatusBadGroup) {
        put_err(err, err_len, "a group id was >= n_groups (rows skipped)");
        return PAC_E_INVALID;
    }
    if (h & pacgpu::kStatusOverflow) {
        put_err(err, err_len, "an int64 SUM did not fit and was saturated (AVG is still exact)");
        return PAC_E_OVERFLOW;
    }
    return PAC_OK;
}
