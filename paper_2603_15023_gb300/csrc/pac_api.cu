// pac_api.cu -- the C ABI (include/pac.h): argument checking, path choice,
// context-owned workspace and the launches of the PAC kernels.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "pac_ctx.h"
#include "pac_internal.cuh"
#include "pac_kernels.h"
#include "pac_mma.h"
#include "pac_part_mma.h"
#include "pac_small.h"
#include "pac_validate.h"
#include "pac_batch.h"

using namespace pacgpu;

namespace {

pac_status run_bitloop(pac_ctx *ctx, const pac_input *in, const pac_agg_spec *specs, int32_t n_specs,
                       uint64_t *meta, cudaStream_t stream, int *launches) {
    BitloopParams p{};
    p.in = make_input(in);
    p.meta = meta;
    p.status = ctx->d_status;
    // one state slot per distinct (op, column)
    int slot_of[PAC_MAX_SPECS];
    for (int i = 0; i < n_specs; i++) {
        slot_of[i] = -1;
        const int op = spec_op(specs[i]);
        if (op < 0) continue;
        for (int k = 0; k < p.n_slots; k++)
            if (p.slot[k].op == op && p.slot[k].values == specs[i].values && p.slot[k].vtype == specs[i].vtype)
                slot_of[i] = k;
        if (slot_of[i] < 0) {
            p.slot[p.n_slots].op = op;
            p.slot[p.n_slots].vtype = specs[i].vtype;
            p.slot[p.n_slots].values = specs[i].values;
            slot_of[i] = p.n_slots++;
        }
    }
    for (int i = 0; i < n_specs; i++) {
        if (spec_is_cascade(specs[i])) continue;
        p.outs[p.n_out].kind = specs[i].kind;
        p.outs[p.n_out].slot = slot_of[i];
        p.outs[p.n_out].out = specs[i].out;
        p.n_out++;
    }
    const uint32_t G = in->n_groups;
    const int ns = bitloop_pick_ns(p.n_slots);
    int n_warps = 8;
    while (n_warps > 1 && bitloop_smem_bytes(n_warps, p.n_slots, G, ns) > 200 * 1024) n_warps /= 2;
    const bool lowcard = bitloop_smem_bytes(n_warps, p.n_slots, G, ns) <= 200 * 1024;
    const size_t per_part = static_cast<size_t>(1 + p.n_slots) * G * kWorlds * 8;
    if (lowcard) {
        const int ctas_per_sm = n_warps >= 8 ? 2 : 4;
        uint64_t n_ctas = static_cast<uint64_t>(ctx->n_sms) * ctas_per_sm;
        const uint64_t min_rows = 4096;
        if (in->n / min_rows < n_ctas) n_ctas = in->n / min_rows;
        if (n_ctas < 1) n_ctas = 1;
        p.rows_per_cta = (in->n + n_ctas - 1) / n_ctas;
        p.rows_per_cta = align_up(p.rows_per_cta, 32);
        if (p.rows_per_cta == 0) p.rows_per_cta = 32;
        n_ctas = (in->n + p.rows_per_cta - 1) / p.rows_per_cta;
        if (n_ctas < 1) n_ctas = 1;
        const size_t need = n_ctas * per_part + 256 + n_ctas * G * 8 + 256;
        pac_status st = ensure_buffer(ctx, &ctx->ws, &ctx->ws_bytes, need);
        if (st != PAC_OK) return st;
        Carver cv(ctx->ws);
        p.partials = cv.take(n_ctas * per_part);
        p.ng_partials = static_cast<uint64_t *>(cv.take(n_ctas * G * 8));
        PAC_CUDA(ctx, launch_bitloop_lowcard(p, static_cast<int>(n_ctas), n_warps, stream));
        PAC_CUDA(ctx, launch_bitloop_merge(p, static_cast<int>(n_ctas), false, stream));
        *launches += 2;
    } else {
        const size_t need = per_part + 256 + G * 8 + 256 + 256;
        pac_status st = ensure_buffer(ctx, &ctx->ws, &ctx->ws_bytes, need);
        if (st != PAC_OK) return st;
        Carver cv(ctx->ws);
        p.partials = cv.take(per_part);
        p.ng_partials = static_cast<uint64_t *>(cv.take(G * 8));
        p.abs_total = static_cast<unsigned long long *>(cv.take(8));
        PAC_CUDA(ctx, cudaMemsetAsync(p.abs_total, 0, 8, stream));
        int n_ctas = ctx->n_sms * 8;
        PAC_CUDA(ctx, launch_bitloop_atomic(p, n_ctas, stream));
        PAC_CUDA(ctx, launch_bitloop_merge(p, 1, true, stream));
        *launches += 3;
    }
    ctx->last_path = 1;
    return PAC_OK;
}

// The per-bit engine of the batched path (warp bit-transpose, warp-private
// or atomic states) on one query: a one-query plan placed in the context's
// workspace, its descriptors staged in pinned memory.
// tensor: the many-group tensor-core path instead -- the same plan, ending
// with the partition, then the tensor-core kernel over the group-ordered
// copies (its partial records placed after the plan in the workspace).
pac_status run_engine(pac_ctx *ctx, const pac_input *in, const pac_agg_spec *specs, int32_t n_specs,
                      uint64_t *meta, cudaStream_t stream, int *launches, bool tensor = false) {
    pac_agg_spec kept[PAC_MAX_SPECS];
    int k = 0;
    for (int i = 0; i < n_specs; i++)
        if (!spec_is_cascade(specs[i])) kept[k++] = specs[i];
    if (k == 0 && !meta) return PAC_OK;
    pac_query q{};
    q.in = *in;
    q.specs = kept;
    q.n_specs = k;
    q.fin_mode = -1;
    q.meta = meta;
    // one query: work items small enough that every SM gets a few (a
    // power of two from 4K rows up to the default size), and no more than
    // 2048 of them, since the merge reads one partial state per item
    BatchConfig cfg = kBatchDefault;
    const uint64_t per_slot = in->n / (static_cast<uint64_t>(ctx->n_sms) * 4);
    uint32_t rows = 4096;
    while (rows < per_slot && rows < cfg.item_rows) rows <<= 1;
    while (in->n / rows > 2048 && rows < (1u << 30)) rows <<= 1;
    cfg.item_rows = rows;
    cfg.partition_only = tensor;
    pac_batch *b = nullptr;
    pac_status st = plan_build(ctx, &q, 1, cfg, &b);
    if (st != PAC_OK) return st;
    const size_t part_off = align_up(b->device_bytes, 256);
    st = ensure_buffer(ctx, &ctx->ws, &ctx->ws_bytes,
                       tensor ? part_off + part_mma_scratch_bytes(in->n, in->n_groups, ctx->n_sms) : b->device_bytes);
    if (st == PAC_OK && ctx->pin_bytes < b->image.size()) {
        if (ctx->pin) {
            cudaEventSynchronize(ctx->pin_ev);
            cudaFreeHost(ctx->pin);
            ctx->pin = nullptr;
        }
        ctx->pin_bytes = 0;
        const size_t want = b->image.size() * 2 + 4096;
        if (cudaMallocHost(&ctx->pin, want) != cudaSuccess) {
            cudaGetLastError();
            st = fail(ctx, PAC_E_NOMEM, "pinned staging of %zu bytes", want);
        } else {
            ctx->pin_bytes = want;
        }
    }
    if (st == PAC_OK && !ctx->pin_ev && cudaEventCreateWithFlags(&ctx->pin_ev, cudaEventDisableTiming) != cudaSuccess)
        st = fail(ctx, PAC_E_CUDA, "event");
    if (st != PAC_OK) {
        plan_destroy(b);
        return st;
    }
    cudaEventSynchronize(ctx->pin_ev);  // the previous copy out of the staging is done
    plan_bind(b, ctx->ws);
    b->d_status = ctx->d_status;
    std::memcpy(ctx->pin, b->image.data(), b->image.size());
    st = plan_setup_kernel(ctx, b);
    if (st == PAC_OK) st = plan_enqueue(ctx, b, stream, ctx->pin);
    if (st == PAC_OK && cudaEventRecord(ctx->pin_ev, stream) != cudaSuccess) st = fail(ctx, PAC_E_CUDA, "event record");
    const bool b_atomic = b->n_atomic > 0;
    const int n_wide = b->n_wide;
    if (st == PAC_OK && tensor) {
        char *base = static_cast<char *>(ctx->ws);
        PartMmaArgs a{};
        a.in = make_input(in);
        a.rec = base + b->rel_smask[0];
        a.sgid = reinterpret_cast<const uint32_t *>(base + b->rel_sgid[0]);
        a.pcnt = reinterpret_cast<const uint32_t *>(base + b->rel_pcnt[0]);
        a.pend = reinterpret_cast<const uint32_t *>(base + b->rel_pcur[0]);
        // the plan packs the group id into the records under balanced keys
        a.packed = ((in->in_flags & PAC_IN_MASKS) == 0 && in->hash_mode == PAC_HASH_BALANCED) ? 1 : 0;
        a.specs = kept;
        a.n_specs = k;
        a.meta = meta;
        a.scratch = base + part_off;
        a.status = ctx->d_status;
        a.n_sms = ctx->n_sms;
        a.wait_ns = static_cast<uint64_t>(ctx->opt_wait_ns);
        const char *why = "";
        st = part_mma_launch(a, stream, launches, &why);
        if (st != PAC_OK) st = fail(ctx, st, "many-group tensor-core path: %s", why);
    }
    plan_destroy(b);
    if (st != PAC_OK) return st;
    if (tensor) {
        *launches += 3 + 2 * n_wide;  // histogram, scan, scatter (+ the wide scan)
        ctx->last_path = 5;
    } else {
        *launches += 2 + (b_atomic ? 3 : 0) + 2 * n_wide;
        ctx->last_path = 3;
    }
    return PAC_OK;
}

// counts / n_counts / meta: COUNT specs and the metadata, produced by the
// first cascade's pass (n_counts = 0 and meta = NULL: none).
pac_status run_cascades(pac_ctx *ctx, const pac_input *in, const pac_agg_spec *specs, int32_t n_specs,
                        cudaStream_t stream, int *launches, const pac_agg_spec *counts = nullptr,
                        int n_counts = 0, uint64_t *meta = nullptr) {
    bool first = true;
    for (int i = 0; i < n_specs; i++) {
        if (!spec_is_cascade(specs[i])) continue;
        // one cascade per distinct column serves its SUM and AVG specs
        bool seen = false;
        for (int k = 0; k < i; k++)
            if (spec_is_cascade(specs[k]) && specs[k].values == specs[i].values) seen = true;
        if (seen) continue;
        int first_sum = -1, first_avg = -1;
        for (int k = i; k < n_specs; k++) {
            if (!spec_is_cascade(specs[k]) || specs[k].values != specs[i].values) continue;
            if (specs[k].kind == PAC_SUM && first_sum < 0) first_sum = k;
            if (specs[k].kind == PAC_AVG && first_avg < 0) first_avg = k;
        }
        ApxParams p{};
        p.in = make_input(in);
        p.values = static_cast<const int64_t *>(specs[i].values);
        p.status = ctx->d_status;
        const size_t states = apx_scratch_bytes(in->n, in->n_groups);
        pac_status st = ensure_buffer(ctx, &ctx->ws, &ctx->ws_bytes, states + 1024);
        if (st != PAC_OK) return st;
        Carver cv(ctx->ws);
        p.ng = static_cast<uint64_t *>(cv.take(in->n_groups * sizeof(uint64_t)));
        if (first && (n_counts > 0 || meta)) {
            p.cnt = static_cast<unsigned long long *>(cv.take(static_cast<size_t>(in->n_groups) * kWorlds * 8));
            p.count_out = n_counts > 0 ? static_cast<unsigned long long *>(counts[0].out) : nullptr;
            p.meta = meta;
        }
        p.states = static_cast<ApxState *>(cv.take(states));
        PAC_CUDA(ctx, launch_approx(p, first_sum >= 0 ? specs[first_sum].out : nullptr,
                                    first_avg >= 0 ? specs[first_avg].out : nullptr, stream, launches));
        // further output buffers for the same (column, kind) get a copy
        for (int k = i; k < n_specs; k++) {
            if (!spec_is_cascade(specs[k]) || specs[k].values != specs[i].values) continue;
            if (k == first_sum || k == first_avg) continue;
            const void *src = specs[specs[k].kind == PAC_SUM ? first_sum : first_avg].out;
            PAC_CUDA(ctx, cudaMemcpyAsync(specs[k].out, src, static_cast<size_t>(in->n_groups) * kWorlds * 8,
                                          cudaMemcpyDeviceToDevice, stream));
        }
        if (first)
            for (int k = 1; k < n_counts; k++)
                PAC_CUDA(ctx, cudaMemcpyAsync(counts[k].out, counts[0].out, static_cast<size_t>(in->n_groups) * kWorlds * 8,
                                              cudaMemcpyDeviceToDevice, stream));
        first = false;
    }
    return PAC_OK;
}

pac_status aggregate_impl(pac_ctx *ctx, const pac_input *in, const pac_agg_spec *specs, int32_t n_specs,
                          uint64_t *meta, cudaStream_t stream) {
    int launches = 0;
    pac_status st;
    ctx->last_launches = 0;
    // The tensor-core path serves COUNT and exact int64 SUM/AVG over few
    // groups, the one-launch path the same specs of small ungrouped queries;
    // the per-bit engine serves everything else; agg_path 1 forces the plain
    // per-bit kernels (the baseline the other paths are measured against).
    // The approximate integer SUM/AVG specs run their own cascades (below);
    // the path is chosen on the other specs, which also write meta.
    pac_agg_spec ex[PAC_MAX_SPECS];
    int32_t n_ex = 0;
    for (int i = 0; i < n_specs; i++)
        if (!spec_is_cascade(specs[i])) ex[n_ex++] = specs[i];
    bool only_counts = true;
    for (int i = 0; i < n_ex; i++) only_counts = only_counts && ex[i].kind == PAC_COUNT;
    if (n_ex < n_specs && only_counts && ctx->opt_agg_path == 0) {
        // COUNT and meta come out of the first cascade's pass over the rows
        st = run_cascades(ctx, in, specs, n_specs, stream, &launches, ex, n_ex, meta);
        if (st != PAC_OK) return st;
        ctx->last_launches = launches;
        return PAC_OK;
    }
    const int want = static_cast<int>(ctx->opt_agg_path);
    const bool small_ok = (want == 0 || want == 4) && n_ex > 0 && small_supported(in, ex, n_ex) &&
                          (want == 4 || in->n <= kSmallAutoRows);
    if (want == 4 && !small_ok) return fail(ctx, PAC_E_UNSUPPORTED, "one-launch path cannot serve this query");
    bool mma_ok = !small_ok && (want == 0 || want == 2) && mma_supported(in, ex, n_ex);
    if (want == 2 && !mma_ok) return fail(ctx, PAC_E_UNSUPPORTED, "tensor-core path cannot serve this query");
    // many groups: the partition and the tensor cores over the group-ordered rows
    const bool part_ok = !small_ok && !mma_ok && (want == 0 || want == 5) && in->n > 0 && n_ex > 0 &&
                         (want == 5 || in->n_groups > kPartMmaAutoGroups) && part_mma_specs_served(ex, n_ex);
    if (want == 5 && !part_ok)
        return fail(ctx, PAC_E_UNSUPPORTED, "many-group tensor-core path cannot serve this query");
    if (small_ok) {
        st = run_small(ctx, in, ex, n_ex, meta, stream, &launches);
        if (st != PAC_OK) return st;
    } else if (mma_ok) {
        st = run_mma(ctx, in, ex, n_ex, meta, stream, &launches);
        if (st != PAC_OK) return st;
        ctx->last_path = 2;
    } else if (part_ok) {
        st = run_engine(ctx, in, ex, n_ex, meta, stream, &launches, true);
        if (st != PAC_OK) return st;
    } else if (want == 1) {
        st = run_bitloop(ctx, in, ex, n_ex, meta, stream, &launches);
        if (st != PAC_OK) return st;
    } else {
        st = run_engine(ctx, in, ex, n_ex, meta, stream, &launches);
        if (st != PAC_OK) return st;
    }
    st = run_cascades(ctx, in, specs, n_specs, stream, &launches);
    if (st != PAC_OK) return st;
    ctx->last_launches = launches;
    return PAC_OK;
}

pac_status check_select(pac_ctx *ctx, const pac_input *in, const pac_select_spec *sel) {
    if (!sel) return fail(ctx, PAC_E_INVALID, "select spec is NULL");
    if (in->n > 0 && !sel->col) return fail(ctx, PAC_E_INVALID, "select column is NULL");
    if (sel->vtype != PAC_I64 && sel->vtype != PAC_F32 && sel->vtype != PAC_F64)
        return fail(ctx, PAC_E_INVALID, "select vtype %d", sel->vtype);
    if (sel->cmp < PAC_CMP_LT || sel->cmp > PAC_CMP_GE) return fail(ctx, PAC_E_INVALID, "select cmp %d", sel->cmp);
    if (!sel->thr || sel->n_thr == 0) return fail(ctx, PAC_E_INVALID, "select operands missing");
    if (!sel->thr_ids && sel->n_thr != 1)
        return fail(ctx, PAC_E_INVALID, "n_thr %u operand vectors need thr_ids", sel->n_thr);
    if (sel->thr_ids && sel->thr_id_bytes != 1 && sel->thr_id_bytes != 2 && sel->thr_id_bytes != 4)
        return fail(ctx, PAC_E_INVALID, "thr_id_bytes %d", sel->thr_id_bytes);
    return PAC_OK;
}

// Sorted operand tables, then the selected masks of every row into `out`
// (two launches).  The tables go to the start of ctx->sws.
pac_status run_select(pac_ctx *ctx, const pac_input *in, const pac_select_spec *sel, uint64_t *out,
                      cudaStream_t stream) {
    SelectDev d;
    d.col = sel->col;
    d.thr = sel->thr;
    d.thr_ids = sel->thr_ids;
    d.vtype = sel->vtype;
    d.cmp = sel->cmp;
    d.thr_id_bytes = sel->thr_ids ? sel->thr_id_bytes : 0;
    d.n_thr = sel->n_thr;
    SelTable *tabs = static_cast<SelTable *>(ctx->sws);
    PAC_CUDA(ctx, launch_select_prep(d, tabs, stream));
    const InputDev di = make_input(in);
    PAC_CUDA(ctx, launch_select(di, d, tabs, out, ctx->d_status, ctx->n_sms, stream));
    return PAC_OK;
}

size_t select_table_bytes(const pac_select_spec *sel) {
    return align_up(static_cast<size_t>(sel->n_thr) * sizeof(SelTable), 256);
}

}  // namespace

namespace pacgpu {
pac_status aggregate_dispatch(pac_ctx *ctx, const pac_input *in, const pac_agg_spec *specs, int32_t n_specs,
                              uint64_t *meta, cudaStream_t stream) {
    return aggregate_impl(ctx, in, specs, n_specs, meta, stream);
}
}  // namespace pacgpu

// ===========================================================================
// exported entry points
// ===========================================================================
extern "C" {

pac_status pac_create(pac_ctx **out, int device) {
    if (!out) return PAC_E_INVALID;
    *out = nullptr;
    pac_ctx *ctx = new (std::nothrow) pac_ctx();
    if (!ctx) return PAC_E_NOMEM;
    ctx->device = device;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || device < 0 || device >= count) {
        delete ctx;
        cudaGetLastError();
        return e != cudaSuccess ? PAC_E_CUDA : PAC_E_INVALID;
    }
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->n_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMalloc(&ctx->d_status, sizeof(uint32_t)) != cudaSuccess ||
        cudaMemset(ctx->d_status, 0, sizeof(uint32_t)) != cudaSuccess ||
        cudaStreamSynchronize(0) != cudaSuccess) {  // cleared before any stream of the caller reads it
        cudaGetLastError();
        if (ctx->d_status) cudaFree(ctx->d_status);
        delete ctx;
        return PAC_E_CUDA;
    }
    *out = ctx;
    return PAC_OK;
}

void pac_destroy(pac_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->qws) cudaFree(ctx->qws);
    if (ctx->sws) cudaFree(ctx->sws);
    if (ctx->small_acc) cudaFree(ctx->small_acc);
    if (ctx->m128) cudaFree(ctx->m128);
    if (ctx->pin_ev) {
        cudaEventSynchronize(ctx->pin_ev);
        cudaEventDestroy(ctx->pin_ev);
    }
    if (ctx->pin) cudaFreeHost(ctx->pin);
    if (ctx->d_status) cudaFree(ctx->d_status);
    delete ctx;
}

const char *pac_last_error(const pac_ctx *ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

const char *pac_status_string(pac_status s) {
    switch (s) {
    case PAC_OK: return "PAC_OK";
    case PAC_E_INVALID: return "PAC_E_INVALID";
    case PAC_E_NOMEM: return "PAC_E_NOMEM";
    case PAC_E_CUDA: return "PAC_E_CUDA";
    case PAC_E_OVERFLOW: return "PAC_E_OVERFLOW";
    case PAC_E_TIMEOUT: return "PAC_E_TIMEOUT";
    case PAC_E_UNSUPPORTED: return "PAC_E_UNSUPPORTED";
    }
    return "unknown";
}

pac_status pac_sync_status(pac_ctx *ctx, pac_stream stream) {
    if (!ctx) return PAC_E_INVALID;
    pac_status st = bind_device(ctx);
    if (st != PAC_OK) return st;
    uint32_t h = 0;
    PAC_CUDA(ctx, cudaMemcpyAsync(&h, ctx->d_status, sizeof(h), cudaMemcpyDeviceToHost, stream));
    PAC_CUDA(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(uint32_t), stream));
    PAC_CUDA(ctx, cudaStreamSynchronize(stream));
    if (h & kStatusTimeout) return fail(ctx, PAC_E_TIMEOUT, "a bounded device wait gave up");
    if (h & kStatusBadGroup) return fail(ctx, PAC_E_INVALID, "a group id was >= n_groups (rows skipped)");
    if (h & kStatusOverflow) return fail(ctx, PAC_E_OVERFLOW, "a result did not fit its output type");
    return PAC_OK;
}

uint64_t pac_query_key(uint64_t seed) {
    return splitmix_mix((seed ^ 0x5041435f4b455921ull) + kGolden);
}

pac_status pac_hash_keys(pac_ctx *ctx, const int64_t *keys, uint64_t *masks, size_t n, uint64_t query_key,
                         int32_t hash_mode, pac_stream stream) {
    if (!ctx) return PAC_E_INVALID;
    if (n > 0 && (!keys || !masks)) return fail(ctx, PAC_E_INVALID, "keys/masks is NULL");
    if (hash_mode != PAC_HASH_BALANCED && hash_mode != PAC_HASH_RAW)
        return fail(ctx, PAC_E_INVALID, "hash_mode %d", hash_mode);
    pac_status st = bind_device(ctx);
    if (st != PAC_OK) return st;
    PAC_CUDA(ctx, launch_hash(keys, masks, n, query_key, hash_mode, ctx->n_sms, stream));
    ctx->last_launches = n ? 1 : 0;
    return PAC_OK;
}

pac_status pac_aggregate_multi(pac_ctx *ctx, const pac_input *in, const pac_agg_spec *specs, int32_t n_specs,
                               uint64_t *meta, pac_stream stream) {
    if (!ctx) return PAC_E_INVALID;
    pac_status st = check_input(ctx, in);
    if (st != PAC_OK) return st;
    st = check_specs(ctx, in, specs, n_specs);
    if (st != PAC_OK) return st;
    if (n_specs == 0 && !meta) return fail(ctx, PAC_E_INVALID, "nothing to compute");
    st = bind_device(ctx);
    if (st != PAC_OK) return st;
    return aggregate_impl(ctx, in, specs, n_specs, meta, stream);
}

pac_status pac_select(pac_ctx *ctx, const pac_input *in, const pac_select_spec *sel, uint64_t *masks_out,
                      pac_stream stream) {
    if (!ctx) return PAC_E_INVALID;
    if (!in) return fail(ctx, PAC_E_INVALID, "input is NULL");
    if (in->n > 0 && (!in->keys_or_masks || !masks_out)) return fail(ctx, PAC_E_INVALID, "keys/masks is NULL");
    const uint32_t base_flags = in->in_flags & ~PAC_IN_DROP_EMPTY;
    if (base_flags != PAC_IN_KEYS && base_flags != PAC_IN_MASKS)
        return fail(ctx, PAC_E_INVALID, "in_flags %u", in->in_flags);
    if (in->hash_mode != PAC_HASH_BALANCED && in->hash_mode != PAC_HASH_RAW)
        return fail(ctx, PAC_E_INVALID, "hash_mode %d", in->hash_mode);
    pac_status st = check_select(ctx, in, sel);
    if (st != PAC_OK) return st;
    st = bind_device(ctx);
    if (st != PAC_OK) return st;
    st = ensure_buffer(ctx, &ctx->sws, &ctx->sws_bytes, select_table_bytes(sel));
    if (st != PAC_OK) return st;
    st = run_select(ctx, in, sel, masks_out, stream);
    if (st != PAC_OK) return st;
    ctx->last_launches = in->n ? 2 : 1;
    return PAC_OK;
}

pac_status pac_aggregate_select(pac_ctx *ctx, const pac_input *in, const pac_select_spec *sel,
                                const pac_agg_spec *specs, int32_t n_specs, uint64_t *meta, pac_stream stream) {
    if (!ctx) return PAC_E_INVALID;
    pac_status st = check_input(ctx, in);
    if (st != PAC_OK) return st;
    st = check_specs(ctx, in, specs, n_specs);
    if (st != PAC_OK) return st;
    if (n_specs == 0 && !meta) return fail(ctx, PAC_E_INVALID, "nothing to compute");
    st = check_select(ctx, in, sel);
    if (st != PAC_OK) return st;
    st = bind_device(ctx);
    if (st != PAC_OK) return st;
    const size_t tb = select_table_bytes(sel);
    st = ensure_buffer(ctx, &ctx->sws, &ctx->sws_bytes, tb + in->n * sizeof(uint64_t));
    if (st != PAC_OK) return st;
    uint64_t *masks = reinterpret_cast<uint64_t *>(static_cast<char *>(ctx->sws) + tb);
    st = run_select(ctx, in, sel, masks, stream);
    if (st != PAC_OK) return st;
    // the selected rows: their masks, and rows left in no world dropped
    pac_input ms = *in;
    ms.keys_or_masks = masks;
    ms.in_flags = PAC_IN_MASKS | PAC_IN_DROP_EMPTY;
    st = aggregate_impl(ctx, &ms, specs, n_specs, meta, stream);
    if (st != PAC_OK) return st;
    ctx->last_launches += in->n ? 2 : 1;
    return PAC_OK;
}

pac_status pac_lift(pac_ctx *ctx, const pac_agg_spec *specs, int32_t n_specs, uint32_t n_groups,
                    const pac_lift_op *prog, int32_t n_ops, double *out, pac_stream stream) {
    if (!ctx) return PAC_E_INVALID;
    if (n_specs < 0 || n_specs > PAC_MAX_SPECS || (n_specs > 0 && !specs))
        return fail(ctx, PAC_E_INVALID, "n_specs %d", n_specs);
    if (!prog || n_ops < 1 || n_ops > PAC_LIFT_MAX_OPS) return fail(ctx, PAC_E_INVALID, "n_ops %d", n_ops);
    if (n_groups > 0 && !out) return fail(ctx, PAC_E_INVALID, "out is NULL");
    LiftParams p{};
    for (int i = 0; i < n_specs; i++) {
        const pac_agg_spec &s = specs[i];
        if (s.kind < PAC_COUNT || s.kind > PAC_LIFTED || (n_groups > 0 && !s.out))
            return fail(ctx, PAC_E_INVALID, "spec %d", i);
        if (s.kind == PAC_LIFTED && s.vtype != PAC_F64)
            return fail(ctx, PAC_E_INVALID, "spec %d: a lifted vector is PAC_F64", i);
        if (s.kind != PAC_COUNT && s.vtype != PAC_I64 && s.vtype != PAC_F32 && s.vtype != PAC_F64)
            return fail(ctx, PAC_E_INVALID, "spec %d: vtype %d", i, s.vtype);
        // stored as: COUNT uint64; AVG, lifted and float aggregates double; else int64
        const int conv = s.kind == PAC_COUNT ? 0 : ((s.kind == PAC_AVG || s.vtype != PAC_I64) ? 2 : 1);
        p.in[i] = s.out;
        p.code[i] = conv | ((s.kind == PAC_COUNT || s.kind == PAC_SUM) ? 4 : 0);
    }
    int depth = 0;  // the program is checked on the host: the kernel trusts it
    for (int k = 0; k < n_ops; k++) {
        const int op = prog[k].op;
        if (op == PAC_LIFT_SPEC || op == PAC_LIFT_CONST) {
            if (op == PAC_LIFT_SPEC && (prog[k].arg < 0 || prog[k].arg >= n_specs))
                return fail(ctx, PAC_E_INVALID, "op %d: no spec %d", k, prog[k].arg);
            if (++depth > PAC_LIFT_DEPTH) return fail(ctx, PAC_E_INVALID, "op %d: deeper than %d", k, PAC_LIFT_DEPTH);
        } else if (op == PAC_LIFT_NEG || op == PAC_LIFT_ABS) {
            if (depth < 1) return fail(ctx, PAC_E_INVALID, "op %d: stack underflow", k);
        } else if (op >= PAC_LIFT_ADD && op <= PAC_LIFT_GE) {
            if (depth < 2) return fail(ctx, PAC_E_INVALID, "op %d: stack underflow", k);
            depth--;
        } else {
            return fail(ctx, PAC_E_INVALID, "op %d: opcode %d", k, op);
        }
        p.prog[k].op = op;
        p.prog[k].arg = prog[k].arg;
        p.prog[k].c = prog[k].c;
    }
    if (depth != 1) return fail(ctx, PAC_E_INVALID, "the program leaves %d values", depth);
    p.n_ops = n_ops;
    p.n_groups = n_groups;
    p.out = out;
    pac_status st = bind_device(ctx);
    if (st != PAC_OK) return st;
    PAC_CUDA(ctx, launch_lift(p, ctx->n_sms, stream));
    ctx->last_launches = n_groups ? 1 : 0;
    return PAC_OK;
}

pac_status pac_filter(pac_ctx *ctx, const double *b, uint32_t n_groups, uint64_t seed, uint8_t *keep,
                      pac_stream stream) {
    if (!ctx) return PAC_E_INVALID;
    if (n_groups > 0 && (!b || !keep)) return fail(ctx, PAC_E_INVALID, "b/keep is NULL");
    pac_status st = bind_device(ctx);
    if (st != PAC_OK) return st;
    PAC_CUDA(ctx, launch_filter(b, n_groups, seed, keep, ctx->n_sms, stream));
    ctx->last_launches = n_groups ? 1 : 0;
    return PAC_OK;
}

pac_status pac_aggregate(pac_ctx *ctx, const void *keys_or_masks, uint32_t in_flags, uint64_t query_key,
                         int32_t hash_mode, const void *values, int32_t vtype, const void *group_ids,
                         int32_t gid_bytes, size_t n, uint32_t n_groups, int32_t kind, int32_t variant, void *out,
                         uint64_t *meta, pac_stream stream) {
    pac_input in;
    in.keys_or_masks = keys_or_masks;
    in.in_flags = in_flags;
    in.hash_mode = hash_mode;
    in.query_key = query_key;
    in.group_ids = group_ids;
    in.gid_bytes = gid_bytes;
    in.n_groups = n_groups;
    in.n = n;
    pac_agg_spec s;
    s.kind = kind;
    s.variant = variant;
    s.vtype = kind == PAC_COUNT ? PAC_I64 : vtype;
    s.reserved = 0;
    s.values = values;
    s.out = out;
    return pac_aggregate_multi(ctx, &in, &s, 1, meta, stream);
}

pac_status pac_finalize(pac_ctx *ctx, const pac_agg_spec *specs, int32_t n_specs, uint32_t n_groups,
                        const uint64_t *meta, uint64_t seed, double budget, int32_t mode, double *noised,
                        uint8_t *is_null, uint32_t *flags, double *posterior, pac_stream stream) {
    if (!ctx) return PAC_E_INVALID;
    FinParams p{};
    pac_status st = build_fin_params(ctx, specs, n_specs, n_groups, meta, seed, budget, mode, noised, is_null,
                                     flags, posterior, p);
    if (st != PAC_OK) return st;
    st = bind_device(ctx);
    if (st != PAC_OK) return st;
    PAC_CUDA(ctx, launch_finalize(p, stream));
    ctx->last_launches = 1;
    return PAC_OK;
}

pac_status pac_query_host(pac_ctx *ctx, const pac_input *in_h, const pac_agg_spec *specs_h, int32_t n_specs,
                          uint64_t seed, double budget, int32_t mode, double *noised, uint8_t *is_null,
                          uint32_t *flags, pac_stream stream) {
    if (!ctx) return PAC_E_INVALID;
    pac_status st = check_input(ctx, in_h);
    if (st != PAC_OK) return st;
    if (n_specs < 1 || n_specs > PAC_MAX_SPECS || !specs_h) return fail(ctx, PAC_E_INVALID, "n_specs %d", n_specs);
    if (!noised || !is_null || !flags) return fail(ctx, PAC_E_INVALID, "NULL host output");
    st = bind_device(ctx);
    if (st != PAC_OK) return st;
    const size_t n = in_h->n;
    const uint32_t G = in_h->n_groups;
    const size_t n_cells = static_cast<size_t>(G) * n_specs;
    const size_t gbytes = in_h->group_ids ? n * in_h->gid_bytes : 0;
    // staging layout: keys | gids | value columns | outs | meta | released cells
    size_t need = align_up(n * 8, 256) + align_up(gbytes, 256) + 4096;
    for (int i = 0; i < n_specs; i++) {
        if (specs_h[i].kind != PAC_COUNT) need += align_up(n * (specs_h[i].vtype == PAC_F32 ? 4 : 8), 256);
        need += align_up(static_cast<size_t>(G) * kWorlds * 8, 256);
    }
    need += align_up(static_cast<size_t>(G) * 16, 256) + 3 * align_up(n_cells * 8, 256);
    st = ensure_buffer(ctx, &ctx->qws, &ctx->qws_bytes, need);
    if (st != PAC_OK) return st;
    Carver cv(ctx->qws);
    pac_input in = *in_h;
    // A query the tensor-core path serves alone reads each input byte once:
    // when every column is pinned host memory, that kernel reads the columns
    // where they are (the same bytes cross the host link, without a staging
    // copy in front of the aggregation).
    const int64_t want = ctx->opt_agg_path;
    bool direct = n > 0 && (((want == 0 || want == 2) && mma_supported(in_h, specs_h, n_specs)) ||
                            ((want == 0 || want == 4) && small_supported(in_h, specs_h, n_specs) &&
                             (want == 4 || n <= kSmallAutoRows)));
    for (int i = 0; i < n_specs && direct; i++) direct = !spec_is_cascade(specs_h[i]);
    auto pinned = [](const void *p) {
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            cudaGetLastError();
            return static_cast<const void *>(nullptr);
        }
        return a.type == cudaMemoryTypeHost ? static_cast<const void *>(a.devicePointer) : nullptr;
    };
    pac_agg_spec direct_specs[PAC_MAX_SPECS];
    if (direct) {
        const void *k = pinned(in_h->keys_or_masks);
        const void *g = in_h->group_ids ? pinned(in_h->group_ids) : nullptr;
        direct = k && (!in_h->group_ids || g);
        for (int i = 0; i < n_specs && direct; i++) {
            direct_specs[i] = specs_h[i];
            if (specs_h[i].kind != PAC_COUNT) {
                direct_specs[i].values = pinned(specs_h[i].values);
                direct = direct_specs[i].values != nullptr;
            }
        }
        if (direct) {
            in.keys_or_masks = k;
            in.group_ids = g;
        }
    }
    void *d_keys = cv.take(n * 8);
    if (n && !direct) PAC_CUDA(ctx, cudaMemcpyAsync(d_keys, in_h->keys_or_masks, n * 8, cudaMemcpyHostToDevice, stream));
    if (!direct) in.keys_or_masks = d_keys;
    if (in_h->group_ids && !direct) {
        void *d_g = cv.take(gbytes);
        if (n) PAC_CUDA(ctx, cudaMemcpyAsync(d_g, in_h->group_ids, gbytes, cudaMemcpyHostToDevice, stream));
        in.group_ids = d_g;
    }
    pac_agg_spec specs[PAC_MAX_SPECS];
    for (int i = 0; i < n_specs; i++) {
        specs[i] = direct ? direct_specs[i] : specs_h[i];
        if (specs[i].kind != PAC_COUNT && !direct) {
            const size_t vb = n * (specs[i].vtype == PAC_F32 ? 4 : 8);
            // a column shared by several specs is copied once
            const void *dv = nullptr;
            for (int k = 0; k < i; k++)
                if (specs_h[k].kind != PAC_COUNT && specs_h[k].values == specs_h[i].values) dv = specs[k].values;
            if (!dv) {
                void *d = cv.take(vb);
                if (n) PAC_CUDA(ctx, cudaMemcpyAsync(d, specs_h[i].values, vb, cudaMemcpyHostToDevice, stream));
                dv = d;
            }
            specs[i].values = dv;
        }
        specs[i].out = cv.take(static_cast<size_t>(G) * kWorlds * 8);
    }
    uint64_t *d_meta = static_cast<uint64_t *>(cv.take(static_cast<size_t>(G) * 16));
    double *d_noised = static_cast<double *>(cv.take(n_cells * 8));
    uint8_t *d_null = static_cast<uint8_t *>(cv.take(n_cells));
    uint32_t *d_flags = static_cast<uint32_t *>(cv.take(n_cells * 4));
    st = pac_aggregate_multi(ctx, &in, specs, n_specs, d_meta, stream);
    if (st != PAC_OK) return st;
    const int64_t agg_launches = ctx->last_launches;
    st = pac_finalize(ctx, specs, n_specs, G, d_meta, seed, budget, mode, d_noised, d_null, d_flags, nullptr, stream);
    if (st != PAC_OK) return st;
    ctx->last_launches += agg_launches;
    PAC_CUDA(ctx, cudaMemcpyAsync(noised, d_noised, n_cells * 8, cudaMemcpyDeviceToHost, stream));
    PAC_CUDA(ctx, cudaMemcpyAsync(is_null, d_null, n_cells, cudaMemcpyDeviceToHost, stream));
    PAC_CUDA(ctx, cudaMemcpyAsync(flags, d_flags, n_cells * 4, cudaMemcpyDeviceToHost, stream));
    return pac_sync_status(ctx, stream);
}

pac_status pac_set_option(pac_ctx *ctx, const char *name, int64_t value) {
    if (!ctx || !name) return PAC_E_INVALID;
    if (strcmp(name, "agg_path") == 0) {
        if (value < 0 || value > 5) return fail(ctx, PAC_E_INVALID, "agg_path %lld", static_cast<long long>(value));
        ctx->opt_agg_path = value;
        return PAC_OK;
    }
    if (strcmp(name, "minmax_prune") == 0) {
        if (value < 0 || value > 1) return fail(ctx, PAC_E_INVALID, "minmax_prune %lld", static_cast<long long>(value));
        ctx->opt_minmax_prune = value;
        return PAC_OK;
    }
    if (strcmp(name, "wait_limit_ns") == 0) {
        if (value < 0) return fail(ctx, PAC_E_INVALID, "wait_limit_ns %lld", static_cast<long long>(value));
        ctx->opt_wait_ns = value;
        return PAC_OK;
    }
    return fail(ctx, PAC_E_INVALID, "unknown option %s", name);
}

pac_status pac_get_info(pac_ctx *ctx, const char *name, int64_t *value) {
    if (!ctx || !name || !value) return PAC_E_INVALID;
    if (strcmp(name, "last_path") == 0) {
        *value = ctx->last_path;
        return PAC_OK;
    }
    if (strcmp(name, "last_launches") == 0) {
        *value = ctx->last_launches;
        return PAC_OK;
    }
    return fail(ctx, PAC_E_INVALID, "unknown info %s", name);
}

}  // extern "C"
