// pac_validate.h -- host-side argument checks and spec classification shared
// by the single-query and batched entry points.
#pragma once

#include "pac_ctx.h"
#include "pac_kernels.h"

namespace pacgpu {

int apx_max_groups();

inline bool is_float(int32_t vtype) { return vtype == PAC_F32 || vtype == PAC_F64; }

// Which per-world state a spec needs on the per-bit path (-1: none).
inline int spec_op(const pac_agg_spec &s) {
    switch (s.kind) {
    case PAC_COUNT: return -1;
    case PAC_SUM:
    case PAC_AVG:
        if (s.vtype == PAC_I64) return s.variant == PAC_APPROX ? -1 : OP_ISUM;
        return s.variant == PAC_APPROX ? OP_FSUM_PLAIN : OP_FSUM_COMP;
    case PAC_MIN: return is_float(s.vtype) ? OP_FMIN : OP_IMIN;
    case PAC_MAX: return is_float(s.vtype) ? OP_FMAX : OP_IMAX;
    }
    return -1;
}

inline bool spec_is_cascade(const pac_agg_spec &s) {
    return (s.kind == PAC_SUM || s.kind == PAC_AVG) && s.vtype == PAC_I64 && s.variant == PAC_APPROX;
}

inline pac_status check_input(pac_ctx *ctx, const pac_input *in) {
    if (!in) return fail(ctx, PAC_E_INVALID, "input is NULL");
    if (in->n > 0 && !in->keys_or_masks) return fail(ctx, PAC_E_INVALID, "keys_or_masks is NULL");
    const uint32_t base_flags = in->in_flags & ~PAC_IN_DROP_EMPTY;
    if (base_flags != PAC_IN_KEYS && base_flags != PAC_IN_MASKS)
        return fail(ctx, PAC_E_INVALID, "in_flags %u", in->in_flags);
    if (in->hash_mode != PAC_HASH_BALANCED && in->hash_mode != PAC_HASH_RAW)
        return fail(ctx, PAC_E_INVALID, "hash_mode %d", in->hash_mode);
    if (in->n_groups == 0) return fail(ctx, PAC_E_INVALID, "n_groups must be >= 1");
    if (!in->group_ids && in->n_groups != 1 && in->n > 0)
        return fail(ctx, PAC_E_INVALID, "ungrouped input needs n_groups == 1");
    if (in->group_ids && in->gid_bytes != 1 && in->gid_bytes != 2 && in->gid_bytes != 4)
        return fail(ctx, PAC_E_INVALID, "gid_bytes %d", in->gid_bytes);
    if (in->group_ids && in->gid_bytes == 1 && in->n_groups > 256)
        return fail(ctx, PAC_E_INVALID, "n_groups %u exceeds 8-bit group ids", in->n_groups);
    if (in->group_ids && in->gid_bytes == 2 && in->n_groups > 65536)
        return fail(ctx, PAC_E_INVALID, "n_groups %u exceeds 16-bit group ids", in->n_groups);
    return PAC_OK;
}

inline pac_status check_specs(pac_ctx *ctx, const pac_input *in, const pac_agg_spec *specs, int32_t n_specs) {
    if (n_specs < 0 || n_specs > PAC_MAX_SPECS) return fail(ctx, PAC_E_INVALID, "n_specs %d", n_specs);
    if (n_specs > 0 && !specs) return fail(ctx, PAC_E_INVALID, "specs is NULL");
    for (int i = 0; i < n_specs; i++) {
        const pac_agg_spec &s = specs[i];
        if (s.kind < PAC_COUNT || s.kind > PAC_MAX) return fail(ctx, PAC_E_INVALID, "spec %d: kind %d", i, s.kind);
        if (s.variant != PAC_EXACT && s.variant != PAC_APPROX)
            return fail(ctx, PAC_E_INVALID, "spec %d: variant %d", i, s.variant);
        if (s.kind != PAC_COUNT && (s.vtype < PAC_I64 || s.vtype > PAC_F64))
            return fail(ctx, PAC_E_INVALID, "spec %d: vtype %d", i, s.vtype);
        if (s.reserved != 0) return fail(ctx, PAC_E_INVALID, "spec %d: reserved must be 0", i);
        if (!s.out) return fail(ctx, PAC_E_INVALID, "spec %d: out is NULL", i);
        if (s.kind != PAC_COUNT && in->n > 0 && !s.values)
            return fail(ctx, PAC_E_INVALID, "spec %d: values is NULL", i);
        if (spec_is_cascade(s) && in->n_groups > static_cast<uint32_t>(apx_max_groups()))
            return fail(ctx, PAC_E_UNSUPPORTED, "spec %d: approximate integer SUM/AVG serves at most %d groups",
                        i, apx_max_groups());
    }
    return PAC_OK;
}

// Argument checks of a release (pac_finalize, pac_finalize128) and its
// launch parameters.
inline pac_status build_fin_params(pac_ctx *ctx, const pac_agg_spec *specs, int32_t n_specs, uint32_t n_groups,
                                   const uint64_t *meta, uint64_t seed, double budget, int32_t mode,
                                   double *noised, uint8_t *is_null, uint32_t *flags, double *posterior,
                                   FinParams &p) {
    if (n_specs < 1 || n_specs > PAC_MAX_SPECS || !specs) return fail(ctx, PAC_E_INVALID, "n_specs %d", n_specs);
    if (n_groups < 1) return fail(ctx, PAC_E_INVALID, "n_groups must be >= 1");
    if (!meta || !noised || !is_null || !flags) return fail(ctx, PAC_E_INVALID, "NULL output or meta");
    if (!(budget > 0.0)) return fail(ctx, PAC_E_INVALID, "budget must be > 0");
    if (mode != PAC_FIN_ADAPTIVE && mode != PAC_FIN_INDEPENDENT) return fail(ctx, PAC_E_INVALID, "mode %d", mode);
    p = FinParams{};
    for (int i = 0; i < n_specs; i++) {
        if (specs[i].kind < PAC_COUNT || specs[i].kind > PAC_LIFTED || !specs[i].out)
            return fail(ctx, PAC_E_INVALID, "spec %d", i);
        if (specs[i].kind == PAC_LIFTED && specs[i].vtype != PAC_F64)
            return fail(ctx, PAC_E_INVALID, "spec %d: a lifted vector is PAC_F64", i);
        p.spec[i].kind = specs[i].kind;
        p.spec[i].vtype = specs[i].kind == PAC_COUNT ? PAC_I64 : specs[i].vtype;
        p.spec[i].variant = specs[i].variant;
        p.spec[i].out = specs[i].out;
    }
    p.n_specs = n_specs;
    p.n_groups = n_groups;
    p.meta = meta;
    p.seed = seed;
    p.budget = budget;
    p.mode = mode;
    p.noised = noised;
    p.is_null = is_null;
    p.flags = flags;
    p.posterior = posterior;
    return PAC_OK;
}

inline InputDev make_input(const pac_input *in) {
    InputDev d;
    d.km = in->keys_or_masks;
    d.gids = in->group_ids;
    d.qkey = in->query_key;
    d.n = in->n;
    d.in_flags = in->in_flags;
    d.hash_mode = in->hash_mode;
    d.gid_bytes = in->group_ids ? in->gid_bytes : 0;
    d.n_groups = in->n_groups;
    return d;
}

}  // namespace pacgpu
