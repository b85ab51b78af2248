/*
 * pac_oracle.c -- plain scalar CPU oracle for PAC stochastic aggregation
 * (SIMD-PAC-DB, arXiv 2603.15023).
 *
 * TEST INFRASTRUCTURE ONLY (see pac_oracle.h).  Slow on purpose: one row at a
 * time, one world at a time, 128-bit integers for exact sums, FP64 with
 * Neumaier compensation for floating-point sums.
 *
 * Readings of the paper that this file fixes where the paper is silent:
 *   R1  pac_hash (Sec. 2 "SIMD-PAC-DB", Sec. 4.2 "PAC Hash"): the engine hash
 *       of the PU key is MurmurHash3's 64-bit finalizer fmix64; the per-query
 *       re-hash is fmix64(inner XOR K) with K drawn per query from SplitMix64;
 *       the balanced transform keeps the low 32 hash bits as worlds 0..31 and
 *       their complement as worlds 32..63, so every PU lies in exactly 32
 *       worlds (Sec. 4.1, balanced subset construction).  "raw" mode keeps all
 *       64 hash bits (binomial popcount).
 *   R2  empty world: COUNT/SUM give 0; AVG/MIN/MAX give 0 (Sec. 3.2 "NULLs":
 *       counters of unset bits are treated as zeros).
 *   R3  approximate integer SUM (Sec. 5 "Approximation"): a value goes to
 *       level l = floor((msb(|v|)-8)/4) clamped at 0, as x = |v| >> 4l; each
 *       level keeps the exact total T[l] of what it received; if T[l]+x would
 *       exceed 0xFFFF the level is flushed first (Sec. 5 "Cascading": flush
 *       before the update); a flush adds C[l][j]>>4 into level l+1 (flushing
 *       l+1 first if its total would overflow), adds T[l]>>4 into T[l+1] and
 *       clears level l.  Negative values go to a second, negated state
 *       (two-sided SUM).  Rows are cut into chunks of ORC_APX_CHUNK
 *       consecutive rows; each chunk fills a fresh state per group; chunk
 *       states are combined level by level (flush on overflow, then add) in a
 *       pairwise tree over chunk index.
 *   R4  AVG: PAC_EXACT is sum_j/count_j (Sec. 4.2 definition); the
 *       approximate variant divides by the exact update count of the group
 *       (Sec. 5 "Cascading"), times 2 for the two-sided result (Sec. 5).
 *   R5  finalize: release scale 2 for COUNT and SUM (Sec. 2, fused
 *       pac_noised_count: count[j*]*2), 1 otherwise; the variance is taken
 *       over the scaled vector; cells are released group by group, specs in
 *       order; NULL per cell with probability (64-popcount(or_g))/64 and no
 *       posterior update; the posterior is kept in log space.
 *   R6  diversity: flag a cell when its group has >= 64 rows but at most 40
 *       worlds ever received an update (Sec. 5 "Diversity Check").  The OR
 *       accumulator of Sec. 3.2 is used (the XOR of Sec. 5 cannot say which
 *       worlds were never updated).
 *   R7  m = 128 worlds (Sec. 2 says m = 128 is possible; the paper runs 64):
 *       two keyed re-hashes of the engine hash, h_a with K and h_b with K2,
 *       the SplitMix64 output after K.  Balanced: worlds 0..31 are the low
 *       word of h_a, 32..63 the low word of h_b, 64..127 the complement of
 *       0..63 (every PU in exactly 64 worlds).  Raw: worlds 0..63 are h_a,
 *       64..127 h_b.  The release is R5/R6 with 128 worlds: j* is the top 7
 *       bits of the first draw, the prior is uniform over 128 worlds, a cell
 *       is NULL with probability (128 - popcount(or_g))/128, and the
 *       diversity flag needs at most 80 updated worlds (the same 5/8).
 */
#include "pac_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

/* ====================================================================== */
/* Hashing                                                                 */
/* ====================================================================== */

/* MurmurHash3 64-bit finalizer (Appleby, public domain): xor-shift by 33,
 * multiply, xor-shift, multiply, xor-shift. */
uint64_t orc_fmix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
}

/* Inverse of an odd multiplier modulo 2^64 by Newton iteration
 * (each step doubles the number of correct low bits). */
static uint64_t inv_odd(uint64_t a) {
    uint64_t x = a; /* correct to 3 bits for odd a */
    for (int i = 0; i < 6; i++) x *= 2 - a * x;
    return x;
}

/* fmix64 is a bijection: x ^ (x >> 33) is its own inverse because 2*33 >= 64,
 * and each multiplier is odd.  Used by the pins, not by the method. */
uint64_t orc_fmix64_inverse(uint64_t h) {
    h ^= h >> 33;
    h *= inv_odd(0xc4ceb9fe1a85ec53ULL);
    h ^= h >> 33;
    h *= inv_odd(0xff51afd7ed558ccdULL);
    h ^= h >> 33;
    return h;
}

/* SplitMix64 (Steele, Lea, Flood 2014; Vigna's reference code): advance the
 * state by the golden gamma, then mix. */
uint64_t orc_splitmix64_next(uint64_t *state) {
    uint64_t z = (*state += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Per-query key K (Sec. 4.2: "K is a randomly sampled key drawn
 * independently for each query"): first SplitMix64 output of the query seed
 * XOR an ASCII domain tag "PAC_KEY!". */
uint64_t orc_query_key(uint64_t seed) {
    uint64_t s = seed ^ 0x5041435f4b455921ULL;
    return orc_splitmix64_next(&s);
}

/* pac_hash_K(key) -> 64-bit world mask (reading R1). */
uint64_t orc_pac_hash(int64_t key, uint64_t query_key, int mode) {
    uint64_t inner = orc_fmix64((uint64_t)key);   /* engine hash of the PU key */
    uint64_t h = orc_fmix64(inner ^ query_key);  /* keyed per-query re-hash */
    if (mode == ORC_RAW) return h;
    uint64_t lo = h & 0xffffffffULL;
    uint64_t hi = (~h) & 0xffffffffULL;
    return lo | (hi << 32);
}

void orc_hash_keys(const int64_t *keys, size_t n, uint64_t query_key, int mode,
                   uint64_t *masks) {
    for (size_t i = 0; i < n; i++) masks[i] = orc_pac_hash(keys[i], query_key, mode);
}

/* ====================================================================== */
/* Counter-based generator for the finalizer                               */
/* ====================================================================== */

/* Draw number `counter` of stream `stream`: the stream's start state is
 * SplitMix64 output number `stream` from the seed; the draw is SplitMix64
 * output number `counter` from that start state.  SplitMix64 output i from
 * state s is mix(s + (i+1)*gamma), which is what the loop-free form below
 * computes by seeking the state. */
uint64_t orc_rng_u64(uint64_t seed, uint64_t stream, uint64_t counter) {
    uint64_t s = seed + stream * 0x9e3779b97f4a7c15ULL;
    uint64_t stream_state = orc_splitmix64_next(&s);
    uint64_t t = stream_state + counter * 0x9e3779b97f4a7c15ULL;
    return orc_splitmix64_next(&t);
}

double orc_u01(uint64_t u) { return (double)(u >> 11) * 0x1.0p-53; }
double orc_u01_open0(uint64_t u) { return (double)((u >> 11) + 1) * 0x1.0p-53; }

/* Box-Muller: z = sqrt(-2 ln u1) cos(2 pi u2), u1 in (0,1], u2 in [0,1). */
double orc_box_muller(uint64_t u1, uint64_t u2) {
    double a = orc_u01_open0(u1);
    double b = orc_u01(u2);
    return sqrt(-2.0 * log(a)) * cos(2.0 * M_PI * b);
}

/* ====================================================================== */
/* Helpers shared by the oracle's own aggregation routines                */
/* ====================================================================== */

static uint32_t gid_at(const void *gids, int gid_bytes, size_t i) {
    if (!gids) return 0;
    switch (gid_bytes) {
    case 1: return ((const uint8_t *)gids)[i];
    case 2: return ((const uint16_t *)gids)[i];
    default: return ((const uint32_t *)gids)[i];
    }
}

static double fval_at(const void *values, int vtype, size_t i) {
    if (vtype == ORC_F32) return (double)((const float *)values)[i];
    return ((const double *)values)[i];
}

static int fits_i64(i128 v) { return v >= (i128)INT64_MIN && v <= (i128)INT64_MAX; }

static int64_t clamp_i64(i128 v, int *status) {
    if (fits_i64(v)) return (int64_t)v;
    *status = 4;
    return v < 0 ? INT64_MIN : INT64_MAX;
}

/* int128 -> double, rounding once: exact int64 conversion when it fits. */
static double i128_to_double(i128 v) {
    if (fits_i64(v)) return (double)(int64_t)v;
    return (double)v;
}

/* Neumaier (improved Kahan-Babuska) compensated FP64 summation. */
typedef struct { double s, c; } nsum;
static void nsum_add(nsum *a, double v) {
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}
static double nsum_get(const nsum *a) { return a->s + a->c; }

/* One group x world accumulator for the exact definition. */
typedef struct {
    uint64_t cnt;
    i128 isum;
    nsum fsum;
    int64_t imin, imax;
    double fmin, fmax;
} acc_t;

static void acc_init(acc_t *a) {
    memset(a, 0, sizeof(*a));
    a->imin = INT64_MAX; a->imax = INT64_MIN;
    a->fmin = INFINITY; a->fmax = -INFINITY;
}

static void acc_update(acc_t *a, const void *values, int vtype, size_t i) {
    a->cnt += 1;
    if (!values) return;
    if (vtype == ORC_I64) {
        int64_t v = ((const int64_t *)values)[i];
        a->isum += v;
        if (v < a->imin) a->imin = v;
        if (v > a->imax) a->imax = v;
    } else {
        double v = fval_at(values, vtype, i);
        nsum_add(&a->fsum, v);
        if (v < a->fmin) a->fmin = v;
        if (v > a->fmax) a->fmax = v;
    }
}

/* Write one world's result (reading R2 for empty worlds). */
static void acc_emit(const acc_t *a, int vtype, int kind, void *out, size_t idx,
                     int *status) {
    if (kind == ORC_COUNT) { ((uint64_t *)out)[idx] = a->cnt; return; }
    int empty = (a->cnt == 0);
    if (vtype == ORC_I64) {
        switch (kind) {
        case ORC_SUM: ((int64_t *)out)[idx] = clamp_i64(a->isum, status); break;
        case ORC_AVG:
            ((double *)out)[idx] = empty ? 0.0 : i128_to_double(a->isum) / (double)a->cnt;
            break;
        case ORC_MIN: ((int64_t *)out)[idx] = empty ? 0 : a->imin; break;
        case ORC_MAX: ((int64_t *)out)[idx] = empty ? 0 : a->imax; break;
        }
    } else {
        double s = nsum_get(&a->fsum);
        switch (kind) {
        case ORC_SUM: ((double *)out)[idx] = s; break;
        case ORC_AVG: ((double *)out)[idx] = empty ? 0.0 : s / (double)a->cnt; break;
        case ORC_MIN: ((double *)out)[idx] = empty ? 0.0 : a->fmin; break;
        case ORC_MAX: ((double *)out)[idx] = empty ? 0.0 : a->fmax; break;
        }
    }
}

/* ====================================================================== */
/* PAC selection (Sec. 4.2 "PAC Selection": the output bit j is set iff    */
/* the row satisfies the predicate on world j's aggregate result and       */
/* pu[j] = 1; Sec. 3.2: pac_select ANDs pu with 64 booleans, and the fused */
/* pac_select_<cmp>(hash, col, list) compares col with each list entry).   */
/* ====================================================================== */
static int holds_i64(int64_t a, int64_t b, int cmp) {
    switch (cmp) {
    case ORC_CMP_LT: return a < b;
    case ORC_CMP_LE: return a <= b;
    case ORC_CMP_EQ: return a == b;
    case ORC_CMP_NE: return a != b;
    case ORC_CMP_GT: return a > b;
    default: return a >= b;
    }
}

static int holds_f64(double a, double b, int cmp) {
    switch (cmp) {
    case ORC_CMP_LT: return a < b;
    case ORC_CMP_LE: return a <= b;
    case ORC_CMP_EQ: return a == b;
    case ORC_CMP_NE: return a != b;
    case ORC_CMP_GT: return a > b;
    default: return a >= b;
    }
}

int orc_select(const uint64_t *masks, const void *col, int vtype, int cmp, const void *thr,
               uint32_t n_thr, const void *thr_ids, int thr_id_bytes, size_t n, uint64_t *out) {
    int status = 0;
    for (size_t i = 0; i < n; i++) {
        uint32_t t = n_thr == 1 ? 0 : gid_at(thr_ids, thr_id_bytes, i);
        if (t >= n_thr) {
            out[i] = 0;
            status = 1;
            continue;
        }
        uint64_t bits = 0;
        for (int j = 0; j < 64; j++) {
            size_t k = (size_t)t * 64 + (size_t)j;
            int h = vtype == ORC_I64 ? holds_i64(((const int64_t *)col)[i], ((const int64_t *)thr)[k], cmp)
                                     : holds_f64(fval_at(col, vtype, i), fval_at(thr, vtype, k), cmp);
            if (h) bits |= 1ULL << j;
        }
        out[i] = masks[i] & bits;
    }
    return status;
}

/* ====================================================================== */
/* Vector-lifted expressions (Sec. 4.2 "Vector-lifted Expression, and      */
/* Lambda Functions": the scalar expression applied world by world, scalar */
/* operands broadcast to every world; Sec. 7 evaluates a ratio of two      */
/* pac_sum vectors this way and noises it once).                           */
/* ====================================================================== */
static int lift_check(uint32_t n_specs, const orc_lift_op *prog, int n_ops) {
    int depth = 0;
    for (int k = 0; k < n_ops; k++) {
        int op = prog[k].op;
        if (op == ORC_LIFT_SPEC || op == ORC_LIFT_CONST) {
            if (op == ORC_LIFT_SPEC && (prog[k].arg < 0 || (uint32_t)prog[k].arg >= n_specs)) return 1;
            if (++depth > ORC_LIFT_DEPTH) return 1;
        } else if (op == ORC_LIFT_NEG || op == ORC_LIFT_ABS) {
            if (depth < 1) return 1;
        } else if (op >= ORC_LIFT_ADD && op <= ORC_LIFT_GE) {
            if (depth < 2) return 1;
            depth--;
        } else {
            return 1;
        }
    }
    return depth == 1 ? 0 : 1;
}

int orc_lift(const double *y, const double *scales, uint32_t n_specs, uint32_t n_groups,
             const orc_lift_op *prog, int n_ops, double *out) {
    if (lift_check(n_specs, prog, n_ops)) return 1;
    for (uint32_t g = 0; g < n_groups; g++) {
        for (int j = 0; j < 64; j++) {
            double st[ORC_LIFT_DEPTH];
            int sp = 0;
            for (int k = 0; k < n_ops; k++) {
                int op = prog[k].op;
                if (op == ORC_LIFT_SPEC) {
                    int s = prog[k].arg;
                    st[sp++] = scales[s] * y[((size_t)g * n_specs + (size_t)s) * 64 + (size_t)j];
                    continue;
                }
                if (op == ORC_LIFT_CONST) { st[sp++] = prog[k].c; continue; }
                if (op == ORC_LIFT_NEG) { st[sp - 1] = -st[sp - 1]; continue; }
                if (op == ORC_LIFT_ABS) { st[sp - 1] = fabs(st[sp - 1]); continue; }
                double b = st[--sp], a = st[sp - 1], r;
                switch (op) {
                case ORC_LIFT_ADD: r = a + b; break;
                case ORC_LIFT_SUB: r = a - b; break;
                case ORC_LIFT_MUL: r = a * b; break;
                case ORC_LIFT_DIV: r = a / b; break;
                case ORC_LIFT_MIN: r = a < b ? a : b; break;
                case ORC_LIFT_MAX: r = a > b ? a : b; break;
                case ORC_LIFT_LT: r = a < b ? 1.0 : 0.0; break;
                case ORC_LIFT_LE: r = a <= b ? 1.0 : 0.0; break;
                case ORC_LIFT_EQ: r = a == b ? 1.0 : 0.0; break;
                case ORC_LIFT_NE: r = a != b ? 1.0 : 0.0; break;
                case ORC_LIFT_GT: r = a > b ? 1.0 : 0.0; break;
                default: r = a >= b ? 1.0 : 0.0; break;
                }
                st[sp - 1] = r;
            }
            out[(size_t)g * 64 + (size_t)j] = st[0];
        }
    }
    return 0;
}

/* ====================================================================== */
/* pac_filter (Sec. 3.2 "Categorical Rewrites"): the fraction of the 64    */
/* booleans that are true is the probability of a random yes/no choice.    */
/* ====================================================================== */
#define STREAM_FILTER 3

void orc_filter(const double *b, uint32_t n_groups, uint64_t seed, uint8_t *keep) {
    for (uint32_t g = 0; g < n_groups; g++) {
        int t = 0;
        for (int j = 0; j < 64; j++) t += b[(size_t)g * 64 + (size_t)j] != 0.0;
        double u = orc_u01(orc_rng_u64(seed, STREAM_FILTER, g));
        keep[g] = u < (double)t / 64.0 ? 1 : 0;
    }
}

/* ====================================================================== */
/* Exact aggregation, row by row: r_j = agg{ e(t) : t in T, pu[j] = 1 }    */
/* (Sec. 4.2 "PAC Aggregation"; the predicated 64-world update loop of     */
/* PacCountUpdate in Sec. 1 and Sec. 5 "Naive"/predication).               */
/* ====================================================================== */
int orc_aggregate_direct(const uint64_t *masks, const void *values, int vtype,
                         const void *gids, int gid_bytes, size_t n,
                         uint32_t n_groups, int kind, void *out,
                         uint64_t *meta_n, uint64_t *meta_or) {
    int status = 0;
    acc_t *acc = (acc_t *)malloc(sizeof(acc_t) * (size_t)n_groups * 64);
    if (!acc) return 2;
    for (size_t k = 0; k < (size_t)n_groups * 64; k++) acc_init(&acc[k]);
    if (meta_n) memset(meta_n, 0, sizeof(uint64_t) * n_groups);
    if (meta_or) memset(meta_or, 0, sizeof(uint64_t) * n_groups);

    for (size_t i = 0; i < n; i++) {
        uint32_t g = gid_at(gids, gid_bytes, i);
        uint64_t key_hash = masks[i];
        if (meta_n) meta_n[g] += 1;
        if (meta_or) meta_or[g] |= key_hash;      /* Sec. 3.2: K <- K | h */
        for (int j = 0; j < 64; j++) {
            if ((key_hash >> j) & 1ULL)
                acc_update(&acc[(size_t)g * 64 + j], values, vtype, i);
        }
    }
    for (size_t k = 0; k < (size_t)n_groups * 64; k++)
        acc_emit(&acc[k], vtype, kind, out, k, &status);
    free(acc);
    return status;
}

/* One world only: r_j for a single j, every group (the same definition,
 * restricted to one world so that large inputs can be sampled). */
int orc_aggregate_world(const uint64_t *masks, const void *values, int vtype,
                        const void *gids, int gid_bytes, size_t n,
                        uint32_t n_groups, int kind, int world, void *out) {
    int status = 0;
    acc_t *acc = (acc_t *)malloc(sizeof(acc_t) * (size_t)n_groups);
    if (!acc) return 2;
    for (uint32_t g = 0; g < n_groups; g++) acc_init(&acc[g]);
    for (size_t i = 0; i < n; i++)
        if ((masks[i] >> world) & 1ULL)
            acc_update(&acc[gid_at(gids, gid_bytes, i)], values, vtype, i);
    for (uint32_t g = 0; g < n_groups; g++) acc_emit(&acc[g], vtype, kind, out, g, &status);
    free(acc);
    return status;
}

/* ====================================================================== */
/* Brute force over materialised worlds (Sec. 4.1 steps (1)-(2); the       */
/* subsets coincide with S_j = { u : pac_hash_K(u)[j] = 1 } as Theorem 2   */
/* assumes).  For each world: build the sample table S_j as a set of PU    */
/* keys, keep the rows whose PU is in S_j (the join with the sample), and  */
/* run an ordinary GROUP BY aggregate over them.                           */
/* ====================================================================== */

typedef struct { int64_t *slot; uint8_t *used; size_t cap; } keyset;

static size_t ks_probe_start(const keyset *s, int64_t k) {
    /* Fibonacci hashing; unrelated to pac_hash on purpose. */
    return (size_t)(((uint64_t)k * 0x9e3779b97f4a7c15ULL) >> 20) & (s->cap - 1);
}
static int ks_init(keyset *s, size_t n) {
    size_t cap = 16;
    while (cap < 2 * n + 16) cap <<= 1;
    s->cap = cap;
    s->slot = (int64_t *)malloc(sizeof(int64_t) * cap);
    s->used = (uint8_t *)calloc(cap, 1);
    return s->slot && s->used;
}
static void ks_free(keyset *s) { free(s->slot); free(s->used); }
static void ks_insert(keyset *s, int64_t k) {
    size_t p = ks_probe_start(s, k);
    while (s->used[p]) {
        if (s->slot[p] == k) return;
        p = (p + 1) & (s->cap - 1);
    }
    s->used[p] = 1; s->slot[p] = k;
}
static int ks_contains(const keyset *s, int64_t k) {
    size_t p = ks_probe_start(s, k);
    while (s->used[p]) {
        if (s->slot[p] == k) return 1;
        p = (p + 1) & (s->cap - 1);
    }
    return 0;
}

int orc_aggregate_brute(const int64_t *keys, uint64_t query_key, int mode,
                        const void *values, int vtype, const void *gids,
                        int gid_bytes, size_t n, uint32_t n_groups, int kind,
                        void *out) {
    int status = 0;
    /* the PU universe: distinct keys */
    keyset universe;
    if (!ks_init(&universe, n)) return 2;
    for (size_t i = 0; i < n; i++) ks_insert(&universe, keys[i]);

    acc_t *acc = (acc_t *)malloc(sizeof(acc_t) * n_groups);
    if (!acc) { ks_free(&universe); return 2; }

    for (int j = 0; j < 64; j++) {
        /* step (1): the j-th sampled PU table */
        keyset sample;
        if (!ks_init(&sample, n)) { free(acc); ks_free(&universe); return 2; }
        for (size_t p = 0; p < universe.cap; p++) {
            if (!universe.used[p]) continue;
            int64_t u = universe.slot[p];
            if ((orc_pac_hash(u, query_key, mode) >> j) & 1ULL) ks_insert(&sample, u);
        }
        /* step (2): the query on the j-th sampled instance */
        for (uint32_t g = 0; g < n_groups; g++) acc_init(&acc[g]);
        for (size_t i = 0; i < n; i++) {
            if (!ks_contains(&sample, keys[i])) continue;
            acc_update(&acc[gid_at(gids, gid_bytes, i)], values, vtype, i);
        }
        for (uint32_t g = 0; g < n_groups; g++)
            acc_emit(&acc[g], vtype, kind, out, (size_t)g * 64 + j, &status);
        ks_free(&sample);
    }
    free(acc);
    ks_free(&universe);
    return status;
}

/* ====================================================================== */
/* Approximate integer SUM (reading R3)                                    */
/* ====================================================================== */

typedef struct {
    uint16_t C[ORC_APX_LEVELS][64];
    uint32_t T[ORC_APX_LEVELS];
} apx_side;
typedef struct { apx_side side[2]; } apx_state; /* [0] positive, [1] negated negatives */

static void apx_flush(apx_side *s, int l, int *ovf) {
    if (l == ORC_APX_LEVELS - 1) { *ovf = 1; return; }
    uint32_t carry_total = s->T[l] >> 4;
    if (s->T[l + 1] + carry_total > 0xFFFF) apx_flush(s, l + 1, ovf);
    for (int j = 0; j < 64; j++) s->C[l + 1][j] = (uint16_t)(s->C[l + 1][j] + (s->C[l][j] >> 4));
    s->T[l + 1] += carry_total;
    memset(s->C[l], 0, sizeof(s->C[l]));
    s->T[l] = 0;
}

static int msb64(uint64_t a) { return 63 - __builtin_clzll(a); }

static void apx_update(apx_state *st, int64_t v, uint64_t key_hash, int *ovf) {
    if (v == 0) return;
    int side = v < 0;
    uint64_t a = side ? (uint64_t)0 - (uint64_t)v : (uint64_t)v;
    int m = msb64(a);
    int l = m < 8 ? 0 : (m - 8) / 4;           /* l(v) = floor((msb(|v|)-8)/4) */
    uint32_t x = (uint32_t)(a >> (4 * l));     /* value in units of 2^(4l) */
    apx_side *s = &st->side[side];
    if (s->T[l] + x > 0xFFFF) apx_flush(s, l, ovf);
    for (int j = 0; j < 64; j++)
        if ((key_hash >> j) & 1ULL) s->C[l][j] = (uint16_t)(s->C[l][j] + x);
    s->T[l] += x;
}

/* dst <- dst (+) src, level by level. */
static void apx_combine(apx_state *dst, const apx_state *src, int *ovf) {
    for (int sd = 0; sd < 2; sd++) {
        apx_side *a = &dst->side[sd];
        const apx_side *b = &src->side[sd];
        for (int l = 0; l < ORC_APX_LEVELS; l++) {
            if (a->T[l] + b->T[l] > 0xFFFF) apx_flush(a, l, ovf);
            for (int j = 0; j < 64; j++) a->C[l][j] = (uint16_t)(a->C[l][j] + b->C[l][j]);
            a->T[l] += b->T[l];
        }
    }
}

static i128 apx_side_value(const apx_side *s, int j) {
    i128 v = 0;
    for (int l = 0; l < ORC_APX_LEVELS; l++) v += (i128)s->C[l][j] << (4 * l);
    return v;
}

/* Runs the chunk schedule and leaves the combined per-group state in
 * `final_states` ([n_groups]).  Returns overflow as status 4. */
/* drop_empty: a row whose mask is 0 is a row of no group (filtered out by a
 * selection): it updates nothing, not even a level total, and the chunks
 * stay over row positions. */
static int apx_run(const uint64_t *masks, const int64_t *values,
                   const void *gids, int gid_bytes, size_t n, uint32_t n_groups,
                   apx_state *final_states, int drop_empty) {
    int ovf = 0;
    size_t n_chunks = (n + ORC_APX_CHUNK - 1) / ORC_APX_CHUNK;
    if (n_chunks == 0) {
        memset(final_states, 0, sizeof(apx_state) * n_groups);
        return 0;
    }
    /* states[c * n_groups + g]: chunk c, group g */
    apx_state *states = (apx_state *)calloc(n_chunks * (size_t)n_groups, sizeof(apx_state));
    if (!states) return 2;
    for (size_t c = 0; c < n_chunks; c++) {
        size_t lo = c * ORC_APX_CHUNK, hi = lo + ORC_APX_CHUNK;
        if (hi > n) hi = n;
        for (size_t i = lo; i < hi; i++) {
            if (drop_empty && masks[i] == 0) continue;
            uint32_t g = gid_at(gids, gid_bytes, i);
            apx_update(&states[c * n_groups + g], values[i], masks[i], &ovf);
        }
    }
    /* pairwise tree over chunk index: width 1, 2, 4, ... */
    for (size_t w = 1; w < n_chunks; w *= 2) {
        for (size_t c = 0; c + w < n_chunks; c += 2 * w) {
            for (uint32_t g = 0; g < n_groups; g++)
                apx_combine(&states[c * n_groups + g], &states[(c + w) * n_groups + g], &ovf);
        }
    }
    memcpy(final_states, states, sizeof(apx_state) * n_groups);
    free(states);
    return ovf ? 4 : 0;
}

int orc_approx_sum_i64(const uint64_t *masks, const int64_t *values,
                       const void *gids, int gid_bytes, size_t n,
                       uint32_t n_groups, int64_t *out) {
    return orc_approx_sum_i64_ex(masks, values, gids, gid_bytes, n, n_groups, out, 0);
}

int orc_approx_sum_i64_ex(const uint64_t *masks, const int64_t *values,
                          const void *gids, int gid_bytes, size_t n,
                          uint32_t n_groups, int64_t *out, int drop_empty) {
    apx_state *fin = (apx_state *)calloc(n_groups ? n_groups : 1, sizeof(apx_state));
    if (!fin) return 2;
    int status = apx_run(masks, values, gids, gid_bytes, n, n_groups, fin, drop_empty);
    for (uint32_t g = 0; g < n_groups; g++)
        for (int j = 0; j < 64; j++) {
            i128 v = apx_side_value(&fin[g].side[0], j) - apx_side_value(&fin[g].side[1], j);
            out[(size_t)g * 64 + j] = clamp_i64(v, &status);
        }
    free(fin);
    return status;
}

int orc_approx_avg_i64(const uint64_t *masks, const int64_t *values,
                       const void *gids, int gid_bytes, size_t n,
                       uint32_t n_groups, double *out) {
    return orc_approx_avg_i64_ex(masks, values, gids, gid_bytes, n, n_groups, out, 0);
}

int orc_approx_avg_i64_ex(const uint64_t *masks, const int64_t *values,
                          const void *gids, int gid_bytes, size_t n,
                          uint32_t n_groups, double *out, int drop_empty) {
    apx_state *fin = (apx_state *)calloc(n_groups ? n_groups : 1, sizeof(apx_state));
    uint64_t *cnt = (uint64_t *)calloc(n_groups ? n_groups : 1, sizeof(uint64_t));
    if (!fin || !cnt) { free(fin); free(cnt); return 2; }
    int status = apx_run(masks, values, gids, gid_bytes, n, n_groups, fin, drop_empty);
    for (size_t i = 0; i < n; i++) /* exact update count */
        if (!(drop_empty && masks[i] == 0)) cnt[gid_at(gids, gid_bytes, i)] += 1;
    for (uint32_t g = 0; g < n_groups; g++)
        for (int j = 0; j < 64; j++) {
            i128 v = apx_side_value(&fin[g].side[0], j) - apx_side_value(&fin[g].side[1], j);
            out[(size_t)g * 64 + j] = cnt[g] ? 2.0 * i128_to_double(v) / (double)cnt[g] : 0.0;
        }
    free(fin); free(cnt);
    return status;
}

/* FLOAT state for DOUBLE sums, rows in order (Sec. 5 "Approximation"). */
int orc_approx_sum_f32state(const uint64_t *masks, const void *values,
                            int vtype, const void *gids, int gid_bytes,
                            size_t n, uint32_t n_groups, double *out) {
    float *st = (float *)calloc((size_t)n_groups * 64, sizeof(float));
    if (!st) return 2;
    for (size_t i = 0; i < n; i++) {
        uint32_t g = gid_at(gids, gid_bytes, i);
        float v = (float)fval_at(values, vtype, i);
        for (int j = 0; j < 64; j++)
            if ((masks[i] >> j) & 1ULL) st[(size_t)g * 64 + j] += v;
    }
    for (size_t k = 0; k < (size_t)n_groups * 64; k++) out[k] = (double)st[k];
    free(st);
    return 0;
}

/* ====================================================================== */
/* Finalize (reading R5/R6)                                                 */
/* ====================================================================== */

#define STREAM_JSTAR 0
#define STREAM_NULL 1
#define STREAM_NOISE 2
#define DIVERSITY_MIN_ROWS 64
#define DIVERSITY_MAX_WORLDS 40

double orc_release_scale(int kind, int variant) {
    (void)variant;
    /* pac_noised returns count[j*]*2 + noise: each world sees about half of
     * the tuples (Sec. 2).  SUM is the same kind of total (Sec. 5, two-sided
     * result 2*(C_pos - C_neg)).  AVG, MIN, MAX are not totals; the
     * approximate AVG already carries its factor 2 (reading R4). */
    return (kind == ORC_COUNT || kind == ORC_SUM) ? 2.0 : 1.0;
}

static void normalize_log(double *logp) {
    double mx = -INFINITY;
    for (int j = 0; j < 64; j++) if (logp[j] > mx) mx = logp[j];
    double s = 0.0;
    for (int j = 0; j < 64; j++) s += exp(logp[j] - mx);
    double lse = mx + log(s);
    for (int j = 0; j < 64; j++) logp[j] -= lse;
}

void orc_finalize(const double *y, const double *scale, uint32_t n_specs,
                  uint32_t n_groups, const uint64_t *meta_n,
                  const uint64_t *meta_or, uint64_t seed, double budget,
                  int mode, double *noised, uint8_t *is_null, uint32_t *flags,
                  double *posterior, int32_t *jstar_out) {
    /* secret world j*, shared by every cell of the query (Sec. 2) */
    int jstar = (int)(orc_rng_u64(seed, STREAM_JSTAR, 0) >> 58);
    if (jstar_out) *jstar_out = jstar;
    /* P_0 = P_S uniform (Sec. 4.1) */
    double logp[64];
    for (int j = 0; j < 64; j++) logp[j] = -log(64.0);

    size_t n_cells = (size_t)n_groups * n_specs;
    for (size_t c = 0; c < n_cells; c++) {
        uint32_t g = (uint32_t)(c / n_specs);
        uint32_t s = (uint32_t)(c % n_specs);
        uint64_t orm = meta_or[g];
        int pop = __builtin_popcountll(orm);
        uint32_t f = 0;
        if (meta_n[g] >= DIVERSITY_MIN_ROWS && pop <= DIVERSITY_MAX_WORLDS) f |= ORC_F_DIVERSITY;

        if (mode == ORC_INDEPENDENT)
            for (int j = 0; j < 64; j++) logp[j] = -log(64.0);

        /* NULL with probability (64 - popcount(K))/64, independent of j* */
        if (pop < 64 && (int)(orc_rng_u64(seed, STREAM_NULL, c) >> 58) < 64 - pop) {
            noised[c] = 0.0; is_null[c] = 1; flags[c] = f | ORC_F_NULL;
            continue;
        }
        is_null[c] = 0;

        /* the released vector: scaled, unset worlds treated as zeros */
        double yv[64];
        for (int j = 0; j < 64; j++)
            yv[j] = ((orm >> j) & 1ULL) ? scale[s] * y[c * 64 + j] : 0.0;

        /* step 1: variance of the outputs under the posterior P; exactly 0
         * when every world the posterior still allows has the same value */
        double p[64], mu = 0.0, var = 0.0;
        int all_equal = 1;
        for (int j = 0; j < 64; j++) p[j] = exp(logp[j]);
        for (int j = 0; j < 64; j++)
            if (p[j] > 0.0 && yv[j] != yv[jstar]) all_equal = 0;
        for (int j = 0; j < 64; j++) mu += p[j] * yv[j];
        for (int j = 0; j < 64; j++) var += p[j] * (yv[j] - mu) * (yv[j] - mu);
        if (all_equal) var = 0.0;
        /* step 2: calibrated noise variance */
        double delta = var / (2.0 * budget);
        /* step 3: release y_{j*} + N(0, delta) */
        double z = orc_box_muller(orc_rng_u64(seed, STREAM_NOISE, 2 * c),
                                  orc_rng_u64(seed, STREAM_NOISE, 2 * c + 1));
        double yt = yv[jstar] + sqrt(delta) * z;
        noised[c] = yt;
        /* step 4: Bayesian update P <- P . W / sum(P . W),
         * W_j = exp(-(yt - y_j)^2 / (2 delta)), in log space */
        if (delta > 0.0) {
            for (int j = 0; j < 64; j++) {
                double d = yt - yv[j];
                logp[j] += -(d * d) / (2.0 * delta);
            }
            normalize_log(logp);
        } else {
            f |= ORC_F_ZEROVAR;
        }
        flags[c] = f;
    }
    if (posterior)
        for (int j = 0; j < 64; j++) posterior[j] = exp(logp[j]);
}

/* ====================================================================== */
/* m = 128 worlds (reading R7).  The same definitions as above with a      */
/* 128-bit world mask, one row at a time, one world at a time.             */
/* ====================================================================== */

uint64_t orc_query_key2(uint64_t seed) {
    uint64_t s = seed ^ 0x5041435f4b455921ULL;
    (void)orc_splitmix64_next(&s);      /* K */
    return orc_splitmix64_next(&s);     /* K2 */
}

void orc_pac_hash128(int64_t key, uint64_t k1, uint64_t k2, int mode, uint64_t *out2) {
    uint64_t inner = orc_fmix64((uint64_t)key);
    uint64_t ha = orc_fmix64(inner ^ k1);
    uint64_t hb = orc_fmix64(inner ^ k2);
    if (mode == ORC_RAW) {
        out2[0] = ha;
        out2[1] = hb;
        return;
    }
    uint64_t w0 = (ha & 0xffffffffULL) | ((hb & 0xffffffffULL) << 32);
    out2[0] = w0;
    out2[1] = ~w0;
}

void orc_hash_keys128(const int64_t *keys, size_t n, uint64_t k1, uint64_t k2, int mode,
                      uint64_t *masks2) {
    for (size_t i = 0; i < n; i++) orc_pac_hash128(keys[i], k1, k2, mode, masks2 + 2 * i);
}

static int world128(const uint64_t *m2, int j) { return (int)((m2[j >> 6] >> (j & 63)) & 1ULL); }

int orc_aggregate128(const uint64_t *masks2, const void *values, int vtype, const void *gids,
                     int gid_bytes, size_t n, uint32_t n_groups, int kind, void *out,
                     uint64_t *meta_n, uint64_t *meta_or2) {
    int status = 0;
    acc_t *acc = (acc_t *)malloc(sizeof(acc_t) * (size_t)n_groups * 128);
    if (!acc) return 2;
    for (size_t k = 0; k < (size_t)n_groups * 128; k++) acc_init(&acc[k]);
    if (meta_n) memset(meta_n, 0, sizeof(uint64_t) * n_groups);
    if (meta_or2) memset(meta_or2, 0, sizeof(uint64_t) * 2 * n_groups);
    for (size_t i = 0; i < n; i++) {
        uint32_t g = gid_at(gids, gid_bytes, i);
        const uint64_t *m2 = masks2 + 2 * i;
        if (meta_n) meta_n[g] += 1;
        if (meta_or2) {
            meta_or2[2 * g] |= m2[0];
            meta_or2[2 * g + 1] |= m2[1];
        }
        for (int j = 0; j < 128; j++)
            if (world128(m2, j)) acc_update(&acc[(size_t)g * 128 + j], values, vtype, i);
    }
    for (size_t k = 0; k < (size_t)n_groups * 128; k++) acc_emit(&acc[k], vtype, kind, out, k, &status);
    free(acc);
    return status;
}

int orc_aggregate_brute128(const int64_t *keys, uint64_t k1, uint64_t k2, int mode, const void *values,
                           int vtype, const void *gids, int gid_bytes, size_t n, uint32_t n_groups,
                           int kind, void *out) {
    int status = 0;
    keyset universe;
    if (!ks_init(&universe, n)) return 2;
    for (size_t i = 0; i < n; i++) ks_insert(&universe, keys[i]);
    acc_t *acc = (acc_t *)malloc(sizeof(acc_t) * n_groups);
    if (!acc) { ks_free(&universe); return 2; }
    for (int j = 0; j < 128; j++) {
        /* step (1): the j-th sampled PU table */
        keyset sample;
        if (!ks_init(&sample, n)) { free(acc); ks_free(&universe); return 2; }
        for (size_t p = 0; p < universe.cap; p++) {
            if (!universe.used[p]) continue;
            uint64_t h2[2];
            orc_pac_hash128(universe.slot[p], k1, k2, mode, h2);
            if (world128(h2, j)) ks_insert(&sample, universe.slot[p]);
        }
        /* step (2): the query on the j-th sampled instance */
        for (uint32_t g = 0; g < n_groups; g++) acc_init(&acc[g]);
        for (size_t i = 0; i < n; i++)
            if (ks_contains(&sample, keys[i])) acc_update(&acc[gid_at(gids, gid_bytes, i)], values, vtype, i);
        for (uint32_t g = 0; g < n_groups; g++) acc_emit(&acc[g], vtype, kind, out, (size_t)g * 128 + j, &status);
        ks_free(&sample);
    }
    free(acc);
    ks_free(&universe);
    return status;
}

static void normalize_log128(double *logp) {
    double mx = -INFINITY;
    for (int j = 0; j < 128; j++) if (logp[j] > mx) mx = logp[j];
    double s = 0.0;
    for (int j = 0; j < 128; j++) s += exp(logp[j] - mx);
    double lse = mx + log(s);
    for (int j = 0; j < 128; j++) logp[j] -= lse;
}

void orc_finalize128(const double *y, const double *scale, uint32_t n_specs, uint32_t n_groups,
                     const uint64_t *meta_n, const uint64_t *meta_or2, uint64_t seed, double budget,
                     int mode, double *noised, uint8_t *is_null, uint32_t *flags, double *posterior,
                     int32_t *jstar_out) {
    int jstar = (int)(orc_rng_u64(seed, STREAM_JSTAR, 0) >> 57);   /* uniform on 0..127 */
    if (jstar_out) *jstar_out = jstar;
    double logp[128];
    for (int j = 0; j < 128; j++) logp[j] = -log(128.0);
    size_t n_cells = (size_t)n_groups * n_specs;
    for (size_t c = 0; c < n_cells; c++) {
        uint32_t g = (uint32_t)(c / n_specs);
        uint32_t s = (uint32_t)(c % n_specs);
        const uint64_t *orm = meta_or2 + 2 * g;
        int pop = __builtin_popcountll(orm[0]) + __builtin_popcountll(orm[1]);
        uint32_t f = 0;
        if (meta_n[g] >= DIVERSITY_MIN_ROWS && pop <= 2 * DIVERSITY_MAX_WORLDS) f |= ORC_F_DIVERSITY;
        if (mode == ORC_INDEPENDENT)
            for (int j = 0; j < 128; j++) logp[j] = -log(128.0);
        if (pop < 128 && (int)(orc_rng_u64(seed, STREAM_NULL, c) >> 57) < 128 - pop) {
            noised[c] = 0.0; is_null[c] = 1; flags[c] = f | ORC_F_NULL;
            continue;
        }
        is_null[c] = 0;
        double yv[128];
        for (int j = 0; j < 128; j++) yv[j] = world128(orm, j) ? scale[s] * y[c * 128 + j] : 0.0;
        double p[128], mu = 0.0, var = 0.0;
        int all_equal = 1;
        for (int j = 0; j < 128; j++) p[j] = exp(logp[j]);
        for (int j = 0; j < 128; j++)
            if (p[j] > 0.0 && yv[j] != yv[jstar]) all_equal = 0;
        for (int j = 0; j < 128; j++) mu += p[j] * yv[j];
        for (int j = 0; j < 128; j++) var += p[j] * (yv[j] - mu) * (yv[j] - mu);
        if (all_equal) var = 0.0;
        double delta = var / (2.0 * budget);
        double z = orc_box_muller(orc_rng_u64(seed, STREAM_NOISE, 2 * c),
                                  orc_rng_u64(seed, STREAM_NOISE, 2 * c + 1));
        double yt = yv[jstar] + sqrt(delta) * z;
        noised[c] = yt;
        if (delta > 0.0) {
            for (int j = 0; j < 128; j++) {
                double d = yt - yv[j];
                logp[j] += -(d * d) / (2.0 * delta);
            }
            normalize_log128(logp);
        } else {
            f |= ORC_F_ZEROVAR;
        }
        flags[c] = f;
    }
    if (posterior)
        for (int j = 0; j < 128; j++) posterior[j] = exp(logp[j]);
}
