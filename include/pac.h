/*
 * pac.h -- C ABI of the GB300 (sm_103a) PAC stochastic-aggregation library
 * (SIMD-PAC-DB, arXiv 2603.15023).
 *
 * The library computes the data-parallel hot path of SIMD-PAC-DB on one GPU:
 *   1. pac_hash_keys      PU key -> 64-bit world mask (Sec. 2 "SIMD-PAC-DB",
 *                         Sec. 4.2 "PAC Hash");
 *   2. pac_aggregate[_multi]
 *                         per-group, per-world COUNT/SUM/AVG/MIN/MAX over the
 *                         set bits of the mask (Sec. 4.2 "PAC Aggregation"),
 *                         exactly or in the approximate variants of Sec. 5
 *                         "Approximation";
 *   3. pac_finalize       variance of each cell's 64 world results under the
 *                         posterior and the PAC noise derived from it (Sec. 2
 *                         "PAC Privacy", Sec. 4.1 noise function steps 1-4,
 *                         Sec. 3.2 "NULLs", Sec. 5 "Diversity Check").
 *
 * Conventions shared by every entry point
 *   - m = 64 worlds: world j <-> bit j of the mask, 0 <= j < 64 (Sec. 5).
 *   - Per-world results are row-major [n_groups][64].
 *   - Unless stated otherwise, data pointers are DEVICE pointers owned by the
 *     caller; the library never frees them and never keeps them after the
 *     call returns.  Calls are asynchronous on the given stream (a
 *     cudaStream_t; NULL = legacy default stream).
 *   - Argument errors are found on the host before any launch and return
 *     PAC_E_INVALID or PAC_E_UNSUPPORTED with nothing enqueued.  Conditions
 *     only the device can see (an exact integer SUM that does not fit int64,
 *     an approximate cascade past its last level, a device wait that timed
 *     out) are recorded in the context's device status word and returned by
 *     the next pac_sync_status().
 *   - No C++ exception crosses this boundary.  A context is used by one host
 *     thread at a time.
 */
#ifndef PAC_H
#define PAC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *pac_stream; /* same type as cudaStream_t */
typedef struct pac_ctx pac_ctx;

typedef enum {
    PAC_OK = 0,
    PAC_E_INVALID = 1,     /* bad argument: null pointer, size, enum value */
    PAC_E_NOMEM = 2,       /* device or host allocation failed */
    PAC_E_CUDA = 3,        /* a CUDA runtime call failed (see pac_last_error) */
    PAC_E_OVERFLOW = 4,    /* a result did not fit its output type */
    PAC_E_TIMEOUT = 5,     /* a bounded device wait gave up */
    PAC_E_UNSUPPORTED = 6  /* valid request this build does not serve */
} pac_status;

/* Aggregates of Sec. 4.2 "PAC Aggregation": agg in {sum,count,avg,min,max}. */
/* PAC_LIFTED (not an aggregate): a vector-lifted expression's [n_groups*64]
 * double result from pac_lift, released by pac_finalize with scale 1. */
typedef enum { PAC_COUNT = 0, PAC_SUM = 1, PAC_AVG = 2, PAC_MIN = 3, PAC_MAX = 4, PAC_LIFTED = 5 } pac_kind;

/* Value column types. */
typedef enum { PAC_I64 = 0, PAC_F32 = 1, PAC_F64 = 2 } pac_dtype;

/* PAC_EXACT: r_j = agg{e(t) : pu[j] = 1} exactly (integers bit-exact; float
 * SUM in FP32 with compensated two-sum partials, within 1e-6 relative of the
 * FP64 sum).  PAC_APPROX: the paper's approximate variants (Sec. 5
 * "Approximation"): integer SUM/AVG through 25 levels of 16-bit counters
 * cascading every 4 bits, two-sided; float SUM with plain FLOAT state. */
typedef enum { PAC_EXACT = 0, PAC_APPROX = 1 } pac_variant;

/* PAC_HASH_BALANCED: every PU lies in exactly 32 worlds (Sec. 2: a hash with
 * guaranteed 32 one-bits); worlds j and j+32 are complements.
 * PAC_HASH_RAW: the 64 bits of the keyed hash (binomial popcount). */
typedef enum { PAC_HASH_BALANCED = 0, PAC_HASH_RAW = 1 } pac_hash_mode;

/* PAC_FIN_ADAPTIVE: the posterior over the secret world is updated after
 * every release (Sec. 2, adaptive composition; Sec. 4.1 step 4).
 * PAC_FIN_INDEPENDENT: every cell is noised under the uniform prior (not the
 * paper's composition; offered for independent releases). */
typedef enum { PAC_FIN_ADAPTIVE = 0, PAC_FIN_INDEPENDENT = 1 } pac_fin_mode;

/* Input selector for pac_aggregate*: the first column holds PU keys (int64,
 * hashed inside the aggregation with query_key and hash_mode) or already
 * computed world masks (uint64, e.g. from pac_hash_keys). */
#define PAC_IN_KEYS 0u
#define PAC_IN_MASKS 1u
/* Or-ed into in_flags: a row whose world mask is 0 is a row of no group --
 * it is skipped like a filtered row and not counted in meta's n_g (the
 * paper's engine drops rows whose updated pu is 0 before the aggregate,
 * Sec. 3.2 "Categorical Rewrites").  Not taken by pac_aggregate_noalloc. */
#define PAC_IN_DROP_EMPTY 2u

/* Per-cell flags written by pac_finalize. */
#define PAC_F_NULL 1u      /* released NULL (Sec. 3.2 "NULLs") */
#define PAC_F_DIVERSITY 2u /* >= 64 rows but <= 40 worlds ever updated (Sec. 5) */
#define PAC_F_ZEROVAR 4u   /* variance under the posterior was exactly 0 */

/* ---------------------------------------------------------------------------
 * Context.  Owns device workspace (grown on demand, freed by pac_destroy),
 * a device status word and the last error message.  `device` is the CUDA
 * ordinal the context's launches use; it is made current in every call.
 * ------------------------------------------------------------------------ */
pac_status pac_create(pac_ctx **ctx, int device);
void pac_destroy(pac_ctx *ctx);
const char *pac_last_error(const pac_ctx *ctx);
const char *pac_status_string(pac_status s);

/* Synchronises `stream`, returns (and clears) the device status word:
 * PAC_OK, PAC_E_OVERFLOW, PAC_E_TIMEOUT, or PAC_E_INVALID when a group id
 * was >= n_groups or a selection's operand id was >= n_thr (such rows are
 * skipped / keep no world, never read or written out of bounds).
 * PAC_E_OVERFLOW: an exact int64 SUM did not fit.  The tensor-core and
 * one-launch paths (agg_path 2 and 4) keep 128-bit totals: a SUM that does
 * not fit is saturated to INT64_MIN / INT64_MAX, and AVG is still the exact
 * total over the count.  The per-bit kernels keep 64-bit partial sums; after
 * an overflow report their SUM and AVG outputs are unspecified. */
pac_status pac_sync_status(pac_ctx *ctx, pac_stream stream);

/* Host-only: the per-query hash key K (Sec. 4.2: drawn independently per
 * query) for a query seed: the first SplitMix64 output of seed XOR the
 * ASCII tag "PAC_KEY!". */
uint64_t pac_query_key(uint64_t seed);

/* ---------------------------------------------------------------------------
 * 1. pac_hash_keys  (Sec. 2 "SIMD-PAC-DB"; Sec. 4.2 "PAC Hash")
 *   keys  [n] int64 PU keys (device); masks [n] uint64 out (device).
 *   mask = balance(fmix64(fmix64(key) XOR query_key)), fmix64 being
 *   MurmurHash3's 64-bit finalizer; balance keeps the low 32 bits and puts
 *   their complement in the high 32 (PAC_HASH_BALANCED) or is the identity
 *   (PAC_HASH_RAW).  n = 0 is a no-op.  keys and masks may alias.
 * ------------------------------------------------------------------------ */
pac_status pac_hash_keys(pac_ctx *ctx, const int64_t *keys, uint64_t *masks, size_t n,
                         uint64_t query_key, int32_t hash_mode, pac_stream stream);

/* ---------------------------------------------------------------------------
 * 2. pac_aggregate / pac_aggregate_multi  (Sec. 4.2 "PAC Aggregation";
 *    Sec. 5 for the approximate variants; Sec. 3.2 "NULLs" for meta)
 *
 * Shared input of one query:
 *   keys_or_masks [n] int64 keys (PAC_IN_KEYS) or uint64 masks (PAC_IN_MASKS)
 *   group_ids     [n] unsigned group id of width gid_bytes (1, 2 or 4), each
 *                 < n_groups; NULL means ungrouped (n_groups must be 1 unless
 *                 n = 0)
 *   n             rows (0 allowed: every output is zero)
 *   n_groups      >= 1
 * One aggregate per spec:
 *   values  [n] column of vtype (ignored, may be NULL, for PAC_COUNT)
 *   out     [n_groups*64] results, type by kind:
 *             COUNT                      -> uint64
 *             SUM, MIN, MAX over PAC_I64 -> int64 (SUM exact; APPROX SUM is
 *                                           the unscaled two-sided sum)
 *             AVG (any), SUM/MIN/MAX over floats -> double
 *           An empty world gives 0 for every kind (Sec. 3.2: unset worlds
 *           count as zeros).
 * meta (optional, may be NULL): [n_groups*2] uint64 {rows n_g, OR of the
 *   masks of the group's rows}, the NULL accumulator of Sec. 3.2.
 * Supported: every kind/vtype with PAC_EXACT; PAC_APPROX for SUM and AVG
 * over PAC_I64 (25-level cascade) and SUM over floats (FLOAT state).
 * ------------------------------------------------------------------------ */
typedef struct {
    const void *keys_or_masks;
    uint32_t in_flags;     /* PAC_IN_KEYS or PAC_IN_MASKS */
    int32_t hash_mode;     /* pac_hash_mode, used with PAC_IN_KEYS */
    uint64_t query_key;    /* K, used with PAC_IN_KEYS */
    const void *group_ids; /* NULL = ungrouped */
    int32_t gid_bytes;     /* 1, 2 or 4 (ignored when ungrouped) */
    uint32_t n_groups;
    size_t n;
} pac_input;

typedef struct {
    int32_t kind;       /* pac_kind */
    int32_t variant;    /* pac_variant */
    int32_t vtype;      /* pac_dtype of values */
    int32_t reserved;   /* must be 0 */
    const void *values; /* device [n] */
    void *out;          /* device [n_groups*64]; an input of pac_finalize */
} pac_agg_spec;

#define PAC_MAX_SPECS 16

pac_status pac_aggregate(pac_ctx *ctx, const void *keys_or_masks, uint32_t in_flags,
                         uint64_t query_key, int32_t hash_mode, const void *values,
                         int32_t vtype, const void *group_ids, int32_t gid_bytes, size_t n,
                         uint32_t n_groups, int32_t kind, int32_t variant, void *out,
                         uint64_t *meta, pac_stream stream);

/* Several aggregates over one pass of the shared key/group columns
 * (n_specs <= PAC_MAX_SPECS; specs is a HOST array). */
pac_status pac_aggregate_multi(pac_ctx *ctx, const pac_input *in, const pac_agg_spec *specs,
                               int32_t n_specs, uint64_t *meta, pac_stream stream);

/* ---------------------------------------------------------------------------
 * 2b. pac_select  (Sec. 4.2 "PAC Selection" and compiler step (3); Sec. 3.2
 *     "Categorical Rewrites": pac_select and the fused pac_select_<cmp>)
 *
 * A selection whose predicate depends on an aggregate computed per world
 * (a correlated subquery, e.g. col < 0.2 * avg(col) of the row's part)
 * updates the PU column: world j of row i is kept iff it was set and
 *   col[i] <cmp> thr[t_i][j]
 * holds.  thr is a [n_thr][64] table of per-world operands (typically a
 * pac_aggregate result, one row per correlation key); t_i = thr_ids[i]
 * picks the row's operand vector (thr_ids NULL and n_thr = 1: one vector
 * for every row).
 *   col, thr     [n] / [n_thr*64] of vtype (PAC_I64 compares as int64,
 *                PAC_F32 / PAC_F64 as IEEE values: every comparison with a
 *                NaN is false except PAC_CMP_NE)
 *   thr_ids      [n] unsigned, width thr_id_bytes (1, 2 or 4), each < n_thr;
 *                a row whose id is out of range keeps no world and the next
 *                pac_sync_status returns PAC_E_INVALID
 * ------------------------------------------------------------------------ */
typedef enum {
    PAC_CMP_LT = 0, /* col <  thr */
    PAC_CMP_LE = 1, /* col <= thr */
    PAC_CMP_EQ = 2, /* col == thr */
    PAC_CMP_NE = 3, /* col != thr */
    PAC_CMP_GT = 4, /* col >  thr */
    PAC_CMP_GE = 5  /* col >= thr */
} pac_cmp;

typedef struct {
    const void *col;      /* device [n], vtype */
    int32_t vtype;        /* pac_dtype of col and thr */
    int32_t cmp;          /* pac_cmp */
    const void *thr;      /* device [n_thr*64], vtype, row-major [t][j] */
    uint32_t n_thr;       /* >= 1 */
    int32_t thr_id_bytes; /* 1, 2 or 4; ignored when thr_ids is NULL */
    const void *thr_ids;  /* device [n] or NULL (then n_thr must be 1) */
} pac_select_spec;

/* masks_out[i] = mask_i AND {j : col[i] <cmp> thr[t_i][j]}, mask_i hashed
 * from the keys (PAC_IN_KEYS) or read (PAC_IN_MASKS); in->group_ids and
 * n_groups are not used.  masks_out: caller-owned device [n]. */
pac_status pac_select(pac_ctx *ctx, const pac_input *in, const pac_select_spec *sel, uint64_t *masks_out,
                      pac_stream stream);

/* pac_aggregate_multi over the selected rows: the masks of pac_select, and
 * rows whose selected mask is 0 dropped (PAC_IN_DROP_EMPTY).  The selected
 * masks live in the context's workspace; nothing is written to the caller's
 * columns. */
pac_status pac_aggregate_select(pac_ctx *ctx, const pac_input *in, const pac_select_spec *sel,
                                const pac_agg_spec *specs, int32_t n_specs, uint64_t *meta,
                                pac_stream stream);

/* ---------------------------------------------------------------------------
 * 3. pac_finalize  (Sec. 2 "PAC Privacy" and fused pac_noised_count;
 *    Sec. 4.1 noise function steps 1-4; Sec. 3.2 "NULLs"; Sec. 5
 *    "Diversity Check")
 *
 * Releases every cell of one query: cell c = g*n_specs + s, for group g and
 * spec s (specs: the HOST array given to pac_aggregate_multi, whose `out`
 * buffers hold the 64 world results).  meta: the device {n_g, or_g} array
 * filled by the aggregation.  For each cell, in that order:
 *   NULL with probability (64 - popcount(or_g))/64 (no posterior update);
 *   y_j = scale * r_j for worlds in or_g, 0 for the others, scale 2 for
 *   COUNT and SUM (count[j*]*2 of Sec. 2) and 1 otherwise;
 *   s^2 = Var_{j~P}[y_j]; Delta = s^2/(2*budget);
 *   release y_{j*} + sqrt(Delta)*z, z standard normal;
 *   P <- P*W/sum(P*W), W_j = exp(-(release - y_j)^2/(2*Delta))
 *   (PAC_FIN_ADAPTIVE only).
 * The secret world j*, the NULL draws and z come from one counter-based
 * SplitMix64 generator keyed by `seed` (draw i of stream t is output i of
 * SplitMix64 started at output t of SplitMix64(seed); streams 0: j*,
 * 1: NULL, 2: Box-Muller pairs).  budget > 0 is the per-cell MI budget B.
 * Outputs (device): noised[n_cells] (0 for NULL cells), is_null[n_cells],
 * flags[n_cells] (PAC_F_*), posterior[64] final P (may be NULL).
 * ------------------------------------------------------------------------ */
pac_status pac_finalize(pac_ctx *ctx, const pac_agg_spec *specs, int32_t n_specs,
                        uint32_t n_groups, const uint64_t *meta, uint64_t seed, double budget,
                        int32_t mode, double *noised, uint8_t *is_null, uint32_t *flags,
                        double *posterior, pac_stream stream);

/* ---------------------------------------------------------------------------
 * 3b. pac_lift  (Sec. 4.2 "Vector-lifted Expression, and Lambda Functions";
 *     Sec. 7: a ratio of two pac_sum vectors evaluated world by world and
 *     noised once)
 *
 * out[g][j] = e(x_1[g][j], ..., x_a[g][j]): a scalar expression applied to
 * world j of every operand, scalar operands broadcast to all 64 worlds.  The
 * expression is a postfix program over a stack of doubles (at most
 * PAC_LIFT_DEPTH values, at most PAC_LIFT_MAX_OPS operations):
 *   PAC_LIFT_SPEC k   push world j of specs[k] times its release scale
 *                     (2 for COUNT and SUM, 1 otherwise: the estimate a
 *                     pac_finalize release of that spec is centred on)
 *   PAC_LIFT_CONST    push c
 *   ADD SUB MUL DIV   pop b, pop a, push a op b (IEEE double: x/0 is +-inf
 *                     or NaN)
 *   MIN MAX           a < b ? a : b, a > b ? a : b
 *   NEG ABS           on the top value
 *   LT LE EQ NE GT GE push 1.0 if a <cmp> b else 0.0 (lifted booleans)
 * specs: HOST array (kind, vtype, out) of the operand vectors (aggregate
 * outputs, or earlier lifted vectors with kind PAC_LIFTED, vtype PAC_F64);
 * out: device [n_groups*64] doubles.  A malformed program (underflow, more
 * than one value left, a missing spec) is PAC_E_INVALID.  Release the result
 * with pac_finalize and a spec {PAC_LIFTED, PAC_EXACT, PAC_F64, -, out},
 * with the meta of the query it came from (its NULL accumulator).
 * ------------------------------------------------------------------------ */
typedef enum {
    PAC_LIFT_SPEC = 0, PAC_LIFT_CONST = 1, PAC_LIFT_ADD = 2, PAC_LIFT_SUB = 3, PAC_LIFT_MUL = 4,
    PAC_LIFT_DIV = 5, PAC_LIFT_NEG = 6, PAC_LIFT_ABS = 7, PAC_LIFT_MIN = 8, PAC_LIFT_MAX = 9,
    PAC_LIFT_LT = 10, PAC_LIFT_LE = 11, PAC_LIFT_EQ = 12, PAC_LIFT_NE = 13, PAC_LIFT_GT = 14,
    PAC_LIFT_GE = 15
} pac_lift_opcode;

typedef struct {
    int32_t op;  /* pac_lift_opcode */
    int32_t arg; /* spec index for PAC_LIFT_SPEC */
    double c;    /* constant for PAC_LIFT_CONST */
} pac_lift_op;

#define PAC_LIFT_DEPTH 8
#define PAC_LIFT_MAX_OPS 32

pac_status pac_lift(pac_ctx *ctx, const pac_agg_spec *specs, int32_t n_specs, uint32_t n_groups,
                    const pac_lift_op *prog, int32_t n_ops, double *out, pac_stream stream);

/* ---------------------------------------------------------------------------
 * 3c. pac_filter  (Sec. 3.2 "Categorical Rewrites": probabilistic filtering
 *     of a WHERE condition on aggregates)
 *
 * b: device [n_groups*64] lifted booleans (a world is true when non-zero).
 * keep[g] = 1 with probability (#true worlds of g)/64: keep[g] = u_g <
 * #true/64 with u_g uniform in [0,1) from the counter generator of `seed`
 * (stream 3, counter g).  The choice does not depend on the secret world
 * and updates no posterior.  keep: device [n_groups] bytes.
 * ------------------------------------------------------------------------ */
pac_status pac_filter(pac_ctx *ctx, const double *b, uint32_t n_groups, uint64_t seed, uint8_t *keep,
                      pac_stream stream);

/* ---------------------------------------------------------------------------
 * End-to-end query from HOST memory: copies the columns named by `in` and
 * `specs` (HOST pointers, ideally pinned) into context-owned device
 * workspace, runs pac_aggregate_multi and pac_finalize there, and copies the
 * released cells back into HOST noised/is_null/flags (n_groups*n_specs
 * each).  The specs' `out` fields are ignored (results live in workspace).
 * Synchronous: returns after the results are on the host, with the device
 * status folded into the return value.
 * ------------------------------------------------------------------------ */
pac_status pac_query_host(pac_ctx *ctx, const pac_input *in, const pac_agg_spec *specs,
                          int32_t n_specs, uint64_t seed, double budget, int32_t mode,
                          double *noised, uint8_t *is_null, uint32_t *flags, pac_stream stream);

/* ---------------------------------------------------------------------------
 * 4. Batched queries: thousands of independent PAC queries (each one the
 *    aggregation of Sec. 4.2 over its own columns, then optionally the
 *    release of Sec. 2 / Sec. 4.1 steps 1-4 over its own cells) in one
 *    persistent aggregation launch.
 *
 * A query of a batch.  `in` and the specs' `values`/`out` are as for
 * pac_aggregate_multi (DEVICE buffers owned by the caller, HOST structs).
 * Every spec must be PAC_EXACT (the approximate integer cascade has its own
 * schedule and runs only through pac_aggregate_multi).
 *   meta      device [n_groups*2] {n_g, or_g}, or NULL (then fin_mode must
 *             be -1).
 *   fin_mode  PAC_FIN_ADAPTIVE or PAC_FIN_INDEPENDENT to release the query's
 *             cells like pac_finalize(seed, budget) would, or -1 for the
 *             aggregation alone.
 *   noised, is_null, flags  device [n_groups*n_specs] release outputs (used
 *             when fin_mode >= 0).
 * ------------------------------------------------------------------------ */
typedef struct {
    pac_input in;
    const pac_agg_spec *specs; /* HOST array of n_specs (1..PAC_MAX_SPECS) */
    int32_t n_specs;
    int32_t fin_mode;
    uint64_t *meta;
    uint64_t seed;
    double budget;
    double *noised;
    uint8_t *is_null;
    uint32_t *flags;
} pac_query;

typedef struct pac_batch pac_batch;

/* Plan flags. */
#define PAC_BATCH_AUTOTUNE 1u /* time candidate work-item sizes and state
                                 placements on this batch and keep the fastest
                                 (the choice is cached in the context) */

/* Plans a batch: checks every query (PAC_E_INVALID / PAC_E_UNSUPPORTED name
 * the first bad query in pac_last_error), chooses per query where its
 * per-world states live (warp-private shared memory or global atomics),
 * cuts all queries into work items and uploads the descriptors once into
 * plan-owned device memory.  Synchronous.  The specs arrays are copied; the
 * device buffers they name must stay valid while the plan is launched.
 * With PAC_BATCH_AUTOTUNE the candidate configurations are launched on this
 * batch (writing its outputs) and timed. */
pac_status pac_batch_plan(pac_ctx *ctx, const pac_query *queries, int32_t n_queries, uint32_t flags,
                          pac_batch **plan);

/* Enqueues the whole batch on `stream`: one memset of the plan's scratch,
 * one persistent aggregation kernel over every query's work items (dynamic
 * scheduling), one merge kernel that writes every query's outputs and meta,
 * and, if any query releases, one finalize kernel (one warp per query).  No
 * allocation, no host synchronisation: the launch can be captured in a CUDA
 * graph and replayed.  Device conditions (overflow, bad group ids) go to the
 * context's status word (pac_sync_status).  Launches of one plan must not
 * overlap on the GPU (they share the plan's scratch). */
pac_status pac_batch_launch(pac_ctx *ctx, pac_batch *plan, pac_stream stream);

/* Frees a plan (synchronises the device first).  NULL is a no-op. */
void pac_batch_free(pac_batch *plan);

/* Plan introspection: "n_items", "item_rows", "smem_cap", "kernels"
 * (kernels per launch), "n_warp_private" (queries with shared-memory
 * states), "n_atomic" (queries with global-atomic states). */
pac_status pac_batch_info(const pac_batch *plan, const char *name, int64_t *value);

/* Plan + launch + synchronise + free.  Returns the device status. */
pac_status pac_batch_run(pac_ctx *ctx, const pac_query *queries, int32_t n_queries, pac_stream stream);

/* ---------------------------------------------------------------------------
 * 5. Serving: continuous batching of incoming PAC queries (each one a
 *    pac_query as above: aggregation of Sec. 4.2, release of Sec. 2 /
 *    Sec. 4.1 when fin_mode >= 0).
 *
 * A server owns a worker thread, a device-memory arena of cfg.mem_budget
 * bytes for the plans of admitted queries (their per-world states, partials
 * and descriptors), a pinned staging area and cfg.n_streams CUDA streams.
 * Submitted queries wait in arrival order; the worker admits as many as the
 * arena's free space, cfg.max_inflight and cfg.max_batch allow as soon as
 * one of its streams is idle, plans them as one batch inside the arena, and
 * enqueues it on that stream, so batches admitted while others run overlap
 * on the device and arrivals during busy periods are batched together.  Completion is
 * stamped on the host by a stream callback; the ticket's latency is from
 * pac_serve_submit to that stamp.  The query's column buffers must stay
 * valid and unmodified, and its output buffers untouched, until the ticket
 * is done.  All entry points are thread-safe.
 * ------------------------------------------------------------------------ */
typedef struct {
    size_t mem_budget;    /* arena bytes for admitted plans (> 0) */
    int32_t max_inflight; /* admitted, unfinished queries at most (>= 1) */
    int32_t max_batch;    /* queries per launch at most (>= 1) */
    int32_t n_streams;    /* streams carrying launches (1..32); a batch is
                             launched only when a stream is idle, with
                             everything queued (up to max_batch) */
    int32_t reserved;     /* must be 0 */
} pac_serve_config;

typedef struct pac_server pac_server;

/* Creates a server on ctx's device (the server keeps its own context). */
pac_status pac_serve_create(pac_ctx *ctx, const pac_serve_config *cfg, pac_server **srv);

/* Queues a copy of *q (its specs array is copied too) and returns its
 * ticket.  PAC_E_INVALID / PAC_E_UNSUPPORTED as pac_batch_plan for a bad
 * query; PAC_E_NOMEM when the query alone needs more than the arena. */
pac_status pac_serve_submit(pac_server *srv, const pac_query *q, uint64_t *ticket);

/* Non-blocking: *done = 1 once the ticket's results are in its output
 * buffers (then *latency_ms, if not NULL, is its latency and the ticket is
 * forgotten), else 0.  Returns the ticket's device status once done. */
pac_status pac_serve_poll(pac_server *srv, uint64_t ticket, int32_t *done, double *latency_ms);

/* Blocks until the ticket is done; as pac_serve_poll otherwise. */
pac_status pac_serve_wait(pac_server *srv, uint64_t ticket, double *latency_ms);

/* Server statistics over completed tickets: "completed", "batches",
 * "mean_batch" (queries per launch), "p50_ms", "p99_ms", "max_ms",
 * "max_inflight_seen", "arena_high_water" (bytes), "max_device_overlap"
 * (the most batches whose aggregation kernels were running on the GPU at one
 * instant, from device-timer stamps the kernels record). */
pac_status pac_serve_stats(pac_server *srv, const char *name, double *value);

/* Finishes every queued and running query, then frees the server. */
void pac_serve_destroy(pac_server *srv);

/* ---------------------------------------------------------------------------
 * pac_aggregate_noalloc -- the paper has no counterpart: this is a service
 * of the library for callers that cannot allocate device memory.
 *
 * Some callers cannot call cudaMalloc: code that runs under a memory pool
 * owning all device memory (a database engine's buffer manager, a
 * framework's caching allocator) and code with a device-memory budget fixed
 * before it starts, where an allocation could fail or stall the device at
 * the wrong time.  This entry point computes what pac_aggregate_multi
 * computes for COUNT and exact int64 SUM/AVG specs (the tensor-core path:
 * at most 4 distinct value columns and 8 groups) without any allocation:
 * it never calls cudaMalloc, cudaFree or an allocating library routine and
 * needs no pac_ctx.  Its scratch is a fixed 263,168-byte __device__ array
 * (plus a 4-byte status word) that every GPU which loads the library holds
 * until the process exits.
 *   in, specs, n_specs, meta: as pac_aggregate_multi (HOST structs, DEVICE
 *       buffers owned by the caller).
 *   stream: work is enqueued on it; the call synchronises it before
 *       returning, then returns the device status (PAC_E_OVERFLOW for an
 *       int64 overflow, PAC_E_INVALID for a group id >= n_groups).
 *   err, err_len: optional HOST buffer for a message (may be NULL).
 * Returns PAC_E_UNSUPPORTED for specs the tensor-core path does not serve
 * (whatever n, so n = 0 is refused for them too).  A query that would need
 * more scratch than the array holds is refused with PAC_E_INVALID; within
 * the limits above none does (the array is sized for the largest).  Every
 * failure writes a message into err.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current) and keeps it for the process: make that
 * first call before any stream capture, and do not use this entry point
 * across cudaDeviceReset.  The call synchronises `stream` before returning.
 * Every call shares the one array and its contents persist between calls
 * (each call clears what must start at zero): calls whose work overlaps on
 * the same GPU (other host threads, other streams) race and must be
 * serialised by the caller.
 * ------------------------------------------------------------------------ */
pac_status pac_aggregate_noalloc(const pac_input *in, const pac_agg_spec *specs, int32_t n_specs,
                                 uint64_t *meta, pac_stream stream, char *err, size_t err_len);

/* ---------------------------------------------------------------------------
 * 6. m = 128 worlds  (Sec. 2 "SIMD-PAC-DB": m = 64 is the paper's choice,
 *    m = 128 is possible with twice the state; the cost at most doubles)
 *
 * A PU's membership in 128 worlds comes from two keyed re-hashes of the same
 * engine hash, h_a = fmix64(fmix64(key) ^ K) and h_b = fmix64(fmix64(key) ^
 * K2), K2 being the SplitMix64 output after K (pac_query_key2).  Mask word 0
 * holds worlds 0..63, word 1 worlds 64..127:
 *   PAC_HASH_BALANCED: word 0 = low 32 bits of h_a | (low 32 bits of h_b)
 *                      << 32, word 1 = ~word 0 (every PU in exactly 64
 *                      worlds; world 64 + j is the complement of world j);
 *   PAC_HASH_RAW:      word 0 = h_a, word 1 = h_b.
 * Everything else is the m = 64 definition with 128 worlds: results are
 * row-major [n_groups][128]; meta is [n_groups][3] {n_g, OR of mask word 0,
 * OR of mask word 1}.
 * ------------------------------------------------------------------------ */

/* Host-only: K2 for a query seed (the SplitMix64 output after K). */
uint64_t pac_query_key2(uint64_t seed);

/* masks: device [n][2] uint64 (word 0, word 1 of each row); keys: device
 * [n] int64.  n = 0 is a no-op.  keys and masks must not overlap. */
pac_status pac_hash_keys128(pac_ctx *ctx, const int64_t *keys, uint64_t *masks, size_t n,
                            uint64_t query_key, uint64_t query_key2, int32_t hash_mode,
                            pac_stream stream);

/* pac_aggregate_multi over 128 worlds.  in->keys_or_masks: [n] int64 keys
 * (PAC_IN_KEYS, hashed with in->query_key and query_key2) or [n][2] uint64
 * masks (PAC_IN_MASKS).  Every exact kind and vtype is served
 * (PAC_E_UNSUPPORTED for PAC_APPROX and PAC_IN_DROP_EMPTY).  specs[i].out:
 * device [n_groups*128] of the kind's output type; meta: device
 * [n_groups*3] or NULL.  COUNT and exact int64 SUM/AVG over at most 8 groups
 * and 4 value columns run on the tensor cores with 128-row accumulator
 * tiles; the other queries run the per-bit engine on each 64-world half. */
pac_status pac_aggregate128(pac_ctx *ctx, const pac_input *in, uint64_t query_key2,
                            const pac_agg_spec *specs, int32_t n_specs, uint64_t *meta,
                            pac_stream stream);

/* pac_finalize over 128 worlds: the release of every cell (Sec. 4.1 steps
 * 1-4, Sec. 3.2 NULLs) with j* the top 7 bits of the first draw of stream 0,
 * a uniform prior over 128 worlds, a cell NULL with probability
 * (128 - popcount(or_g))/128, the diversity flag at >= 64 rows and <= 80
 * updated worlds.  meta: device [n_groups*3] from pac_aggregate128;
 * posterior: device [128] or NULL. */
pac_status pac_finalize128(pac_ctx *ctx, const pac_agg_spec *specs, int32_t n_specs, uint32_t n_groups,
                           const uint64_t *meta, uint64_t seed, double budget, int32_t mode,
                           double *noised, uint8_t *is_null, uint32_t *flags, double *posterior,
                           pac_stream stream);

/* ---------------------------------------------------------------------------
 * Path selection and introspection (for benchmarks and tests).
 *   pac_set_option(ctx, name, value): "agg_path" 0 = automatic (the
 *   one-launch path for ungrouped COUNT / exact int64 SUM / AVG queries of at
 *   most 8M rows, the tensor-core path where it applies, else the per-bit
 *   engine), 1 = force the plain per-bit CUDA-core kernels, 2 = force the
 *   tensor-core path (PAC_E_UNSUPPORTED where it cannot serve), 3 = force the
 *   per-bit engine (warp bit-transpose; the engine of the batched path),
 *   4 = force the one-launch path (one group, COUNT / exact int64 SUM / AVG
 *   over at most 4 value columns, any row count; PAC_E_UNSUPPORTED
 *   otherwise), 5 = force the many-group tensor-core path (rows partitioned
 *   into group order, then tensor-core sums over the group-ordered rows;
 *   COUNT and exact int64 SUM / AVG of one value column, any group count;
 *   PAC_E_UNSUPPORTED otherwise).  The automatic choice takes path 5 above
 *   64 groups when it can serve the query.  The one-launch path keeps its
 *   accumulators in the context, so calls on one context must not overlap.
 *   "minmax_prune" 1 (default) = MIN/MAX bound pruning on the per-bit
 *   engine (Sec. 5 "Pruning": rows whose value improves no world's current
 *   extreme skip the update; results are identical), 0 = every row updated.
 *   Plans built by pac_batch_plan take the setting current at plan time.
 *   "wait_limit_ns" (for tests of the give-up path): the wall-time limit of
 *   the tensor-core kernel's pipeline waits, 0 (default) = 2 s.  A wait that
 *   runs out stops the kernel's tensor-core work, its results are discarded
 *   and the next pac_sync_status returns PAC_E_TIMEOUT; a very short limit
 *   makes ordinary launches run out.  The kernel's final wait for its own
 *   tensor-core operations keeps the 2 s limit.
 *   pac_get_info(ctx, name, &value): "last_path" (1 plain per-bit, 2 tensor
 *   core, 3 per-bit engine, 4 one-launch, 5 many-group tensor core),
 *   "last_launches" kernels launched by the last call.
 * ------------------------------------------------------------------------ */
pac_status pac_set_option(pac_ctx *ctx, const char *name, int64_t value);
pac_status pac_get_info(pac_ctx *ctx, const char *name, int64_t *value);

#ifdef __cplusplus
}
#endif
#endif /* PAC_H */
