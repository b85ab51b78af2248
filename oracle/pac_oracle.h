/*
 * pac_oracle.h -- plain scalar CPU oracle for PAC stochastic aggregation
 * (SIMD-PAC-DB, arXiv 2603.15023).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline / reference legs of the benchmark may load this library.  The
 * product path (the CUDA library and its Python binding) never links, imports
 * or calls it, and it shares no code, header, table or constant generator
 * with the CUDA path.
 *
 * Everything here is written to be checked against the paper by eye: one row
 * at a time, one world at a time, 128-bit integers for exact sums and FP64 for
 * floating point.  No blocking, fusion or reordering beyond what the cited
 * definitions state.
 *
 * Conventions
 *   m = 64 possible worlds; world j <-> bit j of a 64-bit mask, 0 <= j < 64
 *   (Sec. 5, first paragraph).
 *   Per-world outputs are row-major [n_groups][64].
 *   Status: 0 ok, 4 overflow (a result did not fit its output type).
 */
#ifndef PAC_ORACLE_H
#define PAC_ORACLE_H
#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- aggregate kinds / value types / variants (oracle-local numbering) --- */
enum { ORC_COUNT = 0, ORC_SUM = 1, ORC_AVG = 2, ORC_MIN = 3, ORC_MAX = 4, ORC_LIFTED = 5 };
enum { ORC_I64 = 0, ORC_F32 = 1, ORC_F64 = 2 };
enum { ORC_EXACT = 0, ORC_APPROX = 1 };
enum { ORC_BALANCED = 0, ORC_RAW = 1 };
enum { ORC_ADAPTIVE = 0, ORC_INDEPENDENT = 1 };

/* flags written per finalized cell */
#define ORC_F_NULL      1u
#define ORC_F_DIVERSITY 2u
#define ORC_F_ZEROVAR   4u

/* ---- hashing (Sec. 2 "SIMD-PAC-DB", Sec. 4.2 "PAC Hash") ----------------- */
uint64_t orc_fmix64(uint64_t k);
uint64_t orc_fmix64_inverse(uint64_t h);
uint64_t orc_splitmix64_next(uint64_t *state);
uint64_t orc_query_key(uint64_t seed);
uint64_t orc_pac_hash(int64_t key, uint64_t query_key, int mode);
void orc_hash_keys(const int64_t *keys, size_t n, uint64_t query_key, int mode,
                   uint64_t *masks);

/* ---- counter-based generator used by the finalizer ----------------------- */
uint64_t orc_rng_u64(uint64_t seed, uint64_t stream, uint64_t counter);

/* ---- PAC selection (Sec. 4.2 "PAC Selection"; Sec. 3.2 pac_select and the
 *      fused pac_select_<cmp>) ----------------------------------------------
 * out[i] = masks[i] AND { bit j : col[i] <cmp> thr[t_i][j] }, the updated pu
 * column of Sec. 4.2 compiler step (3).  col/thr: int64, float or double by
 * vtype (int64 compares as integers, floats as doubles); cmp: ORC_CMP_*;
 * thr: [n_thr][64]; t_i = thr_ids[i] (width thr_id_bytes) or 0 when n_thr is
 * 1.  A row whose t_i >= n_thr selects no world and makes the status 1. */
#define ORC_CMP_LT 0
#define ORC_CMP_LE 1
#define ORC_CMP_EQ 2
#define ORC_CMP_NE 3
#define ORC_CMP_GT 4
#define ORC_CMP_GE 5
int orc_select(const uint64_t *masks, const void *col, int vtype, int cmp, const void *thr,
               uint32_t n_thr, const void *thr_ids, int thr_id_bytes, size_t n, uint64_t *out);

/* ---- vector-lifted expressions (Sec. 4.2 "Vector-lifted Expression, and
 *      Lambda Functions": e applied world by world, scalars broadcast) -----
 * y[n_groups][n_specs][64]: stored world results as doubles; scales: each
 * spec's release scale; prog: postfix program over a stack of values:
 *   SPEC k  push scales[k] * y[g][k][j]      CONST  push c
 *   ADD SUB MUL DIV  pop b, pop a, push a op b (IEEE double)
 *   MIN MAX  a < b ? a : b,  a > b ? a : b    NEG ABS  on the top value
 *   LT LE EQ NE GT GE  push 1.0 if a <cmp> b else 0.0
 * out[n_groups][64] = the program's single result per world.  Returns 1
 * (out untouched) for a program that underflows, exceeds ORC_LIFT_DEPTH
 * values, names a missing spec or does not end with one value. */
enum {
    ORC_LIFT_SPEC = 0, ORC_LIFT_CONST = 1, ORC_LIFT_ADD = 2, ORC_LIFT_SUB = 3, ORC_LIFT_MUL = 4,
    ORC_LIFT_DIV = 5, ORC_LIFT_NEG = 6, ORC_LIFT_ABS = 7, ORC_LIFT_MIN = 8, ORC_LIFT_MAX = 9,
    ORC_LIFT_LT = 10, ORC_LIFT_LE = 11, ORC_LIFT_EQ = 12, ORC_LIFT_NE = 13, ORC_LIFT_GT = 14,
    ORC_LIFT_GE = 15
};
#define ORC_LIFT_DEPTH 8
typedef struct {
    int32_t op;
    int32_t arg;
    double c;
} orc_lift_op;
int orc_lift(const double *y, const double *scales, uint32_t n_specs, uint32_t n_groups,
             const orc_lift_op *prog, int n_ops, double *out);

/* ---- pac_filter (Sec. 3.2 "Categorical Rewrites": probabilistic filtering)
 * b[n_groups][64]: a lifted boolean list per group (true = non-zero).  The
 * fraction of true worlds is the probability of keeping the group's row:
 * keep[g] = u_g < #true/64, u_g uniform in [0,1) from counter stream 3 of
 * the seed at counter g.  It does not depend on the secret world and makes
 * no posterior update. */
void orc_filter(const double *b, uint32_t n_groups, uint64_t seed, uint8_t *keep);

/* ---- exact aggregation, row by row (Sec. 4.2 "PAC Aggregation") ---------- */
/* values: int64 / float / double column selected by vtype (NULL for COUNT).
 * gids:   group id per row, width gid_bytes (1, 2, 4); NULL => one group.
 * out:    [n_groups][64] of uint64 (COUNT), int64 (SUM/MIN/MAX over I64),
 *         double (AVG, and SUM/MIN/MAX over floats).
 * meta_n/meta_or: per-group row count and OR of masks (Sec. 3.2 "NULLs"),
 *         may be NULL.  Returns a status. */
int orc_aggregate_direct(const uint64_t *masks, const void *values, int vtype,
                         const void *gids, int gid_bytes, size_t n,
                         uint32_t n_groups, int kind, void *out,
                         uint64_t *meta_n, uint64_t *meta_or);

/* r_j of one world j for every group: out[n_groups] (sampling large inputs). */
int orc_aggregate_world(const uint64_t *masks, const void *values, int vtype,
                        const void *gids, int gid_bytes, size_t n,
                        uint32_t n_groups, int kind, int world, void *out);

/* ---- the same definition, computed world by world on materialised
 *      subsamples (Sec. 4.1 compilation procedure steps (1)-(2), with the
 *      hash-coupled SamplePU of Theorem 2) ------------------------------- */
int orc_aggregate_brute(const int64_t *keys, uint64_t query_key, int mode,
                        const void *values, int vtype, const void *gids,
                        int gid_bytes, size_t n, uint32_t n_groups, int kind,
                        void *out);

/* ---- approximate integer SUM, 25 levels of 16-bit counters, two-sided
 *      (Sec. 5 "Approximation"); AVG variant divides by the update count --- */
#define ORC_APX_LEVELS 25
#define ORC_APX_CHUNK 4096
int orc_approx_sum_i64(const uint64_t *masks, const int64_t *values,
                       const void *gids, int gid_bytes, size_t n,
                       uint32_t n_groups, int64_t *out);
int orc_approx_avg_i64(const uint64_t *masks, const int64_t *values,
                       const void *gids, int gid_bytes, size_t n,
                       uint32_t n_groups, double *out);

/* ---- approximate float SUM with FLOAT state (Sec. 5 "Approximation") ---- */
/* The same two with drop_empty: rows whose mask is 0 (filtered out by a
 * selection) update nothing and count in no group; chunks stay over row
 * positions. */
int orc_approx_sum_i64_ex(const uint64_t *masks, const int64_t *values,
                          const void *gids, int gid_bytes, size_t n,
                          uint32_t n_groups, int64_t *out, int drop_empty);
int orc_approx_avg_i64_ex(const uint64_t *masks, const int64_t *values,
                          const void *gids, int gid_bytes, size_t n,
                          uint32_t n_groups, double *out, int drop_empty);
int orc_approx_sum_f32state(const uint64_t *masks, const void *values,
                            int vtype, const void *gids, int gid_bytes,
                            size_t n, uint32_t n_groups, double *out);

/* ---- finalize: variance under the posterior and PAC noise
 *      (Sec. 2 "PAC Privacy", Sec. 4.1 noise function steps 1-4,
 *       Sec. 2 fused pac_noised_count, Sec. 3.2 "NULLs", Sec. 5
 *       "Diversity Check") -------------------------------------------- */
double orc_release_scale(int kind, int variant);
/* y:       [n_groups*n_specs][64] unscaled aggregate results as doubles,
 *          cell c = g*n_specs + s.
 * scale:   [n_specs] release scale per spec (orc_release_scale).
 * outputs: noised[c], is_null[c], flags[c]; posterior[64] may be NULL;
 *          *jstar receives the secret world.  */
void orc_finalize(const double *y, const double *scale, uint32_t n_specs,
                  uint32_t n_groups, const uint64_t *meta_n,
                  const uint64_t *meta_or, uint64_t seed, double budget,
                  int mode, double *noised, uint8_t *is_null, uint32_t *flags,
                  double *posterior, int32_t *jstar);

/* building blocks exposed for the pins */
double orc_u01_open0(uint64_t u);     /* (0,1] */
double orc_u01(uint64_t u);           /* [0,1) */
double orc_box_muller(uint64_t u1, uint64_t u2);

/* m = 128 worlds (reading R7): masks are [n][2] words, world j in bit j % 64
 * of word j / 64; outputs are [n_groups][128]; meta_or2 is [n_groups][2]. */
uint64_t orc_query_key2(uint64_t seed);
void orc_pac_hash128(int64_t key, uint64_t k1, uint64_t k2, int mode, uint64_t *out2);
void orc_hash_keys128(const int64_t *keys, size_t n, uint64_t k1, uint64_t k2, int mode,
                      uint64_t *masks2);
int orc_aggregate128(const uint64_t *masks2, const void *values, int vtype, const void *gids,
                     int gid_bytes, size_t n, uint32_t n_groups, int kind, void *out,
                     uint64_t *meta_n, uint64_t *meta_or2);
int orc_aggregate_brute128(const int64_t *keys, uint64_t k1, uint64_t k2, int mode, const void *values,
                           int vtype, const void *gids, int gid_bytes, size_t n, uint32_t n_groups,
                           int kind, void *out);
void orc_finalize128(const double *y, const double *scale, uint32_t n_specs, uint32_t n_groups,
                     const uint64_t *meta_n, const uint64_t *meta_or2, uint64_t seed, double budget,
                     int mode, double *noised, uint8_t *is_null, uint32_t *flags, double *posterior,
                     int32_t *jstar_out);

#ifdef __cplusplus
}
#endif

#endif
