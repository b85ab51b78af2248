// pac_finalize.cu -- per-cell variance under the posterior and PAC noise
// (Sec. 2 "PAC Privacy"; Sec. 4.1 noise function steps 1-4; Sec. 2 fused
// pac_noised_count, count[j*]*2; Sec. 3.2 "NULLs"; Sec. 5 "Diversity Check").
//
// A cell (group g, spec s) has 64 world results y_t (scaled by 2 for COUNT
// and SUM, 0 for worlds outside the group's OR mask).  Its release:
//   step 1  mu = sum_t p_t y_t, var = sum_t p_t (y_t - mu)^2 under the
//           posterior p, exactly 0 when every world of non-zero posterior
//           has y_t == y_j* (j* the secret world);
//   step 2  delta = var / (2 B);
//   step 3  release y_j* + sqrt(delta) z, z standard normal (Box-Muller);
//   step 4  if delta > 0: log p_t += -(release - y_t)^2 / (2 delta), then
//           normalise.
// A NULL draw (Sec. 3.2) replaces the release of a cell whose group misses
// worlds.  In the adaptive mode every release depends on the posterior left
// by the previous one, so one chain of threads walks all cells of the query
// in order (group-major, then spec order); in the independent mode every
// cell starts from the uniform prior and cells are released in parallel.
// FP64 is used only here.
#include <cmath>

#include "pac_internal.cuh"
#include "pac_kernels.h"

namespace pacgpu {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint64_t kStreamJstar = 0, kStreamNull = 1, kStreamNoise = 2;
constexpr uint64_t kDiversityMinRows = 64;

// W = 64 or 128 worlds.  meta per group: {n_g, OR word 0[, OR word 1]}; j*
// is the top log2(W) bits of the first draw; the diversity flag needs at most
// 5/8 of the worlds updated (40 of 64, 80 of 128).
template <int W>
struct Worlds {
    static constexpr int kWords = W / 64;
    static constexpr int kMetaStride = 1 + kWords;
    static constexpr int kJShift = W == 64 ? 58 : 57;
    static constexpr int kDiversityMaxWorlds = W * 5 / 8;
};

// The OR of a group's mask words: world t was updated by some row.
template <int W>
struct OrMask {
    unsigned long long w[W / 64];
    __device__ __forceinline__ bool bit(int t) const { return (w[t >> 6] >> (t & 63)) & 1ull; }
    __device__ __forceinline__ int popc() const {
        int c = 0;
#pragma unroll
        for (int k = 0; k < W / 64; k++) c += __popcll(w[k]);
        return c;
    }
    __device__ __forceinline__ OrMask shfl(int src) const {
        OrMask o;
#pragma unroll
        for (int k = 0; k < W / 64; k++) o.w[k] = __shfl_sync(0xffffffffu, w[k], src);
        return o;
    }
};

template <int W>
__device__ __forceinline__ OrMask<W> group_or(const FinParams &p, uint32_t g) {
    OrMask<W> o;
#pragma unroll
    for (int k = 0; k < W / 64; k++) o.w[k] = p.meta[static_cast<size_t>(Worlds<W>::kMetaStride) * g + 1 + k];
    return o;
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ double uniform01(uint64_t u) { return static_cast<double>(u >> 11) * 0x1.0p-53; }
__device__ __forceinline__ double uniform01_open0(uint64_t u) {
    return static_cast<double>((u >> 11) + 1) * 0x1.0p-53;
}

// How the 64-bit words of a spec's result array read as the release's value:
// bits 0-1 conversion (0 unsigned count, 1 int64, 2 float64), bit 2 the
// factor 2 of COUNT and SUM (Sec. 2: the secret world's result is doubled).
__device__ __forceinline__ int cell_code(const FinSpec &sp) {
    const int conv = sp.kind == PAC_COUNT ? 0 : ((sp.kind == PAC_AVG || sp.vtype != PAC_I64) ? 2 : 1);
    return conv | ((sp.kind == PAC_COUNT || sp.kind == PAC_SUM) ? 4 : 0);
}

__device__ __forceinline__ double raw_to_double(unsigned long long b, int code) {
    const int conv = code & 3;
    const double v = conv == 0   ? static_cast<double>(b)
                     : conv == 1 ? static_cast<double>(static_cast<long long>(b))
                                 : __longlong_as_double(static_cast<long long>(b));
    return (code & 4) ? 2.0 * v : v;
}

// raw_to_double(a) == raw_to_double(b), mostly decided on the integers.
__device__ __forceinline__ bool same_value(unsigned long long a, unsigned long long b, int code) {
    const int conv = code & 3;
    bool exact;  // the integer comparison decides
    if (conv == 2) {
        const unsigned long long ma = a << 1, mb = b << 1;  // without the sign
        if ((ma | mb) == 0) return true;                   // +0 and -0
        if (a == b) return ma <= (0x7FF0000000000000ull << 1);  // NaN is unequal to itself
        // distinct doubles stay distinct after doubling unless both overflow
        exact = !((code & 4) && ma >= (0x7FE0000000000000ull << 1) && mb >= (0x7FE0000000000000ull << 1));
    } else {
        if (a == b) return true;
        // distinct integers of magnitude <= 2^53 convert to distinct doubles
        constexpr unsigned long long k53 = 1ull << 53;
        exact = conv == 0 ? (a <= k53 && b <= k53) : (a + k53 <= 2 * k53 && b + k53 <= 2 * k53);
    }
    return exact ? false : raw_to_double(a, code) == raw_to_double(b, code);
}

// The release value is not finite (after the factor 2): the variance sums
// would carry it into NaN even at zero weight.
__device__ __forceinline__ bool raw_nonfinite(unsigned long long b, int code) {
    if ((code & 3) != 2) return false;
    const unsigned e = static_cast<unsigned>(b >> 52) & 0x7FFu;
    return e >= ((code & 4) ? 0x7FEu : 0x7FFu);
}

struct CellRaw {
    unsigned long long y, yj;  // this thread's world and the secret world, as stored
    int code;
};

template <int W>
__device__ __forceinline__ CellRaw load_raw(const FinParams &p, uint32_t g, int s, int t, int jstar) {
    const FinSpec &sp = p.spec[s];
    const unsigned long long *o = static_cast<const unsigned long long *>(sp.out) + static_cast<size_t>(g) * W;
    CellRaw r;
    r.y = o[t];
    r.yj = o[jstar];
    r.code = cell_code(sp);
    return r;
}

// Per-lane facts of cell c that do not depend on the posterior.
template <int W>
struct CellDraw {
    OrMask<W> orm;
    bool null_, diversity;
};

template <int W>
__device__ __forceinline__ CellDraw<W> draw_cell(const FinParams &p, uint64_t c) {
    const uint32_t g = static_cast<uint32_t>(c / p.n_specs);
    CellDraw<W> d;
    d.orm = group_or<W>(p, g);
    const uint64_t rows = p.meta[static_cast<size_t>(Worlds<W>::kMetaStride) * g];
    const int pop = d.orm.popc();
    d.null_ = pop < W && static_cast<int>(counter_draw(p.seed, kStreamNull, c) >> Worlds<W>::kJShift) < W - pop;
    d.diversity = rows >= kDiversityMinRows && pop <= Worlds<W>::kDiversityMaxWorlds;
    return d;
}

template <int W>
__device__ __forceinline__ CellDraw<W> no_cell() {
    CellDraw<W> d;
#pragma unroll
    for (int k = 0; k < W / 64; k++) d.orm.w[k] = 0ull;
    d.null_ = true;
    d.diversity = false;
    return d;
}

// The standard normal of cell c (Box-Muller on two counter draws).
__device__ __forceinline__ double normal_draw(uint64_t seed, uint64_t c) {
    const double u1 = uniform01_open0(counter_draw(seed, kStreamNoise, 2 * c));
    const double u2 = uniform01(counter_draw(seed, kStreamNoise, 2 * c + 1));
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}


// ---------------------------------------------------------------------------
// Independent mode: every cell starts from the uniform prior, so step 1 is
// the plain mean and variance of the W worlds (p_t = 1/W) and the posterior
// after a release is needed for the last cell only (the one the caller can
// read back).  One warp takes 32 consecutive cells: lane k makes cell k's
// NULL decision and normal draw, then the warp releases the cells one by
// one, lane l holding worlds l, l+32, ... (W/32 of them), and lane k stores
// cell k.
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(256) k_finalize_independent(const __grid_constant__ FinParams p) {
    constexpr int V = W / 32;
    const int lane = threadIdx.x & 31;
    const int jstar = static_cast<int>(counter_draw(p.seed, kStreamJstar, 0) >> Worlds<W>::kJShift);
    const double inv2b = 1.0 / (2.0 * p.budget);
    const double log_uniform = -log(static_cast<double>(W));
    const uint64_t n_cells = static_cast<uint64_t>(p.n_groups) * p.n_specs;
    const uint64_t n_blk = (n_cells + 31) / 32;
    const uint64_t wid = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_w = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
    for (uint64_t blk = wid; blk < n_blk; blk += n_w) {
        const uint64_t c0 = blk * 32;
        const uint64_t rem = n_cells - c0;
        const int kend = rem < 32 ? static_cast<int>(rem) : 32;
        CellDraw<W> dl = no_cell<W>();
        double zc = 0.0;
        if (lane < kend) {
            dl = draw_cell<W>(p, c0 + lane);
            if (!dl.null_) zc = normal_draw(p.seed, c0 + lane);
        }
        const uint32_t nulls = __ballot_sync(kFull, dl.null_);
        double my_yt = 0.0;
        bool my_zv = false;
        uint32_t g = static_cast<uint32_t>(c0 / p.n_specs);
        int s = static_cast<int>(c0 % p.n_specs);
        for (int k = 0; k < kend; k++, s = (s + 1 == p.n_specs) ? (g++, 0) : s + 1) {
            const uint64_t c = c0 + k;
            const bool last = p.posterior && c == n_cells - 1;
            if ((nulls >> k) & 1u) {
                if (last)
#pragma unroll
                    for (int v = 0; v < V; v++) p.posterior[lane + 32 * v] = exp(log_uniform);
                continue;
            }
            const OrMask<W> orm = dl.orm.shfl(k);
            const double z = __shfl_sync(kFull, zc, k);
            const FinSpec &sp = p.spec[s];
            const int code = cell_code(sp);
            const unsigned long long *o =
                static_cast<const unsigned long long *>(sp.out) + static_cast<size_t>(g) * W;
            unsigned long long r[V];
            bool agree = true;
            const unsigned long long rj = orm.bit(jstar) ? o[jstar] : 0ull;
#pragma unroll
            for (int v = 0; v < V; v++) {
                r[v] = orm.bit(lane + 32 * v) ? o[lane + 32 * v] : 0ull;
                agree = agree && same_value(r[v], rj, code);
            }
            const double yj = raw_to_double(rj, code);
            double var = 0.0, y[V];
#pragma unroll
            for (int v = 0; v < V; v++) y[v] = 0.0;
            if (!__all_sync(kFull, agree)) {
                double sum = 0.0;
#pragma unroll
                for (int v = 0; v < V; v++) {
                    y[v] = raw_to_double(r[v], code);
                    sum += y[v];
                }
                const double mu = warp_sum(sum) * (1.0 / W);
                double sq = 0.0;
#pragma unroll
                for (int v = 0; v < V; v++) {
                    const double d = y[v] - mu;
                    sq = fma(d, d, sq);
                }
                var = warp_sum(sq) * (1.0 / W);
            }
            const double delta = var * inv2b;
            const double yt = delta == 0.0 ? yj : yj + sqrt(delta) * z;
            if (last) {
                double l[V];
#pragma unroll
                for (int v = 0; v < V; v++) l[v] = log_uniform;
                if (delta > 0.0) {
                    double mx = -INFINITY;
#pragma unroll
                    for (int v = 0; v < V; v++) {
                        const double e = yt - y[v];
                        l[v] += -(e * e) / (2.0 * delta);
                        mx = fmax(mx, l[v]);
                    }
                    for (int o2 = 16; o2; o2 >>= 1) mx = fmax(mx, __shfl_xor_sync(kFull, mx, o2));
                    double se = 0.0;
#pragma unroll
                    for (int v = 0; v < V; v++) se += exp(l[v] - mx);
                    const double lse = mx + log(warp_sum(se));
#pragma unroll
                    for (int v = 0; v < V; v++) l[v] -= lse;
                }
#pragma unroll
                for (int v = 0; v < V; v++) p.posterior[lane + 32 * v] = exp(l[v]);
            }
            if (lane == k) {
                my_yt = yt;
                my_zv = !(delta > 0.0);
            }
        }
        if (lane < kend) {
            const uint64_t c = c0 + lane;
            const uint32_t f = dl.diversity ? PAC_F_DIVERSITY : 0u;
            p.noised[c] = dl.null_ ? 0.0 : my_yt;
            p.is_null[c] = dl.null_ ? 1 : 0;
            p.flags[c] = f | (dl.null_ ? PAC_F_NULL : (my_zv ? PAC_F_ZEROVAR : 0u));
        }
    }
    if (p.posterior && n_cells == 0 && blockIdx.x == 0 && threadIdx.x < 32)
#pragma unroll
        for (int v = 0; v < V; v++) p.posterior[lane + 32 * v] = exp(log_uniform);
}

// ---------------------------------------------------------------------------
// The posterior chain of one query (adaptive mode, and every batched query).
// 64 threads, thread t holding world t.  The chain is bound by the latency of
// dependent FP64 operations, so the state is kept in a form that needs one
// exp and no log per update:
//   L_t   log-weight of world t, shifted so that max_t L_t = 0 (all L_t <= 0),
//   w_t   = exp(L_t), the weight left by the last update,
//   se    = sum_t w_t,
// which is the posterior of Sec. 4.1 step 4 up to normalisation:
// p_t = w_t / se, log p_t = L_t - log(se).  The mean and variance of step 1
// divide the weighted sums by se; the update adds -(e_t^2)/(2 delta) to L_t,
// subtracts the new maximum (found as the least IEEE bit pattern, since every
// L_t <= 0) and takes exp once.  In exact arithmetic every quantity is the
// one of steps 1-4 above; rounding differs by a few ulps.
//
// Step 1's test "all worlds of non-zero posterior agree" runs first, on the
// raw 64-bit words, and skips both sums when it holds.  Once a single world
// keeps non-zero weight (adaptive mode), every later release has variance 0
// and the posterior no longer changes, so the remaining cells are released
// in parallel, one per lane (collapsed_tail).  Draws that do not depend on
// the posterior (the NULL decision and the Box-Muller normal of a cell) are
// computed 32 cells at a time, one cell per lane, and world values are
// loaded kAhead cells ahead of the chain.
// ---------------------------------------------------------------------------
constexpr int kAhead = 4;
constexpr int kMaxChainWarps = kWorlds128 / 32;

// W threads (thread t holds world t), W/32 warps.
struct ChainShared {
    double part[4][kMaxChainWarps];  // per-warp partials, rotating slots (one barrier per reduction)
    unsigned long long bits[4][kMaxChainWarps];
};

template <int NW>
__device__ __forceinline__ double chain_sum(double v, ChainShared &sh, int &slot, int warp, int lane) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    double *pp = sh.part[slot];
    slot = (slot + 1) & 3;
    if (lane == 0) pp[warp] = v;
    __syncthreads();
    double t = pp[0] + pp[1];
#pragma unroll
    for (int w = 2; w < NW; w++) t += pp[w];
    return t;
}

// chain_sum, also counting the threads whose flag b is set.
template <int NW>
__device__ __forceinline__ double chain_sum_count(double v, bool b, int &cnt, ChainShared &sh, int &slot, int warp,
                                                  int lane) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    const unsigned bal = __ballot_sync(kFull, b);
    double *pp = sh.part[slot];
    unsigned long long *pb = sh.bits[slot];
    slot = (slot + 1) & 3;
    if (lane == 0) {
        pp[warp] = v;
        pb[warp] = bal;
    }
    __syncthreads();
    cnt = 0;
    double t = pp[0] + pp[1];
#pragma unroll
    for (int w = 0; w < NW; w++) cnt += __popc(static_cast<unsigned>(pb[w]));
#pragma unroll
    for (int w = 2; w < NW; w++) t += pp[w];
    return t;
}

// Maximum of non-positive doubles: the least bit pattern (+0 < -0 < -tiny <
// ... < -inf as unsigned integers).
template <int NW>
__device__ __forceinline__ double chain_max_nonpos(double x, ChainShared &sh, int &slot, int warp, int lane) {
    unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(kFull, b, o);
        b = u < b ? u : b;
    }
    unsigned long long *pp = sh.bits[slot];
    slot = (slot + 1) & 3;
    if (lane == 0) pp[warp] = b;
    __syncthreads();
    b = pp[0];
#pragma unroll
    for (int w = 1; w < NW; w++) b = pp[w] < b ? pp[w] : b;
    return __longlong_as_double(static_cast<long long>(b));
}

__device__ __forceinline__ bool chain_all(bool x) { return __syncthreads_and(x) != 0; }

template <int NW>
__device__ __forceinline__ unsigned chain_or(unsigned m, ChainShared &sh, int &slot, int warp, int lane) {
    m = __reduce_or_sync(kFull, m);
    unsigned long long *pp = sh.bits[slot];
    slot = (slot + 1) & 3;
    if (lane == 0) pp[warp] = m;
    __syncthreads();
    unsigned long long o = 0;
#pragma unroll
    for (int w = 0; w < NW; w++) o |= pp[w];
    return static_cast<unsigned>(o);
}

// Releases cells c0 .. n_cells-1 once world sw alone has non-zero weight
// (w = 1, se = 1).  For each cell: if y_sw == y_j* the worlds agree and the
// variance is 0; otherwise every other world has weight exactly 0, so the
// mean is y_sw and the variance 0, unless some release value is not finite,
// which makes the sums NaN.  No posterior update happens either way.
template <int W>
__device__ void collapsed_tail(const FinParams &p, uint64_t c0, uint64_t n_cells, int jstar, int sw,
                               ChainShared &sh, int &slot) {
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    bool any_float = false;
    for (int s = 0; s < p.n_specs; s++) any_float = any_float || (cell_code(p.spec[s]) & 3) == 2;
    for (; c0 < n_cells; c0 += 32) {
        const uint64_t rem = n_cells - c0;
        const int kend = rem < 32 ? static_cast<int>(rem) : 32;
        unsigned bad = 0;
        if (any_float) {
            // bit k: this thread's world value of cell c0+k is not finite
            uint32_t g = static_cast<uint32_t>(c0 / p.n_specs);
            int s = static_cast<int>(c0 % p.n_specs);
            for (int k = 0; k < kend; k++) {
                const int code = cell_code(p.spec[s]);
                if ((code & 3) == 2 && group_or<W>(p, g).bit(t)) {
                    const unsigned long long v =
                        static_cast<const unsigned long long *>(p.spec[s].out)[static_cast<size_t>(g) * W + t];
                    if (raw_nonfinite(v, code)) bad |= 1u << k;
                }
                if (++s == p.n_specs) s = 0, g++;
            }
            bad = chain_or<W / 32>(bad, sh, slot, warp, lane);
        }
        if (warp == 0 && lane < kend) {
            const uint64_t c = c0 + lane;
            const CellDraw<W> d = draw_cell<W>(p, c);
            uint32_t f = d.diversity ? PAC_F_DIVERSITY : 0u;
            if (d.null_) {
                p.noised[c] = 0.0;
                p.is_null[c] = 1;
                p.flags[c] = f | PAC_F_NULL;
            } else {
                const uint32_t g = static_cast<uint32_t>(c / p.n_specs);
                const FinSpec &sp = p.spec[c % p.n_specs];
                const int code = cell_code(sp);
                const unsigned long long *o =
                    static_cast<const unsigned long long *>(sp.out) + static_cast<size_t>(g) * W;
                const double yj = raw_to_double(d.orm.bit(jstar) ? o[jstar] : 0ull, code);
                const double ys = raw_to_double(d.orm.bit(sw) ? o[sw] : 0ull, code);
                p.noised[c] = (ys == yj || !((bad >> lane) & 1u)) ? yj : __longlong_as_double(0x7FF8000000000000ll);
                p.is_null[c] = 0;
                p.flags[c] = f | PAC_F_ZEROVAR;
            }
        }
    }
}

template <int W>
__device__ void finalize_chain(const FinParams &p) {
    constexpr int NW = W / 32;
    __shared__ ChainShared sh;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int jstar = static_cast<int>(counter_draw(p.seed, kStreamJstar, 0) >> Worlds<W>::kJShift);
    const double inv2b = 1.0 / (2.0 * p.budget);
    const bool adaptive = p.mode != PAC_FIN_INDEPENDENT;
    double L = 0.0, w = 1.0, se = static_cast<double>(W), rse = 1.0 / se;
    bool sup = true;     // posterior of world t is non-zero
    bool single = false; // one world alone has non-zero weight
    int slot = 0;
    const uint64_t n_cells = static_cast<uint64_t>(p.n_groups) * p.n_specs;
    // world values of cells pc - kAhead .. pc - 1, oldest first
    CellRaw ring[kAhead];
    uint32_t pg = 0;
    int ps = 0;
    uint64_t pc = 0;
#pragma unroll
    for (int i = 0; i < kAhead; i++) {
        if (pc < n_cells) {
            ring[i] = load_raw<W>(p, pg, ps, t, jstar);
            pc++;
            if (++ps == p.n_specs) ps = 0, pg++;
        }
    }
    uint64_t c0 = 0;
    while (c0 < n_cells && !single) {
        const uint64_t rem = n_cells - c0;
        const int kend = rem < 32 ? static_cast<int>(rem) : 32;
        // posterior-free draws of cells c0 .. c0+31, one per lane
        CellDraw<W> dl = no_cell<W>();
        double zc = 0.0;
        if (lane < kend) {
            const uint64_t cl = c0 + lane;
            dl = draw_cell<W>(p, cl);
            if (!dl.null_) zc = normal_draw(p.seed, cl);
        }
        const uint32_t nulls = __ballot_sync(kFull, dl.null_);
        double my_yt = 0.0;
        bool my_zv = false;
        int kc = 0;
        for (; kc < kend && !single; kc++) {
            const CellRaw cur = ring[0];
#pragma unroll
            for (int i = 0; i + 1 < kAhead; i++) ring[i] = ring[i + 1];
            if (pc < n_cells) {
                ring[kAhead - 1] = load_raw<W>(p, pg, ps, t, jstar);
                pc++;
                if (++ps == p.n_specs) ps = 0, pg++;
            }
            if (!adaptive) {
                L = 0.0, w = 1.0, se = static_cast<double>(W), rse = 1.0 / se;
                sup = true;
            }
            if ((nulls >> kc) & 1u) continue;
            const OrMask<W> orm = dl.orm.shfl(kc);
            const double z = __shfl_sync(kFull, zc, kc);
            const unsigned long long yr = orm.bit(t) ? cur.y : 0ull;
            const unsigned long long yjr = orm.bit(jstar) ? cur.yj : 0ull;
            const double yj = raw_to_double(yjr, cur.code);
            // step 1: variance under the posterior, exactly 0 when all worlds of
            // non-zero posterior agree (then neither sum is needed)
            double var = 0.0, y = 0.0;
            if (!chain_all(!sup || same_value(yr, yjr, cur.code))) {
                y = raw_to_double(yr, cur.code);
                const double mu = chain_sum<NW>(w * y, sh, slot, warp, lane) * rse;
                const double d = y - mu;
                var = chain_sum<NW>(w * d * d, sh, slot, warp, lane) * rse;
            }
            // step 2: noise variance; step 3: release
            const double delta = var * inv2b;
            // sqrt(delta) and -1/(2 delta) both from one reciprocal square root
            // (the chain is bound by dependent FP64 instructions); delta = inf
            // and deltas near the bottom of the range take the plain forms
            const double rs = rsqrt(delta);
            const bool plain = !(delta > 1e-300) || isinf(delta);
            const double yt = delta == 0.0 ? yj : yj + (plain ? sqrt(delta) : delta * rs) * z;
            // step 4: Bayesian update of the log-weights
            const bool upd = delta > 0.0;
            // independent mode: the next cell starts from the uniform prior, so
            // only the last cell's update is ever read
            if (upd && (adaptive || c0 + kc + 1 == n_cells)) {
                const double e = yt - y;
                L = fma(e * e, plain ? -0.5 / delta : -0.5 * rs * rs, L);
                L -= chain_max_nonpos<NW>(L, sh, slot, warp, lane);
                w = exp(L);
                if (adaptive) {
                    int cnt;
                    se = chain_sum_count<NW>(w, w > 0.0, cnt, sh, slot, warp, lane);
                    single = cnt == 1;
                } else {
                    se = chain_sum<NW>(w, sh, slot, warp, lane);
                }
                rse = 1.0 / se;
                sup = w * rse > 0.0;
            }
            if (lane == kc) {
                my_yt = yt;
                my_zv = !upd;
            }
        }
        // outputs of cells c0 .. c0+kc-1, one per lane of warp 0
        if (warp == 0 && lane < kc) {
            const uint64_t c = c0 + lane;
            const bool nul = (nulls >> lane) & 1u;
            const uint32_t f = dl.diversity ? PAC_F_DIVERSITY : 0u;
            p.noised[c] = nul ? 0.0 : my_yt;
            p.is_null[c] = nul ? 1 : 0;
            p.flags[c] = f | (nul ? PAC_F_NULL : (my_zv ? PAC_F_ZEROVAR : 0u));
        }
        c0 += kc;
    }
    if (single && c0 < n_cells) {
        // the world left with weight 1
        const unsigned bal = __ballot_sync(kFull, w > 0.0);
        unsigned long long *pp = sh.bits[slot];
        slot = (slot + 1) & 3;
        if (lane == 0) pp[warp] = bal;
        __syncthreads();
        int sw = 0;
#pragma unroll
        for (int k = NW - 1; k >= 0; k--)
            if (pp[k]) sw = 32 * k + __ffs(static_cast<int>(pp[k])) - 1;
        collapsed_tail<W>(p, c0, n_cells, jstar, sw, sh, slot);
    }
    if (p.posterior) p.posterior[t] = w * rse;
}

template <int W>
__global__ void __launch_bounds__(W) k_finalize_adaptive(const __grid_constant__ FinParams p) {
    finalize_chain<W>(p);
}

// One posterior chain per query of a batch.
__global__ void __launch_bounds__(kWorlds) k_finalize_batch(const FinParams *__restrict__ ps, int n) {
    if (static_cast<int>(blockIdx.x) < n) finalize_chain<kWorlds>(ps[blockIdx.x]);
}

template <int W>
cudaError_t launch_finalize_w(const FinParams &p, cudaStream_t s) {
    const uint64_t n_cells = static_cast<uint64_t>(p.n_groups) * p.n_specs;
    if (p.mode == PAC_FIN_ADAPTIVE) {
        k_finalize_adaptive<W><<<1, W, 0, s>>>(p);
    } else {
        uint64_t blocks = (n_cells * 32 + 255) / 256;
        if (blocks > 152 * 16) blocks = 152 * 16;
        if (blocks == 0) blocks = 1;
        k_finalize_independent<W><<<static_cast<unsigned>(blocks), 256, 0, s>>>(p);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_finalize(const FinParams &p, cudaStream_t s) { return launch_finalize_w<kWorlds>(p, s); }

cudaError_t launch_finalize128(const FinParams &p, cudaStream_t s) { return launch_finalize_w<kWorlds128>(p, s); }

cudaError_t launch_finalize_batch(const FinParams *d_params, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_finalize_batch<<<static_cast<unsigned>(n), kWorlds, 0, s>>>(d_params, n);
    return cudaGetLastError();
}

}  // namespace pacgpu
