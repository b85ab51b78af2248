// pac_finalize.cu -- per-cell variance under the posterior and PAC noise
// (Sec. 2 "PAC Privacy"; Sec. 4.1 noise function steps 1-4; Sec. 2 fused
// pac_noised_count, count[j*]*2; Sec. 3.2 "NULLs"; Sec. 5 "Diversity Check").
//
// In the adaptive mode every release depends on the posterior left by the
// previous one, so one 64-thread chain walks all cells of the query in order
// (group-major, then spec order), thread t holding world t; the independent
// mode gives every cell its own warp (lane l: worlds l and l+32) under the
// uniform prior.  FP64 is used only here.
#include <cmath>

#include "pac_internal.cuh"
#include "pac_kernels.h"

namespace pacgpu {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint64_t kStreamJstar = 0, kStreamNull = 1, kStreamNoise = 2;
constexpr uint64_t kDiversityMinRows = 64;
constexpr int kDiversityMaxWorlds = 40;

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

__device__ __forceinline__ double world_value(const FinSpec &s, size_t idx) {
    if (s.kind == PAC_COUNT) return static_cast<double>(static_cast<const unsigned long long *>(s.out)[idx]);
    if (s.kind == PAC_AVG || s.vtype != PAC_I64) return static_cast<const double *>(s.out)[idx];
    return static_cast<double>(static_cast<const long long *>(s.out)[idx]);
}

__device__ __forceinline__ double uniform01(uint64_t u) { return static_cast<double>(u >> 11) * 0x1.0p-53; }
__device__ __forceinline__ double uniform01_open0(uint64_t u) {
    return static_cast<double>((u >> 11) + 1) * 0x1.0p-53;
}

// Releases cell c; logp0/logp1 are this lane's log-posterior entries.
__device__ void release_cell(const FinParams &p, uint64_t c, int jstar, double &logp0, double &logp1) {
    const int lane = threadIdx.x & 31;
    const uint32_t g = static_cast<uint32_t>(c / p.n_specs);
    const int s = static_cast<int>(c % p.n_specs);
    const FinSpec &sp = p.spec[s];
    const uint64_t orm = p.meta[2 * g + 1];
    const uint64_t rows = p.meta[2 * g];
    const int pop = __popcll(orm);
    uint32_t f = (rows >= kDiversityMinRows && pop <= kDiversityMaxWorlds) ? PAC_F_DIVERSITY : 0u;

    if (p.mode == PAC_FIN_INDEPENDENT) {
        logp0 = -log(64.0);
        logp1 = -log(64.0);
    }
    if (pop < 64 && static_cast<int>(counter_draw(p.seed, kStreamNull, c) >> 58) < 64 - pop) {
        if (lane == 0) {
            p.noised[c] = 0.0;
            p.is_null[c] = 1;
            p.flags[c] = f | PAC_F_NULL;
        }
        return;
    }
    const double scale = (sp.kind == PAC_COUNT || sp.kind == PAC_SUM) ? 2.0 : 1.0;
    const size_t base = static_cast<size_t>(g) * kWorlds;
    const double y0 = ((orm >> lane) & 1ull) ? scale * world_value(sp, base + lane) : 0.0;
    const double y1 = ((orm >> (lane + 32)) & 1ull) ? scale * world_value(sp, base + lane + 32) : 0.0;
    const double yj = __shfl_sync(kFull, jstar < 32 ? y0 : y1, jstar & 31);

    // step 1: variance under the posterior (exactly 0 when all allowed worlds agree)
    const double p0 = exp(logp0), p1 = exp(logp1);
    const bool same = (!(p0 > 0.0) || y0 == yj) && (!(p1 > 0.0) || y1 == yj);
    const bool all_equal = __all_sync(kFull, same);
    const double mu = warp_sum(p0 * y0 + p1 * y1);
    const double d0 = y0 - mu, d1 = y1 - mu;
    double var = warp_sum(p0 * d0 * d0 + p1 * d1 * d1);
    if (all_equal) var = 0.0;
    // step 2: noise variance; step 3: release
    const double delta = var / (2.0 * p.budget);
    const double u1 = uniform01_open0(counter_draw(p.seed, kStreamNoise, 2 * c));
    const double u2 = uniform01(counter_draw(p.seed, kStreamNoise, 2 * c + 1));
    const double z = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
    const double yt = yj + sqrt(delta) * z;
    // step 4: Bayesian update in log space
    if (delta > 0.0) {
        const double e0 = yt - y0, e1 = yt - y1;
        logp0 += -(e0 * e0) / (2.0 * delta);
        logp1 += -(e1 * e1) / (2.0 * delta);
        const double mx = warp_max(fmax(logp0, logp1));
        const double se = warp_sum(exp(logp0 - mx) + exp(logp1 - mx));
        const double lse = mx + log(se);
        logp0 -= lse;
        logp1 -= lse;
    } else {
        f |= PAC_F_ZEROVAR;
    }
    if (lane == 0) {
        p.noised[c] = yt;
        p.is_null[c] = 0;
        p.flags[c] = f;
    }
}

// ---------------------------------------------------------------------------
// The posterior chain of one query (adaptive mode, and every batched query):
// 64 threads, thread t holds world t of the result vector and of the
// log-posterior, so the FP64 work of a cell is split across two warps (two
// SM sub-partitions).  Draws that do not depend on the posterior (the NULL
// decision and the Box-Muller normal of a cell) are computed 32 cells at a
// time, one cell per lane, and the next cell's world values are loaded while
// the current cell's chain runs.  The arithmetic per cell is that of
// release_cell above.
// ---------------------------------------------------------------------------
constexpr int kChainThreads = 64;

struct ChainShared {
    double part[8][2];  // per-warp partials, rotating slots (one barrier per reduction)
};

__device__ __forceinline__ double chain_reduce(double v, bool is_max, ChainShared &sh, int &slot, int warp,
                                               int lane) {
    for (int o = 16; o; o >>= 1) {
        const double t = __shfl_xor_sync(kFull, v, o);
        v = is_max ? fmax(v, t) : v + t;
    }
    double *pp = sh.part[slot];
    slot = (slot + 1) & 7;
    if (lane == 0) pp[warp] = v;
    __syncthreads();
    return is_max ? fmax(pp[0], pp[1]) : pp[0] + pp[1];
}

struct CellLoad {
    uint64_t orm, rows;
    double y, yj;  // this thread's world value and the secret world's, scaled and masked
};

__device__ __forceinline__ CellLoad load_cell(const FinParams &p, uint64_t c, int world, int jstar) {
    CellLoad L;
    const uint32_t g = static_cast<uint32_t>(c / p.n_specs);
    const int s = static_cast<int>(c % p.n_specs);
    const FinSpec &sp = p.spec[s];
    L.orm = p.meta[2 * g + 1];
    L.rows = p.meta[2 * g];
    const double scale = (sp.kind == PAC_COUNT || sp.kind == PAC_SUM) ? 2.0 : 1.0;
    const size_t base = static_cast<size_t>(g) * kWorlds;
    const double v = world_value(sp, base + world);
    const double vj = world_value(sp, base + jstar);
    L.y = ((L.orm >> world) & 1ull) ? scale * v : 0.0;
    L.yj = ((L.orm >> jstar) & 1ull) ? scale * vj : 0.0;
    return L;
}

__device__ void finalize_chain(const FinParams &p) {
    __shared__ ChainShared sh;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int jstar = static_cast<int>(counter_draw(p.seed, kStreamJstar, 0) >> 58);
    const double log_uniform = -log(64.0);
    double logp = log_uniform;
    int slot = 0;
    const uint64_t n_cells = static_cast<uint64_t>(p.n_groups) * p.n_specs;
    CellLoad nxt{};
    if (n_cells > 0) nxt = load_cell(p, 0, t, jstar);
    for (uint64_t c0 = 0; c0 < n_cells; c0 += 32) {
        // posterior-free draws of cells c0 .. c0+31, one per lane
        const uint64_t cl = c0 + lane;
        double zc = 0.0;
        bool nl = false;
        if (cl < n_cells) {
            const uint64_t orm = p.meta[2 * static_cast<uint32_t>(cl / p.n_specs) + 1];
            const int pop = __popcll(orm);
            nl = pop < 64 && static_cast<int>(counter_draw(p.seed, kStreamNull, cl) >> 58) < 64 - pop;
            if (!nl) {
                const double u1 = uniform01_open0(counter_draw(p.seed, kStreamNoise, 2 * cl));
                const double u2 = uniform01(counter_draw(p.seed, kStreamNoise, 2 * cl + 1));
                zc = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
            }
        }
        const uint32_t nulls = __ballot_sync(kFull, nl);
        const uint64_t rem = n_cells - c0;
        const int kend = rem < 32 ? static_cast<int>(rem) : 32;
        for (int k = 0; k < kend; k++) {
            const uint64_t c = c0 + k;
            const CellLoad cur = nxt;
            if (c + 1 < n_cells) nxt = load_cell(p, c + 1, t, jstar);
            const int pop = __popcll(cur.orm);
            uint32_t f = (cur.rows >= kDiversityMinRows && pop <= kDiversityMaxWorlds) ? PAC_F_DIVERSITY : 0u;
            if (p.mode == PAC_FIN_INDEPENDENT) logp = log_uniform;
            if ((nulls >> k) & 1u) {
                if (t == 0) {
                    p.noised[c] = 0.0;
                    p.is_null[c] = 1;
                    p.flags[c] = f | PAC_F_NULL;
                }
                continue;
            }
            const double z = __shfl_sync(kFull, zc, k);
            // step 1: variance under the posterior (exactly 0 when all allowed worlds agree)
            const double pw = exp(logp);
            const bool same = !(pw > 0.0) || cur.y == cur.yj;
            const bool all_equal = __syncthreads_and(same) != 0;
            const double mu = chain_reduce(pw * cur.y, false, sh, slot, warp, lane);
            const double d = cur.y - mu;
            double var = chain_reduce(pw * d * d, false, sh, slot, warp, lane);
            if (all_equal) var = 0.0;
            // step 2: noise variance; step 3: release
            const double delta = var / (2.0 * p.budget);
            const double yt = cur.yj + sqrt(delta) * z;
            // step 4: Bayesian update in log space
            if (delta > 0.0) {
                const double e = yt - cur.y;
                logp += -(e * e) / (2.0 * delta);
                const double mx = chain_reduce(logp, true, sh, slot, warp, lane);
                const double se = chain_reduce(exp(logp - mx), false, sh, slot, warp, lane);
                logp -= mx + log(se);
            } else {
                f |= PAC_F_ZEROVAR;
            }
            if (t == 0) {
                p.noised[c] = yt;
                p.is_null[c] = 0;
                p.flags[c] = f;
            }
        }
    }
    if (p.posterior) p.posterior[t] = exp(logp);
}

__global__ void __launch_bounds__(kChainThreads) k_finalize_adaptive(const __grid_constant__ FinParams p) {
    finalize_chain(p);
}

__global__ void __launch_bounds__(256) k_finalize_independent(const __grid_constant__ FinParams p) {
    const int lane = threadIdx.x & 31;
    const int jstar = static_cast<int>(counter_draw(p.seed, kStreamJstar, 0) >> 58);
    const uint64_t n_cells = static_cast<uint64_t>(p.n_groups) * p.n_specs;
    const uint64_t wid = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_w = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
    for (uint64_t c = wid; c < n_cells; c += n_w) {
        double logp0, logp1;
        release_cell(p, c, jstar, logp0, logp1);
        // the posterior left by the last release (uniform prior + one update)
        if (p.posterior && c == n_cells - 1) {
            p.posterior[lane] = exp(logp0);
            p.posterior[lane + 32] = exp(logp1);
        }
    }
    if (p.posterior && n_cells == 0 && blockIdx.x == 0 && threadIdx.x < 32) {
        p.posterior[lane] = exp(-log(64.0));
        p.posterior[lane + 32] = exp(-log(64.0));
    }
}

// One posterior chain (64 threads) per query of a batch.
__global__ void __launch_bounds__(kChainThreads) k_finalize_batch(const FinParams *__restrict__ ps, int n) {
    if (static_cast<int>(blockIdx.x) < n) finalize_chain(ps[blockIdx.x]);
}

}  // namespace

cudaError_t launch_finalize(const FinParams &p, cudaStream_t s) {
    const uint64_t n_cells = static_cast<uint64_t>(p.n_groups) * p.n_specs;
    if (p.mode == PAC_FIN_ADAPTIVE) {
        k_finalize_adaptive<<<1, kChainThreads, 0, s>>>(p);
    } else {
        uint64_t blocks = (n_cells * 32 + 255) / 256;
        if (blocks > 152 * 16) blocks = 152 * 16;
        if (blocks == 0) blocks = 1;
        k_finalize_independent<<<static_cast<unsigned>(blocks), 256, 0, s>>>(p);
    }
    return cudaGetLastError();
}

cudaError_t launch_finalize_batch(const FinParams *d_params, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_finalize_batch<<<static_cast<unsigned>(n), kChainThreads, 0, s>>>(d_params, n);
    return cudaGetLastError();
}

}  // namespace pacgpu
