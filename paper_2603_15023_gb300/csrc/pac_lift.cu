// pac_lift.cu -- vector-lifted expressions (Sec. 4.2 "Vector-lifted
// Expression, and Lambda Functions": a scalar expression applied world by
// world, scalar operands broadcast; Sec. 7 evaluates the ratio of two
// pac_sum vectors this way and noises it once) and pac_filter (Sec. 3.2
// "Categorical Rewrites": the fraction of true worlds is the probability of
// a random yes/no choice).
//
// k_lift: one thread per (group, world) cell runs the postfix program, which
// sits in the kernel parameters, so every thread takes the same branches.
// Memory-bound: 8 bytes per operand in, 8 out per cell.
// k_filter: one warp per group counts its true worlds with two ballots.
#include "pac_internal.cuh"
#include "pac_kernels.h"

namespace pacgpu {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint64_t kStreamFilter = 3;

__device__ __forceinline__ double operand(const LiftParams &p, int k, uint64_t cell) {
    const int code = p.code[k];
    const unsigned long long b = __ldg(static_cast<const unsigned long long *>(p.in[k]) + cell);
    const double v = (code & 3) == 0   ? static_cast<double>(b)
                     : (code & 3) == 1 ? static_cast<double>(static_cast<long long>(b))
                                       : __longlong_as_double(static_cast<long long>(b));
    return (code & 4) ? 2.0 * v : v;
}

__global__ void __launch_bounds__(256) k_lift(const __grid_constant__ LiftParams p) {
    const uint64_t n = static_cast<uint64_t>(p.n_groups) * kWorlds;
    const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    for (uint64_t cell = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; cell < n; cell += stride) {
        double st[PAC_LIFT_DEPTH];
        int sp = 0;
        for (int k = 0; k < p.n_ops; k++) {
            const int op = p.prog[k].op;
            if (op == PAC_LIFT_SPEC) {
                st[sp++] = operand(p, p.prog[k].arg, cell);
                continue;
            }
            if (op == PAC_LIFT_CONST) {
                st[sp++] = p.prog[k].c;
                continue;
            }
            if (op == PAC_LIFT_NEG) {
                st[sp - 1] = -st[sp - 1];
                continue;
            }
            if (op == PAC_LIFT_ABS) {
                st[sp - 1] = fabs(st[sp - 1]);
                continue;
            }
            const double b = st[--sp], a = st[sp - 1];
            double r;
            switch (op) {
            case PAC_LIFT_ADD: r = a + b; break;
            case PAC_LIFT_SUB: r = a - b; break;
            case PAC_LIFT_MUL: r = a * b; break;
            case PAC_LIFT_DIV: r = a / b; break;
            case PAC_LIFT_MIN: r = a < b ? a : b; break;
            case PAC_LIFT_MAX: r = a > b ? a : b; break;
            case PAC_LIFT_LT: r = a < b ? 1.0 : 0.0; break;
            case PAC_LIFT_LE: r = a <= b ? 1.0 : 0.0; break;
            case PAC_LIFT_EQ: r = a == b ? 1.0 : 0.0; break;
            case PAC_LIFT_NE: r = a != b ? 1.0 : 0.0; break;
            case PAC_LIFT_GT: r = a > b ? 1.0 : 0.0; break;
            default: r = a >= b ? 1.0 : 0.0; break;
            }
            st[sp - 1] = r;
        }
        p.out[cell] = st[0];
    }
}

__global__ void __launch_bounds__(256) k_filter(const double *__restrict__ b, uint32_t n_groups, uint64_t seed,
                                                uint8_t *__restrict__ keep) {
    const int lane = threadIdx.x & 31;
    const uint64_t wid = (blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x) >> 5;
    const uint64_t n_w = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
    for (uint64_t g = wid; g < n_groups; g += n_w) {
        const double *row = b + g * kWorlds;
        const uint32_t t0 = __ballot_sync(kFull, __ldg(row + lane) != 0.0);
        const uint32_t t1 = __ballot_sync(kFull, __ldg(row + lane + 32) != 0.0);
        if (lane == 0) {
            const int t = __popc(t0) + __popc(t1);
            const double u = static_cast<double>(counter_draw(seed, kStreamFilter, g) >> 11) * 0x1.0p-53;
            keep[g] = u < static_cast<double>(t) / 64.0 ? 1 : 0;
        }
    }
}

}  // namespace

cudaError_t launch_lift(const LiftParams &p, int n_sms, cudaStream_t s) {
    const uint64_t n = static_cast<uint64_t>(p.n_groups) * kWorlds;
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + 255) / 256;
    const uint64_t cap = static_cast<uint64_t>(n_sms) * 8;
    if (blocks > cap) blocks = cap;
    k_lift<<<static_cast<unsigned>(blocks), 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_filter(const double *b, uint32_t n_groups, uint64_t seed, uint8_t *keep, int n_sms,
                          cudaStream_t s) {
    if (n_groups == 0) return cudaSuccess;
    uint64_t blocks = (static_cast<uint64_t>(n_groups) * 32 + 255) / 256;
    const uint64_t cap = static_cast<uint64_t>(n_sms) * 8;
    if (blocks > cap) blocks = cap;
    k_filter<<<static_cast<unsigned>(blocks), 256, 0, s>>>(b, n_groups, seed, keep);
    return cudaGetLastError();
}

}  // namespace pacgpu
