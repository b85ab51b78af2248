// pac_ops.cuh -- per-world state operations of the per-bit CUDA-core paths
// (single-query kernels and the batched persistent kernel): the identity of
// each state, the update of one world's state by one row, the merge of two
// partial states, and the 64-bit pattern a row contributes.
#pragma once

#include <cfloat>
#include <climits>

#include "pac_kernels.h"

namespace pacgpu {
namespace ops {

__device__ __forceinline__ uint64_t op_identity(int op) {
    switch (op) {
    case OP_IMIN: return static_cast<uint64_t>(LLONG_MAX);
    case OP_IMAX: return static_cast<uint64_t>(LLONG_MIN);
    case OP_FMIN: return 0x7ff0000000000000ull;  // +inf
    case OP_FMAX: return 0xfff0000000000000ull;  // -inf
    default: return 0ull;
    }
}

// Knuth's two-sum: s + e == a + b exactly, s = fl(a + b).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

// state <- state (+) one value for one world; `in` is 0/1 membership.
__device__ __forceinline__ void op_update(int op, uint64_t &st, uint64_t vbits, uint32_t in) {
    switch (op) {
    case OP_ISUM:
        st += in ? vbits : 0ull;
        break;
    case OP_FSUM_COMP: {
        const float x = in ? __int_as_float(static_cast<int>(vbits)) : 0.0f;
        float s = __int_as_float(static_cast<int>(st)), c = __int_as_float(static_cast<int>(st >> 32));
        float ns, e;
        two_sum(s, x, ns, e);
        c += e;
        st = static_cast<uint32_t>(__float_as_int(ns)) | (static_cast<uint64_t>(static_cast<uint32_t>(__float_as_int(c))) << 32);
        break;
    }
    case OP_FSUM_PLAIN: {
        const float x = in ? __int_as_float(static_cast<int>(vbits)) : 0.0f;
        st = static_cast<uint32_t>(__float_as_int(__int_as_float(static_cast<int>(st)) + x));
        break;
    }
    case OP_IMIN: {
        const long long v = static_cast<long long>(vbits);
        if (in && v < static_cast<long long>(st)) st = vbits;
        break;
    }
    case OP_IMAX: {
        const long long v = static_cast<long long>(vbits);
        if (in && v > static_cast<long long>(st)) st = vbits;
        break;
    }
    case OP_FMIN: {
        const double v = __longlong_as_double(static_cast<long long>(vbits));
        if (in && v < __longlong_as_double(static_cast<long long>(st))) st = vbits;
        break;
    }
    case OP_FMAX: {
        const double v = __longlong_as_double(static_cast<long long>(vbits));
        if (in && v > __longlong_as_double(static_cast<long long>(st))) st = vbits;
        break;
    }
    }
}

// a <- a (+) b for two partial states of the same world.
__device__ __forceinline__ void op_merge(int op, uint64_t &a, uint64_t b) {
    switch (op) {
    case OP_ISUM: a += b; break;
    case OP_FSUM_COMP: {
        float s1 = __int_as_float(static_cast<int>(a)), c1 = __int_as_float(static_cast<int>(a >> 32));
        float s2 = __int_as_float(static_cast<int>(b)), c2 = __int_as_float(static_cast<int>(b >> 32));
        float s, e;
        two_sum(s1, s2, s, e);
        const float c = c1 + c2 + e;
        a = static_cast<uint32_t>(__float_as_int(s)) | (static_cast<uint64_t>(static_cast<uint32_t>(__float_as_int(c))) << 32);
        break;
    }
    case OP_FSUM_PLAIN:
        a = static_cast<uint32_t>(__float_as_int(__int_as_float(static_cast<int>(a)) + __int_as_float(static_cast<int>(b))));
        break;
    default: op_update(op, a, b, 1u); break;
    }
}

// Raw 64-bit value pattern of row i for a slot: int64 as is, floats as
// float bits (SUM) or double bits (MIN/MAX).
__device__ __forceinline__ uint64_t load_slot_value(const SlotDev &s, uint64_t i) {
    switch (s.op) {
    case OP_ISUM: case OP_IMIN: case OP_IMAX:
        return static_cast<uint64_t>(row_i64(s.values, i));
    case OP_FSUM_COMP: case OP_FSUM_PLAIN:
        return static_cast<uint32_t>(__float_as_int(static_cast<float>(row_f(s.values, s.vtype, i))));
    default:
        return static_cast<uint64_t>(__double_as_longlong(row_f(s.values, s.vtype, i)));
    }
}

}  // namespace ops
}  // namespace pacgpu
