// Exact BF16 slicing of float pairs for the tensor-core products (C1/C5 and
// the Gauss-Jordan updates): a value with |x| < 2^E is cut into kC15Slices
// slices s_j = q_j 2^(E - 7 (j + 1)), q_j integer (|q_0| <= 128, |q_j| <= 65
// for j >= 1), each exact in BF16; the remainder is below 2^(E - 42).
#pragma once

#include <cuda_bf16.h>

#include "ff_math.cuh"
#include "qmc_internal.cuh"

namespace qmc {

__device__ __forceinline__ int exp_bound(float x)   // 2^E > 1.001 x (x >= 0)
{
    const float y = x * 1.001f;
    return ((__float_as_int(y) >> 23) & 0xff) - 126;
}

// Slices of the float pair x with |x| < 2^E: s_j = rint(r 2^(7(j+1))) 2^(-7(j+1)),
// r the remainder, computed exactly in float pairs.
__device__ __forceinline__ void slice6(float2 x, int E, float (&s)[kC15Slices])
{
    E = min(max(E, -125), 126);
    const float sc = __int_as_float((127 - E) << 23);
    float2 r = make_float2(x.x * sc, x.y * sc);
#pragma unroll
    for (int j = 0; j < kC15Slices; ++j) {
        const int sh = kC15SliceBits * (j + 1);
        const float q = rintf(r.x * __int_as_float((127 + sh) << 23));
        const float sj = q * __int_as_float((127 - sh) << 23);
        s[j] = sj;
        r = ff::sub(r, make_float2(sj, 0.f));
    }
}

// The same with S slices (S = 7: 49 bits, the Gauss-Jordan updates).
template <int S>
__device__ __forceinline__ void slice_n(float2 x, int E, float (&s)[S])
{
    E = min(max(E, -125), 126);
    const float sc = __int_as_float((127 - E) << 23);
    float2 r = make_float2(x.x * sc, x.y * sc);
#pragma unroll
    for (int j = 0; j < S; ++j) {
        const int sh = kC15SliceBits * (j + 1);
        const float q = rintf(r.x * __int_as_float((127 + sh) << 23));
        const float sj = q * __int_as_float((127 - sh) << 23);
        s[j] = sj;
        r = ff::sub(r, make_float2(sj, 0.f));
    }
}

// x * 2^e exactly (barring underflow or overflow of the result) for |e| <= 250,
// as two multiplications by powers of two that are normal FP32 numbers
__device__ __forceinline__ float scale_pow2(float x, int e)
{
    e = min(max(e, -250), 250);
    const int e1 = e / 2, e2 = e - e1;
    return __fmul_rn(__fmul_rn(x, __int_as_float((127 + e1) << 23)), __int_as_float((127 + e2) << 23));
}

__device__ __forceinline__ uint32_t bf16_pair(float lo, float hi)   // exact: both have <= 8 significant bits
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

}  // namespace qmc
