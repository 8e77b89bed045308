// Float-float ("double-float") arithmetic on the FP32 pipes: a value is an
// unevaluated sum x + y of two floats (float2: .x high part, .y low part,
// |y| <= ulp(x)/2), ~48 significant bits.  The FP32 pipe of this GPU runs 64
// lanes of FMA for each FP64 lane, so FP64-class quantities on the mixed path
// are computed this way.
//
// Error-free transformations: Knuth's TwoSum, Dekker's Fast2Sum and the FMA
// product error.  Every addition and multiplication whose rounding error is
// recovered afterwards is written with the _rn intrinsics, which the compiler
// never contracts into an FMA (a contracted s = fma(a, b, c) would no longer
// be the rounded sum the error term is computed for).
//
// exp(-x): Cody-Waite reduction by ln 2 (W. J. Cody and W. Waite, "Software
// Manual for the Elementary Functions", 1980), a table of exp(-j/32) (P. T. P.
// Tang, "Table-driven implementation of the exponential function in IEEE
// floating-point arithmetic", ACM TOMS 15, 1989) and the Taylor series of the
// remaining factor.
#pragma once

#include <cuda_runtime.h>

namespace qmc {
namespace ff {

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)   // |a| >= |b| or a == 0
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ float2 renorm(float a, float b)
{
    float s, e;
    fast_two_sum(a, b, s, e);
    return make_float2(s, e);
}

__device__ __forceinline__ float2 add(float2 a, float2 b)
{
    float s, e;
    two_sum(a.x, b.x, s, e);
    e = __fadd_rn(e, __fadd_rn(a.y, b.y));
    return renorm(s, e);
}

__device__ __forceinline__ float2 neg(float2 x) { return make_float2(-x.x, -x.y); }
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return add(a, neg(b)); }

__device__ __forceinline__ float2 mul(float2 a, float2 b)
{
    const float p = __fmul_rn(a.x, b.x);
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    return renorm(p, e);
}

__device__ __forceinline__ float2 mulf(float2 a, float b)   // b a float
{
    const float p = __fmul_rn(a.x, b);
    const float e = fmaf(a.y, b, fmaf(a.x, b, -p));
    return renorm(p, e);
}

// acc + x * y
__device__ __forceinline__ float2 fma2(float2 acc, float2 x, float2 y)
{
    const float p = __fmul_rn(x.x, y.x);
    float pe = fmaf(x.x, y.x, -p);
    pe = fmaf(x.x, y.y, pe);
    pe = fmaf(x.y, y.x, pe);
    float s, se;
    two_sum(acc.x, p, s, se);
    se = __fadd_rn(se, __fadd_rn(acc.y, pe));
    return renorm(s, se);
}

// 1 / x: FP32 reciprocal refined by one Newton step in float-float
__device__ __forceinline__ float2 inv(float2 x)
{
    const float q = 1.0f / x.x;
    const float2 px = mulf(x, q);
    float rh, rl;
    two_sum(1.0f, -px.x, rh, rl);
    rl = __fsub_rn(rl, px.y);
    const float r = __fadd_rn(rh, rl);
    return renorm(q, __fmul_rn(q, r));
}

__device__ __forceinline__ double val(float2 x) { return (double)x.x + (double)x.y; }

__device__ __forceinline__ float2 from_double(double v)
{
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}

// exp(-x) for x >= 0 (a float pair), 0 for x >= 87 (below the FP32 range).
//   x = k ln2 + r,  |r| <= ln2/2, ln2 = L1 + L2 with L1 of 15 significant bits
//                   so that k L1 (k <= 126) and x - k L1 are exact;
//   r = j/32 + s,   |s| <= 1/64, T[j + 12] = exp(-j/32) as a float pair;
//   exp(-s) = 1 - s + s^2/2 + tail, the tail -s^3/6 + ... + s^6/720 in FP32
//   (|tail| < 2^-19, its rounding < 2^-43; the first omitted term < 2^-54).
// exp(-x) = 2^-k T[j] exp(-s), the power of two applied by multiplication.
__device__ __forceinline__ float2 exp_neg(float2 x, const float2 *__restrict__ T)
{
    if (!(x.x < 87.0f)) return make_float2(0.f, 0.f);
    constexpr float kInvLn2 = 1.44269504088896340736f;
    constexpr float kL1 = 0x1.62e4p-1f;
    const float2 kL2 = make_float2(0x1.7f7d1cp-20f, 0x1.ef357ap-45f);
    const float kf = rintf(__fmul_rn(x.x, kInvLn2));
    float rh, rl;
    two_sum(__fsub_rn(x.x, __fmul_rn(kf, kL1)), x.y, rh, rl);
    const float2 r = sub(make_float2(rh, rl), mulf(kL2, kf));
    const float jf = rintf(__fmul_rn(r.x, 32.0f));
    float sh, sl;
    two_sum(__fsub_rn(r.x, __fmul_rn(jf, 0.03125f)), r.y, sh, sl);
    const float2 sv = make_float2(sh, sl);
    const float s = sh;
    const float tail = s * s * s * (-1.0f / 6.0f + s * (1.0f / 24.0f + s * (-1.0f / 120.0f + s * (1.0f / 720.0f))));
    const float2 s2 = mul(sv, sv);
    float2 p = add(make_float2(1.0f, 0.f), neg(sv));
    p = add(p, make_float2(0.5f * s2.x, 0.5f * s2.y));
    p = add(p, make_float2(tail, 0.f));
    const float2 e = mul(p, T[(int)jf + 12]);
    const float scale = __int_as_float((127 - (int)kf) << 23);   // 2^-k, k in [0, 126]: a normal float
    return make_float2(__fmul_rn(e.x, scale), __fmul_rn(e.y, scale));
}

}  // namespace ff
}  // namespace qmc
