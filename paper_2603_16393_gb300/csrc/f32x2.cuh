// f32x2.cuh -- packed single-precision arithmetic of sm_100-class GPUs.
//
// One instruction performs the same IEEE float operation (round to nearest
// even) on both halves of a 64-bit register pair, so a thread that updates
// two cells with the same arithmetic issues half the ALU instructions.  The
// results are bitwise those of the scalar operations on each half.
#pragma once

#include <cuda_runtime.h>

namespace fwi {
namespace f2 {

__device__ __forceinline__ unsigned long long bits(float2 a)
{
    return (unsigned long long)__float_as_uint(a.x) |
           ((unsigned long long)__float_as_uint(a.y) << 32);
}

__device__ __forceinline__ float2 from_bits(unsigned long long d)
{
    return make_float2(__uint_as_float((unsigned)d), __uint_as_float((unsigned)(d >> 32)));
}

__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }

__device__ __forceinline__ float2 sub(float2 a, float2 b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(bits(a)), "l"(bits(b)));
    return from_bits(d);
}

__device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }

// a * b + c with one rounding per half
__device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ float2 splat(float s) { return make_float2(s, s); }

__device__ __forceinline__ float2 ld(const float *p) { return *reinterpret_cast<const float2 *>(p); }

__device__ __forceinline__ void st(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }

}  // namespace f2
}  // namespace fwi
