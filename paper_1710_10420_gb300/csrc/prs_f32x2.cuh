// prs_f32x2.cuh -- packed FP32 pairs for sm_103a.
//
// Blackwell's add/mul/fma .f32x2 instructions apply one FP32 operation, correctly rounded
// exactly as the scalar instruction would (round to nearest even, no flush of
// subnormals), to the two halves of a 64-bit register pair.  The leapfrog update of
// Eqs. 3-5 is the same chain of operations at every site, so the four sites of a float4
// are updated as two pairs: half the arithmetic instructions of the scalar form, and the
// same result bits as a scalar evaluation in the same order with the same fused
// multiply-adds.
#pragma once

#include <cuda_runtime.h>

namespace prs {

struct f2 {
    unsigned long long r;
};

__device__ __forceinline__ f2 pk2(float a, float b)
{
    f2 p;
    asm("mov.b64 %0, {%1, %2};" : "=l"(p.r) : "f"(a), "f"(b));
    return p;
}

__device__ __forceinline__ void upk2(f2 p, float& a, float& b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(p.r)); }

__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
    return d;
}

__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.r) : "l"(a.r), "l"(b.r));
    return d;
}

// a * b + c with one rounding
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.r) : "l"(a.r), "l"(b.r), "l"(c.r));
    return d;
}

}  // namespace prs
