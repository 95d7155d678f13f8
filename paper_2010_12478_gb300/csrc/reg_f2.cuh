// Packed FP32x2 helpers (sm_100 and later execute add/mul/fma on two floats per instruction).
// Each lane of a float2 is an independent FP32 value rounded exactly as the scalar operation.
#pragma once

#include <cuda_runtime.h>

namespace reg {

__device__ __forceinline__ float2 f2(float x)
{
    return make_float2(x, x);
}

__device__ __forceinline__ float2 f2sub(float2 a, float2 b)
{
    float2 d;
    asm("{\n .reg .b64 x, y, z;\n mov.b64 x, {%2, %3};\n mov.b64 y, {%4, %5};\n sub.rn.f32x2 z, x, y;\n"
        " mov.b64 {%0, %1}, z;\n}\n"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

// (hi, lo) += x per lane: TwoSum of hi and x, the rounding error into lo.
__device__ __forceinline__ void ff_acc2(float2 &hi, float2 &lo, float2 x)
{
    const float2 s = __fadd2_rn(hi, x);
    const float2 bp = f2sub(s, hi);
    const float2 e = __fadd2_rn(f2sub(hi, f2sub(s, bp)), f2sub(x, bp));
    hi = s;
    lo = __fadd2_rn(lo, e);
}

// acc += x*y per lane, the exact rounding error of each product kept in err.
__device__ __forceinline__ void acc_prod2(float2 &acc, float2 &err, float2 x, float2 y)
{
    const float2 p = __fmul2_rn(x, y);
    err = __fadd2_rn(err, __ffma2_rn(x, y, make_float2(-p.x, -p.y)));
    acc = __fadd2_rn(acc, p);
}

}  // namespace reg
