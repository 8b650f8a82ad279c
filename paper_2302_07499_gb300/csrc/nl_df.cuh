// Double-float (hi + lo) arithmetic on the FP32 pipes, shared by the
// assembly and the reduction of the FP32 path.
#pragma once

namespace nla {

// Error-free
// transformations (Knuth's TwoSum, and the exact product by fused
// multiply-add), so that strip sums keep about 44 bits without touching the
// narrow FP64 pipe.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF df_add(DF a, DF b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b.hi - bb);
    e += a.lo + b.lo;
    const float h = s + e;
    return DF{h, e - (h - s)};
}
__device__ __forceinline__ DF df_mul(DF a, float x)
{
    const float p = a.hi * x;
    float e = __fmaf_rn(a.hi, x, -p);
    e = __fmaf_rn(a.lo, x, e);
    const float h = p + e;
    return DF{h, e - (h - p)};
}
// double-float times double-float (the products' low parts by fused
// multiply-add; the lo x lo term is below the result's precision)
__device__ __forceinline__ DF df_mul2(DF a, DF b)
{
    const float p = a.hi * b.hi;
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float h = p + e;
    return DF{h, e - (h - p)};
}
// a double constant as float hi + lo (folded at compile time)
__device__ __forceinline__ DF df_const(double d)
{
    const float h = (float)d;
    return DF{h, (float)(d - (double)h)};
}
__device__ __forceinline__ DF df_from(double d)
{
    const float h = (float)d;
    return DF{h, (float)(d - (double)h)};
}
__device__ __forceinline__ double df_to(DF a) { return (double)a.hi + (double)a.lo; }

}  // namespace nla
