// Shared device helpers for the S2LET GPU library: complex arithmetic on
// double2 / float2 and error-free FP32 operations for float-float values.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace s2g {

template <typename R> struct ctype;
template <> struct ctype<double> { using T = double2; };
template <> struct ctype<float> { using T = float2; };
template <typename R> using cplx_t = typename ctype<R>::T;

__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b)
{
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b)
{
    C r;
    r.x = a.x * b.x + a.y * b.y;
    r.y = a.y * b.x - a.x * b.y;
    return r;
}
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) { a.x *= s; a.y *= s; return a; }

template <typename Cd, typename Cs> __device__ __forceinline__ Cd ccast(Cs a)
{
    Cd r;
    r.x = a.x;
    r.y = a.y;
    return r;
}

// ---------------------------------------------------------------- float-float
// Unevaluated sums hi + lo of two FP32 numbers.  The _rn intrinsics are never
// contracted into FMAs by the compiler, which the error-free transformations
// below rely on.
struct ff {
    float h, l;
};

// hi + lo = a * b exactly (FMA-based product).
__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    float ph = __fmul_rn(a.h, b.h);
    float pl = __fmaf_rn(a.h, b.h, -ph);
    pl = __fmaf_rn(a.h, b.l, pl);
    pl = __fmaf_rn(a.l, b.h, pl);
    ff r;
    r.h = ph;
    r.l = pl;
    return r;
}

// a - b with a two-sum on the high parts and renormalisation.
__device__ __forceinline__ ff ff_sub(ff a, ff b)
{
    float sh = __fsub_rn(a.h, b.h);
    float v = __fsub_rn(sh, a.h);
    float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(sh, v)), __fsub_rn(-b.h, v));
    float rl = __fadd_rn(e, __fsub_rn(a.l, b.l));
    ff r;
    r.h = __fadd_rn(sh, rl);
    r.l = __fsub_rn(rl, __fsub_rn(r.h, sh));
    return r;
}

}  // namespace s2g
