// krig_ff.cuh -- float-float arithmetic for the class solves.
//
// A value is carried as the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2, about 48 significant bits.  This GPU issues FP64 at
// 1/64 of the FP32 rate (2 DFMA against 128 FFMA per SM and cycle), so the
// small class solves keep their extended-precision steps (residuals of the
// FP32 factorisation, the ordinary-kriging combine, the adjoint) in this form.
// Building blocks are the exact transformations TwoSum (Knuth), FastTwoSum
// (Dekker) and TwoProduct by one FMA, composed as in the double-double
// literature (Dekker 1971; Hida, Li and Bailey 2001), and the compensated dot
// product Dot2 (Ogita, Rump and Oishi 2005).  The _rn
// intrinsics keep the compiler from contracting the transformations into FMAs.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_make(float a) { return {a, 0.0f}; }

// s + e = a + b exactly, s = fl(a + b)
__device__ __forceinline__ ff ff_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// the same when |a| >= |b| (or a == 0)
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// p + e = a * b exactly, p = fl(a * b)
__device__ __forceinline__ ff ff_two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    ff s = ff_two_sum(a.hi, b.hi);
    const ff t = ff_two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = ff_fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return ff_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    ff p = ff_two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return ff_fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ ff ff_mul_f(ff a, float b)
{
    ff p = ff_two_prod(a.hi, b);
    p.lo = __fmaf_rn(a.lo, b, p.lo);
    return ff_fast_two_sum(p.hi, p.lo);
}

// exact scaling by a power of two
__device__ __forceinline__ ff ff_scale2(ff a, float p2) { return {__fmul_rn(a.hi, p2), __fmul_rn(a.lo, p2)}; }

// a / b: the FP32 quotient and two correction terms from the float-float remainders
__device__ __forceinline__ ff ff_div(ff a, ff b)
{
    const float q1 = __fdiv_rn(a.hi, b.hi);
    ff r = ff_sub(a, ff_mul_f(b, q1));
    const float q2 = __fdiv_rn(r.hi, b.hi);
    r = ff_sub(r, ff_mul_f(b, q2));
    const float q3 = __fdiv_rn(r.hi, b.hi);
    return ff_add(ff_fast_two_sum(q1, q2), ff_make(q3));
}

// nearest FP32 value of a normalised pair
__device__ __forceinline__ float ff_round(ff a) { return __fadd_rn(a.hi, a.lo); }

__device__ __forceinline__ ff ff_from_double(double d)
{
    const float h = __double2float_rn(d);
    return {h, __double2float_rn(d - (double)h)};
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// Sum over the 32 lanes of a warp (every lane gets the same bits: TwoSum and
// the pair addition are symmetric in their operands).
__device__ __forceinline__ ff ff_warp_sum(ff v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const ff w = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        v = ff_add(v, w);
    }
    return v;
}

// Compensated accumulation acc + sum t_j * x_j (Dot2): the running sum s and
// a compensation c that collects the exact product and sum errors; t_j carries
// a low part that enters c directly.
struct ff_dot {
    float s, c;
    __device__ __forceinline__ explicit ff_dot(ff init) : s(init.hi), c(init.lo) {}
    __device__ __forceinline__ void add(ff t, float x)
    {
        const ff p = ff_two_prod(t.hi, x);
        const ff q = ff_two_sum(s, p.hi);
        s = q.hi;
        c = __fadd_rn(c, __fadd_rn(p.lo, q.lo));
        c = __fmaf_rn(t.lo, x, c);
    }
    __device__ __forceinline__ ff value() const { return ff_two_sum(s, c); }
};
