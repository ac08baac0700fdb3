// Float-float ("double-float") arithmetic: a value is hi + lo with two FP32
// numbers, |lo| <= ulp(hi)/2, about 48 significant bits.  On this GPU the
// FP64 pipe runs at about 1/64 of the FP32 rate, so FP64-accurate operator
// applications (the refinement residual and the right-hand side) use this
// type on the FP32 units.  Built from the error-free transformations of
// Knuth (TwoSum), Dekker (FastTwoSum) and the FMA form of TwoProduct; the
// _rn intrinsics keep the compiler from fusing them into FMAs.
#pragma once
#include <cuda_runtime.h>

struct ff {
    float hi, lo;
    __host__ __device__ ff() {}
    __host__ __device__ constexpr ff(float a, float b) : hi(a), lo(b) {}
    __host__ __device__ constexpr ff(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ constexpr ff(float f) : hi(f), lo(0.f) {}
    __host__ __device__ constexpr ff(int i) : hi((float)i), lo(0.f) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ void ff_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void ff_fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ ff operator+(ff a, ff b) {
    float s, e, t, f;
    ff_two_sum(a.hi, b.hi, s, e);
    ff_two_sum(a.lo, b.lo, t, f);
    e = __fadd_rn(e, t);
    ff_fast_two_sum(s, e, s, e);
    e = __fadd_rn(e, f);
    ff_fast_two_sum(s, e, s, e);
    return ff(s, e);
}
__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff operator*(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    float s;
    ff_fast_two_sum(p, e, s, e);
    return ff(s, e);
}
__device__ __forceinline__ ff operator*(ff a, float b) {
    const float p = __fmul_rn(a.hi, b);
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    float s;
    ff_fast_two_sum(p, e, s, e);
    return ff(s, e);
}
__device__ __forceinline__ ff operator*(float b, ff a) { return a * b; }
__device__ __forceinline__ ff operator*(int b, ff a) { return a * (float)b; }
__device__ __forceinline__ ff& operator+=(ff& a, ff b) { a = a + b; return a; }
__device__ __forceinline__ ff& operator-=(ff& a, ff b) { a = a - b; return a; }

struct ffc {
    ff x, y;
};

// storage conversions
__device__ __forceinline__ ffc to_ffc(double2 v) {
    ffc r;
    r.x = ff(v.x);
    r.y = ff(v.y);
    return r;
}
__device__ __forceinline__ double2 to_double2(ffc v) { return make_double2((double)v.x, (double)v.y); }
