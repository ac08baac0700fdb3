// Float-float ("double-float") arithmetic: a value is the unevaluated sum
// hi + lo of two FP32 numbers.  On this GPU the FP64 pipe runs at about 1/64
// of the FP32 rate, so FP64-accurate operator applications (the refinement
// residual and the right-hand side) use this type on the FP32 units.
//
// The operations are the lazy (unnormalised) forms: the leading parts go
// through an error-free transformation -- Knuth's TwoSum for a sum, the FMA
// form of TwoProduct for a product -- and everything smaller is gathered in
// the trailing part with plain FP32 operations, without renormalising the
// pair afterwards.  The pair still represents its value exactly as a sum;
// only the error bound changes from a componentwise to a normwise one: after
// d dependent operations on data of magnitude M the trailing part stays near
// d * 2^-24 * M, so its own rounding adds about d * 2^-48 * M.  FFTs, the
// mode mix and the epilogue need only that normwise bound (a few 1e-14 for
// the depths here), at 8 instructions per addition (20 renormalised) and 4
// per product (7).  The _rn intrinsics keep the compiler from contracting
// the transformations into FMAs.
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

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void ff_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ ff operator+(ff a, ff b) {
    float s, e;
    ff_two_sum(a.hi, b.hi, s, e);
    return ff(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) {
    float s, e;
    ff_two_sum(a.hi, -b.hi, s, e);
    return ff(s, __fadd_rn(e, __fsub_rn(a.lo, b.lo)));
}
// the lo * lo term is below the normwise bound and is dropped
__device__ __forceinline__ ff operator*(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return ff(p, e);
}
__device__ __forceinline__ ff operator*(ff a, float b) {
    const float p = __fmul_rn(a.hi, b);
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return ff(p, e);
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
