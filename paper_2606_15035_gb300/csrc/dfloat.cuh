// FP32-pair ("double-float") arithmetic on the FP32 pipes (sm_103a).
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2, which carries
// a 48-bit significand (relative rounding ~2^-48 = 3.6e-15) at FP32 throughput: on this GPU the
// FP32 pipes issue 64 times as many FMAs per clock as the FP64 pipe, and one pair operation
// costs 3 to 11 FP32 instructions.  The building blocks are the classical error-free
// transformations: Knuth's TwoSum (a + b = s + e exactly), Dekker's Fast2Sum (the same for
// |a| >= |b|) and the FMA product error (a b = p + e exactly with e = fma(a, b, -p)).  Sums use
// the short form (one TwoSum of the high parts, the low parts added once, renormalised), whose
// error is ~2^-47 of the larger operand; that absolute accuracy is what the orbit integrals
// need, because every quantity they combine is bounded by the particle's speed or the mesh
// fields' size.
#pragma once

#include <cuda_runtime.h>

namespace pic {

// The pair overloads below sit beside the standard ones, so that code in this namespace
// still finds floor(double), fmin(double, double), ... by ordinary lookup.
using ::ceil;
using ::fabs;
using ::floor;
using ::fmax;
using ::fmin;

struct DF {
    float hi, lo;
    __host__ __device__ __forceinline__ DF() : hi(0.f), lo(0.f) {}
    __host__ __device__ __forceinline__ DF(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ __forceinline__ DF(float a) : hi(a), lo(0.f) {}
    __host__ __device__ __forceinline__ DF(int a) : hi((float)a), lo(0.f) {}
    // from a double constant or value: the nearest float and the float of the remainder
    __host__ __device__ __forceinline__ DF(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    // an integral pair (a floor or ceil of a position in cells, |value| < 2^24) as an int
    __device__ __forceinline__ explicit operator int() const { return (int)hi + (int)lo; }
};

__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return DF(s, (a - (s - bb)) + (b - bb));
}

__device__ __forceinline__ DF fast_two_sum(float a, float b) {
    const float s = a + b;
    return DF(s, b - (s - a));
}

__device__ __forceinline__ DF two_prod(float a, float b) {
    const float p = a * b;
    return DF(p, fmaf(a, b, -p));
}

__device__ __forceinline__ DF operator-(DF a) { return DF(-a.hi, -a.lo); }

__device__ __forceinline__ DF operator+(DF a, DF b) {
    const DF s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ DF operator-(DF a, DF b) { return a + (-b); }

__device__ __forceinline__ DF operator*(DF a, DF b) {
    const DF p = two_prod(a.hi, b.hi);
    return fast_two_sum(p.hi, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo)));
}

__device__ __forceinline__ DF operator*(DF a, float b) {
    const DF p = two_prod(a.hi, b);
    return fast_two_sum(p.hi, fmaf(a.lo, b, p.lo));
}

__device__ __forceinline__ DF operator*(float b, DF a) { return a * b; }

// One float quotient, then one correction from the exact-enough remainder a - q b.
__device__ __forceinline__ DF operator/(DF a, DF b) {
    const float q1 = a.hi / b.hi;
    const DF r = a - b * q1;
    const float q2 = r.hi / b.hi;
    return fast_two_sum(q1, q2);
}

__device__ __forceinline__ DF& operator+=(DF& a, DF b) { return a = a + b; }
__device__ __forceinline__ DF& operator-=(DF& a, DF b) { return a = a - b; }
__device__ __forceinline__ DF& operator*=(DF& a, DF b) { return a = a * b; }

__device__ __forceinline__ bool operator<(DF a, DF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(DF a, DF b) { return b < a; }
__device__ __forceinline__ bool operator<=(DF a, DF b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(DF a, DF b) { return !(a < b); }
__device__ __forceinline__ bool operator==(DF a, DF b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(DF a, DF b) { return !(a == b); }

__device__ __forceinline__ DF floor(DF a) {
    const float fh = floorf(a.hi);
    if (fh != a.hi) return DF(fh, 0.f);
    return fast_two_sum(fh, floorf(a.lo));
}

__device__ __forceinline__ DF ceil(DF a) {
    const float ch = ceilf(a.hi);
    if (ch != a.hi) return DF(ch, 0.f);
    return fast_two_sum(ch, ceilf(a.lo));
}

__device__ __forceinline__ DF fmin(DF a, DF b) { return b < a ? b : a; }
__device__ __forceinline__ DF fmax(DF a, DF b) { return a < b ? b : a; }
__device__ __forceinline__ DF fabs(DF a) { return a.hi < 0.f ? -a : a; }

// double -> pair and pair -> double (two FP64 operations each way; used at the kernel's edges)
__device__ __forceinline__ DF df_of(double d) {
    const float h = (float)d;
    return DF(h, (float)(d - (double)h));
}
__device__ __forceinline__ double dbl_of(DF a) { return (double)a.hi + (double)a.lo; }

}  // namespace pic
