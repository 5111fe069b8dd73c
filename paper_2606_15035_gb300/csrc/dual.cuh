// Forward-mode dual numbers (value + one directional derivative) for the adjoint of the step.
//
// The per-particle part of the step -- the orbit breakpoints, the Appendix A/B closed-form
// orbit integrals, the gathers and the point interpolant -- is a piecewise polynomial in the
// particle's start position and displacement.  Evaluating the same templated code with Dual
// seeds one input direction and returns the exact derivative of every result along it: the
// breakpoints s_m = (knot - x0) / beta carry their own derivative, so the motion of the piece
// limits (and with it the jump terms of the D_i A integrand at knot crossings, §4.3) is part
// of the result.  Comparisons, floor and ceil act on the value (the piece structure is
// locally constant); the derivative of floor is zero.
#pragma once

#include <cuda_runtime.h>

namespace pic {

using ::ceil;
using ::fabs;
using ::floor;
using ::fmax;
using ::fmin;

struct Dual {
    double v, d;
    __host__ __device__ __forceinline__ Dual() : v(0.0), d(0.0) {}
    __host__ __device__ __forceinline__ Dual(double a) : v(a), d(0.0) {}
    __host__ __device__ __forceinline__ Dual(int a) : v((double)a), d(0.0) {}
    __host__ __device__ __forceinline__ Dual(double a, double b) : v(a), d(b) {}
    __device__ __forceinline__ explicit operator int() const { return (int)v; }
};

__device__ __forceinline__ Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
    const double q = a.v / b.v;
    return Dual(q, (a.d - q * b.d) / b.v);
}
__device__ __forceinline__ Dual& operator+=(Dual& a, Dual b) { return a = a + b; }
__device__ __forceinline__ Dual& operator-=(Dual& a, Dual b) { return a = a - b; }
__device__ __forceinline__ Dual& operator*=(Dual& a, Dual b) { return a = a * b; }

__device__ __forceinline__ bool operator<(Dual a, Dual b) { return a.v < b.v; }
__device__ __forceinline__ bool operator>(Dual a, Dual b) { return a.v > b.v; }
__device__ __forceinline__ bool operator<=(Dual a, Dual b) { return a.v <= b.v; }
__device__ __forceinline__ bool operator>=(Dual a, Dual b) { return a.v >= b.v; }
__device__ __forceinline__ bool operator==(Dual a, Dual b) { return a.v == b.v; }
__device__ __forceinline__ bool operator!=(Dual a, Dual b) { return a.v != b.v; }

__device__ __forceinline__ Dual floor(Dual a) { return Dual(::floor(a.v), 0.0); }
__device__ __forceinline__ Dual ceil(Dual a) { return Dual(::ceil(a.v), 0.0); }
__device__ __forceinline__ Dual fmin(Dual a, Dual b) { return b.v < a.v ? b : a; }
__device__ __forceinline__ Dual fmax(Dual a, Dual b) { return a.v < b.v ? b : a; }
__device__ __forceinline__ Dual fabs(Dual a) { return a.v < 0.0 ? -a : a; }

}  // namespace pic
