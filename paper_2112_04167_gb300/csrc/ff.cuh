// Float-float arithmetic: a value is the unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi) / 2, about 48 significant bits, evaluated on the FP32 pipes.  GB300
// executes FP64 at a small fraction of its FP32 rate; the FP64-bound explicit operators use
// this type for their arithmetic while their inputs and outputs stay FP64 in memory.
//
// Error-free transformations (Knuth's TwoSum, Dekker's FastTwoSum, and the product error
// obtained exactly with one fused multiply-add) give sums and products with a relative
// error of a few units of 2^-48; the addition is the short form that adds the low parts
// without a second TwoSum, so the error of a sum is bounded by that unit times the sum of
// the operands' magnitudes (as for a rounded FP64 addition of rounded operands).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace imex {

struct ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ ff(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ constexpr ff(float x) : hi(x), lo(0.f) {}
  __host__ __device__ constexpr ff(int x) : hi((float)x), lo(0.f) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly (no precondition on the magnitudes)
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return ff(s, e);
}
// s + e = a + b exactly when |a| >= |b|
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
  const float s = a + b;
  return ff(s, b - (s - a));
}

__device__ __forceinline__ ff operator+(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, b.hi);
  return ff_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);                // exact error of the leading product
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ ff operator/(ff a, ff b) {
  const float q1 = a.hi / b.hi;
  const ff r = a - b * ff(q1);
  const float q2 = r.hi / b.hi;
  return ff_fast_two_sum(q1, q2);
}
__device__ __forceinline__ ff& operator+=(ff& a, ff b) { return a = a + b; }
__device__ __forceinline__ ff& operator-=(ff& a, ff b) { return a = a - b; }
__device__ __forceinline__ ff& operator*=(ff& a, ff b) { return a = a * b; }
__device__ __forceinline__ bool operator<(ff a, ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(ff a, ff b) { return b < a; }

// Compensated dot product of float-float operands (the Dot2 scheme of Ogita, Rump and Oishi,
// "Accurate sum and dot product", 2005, with the low parts' cross products added by FMA): the
// high parts' products and running sum are kept exactly by TwoProd / TwoSum, their errors
// and the cross terms m.hi v.lo + m.lo v.hi gather in two FP32 accumulators, and one
// renormalisation at the end gives the float-float result -- as accurate as the operator
// arithmetic above, in about two thirds of its instructions per term.
struct ff_dot {
  float s = 0.f, err = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(ff m, ff v) {
    const float p = m.hi * v.hi;
    const float ep = fmaf(m.hi, v.hi, -p);
    const float t = s + p;
    const float bb = t - s;
    const float es = (s - (t - bb)) + (p - bb);
    s = t;
    err += es + ep;
    lo = fmaf(m.hi, v.lo, fmaf(m.lo, v.hi, lo));
  }
  __device__ __forceinline__ ff value() const {
    const float t = s + (err + lo);
    return ff(t, (err + lo) - (t - s));
  }
};

// Sum of products in the arithmetic type T: plain accumulation for float and double (the
// order of the terms as written), the compensated dot product for float-float
template <typename T>
struct DotAcc {
  T s = T(0);
  __device__ __forceinline__ void add(T m, T v) { s += m * v; }
  __device__ __forceinline__ T value() const { return s; }
};
template <>
struct DotAcc<ff> {
  ff_dot d;
  __device__ __forceinline__ void add(ff m, ff v) { d.add(m, v); }
  __device__ __forceinline__ ff value() const { return d.value(); }
};

template <> __host__ __device__ __forceinline__ ff geom_h<ff>(const Geom& g, int k) { return ff(geom_h<double>(g, k)); }
template <> __host__ __device__ __forceinline__ ff geom_nu0<ff>(const Geom& g) { return ff(g.inu0); }

// table (storage) type of an arithmetic type: ff kernels read the FP64 tables
template <typename T> struct TableType { using type = T; };
template <> struct TableType<ff> { using type = double; };

}  // namespace imex
