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
  __host__ __device__ inline ff(double x);
  __host__ __device__ constexpr ff(float x) : hi(x), lo(0.f) {}
  __host__ __device__ constexpr ff(int x) : hi((float)x), lo(0.f) {}
  __host__ __device__ inline explicit operator double() const;
};

// Conversions between FP64 and float-float.  On this GPU the FP64 pipe -- which also
// executes the FP32 <-> FP64 conversions -- issues at a small fraction of the FP32 rate, so
// a kernel that converts every FP64 value it loads or stores spends most of its time there.
// The device forms below work on the bit patterns with integer operations instead; values
// whose parts would leave the normal FP32 range take the FP64 route (the host always does).
namespace ffbits {
__host__ __device__ __forceinline__ unsigned long long d2u(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long u;
  __builtin_memcpy(&u, &x, 8);
  return u;
#endif
}
__host__ __device__ __forceinline__ double u2d(unsigned long long u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double x;
  __builtin_memcpy(&x, &u, 8);
  return x;
#endif
}
__host__ __device__ __forceinline__ unsigned f2u(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  unsigned u;
  __builtin_memcpy(&u, &x, 4);
  return u;
#endif
}
__host__ __device__ __forceinline__ float u2f(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float x;
  __builtin_memcpy(&x, &u, 4);
  return x;
#endif
}
}  // namespace ffbits

// the FP64 route: hi = x rounded to FP32, lo = the rest rounded to FP32
__host__ __device__ __forceinline__ ff ff_split_fp64(double x) {
  const float h = (float)x;
  return ff(h, (float)(x - (double)h));
}
__host__ __device__ __forceinline__ double ff_join_fp64(ff a) { return (double)a.hi + (double)a.lo; }
// the same out of line, for the rare operands of the integer forms: a call keeps their FP64
// instructions on a branch of their own (inlined, they would be predicated into every use)
static __host__ __device__ __noinline__ ff ff_split_rare(double x) { return ff_split_fp64(x); }
static __host__ __device__ __noinline__ double ff_join_rare(ff a) { return ff_join_fp64(a); }

// x = M 2^(e - 1075) with the 53-bit significand M, in 32-bit words: hi takes M's leading 24
// bits rounded to nearest (ties to even), lo the remainder R (|R| <= 2^28) rounded to FP32
// and scaled by the exact power of two -- the FP64 route's result bit for bit.  Both parts
// are normal floats for biased exponents e in [953, 1149]; zero is exact; anything else
// takes the FP64 route.
__host__ __device__ __forceinline__ ff ff_split_bits(double x) {
  using namespace ffbits;
  const unsigned long long b = d2u(x);
  const unsigned bh = (unsigned)(b >> 32), bl = (unsigned)b;
  if (((bh << 1) | bl) == 0u) return ff(u2f(bh), 0.f);                     // +-0
  const unsigned e = (bh >> 20) & 0x7ffu;
  if (e - 953u > 196u) return ff_split_rare(x);
  // rounding bit 28 of the low word, to even on a tie
  const unsigned rnd = (bl >> 28) & (((bl & 0x0fffffffu) != 0u) | (bl >> 29)) & 1u;
  // exponent and the leading 23 fraction bits (the sign and the exponent's top bits shift
  // out; the rebias is taken modulo 2^32), a carried rounding moves into the exponent
  const unsigned hmag = (((bh << 3) | (bl >> 29)) - (896u << 23)) + rnd;
  const int R = (int)(bl & 0x1fffffffu) - (int)(rnd << 29);
  const float scale = u2f((e - 948u) << 23);                                // 2^(e - 1075)
  return ff(u2f((bh & 0x80000000u) | hmag), (float)((bh >> 31) ? -R : R) * scale);
}

// hi + lo to FP64 in 32-bit words: FP64 bits of hi, then lo's significand added to (or taken
// from) the 64-bit pattern in units of hi's FP64 last place (rounded to that unit: within one
// unit of the correctly rounded sum).  A normalised lo never carries into the exponent; when
// hi is a power of two and lo has the other sign the sum lies in the binade below, whose unit
// is half as large.  Zero, subnormal or non-finite high parts, subnormal low parts and low
// parts that are not normalised take the FP64 route.
__host__ __device__ __forceinline__ double ff_join_bits(ff a) {
  using namespace ffbits;
  const unsigned hb = f2u(a.hi), lb = f2u(a.lo);
  const unsigned eh = (hb >> 23) & 0xffu;
  if (eh - 1u > 253u) return ff_join_rare(a);
  const unsigned hw = (hb & 0x80000000u) | (((hb & 0x7fffffffu) >> 3) + (896u << 20));
  unsigned long long v = ((unsigned long long)hw << 32) | (unsigned long long)(hb << 29);
  if ((lb << 1) != 0u) {
    const unsigned el = (lb >> 23) & 0xffu;
    const int d = (int)eh - (int)el;
    if (el == 0u || d < 24) return ff_join_rare(a);
    const bool opp = ((hb ^ lb) & 0x80000000u) != 0u;
    const int sh = 29 - d + ((opp && (hb & 0x7fffffu) == 0u) ? 1 : 0);
    const unsigned Sl = (lb & 0x7fffffu) | 0x800000u;
    const unsigned L = sh >= 0 ? (Sl << sh) : (sh > -25 ? ((Sl + (1u << (-sh - 1))) >> (-sh)) : 0u);
    v = opp ? v - L : v + L;
  }
  return u2d(v);
}

__host__ __device__ inline ff::ff(double x) {
#ifdef __CUDA_ARCH__
  *this = ff_split_bits(x);
#else
  *this = ff_split_fp64(x);
#endif
}
__host__ __device__ inline ff::operator double() const {
#ifdef __CUDA_ARCH__
  return ff_join_bits(*this);
#else
  return ff_join_fp64(*this);
#endif
}

// The operations below compile for the host as well (the same FP32 operations), so that
// host programs can check them against exact arithmetic.

// s + e = a + b exactly (no precondition on the magnitudes)
__host__ __device__ __forceinline__ ff ff_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return ff(s, e);
}
// s + e = a + b exactly when |a| >= |b|
__host__ __device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
  const float s = a + b;
  return ff(s, b - (s - a));
}

__host__ __device__ __forceinline__ ff operator+(ff a, ff b) {
  const ff s = ff_two_sum(a.hi, b.hi);
  return ff_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__host__ __device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__host__ __device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);                // exact error of the leading product
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return ff_fast_two_sum(p, e);
}
__host__ __device__ __forceinline__ ff operator/(ff a, ff b) {
  const float q1 = a.hi / b.hi;
  const ff r = a - b * ff(q1);
  const float q2 = r.hi / b.hi;
  return ff_fast_two_sum(q1, q2);
}
__host__ __device__ __forceinline__ ff& operator+=(ff& a, ff b) { return a = a + b; }
__host__ __device__ __forceinline__ ff& operator-=(ff& a, ff b) { return a = a - b; }
__host__ __device__ __forceinline__ ff& operator*=(ff& a, ff b) { return a = a * b; }
__host__ __device__ __forceinline__ bool operator<(ff a, ff b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__host__ __device__ __forceinline__ bool operator>(ff a, ff b) { return b < a; }

// Compensated dot product of float-float operands (the Dot2 scheme of Ogita, Rump and Oishi,
// "Accurate sum and dot product", 2005, with the low parts' cross products added by FMA): the
// high parts' products and running sum are kept exactly by TwoProd / TwoSum, their errors
// and the cross terms m.hi v.lo + m.lo v.hi gather in two FP32 accumulators, and one
// renormalisation at the end gives the float-float result -- as accurate as the operator
// arithmetic above, in about two thirds of its instructions per term.
struct ff_dot {
  float s = 0.f, err = 0.f, lo = 0.f;
  __host__ __device__ __forceinline__ void add(ff m, ff v) {
    const float p = m.hi * v.hi;
    const float ep = fmaf(m.hi, v.hi, -p);
    const float t = s + p;
    const float bb = t - s;
    const float es = (s - (t - bb)) + (p - bb);
    s = t;
    err += es + ep;
    lo = fmaf(m.hi, v.lo, fmaf(m.lo, v.hi, lo));
  }
  __host__ __device__ __forceinline__ ff value() const {
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
