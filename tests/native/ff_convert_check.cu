// Host check of the float-float conversions of ff.cuh: the integer (bit-pattern) forms that
// the GPU kernels use against the FP64 route.  The split must equal the FP64 route bit for
// bit; the join must lie within one unit in the last place of the correctly rounded sum.
// Prints one summary line and exits non-zero on a mismatch.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

#include "ff.cuh"

using namespace imex;

static bool join_ok(ff p, long& bad) {
  const double a = ff_join_bits(p), b = ff_join_fp64(p);
  if (a == b || (std::isnan(a) && std::isnan(b))) return true;
  const double ulp = std::fabs(std::nextafter(b, INFINITY) - b);
  if (std::fabs(a - b) <= ulp) return true;
  if (bad < 5) std::printf("join (%a, %a): bits %.17g fp64 %.17g\n", p.hi, p.lo, a, b);
  ++bad;
  return false;
}

int main(int argc, char** argv) {
  const long n = argc > 1 ? std::atol(argv[1]) : 2000000;
  std::mt19937_64 rng(20211208);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  long bad_split = 0, bad_join = 0, tested = 0;
  for (long it = 0; it < n; ++it) {
    double x = 0.0;
    switch (it % 4) {
      case 0: x = u(rng); break;
      case 1: x = u(rng) * std::ldexp(1.0, (int)(rng() % 240) - 120); break;
      case 2: {                                   // arbitrary finite bit patterns
        const unsigned long long b = rng();
        std::memcpy(&x, &b, 8);
        if (!std::isfinite(x)) continue;
        break;
      }
      default:                                    // exact float plus a small remainder
        x = (double)(float)u(rng) + std::ldexp(u(rng), -24 - (int)(rng() % 12));
    }
    ++tested;
    const ff a = ff_split_bits(x), r = ff_split_fp64(x);
    if (std::memcmp(&a, &r, sizeof(ff)) != 0) {
      if (bad_split < 5) std::printf("split %.17g: bits (%a, %a) fp64 (%a, %a)\n", x, a.hi, a.lo, r.hi, r.lo);
      ++bad_split;
    }
    join_ok(r, bad_join);
    // pairs whose low part reaches below the FP64 significand of the sum
    const float h = (float)u(rng) * std::ldexp(1.0f, (int)(rng() % 120) - 60);
    const float l = (float)(u(rng) * std::ldexp((double)std::fabs(h), -24 - (int)(rng() % 30)));
    join_ok(ff(h, l), bad_join);
  }
  const double special[] = {0.0, -0.0, 1.0, -1.0, 0.5, 2.0, 1e-300, -1e-300, 1e300, 3.4e38, -3.5e38, 1e-38, 5e-324,
                            std::ldexp(1.0, -74), std::ldexp(1.0, 126), std::ldexp(1.0, 127), INFINITY, -INFINITY};
  for (double x : special) {
    const ff a = ff_split_bits(x), r = ff_split_fp64(x);
    const bool same = std::memcmp(&a, &r, sizeof(ff)) == 0 || (std::isnan(a.lo) && std::isnan(r.lo) && a.hi == r.hi);
    if (!same) {
      std::printf("special split %g: bits (%a, %a) fp64 (%a, %a)\n", x, a.hi, a.lo, r.hi, r.lo);
      ++bad_split;
    }
    join_ok(r, bad_join);
  }
  std::printf("tested %ld split_mismatch %ld join_mismatch %ld\n", tested, bad_split, bad_join);
  return (bad_split || bad_join) ? 1 : 0;
}
