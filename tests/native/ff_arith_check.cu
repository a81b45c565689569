// Host run of the float-float arithmetic of ff.cuh (the operations the float-float kernels
// execute): for seeded random operands of mixed magnitudes and signs, including near
// cancellations, prints one line per operation with every float in hex, so that a checker
// can compare each result with the exact rational value:
//   add a.hi a.lo b.hi b.lo r.hi r.lo      (and mul, div likewise)
//   dot k m0.hi m0.lo v0.hi v0.lo ... r.hi r.lo
#include <cstdio>
#include <cstdlib>
#include <random>

#include "ff.cuh"

using namespace imex;

static ff rnd(std::mt19937_64& g, int emin, int emax) {
  std::uniform_real_distribution<double> m(0.5, 1.0);
  std::uniform_int_distribution<int> e(emin, emax);
  const double x = std::ldexp(m(g), e(g)) * ((g() & 1) ? -1.0 : 1.0);
  return ff_split_fp64(x);
}

static void pr(ff a) { std::printf(" %a %a", (double)a.hi, (double)a.lo); }

int main(int argc, char** argv) {
  const int n = argc > 1 ? std::atoi(argv[1]) : 2000;
  std::mt19937_64 g(20211208);
  for (int i = 0; i < n; ++i) {
    ff a = rnd(g, -20, 20), b = rnd(g, -20, 20);
    if (i % 4 == 0) b = ff_split_fp64(-(double)a * (1.0 + std::ldexp(1.0, -(int)(g() % 40))));  // cancellation
    std::printf("add");
    pr(a); pr(b); pr(a + b);
    std::printf("\nmul");
    pr(a); pr(b); pr(a * b);
    std::printf("\ndiv");
    pr(a); pr(b); pr(a / b);
    std::printf("\n");
  }
  for (int i = 0; i < n / 4; ++i) {
    const int k = 1 + (int)(g() % 14);
    ff_dot d;
    std::printf("dot %d", k);
    for (int j = 0; j < k; ++j) {
      const ff m = rnd(g, -6, 6), v = rnd(g, -6, 6);
      d.add(m, v);
      pr(m); pr(v);
    }
    pr(d.value());
    std::printf("\n");
  }
  return 0;
}
