// Host dump of the one-dimensional tables the kernels read (basis.cpp build_tables,
// gll_interp and build_line_ops): one line per table, "name N [indices] v0 v1 ...", every
// value printed with 17 significant digits, for N = 2 .. IMEX_MAXN points per direction.
// Only host code runs.
#include <cstdio>

#include "common.cuh"

using namespace imex;

static void row(const char* name, int N, const double* v, int n) {
  std::printf("%s %d", name, N);
  for (int i = 0; i < n; ++i) std::printf(" %.17g", v[i]);
  std::printf("\n");
}

int main() {
  static Tables<double> t;
  static Tables<float> f;
  build_tables(&t, &f);
  for (int N = 2; N <= IMEX_MAXN; ++N) {
    row("x", N, t.x[N], N);
    row("w", N, t.w[N], N);
    row("D", N, t.D[N], N * N);
    if (N >= 3) {
      row("Ipv", N, t.Ipv[N], N * (N - 1));
      row("Gpv", N, t.Gpv[N], N * (N - 1));
    }
    const int Q = t.Q[N];
    std::printf("Q %d %d\n", N, Q);
    if (Q <= IMEX_MAXQ) {
      row("gw", N, t.gw[N], Q);
      row("IG", N, t.IG[N], Q * N);
      row("DG", N, t.DG[N], Q * N);
    }
    // the FP32 copy is the FP64 table rounded
    double xf[IMEX_MAXN];
    for (int i = 0; i < N; ++i) xf[i] = (double)f.x[N][i];
    row("x32", N, xf, N);
  }
  // p-multigrid prolongation factors between GLL sets (coarse Nc, fine Nf)
  static double E[IMEX_MAXN * IMEX_MAXN];
  for (int Nf = 3; Nf <= IMEX_MAXN; ++Nf)
    for (int Nc = 2; Nc < Nf; ++Nc) {
      gll_interp(Nc, Nf, E);
      std::printf("E %d %d", Nc, Nf);
      for (int i = 0; i < Nc * Nf; ++i) std::printf(" %.17g", E[i]);
      std::printf("\n");
    }
  // 1D SIPG line operators of a unit element (h = 1, unit viscosity): own blocks for every
  // pair of face kinds, the neighbour couplings of every side and face kind, the rows forming
  // a neighbour's normal derivative
  static LineOps<double> o;
  static LineOps<float> of;
  const double one[3] = {1.0, 1.0, 1.0};
  for (int N = 2; N <= IMEX_MAXN; ++N) {
    build_line_ops(t, N, one, 1, &o, &of);
    for (int kl = 0; kl < 3; ++kl)
      for (int kr = 0; kr < 3; ++kr) {
        std::printf("LA %d %d %d", N, kl, kr);
        for (int i = 0; i < N * N; ++i) std::printf(" %.17g", o.A[0][3 * kl + kr][i]);
        std::printf("\n");
      }
    for (int side = 0; side < 2; ++side) {
      for (int kind = 0; kind < 3; ++kind)
        for (int c = 0; c < 2; ++c) {
          std::printf("LC %d %d %d %d", N, side, kind, c);
          for (int i = 0; i < N; ++i) std::printf(" %.17g", o.C[0][side][kind][c][i]);
          std::printf("\n");
        }
      std::printf("LDN %d %d", N, side);
      for (int j = 0; j < N; ++j) std::printf(" %.17g", o.dn[0][side][j]);
      std::printf("\n");
    }
  }
  return 0;
}
