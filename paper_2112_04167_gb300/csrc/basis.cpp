// One-dimensional GLL and Gauss tables for the kernels (host side, FP64).
//
// GLL points of degree P (Sec. 3.3 basis): -1, 1 and the roots of L_P', found
// by Newton's method from Chebyshev-Gauss-Lobatto guesses; weights
// 2 / (P (P+1) L_P(x_i)^2); differentiation matrix in its closed form
// D_ij = L_P(x_i) / (L_P(x_j) (x_i - x_j)), D_00 = -P(P+1)/4, D_PP = P(P+1)/4.
// Gauss-Legendre points: roots of L_Q by Newton's method, weights
// 2 / ((1 - x^2) L_Q'(x)^2).  Evaluation of Lagrange bases at other points
// uses the barycentric formula; derivatives there are l'(z) = sum_i l_i(z) D_ij,
// exact because l_j' has degree N-2.
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace imex {
namespace {

// Legendre L_n(x) and its derivative by the three-term recurrence.
void legendre(int n, double x, double* L, double* dL) {
  if (n == 0) { *L = 1.0; *dL = 0.0; return; }
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    double d2 = d0 + (2.0 * k - 1.0) * p1;
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *L = p1; *dL = d1;
}

void gll(int N, double* x, double* w) {
  const int P = N - 1;
  x[0] = -1.0; x[P] = 1.0;
  for (int i = 1; i < P; ++i) {
    double z = -std::cos(M_PI * i / P);
    for (int it = 0; it < 100; ++it) {
      double L, dL;
      legendre(P, z, &L, &dL);
      double d2L = (2.0 * z * dL - P * (P + 1.0) * L) / (1.0 - z * z);
      double dz = dL / d2L;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
  }
  for (int i = 0; i < N; ++i) {
    double L, dL;
    legendre(P, x[i], &L, &dL);
    w[i] = 2.0 / (P * (P + 1.0) * L * L);
  }
}

void gauss(int Q, double* x, double* w) {
  for (int i = 0; i < Q; ++i) {
    double z = -std::cos(M_PI * (i + 0.75) / (Q + 0.5));
    for (int it = 0; it < 100; ++it) {
      double L, dL;
      legendre(Q, z, &L, &dL);
      double dz = L / dL;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double L, dL;
    legendre(Q, z, &L, &dL);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dL * dL);
  }
}

void gll_dmatrix(int N, const double* x, double* D) {
  const int P = N - 1;
  std::vector<double> L(N);
  for (int i = 0; i < N; ++i) { double dL; legendre(P, x[i], &L[i], &dL); }
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j)
      D[i * N + j] = (i == j) ? 0.0 : L[i] / (L[j] * (x[i] - x[j]));
  D[0] = -P * (P + 1.0) / 4.0;
  D[P * N + P] = P * (P + 1.0) / 4.0;
}

// E[i*n + j] = l_j(z_i) for the Lagrange basis on nodes x[0..n-1]
void lagrange_at(int n, const double* x, int m, const double* z, double* E) {
  std::vector<double> lam(n);
  for (int j = 0; j < n; ++j) {
    double p = 1.0;
    for (int k = 0; k < n; ++k) if (k != j) p *= (x[j] - x[k]);
    lam[j] = 1.0 / p;
  }
  for (int i = 0; i < m; ++i) {
    int hit = -1;
    for (int j = 0; j < n; ++j) if (z[i] == x[j]) hit = j;
    if (hit >= 0) {
      for (int j = 0; j < n; ++j) E[i * n + j] = (j == hit) ? 1.0 : 0.0;
      continue;
    }
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += lam[j] / (z[i] - x[j]);
    for (int j = 0; j < n; ++j) E[i * n + j] = (lam[j] / (z[i] - x[j])) / s;
  }
}

}  // namespace

void build_tables(Tables<double>* t, Tables<float>* f) {
  std::memset(t, 0, sizeof(*t));
  for (int N = 2; N <= IMEX_MAXN; ++N) {
    gll(N, t->x[N], t->w[N]);
    gll_dmatrix(N, t->x[N], t->D[N]);
    // pressure basis (N-1 GLL points) at the N velocity points
    if (N >= 3) {
      const int Np = N - 1;
      double xp[IMEX_MAXN], wp[IMEX_MAXN], Dp[IMEX_MAXN * IMEX_MAXN];
      gll(Np, xp, wp);
      gll_dmatrix(Np, xp, Dp);
      lagrange_at(Np, xp, N, t->x[N], t->Ipv[N]);
      for (int i = 0; i < N; ++i)
        for (int a = 0; a < Np; ++a) {
          double s = 0.0;
          for (int b = 0; b < Np; ++b) s += t->Ipv[N][i * Np + b] * Dp[b * Np + a];
          t->Gpv[N][i * Np + a] = s;
        }
    }
    const int Q = over_q(N);
    t->Q[N] = Q;
    if (Q <= IMEX_MAXQ) {
      double xg[IMEX_MAXQ];
      gauss(Q, xg, t->gw[N]);
      lagrange_at(N, t->x[N], Q, xg, t->IG[N]);
      for (int g = 0; g < Q; ++g)
        for (int j = 0; j < N; ++j) {
          double s = 0.0;
          for (int i = 0; i < N; ++i) s += t->IG[N][g * N + i] * t->D[N][i * N + j];
          t->DG[N][g * N + j] = s;
        }
    }
  }
  // FP32 copy
  const double* src = reinterpret_cast<const double*>(t);
  const size_t nd = offsetof(Tables<double>, Q) / sizeof(double);
  float* dst = reinterpret_cast<float*>(f);
  for (size_t i = 0; i < nd; ++i) dst[i] = static_cast<float>(src[i]);
  std::memcpy(f->Q, t->Q, sizeof(t->Q));
}

// E[i * Nc + j] = l_j(x_i): the Lagrange cardinal polynomials of the Nc GLL points evaluated
// at the Nf GLL points (the 1D factor of the p-multigrid prolongation)
void gll_interp(int Nc, int Nf, double* E) {
  double xc[IMEX_MAXN], wc[IMEX_MAXN], xf[IMEX_MAXN], wf[IMEX_MAXN];
  gll(Nc, xc, wc);
  gll(Nf, xf, wf);
  lagrange_at(Nc, xc, Nf, xf, E);
}

// 1D SIPG line operators (unit viscosity) for each direction of a Cartesian mesh:
// volume (2/h) sum_q w_q D_qi D_qj, plus the own-element face terms of the interior-penalty
// form at the left (outward normal -1) and right (+1) ends, factor 1/2 on interior faces,
// 1 with penalty 2 tau on Dirichlet faces, nothing on Neumann faces, tau = N^2 / h.
void build_line_ops(const Tables<double>& t, int N, const double* h, int d, LineOps<double>* o,
                    LineOps<float>* f) {
  std::memset(o, 0, sizeof(*o));
  const double* D = t.D[N];
  const double* w = t.w[N];
  for (int k = 0; k < d; ++k) {
    const double s = 2.0 / h[k];
    const double tau = N * N / h[k];
    for (int i = 0; i < N; ++i) o->Wt[k][i] = 0.5 * h[k] * w[i];
    for (int j = 0; j < N; ++j) {
      o->dn[k][0][j] = s * D[(N - 1) * N + j];   // left neighbour: derivative at its right end
      o->dn[k][1][j] = s * D[0 * N + j];         // right neighbour: derivative at its left end
    }
    for (int kl = 0; kl < 3; ++kl)
      for (int kr = 0; kr < 3; ++kr) {
        double* A = o->A[k][3 * kl + kr];
        for (int i = 0; i < N; ++i)
          for (int j = 0; j < N; ++j) {
            double v = 0.0;
            for (int q = 0; q < N; ++q) v += w[q] * D[q * N + i] * D[q * N + j];
            A[i * N + j] = s * v;
          }
        const double fl = (kl == 1) ? 0.5 : (kl == 2 ? 1.0 : 0.0);
        const double fr = (kr == 1) ? 0.5 : (kr == 2 ? 1.0 : 0.0);
        const double tl = (kl == 1) ? tau : (kl == 2 ? 2.0 * tau : 0.0);
        const double tr = (kr == 1) ? tau : (kr == 2 ? 2.0 * tau : 0.0);
        for (int i = 0; i < N; ++i)
          for (int j = 0; j < N; ++j) {
            double v = 0.0;
            // left end, n = -1
            if (i == 0) v += fl * s * D[0 * N + j];
            if (j == 0) v += fl * s * D[0 * N + i];
            if (i == 0 && j == 0) v += tl;
            // right end, n = +1
            if (i == N - 1) v -= fr * s * D[(N - 1) * N + j];
            if (j == N - 1) v -= fr * s * D[(N - 1) * N + i];
            if (i == N - 1 && j == N - 1) v += tr;
            A[i * N + j] += v;
          }
      }
    for (int kind = 0; kind < 3; ++kind) {
      const double fac = (kind == 1) ? 0.5 : (kind == 2 ? 1.0 : 0.0);
      const double pen = (kind == 1) ? tau : (kind == 2 ? 2.0 * tau : 0.0);
      for (int i = 0; i < N; ++i) {
        // left face: trace (or datum) and normal derivative of the neighbour
        o->C[k][0][kind][0][i] = -fac * s * D[0 * N + i] - (i == 0 ? pen : 0.0);
        o->C[k][0][kind][1][i] = (kind == 1 && i == 0) ? 0.5 : 0.0;
        // right face
        o->C[k][1][kind][0][i] = fac * s * D[(N - 1) * N + i] - (i == N - 1 ? pen : 0.0);
        o->C[k][1][kind][1][i] = (kind == 1 && i == N - 1) ? -0.5 : 0.0;
      }
    }
  }
  const double* src = reinterpret_cast<const double*>(o);
  float* dst = reinterpret_cast<float*>(f);
  const size_t n = sizeof(LineOps<double>) / sizeof(double);
  for (size_t i = 0; i < n; ++i) dst[i] = static_cast<float>(src[i]);
}

}  // namespace imex
