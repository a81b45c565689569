// Flow statistics of Sec. 4.3 (evaluated between steps, not part of a step):
//
//   * the viscous dissipation rate eps = (1 / |Omega|) int nu grad v : grad v, with the
//     element-local (broken) gradient of the DG velocity and the GLL quadrature of its nodes:
//     one block per element computes its element's integral, a reduction adds them;
//   * the energy spectrum E(k): the velocity interpolated to a regular grid of M points per
//     direction (the point x_j = lo + j L / M evaluated by the Lagrange interpolant of the
//     element containing it), a forward DFT along every axis (radix-2, one block per grid
//     line, the line in shared memory), and E(k) = |Omega| / 2 times the summed |v^(n)|^2 of
//     the wave vectors with k - 1/2 <= |n| < k + 1/2 (v^ normalised by M^-d), binned per
//     block in shared memory and added over the blocks by one thread per shell.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace imex {
namespace {

// per element: sum over the nodes of W_q nu_q sum_{c,k} (d v_c / d x_k)^2 (eps of Sec. 4.3)
template <int D, int N>
__global__ void dissipation_kernel(Geom g, const double* __restrict__ v, long long stride, const double* __restrict__ nu,
                                   double nu0, double* __restrict__ out) {
  constexpr int ND = ipow(N, D);
  __shared__ double tile[D][ND];
  __shared__ double red[ND];
  const int e = blockIdx.x;
  const int node = threadIdx.x;
  const Tables<double>& tb = tab<double>(g);
  for (int c = 0; c < D; ++c) tile[c][node] = v[(size_t)c * stride + (size_t)e * ND + node];
  __syncthreads();
  int el = 0;
  const Geom gl = local_geom(g, e, el);
  const int id[3] = {node % N, (D > 1) ? (node / N) % N : 0, (D > 2) ? node / (N * N) : 0};
  const double* Dm = tb.D[N];
  double W = 1.0, s = 0.0;
  int stride_k = 1;
  for (int k = 0; k < D; ++k) {
    const double hk = geom_h<double>(gl, k);
    W *= 0.5 * hk * tb.w[N][id[k]];
    const int base = node - id[k] * stride_k;
    for (int c = 0; c < D; ++c) {
      double dv = 0.0;
      for (int j = 0; j < N; ++j) dv += Dm[id[k] * N + j] * tile[c][base + j * stride_k];
      dv *= 2.0 / hk;
      s += dv * dv;
    }
    stride_k *= N;
  }
  red[node] = W * (nu ? nu[(size_t)e * ND + node] : nu0) * s;
  __syncthreads();
  if (node == 0) {
    double acc = 0.0;
    for (int i = 0; i < ND; ++i) acc += red[i];
    out[e] = acc;
  }
}

// v on the regular grid (component c of point i at out[c * M^D + i], x fastest), complex
// (the grid of E(k), Sec. 4.3)
template <int D, int N>
__global__ void regular_grid_kernel(Geom g, const double* __restrict__ v, long long stride, int M,
                                    double2* __restrict__ out) {
  constexpr int ND = ipow(N, D);
  size_t npts = 1;
  for (int k = 0; k < D; ++k) npts *= (size_t)M;
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= npts) return;
  const double* xg = tab<double>(g).x[N];
  int ec[3] = {0, 0, 0};
  double L[3][N];
  size_t r = i;
  for (int k = 0; k < D; ++k) {
    const int j = (int)(r % M);
    r /= M;
    const double len = geom_h<double>(g, k) * geom_n(g, k);
    const double x = j * len / M;                      // offset from lo
    int e = (int)(x / geom_h<double>(g, k));
    if (e > geom_n(g, k) - 1) e = geom_n(g, k) - 1;
    ec[k] = e;
    const double xi = 2.0 * (x - e * geom_h<double>(g, k)) / geom_h<double>(g, k) - 1.0;
    for (int a = 0; a < N; ++a) {
      double p = 1.0;
      for (int m = 0; m < N; ++m)
        if (m != a) p *= (xi - xg[m]) / (xg[a] - xg[m]);
      L[k][a] = p;
    }
  }
  const int e = ec[0] + g.n[0] * (ec[1] + g.n[1] * ec[2]);
  for (int c = 0; c < D; ++c) {
    const double* ve = v + (size_t)c * stride + (size_t)e * ND;
    double acc = 0.0;
    for (int q = 0; q < ND; ++q) {
      const int a0 = q % N, a1 = (D > 1) ? (q / N) % N : 0, a2 = (D > 2) ? q / (N * N) : 0;
      double w = L[0][a0];
      if (D > 1) w *= L[1][a1];
      if (D > 2) w *= L[2][a2];
      acc += w * ve[q];
    }
    out[(size_t)c * npts + i] = make_double2(acc, 0.0);
  }
}

// forward DFT of every grid line along `axis` (length M, a power of two <= 1024): the line
// loaded into shared memory in bit-reversed order, log2 M butterfly stages (E(k))
__global__ void fft_lines_kernel(double2* __restrict__ a, int M, int logM, int D, int axis) {
  extern __shared__ double2 sl[];
  size_t axstride = 1;
  for (int k = 0; k < axis; ++k) axstride *= (size_t)M;
  // line index -> (component, position with the axis coordinate 0)
  size_t line = blockIdx.x;
  const size_t per_comp = (size_t)gridDim.x / D;
  const size_t comp = line / per_comp;
  size_t rem = line % per_comp;
  const size_t lo = rem % axstride;
  const size_t hi = rem / axstride;
  size_t npts = 1;
  for (int k = 0; k < D; ++k) npts *= (size_t)M;
  const size_t base = comp * npts + hi * axstride * M + lo;
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    const unsigned rv = __brev((unsigned)j) >> (32 - logM);
    sl[rv] = a[base + (size_t)j * axstride];
  }
  __syncthreads();
  for (int len = 2; len <= M; len <<= 1) {
    const int half = len >> 1;
    for (int b = threadIdx.x; b < M / 2; b += blockDim.x) {
      const int grp = b / half, pos = b % half;
      const int i0 = grp * len + pos, i1 = i0 + half;
      double s, co;
      sincospi(-2.0 * pos / len, &s, &co);          // exp(-2 pi i pos / len)
      const double2 u = sl[i0], w = sl[i1];
      const double2 t = make_double2(co * w.x - s * w.y, co * w.y + s * w.x);
      sl[i0] = make_double2(u.x + t.x, u.y + t.y);
      sl[i1] = make_double2(u.x - t.x, u.y - t.y);
    }
    __syncthreads();
  }
  for (int j = threadIdx.x; j < M; j += blockDim.x) a[base + (size_t)j * axstride] = sl[j];
}

// per block: shell sums of |a|^2 (all components), kmax shells, into part[block][kmax]
// (E(k) of Sec. 4.3)
__global__ void shell_bin_kernel(const double2* __restrict__ a, int M, int D, int kmax, double scale,
                                 double* __restrict__ part) {
  extern __shared__ double hist[];
  for (int k = threadIdx.x; k < kmax; k += blockDim.x) hist[k] = 0.0;
  __syncthreads();
  size_t npts = 1;
  for (int k = 0; k < D; ++k) npts *= (size_t)M;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < npts; i += (size_t)gridDim.x * blockDim.x) {
    size_t r = i;
    double n2 = 0.0;
    for (int k = 0; k < D; ++k) {
      const int j = (int)(r % M);
      r /= M;
      const int nk = j < M / 2 ? j : j - M;
      n2 += (double)nk * nk;
    }
    const int shell = (int)floor(sqrt(n2) + 0.5);
    if (shell >= kmax) continue;
    double p = 0.0;
    for (int c = 0; c < D; ++c) {
      const double2 z = a[(size_t)c * npts + i];
      p += z.x * z.x + z.y * z.y;
    }
    atomicAdd(&hist[shell], scale * p);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < kmax; k += blockDim.x) part[(size_t)blockIdx.x * kmax + k] = hist[k];
}

// fixed-order total of the blocks' shell sums into E(k) (Sec. 4.3)
__global__ void shell_sum_kernel(const double* __restrict__ part, int nblocks, int kmax, double* __restrict__ E) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= kmax) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * kmax + k];
  E[k] = s;
}

}  // namespace

int dissipation_elems(const Geom& g, int N, const double* v, long long stride, const double* nu, double nu0,
                      double* out, cudaStream_t st) {
#define IMEX_DIS(DD, NN)                                                                          \
  if (g.d == DD && N == NN) {                                                                     \
    IMEX_COUNTED((dissipation_kernel<DD, NN><<<g.ne, ipow(NN, DD), 0, st>>>(g, v, stride, nu, nu0, out))); \
    return 0;                                                                                     \
  }
  IMEX_DIS(2, 3) IMEX_DIS(2, 4) IMEX_DIS(2, 5) IMEX_DIS(2, 6) IMEX_DIS(2, 7) IMEX_DIS(2, 8) IMEX_DIS(2, 9)
  IMEX_DIS(3, 3) IMEX_DIS(3, 4) IMEX_DIS(3, 5) IMEX_DIS(3, 6) IMEX_DIS(3, 7) IMEX_DIS(3, 8) IMEX_DIS(3, 9)
#undef IMEX_DIS
  return -1;
}

int energy_spectrum(const Geom& g, int N, const double* v, long long stride, int M, int kmax, double vol,
                    double2* grid, double* part, int nbin_blocks, double* E, cudaStream_t st) {
  int logM = 0;
  while ((1 << logM) < M) ++logM;
  if ((1 << logM) != M || M < 2 || M > 1024) return -1;
  size_t npts = 1;
  for (int k = 0; k < g.d; ++k) npts *= (size_t)M;
  const unsigned gb = (unsigned)((npts + 255) / 256);
#define IMEX_GRID(DD, NN)                                                                              \
  if (g.d == DD && N == NN) {                                                                          \
    IMEX_COUNTED((regular_grid_kernel<DD, NN><<<gb, 256, 0, st>>>(g, v, stride, M, grid)));            \
  } else
  IMEX_GRID(2, 3) IMEX_GRID(2, 4) IMEX_GRID(2, 5) IMEX_GRID(2, 6) IMEX_GRID(2, 7) IMEX_GRID(2, 8) IMEX_GRID(2, 9)
  IMEX_GRID(3, 3) IMEX_GRID(3, 4) IMEX_GRID(3, 5) IMEX_GRID(3, 6) IMEX_GRID(3, 7) IMEX_GRID(3, 8) IMEX_GRID(3, 9)
  return -1;
#undef IMEX_GRID
  const unsigned lines = (unsigned)(g.d * (npts / M));
  const int threads = M / 2 < 256 ? (M / 2 > 32 ? M / 2 : 32) : 256;
  for (int axis = 0; axis < g.d; ++axis)
    IMEX_COUNTED((fft_lines_kernel<<<lines, threads, M * sizeof(double2), st>>>(grid, M, logM, g.d, axis)));
  const double scale = 0.5 * vol / ((double)npts * (double)npts);
  IMEX_COUNTED((shell_bin_kernel<<<nbin_blocks, 256, kmax * sizeof(double), st>>>(grid, M, g.d, kmax, scale, part)));
  IMEX_COUNTED((shell_sum_kernel<<<(kmax + 127) / 128, 128, 0, st>>>(part, nbin_blocks, kmax, E)));
  return 0;
}

}  // namespace imex
