// Matrix-free symmetric interior penalty (SIPG) operator, Sec. 3.3 of the paper
// ("interior penalty method for pressure and viscous diffusion equations"),
// applied by sum factorisation on one element per thread group.
//
//   a(u, w) = sum_K sum_q W_q nu_q grad u . grad w                        (volume, GLL quadrature)
//           - sum_F sum_f W_f ({nu du/dn} [w] + {nu dw/dn} [u])            (consistency, symmetry)
//           + sum_F sum_f W_f tau [u] [w]                                   (penalty)
//   tau = N^2 / h_perp * max(nu-, nu+) on interior faces, 2 N^2 / h * nu on Dirichlet faces,
//   N = nodes per direction.  Dirichlet data g enters through [u] = u - g (Nitsche), so
//   the kernel returns  y = alpha M x + beta (A x - r_b(g))  and optionally M^{-1} y.
//
// Per element the kernel stages the element tile and, for each of its 2d faces,
// the neighbour's trace, normal derivative and viscosity in shared memory; the
// symmetric face term is folded into the volume flux at the face nodes, so one
// transposed derivative pass per direction produces the whole result.
#include "common.cuh"
#include "kernels.h"

namespace imex {

template <typename T, int D, int N>
struct SipgShape {
  static constexpr int ND = ipow(N, D);
  static constexpr int NF = ipow(N, D - 1);
  static constexpr int EPB = (ND >= 128) ? 1 : (256 / ND);       // elements per block
  static constexpr int THREADS = EPB * ND;
};

template <typename T, int D, int N>
__global__ void __launch_bounds__(SipgShape<T, D, N>::THREADS)
sipg_apply_kernel(Geom g, SipgArgs<T> a) {
  using S = SipgShape<T, D, N>;
  constexpr int ND = S::ND, NF = S::NF, EPB = S::EPB;
  __shared__ T sD[N * N];
  __shared__ T sw[N];
  __shared__ T su[EPB][ND];
  __shared__ T snu[EPB][ND];
  __shared__ T sQ[D][EPB][ND];
  __shared__ T sfu[EPB][2 * D][NF];
  __shared__ T sfdu[EPB][2 * D][NF];
  __shared__ T sfnu[EPB][2 * D][NF];
  __shared__ int snb[EPB][2 * D];

  const Tables<T>& tb = tab<T>(g);
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) sD[i] = tb.D[N][i];
  for (int i = threadIdx.x; i < N; i += blockDim.x) sw[i] = tb.w[N][i];

  const int le = threadIdx.x / ND;
  const int node = threadIdx.x % ND;
  const int e = blockIdx.x * EPB + le;
  const bool valid = e < g.ne;
  int ec[3] = {0, 0, 0};
  if (valid) elem_coords(g, e, ec);
  int id[3];
  id[0] = node % N;
  id[1] = (D > 1) ? (node / N) % N : 0;
  id[2] = (D > 2) ? node / (N * N) : 0;

  // neighbours (-1: boundary)
  if (valid && node < 2 * D) {
    const int k = node >> 1, side = node & 1;
    snb[le][node] = neighbor(g, ec, k, side ? 1 : -1);
  }
  // viscosity of the element
  if (valid) snu[le][node] = a.nu ? a.nu[(size_t)e * ND + node] : a.nu0;
  __syncthreads();

  T hinv2[D];
  T jac = T(1);
  for (int k = 0; k < D; ++k) { hinv2[k] = T(2) / T(g.h[k]); jac *= T(g.h[k]) * T(0.5); }
  T Wq = jac;
  for (int k = 0; k < D; ++k) Wq *= sw[id[k]];

  // face viscosity of the neighbours (once for all systems)
  if (valid) {
    for (int t = node; t < 2 * D * NF; t += ND) {
      const int fi = t / NF, f = t % NF, k = fi >> 1, side = fi & 1;
      const int nb = snb[le][fi];
      int c[3];
      {  // face-node coordinates over the directions other than k
        int r = f, q = 0;
        for (int j = 0; j < D; ++j) {
          if (j == k) continue;
          c[j] = r % N; r /= N; ++q;
        }
      }
      if (nb >= 0) {
        c[k] = side ? 0 : N - 1;                       // matching face of the neighbour
        int nn = c[0] + N * ((D > 1 ? c[1] : 0) + N * (D > 2 ? c[2] : 0));
        sfnu[le][fi][f] = a.nu ? a.nu[(size_t)nb * ND + nn] : a.nu0;
      } else {
        c[k] = side ? N - 1 : 0;
        int nn = c[0] + N * ((D > 1 ? c[1] : 0) + N * (D > 2 ? c[2] : 0));
        sfnu[le][fi][f] = snu[le][nn];
      }
    }
  }

  for (int s = 0; s < a.nsys; ++s) {
    const T* x = a.x + (size_t)s * a.sys_stride;
    const T* gd = a.gdata ? a.gdata + (size_t)s * a.g_stride : nullptr;
    T* y = a.y + (size_t)s * a.sys_stride;
    __syncthreads();
    if (valid) su[le][node] = x[(size_t)e * ND + node];
    // neighbour traces and normal derivatives
    if (valid) {
      for (int t = node; t < 2 * D * NF; t += ND) {
        const int fi = t / NF, f = t % NF, k = fi >> 1, side = fi & 1;
        const int nb = snb[le][fi];
        int c[3] = {0, 0, 0};
        {
          int r = f;
          for (int j = 0; j < D; ++j) {
            if (j == k) continue;
            c[j] = r % N; r /= N;
          }
        }
        if (nb >= 0) {
          const int iface = side ? 0 : N - 1;            // neighbour's own index on the shared face
          int stride = 1;
          for (int j = 0; j < k; ++j) stride *= N;
          c[k] = 0;
          const int base = c[0] + N * ((D > 1 ? c[1] : 0) + N * (D > 2 ? c[2] : 0));
          const T* xl = x + (size_t)nb * ND + base;
          T acc = T(0), tr = T(0);
#pragma unroll
          for (int j = 0; j < N; ++j) {
            T v = xl[j * stride];
            acc += sD[iface * N + j] * v;
            if (j == iface) tr = v;
          }
          sfu[le][fi][f] = tr;
          sfdu[le][fi][f] = acc * hinv2[k];
        } else {
          c[k] = side ? N - 1 : 0;
          const int nn = c[0] + N * ((D > 1 ? c[1] : 0) + N * (D > 2 ? c[2] : 0));
          sfu[le][fi][f] = gd ? gd[(size_t)e * ND + nn] : T(0);
          sfdu[le][fi][f] = T(0);
        }
      }
    }
    __syncthreads();

    T yface = T(0);
    if (valid) {
      const T uo = su[le][node];
      const T nuq = snu[le][node];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        int stride = 1;
        for (int j = 0; j < k; ++j) stride *= N;
        const int base = node - id[k] * stride;
        T acc = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) acc += sD[id[k] * N + j] * su[le][base + j * stride];
        const T gk = acc * hinv2[k];
        T Qk = Wq * nuq * gk;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          if (id[k] != (side ? N - 1 : 0)) continue;
          const int fi = 2 * k + side;
          const int nb = snb[le][fi];
          const int bc = g.bc[k];
          if (nb < 0 && bc != 1) continue;                 // Neumann: no face terms
          T Wf = jac / (T(g.h[k]) * T(0.5));
          int f = 0, mul = 1;
          for (int j = 0; j < D; ++j) {
            if (j == k) continue;
            Wf *= sw[id[j]];
            f += id[j] * mul; mul *= N;
          }
          const T n = side ? T(1) : T(-1);
          const T un = sfu[le][fi][f];
          const T jump = uo - un;
          const T pen = T(N * N) * T(0.5) * hinv2[k];       // N^2 / h
          if (nb >= 0) {
            const T nun = sfnu[le][fi][f];
            Qk += -Wf * T(0.5) * nuq * jump * n;
            const T tau = pen * (nuq > nun ? nuq : nun);
            yface += Wf * (-T(0.5) * (nuq * n * gk + nun * n * sfdu[le][fi][f]) + tau * jump);
          } else {
            Qk += -Wf * nuq * jump * n;
            yface += Wf * (-nuq * n * gk + T(2) * pen * nuq * jump);
          }
        }
        sQ[k][le][node] = Qk;
      }
    }
    __syncthreads();
    if (valid) {
      T yv = yface;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        int stride = 1;
        for (int j = 0; j < k; ++j) stride *= N;
        const int base = node - id[k] * stride;
        T acc = T(0);
#pragma unroll
        for (int q = 0; q < N; ++q) acc += sD[q * N + id[k]] * sQ[k][le][base + q * stride];
        yv += acc * hinv2[k];
      }
      T out = a.alpha * Wq * su[le][node] + a.beta * yv;
      if (a.minv) out /= Wq;
      y[(size_t)e * ND + node] = out;
    }
  }
}

// Diagonal of alpha M + beta A (Jacobi preconditioner).
template <typename T, int D, int N>
__global__ void __launch_bounds__(SipgShape<T, D, N>::THREADS)
sipg_diag_kernel(Geom g, SipgArgs<T> a) {
  using S = SipgShape<T, D, N>;
  constexpr int ND = S::ND, NF = S::NF, EPB = S::EPB;
  __shared__ T sD[N * N];
  __shared__ T sw[N];
  __shared__ T snu[EPB][ND];
  const Tables<T>& tb = tab<T>(g);
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) sD[i] = tb.D[N][i];
  for (int i = threadIdx.x; i < N; i += blockDim.x) sw[i] = tb.w[N][i];
  const int le = threadIdx.x / ND;
  const int node = threadIdx.x % ND;
  const int e = blockIdx.x * EPB + le;
  const bool valid = e < g.ne;
  if (valid) snu[le][node] = a.nu ? a.nu[(size_t)e * ND + node] : a.nu0;
  __syncthreads();
  if (!valid) return;
  (void)NF;
  int ec[3];
  elem_coords(g, e, ec);
  int id[3];
  id[0] = node % N;
  id[1] = (D > 1) ? (node / N) % N : 0;
  id[2] = (D > 2) ? node / (N * N) : 0;
  T hinv2[D];
  T jac = T(1);
  for (int k = 0; k < D; ++k) { hinv2[k] = T(2) / T(g.h[k]); jac *= T(g.h[k]) * T(0.5); }
  T Wq = jac;
  for (int k = 0; k < D; ++k) Wq *= sw[id[k]];
  const T nuq = snu[le][node];
  T diag = T(0);
  for (int k = 0; k < D; ++k) {
    int stride = 1;
    for (int j = 0; j < k; ++j) stride *= N;
    const int base = node - id[k] * stride;
    // volume: sum over the k-line of W_q nu_q (2/h D_{q,i})^2
    T Wrest = jac;
    for (int j = 0; j < D; ++j) if (j != k) Wrest *= sw[id[j]];
    T acc = T(0);
    for (int q = 0; q < N; ++q) {
      T dq = sD[q * N + id[k]] * hinv2[k];
      acc += Wrest * sw[q] * snu[le][base + q * stride] * dq * dq;
    }
    diag += acc;
    for (int side = 0; side < 2; ++side) {
      if (id[k] != (side ? N - 1 : 0)) continue;
      const int nb = neighbor(g, ec, k, side ? 1 : -1);
      if (nb < 0 && g.bc[k] != 1) continue;
      T Wf = jac / (T(g.h[k]) * T(0.5));
      for (int j = 0; j < D; ++j) if (j != k) Wf *= sw[id[j]];
      const T n = side ? T(1) : T(-1);
      const T dself = n * sD[id[k] * N + id[k]] * hinv2[k];   // d(e_j)/dn at its own face node
      const T pen = T(N * N) * T(0.5) * hinv2[k];
      if (nb >= 0) {
        int c[3] = {id[0], id[1], id[2]};
        c[k] = side ? 0 : N - 1;
        const int nn = c[0] + N * ((D > 1 ? c[1] : 0) + N * (D > 2 ? c[2] : 0));
        const T nun = a.nu ? a.nu[(size_t)nb * ND + nn] : a.nu0;
        diag += -Wf * nuq * dself + Wf * pen * (nuq > nun ? nuq : nun);
      } else {
        diag += -T(2) * Wf * nuq * dself + Wf * T(2) * pen * nuq;
      }
    }
  }
  a.y[(size_t)e * ND + node] = a.alpha * Wq + a.beta * diag;
}

template <typename T, int D, int N>
static void launch_apply(const Geom& g, const SipgArgs<T>& a, cudaStream_t st) {
  using S = SipgShape<T, D, N>;
  int blocks = (g.ne + S::EPB - 1) / S::EPB;
  IMEX_COUNTED(sipg_apply_kernel<T, D, N><<<blocks, S::THREADS, 0, st>>>(g, a));
}

template <typename T, int D, int N>
static void launch_diag(const Geom& g, const SipgArgs<T>& a, cudaStream_t st) {
  using S = SipgShape<T, D, N>;
  int blocks = (g.ne + S::EPB - 1) / S::EPB;
  IMEX_COUNTED(sipg_diag_kernel<T, D, N><<<blocks, S::THREADS, 0, st>>>(g, a));
}

#define IMEX_DISPATCH_N(D, FN, ...)                 \
  switch (N) {                                      \
    case 2: FN<T, D, 2>(__VA_ARGS__); break;        \
    case 3: FN<T, D, 3>(__VA_ARGS__); break;        \
    case 4: FN<T, D, 4>(__VA_ARGS__); break;        \
    case 5: FN<T, D, 5>(__VA_ARGS__); break;        \
    case 6: FN<T, D, 6>(__VA_ARGS__); break;        \
    case 7: FN<T, D, 7>(__VA_ARGS__); break;        \
    case 8: FN<T, D, 8>(__VA_ARGS__); break;        \
    case 9: FN<T, D, 9>(__VA_ARGS__); break;        \
    default: return -1;                             \
  }

template <typename T>
int sipg_apply(const Geom& g, int N, const SipgArgs<T>& a, cudaStream_t st) {
  if (g.d == 2) { IMEX_DISPATCH_N(2, launch_apply, g, a, st) }
  else { IMEX_DISPATCH_N(3, launch_apply, g, a, st) }
  return 0;
}

template <typename T>
int sipg_diag(const Geom& g, int N, const SipgArgs<T>& a, cudaStream_t st) {
  if (g.d == 2) { IMEX_DISPATCH_N(2, launch_diag, g, a, st) }
  else { IMEX_DISPATCH_N(3, launch_diag, g, a, st) }
  return 0;
}

template int sipg_apply<double>(const Geom&, int, const SipgArgs<double>&, cudaStream_t);
template int sipg_apply<float>(const Geom&, int, const SipgArgs<float>&, cudaStream_t);
template int sipg_diag<double>(const Geom&, int, const SipgArgs<double>&, cudaStream_t);
template int sipg_diag<float>(const Geom&, int, const SipgArgs<float>&, cudaStream_t);

}  // namespace imex
