// Divergence / mass-flux stabilisation of the projected velocity (Sec. 3.3 adds it for
// pressure robustness after the works it cites, whose form it does not state).  Reading: the
// penalised projection (M + A_D + A_C) v~ = M v'' with
//   A_D = sum_K tau_D,K B_K^T W_K B_K,  tau_D,K = zeta_D |u_K| h_K / (P + 1) dt,
//   A_C = sum_F tau_C,F J_F^T W_F J_F,  tau_C,F = zeta_C (|u_K-| + |u_K+|) / 2 dt,
// B_K the element-local divergence at the GLL nodes, W_K the GLL volume weights, J_F the
// jump of the normal velocity component across an interior face normal to k (the face's GLL
// weights W_F), |u_K| the magnitude of the element's mass-weighted mean velocity and
// h_K = (h_1 ... h_d)^(1/d).  The operator couples the d components inside an element
// (divergence) and component k across the faces normal to k (jumps); it is solved by CG.
//
// Kernels: the element mean speeds (one block per element), and the operator apply (one
// block per element, a thread per node; the element's d component tiles and the weighted
// divergence in shared memory).
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace imex {
namespace {

// element mean speeds |u_K| of the stabilisation penalties (Sec. 3.3)
template <int D, int N>
__global__ void stab_speed_kernel(Geom g, const double* __restrict__ v, long long stride, double* __restrict__ speed) {
  constexpr int ND = ipow(N, D);
  __shared__ double red[D + 1][ND];
  const int e = blockIdx.x, node = threadIdx.x;
  const Tables<double>& tb = tab<double>(g);
  const int id[3] = {node % N, (D > 1) ? (node / N) % N : 0, (D > 2) ? node / (N * N) : 0};
  double W = 1.0;
  for (int k = 0; k < D; ++k) W *= tb.w[N][id[k]];
  for (int c = 0; c < D; ++c) red[c][node] = W * v[(size_t)c * stride + (size_t)e * ND + node];
  red[D][node] = W;
  __syncthreads();
  if (node == 0) {
    double s2 = 0.0, wsum = 0.0;
    for (int i = 0; i < ND; ++i) wsum += red[D][i];
    for (int c = 0; c < D; ++c) {
      double m = 0.0;
      for (int i = 0; i < ND; ++i) m += red[c][i];
      m /= wsum;
      s2 += m * m;
    }
    speed[e] = sqrt(s2);
  }
}

// y = (M + A_D + A_C) u, the operator of the stabilised projection (Sec. 3.3)
template <int D, int N>
__global__ void stab_apply_kernel(Geom g, const double* __restrict__ u, double* __restrict__ y, long long stride,
                                  const double* __restrict__ speed, double zd, double zc, double dt, int P) {
  constexpr int ND = ipow(N, D);
  __shared__ double su[D][ND];
  __shared__ double ss[ND];
  const int e = blockIdx.x, node = threadIdx.x;
  const Tables<double>& tb = tab<double>(g);
  const double* Dm = tb.D[N];
  const double* w = tb.w[N];
  for (int c = 0; c < D; ++c) su[c][node] = u[(size_t)c * stride + (size_t)e * ND + node];
  int el = 0;
  const Geom gl = local_geom(g, e, el);
  int ec[3];
  elem_coords(gl, el, ec);
  const int id[3] = {node % N, (D > 1) ? (node / N) % N : 0, (D > 2) ? node / (N * N) : 0};
  double h[3], W = 1.0, hprod = 1.0;
  for (int k = 0; k < D; ++k) {
    h[k] = geom_h<double>(gl, k);
    W *= 0.5 * h[k] * w[id[k]];
    hprod *= h[k];
  }
  const double hK = D == 2 ? sqrt(hprod) : cbrt(hprod);
  const double tau_d = zd * speed[e] * hK / (P + 1) * dt;
  __syncthreads();
  // weighted broken divergence at this node
  double dv = 0.0;
  int sk = 1;
  for (int k = 0; k < D; ++k) {
    const int base = node - id[k] * sk;
    double a = 0.0;
    for (int j = 0; j < N; ++j) a += Dm[id[k] * N + j] * su[k][base + j * sk];
    dv += 2.0 / h[k] * a;
    sk *= N;
  }
  ss[node] = tau_d * W * dv;
  __syncthreads();
  sk = 1;
  for (int c = 0; c < D; ++c) {
    // mass + transposed derivative of the weighted divergence along c
    const int base = node - id[c] * sk;
    double a = 0.0;
    for (int j = 0; j < N; ++j) a += Dm[j * N + id[c]] * ss[base + j * sk];
    double out = W * su[c][node] + 2.0 / h[c] * a;
    // normal-velocity jumps on the two faces normal to c
    for (int side = 0; side < 2; ++side) {
      if (id[c] != (side ? N - 1 : 0)) continue;
      const int nb = neighbor(gl, ec, c, side ? 1 : -1);
      if (nb < 0) continue;
      double Wf = 1.0;
      for (int j = 0; j < D; ++j)
        if (j != c) Wf *= 0.5 * h[j] * w[id[j]];
      const double tau_c = zc * 0.5 * (speed[e] + speed[nb]) * dt;
      const int mirror = node + (side ? -(N - 1) : (N - 1)) * sk;
      out += tau_c * Wf * (su[c][node] - u[(size_t)c * stride + (size_t)nb * ND + mirror]);
    }
    y[(size_t)c * stride + (size_t)e * ND + node] = out;
    sk *= N;
  }
}

}  // namespace

#define IMEX_STAB_CASES(X)                                                                                     \
  X(2, 3) X(2, 4) X(2, 5) X(2, 6) X(2, 7) X(2, 8) X(2, 9) X(3, 3) X(3, 4) X(3, 5) X(3, 6) X(3, 7) X(3, 8) X(3, 9)

int stab_speed(const Geom& g, int N, const double* v, long long stride, double* speed, cudaStream_t st) {
#define IMEX_SP(DD, NN)                                                                                        \
  if (g.d == DD && N == NN) {                                                                                  \
    IMEX_COUNTED((stab_speed_kernel<DD, NN><<<g.ne, ipow(NN, DD), 0, st>>>(g, v, stride, speed)));             \
    return 0;                                                                                                  \
  }
  IMEX_STAB_CASES(IMEX_SP)
#undef IMEX_SP
  return -1;
}

int stab_apply(const Geom& g, int N, const double* u, double* y, long long stride, const double* speed, double zd,
               double zc, double dt, cudaStream_t st) {
#define IMEX_SA(DD, NN)                                                                                        \
  if (g.d == DD && N == NN) {                                                                                  \
    IMEX_COUNTED((stab_apply_kernel<DD, NN><<<g.ne, ipow(NN, DD), 0, st>>>(g, u, y, stride, speed, zd, zc, dt, \
                                                                           NN - 1)));                          \
    return 0;                                                                                                  \
  }
  IMEX_STAB_CASES(IMEX_SA)
#undef IMEX_SA
  return -1;
}

}  // namespace imex
