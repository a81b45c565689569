// DG-SEM first-order operators of Sec. 3.2 / 3.3 of the paper:
//   * weak divergence B into the pressure test space (Poisson right-hand side,
//     consistent pressure operator),
//   * DG gradient G = M^{-1} B^T of a pressure field (projection v'' = v' - G psi),
//   * nodal DG derivatives with central lifting (grad-div terms F_d2, F_d3),
//   * the over-integrated convection term F_c with local Lax-Friedrichs flux.
// Every kernel works on one element per thread group with its tiles in shared
// memory and sum-factorised 1D contractions.
//
// Kernel templates; instantiated by k_dg.cu (FP64 / FP32 arithmetic) and k_dg_ff.cu
// (float-float arithmetic on FP64 fields).
#pragma once
#include <type_traits>

#include "common.cuh"
#include "ff.cuh"
#include "kernels.h"

namespace imex {

// ----------------------------------------------------------------------------
// 1D contraction along dimension M of a tensor with extents S0 x S1 x S2
//   out[.., a, ..] (+)= sum_x Mat[a*SA + x*SX] * in[.., x, ..]    (a < NA)
// executed by `nt` threads starting at thread `t` of the block.  All extents and strides
// are compile-time constants: the index arithmetic divides by constants and the inner sum
// unrolls.
// ----------------------------------------------------------------------------
template <typename T, int S0, int S1, int S2, int M, int NA, int SA, int SX, bool ACC>
__device__ __forceinline__ void contract_ct(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ Mat,
                                            int t, int nt) {
  constexpr int O0 = (M == 0) ? NA : S0, O1 = (M == 1) ? NA : S1, O2 = (M == 2) ? NA : S2;
  constexpr int TOTAL = O0 * O1 * O2;
  constexpr int SIN = (M == 0) ? 1 : (M == 1) ? S0 : S0 * S1;       // input stride along M
  constexpr int SM = (M == 0) ? S0 : (M == 1) ? S1 : S2;            // summed extent
  for (int o = t; o < TOTAL; o += nt) {
    const int c0 = o % O0, r = o / O0, c1 = r % O1, c2 = r / O1;
    const int a = (M == 0) ? c0 : (M == 1) ? c1 : c2;
    const int ib = ((M == 0) ? 0 : c0) + S0 * (((M == 1) ? 0 : c1) + S1 * ((M == 2) ? 0 : c2));
    T s;
    if constexpr (std::is_same<T, ff>::value) {
      ff_dot acc;                                 // compensated float-float dot product
#pragma unroll
      for (int x = 0; x < SM; ++x) acc.add(Mat[a * SA + x * SX], in[ib + x * SIN]);
      s = acc.value();
    } else {
      s = T(0);
#pragma unroll
      for (int x = 0; x < SM; ++x) s += Mat[a * SA + x * SX] * in[ib + x * SIN];
    }
    out[o] = ACC ? out[o] + s : s;
  }
}

// N^D nodal values -> Q^D points, one direction per pass (w1, w2 scratch of Q^D)
template <typename T, int D, int N, int Q>
__device__ __forceinline__ void to_points(const T* in, T* out, T* w1, T* w2, const T* IG, int t, int nt) {
  if constexpr (D == 2) {
    contract_ct<T, N, N, 1, 0, Q, N, 1, false>(in, w1, IG, t, nt);
    __syncthreads();
    contract_ct<T, Q, N, 1, 1, Q, N, 1, false>(w1, out, IG, t, nt);
    __syncthreads();
  } else {
    contract_ct<T, N, N, N, 0, Q, N, 1, false>(in, w1, IG, t, nt);
    __syncthreads();
    contract_ct<T, Q, N, N, 1, Q, N, 1, false>(w1, w2, IG, t, nt);
    __syncthreads();
    contract_ct<T, Q, Q, N, 2, Q, N, 1, false>(w2, out, IG, t, nt);
    __syncthreads();
  }
}

// Q^D point values (in w1) tested against the N^D basis with the matrices M0, M1, M2 per
// direction (transposed: out[j] = sum_g M[g N + j] in[g]), added into acc
template <typename T, int D, int N, int Q>
__device__ __forceinline__ void to_nodes_add(T* acc, T* w1, T* w2, const T* M0, const T* M1, const T* M2, int t,
                                             int nt) {
  if constexpr (D == 2) {
    contract_ct<T, Q, Q, 1, 0, N, 1, N, false>(w1, w2, M0, t, nt);
    __syncthreads();
    contract_ct<T, N, Q, 1, 1, N, 1, N, true>(w2, acc, M1, t, nt);
    __syncthreads();
  } else {
    contract_ct<T, Q, Q, Q, 0, N, 1, N, false>(w1, w2, M0, t, nt);
    __syncthreads();
    contract_ct<T, N, Q, Q, 1, N, 1, N, false>(w2, w1, M1, t, nt);
    __syncthreads();
    contract_ct<T, N, N, Q, 2, N, 1, N, true>(w1, acc, M2, t, nt);
    __syncthreads();
  }
}

__device__ __forceinline__ int flat3(const int* c, int N, int D) {
  return c[0] + N * ((D > 1 ? c[1] : 0) + N * (D > 2 ? c[2] : 0));
}

// face-node index f (over the directions other than k, lowest fastest) -> coordinates
template <int D>
__device__ __forceinline__ void face_coords(int f, int k, int N, int* c) {
  for (int j = 0; j < D; ++j) {
    if (j == k) continue;
    c[j] = f % N;
    f /= N;
  }
}

// ----------------------------------------------------------------------------
// weak divergence
//   b_a = sum_k sum_x W_x v_k(x) d_k phi_a(x) - sum_faces sum_f W_f c_f phi_a(f)
//   c_f = n . {v} on interior faces, n . w on Dirichlet faces (w = data or own trace)
// on the velocity points; phi_a = pressure basis.  Sum factorisation: per direction m
//   U <- Ip^T U + (2/h_m) Gp^T V_m,  V_k <- Ip^T V_k (k > m),  U_0 = S, V_k = W v_k.
// ----------------------------------------------------------------------------
// contract2 with compile-time extents (inputs S0 x S1 x S2, direction M, output extent NA)
template <typename T, int S0, int S1, int S2, int M, int NA>
__device__ __forceinline__ void contract2_ct(const T* __restrict__ in1, const T* __restrict__ in2, T s2,
                                             T* __restrict__ out, const T* __restrict__ M1,
                                             const T* __restrict__ M2, int t, int nt) {
  constexpr int O0 = (M == 0) ? NA : S0, O1 = (M == 1) ? NA : S1, O2 = (M == 2) ? NA : S2;
  constexpr int TOTAL = O0 * O1 * O2;
  constexpr int SIN = (M == 0) ? 1 : (M == 1) ? S0 : S0 * S1;
  constexpr int SM = (M == 0) ? S0 : (M == 1) ? S1 : S2;
  for (int o = t; o < TOTAL; o += nt) {
    const int c0 = o % O0, r0 = o / O0, c1 = r0 % O1, c2 = r0 / O1;
    const int am = (M == 0) ? c0 : (M == 1) ? c1 : c2;
    const int ib = ((M == 0) ? 0 : c0) + S0 * (((M == 1) ? 0 : c1) + S1 * ((M == 2) ? 0 : c2));
    T s = T(0), r = T(0);
#pragma unroll
    for (int x = 0; x < SM; ++x) {
      s += M1[x * NA + am] * in1[ib + x * SIN];
      r += M2[x * NA + am] * in2[ib + x * SIN];
    }
    out[o] = s + s2 * r;
  }
}

// pass M of the weak divergence: U <- Ip^T U + hm Gp^T V_M, V_k <- Ip^T V_k (k > M); the
// directions before M are already on the NV - 1 pressure points
template <typename T, int D, int NV, int M>
__device__ __forceinline__ void div_pass(const T* src, T* dst, T hm, const T* sIp, const T* sGp, int t, int nt) {
  constexpr int NP = NV - 1, ND = ipow(NV, D);
  constexpr int S0 = (M > 0) ? NP : NV, S1 = (D > 1) ? ((M > 1) ? NP : NV) : 1, S2 = (D > 2) ? NV : 1;
  contract2_ct<T, S0, S1, S2, M, NP>(src, src + (1 + M) * ND, hm, dst, sIp, sGp, t, nt);
#pragma unroll
  for (int k = M + 1; k < D; ++k)
    contract_ct<T, S0, S1, S2, M, NP, 1, NP, false>(src + (1 + k) * ND, dst + (1 + k) * ND, sIp, t, nt);
}

// the weak divergence of the projection's Poisson right-hand side (Alg. 3, Sec. 3.3)
template <typename T, int D, int NV, typename TS = T>
__global__ void dg_div_kernel(Geom g, DivArgs<TS> a) {
  using TT = typename TableType<T>::type;
  constexpr int NP = NV - 1;
  constexpr int ND = ipow(NV, D);
  constexpr int NDP = ipow(NP, D);
  extern __shared__ unsigned char smem_raw[];
  T* sIp = reinterpret_cast<T*>(smem_raw);
  T* sGp = sIp + NV * NP;
  T* sw = sGp + NV * NP;
  T* buf = sw + NV;                       // [2][D+1][ND]
  const Tables<TT>& tb = tab<TT>(g);
  for (int i = threadIdx.x; i < NV * NP; i += blockDim.x) { sIp[i] = T(tb.Ipv[NV][i]); sGp[i] = T(tb.Gpv[NV][i]); }
  for (int i = threadIdx.x; i < NV; i += blockDim.x) sw[i] = T(tb.w[NV][i]);
  const int e = blockIdx.x;
  int el = 0;
  const Geom gl = local_geom(g, e, el);
  int ec[3];
  elem_coords(gl, el, ec);
  __syncthreads();
  T jac = T(1);
  for (int k = 0; k < D; ++k) jac *= geom_h<T>(gl, k) * T(0.5);
  for (int node = threadIdx.x; node < ND; node += blockDim.x) {
    int id[3] = {node % NV, (D > 1) ? (node / NV) % NV : 0, (D > 2) ? node / (NV * NV) : 0};
    T Wq = jac;
    for (int k = 0; k < D; ++k) Wq *= sw[id[k]];
    T S = T(0);
    for (int k = 0; k < D; ++k) {
      const T vk = T(a.v[(size_t)k * a.v_stride + (size_t)e * ND + node]);
      buf[(1 + k) * ND + node] = Wq * vk;
      for (int side = 0; side < 2; ++side) {
        if (id[k] != (side ? NV - 1 : 0)) continue;
        const int nb = neighbor(gl, ec, k, side ? 1 : -1);
        const T n = side ? T(1) : T(-1);
        T Wf = jac / (geom_h<T>(gl, k) * T(0.5));
        for (int j = 0; j < D; ++j) if (j != k) Wf *= sw[id[j]];
        T cflux = T(0);
        if (nb >= 0) {
          int c[3] = {id[0], id[1], id[2]};
          c[k] = side ? 0 : NV - 1;
          const T vn = T(a.v[(size_t)k * a.v_stride + (size_t)nb * ND + flat3(c, NV, D)]);
          cflux = T(0.5) * (vk + vn) * n;
        } else if (a.mode == 1) {
          cflux = T(a.wdata[(size_t)k * a.v_stride + (size_t)e * ND + node]) * n;
        } else if (a.mode == 2) {
          cflux = vk * n;
        }
        S -= Wf * cflux;
      }
    }
    buf[node] = S;
  }
  __syncthreads();
  // one pass per direction, alternating between the two halves of buf
  T* b0 = buf;
  T* b1 = buf + (size_t)(D + 1) * ND;
  div_pass<T, D, NV, 0>(b0, b1, T(2) / geom_h<T>(gl, 0), sIp, sGp, threadIdx.x, blockDim.x);
  __syncthreads();
  div_pass<T, D, NV, 1>(b1, b0, T(2) / geom_h<T>(gl, 1), sIp, sGp, threadIdx.x, blockDim.x);
  __syncthreads();
  if constexpr (D == 3) {
    div_pass<T, D, NV, 2>(b0, b1, T(2) / geom_h<T>(gl, 2), sIp, sGp, threadIdx.x, blockDim.x);
    __syncthreads();
  }
  const T* res = (D == 3) ? b1 : b0;
  for (int i = threadIdx.x; i < NDP; i += blockDim.x) a.b[(size_t)e * NDP + i] = (TS)(T(a.coef) * res[i]);
}

// ----------------------------------------------------------------------------
// DG gradient of a pressure field: out_k = base_k + coef * (d_k psi - lifting of [psi])
// ----------------------------------------------------------------------------
// the DG gradient M^{-1} B^T psi of the projection's correction (Alg. 3)
template <typename T, int D, int NV, typename TS = T>
__global__ void dg_grad_kernel(Geom g, GradArgs<TS> a) {
  using TT = typename TableType<T>::type;
  constexpr int NP = NV - 1;
  constexpr int ND = ipow(NV, D);
  constexpr int NDP = ipow(NP, D);
  constexpr int NFV = ipow(NV, D - 1);
  constexpr int NFP = ipow(NP, D - 1);
  __shared__ T sIp[NV * NP], sGp[NV * NP], sw[NV];
  __shared__ T sp[NDP];
  __shared__ T b1[ND], b2[ND];
  __shared__ T sjump[2 * D][NFV];
  __shared__ T sjp[2 * D][NFP];
  const Tables<TT>& tb = tab<TT>(g);
  for (int i = threadIdx.x; i < NV * NP; i += blockDim.x) { sIp[i] = T(tb.Ipv[NV][i]); sGp[i] = T(tb.Gpv[NV][i]); }
  for (int i = threadIdx.x; i < NV; i += blockDim.x) sw[i] = T(tb.w[NV][i]);
  const int e = blockIdx.x;
  int el = 0;
  const Geom gl = local_geom(g, e, el);
  int ec[3];
  elem_coords(gl, el, ec);
  for (int i = threadIdx.x; i < NDP; i += blockDim.x) sp[i] = T(a.psi[(size_t)e * NDP + i]);
  __syncthreads();
  // pressure jumps on the pressure face grid: own - neighbour, interior faces only
  for (int t = threadIdx.x; t < 2 * D * NFP; t += blockDim.x) {
    const int fi = t / NFP, f = t % NFP, k = fi >> 1, side = fi & 1;
    const int nb = neighbor(gl, ec, k, side ? 1 : -1);
    int c[3] = {0, 0, 0};
    face_coords<D>(f, k, NP, c);
    if (nb >= 0) {
      c[k] = side ? NP - 1 : 0;
      const T own = sp[flat3(c, NP, D)];
      c[k] = side ? 0 : NP - 1;
      const T nbv = T(a.psi[(size_t)nb * NDP + flat3(c, NP, D)]);
      sjp[fi][f] = own - nbv;
    } else {
      sjp[fi][f] = T(0);
    }
  }
  __syncthreads();
  // tangential interpolation of the jumps to the velocity face points
  for (int t = threadIdx.x; t < 2 * D * NFV; t += blockDim.x) {
    const int fi = t / NFV, f = t % NFV, k = fi >> 1;
    int cv[3] = {0, 0, 0};
    face_coords<D>(f, k, NV, cv);
    T s = T(0);
    if (D == 2) {
      const int j = (k == 0) ? 1 : 0;
      for (int p = 0; p < NP; ++p) s += sIp[cv[j] * NP + p] * sjp[fi][p];
    } else {
      int j0 = (k == 0) ? 1 : 0, j1 = (k == 2) ? 1 : 2;
      for (int q = 0; q < NP; ++q) {
        T r = T(0);
        for (int p = 0; p < NP; ++p) r += sIp[cv[j0] * NP + p] * sjp[fi][p + NP * q];
        s += sIp[cv[j1] * NP + q] * r;
      }
    }
    sjump[fi][f] = s;
  }
  __syncthreads();
  const T wend = sw[0];
  for (int k = 0; k < D; ++k) {
    // d_k psi at the velocity points: Gp' in dim k, Ip elsewhere (generic contractions)
    const T* in;
    {
      const T* M0 = (k == 0) ? sGp : sIp;
      const T* M1 = (k == 1) ? sGp : sIp;
      contract_ct<T, NP, (D > 1 ? NP : 1), (D > 2 ? NP : 1), 0, NV, NP, 1, false>(sp, b1, M0, threadIdx.x,
                                                                                 blockDim.x);
      __syncthreads();
      contract_ct<T, NV, (D > 1 ? NP : 1), (D > 2 ? NP : 1), 1, NV, NP, 1, false>(b1, b2, M1, threadIdx.x,
                                                                                 blockDim.x);
      __syncthreads();
      in = b2;
      if constexpr (D == 3) {
        const T* M2 = (k == 2) ? sGp : sIp;
        contract_ct<T, NV, NV, NP, 2, NV, NP, 1, false>(b2, b1, M2, threadIdx.x, blockDim.x);
        __syncthreads();
        in = b1;
      }
    }
    const T hk = T(2) / geom_h<T>(gl, k);
    for (int node = threadIdx.x; node < ND; node += blockDim.x) {
      int id[3] = {node % NV, (D > 1) ? (node / NV) % NV : 0, (D > 2) ? node / (NV * NV) : 0};
      T val = hk * in[node];
      for (int side = 0; side < 2; ++side) {
        if (id[k] != (side ? NV - 1 : 0)) continue;
        int f = 0, mul = 1;
        for (int j = 0; j < D; ++j) { if (j == k) continue; f += id[j] * mul; mul *= NV; }
        const T n = side ? T(1) : T(-1);
        val -= hk / wend * T(0.5) * sjump[2 * k + side][f] * n;
      }
      const size_t o = (size_t)k * a.stride + (size_t)e * ND + node;
      a.out[o] = (TS)((a.base ? T(a.base[o]) : T(0)) + T(a.coef) * val);
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------
// nodal DG derivative D_k u at node `node` of element e (central lifting inside)
// ----------------------------------------------------------------------------
template <typename T, int D, int N, typename TS>
__device__ __forceinline__ T nodal_deriv(const Geom& g, const int* ec, int e, const int* id, int node,
                                         int k, const T* su, const TS* gfield, const T* sD, T wend) {
  constexpr int ND = ipow(N, D);
  int stride = 1;
  for (int j = 0; j < k; ++j) stride *= N;
  const int base = node - id[k] * stride;
  DotAcc<T> dacc;
#pragma unroll
  for (int j = 0; j < N; ++j) dacc.add(sD[id[k] * N + j], su[base + j * stride]);
  const T acc = dacc.value();
  const T hk = T(2) / geom_h<T>(g, k);
  T val = hk * acc;
  for (int side = 0; side < 2; ++side) {
    if (id[k] != (side ? N - 1 : 0)) continue;
    const int nb = neighbor(g, ec, k, side ? 1 : -1);
    if (nb < 0) continue;
    int c[3] = {id[0], id[1], id[2]};
    c[k] = side ? 0 : N - 1;
    const T un = T(gfield[(size_t)nb * ND + flat3(c, N, D)]);
    const T n = side ? T(1) : T(-1);
    val += hk / wend * T(0.5) * (un - su[node]) * n;
  }
  return val;
}

// the nodal DG derivatives of F_d2, F_d3 (Sec. 3.2; central lifting inside, own trace on the boundary)
// T: arithmetic type (double, or the float-float ff); TS: storage type of the fields
template <typename T, int D, int N, typename TS = T>
__global__ void __launch_bounds__(ipow(N, D)) dg_deriv_kernel(Geom g, DerivArgs<TS> a) {
  using TT = typename TableType<T>::type;
  constexpr int ND = ipow(N, D);
  __shared__ T sD[N * N], sw[N];
  __shared__ T su[D][ND];
  const Tables<TT>& tb = tab<TT>(g);
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) sD[i] = T(tb.D[N][i]);
  for (int i = threadIdx.x; i < N; i += blockDim.x) sw[i] = T(tb.w[N][i]);
  const int e = blockIdx.x;
  int el = 0;
  const Geom gl = local_geom(g, e, el);
  const int node = threadIdx.x;
  int ec[3];
  elem_coords(gl, el, ec);
  int id[3] = {node % N, (D > 1) ? (node / N) % N : 0, (D > 2) ? node / (N * N) : 0};
  const size_t o = (size_t)e * ND + node;
  const T nu = a.nu ? T(a.nu[o]) : (a.inst_nu ? geom_nu0<T>(gl) : T(a.nu0));
  const T coef = T(a.coef);
  // op 3 runs one output component per pass over its d input fields
  const int passes = (a.op == 3) ? D : 1;
  for (int c3 = 0; c3 < passes; ++c3) {
    const int nin = (a.op == 1) ? 1 : D;
    const int f0 = (a.op == 3) ? c3 * D : 0;
    __syncthreads();
    for (int f = 0; f < nin; ++f) su[f][node] = T(a.in[(size_t)(f0 + f) * a.stride + o]);
    __syncthreads();
    const T wend = sw[0];
    if (a.op == 0) {
      T s = T(0);
      for (int k = 0; k < D; ++k)
        s += nodal_deriv<T, D, N>(gl, ec, e, id, node, k, su[k], a.in + (size_t)k * a.stride, sD, wend);
      a.out[o] = (TS)(nu * s);
    } else if (a.op == 1) {
      for (int c = 0; c < D; ++c)
        a.out[(size_t)c * a.stride + o] =
            (TS)(coef * nodal_deriv<T, D, N>(gl, ec, e, id, node, c, su[0], a.in, sD, wend));
    } else if (a.op == 2) {
      for (int c = 0; c < D; ++c)
        for (int k = 0; k < D; ++k)
          a.out[(size_t)(c * D + k) * a.stride + o] = (TS)(
              nu * nodal_deriv<T, D, N>(gl, ec, e, id, node, c, su[k], a.in + (size_t)k * a.stride, sD, wend));
    } else {
      T s = T(0);
      for (int k = 0; k < D; ++k)
        s += nodal_deriv<T, D, N>(gl, ec, e, id, node, k, su[k], a.in + (size_t)(f0 + k) * a.stride, sD, wend);
      const size_t oc = (size_t)c3 * a.stride + o;
      a.out[oc] = (TS)(T(a.out[oc]) + coef * s);
    }
  }
}

// ----------------------------------------------------------------------------
// convection with LLF flux, over-integrated on Q Gauss points per direction
// ----------------------------------------------------------------------------
template <typename T, int D, int N>
struct ConvShape {
  static constexpr int Q = over_q(N);
  static constexpr int ND = ipow(N, D);
  static constexpr int NQ = ipow(Q, D);
  static constexpr int NF = ipow(N, D - 1);
  static constexpr int NFQ = ipow(Q, D - 1);
  static constexpr int THREADS = (ND < 128) ? 128 : ((ND + 31) / 32) * 32;
  // face phase, all 2D faces x D components x {own, neighbour} in every pass, in two
  // alternating regions: R2 (first tangential pass, flux, result on the face nodes) from the
  // start of sv, R1 (traces, Gauss-point values, first pass back) after R2 and after sv
  // (the traces are written while sv is still read)
  static constexpr int NFC = 2 * D;
  static constexpr int R1 = NFC * D * 2 * NFQ;
  static constexpr int R2 = D == 3 ? NFC * D * 2 * Q * N : NFC * D * 2 * Q;
  static constexpr int R1_OFF = R2 > D * ND ? R2 : D * ND;
  // free after the volume term: sv, vg, w1, w2 (contiguous, the end of the layout)
  static constexpr int FREE = D * ND + D * NQ + 2 * NQ;
  static constexpr int EXTRA = R1_OFF + R1 > FREE ? R1_OFF + R1 - FREE : 0;
  // shared: tables + acc[D][ND] + sv[D][ND] + vg[D][NQ] + 2 work[NQ] + extra face scratch
  static constexpr size_t SMEM = sizeof(T) * (size_t)(2 * Q * N + Q + N + D * ND + FREE + EXTRA);
};


// the convective term F_c = -div(v v) of Sec. 3.2 as Sec. 3.3 discretises it: LLF flux with the
// pointwise max |v.n|, over-integration on ceil(3N/2) Gauss points per direction
// T: arithmetic type (double, float, or the float-float ff for FP64-class accuracy on the
// FP32 pipes); TS: storage type of the fields (double for ff)
template <typename T, int D, int N, typename TS = T>
__global__ void dg_conv_kernel(Geom g, ConvArgs<TS> a) {
  using S = ConvShape<T, D, N>;
  using TT = typename TableType<T>::type;
  constexpr int Q = S::Q, ND = S::ND, NQ = S::NQ, NF = S::NF, NFQ = S::NFQ;
  extern __shared__ unsigned char smem_raw[];
  T* sIG = reinterpret_cast<T*>(smem_raw);     // [Q*N]
  T* sDG = sIG + Q * N;                         // [Q*N]
  T* sgw = sDG + Q * N;                         // [Q]
  T* sw = sgw + Q;                              // [N]
  T* acc = sw + N;                              // [D][ND]
  T* sv = acc + D * ND;                         // [D][ND]
  T* vg = sv + D * ND;                          // [D][NQ]
  T* w1 = vg + D * NQ;                          // [NQ]
  T* w2 = w1 + NQ;                              // [NQ]
  __shared__ int snb[6];
  const Tables<TT>& tb = tab<TT>(g);
  for (int i = threadIdx.x; i < Q * N; i += blockDim.x) { sIG[i] = T(tb.IG[N][i]); sDG[i] = T(tb.DG[N][i]); }
  for (int i = threadIdx.x; i < Q; i += blockDim.x) sgw[i] = T(tb.gw[N][i]);
  for (int i = threadIdx.x; i < N; i += blockDim.x) sw[i] = T(tb.w[N][i]);
  const int e = blockIdx.x;
  int el = 0;
  const Geom gl = local_geom(g, e, el);
  int ec[3];
  elem_coords(gl, el, ec);
  for (int c = 0; c < D; ++c)
    for (int i = threadIdx.x; i < ND; i += blockDim.x) {
      sv[c * ND + i] = T(a.v[(size_t)c * a.stride + (size_t)e * ND + i]);
      acc[c * ND + i] = T(0);
    }
  __syncthreads();
  const int t = threadIdx.x, nt = blockDim.x;
  T jac = T(1);
  for (int k = 0; k < D; ++k) jac *= geom_h<T>(gl, k) * T(0.5);
  // --- interpolate v to the Gauss points
  for (int c = 0; c < D; ++c) to_points<T, D, N, Q>(sv + c * ND, vg + c * NQ, w1, w2, sIG, t, nt);
  // --- volume term: acc_c += sum_k (test derivative in k) [W_g v_c v_k]
  for (int c = 0; c < D; ++c) {
    for (int k = 0; k < D; ++k) {
      const T hk = T(2) / geom_h<T>(gl, k);                 // derivative scale of the test function
      for (int q = t; q < NQ; q += nt) {
        int r = q;
        T W = jac * hk;
        for (int j = 0; j < D; ++j) { W *= sgw[r % Q]; r /= Q; }
        w1[q] = W * vg[c * NQ + q] * vg[k * NQ + q];
      }
      __syncthreads();
      // contract the directions in order; the last pass adds into acc
      to_nodes_add<T, D, N, Q>(acc + c * ND, w1, w2, k == 0 ? sDG : sIG, k == 1 ? sDG : sIG, k == 2 ? sDG : sIG,
                               t, nt);
    }
  }
  __syncthreads();
  // --- face terms: every face, component and side in each pass
  constexpr int NFC = S::NFC;
  if (t < NFC) snb[t] = neighbor(gl, ec, t >> 1, (t & 1) ? 1 : -1);
  __syncthreads();
  T* const R2 = sv;                             // see ConvShape
  T* const R1 = sv + S::R1_OFF;
  // traces at the face nodes, R1[((f D + c) 2 + s) NF + node], s = 0 own, 1 neighbour
  // (Dirichlet data, or the own trace without data, on a domain boundary)
  for (int task = t; task < NFC * D * NF; task += nt) {
    const int f = task / (D * NF), rem = task - f * (D * NF), c = rem / NF, fn = rem - c * NF;
    const int k = f >> 1, side = f & 1;
    int cc[3] = {0, 0, 0};
    face_coords<D>(fn, k, N, cc);
    cc[k] = side ? N - 1 : 0;
    const int own = flat3(cc, N, D);
    const T ov = sv[c * ND + own];
    const int nb = snb[f];
    T pv;
    if (nb >= 0) {
      cc[k] = side ? 0 : N - 1;
      pv = T(a.v[(size_t)c * a.stride + (size_t)nb * ND + flat3(cc, N, D)]);
    } else {
      pv = a.vb ? T(a.vb[(size_t)c * a.stride + (size_t)e * ND + own]) : ov;
    }
    const int base = ((f * D + c) * 2) * NF + fn;
    R1[base] = ov;
    R1[base + NF] = pv;
  }
  __syncthreads();
  // the traces at the face Gauss points, R1[((f D + c) 2 + s) NFQ + q] (tangential
  // interpolation; in 3D the first tangential direction into R2 first)
  constexpr int NTR = NFC * D * 2;              // trace fields
  if constexpr (D == 2) {
    for (int task = t; task < NTR * Q; task += nt) {
      const int fld = task / Q, q = task - fld * Q;
      DotAcc<T> s1;
#pragma unroll
      for (int j = 0; j < N; ++j) s1.add(sIG[q * N + j], R1[fld * NF + j]);
      R2[fld * Q + q] = s1.value();
    }
    __syncthreads();
    for (int task = t; task < NTR * Q; task += nt) R1[task] = R2[task];
  } else {
    for (int task = t; task < NTR * Q * N; task += nt) {
      const int fld = task / (Q * N), o = task - fld * (Q * N), q0 = o % Q, j1 = o / Q;
      DotAcc<T> s1;
#pragma unroll
      for (int j = 0; j < N; ++j) s1.add(sIG[q0 * N + j], R1[fld * NF + j + N * j1]);
      R2[task] = s1.value();
    }
    __syncthreads();
    for (int task = t; task < NTR * NFQ; task += nt) {
      const int fld = task / NFQ, o = task - fld * NFQ, q0 = o % Q, q1 = o / Q;
      DotAcc<T> s1;
#pragma unroll
      for (int j = 0; j < N; ++j) s1.add(sIG[q1 * N + j], R2[fld * (Q * N) + q0 + Q * j]);
      R1[task] = s1.value();
    }
  }
  __syncthreads();
  // LLF flux of every face and component at the face Gauss points, weighted:
  // R2[(f D + c) NFQ + q]
  for (int task = t; task < NFC * D * NFQ; task += nt) {
    const int f = task / (D * NFQ), rem = task - f * (D * NFQ), c = rem / NFQ, q = rem - c * NFQ;
    const int k = f >> 1;
    const T n = (f & 1) ? T(1) : T(-1);
    T W = jac / (geom_h<T>(gl, k) * T(0.5));
    int r = q;
    for (int j = 0; j < D - 1; ++j) { W *= sgw[r % Q]; r /= Q; }
    const T* fk = R1 + ((f * D + k) * 2) * NFQ;           // normal component, own / neighbour
    const T* fc = R1 + ((f * D + c) * 2) * NFQ;
    const T vmn = n * fk[q];
    const T vpn = n * fk[NFQ + q];
    const T am = vmn < T(0) ? -vmn : vmn;
    const T ap = vpn < T(0) ? -vpn : vpn;
    const T lam = am > ap ? am : ap;
    const T H = T(0.5) * (fc[q] * vmn + fc[NFQ + q] * vpn) + T(0.5) * lam * (fc[q] - fc[NFQ + q]);
    R2[task] = W * H;
  }
  __syncthreads();
  // tested against the face basis: back to the face nodes, R2[(f D + c) NF + node]
  constexpr int NHF = NFC * D;                  // flux fields
  if constexpr (D == 2) {
    for (int task = t; task < NHF * N; task += nt) {
      const int fld = task / N, j0 = task - fld * N;
      DotAcc<T> s1;
#pragma unroll
      for (int q = 0; q < Q; ++q) s1.add(sIG[q * N + j0], R2[fld * Q + q]);
      R1[task] = s1.value();
    }
    __syncthreads();
    for (int task = t; task < NHF * N; task += nt) R2[task] = R1[task];
  } else {
    for (int task = t; task < NHF * N * Q; task += nt) {
      const int fld = task / (N * Q), o = task - fld * (N * Q), j0 = o % N, q1 = o / N;
      DotAcc<T> s1;
#pragma unroll
      for (int q = 0; q < Q; ++q) s1.add(sIG[q * N + j0], R2[fld * NFQ + q + Q * q1]);
      R1[task] = s1.value();
    }
    __syncthreads();
    for (int task = t; task < NHF * NF; task += nt) {
      const int fld = task / NF, o = task - fld * NF, j0 = o % N, j1 = o / N;
      DotAcc<T> s1;
#pragma unroll
      for (int q = 0; q < Q; ++q) s1.add(sIG[q * N + j1], R1[fld * (N * Q) + j0 + N * q]);
      R2[task] = s1.value();
    }
  }
  __syncthreads();
  // subtract from the nodes on the faces (a node on an edge or corner: every face it is on)
  for (int task = t; task < D * ND; task += nt) {
    const int c = task / ND, node = task - c * ND;
    const int id[3] = {node % N, D > 1 ? (node / N) % N : 0, D > 2 ? node / (N * N) : 0};
    T s1 = acc[task];
#pragma unroll
    for (int f = 0; f < NFC; ++f) {
      const int k = f >> 1;
      if (id[k] != ((f & 1) ? N - 1 : 0)) continue;
      int fn = 0, mul = 1;
      for (int j = 0; j < D; ++j) {
        if (j == k) continue;
        fn += id[j] * mul;
        mul *= N;
      }
      s1 -= R2[(f * D + c) * NF + fn];
    }
    acc[task] = s1;
  }
  __syncthreads();
  // --- M^{-1}
  for (int c = 0; c < D; ++c)
    for (int i = t; i < ND; i += nt) {
      int r = i;
      T W = jac;
      for (int j = 0; j < D; ++j) { W *= sw[r % N]; r /= N; }
      a.out[(size_t)c * a.stride + (size_t)e * ND + i] = (TS)(T(a.coef) * acc[c * ND + i] / W);
    }
}

#define IMEX_DISPATCH_NV(D, FN, ...)                \
  switch (N) {                                      \
    case 3: FN<T, D, 3>(__VA_ARGS__); break;        \
    case 4: FN<T, D, 4>(__VA_ARGS__); break;        \
    case 5: FN<T, D, 5>(__VA_ARGS__); break;        \
    case 6: FN<T, D, 6>(__VA_ARGS__); break;        \
    case 7: FN<T, D, 7>(__VA_ARGS__); break;        \
    case 8: FN<T, D, 8>(__VA_ARGS__); break;        \
    case 9: FN<T, D, 9>(__VA_ARGS__); break;        \
    default: return -1;                             \
  }

}  // namespace imex
