// DG-SEM first-order operators of Sec. 3.2 / 3.3 of the paper:
//   * weak divergence B into the pressure test space (Poisson right-hand side,
//     consistent pressure operator),
//   * DG gradient G = M^{-1} B^T of a pressure field (projection v'' = v' - G psi),
//   * nodal DG derivatives with central lifting (grad-div terms F_d2, F_d3),
//   * the over-integrated convection term F_c with local Lax-Friedrichs flux.
// Every kernel works on one element per thread group with its tiles in shared
// memory and sum-factorised 1D contractions.
#include <type_traits>

#include "common.cuh"
#include "ff.cuh"
#include "kernels.h"

namespace imex {

// ----------------------------------------------------------------------------
// generic 1D contraction along dimension m of a tensor with per-dimension sizes
//   out[.., a, ..] (+)= sum_x Mat[a*sa + x*sx] * in[.., x, ..]
// executed by `nt` threads starting at thread `t0` of the block
// ----------------------------------------------------------------------------
template <typename T, int D>
__device__ __forceinline__ void contract(const T* __restrict__ in, T* __restrict__ out, const int* sz,
                                         int m, int na, const T* Mat, int sa, int sx, bool acc,
                                         int t, int nt) {
  int szo[3] = {sz[0], D > 1 ? sz[1] : 1, D > 2 ? sz[2] : 1};
  szo[m] = na;
  int total = szo[0] * szo[1] * szo[2];
  int sin_m = 1;
  for (int j = 0; j < m; ++j) sin_m *= sz[j];
  for (int o = t; o < total; o += nt) {
    int c0 = o % szo[0];
    int r = o / szo[0];
    int c1 = r % szo[1];
    int c2 = r / szo[1];
    int c[3] = {c0, c1, c2};
    int a = c[m];
    c[m] = 0;
    int ib = c[0] + sz[0] * (c[1] + (D > 1 ? sz[1] : 1) * c[2]);
    T s = T(0);
    for (int x = 0; x < sz[m]; ++x) s += Mat[a * sa + x * sx] * in[ib + x * sin_m];
    out[o] = acc ? out[o] + s : s;
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
template <typename T, int D>
__device__ __forceinline__ void contract2(const T* in1, const T* in2, T s2, T* out, const int* sz,
                                          int m, int na, const T* M1, const T* M2, int t, int nt) {
  int szo[3] = {sz[0], D > 1 ? sz[1] : 1, D > 2 ? sz[2] : 1};
  szo[m] = na;
  const int total = szo[0] * szo[1] * szo[2];
  int sin_m = 1;
  for (int j = 0; j < m; ++j) sin_m *= sz[j];
  for (int o = t; o < total; o += nt) {
    int c[3] = {o % szo[0], (o / szo[0]) % szo[1], o / (szo[0] * szo[1])};
    const int am = c[m];
    c[m] = 0;
    const int ib = c[0] + sz[0] * (c[1] + (D > 1 ? sz[1] : 1) * c[2]);
    T s = T(0), r = T(0);
    for (int x = 0; x < sz[m]; ++x) {
      s += M1[x * na + am] * in1[ib + x * sin_m];
      if (in2) r += M2[x * na + am] * in2[ib + x * sin_m];
    }
    out[o] = s + s2 * r;
  }
}

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
  int sz[3] = {NV, D > 1 ? NV : 1, D > 2 ? NV : 1};
  int cur = 0;
  for (int m = 0; m < D; ++m) {
    T* src = buf + (size_t)cur * (D + 1) * ND;
    T* dst = buf + (size_t)(1 - cur) * (D + 1) * ND;
    const T hm = T(2) / geom_h<T>(gl, m);
    contract2<T, D>(src, src + (1 + m) * ND, hm, dst, sz, m, NP, sIp, sGp, threadIdx.x, blockDim.x);
    for (int k = m + 1; k < D; ++k)
      contract2<T, D>(src + (1 + k) * ND, (const T*)nullptr, T(0), dst + (1 + k) * ND, sz, m, NP, sIp,
                      sIp, threadIdx.x, blockDim.x);
    __syncthreads();
    sz[m] = NP;
    cur ^= 1;
  }
  const T* res = buf + (size_t)cur * (D + 1) * ND;
  for (int i = threadIdx.x; i < NDP; i += blockDim.x) a.b[(size_t)e * NDP + i] = (TS)(T(a.coef) * res[i]);
}

// ----------------------------------------------------------------------------
// DG gradient of a pressure field: out_k = base_k + coef * (d_k psi - lifting of [psi])
// ----------------------------------------------------------------------------
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
    int sz[3] = {NP, D > 1 ? NP : 1, D > 2 ? NP : 1};
    const T* in = sp;
    T* bufs[2] = {b1, b2};
    int cur = 0;
    for (int m = 0; m < D; ++m) {
      const T* M = (m == k) ? sGp : sIp;
      contract<T, D>(in, bufs[cur], sz, m, NV, M, NP, 1, false, threadIdx.x, blockDim.x);
      __syncthreads();
      sz[m] = NV;
      in = bufs[cur];
      cur ^= 1;
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
template <typename T, int D, int N>
__device__ __forceinline__ T nodal_deriv(const Geom& g, const int* ec, int e, const int* id, int node,
                                         int k, const T* su, const T* gfield, const T* sD, T wend) {
  constexpr int ND = ipow(N, D);
  int stride = 1;
  for (int j = 0; j < k; ++j) stride *= N;
  const int base = node - id[k] * stride;
  T acc = T(0);
#pragma unroll
  for (int j = 0; j < N; ++j) acc += sD[id[k] * N + j] * su[base + j * stride];
  const T hk = T(2) / T(g.h[k]);
  T val = hk * acc;
  for (int side = 0; side < 2; ++side) {
    if (id[k] != (side ? N - 1 : 0)) continue;
    const int nb = neighbor(g, ec, k, side ? 1 : -1);
    if (nb < 0) continue;
    int c[3] = {id[0], id[1], id[2]};
    c[k] = side ? 0 : N - 1;
    const T un = gfield[(size_t)nb * ND + flat3(c, N, D)];
    const T n = side ? T(1) : T(-1);
    val += hk / wend * T(0.5) * (un - su[node]) * n;
  }
  return val;
}

template <typename T, int D, int N>
__global__ void __launch_bounds__(ipow(N, D)) dg_deriv_kernel(Geom g, DerivArgs<T> a) {
  constexpr int ND = ipow(N, D);
  __shared__ T sD[N * N], sw[N];
  __shared__ T su[D][ND];
  const Tables<T>& tb = tab<T>(g);
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) sD[i] = tb.D[N][i];
  for (int i = threadIdx.x; i < N; i += blockDim.x) sw[i] = tb.w[N][i];
  const int e = blockIdx.x;
  int el = 0;
  const Geom gl = local_geom(g, e, el);
  const int node = threadIdx.x;
  int ec[3];
  elem_coords(gl, el, ec);
  int id[3] = {node % N, (D > 1) ? (node / N) % N : 0, (D > 2) ? node / (N * N) : 0};
  const size_t o = (size_t)e * ND + node;
  const T nu = a.nu ? a.nu[o] : (a.inst_nu ? geom_nu0<T>(gl) : a.nu0);
  // op 3 runs one output component per pass over its d input fields
  const int passes = (a.op == 3) ? D : 1;
  for (int c3 = 0; c3 < passes; ++c3) {
    const int nin = (a.op == 1) ? 1 : D;
    const int f0 = (a.op == 3) ? c3 * D : 0;
    __syncthreads();
    for (int f = 0; f < nin; ++f) su[f][node] = a.in[(size_t)(f0 + f) * a.stride + o];
    __syncthreads();
    const T wend = sw[0];
    if (a.op == 0) {
      T s = T(0);
      for (int k = 0; k < D; ++k)
        s += nodal_deriv<T, D, N>(gl, ec, e, id, node, k, su[k], a.in + (size_t)k * a.stride, sD, wend);
      a.out[o] = nu * s;
    } else if (a.op == 1) {
      for (int c = 0; c < D; ++c)
        a.out[(size_t)c * a.stride + o] =
            a.coef * nodal_deriv<T, D, N>(gl, ec, e, id, node, c, su[0], a.in, sD, wend);
    } else if (a.op == 2) {
      for (int c = 0; c < D; ++c)
        for (int k = 0; k < D; ++k)
          a.out[(size_t)(c * D + k) * a.stride + o] =
              nu * nodal_deriv<T, D, N>(gl, ec, e, id, node, c, su[k], a.in + (size_t)k * a.stride, sD, wend);
    } else {
      T s = T(0);
      for (int k = 0; k < D; ++k)
        s += nodal_deriv<T, D, N>(gl, ec, e, id, node, k, su[k], a.in + (size_t)(f0 + k) * a.stride, sD, wend);
      a.out[(size_t)c3 * a.stride + o] += a.coef * s;
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
  // shared: tables + sv[D][ND] + vg[D][NQ] + 2 work[NQ] + acc[D][ND] + face buffers
  static constexpr size_t SMEM =
      sizeof(T) * (size_t)(2 * Q * N + Q + N + D * ND + D * NQ + 2 * NQ + D * ND +
                           2 * D * NFQ + 2 * NFQ + NF);
};


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
  T* sv = sw + N;                               // [D][ND]
  T* vg = sv + D * ND;                          // [D][NQ]
  T* w1 = vg + D * NQ;                          // [NQ]
  T* w2 = w1 + NQ;                              // [NQ]
  T* acc = w2 + NQ;                             // [D][ND]
  T* fm = acc + D * ND;                         // [D][NFQ] own trace at face Gauss points
  T* fp = fm + D * NFQ;                         // [D][NFQ] neighbour trace
  T* fh = fp + D * NFQ;                         // [NFQ] flux of one component
  T* ft = fh + NFQ;                             // [NFQ] scratch
  T* fo = ft + NFQ;                             // [NF] result on the face nodes
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
  for (int c = 0; c < D; ++c) {
    int sz[3] = {N, D > 1 ? N : 1, D > 2 ? N : 1};
    const T* in = sv + c * ND;
    T* bufs[2] = {w1, w2};
    int cur = 0;
    for (int m = 0; m < D; ++m) {
      T* out = (m == D - 1) ? (vg + c * NQ) : bufs[cur];
      contract<T, D>(in, out, sz, m, Q, sIG, N, 1, false, t, nt);
      __syncthreads();
      sz[m] = Q;
      in = out;
      cur ^= 1;
    }
  }
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
      int sz[3] = {Q, D > 1 ? Q : 1, D > 2 ? Q : 1};
      const T* in = w1;
      T* bufs[2] = {w2, w1};
      int cur = 0;
      // contract dims in order; the last writes into acc (accumulating)
      for (int m = 0; m < D; ++m) {
        const T* M = (m == k) ? sDG : sIG;
        const bool last = (m == D - 1);
        T* out = last ? (acc + c * ND) : bufs[cur];
        // backward: out[j] = sum_g M[g*N + j] in[g]
        contract<T, D>(in, out, sz, m, N, M, 1, N, last, t, nt);
        __syncthreads();
        sz[m] = N;
        in = out;
        cur ^= 1;
      }
    }
  }
  __syncthreads();
  // --- face terms
  for (int k = 0; k < D; ++k) {
    for (int side = 0; side < 2; ++side) {
      const int nb = neighbor(gl, ec, k, side ? 1 : -1);
      const T n = side ? T(1) : T(-1);
      // traces on the N^{D-1} face nodes -> interpolate tangentially to Q^{D-1}
      for (int c = 0; c < D; ++c) {
        for (int f = t; f < NF; f += nt) {
          int cc[3] = {0, 0, 0};
          face_coords<D>(f, k, N, cc);
          cc[k] = side ? N - 1 : 0;
          const int own = flat3(cc, N, D);
          fo[f] = sv[c * ND + own];
          T pv;
          if (nb >= 0) {
            cc[k] = side ? 0 : N - 1;
            pv = T(a.v[(size_t)c * a.stride + (size_t)nb * ND + flat3(cc, N, D)]);
          } else {
            pv = a.vb ? T(a.vb[(size_t)c * a.stride + (size_t)e * ND + own]) : sv[c * ND + own];
          }
          ft[f] = pv;
        }
        __syncthreads();
        // tangential interpolation (D-1 dims)
        if (D == 2) {
          for (int q = t; q < Q; q += nt) {
            T s1 = T(0), s2 = T(0);
            for (int j = 0; j < N; ++j) { s1 += sIG[q * N + j] * fo[j]; s2 += sIG[q * N + j] * ft[j]; }
            fm[c * NFQ + q] = s1;
            fp[c * NFQ + q] = s2;
          }
        } else {
          // first tangential dim: (N x N) -> (Q x N), stored in fh / w1 scratch
          for (int o = t; o < Q * N; o += nt) {
            const int q0 = o % Q, j1 = o / Q;
            T s1 = T(0), s2 = T(0);
            for (int j = 0; j < N; ++j) {
              s1 += sIG[q0 * N + j] * fo[j + N * j1];
              s2 += sIG[q0 * N + j] * ft[j + N * j1];
            }
            w1[o] = s1;
            w2[o] = s2;
          }
          __syncthreads();
          for (int o = t; o < NFQ; o += nt) {
            const int q0 = o % Q, q1 = o / Q;
            T s1 = T(0), s2 = T(0);
            for (int j = 0; j < N; ++j) {
              s1 += sIG[q1 * N + j] * w1[q0 + Q * j];
              s2 += sIG[q1 * N + j] * w2[q0 + Q * j];
            }
            fm[c * NFQ + o] = s1;
            fp[c * NFQ + o] = s2;
          }
        }
        __syncthreads();
      }
      // LLF flux per component, weighted, projected back onto the face nodes
      for (int c = 0; c < D; ++c) {
        for (int q = t; q < NFQ; q += nt) {
          T W = jac / (geom_h<T>(gl, k) * T(0.5));
          int r = q;
          for (int j = 0; j < D - 1; ++j) { W *= sgw[r % Q]; r /= Q; }
          const T vmn = n * fm[k * NFQ + q];
          const T vpn = n * fp[k * NFQ + q];
          const T am = vmn < T(0) ? -vmn : vmn;
          const T ap = vpn < T(0) ? -vpn : vpn;
          const T lam = am > ap ? am : ap;
          const T H = T(0.5) * (fm[c * NFQ + q] * vmn + fp[c * NFQ + q] * vpn) +
                      T(0.5) * lam * (fm[c * NFQ + q] - fp[c * NFQ + q]);
          fh[q] = W * H;
        }
        __syncthreads();
        if (D == 2) {
          for (int f = t; f < N; f += nt) {
            T s = T(0);
            for (int q = 0; q < Q; ++q) s += sIG[q * N + f] * fh[q];
            fo[f] = s;
          }
        } else {
          for (int o = t; o < N * Q; o += nt) {      // (Q x Q) -> (N x Q)
            const int j0 = o % N, q1 = o / N;
            T s = T(0);
            for (int q = 0; q < Q; ++q) s += sIG[q * N + j0] * fh[q + Q * q1];
            ft[o] = s;
          }
          __syncthreads();
          for (int o = t; o < NF; o += nt) {          // (N x Q) -> (N x N)
            const int j0 = o % N, j1 = o / N;
            T s = T(0);
            for (int q = 0; q < Q; ++q) s += sIG[q * N + j1] * ft[j0 + N * q];
            fo[o] = s;
          }
        }
        __syncthreads();
        for (int f = t; f < NF; f += nt) {
          int cc[3] = {0, 0, 0};
          face_coords<D>(f, k, N, cc);
          cc[k] = side ? N - 1 : 0;
          acc[c * ND + flat3(cc, N, D)] -= fo[f];
        }
        __syncthreads();
      }
    }
  }
  // --- M^{-1}
  for (int c = 0; c < D; ++c)
    for (int i = t; i < ND; i += nt) {
      int r = i;
      T W = jac;
      for (int j = 0; j < D; ++j) { W *= sw[r % N]; r /= N; }
      a.out[(size_t)c * a.stride + (size_t)e * ND + i] = (TS)(T(a.coef) * acc[c * ND + i] / W);
    }
}

// ----------------------------------------------------------------------------
template <typename T, int D, int N>
static void launch_div(const Geom& g, const DivArgs<T>& a, cudaStream_t st) {
  constexpr int ND = ipow(N, D);
  const size_t smem = sizeof(T) * (size_t)(2 * N * (N - 1) + N + 2 * (D + 1) * ND);
  smem_limit_once((const void*)dg_div_kernel<T, D, N>, (int)smem);
  int threads = ND < 128 ? 128 : ((ND + 31) / 32) * 32;
  if (threads > 512) threads = 512;
  IMEX_COUNTED(dg_div_kernel<T, D, N><<<g.ne, threads, smem, st>>>(g, a));
}
template <typename T, int D, int N>
static void launch_grad(const Geom& g, const GradArgs<T>& a, cudaStream_t st) {
  constexpr int ND = ipow(N, D);
  IMEX_COUNTED(dg_grad_kernel<T, D, N><<<g.ne, ((ND + 31) / 32) * 32, 0, st>>>(g, a));
}
template <typename T, int D, int N>
static void launch_div_ff(const Geom& g, const DivArgs<double>& a, cudaStream_t st) {
  constexpr int ND = ipow(N, D);
  const size_t smem = sizeof(ff) * (size_t)(2 * N * (N - 1) + N + 2 * (D + 1) * ND);
  smem_limit_once((const void*)dg_div_kernel<ff, D, N, double>, (int)smem);
  int threads = ND < 128 ? 128 : ((ND + 31) / 32) * 32;
  if (threads > 512) threads = 512;
  IMEX_COUNTED(dg_div_kernel<ff, D, N, double><<<g.ne, threads, smem, st>>>(g, a));
}
template <typename T, int D, int N>
static void launch_grad_ff(const Geom& g, const GradArgs<double>& a, cudaStream_t st) {
  constexpr int ND = ipow(N, D);
  IMEX_COUNTED(dg_grad_kernel<ff, D, N, double><<<g.ne, ((ND + 31) / 32) * 32, 0, st>>>(g, a));
}
template <typename T, int D, int N>
static void launch_deriv(const Geom& g, const DerivArgs<T>& a, cudaStream_t st) {
  constexpr int ND = ipow(N, D);
  IMEX_COUNTED(dg_deriv_kernel<T, D, N><<<g.ne, ND, 0, st>>>(g, a));
}
template <typename T, int D, int N>
static void launch_conv(const Geom& g, const ConvArgs<T>& a, cudaStream_t st) {
  using S = ConvShape<T, D, N>;
  smem_limit_once((const void*)dg_conv_kernel<T, D, N>, (int)S::SMEM);
  IMEX_COUNTED(dg_conv_kernel<T, D, N><<<g.ne, S::THREADS, S::SMEM, st>>>(g, a));
}
template <typename T, int D, int N>
static void launch_conv_ff(const Geom& g, const ConvArgs<double>& a, cudaStream_t st) {
  using S = ConvShape<ff, D, N>;
  smem_limit_once((const void*)dg_conv_kernel<ff, D, N, double>, (int)S::SMEM);
  IMEX_COUNTED(dg_conv_kernel<ff, D, N, double><<<g.ne, S::THREADS, S::SMEM, st>>>(g, a));
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

template <typename T>
int dg_div(const Geom& g, int N, const DivArgs<T>& a, cudaStream_t st) {
  if (g.d == 2) { IMEX_DISPATCH_NV(2, launch_div, g, a, st) } else { IMEX_DISPATCH_NV(3, launch_div, g, a, st) }
  return 0;
}
template <typename T>
int dg_grad(const Geom& g, int N, const GradArgs<T>& a, cudaStream_t st) {
  if (g.d == 2) { IMEX_DISPATCH_NV(2, launch_grad, g, a, st) } else { IMEX_DISPATCH_NV(3, launch_grad, g, a, st) }
  return 0;
}
template <typename T>
int dg_deriv(const Geom& g, int N, const DerivArgs<T>& a, cudaStream_t st) {
  if (g.d == 2) { IMEX_DISPATCH_NV(2, launch_deriv, g, a, st) } else { IMEX_DISPATCH_NV(3, launch_deriv, g, a, st) }
  return 0;
}
template <typename T>
int dg_conv(const Geom& g, int N, const ConvArgs<T>& a, cudaStream_t st) {
  if (g.d == 2) { IMEX_DISPATCH_NV(2, launch_conv, g, a, st) } else { IMEX_DISPATCH_NV(3, launch_conv, g, a, st) }
  return 0;
}

// weak divergence and DG gradient with float-float arithmetic on FP64 fields
int dg_div_ff(const Geom& g, int N, const DivArgs<double>& a, cudaStream_t st) {
  using T = double;
  if (g.d == 2) { IMEX_DISPATCH_NV(2, launch_div_ff, g, a, st) } else { IMEX_DISPATCH_NV(3, launch_div_ff, g, a, st) }
  return 0;
}
int dg_grad_ff(const Geom& g, int N, const GradArgs<double>& a, cudaStream_t st) {
  using T = double;
  if (g.d == 2) { IMEX_DISPATCH_NV(2, launch_grad_ff, g, a, st) } else { IMEX_DISPATCH_NV(3, launch_grad_ff, g, a, st) }
  return 0;
}

// convection with float-float arithmetic on FP64 fields
int dg_conv_ff(const Geom& g, int N, const ConvArgs<double>& a, cudaStream_t st) {
  using T = double;
  if (g.d == 2) { IMEX_DISPATCH_NV(2, launch_conv_ff, g, a, st) } else { IMEX_DISPATCH_NV(3, launch_conv_ff, g, a, st) }
  return 0;
}

template int dg_div<double>(const Geom&, int, const DivArgs<double>&, cudaStream_t);
template int dg_grad<double>(const Geom&, int, const GradArgs<double>&, cudaStream_t);
template int dg_deriv<double>(const Geom&, int, const DerivArgs<double>&, cudaStream_t);
template int dg_conv<double>(const Geom&, int, const ConvArgs<double>&, cudaStream_t);
template int dg_conv<float>(const Geom&, int, const ConvArgs<float>&, cudaStream_t);
template int dg_div<float>(const Geom&, int, const DivArgs<float>&, cudaStream_t);
template int dg_grad<float>(const Geom&, int, const GradArgs<float>&, cudaStream_t);

}  // namespace imex
