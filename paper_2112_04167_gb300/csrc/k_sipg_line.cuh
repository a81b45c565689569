// Line-owner SIPG kernels of the periodic constant-viscosity meshes (2D line apply, 3D
// periodic apply with its fused CG dot / Chebyshev stages, the persistent FP32 CG) and their
// launchers; instantiated per precision by k_sipg_line32.cu (FP32) and k_sipg_line64.cu
// (FP64 and float-float), each holding the constant-memory line operators of its type.
#pragma once
#include "k_sipg.cuh"

namespace imex {

// ---------------------------------------------------------------------------------
// Periodic constant-viscosity path (every face interior): the unit-size line operator of
// the element (interior on both ends), its neighbour coefficients and the derivative rows
// live in constant memory.  For element size h the line operator is
//   (1/h) [A1 u + C_tr1 trace_nb + C_dn1 (dn1 . u_nb)]
// with every unit-size quantity (A, the trace coefficients and the derivative rows scale
// as 1/h, the derivative coefficients are dimensionless), and the weights scale as h/2.
// The z-direction terms use compile-time offsets into constant memory, the x rows are read
// from the shared tile with vector loads, the y columns with scalar loads.
// ---------------------------------------------------------------------------------
// the arrays of one precision live in the translation unit that instantiates its kernels,
// which defines cline<T> for that type
template <typename T> __device__ __forceinline__ const ConstLine<T>& cline(int N);

// 2D periodic line-owner apply: two passes (y, then x), in each a thread owns one whole line
// of an element; the block's elements are contiguous in memory and are staged into shared
// memory with fully coalesced loads.  Many elements per block keep the grid within about
// one wave of resident blocks.
// elements per block of the tuned kernels: variant 0 the default, 1 half of it, 2 twice it,
// 3 (3D FP32, N = 7 and 9 only) one more element -- the N^2 lines per element of those N
// fill whole warps badly at the default (4 x 49 = 196 threads in 7 warps, 5 x 49 = 245 in 8)
__host__ __device__ constexpr int epb_variant(int base, int V) {
  return V == 1 ? (base / 2 > 0 ? base / 2 : 1) : (V == 2 ? base * 2 : (V == 3 ? base + 1 : base));
}

template <typename T, int N, int V = 0>
struct Sipg2lShape {
  static constexpr int NN = N * N;
  static constexpr int EPB = epb_variant(256 / N, V);
  static constexpr int THREADS = EPB * N;
  static constexpr int VEC = 16 / sizeof(T);
  static constexpr int NP = ((N + VEC - 1) / VEC) * VEC;
};

// The periodic constant-viscosity SIPG operator of Sec. 3.3 in 2D by line-owner passes.
// EP: the output stage, fixed at compile time for the FP32 applies (as in 3D), which then
// write the x pass's results into the accumulator tile and run the stage by columns
template <typename T, int N, int V = 0, int EP = SIPG_EP_ANY>
__global__ void __launch_bounds__(Sipg2lShape<T, N, V>::THREADS)
sipg2l_apply_kernel(Geom g, SipgArgs<T> a) {
  constexpr bool COAL = EP != SIPG_EP_ANY;
  using S = Sipg2lShape<T, N, V>;
  constexpr int NN = S::NN, EPB = S::EPB, NP = S::NP, VEC = S::VEC;
  __shared__ __align__(16) T tile[EPB][N][NP];
  __shared__ T acc[EPB][NN];
  __shared__ double red[S::THREADS];
  const ConstLine<T>& L = cline<T>(N);
  const int le = threadIdx.x / N, ta = threadIdx.x - le * N;
  const int e0 = blockIdx.x * EPB;
  const int e = e0 + le;
  const bool valid = e < g.ne;
  int el = 0;
  Geom gl = g;
  if (valid) gl = local_geom(g, e, el);
  int nb[4] = {0, 0, 0, 0};
  if (valid) {
    if (g.nbr) {                                                  // the layout's table
      const int4 q = reinterpret_cast<const int4*>(g.nbr)[e];
      nb[0] = q.x; nb[1] = q.y; nb[2] = q.z; nb[3] = q.w;
    } else {
      int ec[3];
      elem_coords(gl, el, ec);
#pragma unroll
      for (int f = 0; f < 4; ++f) nb[f] = neighbor(gl, ec, f >> 1, (f & 1) ? 1 : -1);
    }
  }
  const T hx = geom_h<T>(gl, 0), hy = geom_h<T>(gl, 1);
  const T ihx = T(1) / hx, ihy = T(1) / hy;
  const T scale = sipg_beta(a, gl) * sipg_nu0(a, gl);
  const int nvalid = min(EPB, g.ne - e0);
  // the GLL weight at the thread's line coordinate, from the global tables (the constant
  // cache would serialise the warp's distinct addresses)
  const T wta = tab<T>(g).w[N][ta];
  for (int s = 0; s < a.nsys; ++s) {
    const T* x = a.x + (size_t)s * a.sys_stride;
    T* y = a.y + (size_t)s * a.sys_stride;
    if (s > 0) __syncthreads();
    if (cg_system_stopped(a, s)) {            // its CG iteration has stopped: A p not needed
      if (a.dot_out && threadIdx.x == 0) put_dot_partial(a, s, 0.0);
      continue;
    }
    pdl_wait();
    const bool live = valid && !elem_stopped(a, g, e, s);
    // the block's elements, contiguous: coalesced loads into the row tiles
    for (int i = threadIdx.x; i < nvalid * NN; i += blockDim.x) {
      const int q = i / NN, r = i - q * NN;
      tile[q][r / N][r % N] = x[(size_t)e0 * NN + i];
    }
    __syncthreads();
    // pass y: column x = ta of element le
    if (live) {
      T v[N], vl[N], vr[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = tile[le][j][ta];
      const T* cl = x + (size_t)nb[2] * NN + ta;
      const T* cr = x + (size_t)nb[3] * NN + ta;
#pragma unroll
      for (int j = 0; j < N; ++j) { vl[j] = cl[j * N]; vr[j] = cr[j * N]; }
      T dl = T(0), dr = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) { dl += L.dnL[j] * vl[j]; dr += L.dnR[j] * vr[j]; }
      const T tl = vl[N - 1], tr = vr[0];
      const T wt = (T(0.5) * hx * wta) * ihy;
#pragma unroll
      for (int o = 0; o < N; ++o) {
        T so = L.ctrL[o] * tl + L.cdnL[o] * dl + L.ctrR[o] * tr + L.cdnR[o] * dr;
#pragma unroll
        for (int j = 0; j < N; ++j) so += L.A[o * N + j] * v[j];
        acc[le][o * N + ta] = wt * so;
      }
    }
    __syncthreads();
    // pass x: row y = ta of element le, and the result
    T dacc = T(0);
    if (live) {
      T v[NP], vl[N], vr[N];
      using VT = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
      const VT* rv = reinterpret_cast<const VT*>(&tile[le][ta][0]);
#pragma unroll
      for (int q = 0; q < NP / VEC; ++q) {
        const VT w4 = rv[q];
        const T* pw = reinterpret_cast<const T*>(&w4);
#pragma unroll
        for (int j = 0; j < VEC; ++j) v[q * VEC + j] = pw[j];
      }
      const T* rl = x + (size_t)nb[0] * NN + ta * N;
      const T* rr = x + (size_t)nb[1] * NN + ta * N;
#pragma unroll
      for (int j = 0; j < N; ++j) { vl[j] = rl[j]; vr[j] = rr[j]; }
      T dl = T(0), dr = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) { dl += L.dnL[j] * vl[j]; dr += L.dnR[j] * vr[j]; }
      const T tl = vl[N - 1], tr = vr[0];
      const T wy = T(0.5) * hy * wta;
      const T wt = wy * ihx;
#pragma unroll
      for (int o = 0; o < N; ++o) {
        T so = L.ctrL[o] * tl + L.cdnL[o] * dl + L.ctrR[o] * tr + L.cdnR[o] * dr;
#pragma unroll
        for (int j = 0; j < N; ++j) so += L.A[o * N + j] * v[j];
        const T W = wy * (T(0.5) * hx * L.w[o]);
        const T res = a.alpha * W * v[o] + scale * (acc[le][ta * N + o] + wt * so);
        if constexpr (COAL) {
          acc[le][ta * N + o] = res;            // own row: staged for the column-ordered stage
        } else {
          T out = res;
          if (a.minv) out /= W;
          sipg_out<T, T>(a, y, (size_t)e * NN + ta * N + o, v[o], out);
          dacc += v[o] * out;
        }
      }
    }
    if constexpr (COAL) {
      // the output stage by columns (x = ta): a warp's accesses are contiguous
      __syncthreads();
      if (live) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const T xin = tile[le][j][ta];
          const T out = sipg_out_ep<EP, T, T>(a, y, (size_t)e * NN + j * N + ta, xin, acc[le][j * N + ta], T(1));
          dacc += xin * out;
        }
      }
    }
    if (a.dot_out) {
      const double bs = block_sum_any_t<T>(dacc, red);
      if (threadIdx.x == 0) put_dot_partial(a, s, bs);
    }
  }
  if (a.dot_out) fused_dot_finish(a, red);
}

template <typename T, int N, int V = 0>
struct Sipg3pShape {
  static constexpr int NN = N * N;
  static constexpr int VEC = 16 / sizeof(T);                       // elements per 16-byte load
  static constexpr int NP = ((N + VEC - 1) / VEC) * VEC;           // padded row length
  static constexpr int TILE = N * N * NP;
  static constexpr int EPB = epb_variant((NN >= 49) ? 4 : (NN >= 16 ? 256 / NN : 16), V);
  static constexpr int THREADS = EPB * NN;
};

// Line-owner form of the same group apply: three passes over the element, one per direction,
// in each of which a thread owns one whole line of N nodes along that direction (z: column
// (i0, i1), y: column (i0, k), x: row (i1, k)).  It reads its line once (registers for z, the
// shared tile for y and x), loads the two neighbours' lines along the same direction from
// global memory (coalesced across the threads of a warp), and produces the N outputs of the
// 1D operator from registers; the three directional contributions meet in a shared
// accumulator.  Per node: about one shared load and two global loads per pass instead of a
// strided shared read for every term.
template <typename T, int N, int V = 0>
struct Sipg3lShape {
  static constexpr int NN = N * N;
  static constexpr int ND = N * N * N;
  static constexpr int EPB = epb_variant((NN >= 49) ? 4 : (NN >= 16 ? 256 / NN : 16), V);
  static constexpr int THREADS = EPB * NN;
  static constexpr int VEC = 16 / sizeof(T);
  static constexpr int NP = ((N + VEC - 1) / VEC) * VEC;
  static constexpr int TILE = N * N * NP;
};

// vectors of the output stage EP copied into shared memory ahead of it (Chebyshev step: r,
// D^{-1}, s; first step: b, D^{-1}), FP32 only
template <typename T, int EP>
__host__ __device__ constexpr int sipg3l_staged() {
  return sizeof(T) != 4 ? 0 : (EP == SIPG_EP_CHEB ? 3 : (EP == SIPG_EP_CHEB_FIRST ? 2 : 0));
}
template <typename T, int N, int V = 0, int EP = SIPG_EP_ANY>
constexpr size_t sipg3l_smem() {
  using S = Sipg3lShape<T, N, V>;
  return sizeof(T) * (size_t)(S::EPB * S::TILE + S::EPB * S::ND * (1 + sipg3l_staged<T, EP>()));
}

// 4-byte asynchronous copy global -> shared (no register holds the value in flight)
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// what a line's face terms need of the two neighbour lines along its direction: the
// neighbours' traces at the shared faces and their normal derivatives there (unit size)
template <typename T>
struct LineFaces {
  T tl, dl, tr, dr;
};
template <typename T, int N, typename TS>
__device__ __forceinline__ LineFaces<T> line_faces(const ConstLine<T>& L, const TS* cl, const TS* cr, int stride) {
  T vl[N], vr[N];
#pragma unroll
  for (int j = 0; j < N; ++j) { vl[j] = T(cl[j * stride]); vr[j] = T(cr[j * stride]); }
  LineFaces<T> f{vl[N - 1], T(0), vr[0], T(0)};
#pragma unroll
  for (int j = 0; j < N; ++j) { f.dl += L.dnL[j] * vl[j]; f.dr += L.dnR[j] * vr[j]; }
  return f;
}

// TX: the input's storage type (TS, or float-float pairs converted beforehand)
template <typename T, int N, typename TS = T, int V = 0, int EP = SIPG_EP_ANY, typename TX = TS>
__device__ __forceinline__ T sipg3l_group(const Geom& g, const SipgArgs<TS>& a, const TX* __restrict__ x,
                                          TS* __restrict__ y, int grp, int sys = 0) {
  using S = Sipg3lShape<T, N, V>;
  constexpr int NN = S::NN, ND = S::ND, EPB = S::EPB, NP = S::NP, TILE = S::TILE, VEC = S::VEC;
  constexpr int NSTG = sipg3l_staged<T, EP>();
  // FP32 up to N = 8: all neighbour lines are loaded before the first pass, so that their
  // latency is paid once rather than after each of the two barriers (12 scalars stay live);
  // the wider types and N = 9 load them pass by pass (register pressure)
#ifndef IMEX_SIPG3L_HOIST
#define IMEX_SIPG3L_HOIST 1
#endif
  constexpr bool HOIST = IMEX_SIPG3L_HOIST && sizeof(T) == 4 && N <= 8;
  // the fixed output stages (no M^{-1}) write through the shared accumulator tile
  constexpr bool COAL = EP != SIPG_EP_ANY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);                       // [EPB][z][y][NP]
  T* acc = tile + EPB * TILE;                                     // [EPB][z][y][x]
  T* stg = acc + EPB * ND;                                        // [NSTG][EPB][z][y][x]
  const ConstLine<T>& L = cline<T>(N);
  const int le = threadIdx.x / NN;
  const int t = threadIdx.x - le * NN;
  const int e = grp * EPB + le;
  const bool valid = e < g.ne;
  int el = 0;
  Geom gl = g;
  if (valid) gl = local_geom(g, e, el);
  int nb[6] = {0, 0, 0, 0, 0, 0};
  if (valid) {
    if (g.nbr) {                                                  // the layout's table
      const int2* p = reinterpret_cast<const int2*>(g.nbr) + (size_t)e * 3;
      const int2 a0 = p[0], a1 = p[1], a2 = p[2];
      nb[0] = a0.x; nb[1] = a0.y; nb[2] = a1.x; nb[3] = a1.y; nb[4] = a2.x; nb[5] = a2.y;
    } else {
      int ec[3];
      elem_coords(gl, el, ec);
#pragma unroll
      for (int f = 0; f < 6; ++f) nb[f] = neighbor(gl, ec, f >> 1, (f & 1) ? 1 : -1);
    }
  }
  const T hx = geom_h<T>(gl, 0), hy = geom_h<T>(gl, 1), hz = geom_h<T>(gl, 2);
  const T ihx = T(1) / hx, ihy = T(1) / hy, ihz = T(1) / hz;
  const T scale = T(sipg_beta(a, gl)) * T(sipg_nu0(a, gl));
  const T alpha = T(a.alpha);
  T* mt = tile + le * TILE;
  T* ma = acc + le * ND;
  const size_t eb = (size_t)e * ND;
  const int ta = t % N, tb = t / N;                               // the thread's two line coordinates
  // the GLL weights at the thread's two line coordinates, read once: FP32 and FP64 from the
  // global tables (an L1 hit; the constant cache would serialise the warp's distinct
  // addresses), float-float from constant memory
  T wa, wb;
  if constexpr (std::is_same<T, ff>::value) {
    wa = L.w[ta];
    wb = L.w[tb];
  } else {
    const Tables<T>& tbl = tab<T>(g);
    wa = tbl.w[N][ta];
    wb = tbl.w[N][tb];
  }
  // neighbour lines: z at (x = ta, y = tb), y at (x = ta, z = tb), x at (y = ta, z = tb)
  const TX* zl = x + (size_t)nb[4] * ND + t;
  const TX* zr = x + (size_t)nb[5] * ND + t;
  const TX* yl = x + (size_t)nb[2] * ND + tb * NN + ta;
  const TX* yr = x + (size_t)nb[3] * ND + tb * NN + ta;
  const TX* xl = x + (size_t)nb[0] * ND + tb * NN + ta * N;
  const TX* xr = x + (size_t)nb[1] * ND + tb * NN + ta * N;
  // own element into the shared tile; the z-column (ta, tb) stays in registers
  T u[N];
#pragma unroll
  for (int k = 0; k < N; ++k) u[k] = T(0);
  LineFaces<T> fz{}, fy{}, fx{};
  pdl_wait();
  const bool live = valid && !elem_stopped(a, g, e, sys);
  if (live) {
#pragma unroll
    for (int k = 0; k < N; ++k) u[k] = T(x[eb + k * NN + t]);
    if (HOIST) {
      fz = line_faces<T, N>(L, zl, zr, NN);
      fy = line_faces<T, N>(L, yl, yr, N);
      fx = line_faces<T, N>(L, xl, xr, 1);
    }
#pragma unroll
    for (int k = 0; k < N; ++k) mt[(k * N + tb) * NP + ta] = u[k];
    // the output stage's vectors at the thread's z-column, copied into shared memory while
    // the three passes run
    if constexpr (NSTG > 0) {
      const TS* src[3] = {EP == SIPG_EP_CHEB ? a.ch_r : a.ch_b, a.ch_dinv, a.ch_s};
#pragma unroll
      for (int v = 0; v < NSTG; ++v)
#pragma unroll
        for (int k = 0; k < N; ++k) cp_async4(stg + (v * EPB + le) * ND + k * NN + t, src[v] + eb + k * NN + t);
    }
  }
  // pass z: line (x = ta, y = tb) along z
  if (live) {
    if (!HOIST) fz = line_faces<T, N>(L, zl, zr, NN);
    const T wt = (T(0.5) * hx * wa) * (T(0.5) * hy * wb) * ihz;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      T sk = L.ctrL[k] * fz.tl + L.cdnL[k] * fz.dl + L.ctrR[k] * fz.tr + L.cdnR[k] * fz.dr;
#pragma unroll
      for (int j = 0; j < N; ++j) sk += L.A[k * N + j] * u[j];
      ma[k * NN + t] = wt * sk;
    }
  }
  __syncthreads();
  // pass y: line (x = ta, z = tb) along y
  if (live) {
    T v[N];
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = mt[(tb * N + j) * NP + ta];
    if (!HOIST) fy = line_faces<T, N>(L, yl, yr, N);
    const T wt = (T(0.5) * hx * wa) * (T(0.5) * hz * wb) * ihy;
#pragma unroll
    for (int o = 0; o < N; ++o) {
      T so = L.ctrL[o] * fy.tl + L.cdnL[o] * fy.dl + L.ctrR[o] * fy.tr + L.cdnR[o] * fy.dr;
#pragma unroll
      for (int j = 0; j < N; ++j) so += L.A[o * N + j] * v[j];
      ma[(tb * N + o) * N + ta] += wt * so;
    }
  }
  __syncthreads();
  // pass x: line (y = ta, z = tb) along x, and the result
  T dacc = T(0);
  if (live) {
    T v[NP];
    using VT = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    const VT* rv = reinterpret_cast<const VT*>(mt + (tb * N + ta) * NP);
#pragma unroll
    for (int q = 0; q < NP / VEC; ++q) {
      const VT w4 = rv[q];
      const T* pw = reinterpret_cast<const T*>(&w4);
#pragma unroll
      for (int j = 0; j < VEC; ++j) v[q * VEC + j] = pw[j];
    }
    if (!HOIST) fx = line_faces<T, N>(L, xl, xr, 1);
    const T wyz = (T(0.5) * hy * wa) * (T(0.5) * hz * wb);
    const T wt = wyz * ihx;
#pragma unroll
    for (int o = 0; o < N; ++o) {
      T so = L.ctrL[o] * fx.tl + L.cdnL[o] * fx.dl + L.ctrR[o] * fx.tr + L.cdnR[o] * fx.dr;
#pragma unroll
      for (int j = 0; j < N; ++j) so += L.A[o * N + j] * v[j];
      const int node = (tb * N + ta) * N + o;
      const T W = wyz * (T(0.5) * hx * L.w[o]);
      const T res = alpha * W * v[o] + scale * (ma[node] + wt * so);
      if constexpr (COAL) {
        ma[node] = res;                         // staged: the output stage runs by z-columns
      } else {
        const T out = sipg_out_ep<EP, T, TS>(a, y, eb + node, v[o], res, W);
        dacc += v[o] * out;
      }
    }
  }
  if constexpr (COAL) {
    // the fixed output stages by z-columns (x = ta, y = tb): a warp's accesses to y and to
    // the Chebyshev vectors are contiguous, where the x-lines of the pass are 4N bytes apart
    if constexpr (NSTG > 0) cp_async_wait_all();
    __syncthreads();
    if (live) {
      const T* s0 = stg + le * ND;                                // r (or b), D^{-1}, s
      const T* s1 = s0 + EPB * ND;
      const T* s2 = s1 + EPB * ND;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const int node = k * NN + t;
        const size_t i = eb + node;
        const T xin = mt[(k * N + tb) * NP + ta];
        const T out = ma[node];
        if constexpr (NSTG > 0 && EP == SIPG_EP_CHEB) {
          const T r = s0[node] - out;
          const T dn = T(a.ch_c1) * xin + T(a.ch_c2) * s1[node] * r;
          a.ch_s[i] = (TS)(s2[node] + (a.ch_addx ? xin + dn : dn));
          if (!a.ch_last) {
            a.ch_r[i] = (TS)r;
            a.ch_dout[i] = (TS)dn;
          }
        } else if constexpr (NSTG > 0 && EP == SIPG_EP_CHEB_FIRST) {
          const T r = s0[node] - out;
          a.ch_r[i] = (TS)r;
          a.ch_dout[i] = (TS)(T(a.ch_c1) * s1[node] * r);
        } else {
          sipg_out_ep<EP, T, TS>(a, y, i, xin, out, T(1));
        }
        dacc += xin * out;
      }
    }
  }
  return dacc;
}

// FP32 up to N = 8: at least IMEX_SIPG3P_MINB resident blocks per SM (a register cap; 5
// keeps the hoisted neighbour loads at 56 registers for N = 7 without spills; measured on
// the 16^3, N = 7 pressure apply: 21.0 us against 22.0 us for the unhoisted form)
#ifndef IMEX_SIPG3P_MINB
#define IMEX_SIPG3P_MINB 5
#endif
// resident blocks asked of the compiler: IMEX_SIPG3P_MINB for the FP32 default and halved
// shapes; none for the doubled blocks (a forced count would make them spill)
// float-float: two resident blocks (128 registers; uncapped, the unrolled neighbour-line
// conversions take 255 registers and spill)
__host__ __device__ constexpr int sipg3p_minb(int V, bool f32, bool isff) {
  return V == 2 ? 1 : (f32 ? IMEX_SIPG3P_MINB : (isff ? 2 : 1));
}
// The periodic constant-viscosity SIPG operator of Sec. 3.3 in 3D by line-owner passes (the
// CG and V-cycle applies; the Chebyshev step fused in the output stage).
// XFF: the input is a.xff, float-float pairs converted from a.x beforehand (float-float
// applies: no FP64 conversions in the kernel)
template <typename T, int N, typename TS = T, int V = 0, int EP = SIPG_EP_ANY, bool XFF = false>
__global__ void __launch_bounds__(Sipg3pShape<T, N, V>::THREADS,
                                  sipg3p_minb(V, sizeof(T) == 4 && N <= 8, std::is_same<T, ff>::value))
sipg3p_apply_kernel(Geom g, SipgArgs<TS> a) {
  __shared__ double red[Sipg3pShape<T, N, V>::THREADS];
  pdl_trigger();
  for (int s = 0; s < a.nsys; ++s) {
    if (s > 0) __syncthreads();
    if (cg_system_stopped(a, s)) {            // its CG iteration has stopped: A p not needed
      if (a.dot_out && threadIdx.x == 0) put_dot_partial(a, s, 0.0);
      continue;
    }
    T dacc;
    if constexpr (XFF)
      dacc = sipg3l_group<T, N, TS, V, EP, ff>(g, a, reinterpret_cast<const ff*>(a.xff) + (size_t)s * a.sys_stride,
                                               a.y + (size_t)s * a.sys_stride, blockIdx.x, s);
    else
      dacc = sipg3l_group<T, N, TS, V, EP>(g, a, a.x + (size_t)s * a.sys_stride, a.y + (size_t)s * a.sys_stride,
                                           blockIdx.x, s);
    if (a.dot_out) {
      const double bs = block_sum_any_t<T>(dacc, red);
      if (threadIdx.x == 0) put_dot_partial(a, s, bs);
    }
  }
  if (a.dot_out) fused_dot_finish(a, red);
}

// ---------------------------------------------------------------------------------
// Persistent projected CG (FP32 inner iterations of the mixed form) for the periodic
// constant-coefficient pressure operator of one instance: one cooperative launch runs
// iterations -- apply A p with (p, A p), step, direction -- separated by grid barriers, until
// the recursive residual meets the tolerance, falls below the replacement threshold, the
// iteration limit is reached or the step breaks down.  Every block adds the per-block
// partial sums in the same order, so all blocks hold identical scalars without a
// broadcast.  The vectors (p, A p, r, y, D^{-1}) are L2-resident at the sizes this serves.
// ---------------------------------------------------------------------------------
struct PcgPersist {
  float* y;
  float* r;
  float* p;
  float* Ap;
  const float* dinv;
  long long n;
  double stop_rr;          // leave for a residual replacement once (r', r') < stop_rr
  double* partial;         // [5][gridDim.x]
  unsigned int* bar;       // [2]: arrival counter, generation (zero at launch)
  int* err;                // set when a barrier wait gives up
};

// grid-wide barrier of a cooperative launch; bounded wait (gives up with *err = 1)
__device__ __forceinline__ void grid_barrier(unsigned int* bar, unsigned int& gen, int* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int g = gen;
    if (atomicAdd(&bar[0], 1u) == gridDim.x - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicExch(&bar[1], g + 1u);
    } else {
      volatile unsigned int* vg = bar + 1;
      long long spins = 0;
      while (*vg == g) {
        __nanosleep(32);
        if (++spins > (1LL << 25)) {
          atomicExch(err, 1);
          break;
        }
      }
    }
    __threadfence();
  }
  gen++;
  __syncthreads();
}

// K sums over the block (any block size) into out[] (valid in every thread): per-thread
// values summed in FP32 by warp 0, the K results converted once
template <int K>
__device__ __forceinline__ void persist_block_sum(const float (&v)[K], double (&out)[K], double* red) {
  float* rf = reinterpret_cast<float*>(red);
  __shared__ double res[8];
  __syncthreads();
  for (int k = 0; k < K; ++k) rf[k * blockDim.x + threadIdx.x] = v[k];
  __syncthreads();
  if (threadIdx.x < 32) {
    for (int k = 0; k < K; ++k) {
      float s = 0.f;
      for (int i = threadIdx.x; i < (int)blockDim.x; i += 32) s += rf[k * blockDim.x + i];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (threadIdx.x == 0) res[k] = (double)s;
    }
  }
  __syncthreads();
  for (int k = 0; k < K; ++k) out[k] = res[k];
}

// totals over the blocks of K partial arrays (fixed order; identical in every block): the
// threads' strided shares through shared memory, added by warp 0
template <int K>
__device__ __forceinline__ void persist_totals(const double* partial, int q0, double (&out)[K], double* red) {
  __syncthreads();
  for (int k = 0; k < K; ++k) {
    double v = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) v += partial[(size_t)(q0 + k) * gridDim.x + b];
    red[k * blockDim.x + threadIdx.x] = v;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int i = threadIdx.x; i < (int)blockDim.x; i += 32) s += red[k * blockDim.x + i];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (threadIdx.x == 0) red[K * blockDim.x + k] = s;
    }
  }
  __syncthreads();
  for (int k = 0; k < K; ++k) out[k] = red[K * blockDim.x + k];
}

// the whole FP32 Jacobi-preconditioned pressure CG of Alg. 3's projection in one cooperative
// launch (opt-in; the projected iteration of the singular system)
template <int N>
__global__ void __launch_bounds__(Sipg3pShape<float, N>::THREADS, (N <= 8) ? 5 : 1)
pcg_persist_kernel(Geom g, SipgArgs<float> a, PcgPersist q, CgScalars sc, int maxit) {
  using S = Sipg3pShape<float, N>;
  __shared__ double red[5 * S::THREADS];
  constexpr int NN = N * N, ND = N * N * N;
  const int ngroups = (g.ne + S::EPB - 1) / S::EPB;
  const long long n = q.n;
  const int le = threadIdx.x / NN, tcol = threadIdx.x - le * NN;    // element of the group, column
  unsigned int gen = 0;
  double rz = sc.rz[0];
  const double dsum = sc.dsum[0], thr = sc.tol2 * sc.bb[0];
  const double nd = (double)n;
  int iters = sc.iters[0];
  int done = sc.done[0];
  double rr = sc.rr[0], zmean = sc.zmean[0], rmean = sc.rmean[0], beta = 0.0, rz_old = sc.rz_old[0];
  while (done == 0) {
    // A p and (p, A p)
    float dacc = 0.f;
    for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
      __syncthreads();
      dacc += sipg3l_group<float, N>(g, a, q.p, q.Ap, grp);
    }
    {
      const float v[1] = {dacc};
      double o[1];
      persist_block_sum<1>(v, o, red);
      if (threadIdx.x == 0) q.partial[blockIdx.x] = o[0];
    }
    grid_barrier(q.bar, gen, q.err);
    if (*((volatile int*)q.err)) break;
    double pap[1];
    persist_totals<1>(q.partial, 0, pap, red);
    const double alpha = pap[0] != 0.0 ? rz / pap[0] : 0.0;
    if (!isfinite(alpha)) {
      done = 2;
      break;
    }
    // y += alpha p, r -= alpha A p on this block's element groups (the apply's node mapping:
    // each thread a column of N nodes, all loads issued before the arithmetic); sums of the
    // new residual
    float s4[4] = {0.f, 0.f, 0.f, 0.f};
    const float af = (float)alpha;
    for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
      const int e = grp * S::EPB + le;
      if (e >= g.ne) continue;
      const size_t b0 = (size_t)e * ND + tcol;
      float rv[N], av[N], dv[N], yv[N], pv[N];
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const size_t i = b0 + (size_t)k * NN;
        rv[k] = q.r[i]; av[k] = q.Ap[i]; dv[k] = q.dinv[i]; yv[k] = q.y[i]; pv[k] = q.p[i];
      }
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const size_t i = b0 + (size_t)k * NN;
        const float ri = rv[k] - af * av[k];
        const float zi = ri * dv[k];
        q.y[i] = yv[k] + af * pv[k];
        q.r[i] = ri;
        s4[0] += ri * zi;
        s4[1] += ri * ri;
        s4[2] += zi;
        s4[3] += ri;
      }
    }
    {
      double o[4];
      persist_block_sum<4>(s4, o, red);
      if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) q.partial[(size_t)(1 + k) * gridDim.x + blockIdx.x] = o[k];
    }
    grid_barrier(q.bar, gen, q.err);
    if (*((volatile int*)q.err)) break;
    double tot[4];
    persist_totals<4>(q.partial, 1, tot, red);
    const double rho = tot[3] / nd;
    const double rzn = tot[0] - 2.0 * rho * tot[2] + rho * rho * dsum;
    rr = fmax(tot[1] - nd * rho * rho, 0.0);
    zmean = (tot[2] - rho * dsum) / nd;
    rmean = rho;
    beta = rz != 0.0 ? rzn / rz : 0.0;
    rz_old = rz;
    rz = rzn;
    iters++;
    if (rr != rr || !isfinite(beta)) done = 2;
    else if (rr <= thr) done = 1;
    else if (iters >= maxit) done = 3;
    if (done != 0) break;
    // next direction: p = D^{-1} (r - rho) - zmean + beta p, r -= rho
    const float bf = (float)beta, zm = (float)zmean, rm = (float)rmean;
    for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
      const int e = grp * S::EPB + le;
      if (e >= g.ne) continue;
      const size_t b0 = (size_t)e * ND + tcol;
      float rv[N], dv[N], pv[N];
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const size_t i = b0 + (size_t)k * NN;
        rv[k] = q.r[i]; dv[k] = q.dinv[i]; pv[k] = q.p[i];
      }
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const size_t i = b0 + (size_t)k * NN;
        const float ri = rv[k] - rm;
        q.r[i] = ri;
        q.p[i] = (ri * dv[k] - zm) + bf * pv[k];
      }
    }
    if (rr < q.stop_rr) break;                        // residual replacement is due (p is current)
    grid_barrier(q.bar, gen, q.err);
    if (*((volatile int*)q.err)) break;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc.rz[0] = rz;
    sc.rz_old[0] = rz_old;
    sc.rr[0] = rr;
    sc.zmean[0] = zmean;
    sc.rmean[0] = rmean;
    sc.zmean_f[0] = (float)zmean;
    sc.rmean_f[0] = (float)rmean;
    sc.beta[0] = beta;
    sc.beta_f[0] = (float)beta;
    sc.iters[0] = iters;
    sc.done[0] = *((volatile int*)q.err) ? 2 : done;
  }
}

template <int N>
static int launch_persist(const Geom& g, const SipgArgs<float>& a, const PcgPersist& q, const CgScalars& sc,
                          int maxit, int* grid_out, cudaStream_t st) {
  using S = Sipg3pShape<float, N>;
  constexpr size_t sm = sipg3l_smem<float, N>();
  smem_limit_once((const void*)pcg_persist_kernel<N>, (int)sm);
  int dev = 0, nsm = 0, per = 0, coop = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pcg_persist_kernel<N>, S::THREADS, sm) != cudaSuccess ||
      per < 1)
    return -1;
  const int ngroups = (g.ne + S::EPB - 1) / S::EPB;
  const int grid = std::min(std::min(per * nsm, ngroups), 4096);
  if (grid_out) *grid_out = grid;
  Geom gg = g;
  SipgArgs<float> aa = a;
  PcgPersist qq = q;
  CgScalars ss = sc;
  void* args[] = {&gg, &aa, &qq, &ss, &maxit};
  IMEX_COUNTED(cudaLaunchCooperativeKernel((const void*)pcg_persist_kernel<N>, dim3(grid), dim3(S::THREADS), args,
                                           sm, st));
  return 0;
}

template <typename T, int N, int V, int EP>
static void launch_apply2l_ep(const Geom& g, const SipgArgs<T>& a, cudaStream_t st) {
  using C = Sipg2lShape<T, N, V>;
  IMEX_COUNTED((sipg2l_apply_kernel<T, N, V, EP><<<(g.ne + C::EPB - 1) / C::EPB, C::THREADS, 0, st>>>(g, a)));
}
// FP32: the output stage fixed at compile time unless M^{-1} is asked for
template <typename T, int N, int V>
static void launch_apply2l(const Geom& g, const SipgArgs<T>& a, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (!a.minv) {
      if (a.cheb == 2) launch_apply2l_ep<T, N, V, SIPG_EP_CHEB_FIRST>(g, a, st);
      else if (a.cheb) launch_apply2l_ep<T, N, V, SIPG_EP_CHEB>(g, a, st);
      else launch_apply2l_ep<T, N, V, SIPG_EP_PLAIN>(g, a, st);
    } else {
      launch_apply2l_ep<T, N, 0, SIPG_EP_ANY>(g, a, st);
    }
  } else {
    launch_apply2l_ep<T, N, V, SIPG_EP_ANY>(g, a, st);
  }
}

template <typename T, int N, int V, int EP>
static void launch_apply3p_ep(const Geom& g, const SipgArgs<T>& a, cudaStream_t st) {
  using P = Sipg3pShape<T, N, V>;
  constexpr size_t sm = sipg3l_smem<T, N, V, EP>();
  smem_limit_once((const void*)sipg3p_apply_kernel<T, N, T, V, EP>, (int)sm);
  launch_cg_kernel(sipg3p_apply_kernel<T, N, T, V, EP>, (g.ne + P::EPB - 1) / P::EPB, P::THREADS, sm, st, g, a);
}
// FP32 (the CG and V-cycle applies): the output stage fixed at compile time unless M^{-1}
// is asked for
template <typename T, int N, int V>
static void launch_apply3p(const Geom& g, const SipgArgs<T>& a, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (!a.minv) {
      if (a.cheb == 2) launch_apply3p_ep<T, N, V, SIPG_EP_CHEB_FIRST>(g, a, st);
      else if (a.cheb) launch_apply3p_ep<T, N, V, SIPG_EP_CHEB>(g, a, st);
      else launch_apply3p_ep<T, N, V, SIPG_EP_PLAIN>(g, a, st);
    } else {
      launch_apply3p_ep<T, N, 0, SIPG_EP_ANY>(g, a, st);    // M^{-1} A x: the default shape
    }
  } else {
    launch_apply3p_ep<T, N, V, SIPG_EP_ANY>(g, a, st);
  }
}

// the line-owner dispatch for one precision: the tuned launch shape of the 2D line and the
// 3D periodic applies (twice the elements per block in 2D: FP32 only, for the static shared
// memory; one element more: 3D FP32 at N = 7, 9)
template <typename T, int N>
static void launch_line(const Geom& g, const SipgArgs<T>& a, cudaStream_t st) {
  if (g.d == 2) {
    if (a.variant == 1) launch_apply2l<T, N, 1>(g, a, st);
    else if constexpr (sizeof(T) == 4) {
      if (a.variant == 2) launch_apply2l<T, N, 2>(g, a, st);
      else launch_apply2l<T, N, 0>(g, a, st);
    } else {
      launch_apply2l<T, N, 0>(g, a, st);
    }
    return;
  }
  if (a.variant == 1) launch_apply3p<T, N, 1>(g, a, st);
  else if (a.variant == 2) launch_apply3p<T, N, 2>(g, a, st);
  else if constexpr (sizeof(T) == 4 && (N == 7 || N == 9)) {
    if (a.variant == 3) launch_apply3p<T, N, 3>(g, a, st);
    else launch_apply3p<T, N, 0>(g, a, st);
  } else {
    launch_apply3p<T, N, 0>(g, a, st);
  }
}

template <typename T>
static int sipg_apply_line_t(const Geom& g, int N, const SipgArgs<T>& a, cudaStream_t st) {
  if (a.nu || !a.ops || g.bc[0] != 0 || g.bc[1] != 0 || (g.d == 3 && g.bc[2] != 0)) return -1;
  switch (N) {
    case 2: launch_line<T, 2>(g, a, st); return 0;
    case 3: launch_line<T, 3>(g, a, st); return 0;
    case 4: launch_line<T, 4>(g, a, st); return 0;
    case 5: launch_line<T, 5>(g, a, st); return 0;
    case 6: launch_line<T, 6>(g, a, st); return 0;
    case 7: launch_line<T, 7>(g, a, st); return 0;
    case 8: launch_line<T, 8>(g, a, st); return 0;
    case 9: launch_line<T, 9>(g, a, st); return 0;
    default: return -1;
  }
}

}  // namespace imex
