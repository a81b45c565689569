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
#include <type_traits>

#include "common.cuh"
#include "ff.cuh"
#include "kernels.h"
#include "vec.h"

namespace imex {

// Output of one node of an apply: y = A x, or the fused Chebyshev step of the p-multigrid
// smoother (a.cheb): r -= A x, d' = c1 x + c2 D^{-1} r, s += d' (xin: this node's input x)
template <typename T, typename TS>
__device__ __forceinline__ void sipg_cheb_out(const SipgArgs<TS>& a, size_t i, T xin, T out) {
  const T r = T(a.ch_r[i]) - out;
  const T dn = T(a.ch_c1) * xin + T(a.ch_c2) * T(a.ch_dinv[i]) * r;
  a.ch_s[i] = (TS)(T(a.ch_s[i]) + dn);
  if (!a.ch_last) {
    a.ch_r[i] = (TS)r;
    a.ch_dout[i] = (TS)dn;
  }
}
template <typename T, typename TS>
__device__ __forceinline__ void sipg_out(const SipgArgs<TS>& a, TS* __restrict__ y, size_t i, T xin, T out) {
  if (!a.cheb) {
    y[i] = (TS)out;
    return;
  }
  sipg_cheb_out<T, TS>(a, i, xin, out);
}
// Output stage chosen at compile time: EP = 0 reads the flags (M^{-1}, Chebyshev) at run
// time, 1 writes y = A x, 2 performs the Chebyshev step.  Fixed stages keep the unused
// branches -- a precise division, the Chebyshev loads and stores -- out of the unrolled
// output loop, where the compiler would otherwise predicate them into every node.
constexpr int SIPG_EP_ANY = 0, SIPG_EP_PLAIN = 1, SIPG_EP_CHEB = 2;
template <int EP, typename T, typename TS>
__device__ __forceinline__ T sipg_out_ep(const SipgArgs<TS>& a, TS* __restrict__ y, size_t i, T xin, T out, T W) {
  if constexpr (EP == SIPG_EP_PLAIN) {
    y[i] = (TS)out;
  } else if constexpr (EP == SIPG_EP_CHEB) {
    sipg_cheb_out<T, TS>(a, i, xin, out);
  } else {
    if (a.minv) out = out / W;
    sipg_out<T, TS>(a, y, i, xin, out);
  }
  return out;
}


// Deterministic block sum for any block size: thread values through shared memory, then
// warp 0 adds them in a fixed order.  Result valid in thread 0.
__device__ __forceinline__ double block_sum_any(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    for (int i = threadIdx.x; i < (int)blockDim.x; i += 32) s += red[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  __syncthreads();
  return s;
}

// The same for a value of the vector type T: the per-thread values are staged in T and
// only warp 0 converts (FP32 kernels keep FP64 arithmetic out of the per-thread path).
template <typename T>
__device__ __forceinline__ double block_sum_any_t(T v, double* red_storage) {
  T* red = reinterpret_cast<T*>(red_storage);
  red[threadIdx.x] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    T ls = T(0);
    for (int i = threadIdx.x; i < (int)blockDim.x; i += 32) ls += red[i];
    s = (double)ls;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  __syncthreads();
  return s;
}

// A block's partial of the fused CG dot; the deferred form stores it in the vector type (the
// block sums are formed in that type), which the step kernel then adds
template <typename T>
__device__ __forceinline__ void put_dot_partial(const SipgArgs<T>& a, int s, double bs) {
  const size_t i = (size_t)s * gridDim.x + blockIdx.x;
  if (a.dot_defer) reinterpret_cast<T*>(a.dot_partial)[i] = (T)bs;
  else a.dot_partial[i] = bs;
}

// In a CG loop (the fused form) the apply skips a system whose iteration has stopped
// (converged, broken down or out of iterations: its flag is set by an earlier kernel), so
// that the tail of a graph-replayed chunk of iterations costs no operator work
template <typename T>
__device__ __forceinline__ bool cg_system_stopped(const SipgArgs<T>& a, int s) {
  if (!a.cg_done) return false;
  pdl_wait();
  return a.cg_done[s] != 0;
}

// In a batch group's CG loop the apply skips the elements whose system has stopped (call
// after pdl_wait: the flags are written by earlier kernels)
template <typename T>
__device__ __forceinline__ bool elem_stopped(const SipgArgs<T>& a, const Geom& g, int e, int s) {
  if (!a.done_flags || !g.elem_inst) return false;
  return a.done_flags[s * a.done_ninst + g.elem_inst[e]] != 0;
}

// Fused CG dot: each block has left its partial per system in a.dot_partial; the last block
// to finish adds the partials in block order and writes a.dot_out and the step length, then
// resets the counter.  The deferred form only records the number of blocks (in *dot_nblk)
// for the step kernel, which adds the partials itself.
template <typename T>
__device__ void fused_dot_finish(const SipgArgs<T>& a, double* red) {
  if (a.dot_defer) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.dot_nblk = gridDim.x;
    return;
  }
  __shared__ int am_last;
  if (threadIdx.x == 0) {
    __threadfence();                       // this block's partials (written by thread 0) are visible
    am_last = (atomicAdd(a.dot_counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  for (int s = 0; s < a.nsys; ++s) {
    double v = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) v += a.dot_partial[(size_t)s * gridDim.x + b];
    v = block_sum_any(v, red);
    if (threadIdx.x == 0) {
      a.dot_out[s] = v;
      if (a.cg_rz) {
        const double al = v != 0.0 ? a.cg_rz[s] / v : 0.0;
        const bool ok = isfinite(al);
        a.cg_alpha[s] = ok ? al : 0.0;
        a.cg_alpha_f[s] = ok ? (float)al : 0.f;
        if (!ok && a.cg_done[s] == 0) a.cg_done[s] = 2;
      }
    }
  }
  if (threadIdx.x == 0) *a.dot_counter = 0u;
}

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
  int el = 0;
  Geom gl = g;
  if (valid) gl = local_geom(g, e, el);
  int ec[3] = {0, 0, 0};
  if (valid) elem_coords(gl, el, ec);
  int id[3];
  id[0] = node % N;
  id[1] = (D > 1) ? (node / N) % N : 0;
  id[2] = (D > 2) ? node / (N * N) : 0;

  // neighbours (-1: boundary)
  if (valid && node < 2 * D) {
    const int k = node >> 1, side = node & 1;
    snb[le][node] = neighbor(gl, ec, k, side ? 1 : -1);
  }
  // viscosity of the element
  if (valid) snu[le][node] = a.nu ? a.nu[(size_t)e * ND + node] : sipg_nu0(a, gl);
  __syncthreads();

  T hinv2[D];
  T jac = T(1);
  for (int k = 0; k < D; ++k) { hinv2[k] = T(2) / geom_h<T>(gl, k); jac *= geom_h<T>(gl, k) * T(0.5); }
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
        sfnu[le][fi][f] = a.nu ? a.nu[(size_t)nb * ND + nn] : sipg_nu0(a, gl);
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
          const int bc = geom_bc(g, k);
          if (nb < 0 && bc != 1) continue;                 // Neumann: no face terms
          T Wf = jac / (geom_h<T>(gl, k) * T(0.5));
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
      T out = a.alpha * Wq * su[le][node] + sipg_beta(a, gl) * yv;
      if (a.minv) out /= Wq;
      y[(size_t)e * ND + node] = out;
    }
  }
}

// ---------------------------------------------------------------------------------
// 3D form: N^2 threads per element, each owning one z-column (i0, i1) of the element
// tile in registers.  x / y derivatives read the tile from shared memory, z
// derivatives stay in registers; the neighbours' traces and normal derivatives on
// the four lateral faces are staged cooperatively (one face node per thread and
// face), those of the two z-faces per thread in registers.
// ---------------------------------------------------------------------------------
template <int N>
struct Sipg3Shape {
  static constexpr int NN = N * N;
  static constexpr int ND = N * N * N;
  static constexpr int EPB = (NN >= 49) ? 4 : (NN >= 16 ? 256 / NN : 16);
  static constexpr int THREADS = EPB * NN;
};

// face contribution at one node: the symmetric term enters the flux Qk, the
// consistency and penalty terms the nodal value yface.  kind: 0 none, 1 interior, 2 Dirichlet
template <typename T>
__device__ __forceinline__ void sipg_face(int kind, T Wf, T n, T uo, T gk, T nuq, T un, T dn, T nun, T pen, T& Qk,
                                          T& yface) {
  if (kind == 1) {
    const T jump = uo - un;
    Qk += -Wf * T(0.5) * nuq * jump * n;
    const T tau = pen * (nuq > nun ? nuq : nun);
    yface += Wf * (-T(0.5) * n * (nuq * gk + nun * dn) + tau * jump);
  } else if (kind == 2) {
    const T jump = uo - un;
    Qk += -Wf * nuq * jump * n;
    yface += Wf * (-nuq * n * gk + T(2) * pen * nuq * jump);
  }
}

template <typename T, int N>
constexpr size_t sipg3_smem() {
  using S = Sipg3Shape<N>;
  return sizeof(T) * (size_t)(N * N + N + 3 * S::EPB * S::ND + 3 * S::EPB * 4 * S::NN);
}

template <typename T, int N, bool VARNU>
__global__ void __launch_bounds__(Sipg3Shape<N>::THREADS)
sipg3_apply_kernel(Geom g, SipgArgs<T> a) {
  using S = Sipg3Shape<N>;
  constexpr int NN = S::NN, ND = S::ND, EPB = S::EPB;
  extern __shared__ unsigned char smem_raw[];
  T* sD = reinterpret_cast<T*>(smem_raw);
  T* sw = sD + N * N;
  T (*su)[ND] = reinterpret_cast<T (*)[ND]>(sw + N);
  T (*sQx)[ND] = su + EPB;
  T (*sQy)[ND] = sQx + EPB;
  T (*sfu)[4][NN] = reinterpret_cast<T (*)[4][NN]>(sQy + EPB);
  T (*sfd)[4][NN] = sfu + EPB;
  T (*sfn)[4][NN] = sfd + EPB;
  __shared__ int snb[EPB][6];

  const Tables<T>& tb = tab<T>(g);
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) sD[i] = tb.D[N][i];
  for (int i = threadIdx.x; i < N; i += blockDim.x) sw[i] = tb.w[N][i];
  const int le = threadIdx.x / NN;
  const int t = threadIdx.x - le * NN;
  const int i0 = t % N, i1 = t / N;
  const int e = blockIdx.x * EPB + le;
  const bool valid = e < g.ne;
  int el = 0;
  Geom gl = g;
  if (valid) gl = local_geom(g, e, el);
  int ec[3] = {0, 0, 0};
  if (valid) elem_coords(gl, el, ec);
  // six neighbours per element: with N = 2 an element has only four threads
  if (valid)
    for (int f = t; f < 6; f += NN) snb[le][f] = neighbor(gl, ec, f >> 1, (f & 1) ? 1 : -1);
  __syncthreads();

  const T hx = T(2) / geom_h<T>(gl, 0), hy = T(2) / geom_h<T>(gl, 1), hz = T(2) / geom_h<T>(gl, 2);
  const T jac = geom_h<T>(gl, 0) * geom_h<T>(gl, 1) * geom_h<T>(gl, 2) * T(0.125);
  const T jfx = geom_h<T>(gl, 1) * geom_h<T>(gl, 2) * T(0.25), jfy = geom_h<T>(gl, 0) * geom_h<T>(gl, 2) * T(0.25),
          jfz = geom_h<T>(gl, 0) * geom_h<T>(gl, 1) * T(0.25);
  const T penx = T(N * N) * T(0.5) * hx, peny = T(N * N) * T(0.5) * hy, penz = T(N * N) * T(0.5) * hz;
  const size_t ebase = (size_t)e * ND;

  // own viscosity column (constant viscosity: one register)
  T nuc[VARNU ? N : 1];
#pragma unroll
  for (int k = 0; k < (VARNU ? N : 1); ++k) nuc[k] = (VARNU && valid) ? a.nu[ebase + k * NN + t] : sipg_nu0(a, gl);
  // face kinds: 0 none (Neumann), 1 interior, 2 Dirichlet
  int kind[6];
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const int nb = valid ? snb[le][f] : -1;
    kind[f] = nb >= 0 ? 1 : (g.bc[f >> 1] == 1 ? 2 : 0);
  }

  for (int s = 0; s < a.nsys; ++s) {
    const T* x = a.x + (size_t)s * a.sys_stride;
    const T* gd = a.gdata ? a.gdata + (size_t)s * a.g_stride : nullptr;
    T* y = a.y + (size_t)s * a.sys_stride;
    T u[N];
    if (s > 0) __syncthreads();
    if (valid) {
#pragma unroll
      for (int k = 0; k < N; ++k) {
        u[k] = x[ebase + k * NN + t];
        su[le][k * NN + t] = u[k];
      }
      // lateral faces: face node t = (c0, c1) with c1 = t / N the z index
      const int c0 = t % N, kk = t / N;
#pragma unroll
      for (int fi = 0; fi < 4; ++fi) {
        const int dir = fi >> 1, side = fi & 1;
        const int nb = snb[le][fi];
        T tr = T(0), dv = T(0), nn = sipg_nu0(a, gl);
        if (nb >= 0) {
          const int iface = side ? 0 : N - 1;                    // neighbour's index on the shared face
          const size_t nbase = (size_t)nb * ND + kk * NN;
          T acc = T(0);
          if (dir == 0) {
            const T* row = x + nbase + c0 * N;                  // neighbour row along x at (y = c0, z = kk)
#pragma unroll
            for (int j = 0; j < N; ++j) { const T v = row[j]; acc += sD[iface * N + j] * v; if (j == iface) tr = v; }
            dv = acc * hx;
            if (VARNU) nn = a.nu[nbase + c0 * N + iface];
          } else {
            const T* col = x + nbase + c0;                      // neighbour column along y at (x = c0, z = kk)
#pragma unroll
            for (int j = 0; j < N; ++j) { const T v = col[j * N]; acc += sD[iface * N + j] * v; if (j == iface) tr = v; }
            dv = acc * hy;
            if (VARNU) nn = a.nu[nbase + iface * N + c0];
          }
        } else if (geom_bc(g, dir) == 1) {
          const int own = side ? N - 1 : 0;
          const size_t on = ebase + kk * NN + (dir == 0 ? c0 * N + own : own * N + c0);
          tr = gd ? gd[on] : T(0);
          if (VARNU) nn = a.nu[on];
        }
        sfu[le][fi][t] = tr;
        sfd[le][fi][t] = dv;
        sfn[le][fi][t] = nn;
      }
    }
    // z-faces: the neighbour columns through this thread's (i0, i1)
    T zu[2] = {T(0), T(0)}, zd[2] = {T(0), T(0)}, zn[2] = {sipg_nu0(a, gl), sipg_nu0(a, gl)};
    if (valid) {
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const int nb = snb[le][4 + side];
        if (nb >= 0) {
          const int iface = side ? 0 : N - 1;
          const T* col = x + (size_t)nb * ND + t;
          T acc = T(0);
#pragma unroll
          for (int j = 0; j < N; ++j) { const T v = col[j * NN]; acc += sD[iface * N + j] * v; if (j == iface) zu[side] = v; }
          zd[side] = acc * hz;
          if (VARNU) zn[side] = a.nu[(size_t)nb * ND + iface * NN + t];
        } else if (g.bc[2] == 1) {
          const int own = side ? N - 1 : 0;
          zu[side] = gd ? gd[ebase + own * NN + t] : T(0);
          zn[side] = nuc[VARNU ? own : 0];
        }
      }
    }
    __syncthreads();
    T Qz[N], yf[N];
    if (valid) {
      const T wxy = sw[i0] * sw[i1];
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const T* plane = &su[le][k * NN];
        T gx = T(0), gy = T(0), gz = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
          gx += sD[i0 * N + j] * plane[i1 * N + j];
          gy += sD[i1 * N + j] * plane[j * N + i0];
          gz += sD[k * N + j] * u[j];
        }
        gx *= hx; gy *= hy; gz *= hz;
        const T nuq = nuc[VARNU ? k : 0];
        const T W = jac * wxy * sw[k];
        T Qx = W * nuq * gx, Qy = W * nuq * gy, Qzk = W * nuq * gz;
        T yface = T(0);
        const int fxy0 = i1 + N * k, fxy1 = i0 + N * k;
        if (i0 == 0) sipg_face<T>(kind[0], jfx * sw[i1] * sw[k], T(-1), u[k], gx, nuq, sfu[le][0][fxy0],
                                  sfd[le][0][fxy0], sfn[le][0][fxy0], penx, Qx, yface);
        if (i0 == N - 1) sipg_face<T>(kind[1], jfx * sw[i1] * sw[k], T(1), u[k], gx, nuq, sfu[le][1][fxy0],
                                      sfd[le][1][fxy0], sfn[le][1][fxy0], penx, Qx, yface);
        if (i1 == 0) sipg_face<T>(kind[2], jfy * sw[i0] * sw[k], T(-1), u[k], gy, nuq, sfu[le][2][fxy1],
                                  sfd[le][2][fxy1], sfn[le][2][fxy1], peny, Qy, yface);
        if (i1 == N - 1) sipg_face<T>(kind[3], jfy * sw[i0] * sw[k], T(1), u[k], gy, nuq, sfu[le][3][fxy1],
                                      sfd[le][3][fxy1], sfn[le][3][fxy1], peny, Qy, yface);
        if (k == 0) sipg_face<T>(kind[4], jfz * wxy, T(-1), u[k], gz, nuq, zu[0], zd[0], zn[0], penz, Qzk, yface);
        if (k == N - 1) sipg_face<T>(kind[5], jfz * wxy, T(1), u[k], gz, nuq, zu[1], zd[1], zn[1], penz, Qzk, yface);
        sQx[le][k * NN + t] = Qx;
        sQy[le][k * NN + t] = Qy;
        Qz[k] = Qzk;
        yf[k] = yface;
      }
    }
    __syncthreads();
    if (valid) {
      const T wxy = sw[i0] * sw[i1];
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const T* px = &sQx[le][k * NN];
        const T* py = &sQy[le][k * NN];
        T ax = T(0), ay = T(0), az = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
          ax += sD[j * N + i0] * px[i1 * N + j];
          ay += sD[j * N + i1] * py[j * N + i0];
          az += sD[j * N + k] * Qz[j];
        }
        const T W = jac * wxy * sw[k];
        const T yv = yf[k] + hx * ax + hy * ay + hz * az;
        T out = a.alpha * W * u[k] + sipg_beta(a, gl) * yv;
        if (a.minv) out /= W;
        y[ebase + k * NN + t] = out;
      }
    }
  }
}

// ---------------------------------------------------------------------------------
// Constant-viscosity fast path.  With constant nu the operator is
//   y = alpha M u + beta nu0 sum_k W_perp,k (A_k u_line + sum_sides C_k (trace, dn)_nb)
// with the precomputed line operators of LineOps: per node one N-term row of A_k per
// direction plus two or four neighbour terms, a single synchronisation per element.
// 3D: N^2 threads per element, each owning a z-column in registers.
// ---------------------------------------------------------------------------------
template <int N>
struct Sipg3cShape {
  static constexpr int NN = N * N;
  static constexpr int ND = N * N * N;
  static constexpr int EPB = (NN >= 49) ? 4 : (NN >= 16 ? 256 / NN : 16);
  static constexpr int THREADS = EPB * NN;
};

template <typename T, int N>
constexpr size_t sipg3c_smem() {
  using S = Sipg3cShape<N>;
  // A[3][9][N*N] + C[3][2][3][2][N] + dn[3][2][N] + Wt[3][N] + tile + 4 lateral faces x (trace, dn)
  return sizeof(T) * (size_t)(27 * N * N + 36 * N + 6 * N + 3 * N + S::EPB * S::ND + S::EPB * 8 * S::NN);
}

template <typename T, int N>
__global__ void __launch_bounds__(Sipg3cShape<N>::THREADS)
sipg3c_apply_kernel(Geom g, SipgArgs<T> a) {
  using S = Sipg3cShape<N>;
  constexpr int NN = S::NN, ND = S::ND, EPB = S::EPB;
  extern __shared__ unsigned char smem_raw[];
  T* sA = reinterpret_cast<T*>(smem_raw);        // [3][9][NN]
  T* sC = sA + 27 * NN;                          // [3][2][3][2][N]
  T* sdn = sC + 36 * N;                          // [3][2][N]
  T* sWt = sdn + 6 * N;                          // [3][N]
  T (*su)[ND] = reinterpret_cast<T (*)[ND]>(sWt + 3 * N);
  T (*sf)[8][NN] = reinterpret_cast<T (*)[8][NN]>(su + EPB);   // [face 0..3][trace | dn]
  __shared__ int snb[EPB][6];
  const LineOps<T>& op = *a.ops;
  for (int i = threadIdx.x; i < 27 * NN; i += blockDim.x) {
    const int kv = i / NN, r = i % NN;
    sA[i] = op.A[kv / 9][kv % 9][r];
  }
  for (int i = threadIdx.x; i < 36 * N; i += blockDim.x) {
    const int q = i / N, r = i % N;   // q = ((k*2 + side)*3 + kind)*2 + which
    sC[i] = op.C[q / 12][(q / 6) % 2][(q / 2) % 3][q % 2][r];
  }
  for (int i = threadIdx.x; i < 6 * N; i += blockDim.x) sdn[i] = op.dn[i / (2 * N)][(i / N) % 2][i % N];
  for (int i = threadIdx.x; i < 3 * N; i += blockDim.x) sWt[i] = op.Wt[i / N][i % N];
  const int le = threadIdx.x / NN;
  const int t = threadIdx.x - le * NN;
  const int i0 = t % N, i1 = t / N;
  const int e = blockIdx.x * EPB + le;
  const bool valid = e < g.ne;
  int el = 0;
  Geom gl = g;
  if (valid) gl = local_geom(g, e, el);
  int ec[3] = {0, 0, 0};
  if (valid) elem_coords(gl, el, ec);
  // six neighbours per element: with N = 2 an element has only four threads
  if (valid)
    for (int f = t; f < 6; f += NN) snb[le][f] = neighbor(gl, ec, f >> 1, (f & 1) ? 1 : -1);
  __syncthreads();
  int kind[6];
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const int nb = valid ? snb[le][f] : -1;
    kind[f] = nb >= 0 ? 1 : (g.bc[f >> 1] == 1 ? 2 : 0);
  }
  const size_t ebase = (size_t)e * ND;
  const T scale = sipg_beta(a, gl) * sipg_nu0(a, gl);
  __shared__ double red[S::THREADS];
  for (int s = 0; s < a.nsys; ++s) {
    const T* x = a.x + (size_t)s * a.sys_stride;
    const T* gd = a.gdata ? a.gdata + (size_t)s * a.g_stride : nullptr;
    T* y = a.y + (size_t)s * a.sys_stride;
    if (s > 0) __syncthreads();
    if (cg_system_stopped(a, s)) {            // its CG iteration has stopped: A p not needed
      if (a.dot_out && threadIdx.x == 0) put_dot_partial(a, s, 0.0);
      continue;
    }
    T u[N];
    T dacc = T(0);
    T zt[2] = {T(0), T(0)}, zd[2] = {T(0), T(0)};
    if (valid) {
#pragma unroll
      for (int k = 0; k < N; ++k) {
        u[k] = x[ebase + k * NN + t];
        su[le][k * NN + t] = u[k];
      }
      // lateral faces: face node t = (c0, kk), kk the z index
      const int c0 = t % N, kk = t / N;
#pragma unroll
      for (int fi = 0; fi < 4; ++fi) {
        const int dir = fi >> 1, side = fi & 1;
        const int nb = snb[le][fi];
        T tr = T(0), dv = T(0);
        if (nb >= 0) {
          const int iface = side ? 0 : N - 1;
          const T* dr = sdn + (dir * 2 + side) * N;
          const size_t nbase = (size_t)nb * ND + kk * NN;
          if (dir == 0) {
            const T* row = x + nbase + c0 * N;
#pragma unroll
            for (int j = 0; j < N; ++j) { const T v = row[j]; dv += dr[j] * v; if (j == iface) tr = v; }
          } else {
            const T* col = x + nbase + c0;
#pragma unroll
            for (int j = 0; j < N; ++j) { const T v = col[j * N]; dv += dr[j] * v; if (j == iface) tr = v; }
          }
        } else if (kind[fi] == 2 && gd) {
          const int own = side ? N - 1 : 0;
          tr = gd[ebase + kk * NN + (dir == 0 ? c0 * N + own : own * N + c0)];
        }
        sf[le][2 * fi][t] = tr;
        sf[le][2 * fi + 1][t] = dv;
      }
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const int nb = snb[le][4 + side];
        if (nb >= 0) {
          const int iface = side ? 0 : N - 1;
          const T* dr = sdn + (2 * 2 + side) * N;
          const T* col = x + (size_t)nb * ND + t;
#pragma unroll
          for (int j = 0; j < N; ++j) { const T v = col[j * NN]; zd[side] += dr[j] * v; if (j == iface) zt[side] = v; }
        } else if (kind[4 + side] == 2 && gd) {
          zt[side] = gd[ebase + (side ? N - 1 : 0) * NN + t];
        }
      }
    }
    __syncthreads();
    if (valid) {
      const T* Ax = sA + (0 * 9 + 3 * kind[0] + kind[1]) * NN + i0 * N;
      const T* Ay = sA + (1 * 9 + 3 * kind[2] + kind[3]) * NN + i1 * N;
      const T* Az = sA + (2 * 9 + 3 * kind[4] + kind[5]) * NN;
      // neighbour coefficients of this thread's rows: C[k][side][kind][which][i]
      const T cxl0 = sC[((0 * 2 + 0) * 3 + kind[0]) * 2 * N + i0], cxl1 = sC[(((0 * 2 + 0) * 3 + kind[0]) * 2 + 1) * N + i0];
      const T cxr0 = sC[((0 * 2 + 1) * 3 + kind[1]) * 2 * N + i0], cxr1 = sC[(((0 * 2 + 1) * 3 + kind[1]) * 2 + 1) * N + i0];
      const T cyl0 = sC[((1 * 2 + 0) * 3 + kind[2]) * 2 * N + i1], cyl1 = sC[(((1 * 2 + 0) * 3 + kind[2]) * 2 + 1) * N + i1];
      const T cyr0 = sC[((1 * 2 + 1) * 3 + kind[3]) * 2 * N + i1], cyr1 = sC[(((1 * 2 + 1) * 3 + kind[3]) * 2 + 1) * N + i1];
      const T* czl = sC + ((2 * 2 + 0) * 3 + kind[4]) * 2 * N;
      const T* czr = sC + ((2 * 2 + 1) * 3 + kind[5]) * 2 * N;
      // unit-size line operators: direction k scales as 1 / h_k, its weights as h_k
      const T hx = geom_h<T>(gl, 0), hy = geom_h<T>(gl, 1), hz = geom_h<T>(gl, 2);
      const T ihx = T(1) / hx, ihy = T(1) / hy, ihz = T(1) / hz;
      const T wx = hx * sWt[i0], wy = hy * sWt[N + i1];
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const T* plane = &su[le][k * NN];
        T yx = T(0), yy = T(0), yz = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
          yx += Ax[j] * plane[i1 * N + j];
          yy += Ay[j] * plane[j * N + i0];
          yz += Az[k * N + j] * u[j];
        }
        const int fx = i1 + N * k, fy = i0 + N * k;
        yx += cxl0 * sf[le][0][fx] + cxl1 * sf[le][1][fx] + cxr0 * sf[le][2][fx] + cxr1 * sf[le][3][fx];
        yy += cyl0 * sf[le][4][fy] + cyl1 * sf[le][5][fy] + cyr0 * sf[le][6][fy] + cyr1 * sf[le][7][fy];
        yz += czl[k] * zt[0] + czl[N + k] * zd[0] + czr[k] * zt[1] + czr[N + k] * zd[1];
        const T wz = hz * sWt[2 * N + k];
        const T W = wx * wy * wz;
        const T yv = wy * wz * ihx * yx + wx * wz * ihy * yy + wx * wy * ihz * yz;
        T out = a.alpha * W * u[k] + scale * yv;
        if (a.minv) out /= W;
        sipg_out<T, T>(a, y, ebase + k * NN + t, u[k], out);
        dacc += u[k] * out;
      }
    }
    if (a.dot_out) {
      const double bs = block_sum_any_t<T>(dacc, red);
      if (threadIdx.x == 0) put_dot_partial(a, s, bs);
    }
  }
  if (a.dot_out) fused_dot_finish(a, red);
}

// 2D: one thread per node, EPB elements per block.
template <int N>
struct Sipg2cShape {
  static constexpr int NN = N * N;
  static constexpr int EPB = (256 / NN) > 0 ? 256 / NN : 1;
  static constexpr int THREADS = EPB * NN;
};

template <typename T, int N>
constexpr size_t sipg2c_smem() {
  using S = Sipg2cShape<N>;
  return sizeof(T) * (size_t)(18 * N * N + 24 * N + 4 * N + 2 * N + S::EPB * S::NN + S::EPB * 8 * N);
}

template <typename T, int N>
__global__ void __launch_bounds__(Sipg2cShape<N>::THREADS)
sipg2c_apply_kernel(Geom g, SipgArgs<T> a) {
  using S = Sipg2cShape<N>;
  constexpr int NN = S::NN, EPB = S::EPB;
  extern __shared__ unsigned char smem_raw[];
  T* sA = reinterpret_cast<T*>(smem_raw);        // [2][9][NN]
  T* sC = sA + 18 * NN;                          // [2][2][3][2][N]
  T* sdn = sC + 24 * N;                          // [2][2][N]
  T* sWt = sdn + 4 * N;                          // [2][N]
  T (*su)[NN] = reinterpret_cast<T (*)[NN]>(sWt + 2 * N);
  T (*sf)[8][N] = reinterpret_cast<T (*)[8][N]>(su + EPB);
  __shared__ int snb[EPB][4];
  const LineOps<T>& op = *a.ops;
  for (int i = threadIdx.x; i < 18 * NN; i += blockDim.x) {
    const int kv = i / NN, r = i % NN;
    sA[i] = op.A[kv / 9][kv % 9][r];
  }
  for (int i = threadIdx.x; i < 24 * N; i += blockDim.x) {
    const int q = i / N, r = i % N;
    sC[i] = op.C[q / 12][(q / 6) % 2][(q / 2) % 3][q % 2][r];
  }
  for (int i = threadIdx.x; i < 4 * N; i += blockDim.x) sdn[i] = op.dn[i / (2 * N)][(i / N) % 2][i % N];
  for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) sWt[i] = op.Wt[i / N][i % N];
  const int le = threadIdx.x / NN;
  const int t = threadIdx.x - le * NN;
  const int i0 = t % N, i1 = t / N;
  const int e = blockIdx.x * EPB + le;
  const bool valid = e < g.ne;
  int el = 0;
  Geom gl = g;
  if (valid) gl = local_geom(g, e, el);
  int ec[3] = {0, 0, 0};
  if (valid) elem_coords(gl, el, ec);
  if (valid && t < 4) snb[le][t] = neighbor(gl, ec, t >> 1, (t & 1) ? 1 : -1);
  __syncthreads();
  int kind[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const int nb = valid ? snb[le][f] : -1;
    kind[f] = nb >= 0 ? 1 : (g.bc[f >> 1] == 1 ? 2 : 0);
  }
  const size_t ebase = (size_t)e * NN;
  const T scale = sipg_beta(a, gl) * sipg_nu0(a, gl);
  __shared__ double red[S::THREADS];
  for (int s = 0; s < a.nsys; ++s) {
    const T* x = a.x + (size_t)s * a.sys_stride;
    const T* gd = a.gdata ? a.gdata + (size_t)s * a.g_stride : nullptr;
    T* y = a.y + (size_t)s * a.sys_stride;
    if (s > 0) __syncthreads();
    if (cg_system_stopped(a, s)) {            // its CG iteration has stopped: A p not needed
      if (a.dot_out && threadIdx.x == 0) put_dot_partial(a, s, 0.0);
      continue;
    }
    T uo = T(0);
    T dacc = T(0);
    if (valid) {
      uo = x[ebase + t];
      su[le][t] = uo;
      // face data: face fi = q / N, face node c = q % N for q = t, t + N^2, ... < 4N
      for (int q = t; q < 4 * N; q += NN) {
        const int fi = q / N, c = q % N, dir = fi >> 1, side = fi & 1;
        const int nb = snb[le][fi];
        T tr = T(0), dv = T(0);
        if (nb >= 0) {
          const int iface = side ? 0 : N - 1;
          const T* dr = sdn + (dir * 2 + side) * N;
          const T* line = x + (size_t)nb * NN + (dir == 0 ? c * N : c);
          const int stride = dir == 0 ? 1 : N;
#pragma unroll
          for (int j = 0; j < N; ++j) { const T v = line[j * stride]; dv += dr[j] * v; if (j == iface) tr = v; }
        } else if (kind[fi] == 2 && gd) {
          const int own = side ? N - 1 : 0;
          tr = gd[ebase + (dir == 0 ? c * N + own : own * N + c)];
        }
        sf[le][2 * fi][c] = tr;
        sf[le][2 * fi + 1][c] = dv;
      }
    }
    __syncthreads();
    if (valid) {
      const T* Ax = sA + (0 * 9 + 3 * kind[0] + kind[1]) * NN + i0 * N;
      const T* Ay = sA + (1 * 9 + 3 * kind[2] + kind[3]) * NN + i1 * N;
      T yx = T(0), yy = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        yx += Ax[j] * su[le][i1 * N + j];
        yy += Ay[j] * su[le][j * N + i0];
      }
      yx += sC[((0 * 2 + 0) * 3 + kind[0]) * 2 * N + i0] * sf[le][0][i1] +
            sC[(((0 * 2 + 0) * 3 + kind[0]) * 2 + 1) * N + i0] * sf[le][1][i1] +
            sC[((0 * 2 + 1) * 3 + kind[1]) * 2 * N + i0] * sf[le][2][i1] +
            sC[(((0 * 2 + 1) * 3 + kind[1]) * 2 + 1) * N + i0] * sf[le][3][i1];
      yy += sC[((1 * 2 + 0) * 3 + kind[2]) * 2 * N + i1] * sf[le][4][i0] +
            sC[(((1 * 2 + 0) * 3 + kind[2]) * 2 + 1) * N + i1] * sf[le][5][i0] +
            sC[((1 * 2 + 1) * 3 + kind[3]) * 2 * N + i1] * sf[le][6][i0] +
            sC[(((1 * 2 + 1) * 3 + kind[3]) * 2 + 1) * N + i1] * sf[le][7][i0];
      // unit-size line operators: direction k scales as 1 / h_k, its weights as h_k
      const T hx = geom_h<T>(gl, 0), hy = geom_h<T>(gl, 1);
      const T wx = hx * sWt[i0], wy = hy * sWt[N + i1];
      const T W = wx * wy;
      T out = a.alpha * W * uo + scale * (wy * yx / hx + wx * yy / hy);
      if (a.minv) out /= W;
      sipg_out<T, T>(a, y, ebase + t, uo, out);
      dacc = uo * out;
    }
    if (a.dot_out) {
      const double bs = block_sum_any_t<T>(dacc, red);
      if (threadIdx.x == 0) put_dot_partial(a, s, bs);
    }
  }
  if (a.dot_out) fused_dot_finish(a, red);
}

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
template <typename T>
struct ConstLine {
  T A[IMEX_MAXN * IMEX_MAXN];
  T ctrL[IMEX_MAXN], cdnL[IMEX_MAXN], ctrR[IMEX_MAXN], cdnR[IMEX_MAXN];
  T dnL[IMEX_MAXN], dnR[IMEX_MAXN];
  T w[IMEX_MAXN];
};
__constant__ ConstLine<float> c_line32[IMEX_MAXN + 1];
__constant__ ConstLine<double> c_line64[IMEX_MAXN + 1];
__constant__ ConstLine<ff> c_lineff[IMEX_MAXN + 1];
template <typename T> __device__ __forceinline__ const ConstLine<T>& cline(int N);
template <> __device__ __forceinline__ const ConstLine<ff>& cline<ff>(int N) { return c_lineff[N]; }
template <> __device__ __forceinline__ const ConstLine<float>& cline<float>(int N) { return c_line32[N]; }
template <> __device__ __forceinline__ const ConstLine<double>& cline<double>(int N) { return c_line64[N]; }

// 2D periodic line-owner apply: two passes (y, then x), in each a thread owns one whole line
// of an element; the block's elements are contiguous in memory and are staged into shared
// memory with fully coalesced loads.  Many elements per block keep the grid within about
// one wave of resident blocks.
// elements per block of the tuned kernels: variant 0 the default, 1 half of it, 2 twice it,
// 3 (3D FP32 only) one more element -- for N = 7 and 9, whose N^2 lines per element fill
// whole warps badly at the default (4 x 49 = 196 threads in 7 warps, 5 x 49 = 245 in 8)
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

template <typename T, int N, int V = 0>
__global__ void __launch_bounds__(Sipg2lShape<T, N, V>::THREADS)
sipg2l_apply_kernel(Geom g, SipgArgs<T> a) {
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
    int ec[3];
    elem_coords(gl, el, ec);
#pragma unroll
    for (int f = 0; f < 4; ++f) nb[f] = neighbor(gl, ec, f >> 1, (f & 1) ? 1 : -1);
  }
  const T hx = geom_h<T>(gl, 0), hy = geom_h<T>(gl, 1);
  const T ihx = T(1) / hx, ihy = T(1) / hy;
  const T scale = sipg_beta(a, gl) * sipg_nu0(a, gl);
  const int nvalid = min(EPB, g.ne - e0);
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
      const T wt = (T(0.5) * hx * L.w[ta]) * ihy;
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
      const T wy = T(0.5) * hy * L.w[ta];
      const T wt = wy * ihx;
#pragma unroll
      for (int o = 0; o < N; ++o) {
        T so = L.ctrL[o] * tl + L.cdnL[o] * dl + L.ctrR[o] * tr + L.cdnR[o] * dr;
#pragma unroll
        for (int j = 0; j < N; ++j) so += L.A[o * N + j] * v[j];
        const T W = wy * (T(0.5) * hx * L.w[o]);
        T out = a.alpha * W * v[o] + scale * (acc[le][ta * N + o] + wt * so);
        if (a.minv) out /= W;
        sipg_out<T, T>(a, y, (size_t)e * NN + ta * N + o, v[o], out);
        dacc += v[o] * out;
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

template <typename T, int N>
constexpr size_t sipg3p_smem() {
  using S = Sipg3pShape<T, N>;
  return sizeof(T) * (size_t)(S::EPB * S::TILE + S::EPB * 8 * S::NN);
}

// One group of EPB elements (group index grp) of the periodic constant-coefficient apply
// y = alpha M x + beta nu0 A x; every thread of the block must call it (it holds a barrier);
// returns this thread's share of (x, y).  Consecutive calls need a barrier in between.
template <typename T, int N>
__device__ __forceinline__ T sipg3p_group(const Geom& g, const SipgArgs<T>& a, const T* __restrict__ x,
                                          T* __restrict__ y, int grp) {
  using S = Sipg3pShape<T, N>;
  constexpr int NN = S::NN, ND = N * N * N, EPB = S::EPB, NP = S::NP, TILE = S::TILE, VEC = S::VEC;
  using VT = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);                       // [EPB][z][y][NP]
  T (*sf)[8][NN] = reinterpret_cast<T (*)[8][NN]>(tile + EPB * TILE);
  const ConstLine<T>& L = cline<T>(N);
  const int le = threadIdx.x / NN;
  const int t = threadIdx.x - le * NN;
  const int i0 = t % N, i1 = t / N;
  const int e = grp * EPB + le;
  const bool valid = e < g.ne;
  int el = 0;
  Geom gl = g;
  if (valid) gl = local_geom(g, e, el);
  int ec[3] = {0, 0, 0};
  int nb[6] = {0, 0, 0, 0, 0, 0};
  if (valid) {
    elem_coords(gl, el, ec);
#pragma unroll
    for (int f = 0; f < 6; ++f) nb[f] = neighbor(gl, ec, f >> 1, (f & 1) ? 1 : -1);
  }
  const T ihx = T(1) / geom_h<T>(gl, 0), ihy = T(1) / geom_h<T>(gl, 1), ihz = T(1) / geom_h<T>(gl, 2);
  const T hx2 = T(0.5) * geom_h<T>(gl, 0), hy2 = T(0.5) * geom_h<T>(gl, 1), hz2 = T(0.5) * geom_h<T>(gl, 2);
  // this thread's rows of the x and y line operators and neighbour coefficients
  T ax[N], ay[N];
#pragma unroll
  for (int j = 0; j < N; ++j) { ax[j] = L.A[i0 * N + j]; ay[j] = L.A[i1 * N + j]; }
  const T cxl0 = L.ctrL[i0], cxl1 = L.cdnL[i0], cxr0 = L.ctrR[i0], cxr1 = L.cdnR[i0];
  const T cyl0 = L.ctrL[i1], cyl1 = L.cdnL[i1], cyr0 = L.ctrR[i1], cyr1 = L.cdnR[i1];
  const T wx = hx2 * L.w[i0], wy = hy2 * L.w[i1];
  const size_t ebase = (size_t)e * ND;
  const T scale = sipg_beta(a, gl) * sipg_nu0(a, gl);
  T* mytile = tile + le * TILE;
  {
    T u[N];
    T zt0 = T(0), zd0 = T(0), zt1 = T(0), zd1 = T(0);
    T dacc = T(0);
    if (valid) {
#pragma unroll
      for (int k = 0; k < N; ++k) {
        u[k] = x[ebase + k * NN + t];
        mytile[(k * N + i1) * NP + i0] = u[k];
      }
      const int c0 = t % N, kk = t / N;
      {  // x-neighbours: rows along x at (y = c0, z = kk)
        const T* rl = x + (size_t)nb[0] * ND + kk * NN + c0 * N;
        const T* rr = x + (size_t)nb[1] * ND + kk * NN + c0 * N;
        T tl = T(0), dl = T(0), tr = T(0), dr = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const T vl = rl[j], vr = rr[j];
          dl += L.dnL[j] * vl;
          dr += L.dnR[j] * vr;
          if (j == N - 1) tl = vl;
          if (j == 0) tr = vr;
        }
        sf[le][0][t] = tl; sf[le][1][t] = dl; sf[le][2][t] = tr; sf[le][3][t] = dr;
      }
      {  // y-neighbours: columns along y at (x = c0, z = kk)
        const T* cl = x + (size_t)nb[2] * ND + kk * NN + c0;
        const T* cr = x + (size_t)nb[3] * ND + kk * NN + c0;
        T tl = T(0), dl = T(0), tr = T(0), dr = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const T vl = cl[j * N], vr = cr[j * N];
          dl += L.dnL[j] * vl;
          dr += L.dnR[j] * vr;
          if (j == N - 1) tl = vl;
          if (j == 0) tr = vr;
        }
        sf[le][4][t] = tl; sf[le][5][t] = dl; sf[le][6][t] = tr; sf[le][7][t] = dr;
      }
      {  // z-neighbours: columns along z through (i0, i1)
        const T* cl = x + (size_t)nb[4] * ND + t;
        const T* cr = x + (size_t)nb[5] * ND + t;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const T vl = cl[j * NN], vr = cr[j * NN];
          zd0 += L.dnL[j] * vl;
          zd1 += L.dnR[j] * vr;
          if (j == N - 1) zt0 = vl;
          if (j == 0) zt1 = vr;
        }
      }
    }
    __syncthreads();
    if (valid) {
#pragma unroll
      for (int k = 0; k < N; ++k) {
        // x: the padded row (y = i1, z = k) by 16-byte loads
        T row[NP];
        const VT* rv = reinterpret_cast<const VT*>(mytile + (k * N + i1) * NP);
#pragma unroll
        for (int q = 0; q < NP / VEC; ++q) {
          const VT v = rv[q];
          if (VEC == 4) {
            const float4 f = *reinterpret_cast<const float4*>(&v);
            reinterpret_cast<float*>(row)[4 * q + 0] = f.x;
            reinterpret_cast<float*>(row)[4 * q + 1] = f.y;
            reinterpret_cast<float*>(row)[4 * q + 2] = f.z;
            reinterpret_cast<float*>(row)[4 * q + 3] = f.w;
          } else {
            const double2 f = *reinterpret_cast<const double2*>(&v);
            reinterpret_cast<double*>(row)[2 * q + 0] = f.x;
            reinterpret_cast<double*>(row)[2 * q + 1] = f.y;
          }
        }
        T yx = T(0), yy = T(0), yz = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
          yx += ax[j] * row[j];
          yy += ay[j] * mytile[(k * N + j) * NP + i0];
          yz += L.A[k * N + j] * u[j];
        }
        const int f = i1 + N * k, fy = i0 + N * k;
        yx += cxl0 * sf[le][0][f] + cxl1 * sf[le][1][f] + cxr0 * sf[le][2][f] + cxr1 * sf[le][3][f];
        yy += cyl0 * sf[le][4][fy] + cyl1 * sf[le][5][fy] + cyr0 * sf[le][6][fy] + cyr1 * sf[le][7][fy];
        yz += L.ctrL[k] * zt0 + L.cdnL[k] * zd0 + L.ctrR[k] * zt1 + L.cdnR[k] * zd1;
        const T wz = hz2 * L.w[k];
        const T W = wx * wy * wz;
        const T yv = wy * wz * ihx * yx + wx * wz * ihy * yy + wx * wy * ihz * yz;
        T out = a.alpha * W * u[k] + scale * yv;
        if (a.minv) out /= W;
        y[ebase + k * NN + t] = out;
        dacc += u[k] * out;
      }
    }
    return dacc;
  }
}

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

template <typename T, int N, int V = 0>
constexpr size_t sipg3l_smem() {
  using S = Sipg3lShape<T, N, V>;
  return sizeof(T) * (size_t)(S::EPB * S::TILE + S::EPB * S::ND);
}

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

template <typename T, int N, typename TS = T, int V = 0, int EP = SIPG_EP_ANY>
__device__ __forceinline__ T sipg3l_group(const Geom& g, const SipgArgs<TS>& a, const TS* __restrict__ x,
                                          TS* __restrict__ y, int grp, int sys = 0) {
  using S = Sipg3lShape<T, N, V>;
  constexpr int NN = S::NN, ND = S::ND, EPB = S::EPB, NP = S::NP, TILE = S::TILE, VEC = S::VEC;
  // FP32 up to N = 8: all neighbour lines are loaded before the first pass, so that their
  // latency is paid once rather than after each of the two barriers (12 scalars stay live);
  // the wider types and N = 9 load them pass by pass (register pressure)
#ifndef IMEX_SIPG3L_HOIST
#define IMEX_SIPG3L_HOIST 1
#endif
  constexpr bool HOIST = IMEX_SIPG3L_HOIST && sizeof(T) == 4 && N <= 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);                       // [EPB][z][y][NP]
  T* acc = tile + EPB * TILE;                                     // [EPB][z][y][x]
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
    int ec[3];
    elem_coords(gl, el, ec);
#pragma unroll
    for (int f = 0; f < 6; ++f) nb[f] = neighbor(gl, ec, f >> 1, (f & 1) ? 1 : -1);
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
  const TS* zl = x + (size_t)nb[4] * ND + t;
  const TS* zr = x + (size_t)nb[5] * ND + t;
  const TS* yl = x + (size_t)nb[2] * ND + tb * NN + ta;
  const TS* yr = x + (size_t)nb[3] * ND + tb * NN + ta;
  const TS* xl = x + (size_t)nb[0] * ND + tb * NN + ta * N;
  const TS* xr = x + (size_t)nb[1] * ND + tb * NN + ta * N;
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
      const T out = sipg_out_ep<EP, T, TS>(a, y, eb + node, v[o], alpha * W * v[o] + scale * (ma[node] + wt * so), W);
      dacc += v[o] * out;
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
template <typename T, int N, typename TS = T, int V = 0, int EP = SIPG_EP_ANY>
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
    const T dacc = sipg3l_group<T, N, TS, V, EP>(g, a, a.x + (size_t)s * a.sys_stride,
                                             a.y + (size_t)s * a.sys_stride, blockIdx.x, s);
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

int pcg_persist_f32(const Geom& g, int N, const SipgArgs<float>& a, float* y, float* r, float* p, float* Ap,
                    const float* dinv, long long n, const CgScalars& sc, double stop_rr, int maxit, double* partial,
                    unsigned int* bar, int* err, cudaStream_t st) {
  if (g.d != 3 || g.inst || g.bc[0] || g.bc[1] || g.bc[2] || a.nu || !a.ops) return -1;
  PcgPersist q{y, r, p, Ap, dinv, n, stop_rr, partial, bar, err};
  SipgArgs<float> aa = a;
  aa.x = p;
  aa.y = Ap;
  aa.nsys = 1;
  aa.dot_out = nullptr;
  switch (N) {
    case 3: return launch_persist<3>(g, aa, q, sc, maxit, nullptr, st);
    case 4: return launch_persist<4>(g, aa, q, sc, maxit, nullptr, st);
    case 5: return launch_persist<5>(g, aa, q, sc, maxit, nullptr, st);
    case 6: return launch_persist<6>(g, aa, q, sc, maxit, nullptr, st);
    case 7: return launch_persist<7>(g, aa, q, sc, maxit, nullptr, st);
    case 8: return launch_persist<8>(g, aa, q, sc, maxit, nullptr, st);
    default: return -1;
  }
}

// fill the constant-memory line operators once per device
static bool g_cline_ready[64] = {false};
void init_const_lines(const Tables<double>& t) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || g_cline_ready[dev]) return;
  static ConstLine<double> h64[IMEX_MAXN + 1];
  static ConstLine<float> h32[IMEX_MAXN + 1];
  LineOps<double>* o = new LineOps<double>();
  LineOps<float>* of = new LineOps<float>();
  const double one[3] = {1.0, 1.0, 1.0};
  for (int N = 2; N <= IMEX_MAXN; ++N) {
    build_line_ops(t, N, one, 1, o, of);
    ConstLine<double>& c = h64[N];
    for (int i = 0; i < N * N; ++i) c.A[i] = o->A[0][4][i];
    for (int i = 0; i < N; ++i) {
      c.ctrL[i] = o->C[0][0][1][0][i];
      c.cdnL[i] = o->C[0][0][1][1][i];
      c.ctrR[i] = o->C[0][1][1][0][i];
      c.cdnR[i] = o->C[0][1][1][1][i];
      c.dnL[i] = o->dn[0][0][i];
      c.dnR[i] = o->dn[0][1][i];
      c.w[i] = t.w[N][i];
    }
    const double* src = reinterpret_cast<const double*>(&c);
    float* dst = reinterpret_cast<float*>(&h32[N]);
    for (size_t i = 0; i < sizeof(ConstLine<double>) / sizeof(double); ++i) dst[i] = (float)src[i];
  }
  delete o;
  delete of;
  if (cudaMemcpyToSymbol(c_line64, h64, sizeof(h64)) == cudaSuccess &&
      cudaMemcpyToSymbol(c_line32, h32, sizeof(h32)) == cudaSuccess) {
    static ConstLine<ff> hff[IMEX_MAXN + 1];
    for (int N = 2; N <= IMEX_MAXN; ++N) {
      const double* src = reinterpret_cast<const double*>(&h64[N]);
      ff* dst = reinterpret_cast<ff*>(&hff[N]);
      for (size_t i = 0; i < sizeof(ConstLine<double>) / sizeof(double); ++i) dst[i] = ff(src[i]);
    }
    if (cudaMemcpyToSymbol(c_lineff, hff, sizeof(hff)) == cudaSuccess) g_cline_ready[dev] = true;
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
  int el = 0;
  Geom gl = g;
  if (valid) gl = local_geom(g, e, el);
  if (valid) snu[le][node] = a.nu ? a.nu[(size_t)e * ND + node] : sipg_nu0(a, gl);
  __syncthreads();
  if (!valid) return;
  (void)NF;
  int ec[3];
  elem_coords(gl, el, ec);
  int id[3];
  id[0] = node % N;
  id[1] = (D > 1) ? (node / N) % N : 0;
  id[2] = (D > 2) ? node / (N * N) : 0;
  T hinv2[D];
  T jac = T(1);
  for (int k = 0; k < D; ++k) { hinv2[k] = T(2) / geom_h<T>(gl, k); jac *= geom_h<T>(gl, k) * T(0.5); }
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
      const int nb = neighbor(gl, ec, k, side ? 1 : -1);
      if (nb < 0 && geom_bc(g, k) != 1) continue;
      T Wf = jac / (geom_h<T>(gl, k) * T(0.5));
      for (int j = 0; j < D; ++j) if (j != k) Wf *= sw[id[j]];
      const T n = side ? T(1) : T(-1);
      const T dself = n * sD[id[k] * N + id[k]] * hinv2[k];   // d(e_j)/dn at its own face node
      const T pen = T(N * N) * T(0.5) * hinv2[k];
      if (nb >= 0) {
        int c[3] = {id[0], id[1], id[2]};
        c[k] = side ? 0 : N - 1;
        const int nn = c[0] + N * ((D > 1 ? c[1] : 0) + N * (D > 2 ? c[2] : 0));
        const T nun = a.nu ? a.nu[(size_t)nb * ND + nn] : sipg_nu0(a, gl);
        diag += -Wf * nuq * dself + Wf * pen * (nuq > nun ? nuq : nun);
      } else {
        diag += -T(2) * Wf * nuq * dself + Wf * T(2) * pen * nuq;
      }
    }
  }
  a.y[(size_t)e * ND + node] = a.alpha * Wq + sipg_beta(a, gl) * diag;
}

template <typename T, int N, int V>
static void launch_apply2l(const Geom& g, const SipgArgs<T>& a, cudaStream_t st) {
  using C = Sipg2lShape<T, N, V>;
  IMEX_COUNTED((sipg2l_apply_kernel<T, N, V><<<(g.ne + C::EPB - 1) / C::EPB, C::THREADS, 0, st>>>(g, a)));
}

template <typename T, int D, int N>
static void launch_apply(const Geom& g, const SipgArgs<T>& a, cudaStream_t st) {
  if (D == 2 && !a.nu && a.ops && g.bc[0] == 0 && g.bc[1] == 0 && N <= IMEX_MAXN) {
    // the variant chosen by the tuner (twice the elements per block: FP32 only, for the
    // static shared memory)
    if (a.variant == 1) launch_apply2l<T, N, 1>(g, a, st);
    else if constexpr (sizeof(T) == 4) {
      if (a.variant == 2) launch_apply2l<T, N, 2>(g, a, st);
      else launch_apply2l<T, N, 0>(g, a, st);
    } else {
      launch_apply2l<T, N, 0>(g, a, st);
    }
    return;
  }
  if (D == 2 && !a.nu && a.ops) {
    using C = Sipg2cShape<N>;
    constexpr size_t sm = sipg2c_smem<T, N>();
    smem_limit_once((const void*)sipg2c_apply_kernel<T, N>, (int)sm);
    IMEX_COUNTED(sipg2c_apply_kernel<T, N><<<(g.ne + C::EPB - 1) / C::EPB, C::THREADS, sm, st>>>(g, a));
    return;
  }
  using S = SipgShape<T, D, N>;
  int blocks = (g.ne + S::EPB - 1) / S::EPB;
  IMEX_COUNTED(sipg_apply_kernel<T, D, N><<<blocks, S::THREADS, 0, st>>>(g, a));
}

template <typename T, int N, int V, int EP>
static void launch_apply3p_ep(const Geom& g, const SipgArgs<T>& a, cudaStream_t st) {
  using P = Sipg3pShape<T, N, V>;
  constexpr size_t sm = sipg3l_smem<T, N, V>();
  smem_limit_once((const void*)sipg3p_apply_kernel<T, N, T, V, EP>, (int)sm);
  launch_cg_kernel(sipg3p_apply_kernel<T, N, T, V, EP>, (g.ne + P::EPB - 1) / P::EPB, P::THREADS, sm, st, g, a);
}
// FP32 (the CG and V-cycle applies): the output stage fixed at compile time unless M^{-1}
// is asked for
template <typename T, int N, int V>
static void launch_apply3p(const Geom& g, const SipgArgs<T>& a, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (!a.minv) {
      if (a.cheb) launch_apply3p_ep<T, N, V, SIPG_EP_CHEB>(g, a, st);
      else launch_apply3p_ep<T, N, V, SIPG_EP_PLAIN>(g, a, st);
      return;
    }
  }
  launch_apply3p_ep<T, N, V, SIPG_EP_ANY>(g, a, st);
}

template <typename T, int D, int N>
static void launch_apply3(const Geom& g, const SipgArgs<T>& a, cudaStream_t st) {
  if (!a.nu && a.ops && g.bc[0] == 0 && g.bc[1] == 0 && g.bc[2] == 0) {
    if (a.variant == 1) launch_apply3p<T, N, 1>(g, a, st);
    else if (a.variant == 2) launch_apply3p<T, N, 2>(g, a, st);
    else if constexpr (sizeof(T) == 4) {
      if (a.variant == 3) launch_apply3p<T, N, 3>(g, a, st);
      else launch_apply3p<T, N, 0>(g, a, st);
    } else {
      launch_apply3p<T, N, 0>(g, a, st);
    }
    return;
  }
  if (!a.nu && a.ops) {
    using C = Sipg3cShape<N>;
    constexpr size_t sm = sipg3c_smem<T, N>();
    smem_limit_once((const void*)sipg3c_apply_kernel<T, N>, (int)sm);
    IMEX_COUNTED(sipg3c_apply_kernel<T, N><<<(g.ne + C::EPB - 1) / C::EPB, C::THREADS, sm, st>>>(g, a));
    return;
  }
  using S = Sipg3Shape<N>;
  const int blocks = (g.ne + S::EPB - 1) / S::EPB;
  constexpr size_t smem = sipg3_smem<T, N>();
  if (a.nu) {
    smem_limit_once((const void*)sipg3_apply_kernel<T, N, true>, (int)smem);
    IMEX_COUNTED(sipg3_apply_kernel<T, N, true><<<blocks, S::THREADS, smem, st>>>(g, a));
  } else {
    smem_limit_once((const void*)sipg3_apply_kernel<T, N, false>, (int)smem);
    IMEX_COUNTED(sipg3_apply_kernel<T, N, false><<<blocks, S::THREADS, smem, st>>>(g, a));
  }
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

template <int N>
static void launch_apply_ff(const Geom& g, const SipgArgs<double>& a, cudaStream_t st) {
  using P = Sipg3pShape<ff, N>;
  constexpr size_t sm = sipg3l_smem<ff, N>();
  smem_limit_once((const void*)sipg3p_apply_kernel<ff, N, double>, (int)sm);
  IMEX_COUNTED(sipg3p_apply_kernel<ff, N, double><<<(g.ne + P::EPB - 1) / P::EPB, P::THREADS, sm, st>>>(g, a));
}

int sipg_apply_ff(const Geom& g, int N, const SipgArgs<double>& a, cudaStream_t st) {
  if (g.d != 3 || g.bc[0] || g.bc[1] || g.bc[2] || a.nu || !a.ops || a.gdata) return -1;
  switch (N) {
    case 3: launch_apply_ff<3>(g, a, st); return 0;
    case 4: launch_apply_ff<4>(g, a, st); return 0;
    case 5: launch_apply_ff<5>(g, a, st); return 0;
    case 6: launch_apply_ff<6>(g, a, st); return 0;
    case 7: launch_apply_ff<7>(g, a, st); return 0;
    case 8: launch_apply_ff<8>(g, a, st); return 0;
    case 9: launch_apply_ff<9>(g, a, st); return 0;
    default: return -1;
  }
}

template <typename T>
int sipg_apply(const Geom& g, int N, const SipgArgs<T>& a, cudaStream_t st) {
  if (a.dot_out && (a.nu || !a.ops)) return -2;     // the fused dot exists on the constant-nu path only
  if (a.cheb && (a.nu || !a.ops || a.gdata)) return -3;  // so does the fused Chebyshev step
  if (g.d == 2) { IMEX_DISPATCH_N(2, launch_apply, g, a, st) }
  else { IMEX_DISPATCH_N(3, launch_apply3, g, a, st) }
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
