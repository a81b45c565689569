// Output stages, block sums and CG hooks shared by the SIPG operator kernels (k_sipg.cu:
// generic and face-kind kernels; k_sipg_line32.cu / k_sipg_line64.cu: the line-owner kernels
// of the constant-viscosity periodic meshes).
#pragma once
#include <type_traits>

#include "common.cuh"
#include "ff.cuh"
#include "kernels.h"
#include "vec.h"

namespace imex {

// Output of one node of an apply: y = A x, or a fused Chebyshev step of the p-multigrid
// smoother (a.cheb = 1: r -= A x, d' = c1 x + c2 D^{-1} r, s += d', xin this node's input x;
// a.cheb = 2, the first step from the current s = x: r = b - A x, d = c1 D^{-1} r)
template <typename T, typename TS>
__device__ __forceinline__ void sipg_cheb_step(const SipgArgs<TS>& a, size_t i, T xin, T out) {
  const T r = T(a.ch_r[i]) - out;
  const T dn = T(a.ch_c1) * xin + T(a.ch_c2) * T(a.ch_dinv[i]) * r;
  a.ch_s[i] = (TS)(T(a.ch_s[i]) + (a.ch_addx ? xin + dn : dn));
  if (!a.ch_last) {
    a.ch_r[i] = (TS)r;
    a.ch_dout[i] = (TS)dn;
  }
}
template <typename T, typename TS>
__device__ __forceinline__ void sipg_cheb_first(const SipgArgs<TS>& a, size_t i, T out) {
  const T r = T(a.ch_b[i]) - out;
  a.ch_r[i] = (TS)r;
  a.ch_dout[i] = (TS)(T(a.ch_c1) * T(a.ch_dinv[i]) * r);
}
template <typename T, typename TS>
__device__ __forceinline__ void sipg_out(const SipgArgs<TS>& a, TS* __restrict__ y, size_t i, T xin, T out) {
  if (!a.cheb) {
    y[i] = (TS)out;
    return;
  }
  if (a.cheb == 2) sipg_cheb_first<T, TS>(a, i, out);
  else sipg_cheb_step<T, TS>(a, i, xin, out);
}
// Output stage chosen at compile time: EP = 0 reads the flags (M^{-1}, Chebyshev) at run
// time, 1 writes y = A x, 2 performs a Chebyshev step, 3 the first step from a nonzero s.
// Fixed stages keep the unused branches -- a precise division, the Chebyshev loads and
// stores -- out of the unrolled output loop, where the compiler would otherwise predicate
// them into every node.
constexpr int SIPG_EP_ANY = 0, SIPG_EP_PLAIN = 1, SIPG_EP_CHEB = 2, SIPG_EP_CHEB_FIRST = 3;
template <int EP, typename T, typename TS>
__device__ __forceinline__ T sipg_out_ep(const SipgArgs<TS>& a, TS* __restrict__ y, size_t i, T xin, T out, T W) {
  if constexpr (EP == SIPG_EP_PLAIN) {
    y[i] = (TS)out;
  } else if constexpr (EP == SIPG_EP_CHEB) {
    sipg_cheb_step<T, TS>(a, i, xin, out);
  } else if constexpr (EP == SIPG_EP_CHEB_FIRST) {
    sipg_cheb_first<T, TS>(a, i, out);
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

// the line-owner kernels of the periodic constant-viscosity meshes (2D line and 3D periodic
// applies): -1 when the mesh or the arguments are not such a case (nothing launched)
int sipg_apply_line(const Geom& g, int N, const SipgArgs<float>& a, cudaStream_t st);
int sipg_apply_line(const Geom& g, int N, const SipgArgs<double>& a, cudaStream_t st);
// constant-memory line operators of the line-owner translation units
template <typename T>
struct ConstLine {
  T A[IMEX_MAXN * IMEX_MAXN];
  T ctrL[IMEX_MAXN], cdnL[IMEX_MAXN], ctrR[IMEX_MAXN], cdnR[IMEX_MAXN];
  T dnL[IMEX_MAXN], dnR[IMEX_MAXN];
  T w[IMEX_MAXN];
};
bool upload_const_lines_f32(const ConstLine<float>* h);
bool upload_const_lines_f64(const ConstLine<double>* h64, const ConstLine<ff>* hff);

}  // namespace imex
