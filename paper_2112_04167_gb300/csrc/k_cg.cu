// Segmented Jacobi-PCG kernels (the linear solves of Alg. 3 / Alg. 4, which Sec. 3.3 solves by
// preconditioned CG: pressure Poisson and viscous Helmholtz problems, both symmetric positive (semi-)definite, preconditioned by the
// operator's diagonal).
//
// The systems solved together (the vector components of one instance, or the instances of
// a batch) are segments of the same vectors.  A 1D grid of blocks covers them, each block
// one chunk of SEG_CHUNK elements of one segment, so uneven segment lengths cost no idle
// blocks.  Per-block partial sums are combined in block order (deterministic) by the last
// block to finish; the per-system scalars never leave device memory.  The step length
// alpha = (r, z) / (p, A p) is the exception: the operator apply (or the dot kernel) only
// leaves its per-block partials of (p, A p), and every block of the step kernel adds those
// of its system in the same fixed order -- identical in all blocks, and no completion
// counter, fence or last-block sum at the end of the apply.
//
// Singular systems (project = 1; null space = the constants) run the projected iteration:
// the residual r' = r - rho 1 (rho = mean r) and the preconditioned residual
// z' = D^{-1} r' - mean(D^{-1} r') are kept out of the null space.  Rounding in A p lets the
// recursive residual pick up a constant part every iteration; the partial sums
// S_rz = (r, D^{-1} r), S_rr = (r, r), S_z = sum D^{-1} r, S_r = sum r of the unprojected r give
// the projected scalars in closed form,
//   (r', z') = S_rz - 2 rho S_z + rho^2 sum D^{-1},  (r', r') = S_rr - n rho^2,
//   mean(D^{-1} r') = (S_z - rho sum D^{-1}) / n,
// and the direction update stores r' back, so the drift never accumulates.
//
// Data movement: every kernel streams its vectors with 16-byte loads (the direction kernel
// issues all of a thread's loads before the arithmetic; the step kernel, with five input
// vectors, one 16-byte group of each at a time, which keeps its register count low enough
// for one wave of blocks), and falls back to scalar accesses for chunks whose addresses are
// not 16-byte aligned.  FP32 instances accumulate per thread and per warp in FP32 and
// switch to FP64 at the per-warp level (GB300 executes FP64 at a small fraction of the FP32
// rate).
#include <cstdint>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"
#include "vec.h"

namespace imex {
namespace {

constexpr int CG_THREADS = 256;

template <typename T> struct Vec16;
template <> struct Vec16<float> { using V = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using V = double2; static constexpr int n = 2; };

__device__ __forceinline__ void vload(const float* p, float (&o)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void vload(const double* p, double (&o)[2]) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  o[0] = v.x; o[1] = v.y;
}
__device__ __forceinline__ void vstore(float* p, const float (&o)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
}
__device__ __forceinline__ void vstore(double* p, const double (&o)[2]) {
  *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
}
__device__ __forceinline__ bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// K block sums of per-thread values in T; out[] valid in thread 0.  Warp sums by shuffles,
// then warp 0 adds the per-warp sums with one more shuffle tree in T (no serial FP64 on one
// thread while the block waits); the K results are converted once.  Ends with a barrier, so
// it may be called repeatedly.  blockDim.x must be a multiple of 32.
template <typename T, int K>
__device__ __forceinline__ void block_sum_k(T (&v)[K], double (&out)[K]) {
  __shared__ T ws[K][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_sum_t(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) ws[k][w] = v[k];
  }
  __syncthreads();
  if (w == 0) {
    const int nw = (int)(blockDim.x >> 5);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const T x = warp_sum_t(lane < nw ? ws[k][lane] : T(0));
      if (lane == 0) out[k] = (double)x;
    }
  }
  __syncthreads();
}

// last block of the grid? (thread 0 publishes; all threads get the answer)
__device__ __forceinline__ bool last_block(unsigned int* counter) {
  __shared__ int am_last;
  if (threadIdx.x == 0) {
    __threadfence();
    am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (am_last) __threadfence();
  return am_last != 0;
}

// Totals over the blocks of each segment of the K partials partial[k * nblk + b], handed to
// fn(q, tot) once per segment (by one thread).  Few segments: the whole block adds each
// segment's partials (one load latency); many short segments (a batch): one thread per
// segment, all segments at once; otherwise one warp per segment.
template <int K, typename Fn>
__device__ __forceinline__ void seg_totals(const SegTable& t, const double* __restrict__ partial, Fn fn) {
  if (t.nseg <= 4) {
    for (int q = 0; q < t.nseg; ++q) {
      double v[K];
#pragma unroll
      for (int k = 0; k < K; ++k) v[k] = 0.0;
      for (int b = t.seg_blk0[q] + threadIdx.x; b < t.seg_blk0[q + 1]; b += blockDim.x) {
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] += partial[(size_t)k * t.nblk + b];
      }
      double tot[K];
      block_sum_k<double, K>(v, tot);
      if (threadIdx.x == 0) fn(q, tot);
    }
  } else if (t.nblk <= 24 * t.nseg) {
    for (int q = threadIdx.x; q < t.nseg; q += blockDim.x) {
      double v[K];
#pragma unroll
      for (int k = 0; k < K; ++k) v[k] = 0.0;
      const int b0 = t.seg_blk0[q], b1 = t.seg_blk0[q + 1];
#pragma unroll 4
      for (int b = b0; b < b1; ++b) {
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] += partial[(size_t)k * t.nblk + b];
      }
      fn(q, v);
    }
  } else {
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5, lane = threadIdx.x & 31;
    for (int q = warp; q < t.nseg; q += nw) {
      double v[K];
#pragma unroll
      for (int k = 0; k < K; ++k) v[k] = 0.0;
#pragma unroll 4
      for (int b = t.seg_blk0[q] + lane; b < t.seg_blk0[q + 1]; b += 32) {
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] += partial[(size_t)k * t.nblk + b];
      }
#pragma unroll
      for (int k = 0; k < K; ++k) v[k] = warp_sum_t(v[k]);
      if (lane == 0) fn(q, v);
    }
  }
}

// projected (or plain) CG scalars of one segment from its totals S_rz, S_rr, S_z, S_r
struct SegSums {
  double rz, rr, zmean, rmean;
};
__device__ __forceinline__ SegSums seg_scalars(const double* tot, double n, double dsum, int project) {
  SegSums o;
  o.rz = tot[0];
  o.rr = tot[1];
  o.zmean = 0.0;
  o.rmean = 0.0;
  if (project) {
    const double rho = tot[3] / n;
    o.rz = tot[0] - 2.0 * rho * tot[2] + rho * rho * dsum;
    o.rr = fmax(tot[1] - n * rho * rho, 0.0);
    o.zmean = (tot[2] - rho * dsum) / n;
    o.rmean = rho;
  }
  return o;
}

// this block's chunk (one 32-byte load)
__device__ __forceinline__ SegBlock chunk_of(const SegTable& t) {
  const int4* p = reinterpret_cast<const int4*>(t.blk + blockIdx.x);
  const int4 a = p[0], b = p[1];
  SegBlock c;
  c.off = ((long long)(unsigned)a.x) | ((long long)a.y << 32);
  c.doff = ((long long)(unsigned)a.z) | ((long long)a.w << 32);
  c.n = b.x;
  c.s = b.y;
  return c;
}

template <typename T> __device__ __forceinline__ T pick(const double* d, const float* f, int s);
template <> __device__ __forceinline__ float pick<float>(const double*, const float* f, int s) { return f[s]; }
template <> __device__ __forceinline__ double pick<double>(const double* d, const float*, int s) { return d[s]; }

__host__ __device__ constexpr int unroll_of(int vec) { return SEG_CHUNK / (vec * CG_THREADS); }

// x += alpha p, r -= alpha A p, and the partial sums of the new residual; the last block
// forms the new scalars, the stopping test of Sec. 4 and the next direction
// coefficient beta = rz_new / rz
// FP32: at least 5 blocks per SM, so that a 1.4 M-node system's 686 blocks run in one wave
// of 152 SMs (4 per SM left 78 blocks for a second wave)
template <typename T>
__global__ void __launch_bounds__(CG_THREADS, sizeof(T) == 4 ? 5 : 2)
seg_xr_kernel(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p, const T* __restrict__ Ap,
              const T* __restrict__ dinv, SegTable t, CgScalars sc, double* __restrict__ partial,
              unsigned int* __restrict__ counter, int maxit) {
  constexpr int VN = Vec16<T>::n, U = unroll_of(VN);
  pdl_trigger();
  const SegBlock c = chunk_of(t);
  T acc[4] = {T(0), T(0), T(0), T(0)};          // (r, z), (r, r), sum z, sum r
  pdl_wait();
  bool run = sc.done[c.s] == 0;
  T a;
  if (sc.apart) {
    // the apply (or the dot kernel) left per-block partials of (p, A p) in T: every block
    // adds those of its system in the same order, so all blocks of a system hold the same
    // alpha
    const T* pp = reinterpret_cast<const T*>(sc.apart);
    int b0, b1;
    if (sc.apart_seg) {
      b0 = t.seg_blk0[c.s];
      b1 = t.seg_blk0[c.s + 1];
    } else {
      const int nb = (int)*sc.apart_n;
      b0 = c.s * nb;
      b1 = b0 + nb;
    }
    T v[1] = {T(0)};
    for (int b = b0 + threadIdx.x; b < b1; b += CG_THREADS) v[0] += pp[b];
    double tot[1];
    block_sum_k<T, 1>(v, tot);
    // alpha = rz / pAp in T: the step uses it in T, and FP32 needs no FP64 division
    __shared__ T s_alpha;
    if (threadIdx.x == 0) {
      const T al = tot[0] != 0.0 ? T(sc.rz[c.s]) / T(tot[0]) : T(0);
      s_alpha = al;
      if (!isfinite(al) && run) atomicCAS(sc.done + c.s, 0, 2);   // breakdown of this system
    }
    __syncthreads();
    a = s_alpha;
    run = run && isfinite(a);
  } else {
    a = pick<T>(sc.alpha, sc.alpha_f, c.s);
  }
  if (run) {
    T* xs = x + c.off;
    T* rs = r + c.off;
    const T* ps = p + c.off;
    const T* aps = Ap + c.off;
    const T* ds = dinv + c.doff;
    const int n = c.n;
    int done_n = 0;
    if (al16(xs) && al16(rs) && al16(ps) && al16(aps) && al16(ds)) {
      const int nv = n / VN;
      // one 16-byte group of each vector at a time (fewer registers: more resident blocks)
#pragma unroll 1
      for (int u = 0; u < U; ++u) {
        const int v = threadIdx.x + u * CG_THREADS;
        if (v < nv) {
          T rv[VN], av[VN], dv[VN], xv[VN], pv[VN];
          vload(rs + v * VN, rv); vload(aps + v * VN, av); vload(ds + v * VN, dv);
          vload(xs + v * VN, xv); vload(ps + v * VN, pv);
#pragma unroll
          for (int j = 0; j < VN; ++j) {
            const T ri = rv[j] - a * av[j];
            const T zi = ri * dv[j];
            xv[j] += a * pv[j];
            rv[j] = ri;
            acc[0] += ri * zi;
            acc[1] += ri * ri;
            acc[2] += zi;
            acc[3] += ri;
          }
          vstore(xs + v * VN, xv);
          vstore(rs + v * VN, rv);
        }
      }
      done_n = nv * VN;
    }
    for (int i = done_n + threadIdx.x; i < n; i += CG_THREADS) {
      const T ri = rs[i] - a * aps[i];
      const T zi = ri * ds[i];
      xs[i] += a * ps[i];
      rs[i] = ri;
      acc[0] += ri * zi;
      acc[1] += ri * ri;
      acc[2] += zi;
      acc[3] += ri;
    }
  }
  double bs[4];
  block_sum_k<T, 4>(acc, bs);
  if (threadIdx.x == 0) {
    for (int k = 0; k < 4; ++k) partial[(size_t)k * t.nblk + blockIdx.x] = bs[k];
  }
  if (!last_block(counter)) return;
  // the scalars the update needs, loaded before the partial sums (their latencies overlap)
  struct Pre {
    double rz, dsum, bb;
    int done, iters, len;
  };
  Pre pre[4];
  if (threadIdx.x == 0 && t.nseg <= 4)
    for (int q = 0; q < t.nseg; ++q) pre[q] = {sc.rz[q], sc.dsum[q], sc.bb[q], sc.done[q], sc.iters[q], t.len[q]};
  seg_totals<4>(t, partial, [&](int q, const double* tot) {
    const Pre v = t.nseg <= 4 ? pre[q]
                              : Pre{sc.rz[q], sc.dsum[q], sc.bb[q], sc.done[q], sc.iters[q], t.len[q]};
    if (v.done != 0) return;
    const SegSums o = seg_scalars(tot, (double)v.len, v.dsum, sc.project);
    const double bt = v.rz != 0.0 ? o.rz / v.rz : 0.0;
    sc.rz_old[q] = v.rz;
    sc.rz[q] = o.rz;
    sc.rr[q] = o.rr;
    sc.zmean[q] = o.zmean;
    sc.rmean[q] = o.rmean;
    sc.zmean_f[q] = (float)o.zmean;
    sc.rmean_f[q] = (float)o.rmean;
    sc.beta[q] = bt;
    sc.beta_f[q] = (float)bt;
    sc.iters[q] = v.iters + 1;
    if (o.rr != o.rr || !isfinite(bt)) sc.done[q] = 2;
    else if (o.rr <= sc.tol2 * v.bb) sc.done[q] = 1;
    else if (v.iters + 1 >= maxit) sc.done[q] = 3;
  });
  if (threadIdx.x == 0) *counter = 0u;
}

// the Jacobi-preconditioned direction of the CG of Sec. 3.3 (projected for singular systems):
// z' = D^{-1} (r - rmean) - zmean, p = z' + beta p (beta = 0 with restart = 1); projected
// systems store r - rmean back
template <typename T>
__global__ void __launch_bounds__(CG_THREADS)
seg_p_kernel(T* __restrict__ p, T* __restrict__ r, const T* __restrict__ dinv, SegTable t, CgScalars sc,
             int restart) {
  constexpr int VN = Vec16<T>::n, U = unroll_of(VN);
  pdl_trigger();
  const SegBlock c = chunk_of(t);
  pdl_wait();
  if (sc.done[c.s] != 0) return;
  const bool proj = sc.project != 0;
  const T beta = restart ? T(0) : pick<T>(sc.beta, sc.beta_f, c.s);
  const T zm = proj ? pick<T>(sc.zmean, sc.zmean_f, c.s) : T(0);
  const T rm = proj ? pick<T>(sc.rmean, sc.rmean_f, c.s) : T(0);
  T* ps = p + c.off;
  T* rs = r + c.off;
  const T* ds = dinv + c.doff;
  const int n = c.n;
  int done_n = 0;
  if (al16(ps) && al16(rs) && al16(ds)) {
    const int nv = n / VN;
    T rv[U][VN], dv[U][VN], pv[U][VN];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int v = threadIdx.x + u * CG_THREADS;
      if (v < nv) {
        vload(rs + v * VN, rv[u]); vload(ds + v * VN, dv[u]);
        if (!restart) {
          vload(ps + v * VN, pv[u]);
        } else {
#pragma unroll
          for (int j = 0; j < VN; ++j) pv[u][j] = T(0);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int v = threadIdx.x + u * CG_THREADS;
      if (v < nv) {
#pragma unroll
        for (int j = 0; j < VN; ++j) {
          const T ri = rv[u][j] - rm;
          const T zi = ri * dv[u][j] - zm;
          rv[u][j] = ri;
          pv[u][j] = zi + beta * pv[u][j];
        }
        if (proj) vstore(rs + v * VN, rv[u]);
        vstore(ps + v * VN, pv[u]);
      }
    }
    done_n = nv * VN;
  }
  for (int i = done_n + threadIdx.x; i < n; i += CG_THREADS) {
    const T ri = rs[i] - rm;
    const T zi = ri * ds[i] - zm;
    if (proj) rs[i] = ri;
    ps[i] = restart ? zi : zi + beta * ps[i];
  }
}

// streaming dot of one chunk into acc (16-byte loads where aligned)
template <typename T>
__device__ __forceinline__ T chunk_dot(const T* xs, const T* ys, int n) {
  constexpr int VN = Vec16<T>::n, U = unroll_of(VN);
  T acc = T(0);
  int done_n = 0;
  if (al16(xs) && al16(ys)) {
    const int nv = n / VN;
    T xv[U][VN], yv[U][VN];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int v = threadIdx.x + u * CG_THREADS;
      if (v < nv) { vload(xs + v * VN, xv[u]); vload(ys + v * VN, yv[u]); }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int v = threadIdx.x + u * CG_THREADS;
      if (v < nv) {
#pragma unroll
        for (int j = 0; j < VN; ++j) acc += xv[u][j] * yv[u][j];
      }
    }
    done_n = nv * VN;
  }
  for (int i = done_n + threadIdx.x; i < n; i += CG_THREADS) acc += xs[i] * ys[i];
  return acc;
}

// dot per segment into out[s] (the CG scalars and residual norms of Sec. 4)
template <typename T>
__global__ void __launch_bounds__(CG_THREADS)
seg_dot_kernel(const T* __restrict__ x, const T* __restrict__ y, SegTable t, double* __restrict__ out,
               double* __restrict__ partial, unsigned int* __restrict__ counter) {
  const SegBlock c = chunk_of(t);
  T acc[1] = {chunk_dot(x + c.off, y + c.off, c.n)};
  double bs[1];
  block_sum_k<T, 1>(acc, bs);
  if (threadIdx.x == 0) partial[blockIdx.x] = bs[0];
  if (!last_block(counter)) return;
  seg_totals<1>(t, partial, [&](int q, const double* tot) { out[q] = tot[0]; });
  if (threadIdx.x == 0) *counter = 0u;
}

// (p, A p) per running system into sc.pAp and the CG step length alpha = rz / pAp
template <typename T>
__global__ void __launch_bounds__(CG_THREADS)
seg_pap_kernel(const T* __restrict__ p, const T* __restrict__ Ap, SegTable t, CgScalars sc,
               double* __restrict__ partial, unsigned int* __restrict__ counter) {
  const SegBlock c = chunk_of(t);
  T acc[1] = {sc.done[c.s] == 0 ? chunk_dot(p + c.off, Ap + c.off, c.n) : T(0)};
  double bs[1];
  block_sum_k<T, 1>(acc, bs);
  if (sc.apart_seg) {
    // deferred: the block's partial in T, added by the step kernel of its segment
    if (threadIdx.x == 0) reinterpret_cast<T*>(const_cast<double*>(sc.apart))[blockIdx.x] = (T)bs[0];
    return;
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = bs[0];
  if (!last_block(counter)) return;
  seg_totals<1>(t, partial, [&](int q, const double* tot) {
    if (sc.done[q] != 0) return;
    const double al = tot[0] != 0.0 ? sc.rz[q] / tot[0] : 0.0;
    const bool ok = isfinite(al);
    sc.pAp[q] = tot[0];
    sc.alpha[q] = ok ? al : 0.0;
    sc.alpha_f[q] = ok ? (float)al : 0.f;
    if (!ok) sc.done[q] = 2;
  });
  if (threadIdx.x == 0) *counter = 0u;
}

// CG scalars of a new residual r for the running systems, with the stopping test of Sec. 4
// (all systems with reset = 1,
// which also restarts their iteration counts and convergence flags); also sum D^{-1}
template <typename T>
__global__ void __launch_bounds__(CG_THREADS)
seg_init_kernel(const T* __restrict__ r, const T* __restrict__ dinv, SegTable t, CgScalars sc,
                double* __restrict__ partial, unsigned int* __restrict__ counter, int reset) {
  const SegBlock c = chunk_of(t);
  T acc[5] = {T(0), T(0), T(0), T(0), T(0)};   // (r, z), (r, r), sum z, sum r, sum D^{-1}
  if (sc.done[c.s] == 0 || reset) {
    const T* rs = r + c.off;
    const T* ds = dinv + c.doff;
    for (int i = threadIdx.x; i < c.n; i += CG_THREADS) {
      const T ri = rs[i];
      const T di = ds[i];
      const T zi = ri * di;
      acc[0] += ri * zi;
      acc[1] += ri * ri;
      acc[2] += zi;
      acc[3] += ri;
      acc[4] += di;
    }
  }
  double bs[5];
  block_sum_k<T, 5>(acc, bs);
  if (threadIdx.x == 0) {
    for (int k = 0; k < 5; ++k) partial[(size_t)k * t.nblk + blockIdx.x] = bs[k];
  }
  if (!last_block(counter)) return;
  seg_totals<5>(t, partial, [&](int q, const double* tot) {
    if (!(reset || sc.done[q] == 0)) return;
    const SegSums o = seg_scalars(tot, (double)t.len[q], tot[4], sc.project);
    sc.dsum[q] = tot[4];
    sc.rz[q] = o.rz;
    sc.rr[q] = o.rr;
    sc.zmean[q] = o.zmean;
    sc.rmean[q] = o.rmean;
    sc.zmean_f[q] = (float)o.zmean;
    sc.rmean_f[q] = (float)o.rmean;
    if (reset) {
      sc.iters[q] = 0;
      sc.done[q] = (o.rr <= sc.tol2 * sc.bb[q]) ? 1 : 0;
    }
  });
  if (threadIdx.x == 0) *counter = 0u;
}

// per-segment mean removal of the singular problems: x -= mean over the segment (two passes)
__global__ void __launch_bounds__(CG_THREADS)
seg_sum_kernel(const double* __restrict__ x, SegTable t, double* __restrict__ out, double* __restrict__ partial,
               unsigned int* __restrict__ counter) {
  const SegBlock c = chunk_of(t);
  double acc[1] = {0.0};
  for (int i = threadIdx.x; i < c.n; i += CG_THREADS) acc[0] += x[c.off + i];
  double bs[1];
  block_sum_k<double, 1>(acc, bs);
  if (threadIdx.x == 0) partial[blockIdx.x] = bs[0];
  if (!last_block(counter)) return;
  seg_totals<1>(t, partial, [&](int q, const double* tot) { out[q] = tot[0] / (double)t.len[q]; });
  if (threadIdx.x == 0) *counter = 0u;
}
// weighted mean per segment (the mass-weighted pressure mean): out[q] = sum w x / sum w
__global__ void __launch_bounds__(CG_THREADS)
seg_wsum_kernel(const double* __restrict__ x, const double* __restrict__ w, SegTable t, double* __restrict__ out,
                double* __restrict__ partial, unsigned int* __restrict__ counter) {
  const SegBlock c = chunk_of(t);
  double acc[2] = {0.0, 0.0};
  for (int i = threadIdx.x; i < c.n; i += CG_THREADS) {
    const double wi = w[c.doff + i];
    acc[0] += wi * x[c.off + i];
    acc[1] += wi;
  }
  double bs[2];
  block_sum_k<double, 2>(acc, bs);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = bs[0];
    partial[(size_t)t.nblk + blockIdx.x] = bs[1];
  }
  if (!last_block(counter)) return;
  seg_totals<2>(t, partial, [&](int q, const double* tot) { out[q] = tot[1] != 0.0 ? tot[0] / tot[1] : 0.0; });
  if (threadIdx.x == 0) *counter = 0u;
}
// x -= the segment's mean (the mean removal of the singular problems)
__global__ void __launch_bounds__(CG_THREADS)
seg_sub_kernel(double* __restrict__ x, SegTable t, const double* __restrict__ mean) {
  const SegBlock c = chunk_of(t);
  const double m = mean[c.s];
  for (int i = threadIdx.x; i < c.n; i += CG_THREADS) x[c.off + i] -= m;
}

// ---- CG with a general preconditioner (see vec.h) --------------------------------------
template <typename T>
__global__ void __launch_bounds__(CG_THREADS)
seg_rproj_kernel(T* __restrict__ r, SegTable t, CgScalars sc) {
  const SegBlock c = chunk_of(t);
  if (sc.done[c.s] != 0) return;
  const T rm = pick<T>(sc.rmean, sc.rmean_f, c.s);
  T* rs = r + c.off;
  for (int i = threadIdx.x; i < c.n; i += CG_THREADS) rs[i] -= rm;
}

// (r, z) and sum z of the V-cycle-preconditioned CG: the last block forms beta, the
// mean of z (projected systems) and the breakdown flag
template <typename T>
__global__ void __launch_bounds__(CG_THREADS)
seg_rz_kernel(const T* __restrict__ r, const T* __restrict__ z, SegTable t, CgScalars sc,
              double* __restrict__ partial, unsigned int* __restrict__ counter, int init) {
  const SegBlock c = chunk_of(t);
  T acc[2] = {T(0), T(0)};                      // (r, z), sum z
  if (sc.done[c.s] == 0) {
    const T* rs = r + c.off;
    const T* zs = z + c.off;
    for (int i = threadIdx.x; i < c.n; i += CG_THREADS) {
      const T zi = zs[i];
      acc[0] += rs[i] * zi;
      acc[1] += zi;
    }
  }
  double bs[2];
  block_sum_k<T, 2>(acc, bs);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = bs[0];
    partial[(size_t)t.nblk + blockIdx.x] = bs[1];
  }
  if (!last_block(counter)) return;
  seg_totals<2>(t, partial, [&](int q, const double* tot) {
    if (sc.done[q] != 0) return;
    // r is mean-free for projected systems, so (r, z - mean z) = (r, z)
    const double rz = tot[0];
    const double zm = sc.project ? tot[1] / (double)t.len[q] : 0.0;
    sc.rz[q] = rz;
    sc.zmean[q] = zm;
    sc.zmean_f[q] = (float)zm;
    if (!init) {
      const double bt = sc.rz_old[q] != 0.0 ? rz / sc.rz_old[q] : 0.0;
      sc.beta[q] = bt;
      sc.beta_f[q] = (float)bt;
      if (!isfinite(bt)) sc.done[q] = 2;
    }
    if (rz != rz) sc.done[q] = 2;
  });
  if (threadIdx.x == 0) *counter = 0u;
}

// direction of the V-cycle-preconditioned CG: p = z - mean z + beta p
template <typename T>
__global__ void __launch_bounds__(CG_THREADS)
seg_pz_kernel(T* __restrict__ p, const T* __restrict__ z, SegTable t, CgScalars sc, int restart) {
  const SegBlock c = chunk_of(t);
  if (sc.done[c.s] != 0) return;
  const T beta = restart ? T(0) : pick<T>(sc.beta, sc.beta_f, c.s);
  const T zm = pick<T>(sc.zmean, sc.zmean_f, c.s);
  T* ps = p + c.off;
  const T* zs = z + c.off;
  for (int i = threadIdx.x; i < c.n; i += CG_THREADS) ps[i] = restart ? zs[i] - zm : (zs[i] - zm) + beta * ps[i];
}

}  // namespace

template <typename T>
void seg_rproj(T* r, const SegTable& t, const CgScalars& sc, cudaStream_t st) {
  IMEX_COUNTED(seg_rproj_kernel<T><<<t.nblk, CG_THREADS, 0, st>>>(r, t, sc));
}
template <typename T>
void seg_rz(const T* r, const T* z, const SegTable& t, const CgScalars& sc, double* partial, unsigned int* counter,
            int init, cudaStream_t st) {
  IMEX_COUNTED(seg_rz_kernel<T><<<t.nblk, CG_THREADS, 0, st>>>(r, z, t, sc, partial, counter, init));
}
template <typename T>
void seg_pz(T* p, const T* z, const SegTable& t, const CgScalars& sc, int restart, cudaStream_t st) {
  IMEX_COUNTED(seg_pz_kernel<T><<<t.nblk, CG_THREADS, 0, st>>>(p, z, t, sc, restart));
}
template void seg_rproj<float>(float*, const SegTable&, const CgScalars&, cudaStream_t);
template void seg_rproj<double>(double*, const SegTable&, const CgScalars&, cudaStream_t);
template void seg_rz<float>(const float*, const float*, const SegTable&, const CgScalars&, double*, unsigned int*,
                            int, cudaStream_t);
template void seg_rz<double>(const double*, const double*, const SegTable&, const CgScalars&, double*,
                             unsigned int*, int, cudaStream_t);
template void seg_pz<float>(float*, const float*, const SegTable&, const CgScalars&, int, cudaStream_t);
template void seg_pz<double>(double*, const double*, const SegTable&, const CgScalars&, int, cudaStream_t);

template <typename T>
void seg_step_xr(T* x, T* r, const T* p, const T* Ap, const T* dinv, const SegTable& t, const CgScalars& sc,
                 int maxit, double* partial, unsigned int* counter, cudaStream_t st) {
  launch_cg_kernel(seg_xr_kernel<T>, t.nblk, CG_THREADS, 0, st, x, r, p, Ap, dinv, t, sc, partial, counter, maxit);
}
template <typename T>
void seg_step_p(T* p, T* r, const T* dinv, const SegTable& t, const CgScalars& sc, int restart, cudaStream_t st) {
  launch_cg_kernel(seg_p_kernel<T>, t.nblk, CG_THREADS, 0, st, p, r, dinv, t, sc, restart);
}
template <typename T>
void seg_dot(const T* x, const T* y, const SegTable& t, double* out, double* partial, unsigned int* counter,
             cudaStream_t st) {
  IMEX_COUNTED(seg_dot_kernel<T><<<t.nblk, CG_THREADS, 0, st>>>(x, y, t, out, partial, counter));
}
template <typename T>
void seg_pap(const T* p, const T* Ap, const SegTable& t, const CgScalars& sc, double* partial, unsigned int* counter,
             cudaStream_t st) {
  IMEX_COUNTED(seg_pap_kernel<T><<<t.nblk, CG_THREADS, 0, st>>>(p, Ap, t, sc, partial, counter));
}
template <typename T>
void seg_init(const T* r, const T* dinv, const SegTable& t, const CgScalars& sc, double* partial,
              unsigned int* counter, int reset, cudaStream_t st) {
  IMEX_COUNTED(seg_init_kernel<T><<<t.nblk, CG_THREADS, 0, st>>>(r, dinv, t, sc, partial, counter, reset));
}
void seg_remove_mean(double* x, const SegTable& t, double* mean, double* partial, unsigned int* counter,
                     cudaStream_t st) {
  IMEX_COUNTED(seg_sum_kernel<<<t.nblk, CG_THREADS, 0, st>>>(x, t, mean, partial, counter));
  IMEX_COUNTED(seg_sub_kernel<<<t.nblk, CG_THREADS, 0, st>>>(x, t, mean));
}

void seg_remove_wmean(double* x, const double* w, const SegTable& t, double* mean, double* partial,
                      unsigned int* counter, cudaStream_t st) {
  IMEX_COUNTED(seg_wsum_kernel<<<t.nblk, CG_THREADS, 0, st>>>(x, w, t, mean, partial, counter));
  IMEX_COUNTED(seg_sub_kernel<<<t.nblk, CG_THREADS, 0, st>>>(x, t, mean));
}

template void seg_step_xr<double>(double*, double*, const double*, const double*, const double*, const SegTable&,
                                  const CgScalars&, int, double*, unsigned int*, cudaStream_t);
template void seg_step_xr<float>(float*, float*, const float*, const float*, const float*, const SegTable&,
                                 const CgScalars&, int, double*, unsigned int*, cudaStream_t);
template void seg_step_p<double>(double*, double*, const double*, const SegTable&, const CgScalars&, int,
                                 cudaStream_t);
template void seg_step_p<float>(float*, float*, const float*, const SegTable&, const CgScalars&, int, cudaStream_t);
template void seg_dot<double>(const double*, const double*, const SegTable&, double*, double*, unsigned int*,
                              cudaStream_t);
template void seg_dot<float>(const float*, const float*, const SegTable&, double*, double*, unsigned int*,
                             cudaStream_t);
template void seg_pap<double>(const double*, const double*, const SegTable&, const CgScalars&, double*,
                              unsigned int*, cudaStream_t);
template void seg_pap<float>(const float*, const float*, const SegTable&, const CgScalars&, double*, unsigned int*,
                             cudaStream_t);
template void seg_init<double>(const double*, const double*, const SegTable&, const CgScalars&, double*,
                               unsigned int*, int, cudaStream_t);
template void seg_init<float>(const float*, const float*, const SegTable&, const CgScalars&, double*,
                              unsigned int*, int, cudaStream_t);

}  // namespace imex
