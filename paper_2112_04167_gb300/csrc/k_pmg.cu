// p-multigrid building blocks for the pressure Poisson solves (the preconditioner of the CG
// of Sec. 3.3's solver statement; the paper's own preconditioners are not described there):
//
//   * element-local transfers between the GLL(NF) and GLL(NC) spaces of two levels on the
//     same mesh: prolongation x_f += (I x I x I) x_c with the 1D interpolation matrix
//     I[i][j] = l_j(x_i) (GLL(NC) cardinal polynomials at the GLL(NF) points), and the
//     restriction of a residual, r_c = (I^T x I^T x I^T)(b_f - A x_f), its transpose;
//   * the vector updates of the Chebyshev-accelerated Jacobi smoother (three-term
//     recurrence, Saad, Iterative Methods, Alg. 12.1): the first step
//     r = b - A x0, d = c0 D^{-1} r, x = x0 + d, and each further step
//     r -= A d, d = c1 d + c2 D^{-1} r, x += d.
//
// The transfers are sum-factorised: three (two in 2D) passes of 1D contractions over the
// element's tile staged in shared memory; a block holds EPB elements.  Memory traffic per
// fine node: the restriction reads two vectors and writes (NC/NF)^d of one; the
// prolongation reads (NC/NF)^d of one and reads and writes one.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace imex {
namespace {

constexpr int XF_THREADS = 128;

template <int D, int N>
struct TileN {
  static constexpr int n = ipow(N, D);
};

// elements per block: enough to give every thread about one fine node
template <int D, int NF>
__host__ __device__ constexpr int xfer_epb() {
  return TileN<D, NF>::n >= XF_THREADS ? 1 : XF_THREADS / TileN<D, NF>::n;
}

// MODE 0: xf += P xc (prolongation and add); MODE 1: rc = P^T (bf - axf) (restriction): the
// GLL transfers between p-multigrid levels
template <typename T, int D, int NF, int NC, int MODE>
__global__ void __launch_bounds__(XF_THREADS)
pmg_transfer_kernel(int ne, const T* __restrict__ in0, const T* __restrict__ in1, T* __restrict__ out, Interp1D I,
                    ChebInit<T> ci) {
  constexpr int EPB = xfer_epb<D, NF>();
  constexpr int NFD = TileN<D, NF>::n, NCD = TileN<D, NC>::n;
  constexpr int BIG = NFD;                        // largest intermediate tile
  __shared__ T sa[EPB][BIG];
  __shared__ T sb[EPB][BIG];
  __shared__ T sI[NF * NC];
  for (int i = threadIdx.x; i < NF * NC; i += blockDim.x) sI[i] = (T)I.m[i];
  const int e0 = blockIdx.x * EPB;
  const int nel = min(EPB, ne - e0);
  if (MODE == 1) {
    // fine residual b - A x into the tile
    for (int i = threadIdx.x; i < nel * NFD; i += blockDim.x) {
      const size_t gi = (size_t)e0 * NFD + i;
      sa[i / NFD][i % NFD] = in0[gi] - in1[gi];
    }
  } else {
    for (int i = threadIdx.x; i < nel * NCD; i += blockDim.x) sa[i / NCD][i % NCD] = in0[(size_t)e0 * NCD + i];
  }
  __syncthreads();
  // pass k contracts direction k; tile sizes before the pass: n0 x n1 x n2 with x fastest
  // (restriction maps NF -> NC along k, prolongation NC -> NF)
  constexpr int NI = MODE == 1 ? NF : NC;        // input points along a direction
  constexpr int NO = MODE == 1 ? NC : NF;        // output points
  int ext[3] = {NI, D > 1 ? NI : 1, D > 2 ? NI : 1};
  T(*src)[BIG] = sa;
  T(*dst)[BIG] = sb;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    int oext[3] = {ext[0], ext[1], ext[2]};
    oext[k] = NO;
    const int ocount = oext[0] * oext[1] * oext[2];
    const int stride_in = k == 0 ? 1 : (k == 1 ? ext[0] : ext[0] * ext[1]);
    for (int i = threadIdx.x; i < nel * ocount; i += blockDim.x) {
      const int q = i / ocount;
      const int o = i - q * ocount;
      const int c0 = o % oext[0];
      const int c1 = (o / oext[0]) % oext[1];
      const int c2 = o / (oext[0] * oext[1]);
      const int ck = k == 0 ? c0 : (k == 1 ? c1 : c2);
      // input index with direction k at 0
      const int base = (k == 0 ? 0 : c0) + ext[0] * ((k == 1 ? 0 : c1) + ext[1] * (k == 2 ? 0 : c2));
      T acc = T(0);
#pragma unroll
      for (int j = 0; j < NI; ++j) {
        const T w = MODE == 1 ? sI[j * NC + ck] : sI[ck * NC + j];
        acc += w * src[q][base + j * stride_in];
      }
      dst[q][o] = acc;
    }
    __syncthreads();
    ext[k] = NO;
    T(*t)[BIG] = src;
    src = dst;
    dst = t;
  }
  if (MODE == 1) {
    for (int i = threadIdx.x; i < nel * NCD; i += blockDim.x) {
      const size_t gi = (size_t)e0 * NCD + i;
      const T v = src[i / NCD][i % NCD];
      out[gi] = v;
      if (ci.x) {                                 // the coarse level's first smoothing step
        const T dd = ci.c0 * ci.dinv[gi] * v;
        ci.r[gi] = v;
        ci.d[gi] = dd;
        ci.x[gi] = dd;
      }
    }
  } else {
    for (int i = threadIdx.x; i < nel * NFD; i += blockDim.x) out[(size_t)e0 * NFD + i] += src[i / NFD][i % NFD];
  }
}

template <typename T, int D, int NF, int NC, int MODE>
void launch_transfer(int ne, const T* in0, const T* in1, T* out, const Interp1D& I, const ChebInit<T>& ci,
                     cudaStream_t st) {
  constexpr int EPB = xfer_epb<D, NF>();
  const int blocks = (ne + EPB - 1) / EPB;
  IMEX_COUNTED((pmg_transfer_kernel<T, D, NF, NC, MODE><<<blocks, XF_THREADS, 0, st>>>(ne, in0, in1, out, I, ci)));
}

template <typename T, int D, int MODE>
int transfer_d(int ne, int NF, int NC, const T* in0, const T* in1, T* out, const Interp1D& I, const ChebInit<T>& ci,
               cudaStream_t st) {
#define IMEX_XF(A, B)                                                    \
  if (NF == A && NC == B) {                                              \
    launch_transfer<T, D, A, B, MODE>(ne, in0, in1, out, I, ci, st);     \
    return 0;                                                            \
  }
  IMEX_XF(9, 5) IMEX_XF(8, 4) IMEX_XF(7, 4) IMEX_XF(6, 3) IMEX_XF(5, 3) IMEX_XF(4, 2) IMEX_XF(3, 2)
#undef IMEX_XF
  return -1;
}

// ---- Chebyshev smoother updates (grid-stride, 16-byte accesses where aligned) ----------
template <typename T>
__global__ void __launch_bounds__(256)
cheb_first_kernel(T* __restrict__ x, T* __restrict__ d, T* __restrict__ r, const T* __restrict__ b,
                  const T* __restrict__ ax, const T* __restrict__ dinv, T c0, size_t n, int add) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const T ri = ax ? b[i] - ax[i] : b[i];
    const T di = c0 * dinv[i] * ri;
    r[i] = ri;
    d[i] = di;
    x[i] = add ? x[i] + di : di;
  }
}

// the same from zero for the residual of a singular (projected) one-segment CG system: the
// segment mean is taken off r first and the projected r written back (the CG keeps it)
template <typename T>
__global__ void __launch_bounds__(256)
cheb_first_proj_kernel(T* __restrict__ x, T* __restrict__ d, T* __restrict__ r, T* __restrict__ b,
                       const T* __restrict__ dinv, T c0, const T* __restrict__ mean, const int* __restrict__ done,
                       size_t n) {
  const bool proj = *done == 0;
  const T m = proj ? *mean : T(0);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const T bi = b[i] - m;
    if (proj) b[i] = bi;
    const T di = c0 * dinv[i] * bi;
    r[i] = bi;
    d[i] = di;
    x[i] = di;
  }
}

// a further Chebyshev step: r -= A d, d = c1 d + c2 D^{-1} r, x += d
template <typename T>
__global__ void __launch_bounds__(256)
cheb_next_kernel(T* __restrict__ x, T* __restrict__ d, T* __restrict__ r, const T* __restrict__ ad,
                 const T* __restrict__ dinv, T c1, T c2, size_t n, int last) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const T ri = r[i] - ad[i];
    const T di = c1 * d[i] + c2 * dinv[i] * ri;
    x[i] += di;
    if (!last) {
      r[i] = ri;
      d[i] = di;
    }
  }
}

// y = s a b elementwise (the power iteration of the Chebyshev bounds)
template <typename T>
__global__ void __launch_bounds__(256)
vec_mul_kernel(T* __restrict__ y, const T* __restrict__ a, const T* __restrict__ b, T s, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = s * a[i] * b[i];
}

int grid_for(size_t n) {
  const size_t b = (n + 255) / 256;
  return (int)(b < (size_t)152 * 8 ? (b > 0 ? b : 1) : (size_t)152 * 8);
}

}  // namespace

template <typename T>
int pmg_prolong(int d, int ne, int NF, int NC, const T* xc, T* xf, const Interp1D& I, cudaStream_t st) {
  const ChebInit<T> none{nullptr, nullptr, nullptr, nullptr, T(0)};
  return d == 2 ? transfer_d<T, 2, 0>(ne, NF, NC, xc, nullptr, xf, I, none, st)
                : transfer_d<T, 3, 0>(ne, NF, NC, xc, nullptr, xf, I, none, st);
}
template <typename T>
int pmg_restrict_cheb(int d, int ne, int NF, int NC, const T* bf, const T* axf, T* rc, const Interp1D& I,
                      const ChebInit<T>& ci, cudaStream_t st) {
  return d == 2 ? transfer_d<T, 2, 1>(ne, NF, NC, bf, axf, rc, I, ci, st)
                : transfer_d<T, 3, 1>(ne, NF, NC, bf, axf, rc, I, ci, st);
}
template <typename T>
int pmg_restrict(int d, int ne, int NF, int NC, const T* bf, const T* axf, T* rc, const Interp1D& I,
                 cudaStream_t st) {
  const ChebInit<T> none{nullptr, nullptr, nullptr, nullptr, T(0)};
  return pmg_restrict_cheb<T>(d, ne, NF, NC, bf, axf, rc, I, none, st);
}
template <typename T>
void cheb_first(T* x, T* dv, T* r, const T* b, const T* ax, const T* dinv, double c0, size_t n, int add,
                cudaStream_t st) {
  IMEX_COUNTED(cheb_first_kernel<T><<<grid_for(n), 256, 0, st>>>(x, dv, r, b, ax, dinv, (T)c0, n, add));
}
template <typename T>
void cheb_first_proj(T* x, T* dv, T* r, T* b, const T* dinv, double c0, const T* mean, const int* done, size_t n,
                     cudaStream_t st) {
  IMEX_COUNTED(cheb_first_proj_kernel<T><<<grid_for(n), 256, 0, st>>>(x, dv, r, b, dinv, (T)c0, mean, done, n));
}
template <typename T>
void cheb_next(T* x, T* dv, T* r, const T* ad, const T* dinv, double c1, double c2, size_t n, int last,
               cudaStream_t st) {
  IMEX_COUNTED(cheb_next_kernel<T><<<grid_for(n), 256, 0, st>>>(x, dv, r, ad, dinv, (T)c1, (T)c2, n, last));
}

void vec_mul(double* y, const double* a, const double* b, double s, size_t n, cudaStream_t st) {
  IMEX_COUNTED(vec_mul_kernel<double><<<grid_for(n), 256, 0, st>>>(y, a, b, s, n));
}

template int pmg_prolong<float>(int, int, int, int, const float*, float*, const Interp1D&, cudaStream_t);
template int pmg_prolong<double>(int, int, int, int, const double*, double*, const Interp1D&, cudaStream_t);
template int pmg_restrict<float>(int, int, int, int, const float*, const float*, float*, const Interp1D&,
                                 cudaStream_t);
template int pmg_restrict<double>(int, int, int, int, const double*, const double*, double*, const Interp1D&,
                                  cudaStream_t);
template int pmg_restrict_cheb<float>(int, int, int, int, const float*, const float*, float*, const Interp1D&,
                                      const ChebInit<float>&, cudaStream_t);
template int pmg_restrict_cheb<double>(int, int, int, int, const double*, const double*, double*, const Interp1D&,
                                       const ChebInit<double>&, cudaStream_t);
template void cheb_first_proj<float>(float*, float*, float*, float*, const float*, double, const float*, const int*,
                                     size_t, cudaStream_t);
template void cheb_first_proj<double>(double*, double*, double*, double*, const double*, double, const double*,
                                      const int*, size_t, cudaStream_t);
template void cheb_first<float>(float*, float*, float*, const float*, const float*, const float*, double, size_t, int,
                                cudaStream_t);
template void cheb_first<double>(double*, double*, double*, const double*, const double*, const double*, double,
                                 size_t, int, cudaStream_t);
template void cheb_next<float>(float*, float*, float*, const float*, const float*, double, double, size_t, int,
                               cudaStream_t);
template void cheb_next<double>(double*, double*, double*, const double*, const double*, double, double, size_t,
                                int, cudaStream_t);

}  // namespace imex
