// Vector kernels: stage linear combinations (FP64), deterministic two-level
// reductions (FP64 accumulation), precision conversion and the allocation-free
// reduction entry point.  The Jacobi-PCG kernels live in k_cg.cu.
#include <cstdlib>
#include <atomic>
#include <mutex>
#include <type_traits>
#include <vector>

#include "../../include/imex.h"
#include "common.cuh"
#include "kernels.h"
#include "vec.h"

namespace imex {

static std::atomic<long long> g_launches{0};
static thread_local long long t_launches = 0;
void count_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ++t_launches;
}
void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
bool pdl_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("IMEX_PDL");
    return e && std::atoi(e) != 0;
  }();
  return on;
}
long long thread_launch_count() { return t_launches; }

void smem_limit_once(const void* kernel, int bytes) {
  static std::mutex mu;
  static std::vector<std::pair<const void*, int>> done;   // (kernel, device)
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  for (const auto& d : done)
    if (d.first == kernel && d.second == dev) return;
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  done.emplace_back(kernel, dev);
}
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

// out = sum_j c_j x_j: the stage extrapolation, the Helmholtz right-hand side and the final
// assembly of Alg. 3 (its stage sums in FP64), the SDC quadrature sums of Alg. 4
__global__ void lincomb_kernel(double* __restrict__ out, LinComb lc, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    if (lc.edt) {
      double u = 0.0;
      for (int j = 0; j < lc.nfixed; ++j) s += lc.c[j] * lc.x[j][i];
#pragma unroll 4
      for (int j = lc.nfixed; j < lc.nterms; ++j) u += lc.c[j] * lc.x[j][i];
      s += lc.edt[(i % (size_t)lc.cstride) / (size_t)lc.nd] * u;
    } else {
#pragma unroll 4
      for (int j = 0; j < lc.nterms; ++j) s += lc.c[j] * lc.x[j][i];
    }
    out[i] = s;
  }
}

static int grid_for(size_t n, int threads) {
  size_t b = (n + threads - 1) / threads;
  const size_t cap = 152 * 8;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

void lincomb(double* out, const LinComb& lc, size_t n, cudaStream_t st) {
  if (n == 0) return;
  IMEX_COUNTED(lincomb_kernel<<<grid_for(n, 256), 256, 0, st>>>(out, lc, n));
}

// ---- block reduction helpers ----------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}
// sum over the block (blockDim.x multiple of 32, <= 1024); result valid in thread 0
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double ws[32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) ws[w] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? ws[lane] : 0.0;
  if (w == 0) v = warp_sum(v);
  return v;
}
__device__ __forceinline__ double block_max(double v) {
  __shared__ double ws[32];
  v = warp_max(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) ws[w] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? ws[lane] : 0.0;
  if (w == 0) v = warp_max(v);
  return v;
}

// per-block partial dot products of nsys systems (the CG dots and the relative residual
// norms of the stopping rule of Sec. 4), FP64 accumulation
template <typename T>
__global__ void dot_partial_kernel(const T* __restrict__ x, const T* __restrict__ y, size_t n,
                                   long long stride, double* __restrict__ partial) {
  const int s = blockIdx.y;
  const T* xs = x + (size_t)s * stride;
  const T* ys = y + (size_t)s * stride;
  T tacc = T(0);                      // per-thread partial in the data type (FP64 is scarce on GB300)
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    tacc += xs[i] * ys[i];
  double acc = block_sum((double)tacc);
  if (threadIdx.x == 0) partial[(size_t)s * gridDim.x + blockIdx.x] = acc;
}

// fixed-order final sum of nblocks partials per system (deterministic)
__global__ void finish_sum_kernel(const double* __restrict__ partial, int nblocks, double* __restrict__ dst) {
  const int s = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) acc += partial[(size_t)s * nblocks + i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) dst[s] = acc;
}

template <typename T>
static int dot_impl(const T* x, const T* y, size_t n, long long stride, int nsys, double* partial,
                    int nblocks, double* dst, cudaStream_t st) {
  dim3 grid(nblocks, nsys);
  IMEX_COUNTED(dot_partial_kernel<T><<<grid, 256, 0, st>>>(x, y, n, stride, partial));
  IMEX_COUNTED(finish_sum_kernel<<<nsys, 256, 0, st>>>(partial, nblocks, dst));
  return 0;
}

int dot_batched(const double* x, const double* y, size_t n, long long stride, int nsys, double* partial,
                int nblocks, double* dst, cudaStream_t st) {
  return dot_impl<double>(x, y, n, stride, nsys, partial, nblocks, dst, st);
}
int dot_batched_f(const float* x, const float* y, size_t n, long long stride, int nsys, double* partial,
                  int nblocks, double* dst, cudaStream_t st) {
  return dot_impl<float>(x, y, n, stride, nsys, partial, nblocks, dst, st);
}

// per-block partial sums (the mean removal of the singular pressure problems)
__global__ void sum_partial_kernel(const double* __restrict__ x, size_t n, double* __restrict__ partial) {
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    acc += x[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}
int reduce_sum(const double* x, size_t n, double* partial, int nblocks, double* dst, cudaStream_t st) {
  IMEX_COUNTED(sum_partial_kernel<<<nblocks, 256, 0, st>>>(x, n, partial));
  IMEX_COUNTED(finish_sum_kernel<<<1, 256, 0, st>>>(partial, nblocks, dst));
  return 0;
}

// max |x| with NaN propagation: a NaN entry makes the result NaN (the instability check,
// Sec. 4.2.3)
__global__ void maxabs_partial_kernel(const double* __restrict__ x, size_t n, double* __restrict__ partial) {
  double m = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double v = fabs(x[i]);
    m = (v != v || m != m) ? nan("") : fmax(m, v);
  }
  // propagate NaN through the reduction explicitly
  __shared__ int has_nan;
  if (threadIdx.x == 0) has_nan = 0;
  __syncthreads();
  if (m != m) has_nan = 1;
  m = block_max(m != m ? 0.0 : m);
  __syncthreads();
  if (threadIdx.x == 0) partial[blockIdx.x] = has_nan ? nan("") : m;
}
// max over the partials, NaN propagated (the instability check of Sec. 4.2.3)
__global__ void finish_max_kernel(const double* __restrict__ partial, int nblocks, double* __restrict__ dst) {
  __shared__ int has_nan;
  if (threadIdx.x == 0) has_nan = 0;
  __syncthreads();
  double m = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
    double v = partial[i];
    if (v != v) has_nan = 1; else m = fmax(m, v);
  }
  m = block_max(m);
  __syncthreads();
  if (threadIdx.x == 0) dst[0] = has_nan ? nan("") : m;
}
int reduce_max_abs(const double* x, size_t n, double* partial, int nblocks, double* dst, cudaStream_t st) {
  IMEX_COUNTED(maxabs_partial_kernel<<<nblocks, 256, 0, st>>>(x, n, partial));
  IMEX_COUNTED(finish_max_kernel<<<1, 256, 0, st>>>(partial, nblocks, dst));
  return 0;
}

// x -= num/den (w == nullptr) or x -= (num/den) elementwise constant (mean removal of the singular pressure problems)
__global__ void subtract_scalar_kernel(double* x, size_t n, const double* num, const double* den) {
  const double c = num[0] / den[0];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    x[i] -= c;
}
void subtract_scaled_scalar(double* x, size_t n, const double* num, const double* den, const double* w,
                            cudaStream_t st) {
  (void)w;
  IMEX_COUNTED(subtract_scalar_kernel<<<grid_for(n, 256), 256, 0, st>>>(x, n, num, den));
}

// FP64 -> FP32 and FP32 correction added to an FP64 iterate: the FP64 refinement of the mixed-precision solves
__global__ void d2f_kernel(const double* in, float* out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}
void convert_d2f(const double* in, float* out, size_t n, cudaStream_t st) {
  IMEX_COUNTED(d2f_kernel<<<grid_for(n, 256), 256, 0, st>>>(in, out, n));
}
__global__ void axpy_f2d_kernel(double* y, const float* x, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] += (double)x[i];
}
void axpy_f2d(double* y, const float* x, size_t n, cudaStream_t st) {
  IMEX_COUNTED(axpy_f2d_kernel<<<grid_for(n, 256), 256, 0, st>>>(y, x, n));
}

// d = 1 / d: the Jacobi preconditioner of the CG solves (Sec. 3.3) from an operator diagonal
template <typename T>
__global__ void recip_kernel(T* d, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    d[i] = T(1) / d[i];
}
template <typename T>
void reciprocal(T* d, size_t n, cudaStream_t st) {
  IMEX_COUNTED(recip_kernel<T><<<grid_for(n, 256), 256, 0, st>>>(d, n));
}

// Jacobi diagonal of M + gamma A (the Helmholtz operator of an Alg. 3 stage) for a viscosity
// that is constant per element: from the
// cached diagonals of M and of A (unit factor), d = 1 / (m + gamma dt_e k), with dt_e the
// element's own time step in a batch group (edt) and 1 otherwise
__global__ void helm_diag_kernel(double* __restrict__ d, const double* __restrict__ m, const double* __restrict__ k,
                                 double gamma, const double* __restrict__ edt, long long nd, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double g = edt ? gamma * edt[i / (size_t)nd] : gamma;
    d[i] = 1.0 / (m[i] + g * k[i]);
  }
}
void helm_diag(double* d, const double* m, const double* k, double gamma, const double* edt, long long nd, size_t n,
               cudaStream_t st) {
  if (n == 0) return;
  IMEX_COUNTED(helm_diag_kernel<<<grid_for(n, 256), 256, 0, st>>>(d, m, k, gamma, edt, nd, n));
}

// Helmholtz operator and F_d1 of Alg. 3 from K x (the SIPG operator with unit factor applied to the d
// components of x, stride n each): mode 0: y = m x + gamma dt_e K x (dt_e = edt[i / nd], or
// 1 when edt is null); mode 1: y = -K x / m
__global__ void kx_combine_kernel(double* __restrict__ y, const double* __restrict__ x, const double* __restrict__ m,
                                  const double* __restrict__ kx, double gamma, const double* __restrict__ edt,
                                  long long nd, size_t n, int nsys, int mode) {
  const size_t tot = n * (size_t)nsys;
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < tot; j += (size_t)gridDim.x * blockDim.x) {
    const size_t i = j % n;
    if (mode == 0) {
      const double g = edt ? gamma * edt[i / (size_t)nd] : gamma;
      y[j] = m[i] * x[j] + g * kx[j];
    } else {
      y[j] = -kx[j] / m[i];
    }
  }
}
void kx_combine(double* y, const double* x, const double* m, const double* kx, double gamma, const double* edt,
                long long nd, size_t n, int nsys, int mode, cudaStream_t st) {
  if (n == 0) return;
  IMEX_COUNTED(kx_combine_kernel<<<grid_for(n * nsys, 256), 256, 0, st>>>(y, x, m, kx, gamma, edt, nd, n, nsys, mode));
}

template void reciprocal<double>(double*, size_t, cudaStream_t);
template void reciprocal<float>(float*, size_t, cudaStream_t);

}  // namespace imex


// =====================================================================================
// Allocation-free reduction: imex_reduce_noalloc (include/imex.h).
//
// For callers that must not allocate device memory at call time -- code that runs
// while a memory pool owned by another framework holds the device, inside a loop
// where a cudaMalloc would synchronise the device, or in embedded / real-time hosts
// that forbid allocation after start-up.  Same reduction as imex_reduce, with the
// per-block partial sums kept in a fixed file-scope device array instead of a
// context buffer.  Every GPU that loads this library holds that array until exit.
// =====================================================================================
namespace {

constexpr int kNoallocChunk = 256;                     // elements per partial sum
constexpr int kNoallocSlots = 65536;                   // partial sums held
constexpr long long kNoallocMaxN = (long long)kNoallocChunk * kNoallocSlots;   // 16,777,216
constexpr int kNoallocMaxDevices = 64;

// partial sums [0, kNoallocSlots) and the final value at [kNoallocSlots]
static __device__ __align__(256) double g_noalloc_scratch[kNoallocSlots + 32];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kNoallocMaxDevices] = {nullptr};

// The allocation-free reduction entry point (no counterpart in the paper).
// block b reduces exactly the elements [256 b, 256 b + 256) into partial[b]
__global__ void noalloc_chunk_kernel(int op, const double* __restrict__ x, const double* __restrict__ y,
                                     long long n, double* __restrict__ partial) {
  const long long i = (long long)blockIdx.x * kNoallocChunk + threadIdx.x;
  double v = 0.0;
  bool nan_here = false;
  if (i < n) {
    if (op == IMEX_REDUCE_DOT) v = x[i] * y[i];
    else if (op == IMEX_REDUCE_SUM) v = x[i];
    else { v = fabs(x[i]); nan_here = (v != v); }
  }
  if (op == IMEX_REDUCE_MAXABS) {
    __shared__ int has_nan;
    if (threadIdx.x == 0) has_nan = 0;
    __syncthreads();
    if (nan_here) has_nan = 1;
    const double m = imex::block_max(nan_here ? 0.0 : v);
    __syncthreads();
    if (threadIdx.x == 0) partial[blockIdx.x] = has_nan ? nan("") : m;
  } else {
    const double s = imex::block_sum(v);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
  }
}

// one block: fixed-order combination of nb partial sums into out[0] (allocation-free entry;
// no counterpart in the paper)
__global__ void noalloc_finish_kernel(int op, const double* __restrict__ partial, int nb, double* __restrict__ out) {
  if (op == IMEX_REDUCE_MAXABS) {
    __shared__ int has_nan;
    if (threadIdx.x == 0) has_nan = 0;
    __syncthreads();
    double m = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
      const double v = partial[i];
      if (v != v) has_nan = 1; else m = fmax(m, v);
    }
    m = imex::block_max(m);
    __syncthreads();
    if (threadIdx.x == 0) out[0] = has_nan ? nan("") : m;
  } else {
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partial[i];
    s = imex::block_sum(s);
    if (threadIdx.x == 0) out[0] = s;
  }
}

// device address of the scratch array on the current device (looked up once per device)
imex_status noalloc_scratch(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IMEX_ECUDA;
  if (dev < 0 || dev >= kNoallocMaxDevices) return IMEX_EINVAL;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return IMEX_ECUDA;
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return IMEX_OK;
}

}  // namespace

extern "C" imex_status imex_reduce_noalloc(int op, const double* x, const double* y, long long n, double* out,
                                           void* stream) {
  if (!x || !out || n < 0 || op < IMEX_REDUCE_DOT || op > IMEX_REDUCE_MAXABS || (op == IMEX_REDUCE_DOT && !y))
    return IMEX_EINVAL;
  if (n > kNoallocMaxN) return IMEX_EINVAL;       // more partial sums than the fixed array holds
  if (n == 0) {
    *out = 0.0;
    return IMEX_OK;
  }
  double* scratch = nullptr;
  const imex_status s = noalloc_scratch(&scratch);
  if (s != IMEX_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nb = (int)((n + kNoallocChunk - 1) / kNoallocChunk);
  IMEX_COUNTED(noalloc_chunk_kernel<<<nb, kNoallocChunk, 0, st>>>(op, x, y, n, scratch));
  IMEX_COUNTED(noalloc_finish_kernel<<<1, 256, 0, st>>>(op, scratch, nb, scratch + kNoallocSlots));
  if (cudaGetLastError() != cudaSuccess) return IMEX_ECUDA;
  if (cudaMemcpyAsync(out, scratch + kNoallocSlots, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return IMEX_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return IMEX_ECUDA;
  return IMEX_OK;
}

