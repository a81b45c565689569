// Which pipe executes each kind of operation the float-float kernels use: one small kernel
// per kind repeats it 256 times per thread over 152 x 8 blocks of 256 threads; run under ncu
// with the per-pipe instruction counters (sm__inst_executed_pipe_{fp64,alu,fma,xu}.sum and
// smsp__inst_executed.sum), each count divided by the number of operations gives the
// instructions per operation on each pipe.  Kinds: FP32 FMA, FP32 division and reciprocal,
// int <-> float conversions, integer division, 64-bit shifts, FP32 <-> FP64 round trip,
// FP64 add, the float-float split and join by integer operations and by the FP64 route, the
// compensated float-float dot product term, float-float multiply-add and division, and the
// selection of one of three doubles followed by a conversion.  Prints the time per launch;
// exits non-zero on a CUDA error.  Build: nvcc -O3 -gencode arch=compute_103a,code=sm_103a
// -I paper_2112_04167_gb300/csrc tests/native/fp64_pipe_probe.cu
#include <cstdio>

#include <cuda_runtime.h>

#include "ff.cuh"

using namespace imex;

namespace {
constexpr int IT = 256;
#define PROBE(name, init, body, outexpr)                                                                        \
  __global__ void name(const float* __restrict__ in, const double* __restrict__ ind, float* __restrict__ out, \
                       int nrt) {                                                                             \
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;                                                    \
    init _Pragma("unroll 4") for (int it = 0; it < IT; ++it) { body }                                         \
    out[gid] = outexpr;                                                                                       \
  }
PROBE(p_fma, float a = in[gid]; float s = 0.f;, s = fmaf(a, s, 1.0001f);, s)
PROBE(p_fdiv, float a = in[gid]; float s = 1.f;, s = (s + 1.f) / (a + (float)0);, s)
PROBE(p_i2f, int v = gid; float s = 0.f;, s += (float)(v + it);, s)
PROBE(p_f2i, float a = in[gid]; int v = 0;, v += (int)(a * (float)it);, (float)v)
PROBE(p_idiv, int v = gid; int s = 0;, s += (v + it) / nrt;, (float)s)
PROBE(p_sh64, unsigned long long u = (unsigned long long)gid * 12345ull; unsigned long long s = 0;,
      s += (u << (it & 31)) >> 7; u += s;, (float)(unsigned)s)
PROBE(p_f2f, float a = in[gid]; double d = 0.0;, d = (double)(a + (float)it); a = (float)d * 0.5f;, a)
PROBE(p_dadd, double d = ind[gid]; double s = 0.0;, s = s + d * 1.0000001;, (float)s)
PROBE(p_split_bits, double d = ind[gid]; float s = 0.f;, ff f = ff_split_bits(d); s += f.hi + f.lo; d += 1e-3;, s)
PROBE(p_split_fp64, double d = ind[gid]; float s = 0.f;, ff f = ff_split_fp64(d); s += f.hi + f.lo; d += 1e-3;, s)
PROBE(p_join_bits, float a = in[gid]; double s = 0.0;, s += ff_join_bits(ff(a, a * 1e-9f)); a += 1.f;, (float)s)
PROBE(p_ffdot, float a = in[gid]; ff_dot acc;, acc.add(ff(a, 1e-9f), ff(a + 1.f, 1e-10f)); a += 0.5f;,
      acc.value().hi)
PROBE(p_ffmul, float a = in[gid]; ff s(1.f);, s = s * ff(a, 1e-9f) + ff(0.5f, 0.f);, s.hi)
PROBE(p_ffdiv, float a = in[gid]; ff s(1.f);, s = ff(1.f) / (s + ff(a, 1e-9f));, s.hi)
PROBE(p_frcp, float a = in[gid]; float s = 0.f;, s += 1.f / (a + (float)it);, s)
PROBE(p_dsel, float s = 0.f; double h0 = ind[gid]; double h1 = h0 * 2; double h2 = h0 * 3;,
      const int k = it % 3; double h = k == 0 ? h0 : (k == 1 ? h1 : h2); s += (float)h;, s)
#undef PROBE
typedef void (*Probe)(const float*, const double*, float*, int);
}  // namespace

int main() {
  const int blocks = 152 * 8, threads = 256, n = blocks * threads;
  float *in = nullptr, *out = nullptr;
  double* ind = nullptr;
  if (cudaMalloc(&in, n * sizeof(float)) != cudaSuccess || cudaMalloc(&out, n * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&ind, n * sizeof(double)) != cudaSuccess)
    return 1;
  cudaMemset(in, 0, n * sizeof(float));
  cudaMemset(ind, 0, n * sizeof(double));
  const Probe ps[] = {p_fma, p_fdiv, p_i2f, p_f2i, p_idiv, p_sh64, p_f2f, p_dadd,
                      p_split_bits, p_split_fp64, p_join_bits, p_ffdot, p_ffmul, p_ffdiv, p_frcp, p_dsel};
  const char* names[] = {"fma", "fdiv", "i2f", "f2i", "idiv", "sh64", "f2f", "dadd",
                         "split_bits", "split_fp64", "join_bits", "ffdot", "ffmul", "ffdiv", "frcp", "dsel"};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int i = 0; i < 16; ++i) {
    ps[i]<<<blocks, threads>>>(in, ind, out, 7);
    cudaEventRecord(e0);
    for (int r = 0; r < 5; ++r) ps[i]<<<blocks, threads>>>(in, ind, out, 7);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    std::printf("%-12s %8.2f us per launch (%d operations per thread)\n", names[i], ms * 1000.f / 5.f, IT);
  }
  const cudaError_t err = cudaDeviceSynchronize();
  std::printf("status %s\n", cudaGetErrorString(err));
  cudaFree(in);
  cudaFree(out);
  cudaFree(ind);
  return err == cudaSuccess ? 0 : 1;
}
