// FP64 and float-float line-owner SIPG kernels (the FP64 form's applies, the float-float
// residual applies of the mixed form) and their constant-memory line operators; the host
// construction of every precision's line operators.
#include "k_sipg_line.cuh"

namespace imex {

__constant__ ConstLine<double> c_line64[IMEX_MAXN + 1];
__constant__ ConstLine<ff> c_lineff[IMEX_MAXN + 1];
template <> __device__ __forceinline__ const ConstLine<double>& cline<double>(int N) { return c_line64[N]; }
template <> __device__ __forceinline__ const ConstLine<ff>& cline<ff>(int N) { return c_lineff[N]; }

bool upload_const_lines_f64(const ConstLine<double>* h64, const ConstLine<ff>* hff) {
  return cudaMemcpyToSymbol(c_line64, h64, sizeof(ConstLine<double>) * (IMEX_MAXN + 1)) == cudaSuccess &&
         cudaMemcpyToSymbol(c_lineff, hff, sizeof(ConstLine<ff>) * (IMEX_MAXN + 1)) == cudaSuccess;
}

int sipg_apply_line(const Geom& g, int N, const SipgArgs<double>& a, cudaStream_t st) {
  return sipg_apply_line_t<double>(g, N, a, st);
}

template <int N, bool XFF>
static void launch_apply_ff(const Geom& g, const SipgArgs<double>& a, cudaStream_t st) {
  using P = Sipg3pShape<ff, N>;
  constexpr size_t sm = sipg3l_smem<ff, N>();
  smem_limit_once((const void*)sipg3p_apply_kernel<ff, N, double, 0, SIPG_EP_ANY, XFF>, (int)sm);
  IMEX_COUNTED((sipg3p_apply_kernel<ff, N, double, 0, SIPG_EP_ANY, XFF>
                <<<(g.ne + P::EPB - 1) / P::EPB, P::THREADS, sm, st>>>(g, a)));
}

namespace {
// x -> float-float pairs (the split of every value, by integer operations)
__global__ void __launch_bounds__(256) to_ff_kernel(const double* __restrict__ x, ff* __restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = ff(x[i]);
}
}  // namespace

int sipg_apply_ff(const Geom& g, int N, const SipgArgs<double>& a, void* scratch, cudaStream_t st) {
  if (g.d != 3 || g.bc[0] || g.bc[1] || g.bc[2] || a.nu || !a.ops || a.gdata || N < 3 || N > 9) return -1;
  SipgArgs<double> aa = a;
  const bool pre = scratch != nullptr;
  if (pre) {
    // the input converted once, so that the apply's loads (each value about seven times:
    // own line and six neighbour lines) take no conversion
    const size_t n = (size_t)a.nsys * (size_t)a.sys_stride;
    const size_t b = (n + 255) / 256;
    IMEX_COUNTED((to_ff_kernel<<<(int)(b < (size_t)152 * 16 ? b : (size_t)152 * 16), 256, 0, st>>>(
        a.x, reinterpret_cast<ff*>(scratch), n)));
    aa.xff = scratch;
  }
  switch (N) {
#define IMEX_FFN(NN)                                                            \
    case NN:                                                                   \
      if (pre) launch_apply_ff<NN, true>(g, aa, st);                           \
      else launch_apply_ff<NN, false>(g, aa, st);                              \
      return 0;
    IMEX_FFN(3) IMEX_FFN(4) IMEX_FFN(5) IMEX_FFN(6) IMEX_FFN(7) IMEX_FFN(8) IMEX_FFN(9)
#undef IMEX_FFN
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
  static ConstLine<ff> hff[IMEX_MAXN + 1];
  for (int N = 2; N <= IMEX_MAXN; ++N) {
    const double* src = reinterpret_cast<const double*>(&h64[N]);
    ff* dst = reinterpret_cast<ff*>(&hff[N]);
    for (size_t i = 0; i < sizeof(ConstLine<double>) / sizeof(double); ++i) dst[i] = ff(src[i]);
  }
  if (upload_const_lines_f32(h32) && upload_const_lines_f64(h64, hff)) g_cline_ready[dev] = true;
}

}  // namespace imex
