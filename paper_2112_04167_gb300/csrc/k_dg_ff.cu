// Float-float instantiations of the DG-SEM first-order operators and the convection term
// (k_dg.cuh): FP64 fields, arithmetic in float-float on the FP32 pipes.
#include "k_dg.cuh"

namespace imex {

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
static void launch_deriv_ff(const Geom& g, const DerivArgs<double>& a, cudaStream_t st) {
  constexpr int ND = ipow(N, D);
  IMEX_COUNTED(dg_deriv_kernel<ff, D, N, double><<<g.ne, ND, 0, st>>>(g, a));
}
template <typename T, int D, int N>
static void launch_conv_ff(const Geom& g, const ConvArgs<double>& a, cudaStream_t st) {
  using S = ConvShape<ff, D, N>;
  smem_limit_once((const void*)dg_conv_kernel<ff, D, N, double>, (int)S::SMEM);
  IMEX_COUNTED(dg_conv_kernel<ff, D, N, double><<<g.ne, S::THREADS, S::SMEM, st>>>(g, a));
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

// nodal DG derivatives with float-float arithmetic on FP64 fields
int dg_deriv_ff(const Geom& g, int N, const DerivArgs<double>& a, cudaStream_t st) {
  using T = double;
  if (g.d == 2) { IMEX_DISPATCH_NV(2, launch_deriv_ff, g, a, st) } else { IMEX_DISPATCH_NV(3, launch_deriv_ff, g, a, st) }
  return 0;
}

// convection with float-float arithmetic on FP64 fields
int dg_conv_ff(const Geom& g, int N, const ConvArgs<double>& a, cudaStream_t st) {
  using T = double;
  if (g.d == 2) { IMEX_DISPATCH_NV(2, launch_conv_ff, g, a, st) } else { IMEX_DISPATCH_NV(3, launch_conv_ff, g, a, st) }
  return 0;
}

}  // namespace imex
