// DG-SEM first-order operators of Sec. 3.2 / 3.3 of the paper:
//   * weak divergence B into the pressure test space (Poisson right-hand side,
//     consistent pressure operator),
//   * DG gradient G = M^{-1} B^T of a pressure field (projection v'' = v' - G psi),
//   * nodal DG derivatives with central lifting (grad-div terms F_d2, F_d3),
//   * the over-integrated convection term F_c with local Lax-Friedrichs flux.
// Every kernel works on one element per thread group with its tiles in shared
// memory and sum-factorised 1D contractions.
//
// This unit: the FP64 and FP32 instantiations and their launchers.
#include "k_dg.cuh"

namespace imex {

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

template int dg_div<double>(const Geom&, int, const DivArgs<double>&, cudaStream_t);
template int dg_grad<double>(const Geom&, int, const GradArgs<double>&, cudaStream_t);
template int dg_deriv<double>(const Geom&, int, const DerivArgs<double>&, cudaStream_t);
template int dg_conv<double>(const Geom&, int, const ConvArgs<double>&, cudaStream_t);
template int dg_conv<float>(const Geom&, int, const ConvArgs<float>&, cudaStream_t);
template int dg_div<float>(const Geom&, int, const DivArgs<float>&, cudaStream_t);
template int dg_grad<float>(const Geom&, int, const GradArgs<float>&, cudaStream_t);

}  // namespace imex
