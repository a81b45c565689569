// Launchers of the device kernels (host-callable, C++ linkage inside the library).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "common.cuh"

namespace imex {

// y = alpha M x + beta (A(nu) x - r_b(g)), optionally scaled by M^{-1}; nsys systems
// (vector components) share nu and the geometry.
template <typename T>
struct SipgArgs {
  const T* x;
  T* y;
  int nsys;
  long long sys_stride;
  const T* nu;      // nodal viscosity, or nullptr for nu0
  T nu0;
  const T* gdata;   // Dirichlet data (nodal), or nullptr
  long long g_stride;
  T alpha, beta;
  int minv;
  const LineOps<T>* ops;   // line operators of this space (constant-viscosity fast path), or nullptr
  // optional fused CG dot (x, y) per system: block partials, completion counter, result
  double* dot_partial;     // [nsys][gridDim.x]
  unsigned int* dot_counter;
  double* dot_out;         // [nsys]
  // optional CG step length from the fused dot: alpha[s] = cg_rz[s] / dot_out[s] in FP64 and
  // FP32; a non-finite step marks a running system (cg_done[s] == 0) as broken down (2)
  const double* cg_rz;
  double* cg_alpha;
  float* cg_alpha_f;
  int* cg_done;
  // deferred form of the fused dot: the blocks only leave their partials, block 0 stores the
  // number of blocks in *dot_nblk, and the next kernel (the CG step) adds them itself -- no
  // completion counter and no last-block reduction at the end of the apply
  int dot_defer;
  unsigned int* dot_nblk;
  // batch groups in a CG loop: elements whose system has stopped are skipped; system s of an
  // element of instance i is segment s * done_ninst + i of done_flags (nullptr: no skipping)
  const int* done_flags;
  int done_ninst;
  // batched meshes: take the constant viscosity from each element's instance instead of nu0
  // (inst_nu), and multiply beta by the instance's time step (inst_dt)
  int inst_nu;
  int inst_dt;
  // launch shape chosen by the tuner for the periodic constant-viscosity kernels (elements
  // per block: 0 the default, 1 half, 2 twice, 3 one more; other kernels ignore it)
  int variant;
  // Chebyshev smoother steps fused into the apply (p-multigrid, constant-viscosity kernels),
  // node by node instead of y = A x:
  //   cheb = 1: r -= A x, d' = c1 x + c2 D^{-1} r, s += d' (x is the previous direction; d'
  //             goes to a buffer other than x); ch_last: only s is stored; ch_addx: s += x + d'
  //             (the first step's direction, not yet added to s)
  //   cheb = 2: the first step from the current s = x: r = b - A x, d = c1 D^{-1} r (s is left
  //             for the next step to add d to, with ch_addx)
  //   cheb = 0: the plain apply.
  int cheb;
  int ch_last;
  int ch_addx;
  T* ch_r;
  T* ch_dout;
  T* ch_s;
  const T* ch_dinv;
  const T* ch_b;
  T ch_c1, ch_c2;
  // float-float applies: the input x converted to float-float pairs (sipg_apply_ff)
  const void* xff;
};

template <typename T>
__device__ __forceinline__ T sipg_nu0(const SipgArgs<T>& a, const Geom& gl) {
  return a.inst_nu ? geom_nu0<T>(gl) : a.nu0;
}
template <typename T>
__device__ __forceinline__ T sipg_beta(const SipgArgs<T>& a, const Geom& gl) {
  return a.inst_dt ? a.beta * geom_dt<T>(gl) : a.beta;
}

template <typename T> int sipg_apply(const Geom& g, int N, const SipgArgs<T>& a, cudaStream_t st);
// the periodic 3D constant-viscosity apply on FP64 fields with float-float arithmetic (about
// 48 significant bits on the FP32 pipes); -1 for any other case (nothing launched)
// scratch: room for nsys * sys_stride float-float pairs (8 bytes each) to hold the input
// converted beforehand, or nullptr (the kernel converts as it loads)
int sipg_apply_ff(const Geom& g, int N, const SipgArgs<double>& a, void* scratch, cudaStream_t st);
// constant-memory line operators of the periodic fast path (once per device)
void init_const_lines(const Tables<double>& t);
template <typename T> int sipg_diag(const Geom& g, int N, const SipgArgs<T>& a, cudaStream_t st);

// Weak divergence into the pressure test space (Nv velocity points, Nv-1 pressure points):
//   b = coef * ( B v - int_{dOmega} (n . w) q ),   w = wdata (mode 1), w = v (mode 2), none (mode 0)
// v, wdata: d components with stride v_stride.
template <typename T>
struct DivArgs {
  const T* v;
  long long v_stride;
  const T* wdata;
  int mode;
  T coef;
  T* b;
};
template <typename T> int dg_div(const Geom& g, int Nv, const DivArgs<T>& a, cudaStream_t st);

// DG gradient of a pressure field into the velocity space, out_k = base_k + coef * (M^{-1} B^T psi)_k.
template <typename T>
struct GradArgs {
  const T* psi;
  const T* base;     // may be nullptr (then 0)
  long long stride;  // component stride of base / out
  T coef;
  T* out;
};
template <typename T> int dg_grad(const Geom& g, int Nv, const GradArgs<T>& a, cudaStream_t st);

// Nodal DG derivatives (central flux inside, own trace at domain boundaries):
//   op 0: out = nu * sum_k D_k in_k                     (in: d fields, out: 1 field)
//   op 1: out_c = coef * D_c in_0                      (in: 1 field,  out: d fields)
//   op 2: out_{c*d+k} = nu * D_c in_k                  (in: d fields, out: d*d fields)
//   op 3: out_c = out_c + coef * sum_k D_k in_{c*d+k}  (in: d*d fields, out: d fields, accumulates)
template <typename T>
struct DerivArgs {
  int op;
  const T* in;
  long long stride;
  const T* nu;
  T nu0;
  T coef;
  T* out;
  int inst_nu;     // batched meshes: constant viscosity of each element's instance
};
template <typename T> int dg_deriv(const Geom& g, int N, const DerivArgs<T>& a, cudaStream_t st);
// the same with float-float arithmetic on FP64 fields
int dg_deriv_ff(const Geom& g, int N, const DerivArgs<double>& a, cudaStream_t st);

// Convection F_c = M^{-1} [ sum_K int (v v) : grad w - sum_F int H . w ], LLF flux, Gauss
// over-integration; vb: Dirichlet data (nodal), out = coef * F_c.
template <typename T>
struct ConvArgs {
  const T* v;
  long long stride;
  const T* vb;
  T coef;
  T* out;
};
template <typename T> int dg_conv(const Geom& g, int N, const ConvArgs<T>& a, cudaStream_t st);
// the same on FP64 fields with float-float arithmetic (about 48 significant bits) on the FP32 pipes
int dg_conv_ff(const Geom& g, int N, const ConvArgs<double>& a, cudaStream_t st);
int dg_div_ff(const Geom& g, int N, const DivArgs<double>& a, cudaStream_t st);
int dg_grad_ff(const Geom& g, int N, const GradArgs<double>& a, cudaStream_t st);

// ---- vector kernels (k_vec.cu) ------------------------------------------------
#define IMEX_MAXTERMS 16
struct LinComb {
  const double* x[IMEX_MAXTERMS];
  double c[IMEX_MAXTERMS];
  int nterms;
  // batched meshes: terms j >= nfixed are also multiplied by the time step of the element
  // holding entry i, edt[(i mod cstride) / nd] (edt == nullptr: no such factor)
  const double* edt;
  long long cstride;
  int nd;
  int nfixed;
};
// out[i] = c0 * x0[i] + sum c_j x_j[i]   (x0 may be out itself)
void lincomb(double* out, const LinComb& lc, size_t n, cudaStream_t st);

// partial sums for deterministic dots: two-level reduction into dst[0..nsys)
int dot_batched(const double* x, const double* y, size_t n, long long stride, int nsys,
                double* partial, int nblocks, double* dst, cudaStream_t st);
int dot_batched_f(const float* x, const float* y, size_t n, long long stride, int nsys,
                  double* partial, int nblocks, double* dst, cudaStream_t st);
int reduce_sum(const double* x, size_t n, double* partial, int nblocks, double* dst, cudaStream_t st);
int reduce_max_abs(const double* x, size_t n, double* partial, int nblocks, double* dst,
                   cudaStream_t st);

// x[i] -= (sum_j w_j x_j) / (sum_j w_j) for a precomputed scalar pair in dev memory
void subtract_scaled_scalar(double* x, size_t n, const double* num, const double* den,
                            const double* w, cudaStream_t st);

void convert_d2f(const double* in, float* out, size_t n, cudaStream_t st);
void axpy_f2d(double* y, const float* x, size_t n, cudaStream_t st);

template <typename T>
void reciprocal(T* d, size_t n, cudaStream_t st);
// over the nsys components (stride n) of x and kx = K x: mode 0: y = m x + gamma dt_e kx;
// mode 1: y = -kx / m  (dt_e = edt[i / nd], or 1 when edt is null)
void kx_combine(double* y, const double* x, const double* m, const double* kx, double gamma, const double* edt,
                long long nd, size_t n, int nsys, int mode, cudaStream_t st);
// d = 1 / (m + gamma dt_e k) over n nodes, dt_e = edt[i / nd] (or 1 when edt is null)
void helm_diag(double* d, const double* m, const double* k, double gamma, const double* edt, long long nd, size_t n,
               cudaStream_t st);

// ---- p-multigrid (k_pmg.cu) -----------------------------------------------------
// 1D interpolation between two levels, m[i * NC + j] = l_j(x_i) (NF x NC)
struct Interp1D {
  double m[IMEX_MAXN * IMEX_MAXN];
};
// xf += P xc over ne elements (element-local tensor-product interpolation NC -> NF points);
// -1 for an unsupported (NF, NC) pair (nothing launched)
template <typename T>
int pmg_prolong(int d, int ne, int NF, int NC, const T* xc, T* xf, const Interp1D& I, cudaStream_t st);
// rc = P^T (bf - axf): restriction of the fine residual
template <typename T>
int pmg_restrict(int d, int ne, int NF, int NC, const T* bf, const T* axf, T* rc, const Interp1D& I, cudaStream_t st);
// the same, with the coarse level's first Chebyshev step from zero fused into the output:
// r = rc, d = x = c0 D^{-1} rc
// The coarsest p-multigrid level (N = 2, 3D, every face periodic, one mesh instance, FP32)
// on one thread-block cluster: pmg_cluster_prepare decides once per device and element
// count whether the GPU can run it (call it outside stream capture); pmg_coarse_cluster then
// runs all `steps` Chebyshev steps from x = 0 for A x = b on [lmax / ratio, lmax] in one
// launch, or returns -1 (nothing launched) when it was not prepared for this mesh
bool pmg_cluster_prepare(const Geom& g, int N);
int pmg_coarse_cluster(const Geom& g, int N, const float* b, const float* dinv, float* x, int steps, double lmax,
                       double ratio, cudaStream_t st);
template <typename T>
struct ChebInit {
  T* x;
  T* d;
  T* r;
  const T* dinv;
  T c0;
};
template <typename T>
int pmg_restrict_cheb(int d, int ne, int NF, int NC, const T* bf, const T* axf, T* rc, const Interp1D& I,
                      const ChebInit<T>& ci, cudaStream_t st);
// Chebyshev smoother steps: first  r = b - ax (ax may be null: r = b), d = c0 D^{-1} r,
// x = (add ? x : 0) + d;  next  r -= ad, d = c1 d + c2 D^{-1} r, x += d (last: r, d not stored)
template <typename T>
void cheb_first(T* x, T* d, T* r, const T* b, const T* ax, const T* dinv, double c0, size_t n, int add,
                cudaStream_t st);
// the first step from zero for a projected one-segment CG residual b (its mean *mean taken
// off and the projected b written back unless *done)
template <typename T>
void cheb_first_proj(T* x, T* d, T* r, T* b, const T* dinv, double c0, const T* mean, const int* done, size_t n,
                     cudaStream_t st);
template <typename T>
void cheb_next(T* x, T* d, T* r, const T* ad, const T* dinv, double c1, double c2, size_t n, int last,
               cudaStream_t st);
// y = s a b elementwise
void vec_mul(double* y, const double* a, const double* b, double s, size_t n, cudaStream_t st);

// ---- flow statistics (k_diag.cu) ------------------------------------------------
// per element e: out[e] = int_e nu grad v : grad v (broken gradient, GLL quadrature); nu:
// nodal viscosity or nullptr for nu0.  -1 for an unsupported (d, N)
int dissipation_elems(const Geom& g, int N, const double* v, long long stride, const double* nu, double nu0,
                      double* out, cudaStream_t st);
// E[0..kmax) of v on an M^d regular grid (M a power of two, 2..1024); grid: d * M^d complex
// scratch, part: nbin_blocks * kmax scratch; vol: |Omega|.  -1 for unsupported arguments
int energy_spectrum(const Geom& g, int N, const double* v, long long stride, int M, int kmax, double vol,
                    double2* grid, double* part, int nbin_blocks, double* E, cudaStream_t st);

// ---- divergence / mass-flux stabilisation (k_stab.cu) ---------------------------
// speed[e] = |mass-weighted mean velocity of element e|
int stab_speed(const Geom& g, int N, const double* v, long long stride, double* speed, cudaStream_t st);
// y = (M + A_D + A_C) u for the d components (stride apart) with the element speeds
int stab_apply(const Geom& g, int N, const double* u, double* y, long long stride, const double* speed, double zd,
               double zc, double dt, cudaStream_t st);

// ---- pointwise fields (k_fields.cu) --------------------------------------------
// what: 0 velocity of a closed-form flow (d components), 1 viscosity (1 component),
//       2 forcing (d components).  kind / p: the flow, viscosity law or forcing and its
//       parameters (imex.h).  v: velocity for velocity-dependent viscosity.
struct FieldSpec {
  int kind;
  double p[8];
};
int eval_field(const Geom& g, int N, int what, const FieldSpec& fs, double t, const double* v,
               long long stride, double* out, cudaStream_t st);

}  // namespace imex
