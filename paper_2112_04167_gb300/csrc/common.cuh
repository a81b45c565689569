// Common definitions of the GB300 (sm_103a) DG-SEM kernels.
//
// Discretisation (Sec. 3.3 of the paper): Cartesian hexahedral / quadrilateral
// elements, tensor-product Lagrange bases on Gauss-Lobatto-Legendre points,
// velocity degree P (N = P+1 points per direction), pressure degree P-1.
// Storage: element-contiguous, nodes lexicographic with x fastest; a vector
// field stores its d components one after the other.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define IMEX_MAXN 9                        // nodes per direction: P <= 8
#define IMEX_MAXQ 14                       // Gauss points for over-integration, ceil(3*9/2)
#define IMEX_WARP 32

namespace imex {

// One instance of a batched mesh: its elements are [e0, e0 + ne) of the union, its own
// Cartesian box, element counts and sizes, constant viscosity, time step and current time,
// and the parameters of its analytic viscosity model, boundary data and forcing.
struct InstGeom {
  int e0;
  int ne;
  int n[3];
  double lo[3];
  double h[3];
  float hf[3];
  double nu0;
  float nu0f;
  double dt;
  float dtf;
  double t;
  double nu_p[8], bc_p[8], f_p[8];
};

// Mesh geometry as seen by every kernel (passed by value).  A batched mesh is the union of
// several instances of the same space (d, N): inst / elem_inst give each element's instance
// and local_geom() the element's own view of it.
struct Geom {
  int d;                 // 2 or 3
  int ne;                // number of elements
  int n[3];              // elements per direction (n[2] = 1 in 2D)
  int bc[3];             // 0 periodic, 1 Dirichlet, 2 homogeneous Neumann (per direction)
  double lo[3];
  double h[3];           // element sizes
  float hf[3];           // the same in FP32 (FP32 kernels take no FP64 conversion per thread)
  const void* tab64;     // device Tables<double>
  const void* tab32;     // device Tables<float>
  const InstGeom* inst;  // batched mesh: per-instance geometry, or nullptr
  const int* elem_inst;  // batched mesh: instance of each element
  // set by local_geom for the element at hand (defaults for a single instance)
  int e0;                // first element of the instance
  double inu0;           // the instance's constant viscosity
  float inu0f;
  double idt;            // the instance's time step
  float idtf;
  // element neighbours across the 2d faces ([element][2d], face 2k + side, side 1 the upper
  // one; -1 on a domain boundary), built on the host for the context's layout, or nullptr
  const int* nbr = nullptr;
};

// per-direction geometry by selects rather than array indexing, so that a Geom held by a
// thread stays in registers when k is not a compile-time constant
template <typename T> __host__ __device__ __forceinline__ T geom_h(const Geom& g, int k);
template <> __host__ __device__ __forceinline__ double geom_h<double>(const Geom& g, int k) {
  return k == 0 ? g.h[0] : (k == 1 ? g.h[1] : g.h[2]);
}
template <> __host__ __device__ __forceinline__ float geom_h<float>(const Geom& g, int k) {
  return k == 0 ? g.hf[0] : (k == 1 ? g.hf[1] : g.hf[2]);
}
__host__ __device__ __forceinline__ int geom_n(const Geom& g, int k) {
  return k == 0 ? g.n[0] : (k == 1 ? g.n[1] : g.n[2]);
}
__host__ __device__ __forceinline__ int geom_bc(const Geom& g, int k) {
  return k == 0 ? g.bc[0] : (k == 1 ? g.bc[1] : g.bc[2]);
}

// 1D tables per number of points N (index N, 2..IMEX_MAXN), in FP64 and FP32.
//   x, w      : GLL points / weights
//   D         : D[i*N+j] = l_j'(x_i)
//   Ipv       : pressure basis (N-1 points) at the N velocity points, [i*(N-1)+a]
//   Gpv       : its derivative there
//   IG, DG    : velocity basis and its derivative at the Q(N) Gauss points, [g*N+j]
//   gw        : Gauss weights
template <typename T>
struct Tables {
  T x[IMEX_MAXN + 1][IMEX_MAXN];
  T w[IMEX_MAXN + 1][IMEX_MAXN];
  T D[IMEX_MAXN + 1][IMEX_MAXN * IMEX_MAXN];
  T Ipv[IMEX_MAXN + 1][IMEX_MAXN * IMEX_MAXN];
  T Gpv[IMEX_MAXN + 1][IMEX_MAXN * IMEX_MAXN];
  T IG[IMEX_MAXN + 1][IMEX_MAXQ * IMEX_MAXN];
  T DG[IMEX_MAXN + 1][IMEX_MAXQ * IMEX_MAXN];
  T gw[IMEX_MAXN + 1][IMEX_MAXQ];
  int Q[IMEX_MAXN + 1];
};

// One-dimensional SIPG line operators of a Cartesian mesh with constant viscosity (unit nu).
// On affine Cartesian elements with GLL collocation the SIPG operator is a sum over the
// directions k of (tangential mass) x (1D SIPG operator along k), so per direction the
// element's own block and its rank-2 coupling to each neighbour along k are fixed matrices:
//   A[k][3*kl + kr][i*N + j] : own block for left / right face kinds kl, kr
//   C[k][side][kind][0][i]   : coefficient of the neighbour's trace (or Dirichlet datum)
//   C[k][side][kind][1][i]   : coefficient of the neighbour's normal derivative
//   dn[k][side][j]           : row forming that derivative from the neighbour's line
//   Wt[k][i]                 : (h_k / 2) w_i, the factor that direction k contributes to
//                              tangential and volume weights
// face kinds: 0 no terms (Neumann), 1 interior, 2 Dirichlet
template <typename T>
struct LineOps {
  T A[3][9][IMEX_MAXN * IMEX_MAXN];
  T C[3][2][3][2][IMEX_MAXN];
  T dn[3][2][IMEX_MAXN];
  T Wt[3][IMEX_MAXN];
};

template <typename T> __device__ __forceinline__ const Tables<T>& tab(const Geom& g);
template <> __device__ __forceinline__ const Tables<double>& tab<double>(const Geom& g) {
  return *reinterpret_cast<const Tables<double>*>(g.tab64);
}
template <> __device__ __forceinline__ const Tables<float>& tab<float>(const Geom& g) {
  return *reinterpret_cast<const Tables<float>*>(g.tab32);
}

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }
__host__ __device__ constexpr int over_q(int N) { return (3 * N + 1) / 2; }

// The geometry of element e as seen from its own instance: box, counts and sizes of the
// instance, and el = e - e0 its index there.  Single-instance meshes return g unchanged.
__device__ __forceinline__ Geom local_geom(const Geom& g, int e, int& el) {
  if (!g.inst) {
    el = e;
    return g;
  }
  const InstGeom& I = g.inst[g.elem_inst[e]];
  Geom l = g;
  for (int k = 0; k < 3; ++k) {
    l.n[k] = I.n[k];
    l.lo[k] = I.lo[k];
    l.h[k] = I.h[k];
    l.hf[k] = I.hf[k];
  }
  l.e0 = I.e0;
  l.inu0 = I.nu0;
  l.inu0f = I.nu0f;
  l.idt = I.dt;
  l.idtf = I.dtf;
  el = e - I.e0;
  return l;
}

template <typename T> __host__ __device__ __forceinline__ T geom_nu0(const Geom& g);
template <> __host__ __device__ __forceinline__ double geom_nu0<double>(const Geom& g) { return g.inu0; }
template <> __host__ __device__ __forceinline__ float geom_nu0<float>(const Geom& g) { return g.inu0f; }
template <typename T> __host__ __device__ __forceinline__ T geom_dt(const Geom& g);
template <> __host__ __device__ __forceinline__ double geom_dt<double>(const Geom& g) { return g.idt; }
template <> __host__ __device__ __forceinline__ float geom_dt<float>(const Geom& g) { return g.idtf; }

// neighbour element (index in the union) across face (k, side) of the element with local
// coordinates ec (side -1 or +1); -1 on a domain boundary.  g is the element's local_geom.
__device__ __forceinline__ int neighbor(const Geom& g, const int ec[3], int k, int side) {
  int cx = ec[0], cy = ec[1], cz = ec[2];
  const int nk = geom_n(g, k);
  int j = (k == 0 ? cx : (k == 1 ? cy : cz)) + side;
  if (j < 0 || j >= nk) {
    if (geom_bc(g, k) != 0) return -1;
    j = j < 0 ? j + nk : j - nk;                 // periodic wrap by one element
  }
  if (k == 0) cx = j;
  else if (k == 1) cy = j;
  else cz = j;
  return g.e0 + cx + g.n[0] * (cy + g.n[1] * cz);
}

// local coordinates of the element with local index el (g: its local_geom)
__device__ __forceinline__ void elem_coords(const Geom& g, int el, int ec[3]) {
  ec[0] = el % g.n[0];
  int r = el / g.n[0];
  ec[1] = r % g.n[1];
  ec[2] = r / g.n[1];
}

// host-side table construction (basis.cpp)
void build_tables(Tables<double>* t64, Tables<float>* t32);
void build_line_ops(const Tables<double>& t, int N, const double* h, int d, LineOps<double>* o64,
                    LineOps<float>* o32);
// E[i * Nc + j] = l_j(x_i): GLL(Nc) cardinal polynomials at the GLL(Nf) points
void gll_interp(int Nc, int Nf, double* E);

// number of kernels this library has launched (all contexts, all threads); add_launches
// accounts for the kernels of a CUDA-graph replay
void count_launch();
void add_launches(long long n);
long long launch_count();
long long thread_launch_count();     // launches issued by the calling thread

// raise a kernel's dynamic shared-memory limit once per device (kept out of the launch path,
// so that launches can be captured into CUDA graphs)
void smem_limit_once(const void* kernel, int bytes);

// Programmatic dependent launch (the kernels of the CG iteration loop).  A kernel launched
// with the programmatic-serialization attribute may be scheduled while its predecessor in
// the stream is still running; it calls pdl_wait() before it reads or writes anything the
// predecessor (or an earlier kernel) touches -- the wait returns once the predecessor has
// completed and its memory operations are visible -- and pdl_trigger() to let its own
// successor be scheduled.  Without the attribute both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
// IMEX_PDL=1 in the environment launches the CG loop kernels with the attribute
bool pdl_enabled();

// launch of a kernel of the CG loop: counted, with the programmatic-serialization attribute
// when enabled
template <typename... KArgs, typename... Args>
void launch_cg_kernel(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                      Args... args) {
  count_launch();
  if (!pdl_enabled()) {
    kernel<<<grid, block, smem, st>>>(args...);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace imex

// every kernel launch of the library goes through this macro, which counts it
#define IMEX_COUNTED(...)    \
  do {                       \
    ::imex::count_launch();  \
    __VA_ARGS__;             \
  } while (0)

