// FP32 line-owner SIPG kernels (the CG and p-multigrid applies of the mixed form, the
// persistent FP32 CG) and their constant-memory line operators.
#include <algorithm>
#include <cooperative_groups.h>

#include "k_sipg_line.cuh"

namespace imex {

__constant__ ConstLine<float> c_line32[IMEX_MAXN + 1];
template <> __device__ __forceinline__ const ConstLine<float>& cline<float>(int N) { return c_line32[N]; }

bool upload_const_lines_f32(const ConstLine<float>* h) {
  return cudaMemcpyToSymbol(c_line32, h, sizeof(ConstLine<float>) * (IMEX_MAXN + 1)) == cudaSuccess;
}

int sipg_apply_line(const Geom& g, int N, const SipgArgs<float>& a, cudaStream_t st) {
  return sipg_apply_line_t<float>(g, N, a, st);
}

int pcg_persist_f32(const Geom& g, int N, const SipgArgs<float>& a, float* y, float* r, float* p, float* Ap,
                    const float* dinv, long long n, const CgScalars& sc, double stop_rr, int maxit, double* partial,
                    unsigned int* bar, int* err, cudaStream_t st) {
  if (g.d != 3 || g.inst || g.bc[0] || g.bc[1] || g.bc[2] || a.nu || !a.ops) return -1;
  PcgPersist q{y, r, p, Ap, dinv, n, stop_rr, partial, bar, err};
  SipgArgs<float> aa = a;
  aa.x = p;
  aa.y = Ap;
  aa.nsys = 1;
  aa.dot_out = nullptr;
  switch (N) {
    case 3: return launch_persist<3>(g, aa, q, sc, maxit, nullptr, st);
    case 4: return launch_persist<4>(g, aa, q, sc, maxit, nullptr, st);
    case 5: return launch_persist<5>(g, aa, q, sc, maxit, nullptr, st);
    case 6: return launch_persist<6>(g, aa, q, sc, maxit, nullptr, st);
    case 7: return launch_persist<7>(g, aa, q, sc, maxit, nullptr, st);
    case 8: return launch_persist<8>(g, aa, q, sc, maxit, nullptr, st);
    default: return -1;
  }
}

// ---------------------------------------------------------------------------------
// The coarsest p-multigrid level (N = 2 points per direction, 3D, every face periodic,
// unit viscosity, FP32) smoothed on one thread-block cluster: all Chebyshev steps of the
// level in one launch instead of one apply per step.  The CTAs of the cluster own
// contiguous element ranges and keep their elements' right-hand side, D^{-1} and two
// iterates in shared memory; values of neighbour elements owned by another CTA are read
// from that CTA's shared memory (distributed shared memory), and a cluster barrier
// separates the steps.  The steps use the three-term form of the Chebyshev recurrence
// (Saad, Iterative Methods for Sparse Linear Systems, Alg. 12.1, with d_k = x_{k+1} - x_k):
//   x_1 = D^{-1} b / theta,
//   x_{k+1} = x_k + c1_k (x_k - x_{k-1}) + c2_k D^{-1} (b - A x_k),   k = 1 .. m - 1,
// the same iterates as the direction form the separate applies use, so that x_{k+1}
// overwrites x_{k-1} node by node (neighbours read only x_k).
// ---------------------------------------------------------------------------------
namespace {
constexpr int PMGC_THREADS = 1024;
constexpr int PMGC_MAXSTEPS = 64;
struct CoarseCheb {
  int steps;                          // m >= 1
  int per;                            // elements per CTA
  float c0;                           // 1 / theta
  float c1[PMGC_MAXSTEPS], c2[PMGC_MAXSTEPS];
};

// The line operator's coefficients at node n = i + 2 j + 4 k, per direction d: the node's
// position p along d selects the row of the 2 x 2 own-line block and the neighbour trace /
// derivative coefficients; wt is the tangential weight over h_d.  Selected once per thread
// (every thread keeps one node index), so that the step loop reads no constant memory at
// thread-dependent addresses.
struct PmgcNode {
  float a0[3], a1[3], ctl[3], cdl[3], ctr[3], cdr[3], wt[3];
  int base[3];
};
__device__ __forceinline__ PmgcNode pmgc_node(const ConstLine<float>& L, int n, const float h[3]) {
  PmgcNode c;
  const float w0 = L.w[0], w1 = L.w[1];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int p = (n >> d) & 1;
    c.base[d] = n - p * (1 << d);
    c.a0[d] = p ? L.A[2] : L.A[0];
    c.a1[d] = p ? L.A[3] : L.A[1];
    c.ctl[d] = p ? L.ctrL[1] : L.ctrL[0];
    c.cdl[d] = p ? L.cdnL[1] : L.cdnL[0];
    c.ctr[d] = p ? L.ctrR[1] : L.ctrR[0];
    c.cdr[d] = p ? L.cdnR[1] : L.cdnR[0];
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    const float wa = ((n >> t1) & 1) ? w1 : w0, wb = ((n >> t2) & 1) ? w1 : w0;
    c.wt[d] = (0.5f * h[t1] * wa) * (0.5f * h[t2] * wb) / h[d];
  }
  return c;
}

// (A x)[n] at the node of c in the element whose values are xe, with the six neighbour
// elements' values xn[f] (face f = 2 direction + side): per direction the line of the node
// (its two values), the neighbours' lines at the same tangential position, the unit-size
// line operator and the tangential weights, as in the line-owner apply
__device__ __forceinline__ float pmgc_apply_node(const PmgcNode& c, float dl0, float dl1, float dr0, float dr1,
                                                 const float* xe, const float* const* xn) {
  float out = 0.f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int sd = 1 << d;
    const int base = c.base[d];
    const float u0 = xe[base], u1 = xe[base + sd];
    const float l0 = xn[2 * d][base], l1 = xn[2 * d][base + sd];
    const float r0 = xn[2 * d + 1][base], r1 = xn[2 * d + 1][base + sd];
    const float dl = dl0 * l0 + dl1 * l1;
    const float dr = dr0 * r0 + dr1 * r1;
    float s = c.ctl[d] * l1 + c.cdl[d] * dl + c.ctr[d] * r0 + c.cdr[d] * dr;
    s += c.a0[d] * u0 + c.a1[d] * u1;
    out += c.wt[d] * s;
  }
  return out;
}

// all Chebyshev steps of the FP32 coarsest (degree-1) p-multigrid level on one thread-block
// cluster (the three-term Chebyshev recurrence)
__global__ void __launch_bounds__(PMGC_THREADS) pmg_coarse_cluster_kernel(Geom g, const float* __restrict__ b,
                                                                          const float* __restrict__ dinv,
                                                                          float* __restrict__ x, CoarseCheb cc) {
  namespace cgr = cooperative_groups;
  cgr::cluster_group cl = cgr::this_cluster();
  const int rank = (int)cl.block_rank();
  const int per = cc.per;
  const int e0 = rank * per;
  const int nloc = max(0, min(per, g.ne - e0));
  extern __shared__ __align__(16) float pmgc_sm[];
  const float** snbp = reinterpret_cast<const float**>(pmgc_sm);   // [per][6] neighbours' slots in xa
  float* xa = reinterpret_cast<float*>(snbp + (size_t)per * 6);    // iterates (alternating)
  float* xb = xa + per * 8;
  float* sbv = xb + per * 8;                 // b
  float* sdv = sbv + per * 8;                // D^{-1}
  const ConstLine<float>& L = cline<float>(2);
  const float h[3] = {g.hf[0], g.hf[1], g.hf[2]};
  static_assert(PMGC_THREADS % 8 == 0, "one node index per thread");
  for (int q = threadIdx.x; q < nloc * 8; q += blockDim.x) {
    const size_t gi = (size_t)e0 * 8 + q;
    const float bv = b[gi], dv = dinv[gi];
    sbv[q] = bv;
    sdv[q] = dv;
    xa[q] = cc.c0 * dv * bv;
  }
  // the neighbours' slots of buffer xa, local or in another CTA's shared memory (the
  // layout is the same in every CTA: buffer xb lies per * 8 floats further)
  for (int t = threadIdx.x; t < nloc * 6; t += blockDim.x) {
    const int le = t / 6, f = t - le * 6;
    int ec[3];
    elem_coords(g, e0 + le, ec);
    const int nb = neighbor(g, ec, f >> 1, (f & 1) ? 1 : -1);
    const int r = nb / per;
    snbp[t] = (r == rank ? xa : cl.map_shared_rank(xa, r)) + (nb - r * per) * 8;
  }
  // the thread's node index is the same in every task (the block size is a multiple of 8)
  const PmgcNode nc = pmgc_node(L, threadIdx.x & 7, h);
  const float dl0 = L.dnL[0], dl1 = L.dnL[1], dr0 = L.dnR[0], dr1 = L.dnR[1];
  cl.sync();
  float* cur = xa;
  float* prev = xb;
  for (int k = 1; k < cc.steps; ++k) {
    const float c1 = cc.c1[k], c2 = cc.c2[k];
    const int boff = cur == xa ? 0 : per * 8;
    for (int q = threadIdx.x; q < nloc * 8; q += blockDim.x) {
      const int le = q >> 3;
      const float* xn[6];
#pragma unroll
      for (int f = 0; f < 6; ++f) xn[f] = snbp[le * 6 + f] + boff;
      const float ax = pmgc_apply_node(nc, dl0, dl1, dr0, dr1, cur + le * 8, xn);
      const float xk = cur[q];
      const float xp = k == 1 ? 0.f : prev[q];
      prev[q] = xk + c1 * (xk - xp) + c2 * sdv[q] * (sbv[q] - ax);
    }
    cl.sync();
    float* t = cur;
    cur = prev;
    prev = t;
  }
  for (int q = threadIdx.x; q < nloc * 8; q += blockDim.x) x[(size_t)e0 * 8 + q] = cur[q];
}

// cluster size per device: 16 CTAs (non-portable size) when the GPU can co-schedule them with
// the largest shared memory the kernel may ask for, else 8, else 0 (not usable)
constexpr size_t PMGC_MAX_SMEM = (size_t)160 * 1024;
int g_pmgc_csize[64];
bool g_pmgc_decided[64];

size_t pmgc_smem(int per) { return (size_t)per * (6 * sizeof(const float*) + 4 * 8 * sizeof(float)); }

int pmgc_decide() {
  if (cudaFuncSetAttribute((const void*)pmg_coarse_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed,
                           1) != cudaSuccess)
    cudaGetLastError();
  if (cudaFuncSetAttribute((const void*)pmg_coarse_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)PMGC_MAX_SMEM) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  for (int cs : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(PMGC_THREADS);
    cfg.dynamicSmemBytes = PMGC_MAX_SMEM;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, (const void*)pmg_coarse_cluster_kernel, &cfg) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (nclusters >= 1) return cs;
  }
  return 0;
}

// elements per CTA for ne elements with cluster size cs, 0 when they do not fit
int pmgc_per(long long ne, int cs) {
  if (cs <= 0) return 0;
  const long long per = (ne + cs - 1) / cs;
  return pmgc_smem((int)std::min<long long>(per, 1 << 20)) <= PMGC_MAX_SMEM ? (int)per : 0;
}
}  // namespace

bool pmg_cluster_prepare(const Geom& g, int N) {
  if (N != 2 || g.d != 3 || g.inst || g.bc[0] || g.bc[1] || g.bc[2] || g.ne < 1) return false;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return false;
  if (!g_pmgc_decided[dev]) {
    g_pmgc_csize[dev] = pmgc_decide();
    g_pmgc_decided[dev] = true;
  }
  return pmgc_per(g.ne, g_pmgc_csize[dev]) > 0;
}

int pmg_coarse_cluster(const Geom& g, int N, const float* b, const float* dinv, float* x, int steps, double lmax,
                       double ratio, cudaStream_t st) {
  if (steps < 1 || steps > PMGC_MAXSTEPS || N != 2 || g.d != 3 || g.inst || g.bc[0] || g.bc[1] || g.bc[2])
    return -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !g_pmgc_decided[dev]) return -1;
  const int cs = g_pmgc_csize[dev];
  const int per = pmgc_per(g.ne, cs);
  if (per <= 0) return -1;
  CoarseCheb cc{};
  cc.steps = steps;
  cc.per = per;
  const double lmin = lmax / ratio;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
  cc.c0 = (float)(1.0 / theta);
  double rho = 1.0 / sigma;
  for (int k = 1; k < steps; ++k) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    cc.c1[k] = (float)(rn * rho);
    cc.c2[k] = (float)(2.0 * rn / delta);
    rho = rn;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(PMGC_THREADS);
  cfg.dynamicSmemBytes = pmgc_smem(per);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  IMEX_COUNTED(cudaLaunchKernelEx(&cfg, pmg_coarse_cluster_kernel, g, b, dinv, x, cc));
  return 0;
}

}  // namespace imex
