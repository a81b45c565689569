// Device-resident scalars and launchers of the Jacobi-PCG kernels (k_vec.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace imex {

// Per-system CG scalars, all in device memory.  done: 0 running, 1 converged,
// 2 NaN in the residual, 3 iteration limit reached (4: converged in the true residual,
// set by the host of the mixed form).
struct CgScalars {
  double* rz;
  double* rz_old;
  double* rr;
  double* bb;
  double* pAp;
  int* done;
  int* iters;
  double tol2;     // (relative tolerance)^2 on ||r||_2 / ||b||_2
  double* zmean;   // projected systems: mean of D^{-1} r'
  double* rmean;   // projected systems: mean of the recursive residual r
  double* dsum;    // projected systems: sum of D^{-1} over the system
  int project;     // 1: singular systems with the constants as null space
  // step coefficients, computed once per iteration by the kernel that finishes the
  // reduction they need, in FP64 and FP32 (the streaming kernels read them directly)
  double* alpha;   // rz / pAp
  double* beta;    // rz / rz_old
  float* alpha_f;
  float* beta_f;
  float* zmean_f;
  float* rmean_f;
  // the partials (p, A p) left in the vector type by a deferred fused apply
  // ([system][*apart_n]) or by the deferred dot kernel (one per segment block, apart_seg = 1),
  // or nullptr: the step kernel then forms pAp and alpha itself
  const double* apart;
  const unsigned int* apart_n;
  int apart_seg;
};

// Segments of a set of CG systems sharing vectors (see k_vec.cu): system s occupies
// [off[s], off[s] + len[s]) of the vectors and [doff[s], doff[s] + len[s]) of the Jacobi
// diagonal; blocks of SEG_CHUNK elements, blk_seg / blk_lo per block, seg_blk0[s] the first
// block of system s (seg_blk0[nseg] = nblk).
constexpr int SEG_CHUNK = 2048;
// one block's chunk: vectors [off, off + n), diagonal [doff, doff + n), system s
struct alignas(16) SegBlock {
  long long off;
  long long doff;
  int n;
  int s;
  int pad[2];
};
struct SegTable {
  int nseg;
  int nblk;
  const long long* off;
  const long long* doff;
  const int* len;
  const int* blk_seg;
  const int* blk_lo;
  const int* seg_blk0;
  const SegBlock* blk;
};
// x += alpha p, r -= alpha A p, the new (projected) CG scalars and the convergence test
template <typename T>
void seg_step_xr(T* x, T* r, const T* p, const T* Ap, const T* dinv, const SegTable& t, const CgScalars& sc,
                 int maxit, double* partial, unsigned int* counter, cudaStream_t st);
// p = z' + beta p with z' the (projected) preconditioned residual (beta = 0 with restart = 1)
template <typename T>
void seg_step_p(T* p, T* r, const T* dinv, const SegTable& t, const CgScalars& sc, int restart, cudaStream_t st);
template <typename T>
void seg_dot(const T* x, const T* y, const SegTable& t, double* out, double* partial, unsigned int* counter,
             cudaStream_t st);
// (p, A p) per system into sc.pAp, and the step length alpha = rz / pAp
template <typename T>
void seg_pap(const T* p, const T* Ap, const SegTable& t, const CgScalars& sc, double* partial, unsigned int* counter,
             cudaStream_t st);
// CG scalars of a new residual (reset = 1: all systems, iteration counts and flags restart)
template <typename T>
void seg_init(const T* r, const T* dinv, const SegTable& t, const CgScalars& sc, double* partial,
              unsigned int* counter, int reset, cudaStream_t st);
void seg_remove_mean(double* x, const SegTable& t, double* mean, double* partial, unsigned int* counter,
                     cudaStream_t st);
// CG with a general preconditioner z = B r (the p-multigrid V-cycle).  The step kernel runs
// with a unit diagonal (it yields alpha, x, r, (r, r), the mean of r and the convergence
// test); then, for the running systems of projected problems, r -= mean(r) (seg_rproj);
// z = B r; seg_rz forms (r, z), the mean of z and beta = (r, z) / (r, z)_old (init = 1: the
// first residual of a cycle, no beta); seg_pz sets p = z - mean(z) + beta p (restart: beta 0).
template <typename T>
void seg_rproj(T* r, const SegTable& t, const CgScalars& sc, cudaStream_t st);
template <typename T>
void seg_rz(const T* r, const T* z, const SegTable& t, const CgScalars& sc, double* partial, unsigned int* counter,
            int init, cudaStream_t st);
template <typename T>
void seg_pz(T* p, const T* z, const SegTable& t, const CgScalars& sc, int restart, cudaStream_t st);
// x -= (sum w x / sum w) per segment; w indexed like the Jacobi diagonal (doff)
void seg_remove_wmean(double* x, const double* w, const SegTable& t, double* mean, double* partial,
                      unsigned int* counter, cudaStream_t st);

// Persistent projected FP32 CG for the periodic 3D constant-coefficient pressure operator
// of one instance (k_sipg.cu): runs iterations in one cooperative launch until the
// recursive residual meets tol^2 bb, drops below stop_rr (replacement due), maxit or a
// breakdown; the scalars in sc are read at start and written back at exit.  partial: 5 x
// (number of SMs x resident blocks) doubles; bar: two zeroed counters; err: zeroed flag set
// when a barrier wait gives up.  Returns -1 when the case is not supported (nothing launched).
struct Geom;
template <typename T> struct SipgArgs;
int pcg_persist_f32(const Geom& g, int N, const SipgArgs<float>& a, float* y, float* r, float* p, float* Ap,
                    const float* dinv, long long n, const CgScalars& sc, double stop_rr, int maxit, double* partial,
                    unsigned int* bar, int* err, cudaStream_t st);

}  // namespace imex
