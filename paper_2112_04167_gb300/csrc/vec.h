// Device-resident scalars and launchers of the Jacobi-PCG kernels (k_vec.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace imex {

// Per-system CG scalars, all in device memory.  done: 0 running, 1 converged,
// 2 NaN in the residual, 3 iteration limit reached.
struct CgScalars {
  double* rz;
  double* rz_old;
  double* rr;
  double* bb;
  double* pAp;
  int* done;
  int* iters;
  double tol2;     // (relative tolerance)^2 on ||r||_2 / ||b||_2
};

template <typename T>
void cg_init(T* p, T* z, const T* r, const T* dinv, size_t n, long long stride, int nsys, const CgScalars& sc,
             double* partial, int nblocks, cudaStream_t st);
template <typename T>
void cg_pap(const T* p, const T* Ap, size_t n, long long stride, int nsys, const CgScalars& sc,
            double* partial, int nblocks, cudaStream_t st);
template <typename T>
void cg_step_xr(T* x, T* r, const T* p, const T* Ap, const T* dinv, T* z, size_t n, long long stride,
                int nsys, const CgScalars& sc, int maxit, double* partial, int nblocks, cudaStream_t st);
template <typename T>
void cg_step_p(T* p, const T* z, size_t n, long long stride, int nsys, const CgScalars& sc, int nblocks,
               cudaStream_t st);

}  // namespace imex
