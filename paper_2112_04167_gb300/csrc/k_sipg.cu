// Matrix-free symmetric interior penalty (SIPG) operator, Sec. 3.3 of the paper
// ("interior penalty method for pressure and viscous diffusion equations"),
// applied by sum factorisation on one element per thread group.
//
//   a(u, w) = sum_K sum_q W_q nu_q grad u . grad w                        (volume, GLL quadrature)
//           - sum_F sum_f W_f ({nu du/dn} [w] + {nu dw/dn} [u])            (consistency, symmetry)
//           + sum_F sum_f W_f tau [u] [w]                                   (penalty)
//   tau = N^2 / h_perp * max(nu-, nu+) on interior faces, 2 N^2 / h * nu on Dirichlet faces,
//   N = nodes per direction.  Dirichlet data g enters through [u] = u - g (Nitsche), so
//   the kernel returns  y = alpha M x + beta (A x - r_b(g))  and optionally M^{-1} y.
//
// Per element the kernel stages the element tile and, for each of its 2d faces,
// the neighbour's trace, normal derivative and viscosity in shared memory; the
// symmetric face term is folded into the volume flux at the face nodes, so one
// transposed derivative pass per direction produces the whole result.
#include "k_sipg.cuh"

namespace imex {

template <typename T, int D, int N>
struct SipgShape {
  static constexpr int ND = ipow(N, D);
  static constexpr int NF = ipow(N, D - 1);
  static constexpr int EPB = (ND >= 128) ? 1 : (256 / ND);       // elements per block
  static constexpr int THREADS = EPB * ND;
};

// the SIPG operator of Sec. 3.3 (penalty N^2 / h max(nu-, nu+)), generic form: y = alpha M x + beta (A(nu) x -
// r_b(g)) for any face kinds and a nodal or constant viscosity
template <typename T, int D, int N>
__global__ void __launch_bounds__(SipgShape<T, D, N>::THREADS)
sipg_apply_kernel(Geom g, SipgArgs<T> a) {
  using S = SipgShape<T, D, N>;
  constexpr int ND = S::ND, NF = S::NF, EPB = S::EPB;
  __shared__ T sD[N * N];
  __shared__ T sw[N];
  __shared__ T su[EPB][ND];
  __shared__ T snu[EPB][ND];
  __shared__ T sQ[D][EPB][ND];
  __shared__ T sfu[EPB][2 * D][NF];
  __shared__ T sfdu[EPB][2 * D][NF];
  __shared__ T sfnu[EPB][2 * D][NF];
  __shared__ int snb[EPB][2 * D];

  const Tables<T>& tb = tab<T>(g);
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) sD[i] = tb.D[N][i];
  for (int i = threadIdx.x; i < N; i += blockDim.x) sw[i] = tb.w[N][i];

  const int le = threadIdx.x / ND;
  const int node = threadIdx.x % ND;
  const int e = blockIdx.x * EPB + le;
  const bool valid = e < g.ne;
  int el = 0;
  Geom gl = g;
  if (valid) gl = local_geom(g, e, el);
  int ec[3] = {0, 0, 0};
  if (valid) elem_coords(gl, el, ec);
  int id[3];
  id[0] = node % N;
  id[1] = (D > 1) ? (node / N) % N : 0;
  id[2] = (D > 2) ? node / (N * N) : 0;

  // neighbours (-1: boundary)
  if (valid && node < 2 * D) {
    const int k = node >> 1, side = node & 1;
    snb[le][node] = neighbor(gl, ec, k, side ? 1 : -1);
  }
  // viscosity of the element
  if (valid) snu[le][node] = a.nu ? a.nu[(size_t)e * ND + node] : sipg_nu0(a, gl);
  __syncthreads();

  T hinv2[D];
  T jac = T(1);
  for (int k = 0; k < D; ++k) { hinv2[k] = T(2) / geom_h<T>(gl, k); jac *= geom_h<T>(gl, k) * T(0.5); }
  T Wq = jac;
  for (int k = 0; k < D; ++k) Wq *= sw[id[k]];

  // face viscosity of the neighbours (once for all systems)
  if (valid) {
    for (int t = node; t < 2 * D * NF; t += ND) {
      const int fi = t / NF, f = t % NF, k = fi >> 1, side = fi & 1;
      const int nb = snb[le][fi];
      int c[3];
      {  // face-node coordinates over the directions other than k
        int r = f, q = 0;
        for (int j = 0; j < D; ++j) {
          if (j == k) continue;
          c[j] = r % N; r /= N; ++q;
        }
      }
      if (nb >= 0) {
        c[k] = side ? 0 : N - 1;                       // matching face of the neighbour
        int nn = c[0] + N * ((D > 1 ? c[1] : 0) + N * (D > 2 ? c[2] : 0));
        sfnu[le][fi][f] = a.nu ? a.nu[(size_t)nb * ND + nn] : sipg_nu0(a, gl);
      } else {
        c[k] = side ? N - 1 : 0;
        int nn = c[0] + N * ((D > 1 ? c[1] : 0) + N * (D > 2 ? c[2] : 0));
        sfnu[le][fi][f] = snu[le][nn];
      }
    }
  }

  for (int s = 0; s < a.nsys; ++s) {
    const T* x = a.x + (size_t)s * a.sys_stride;
    const T* gd = a.gdata ? a.gdata + (size_t)s * a.g_stride : nullptr;
    T* y = a.y + (size_t)s * a.sys_stride;
    __syncthreads();
    if (valid) su[le][node] = x[(size_t)e * ND + node];
    // neighbour traces and normal derivatives
    if (valid) {
      for (int t = node; t < 2 * D * NF; t += ND) {
        const int fi = t / NF, f = t % NF, k = fi >> 1, side = fi & 1;
        const int nb = snb[le][fi];
        int c[3] = {0, 0, 0};
        {
          int r = f;
          for (int j = 0; j < D; ++j) {
            if (j == k) continue;
            c[j] = r % N; r /= N;
          }
        }
        if (nb >= 0) {
          const int iface = side ? 0 : N - 1;            // neighbour's own index on the shared face
          int stride = 1;
          for (int j = 0; j < k; ++j) stride *= N;
          c[k] = 0;
          const int base = c[0] + N * ((D > 1 ? c[1] : 0) + N * (D > 2 ? c[2] : 0));
          const T* xl = x + (size_t)nb * ND + base;
          T acc = T(0), tr = T(0);
#pragma unroll
          for (int j = 0; j < N; ++j) {
            T v = xl[j * stride];
            acc += sD[iface * N + j] * v;
            if (j == iface) tr = v;
          }
          sfu[le][fi][f] = tr;
          sfdu[le][fi][f] = acc * hinv2[k];
        } else {
          c[k] = side ? N - 1 : 0;
          const int nn = c[0] + N * ((D > 1 ? c[1] : 0) + N * (D > 2 ? c[2] : 0));
          sfu[le][fi][f] = gd ? gd[(size_t)e * ND + nn] : T(0);
          sfdu[le][fi][f] = T(0);
        }
      }
    }
    __syncthreads();

    T yface = T(0);
    if (valid) {
      const T uo = su[le][node];
      const T nuq = snu[le][node];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        int stride = 1;
        for (int j = 0; j < k; ++j) stride *= N;
        const int base = node - id[k] * stride;
        T acc = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) acc += sD[id[k] * N + j] * su[le][base + j * stride];
        const T gk = acc * hinv2[k];
        T Qk = Wq * nuq * gk;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
          if (id[k] != (side ? N - 1 : 0)) continue;
          const int fi = 2 * k + side;
          const int nb = snb[le][fi];
          const int bc = geom_bc(g, k);
          if (nb < 0 && bc != 1) continue;                 // Neumann: no face terms
          T Wf = jac / (geom_h<T>(gl, k) * T(0.5));
          int f = 0, mul = 1;
          for (int j = 0; j < D; ++j) {
            if (j == k) continue;
            Wf *= sw[id[j]];
            f += id[j] * mul; mul *= N;
          }
          const T n = side ? T(1) : T(-1);
          const T un = sfu[le][fi][f];
          const T jump = uo - un;
          const T pen = T(N * N) * T(0.5) * hinv2[k];       // N^2 / h
          if (nb >= 0) {
            const T nun = sfnu[le][fi][f];
            Qk += -Wf * T(0.5) * nuq * jump * n;
            const T tau = pen * (nuq > nun ? nuq : nun);
            yface += Wf * (-T(0.5) * (nuq * n * gk + nun * n * sfdu[le][fi][f]) + tau * jump);
          } else {
            Qk += -Wf * nuq * jump * n;
            yface += Wf * (-nuq * n * gk + T(2) * pen * nuq * jump);
          }
        }
        sQ[k][le][node] = Qk;
      }
    }
    __syncthreads();
    if (valid) {
      T yv = yface;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        int stride = 1;
        for (int j = 0; j < k; ++j) stride *= N;
        const int base = node - id[k] * stride;
        T acc = T(0);
#pragma unroll
        for (int q = 0; q < N; ++q) acc += sD[q * N + id[k]] * sQ[k][le][base + q * stride];
        yv += acc * hinv2[k];
      }
      T out = a.alpha * Wq * su[le][node] + sipg_beta(a, gl) * yv;
      if (a.minv) out /= Wq;
      y[(size_t)e * ND + node] = out;
    }
  }
}

// ---------------------------------------------------------------------------------
// 3D form: N^2 threads per element, each owning one z-column (i0, i1) of the element
// tile in registers.  x / y derivatives read the tile from shared memory, z
// derivatives stay in registers; the neighbours' traces and normal derivatives on
// the four lateral faces are staged cooperatively (one face node per thread and
// face), those of the two z-faces per thread in registers.
// ---------------------------------------------------------------------------------
template <int N>
struct Sipg3Shape {
  static constexpr int NN = N * N;
  static constexpr int ND = N * N * N;
  static constexpr int EPB = (NN >= 49) ? 4 : (NN >= 16 ? 256 / NN : 16);
  static constexpr int THREADS = EPB * NN;
};

// face contribution at one node: the symmetric term enters the flux Qk, the
// consistency and penalty terms the nodal value yface.  kind: 0 none, 1 interior, 2 Dirichlet
template <typename T>
__device__ __forceinline__ void sipg_face(int kind, T Wf, T n, T uo, T gk, T nuq, T un, T dn, T nun, T pen, T& Qk,
                                          T& yface) {
  if (kind == 1) {
    const T jump = uo - un;
    Qk += -Wf * T(0.5) * nuq * jump * n;
    const T tau = pen * (nuq > nun ? nuq : nun);
    yface += Wf * (-T(0.5) * n * (nuq * gk + nun * dn) + tau * jump);
  } else if (kind == 2) {
    const T jump = uo - un;
    Qk += -Wf * nuq * jump * n;
    yface += Wf * (-nuq * n * gk + T(2) * pen * nuq * jump);
  }
}

template <typename T, int N>
constexpr size_t sipg3_smem() {
  using S = Sipg3Shape<N>;
  return sizeof(T) * (size_t)(N * N + N + 3 * S::EPB * S::ND + 3 * S::EPB * 4 * S::NN);
}

// the SIPG operator of Sec. 3.3 in 3D, variable or constant viscosity: gradient, flux and
// transposed derivative passes
template <typename T, int N, bool VARNU>
__global__ void __launch_bounds__(Sipg3Shape<N>::THREADS)
sipg3_apply_kernel(Geom g, SipgArgs<T> a) {
  using S = Sipg3Shape<N>;
  constexpr int NN = S::NN, ND = S::ND, EPB = S::EPB;
  extern __shared__ unsigned char smem_raw[];
  T* sD = reinterpret_cast<T*>(smem_raw);
  T* sw = sD + N * N;
  T (*su)[ND] = reinterpret_cast<T (*)[ND]>(sw + N);
  T (*sQx)[ND] = su + EPB;
  T (*sQy)[ND] = sQx + EPB;
  T (*sfu)[4][NN] = reinterpret_cast<T (*)[4][NN]>(sQy + EPB);
  T (*sfd)[4][NN] = sfu + EPB;
  T (*sfn)[4][NN] = sfd + EPB;
  __shared__ int snb[EPB][6];

  const Tables<T>& tb = tab<T>(g);
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) sD[i] = tb.D[N][i];
  for (int i = threadIdx.x; i < N; i += blockDim.x) sw[i] = tb.w[N][i];
  const int le = threadIdx.x / NN;
  const int t = threadIdx.x - le * NN;
  const int i0 = t % N, i1 = t / N;
  const int e = blockIdx.x * EPB + le;
  const bool valid = e < g.ne;
  int el = 0;
  Geom gl = g;
  if (valid) gl = local_geom(g, e, el);
  int ec[3] = {0, 0, 0};
  if (valid) elem_coords(gl, el, ec);
  // six neighbours per element: with N = 2 an element has only four threads
  if (valid)
    for (int f = t; f < 6; f += NN) snb[le][f] = neighbor(gl, ec, f >> 1, (f & 1) ? 1 : -1);
  __syncthreads();

  const T hx = T(2) / geom_h<T>(gl, 0), hy = T(2) / geom_h<T>(gl, 1), hz = T(2) / geom_h<T>(gl, 2);
  const T jac = geom_h<T>(gl, 0) * geom_h<T>(gl, 1) * geom_h<T>(gl, 2) * T(0.125);
  const T jfx = geom_h<T>(gl, 1) * geom_h<T>(gl, 2) * T(0.25), jfy = geom_h<T>(gl, 0) * geom_h<T>(gl, 2) * T(0.25),
          jfz = geom_h<T>(gl, 0) * geom_h<T>(gl, 1) * T(0.25);
  const T penx = T(N * N) * T(0.5) * hx, peny = T(N * N) * T(0.5) * hy, penz = T(N * N) * T(0.5) * hz;
  const size_t ebase = (size_t)e * ND;

  // own viscosity column (constant viscosity: one register)
  T nuc[VARNU ? N : 1];
#pragma unroll
  for (int k = 0; k < (VARNU ? N : 1); ++k) nuc[k] = (VARNU && valid) ? a.nu[ebase + k * NN + t] : sipg_nu0(a, gl);
  // face kinds: 0 none (Neumann), 1 interior, 2 Dirichlet
  int kind[6];
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const int nb = valid ? snb[le][f] : -1;
    kind[f] = nb >= 0 ? 1 : (g.bc[f >> 1] == 1 ? 2 : 0);
  }

  for (int s = 0; s < a.nsys; ++s) {
    const T* x = a.x + (size_t)s * a.sys_stride;
    const T* gd = a.gdata ? a.gdata + (size_t)s * a.g_stride : nullptr;
    T* y = a.y + (size_t)s * a.sys_stride;
    T u[N];
    if (s > 0) __syncthreads();
    if (valid) {
#pragma unroll
      for (int k = 0; k < N; ++k) {
        u[k] = x[ebase + k * NN + t];
        su[le][k * NN + t] = u[k];
      }
      // lateral faces: face node t = (c0, c1) with c1 = t / N the z index
      const int c0 = t % N, kk = t / N;
#pragma unroll
      for (int fi = 0; fi < 4; ++fi) {
        const int dir = fi >> 1, side = fi & 1;
        const int nb = snb[le][fi];
        T tr = T(0), dv = T(0), nn = sipg_nu0(a, gl);
        if (nb >= 0) {
          const int iface = side ? 0 : N - 1;                    // neighbour's index on the shared face
          const size_t nbase = (size_t)nb * ND + kk * NN;
          T acc = T(0);
          if (dir == 0) {
            const T* row = x + nbase + c0 * N;                  // neighbour row along x at (y = c0, z = kk)
#pragma unroll
            for (int j = 0; j < N; ++j) { const T v = row[j]; acc += sD[iface * N + j] * v; if (j == iface) tr = v; }
            dv = acc * hx;
            if (VARNU) nn = a.nu[nbase + c0 * N + iface];
          } else {
            const T* col = x + nbase + c0;                      // neighbour column along y at (x = c0, z = kk)
#pragma unroll
            for (int j = 0; j < N; ++j) { const T v = col[j * N]; acc += sD[iface * N + j] * v; if (j == iface) tr = v; }
            dv = acc * hy;
            if (VARNU) nn = a.nu[nbase + iface * N + c0];
          }
        } else if (geom_bc(g, dir) == 1) {
          const int own = side ? N - 1 : 0;
          const size_t on = ebase + kk * NN + (dir == 0 ? c0 * N + own : own * N + c0);
          tr = gd ? gd[on] : T(0);
          if (VARNU) nn = a.nu[on];
        }
        sfu[le][fi][t] = tr;
        sfd[le][fi][t] = dv;
        sfn[le][fi][t] = nn;
      }
    }
    // z-faces: the neighbour columns through this thread's (i0, i1)
    T zu[2] = {T(0), T(0)}, zd[2] = {T(0), T(0)}, zn[2] = {sipg_nu0(a, gl), sipg_nu0(a, gl)};
    if (valid) {
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const int nb = snb[le][4 + side];
        if (nb >= 0) {
          const int iface = side ? 0 : N - 1;
          const T* col = x + (size_t)nb * ND + t;
          T acc = T(0);
#pragma unroll
          for (int j = 0; j < N; ++j) { const T v = col[j * NN]; acc += sD[iface * N + j] * v; if (j == iface) zu[side] = v; }
          zd[side] = acc * hz;
          if (VARNU) zn[side] = a.nu[(size_t)nb * ND + iface * NN + t];
        } else if (g.bc[2] == 1) {
          const int own = side ? N - 1 : 0;
          zu[side] = gd ? gd[ebase + own * NN + t] : T(0);
          zn[side] = nuc[VARNU ? own : 0];
        }
      }
    }
    __syncthreads();
    T Qz[N], yf[N];
    if (valid) {
      const T wxy = sw[i0] * sw[i1];
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const T* plane = &su[le][k * NN];
        T gx = T(0), gy = T(0), gz = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
          gx += sD[i0 * N + j] * plane[i1 * N + j];
          gy += sD[i1 * N + j] * plane[j * N + i0];
          gz += sD[k * N + j] * u[j];
        }
        gx *= hx; gy *= hy; gz *= hz;
        const T nuq = nuc[VARNU ? k : 0];
        const T W = jac * wxy * sw[k];
        T Qx = W * nuq * gx, Qy = W * nuq * gy, Qzk = W * nuq * gz;
        T yface = T(0);
        const int fxy0 = i1 + N * k, fxy1 = i0 + N * k;
        if (i0 == 0) sipg_face<T>(kind[0], jfx * sw[i1] * sw[k], T(-1), u[k], gx, nuq, sfu[le][0][fxy0],
                                  sfd[le][0][fxy0], sfn[le][0][fxy0], penx, Qx, yface);
        if (i0 == N - 1) sipg_face<T>(kind[1], jfx * sw[i1] * sw[k], T(1), u[k], gx, nuq, sfu[le][1][fxy0],
                                      sfd[le][1][fxy0], sfn[le][1][fxy0], penx, Qx, yface);
        if (i1 == 0) sipg_face<T>(kind[2], jfy * sw[i0] * sw[k], T(-1), u[k], gy, nuq, sfu[le][2][fxy1],
                                  sfd[le][2][fxy1], sfn[le][2][fxy1], peny, Qy, yface);
        if (i1 == N - 1) sipg_face<T>(kind[3], jfy * sw[i0] * sw[k], T(1), u[k], gy, nuq, sfu[le][3][fxy1],
                                      sfd[le][3][fxy1], sfn[le][3][fxy1], peny, Qy, yface);
        if (k == 0) sipg_face<T>(kind[4], jfz * wxy, T(-1), u[k], gz, nuq, zu[0], zd[0], zn[0], penz, Qzk, yface);
        if (k == N - 1) sipg_face<T>(kind[5], jfz * wxy, T(1), u[k], gz, nuq, zu[1], zd[1], zn[1], penz, Qzk, yface);
        sQx[le][k * NN + t] = Qx;
        sQy[le][k * NN + t] = Qy;
        Qz[k] = Qzk;
        yf[k] = yface;
      }
    }
    __syncthreads();
    if (valid) {
      const T wxy = sw[i0] * sw[i1];
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const T* px = &sQx[le][k * NN];
        const T* py = &sQy[le][k * NN];
        T ax = T(0), ay = T(0), az = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
          ax += sD[j * N + i0] * px[i1 * N + j];
          ay += sD[j * N + i1] * py[j * N + i0];
          az += sD[j * N + k] * Qz[j];
        }
        const T W = jac * wxy * sw[k];
        const T yv = yf[k] + hx * ax + hy * ay + hz * az;
        T out = a.alpha * W * u[k] + sipg_beta(a, gl) * yv;
        if (a.minv) out /= W;
        y[ebase + k * NN + t] = out;
      }
    }
  }
}

// ---------------------------------------------------------------------------------
// Constant-viscosity fast path.  With constant nu the operator is
//   y = alpha M u + beta nu0 sum_k W_perp,k (A_k u_line + sum_sides C_k (trace, dn)_nb)
// with the precomputed line operators of LineOps: per node one N-term row of A_k per
// direction plus two or four neighbour terms, a single synchronisation per element.
// 3D: N^2 threads per element, each owning a z-column in registers.
// ---------------------------------------------------------------------------------
template <int N>
struct Sipg3cShape {
  static constexpr int NN = N * N;
  static constexpr int ND = N * N * N;
  static constexpr int EPB = (NN >= 49) ? 4 : (NN >= 16 ? 256 / NN : 16);
  static constexpr int THREADS = EPB * NN;
};

template <typename T, int N>
constexpr size_t sipg3c_smem() {
  using S = Sipg3cShape<N>;
  // A[3][9][N*N] + C[3][2][3][2][N] + dn[3][2][N] + Wt[3][N] + tile + 4 lateral faces x (trace, dn)
  return sizeof(T) * (size_t)(27 * N * N + 36 * N + 6 * N + 3 * N + S::EPB * S::ND + S::EPB * 8 * S::NN);
}

// the constant-viscosity SIPG operator of Sec. 3.3 in 3D with Dirichlet / Neumann sides,
// from the line operators of every face kind
template <typename T, int N>
__global__ void __launch_bounds__(Sipg3cShape<N>::THREADS)
sipg3c_apply_kernel(Geom g, SipgArgs<T> a) {
  using S = Sipg3cShape<N>;
  constexpr int NN = S::NN, ND = S::ND, EPB = S::EPB;
  extern __shared__ unsigned char smem_raw[];
  T* sA = reinterpret_cast<T*>(smem_raw);        // [3][9][NN]
  T* sC = sA + 27 * NN;                          // [3][2][3][2][N]
  T* sdn = sC + 36 * N;                          // [3][2][N]
  T* sWt = sdn + 6 * N;                          // [3][N]
  T (*su)[ND] = reinterpret_cast<T (*)[ND]>(sWt + 3 * N);
  T (*sf)[8][NN] = reinterpret_cast<T (*)[8][NN]>(su + EPB);   // [face 0..3][trace | dn]
  __shared__ int snb[EPB][6];
  const LineOps<T>& op = *a.ops;
  for (int i = threadIdx.x; i < 27 * NN; i += blockDim.x) {
    const int kv = i / NN, r = i % NN;
    sA[i] = op.A[kv / 9][kv % 9][r];
  }
  for (int i = threadIdx.x; i < 36 * N; i += blockDim.x) {
    const int q = i / N, r = i % N;   // q = ((k*2 + side)*3 + kind)*2 + which
    sC[i] = op.C[q / 12][(q / 6) % 2][(q / 2) % 3][q % 2][r];
  }
  for (int i = threadIdx.x; i < 6 * N; i += blockDim.x) sdn[i] = op.dn[i / (2 * N)][(i / N) % 2][i % N];
  for (int i = threadIdx.x; i < 3 * N; i += blockDim.x) sWt[i] = op.Wt[i / N][i % N];
  const int le = threadIdx.x / NN;
  const int t = threadIdx.x - le * NN;
  const int i0 = t % N, i1 = t / N;
  const int e = blockIdx.x * EPB + le;
  const bool valid = e < g.ne;
  int el = 0;
  Geom gl = g;
  if (valid) gl = local_geom(g, e, el);
  int ec[3] = {0, 0, 0};
  if (valid) elem_coords(gl, el, ec);
  // six neighbours per element: with N = 2 an element has only four threads
  if (valid)
    for (int f = t; f < 6; f += NN) snb[le][f] = neighbor(gl, ec, f >> 1, (f & 1) ? 1 : -1);
  __syncthreads();
  int kind[6];
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const int nb = valid ? snb[le][f] : -1;
    kind[f] = nb >= 0 ? 1 : (g.bc[f >> 1] == 1 ? 2 : 0);
  }
  const size_t ebase = (size_t)e * ND;
  const T scale = sipg_beta(a, gl) * sipg_nu0(a, gl);
  __shared__ double red[S::THREADS];
  for (int s = 0; s < a.nsys; ++s) {
    const T* x = a.x + (size_t)s * a.sys_stride;
    const T* gd = a.gdata ? a.gdata + (size_t)s * a.g_stride : nullptr;
    T* y = a.y + (size_t)s * a.sys_stride;
    if (s > 0) __syncthreads();
    if (cg_system_stopped(a, s)) {            // its CG iteration has stopped: A p not needed
      if (a.dot_out && threadIdx.x == 0) put_dot_partial(a, s, 0.0);
      continue;
    }
    T u[N];
    T dacc = T(0);
    T zt[2] = {T(0), T(0)}, zd[2] = {T(0), T(0)};
    if (valid) {
#pragma unroll
      for (int k = 0; k < N; ++k) {
        u[k] = x[ebase + k * NN + t];
        su[le][k * NN + t] = u[k];
      }
      // lateral faces: face node t = (c0, kk), kk the z index
      const int c0 = t % N, kk = t / N;
#pragma unroll
      for (int fi = 0; fi < 4; ++fi) {
        const int dir = fi >> 1, side = fi & 1;
        const int nb = snb[le][fi];
        T tr = T(0), dv = T(0);
        if (nb >= 0) {
          const int iface = side ? 0 : N - 1;
          const T* dr = sdn + (dir * 2 + side) * N;
          const size_t nbase = (size_t)nb * ND + kk * NN;
          if (dir == 0) {
            const T* row = x + nbase + c0 * N;
#pragma unroll
            for (int j = 0; j < N; ++j) { const T v = row[j]; dv += dr[j] * v; if (j == iface) tr = v; }
          } else {
            const T* col = x + nbase + c0;
#pragma unroll
            for (int j = 0; j < N; ++j) { const T v = col[j * N]; dv += dr[j] * v; if (j == iface) tr = v; }
          }
        } else if (kind[fi] == 2 && gd) {
          const int own = side ? N - 1 : 0;
          tr = gd[ebase + kk * NN + (dir == 0 ? c0 * N + own : own * N + c0)];
        }
        sf[le][2 * fi][t] = tr;
        sf[le][2 * fi + 1][t] = dv;
      }
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const int nb = snb[le][4 + side];
        if (nb >= 0) {
          const int iface = side ? 0 : N - 1;
          const T* dr = sdn + (2 * 2 + side) * N;
          const T* col = x + (size_t)nb * ND + t;
#pragma unroll
          for (int j = 0; j < N; ++j) { const T v = col[j * NN]; zd[side] += dr[j] * v; if (j == iface) zt[side] = v; }
        } else if (kind[4 + side] == 2 && gd) {
          zt[side] = gd[ebase + (side ? N - 1 : 0) * NN + t];
        }
      }
    }
    __syncthreads();
    if (valid) {
      const T* Ax = sA + (0 * 9 + 3 * kind[0] + kind[1]) * NN + i0 * N;
      const T* Ay = sA + (1 * 9 + 3 * kind[2] + kind[3]) * NN + i1 * N;
      const T* Az = sA + (2 * 9 + 3 * kind[4] + kind[5]) * NN;
      // neighbour coefficients of this thread's rows: C[k][side][kind][which][i]
      const T cxl0 = sC[((0 * 2 + 0) * 3 + kind[0]) * 2 * N + i0], cxl1 = sC[(((0 * 2 + 0) * 3 + kind[0]) * 2 + 1) * N + i0];
      const T cxr0 = sC[((0 * 2 + 1) * 3 + kind[1]) * 2 * N + i0], cxr1 = sC[(((0 * 2 + 1) * 3 + kind[1]) * 2 + 1) * N + i0];
      const T cyl0 = sC[((1 * 2 + 0) * 3 + kind[2]) * 2 * N + i1], cyl1 = sC[(((1 * 2 + 0) * 3 + kind[2]) * 2 + 1) * N + i1];
      const T cyr0 = sC[((1 * 2 + 1) * 3 + kind[3]) * 2 * N + i1], cyr1 = sC[(((1 * 2 + 1) * 3 + kind[3]) * 2 + 1) * N + i1];
      const T* czl = sC + ((2 * 2 + 0) * 3 + kind[4]) * 2 * N;
      const T* czr = sC + ((2 * 2 + 1) * 3 + kind[5]) * 2 * N;
      // unit-size line operators: direction k scales as 1 / h_k, its weights as h_k
      const T hx = geom_h<T>(gl, 0), hy = geom_h<T>(gl, 1), hz = geom_h<T>(gl, 2);
      const T ihx = T(1) / hx, ihy = T(1) / hy, ihz = T(1) / hz;
      const T wx = hx * sWt[i0], wy = hy * sWt[N + i1];
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const T* plane = &su[le][k * NN];
        T yx = T(0), yy = T(0), yz = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
          yx += Ax[j] * plane[i1 * N + j];
          yy += Ay[j] * plane[j * N + i0];
          yz += Az[k * N + j] * u[j];
        }
        const int fx = i1 + N * k, fy = i0 + N * k;
        yx += cxl0 * sf[le][0][fx] + cxl1 * sf[le][1][fx] + cxr0 * sf[le][2][fx] + cxr1 * sf[le][3][fx];
        yy += cyl0 * sf[le][4][fy] + cyl1 * sf[le][5][fy] + cyr0 * sf[le][6][fy] + cyr1 * sf[le][7][fy];
        yz += czl[k] * zt[0] + czl[N + k] * zd[0] + czr[k] * zt[1] + czr[N + k] * zd[1];
        const T wz = hz * sWt[2 * N + k];
        const T W = wx * wy * wz;
        const T yv = wy * wz * ihx * yx + wx * wz * ihy * yy + wx * wy * ihz * yz;
        T out = a.alpha * W * u[k] + scale * yv;
        if (a.minv) out /= W;
        sipg_out<T, T>(a, y, ebase + k * NN + t, u[k], out);
        dacc += u[k] * out;
      }
    }
    if (a.dot_out) {
      const double bs = block_sum_any_t<T>(dacc, red);
      if (threadIdx.x == 0) put_dot_partial(a, s, bs);
    }
  }
  if (a.dot_out) fused_dot_finish(a, red);
}

// 2D: one thread per node, EPB elements per block.
template <int N>
struct Sipg2cShape {
  static constexpr int NN = N * N;
  static constexpr int EPB = (256 / NN) > 0 ? 256 / NN : 1;
  static constexpr int THREADS = EPB * NN;
};

template <typename T, int N>
constexpr size_t sipg2c_smem() {
  using S = Sipg2cShape<N>;
  return sizeof(T) * (size_t)(18 * N * N + 24 * N + 4 * N + 2 * N + S::EPB * S::NN + S::EPB * 8 * N);
}

// the constant-viscosity SIPG operator of Sec. 3.3 in 2D with Dirichlet / Neumann sides
template <typename T, int N>
__global__ void __launch_bounds__(Sipg2cShape<N>::THREADS)
sipg2c_apply_kernel(Geom g, SipgArgs<T> a) {
  using S = Sipg2cShape<N>;
  constexpr int NN = S::NN, EPB = S::EPB;
  extern __shared__ unsigned char smem_raw[];
  T* sA = reinterpret_cast<T*>(smem_raw);        // [2][9][NN]
  T* sC = sA + 18 * NN;                          // [2][2][3][2][N]
  T* sdn = sC + 24 * N;                          // [2][2][N]
  T* sWt = sdn + 4 * N;                          // [2][N]
  T (*su)[NN] = reinterpret_cast<T (*)[NN]>(sWt + 2 * N);
  T (*sf)[8][N] = reinterpret_cast<T (*)[8][N]>(su + EPB);
  __shared__ int snb[EPB][4];
  const LineOps<T>& op = *a.ops;
  for (int i = threadIdx.x; i < 18 * NN; i += blockDim.x) {
    const int kv = i / NN, r = i % NN;
    sA[i] = op.A[kv / 9][kv % 9][r];
  }
  for (int i = threadIdx.x; i < 24 * N; i += blockDim.x) {
    const int q = i / N, r = i % N;
    sC[i] = op.C[q / 12][(q / 6) % 2][(q / 2) % 3][q % 2][r];
  }
  for (int i = threadIdx.x; i < 4 * N; i += blockDim.x) sdn[i] = op.dn[i / (2 * N)][(i / N) % 2][i % N];
  for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) sWt[i] = op.Wt[i / N][i % N];
  const int le = threadIdx.x / NN;
  const int t = threadIdx.x - le * NN;
  const int i0 = t % N, i1 = t / N;
  const int e = blockIdx.x * EPB + le;
  const bool valid = e < g.ne;
  int el = 0;
  Geom gl = g;
  if (valid) gl = local_geom(g, e, el);
  int ec[3] = {0, 0, 0};
  if (valid) elem_coords(gl, el, ec);
  if (valid && t < 4) snb[le][t] = neighbor(gl, ec, t >> 1, (t & 1) ? 1 : -1);
  __syncthreads();
  int kind[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const int nb = valid ? snb[le][f] : -1;
    kind[f] = nb >= 0 ? 1 : (g.bc[f >> 1] == 1 ? 2 : 0);
  }
  const size_t ebase = (size_t)e * NN;
  const T scale = sipg_beta(a, gl) * sipg_nu0(a, gl);
  __shared__ double red[S::THREADS];
  for (int s = 0; s < a.nsys; ++s) {
    const T* x = a.x + (size_t)s * a.sys_stride;
    const T* gd = a.gdata ? a.gdata + (size_t)s * a.g_stride : nullptr;
    T* y = a.y + (size_t)s * a.sys_stride;
    if (s > 0) __syncthreads();
    if (cg_system_stopped(a, s)) {            // its CG iteration has stopped: A p not needed
      if (a.dot_out && threadIdx.x == 0) put_dot_partial(a, s, 0.0);
      continue;
    }
    T uo = T(0);
    T dacc = T(0);
    if (valid) {
      uo = x[ebase + t];
      su[le][t] = uo;
      // face data: face fi = q / N, face node c = q % N for q = t, t + N^2, ... < 4N
      for (int q = t; q < 4 * N; q += NN) {
        const int fi = q / N, c = q % N, dir = fi >> 1, side = fi & 1;
        const int nb = snb[le][fi];
        T tr = T(0), dv = T(0);
        if (nb >= 0) {
          const int iface = side ? 0 : N - 1;
          const T* dr = sdn + (dir * 2 + side) * N;
          const T* line = x + (size_t)nb * NN + (dir == 0 ? c * N : c);
          const int stride = dir == 0 ? 1 : N;
#pragma unroll
          for (int j = 0; j < N; ++j) { const T v = line[j * stride]; dv += dr[j] * v; if (j == iface) tr = v; }
        } else if (kind[fi] == 2 && gd) {
          const int own = side ? N - 1 : 0;
          tr = gd[ebase + (dir == 0 ? c * N + own : own * N + c)];
        }
        sf[le][2 * fi][c] = tr;
        sf[le][2 * fi + 1][c] = dv;
      }
    }
    __syncthreads();
    if (valid) {
      const T* Ax = sA + (0 * 9 + 3 * kind[0] + kind[1]) * NN + i0 * N;
      const T* Ay = sA + (1 * 9 + 3 * kind[2] + kind[3]) * NN + i1 * N;
      T yx = T(0), yy = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        yx += Ax[j] * su[le][i1 * N + j];
        yy += Ay[j] * su[le][j * N + i0];
      }
      yx += sC[((0 * 2 + 0) * 3 + kind[0]) * 2 * N + i0] * sf[le][0][i1] +
            sC[(((0 * 2 + 0) * 3 + kind[0]) * 2 + 1) * N + i0] * sf[le][1][i1] +
            sC[((0 * 2 + 1) * 3 + kind[1]) * 2 * N + i0] * sf[le][2][i1] +
            sC[(((0 * 2 + 1) * 3 + kind[1]) * 2 + 1) * N + i0] * sf[le][3][i1];
      yy += sC[((1 * 2 + 0) * 3 + kind[2]) * 2 * N + i1] * sf[le][4][i0] +
            sC[(((1 * 2 + 0) * 3 + kind[2]) * 2 + 1) * N + i1] * sf[le][5][i0] +
            sC[((1 * 2 + 1) * 3 + kind[3]) * 2 * N + i1] * sf[le][6][i0] +
            sC[(((1 * 2 + 1) * 3 + kind[3]) * 2 + 1) * N + i1] * sf[le][7][i0];
      // unit-size line operators: direction k scales as 1 / h_k, its weights as h_k
      const T hx = geom_h<T>(gl, 0), hy = geom_h<T>(gl, 1);
      const T wx = hx * sWt[i0], wy = hy * sWt[N + i1];
      const T W = wx * wy;
      T out = a.alpha * W * uo + scale * (wy * yx / hx + wx * yy / hy);
      if (a.minv) out /= W;
      sipg_out<T, T>(a, y, ebase + t, uo, out);
      dacc = uo * out;
    }
    if (a.dot_out) {
      const double bs = block_sum_any_t<T>(dacc, red);
      if (threadIdx.x == 0) put_dot_partial(a, s, bs);
    }
  }
  if (a.dot_out) fused_dot_finish(a, red);
}

// Diagonal of alpha M + beta A (Jacobi preconditioner of the CG solves of Sec. 3.3; the
// self-neighbour term of an element that meets itself across a periodic direction).
template <typename T, int D, int N>
__global__ void __launch_bounds__(SipgShape<T, D, N>::THREADS)
sipg_diag_kernel(Geom g, SipgArgs<T> a) {
  using S = SipgShape<T, D, N>;
  constexpr int ND = S::ND, NF = S::NF, EPB = S::EPB;
  __shared__ T sD[N * N];
  __shared__ T sw[N];
  __shared__ T snu[EPB][ND];
  const Tables<T>& tb = tab<T>(g);
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) sD[i] = tb.D[N][i];
  for (int i = threadIdx.x; i < N; i += blockDim.x) sw[i] = tb.w[N][i];
  const int le = threadIdx.x / ND;
  const int node = threadIdx.x % ND;
  const int e = blockIdx.x * EPB + le;
  const bool valid = e < g.ne;
  int el = 0;
  Geom gl = g;
  if (valid) gl = local_geom(g, e, el);
  if (valid) snu[le][node] = a.nu ? a.nu[(size_t)e * ND + node] : sipg_nu0(a, gl);
  __syncthreads();
  if (!valid) return;
  (void)NF;
  int ec[3];
  elem_coords(gl, el, ec);
  int id[3];
  id[0] = node % N;
  id[1] = (D > 1) ? (node / N) % N : 0;
  id[2] = (D > 2) ? node / (N * N) : 0;
  T hinv2[D];
  T jac = T(1);
  for (int k = 0; k < D; ++k) { hinv2[k] = T(2) / geom_h<T>(gl, k); jac *= geom_h<T>(gl, k) * T(0.5); }
  T Wq = jac;
  for (int k = 0; k < D; ++k) Wq *= sw[id[k]];
  const T nuq = snu[le][node];
  T diag = T(0);
  for (int k = 0; k < D; ++k) {
    int stride = 1;
    for (int j = 0; j < k; ++j) stride *= N;
    const int base = node - id[k] * stride;
    // volume: sum over the k-line of W_q nu_q (2/h D_{q,i})^2
    T Wrest = jac;
    for (int j = 0; j < D; ++j) if (j != k) Wrest *= sw[id[j]];
    T acc = T(0);
    for (int q = 0; q < N; ++q) {
      T dq = sD[q * N + id[k]] * hinv2[k];
      acc += Wrest * sw[q] * snu[le][base + q * stride] * dq * dq;
    }
    diag += acc;
    for (int side = 0; side < 2; ++side) {
      if (id[k] != (side ? N - 1 : 0)) continue;
      const int nb = neighbor(gl, ec, k, side ? 1 : -1);
      if (nb < 0 && geom_bc(g, k) != 1) continue;
      T Wf = jac / (geom_h<T>(gl, k) * T(0.5));
      for (int j = 0; j < D; ++j) if (j != k) Wf *= sw[id[j]];
      const T n = side ? T(1) : T(-1);
      const T dself = n * sD[id[k] * N + id[k]] * hinv2[k];   // d(e_j)/dn at its own face node
      const T pen = T(N * N) * T(0.5) * hinv2[k];
      if (nb >= 0) {
        int c[3] = {id[0], id[1], id[2]};
        c[k] = side ? 0 : N - 1;
        const int nn = c[0] + N * ((D > 1 ? c[1] : 0) + N * (D > 2 ? c[2] : 0));
        const T nun = a.nu ? a.nu[(size_t)nb * ND + nn] : sipg_nu0(a, gl);
        diag += -Wf * nuq * dself + Wf * pen * (nuq > nun ? nuq : nun);
        // one element across a periodic direction is its own neighbour: the face average of
        // the normal derivative then also holds this basis function's derivative at the
        // element's opposite end
        if (nb == e) diag += -Wf * nun * n * sD[(side ? 0 : N - 1) * N + id[k]] * hinv2[k];
      } else {
        diag += -T(2) * Wf * nuq * dself + Wf * T(2) * pen * nuq;
      }
    }
  }
  a.y[(size_t)e * ND + node] = a.alpha * Wq + sipg_beta(a, gl) * diag;
}

template <typename T, int D, int N>
static void launch_apply(const Geom& g, const SipgArgs<T>& a, cudaStream_t st) {
  if (D == 2 && sipg_apply_line(g, N, a, st) == 0) return;      // periodic constant viscosity
  if (D == 2 && !a.nu && a.ops) {
    using C = Sipg2cShape<N>;
    constexpr size_t sm = sipg2c_smem<T, N>();
    smem_limit_once((const void*)sipg2c_apply_kernel<T, N>, (int)sm);
    IMEX_COUNTED(sipg2c_apply_kernel<T, N><<<(g.ne + C::EPB - 1) / C::EPB, C::THREADS, sm, st>>>(g, a));
    return;
  }
  using S = SipgShape<T, D, N>;
  int blocks = (g.ne + S::EPB - 1) / S::EPB;
  IMEX_COUNTED(sipg_apply_kernel<T, D, N><<<blocks, S::THREADS, 0, st>>>(g, a));
}

template <typename T, int D, int N>
static void launch_apply3(const Geom& g, const SipgArgs<T>& a, cudaStream_t st) {
  if (sipg_apply_line(g, N, a, st) == 0) return;                 // periodic constant viscosity
  if (!a.nu && a.ops) {
    using C = Sipg3cShape<N>;
    constexpr size_t sm = sipg3c_smem<T, N>();
    smem_limit_once((const void*)sipg3c_apply_kernel<T, N>, (int)sm);
    IMEX_COUNTED(sipg3c_apply_kernel<T, N><<<(g.ne + C::EPB - 1) / C::EPB, C::THREADS, sm, st>>>(g, a));
    return;
  }
  using S = Sipg3Shape<N>;
  const int blocks = (g.ne + S::EPB - 1) / S::EPB;
  constexpr size_t smem = sipg3_smem<T, N>();
  if (a.nu) {
    smem_limit_once((const void*)sipg3_apply_kernel<T, N, true>, (int)smem);
    IMEX_COUNTED(sipg3_apply_kernel<T, N, true><<<blocks, S::THREADS, smem, st>>>(g, a));
  } else {
    smem_limit_once((const void*)sipg3_apply_kernel<T, N, false>, (int)smem);
    IMEX_COUNTED(sipg3_apply_kernel<T, N, false><<<blocks, S::THREADS, smem, st>>>(g, a));
  }
}

template <typename T, int D, int N>
static void launch_diag(const Geom& g, const SipgArgs<T>& a, cudaStream_t st) {
  using S = SipgShape<T, D, N>;
  int blocks = (g.ne + S::EPB - 1) / S::EPB;
  IMEX_COUNTED(sipg_diag_kernel<T, D, N><<<blocks, S::THREADS, 0, st>>>(g, a));
}

#define IMEX_DISPATCH_N(D, FN, ...)                 \
  switch (N) {                                      \
    case 2: FN<T, D, 2>(__VA_ARGS__); break;        \
    case 3: FN<T, D, 3>(__VA_ARGS__); break;        \
    case 4: FN<T, D, 4>(__VA_ARGS__); break;        \
    case 5: FN<T, D, 5>(__VA_ARGS__); break;        \
    case 6: FN<T, D, 6>(__VA_ARGS__); break;        \
    case 7: FN<T, D, 7>(__VA_ARGS__); break;        \
    case 8: FN<T, D, 8>(__VA_ARGS__); break;        \
    case 9: FN<T, D, 9>(__VA_ARGS__); break;        \
    default: return -1;                             \
  }

template <typename T>
int sipg_apply(const Geom& g, int N, const SipgArgs<T>& a, cudaStream_t st) {
  if (a.dot_out && (a.nu || !a.ops)) return -2;     // the fused dot exists on the constant-nu path only
  if (a.cheb && (a.nu || !a.ops || a.gdata)) return -3;  // so does the fused Chebyshev step
  if (g.d == 2) { IMEX_DISPATCH_N(2, launch_apply, g, a, st) }
  else { IMEX_DISPATCH_N(3, launch_apply3, g, a, st) }
  return 0;
}

template <typename T>
int sipg_diag(const Geom& g, int N, const SipgArgs<T>& a, cudaStream_t st) {
  if (g.d == 2) { IMEX_DISPATCH_N(2, launch_diag, g, a, st) }
  else { IMEX_DISPATCH_N(3, launch_diag, g, a, st) }
  return 0;
}

template int sipg_apply<double>(const Geom&, int, const SipgArgs<double>&, cudaStream_t);
template int sipg_apply<float>(const Geom&, int, const SipgArgs<float>&, cudaStream_t);
template int sipg_diag<double>(const Geom&, int, const SipgArgs<double>&, cudaStream_t);
template int sipg_diag<float>(const Geom&, int, const SipgArgs<float>&, cudaStream_t);

}  // namespace imex
