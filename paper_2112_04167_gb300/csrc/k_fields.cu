// Pointwise fields evaluated on the device at the GLL nodes: closed-form flows
// used as initial / boundary data (Sec. 4.1 traveling Taylor-Green vortex, the
// decaying 2D Taylor-Green vortex, the 3D Taylor-Green initial field of
// Sec. 4.3, the travelling vortex array of Sec. 4.2), viscosity laws (constant,
// nu(x, y, t), nu(|v|) of Sec. 4.2) and the manufactured forcing that makes the traveling
// vortex exact under nu(x, y, t) and the vortex array exact under nu(|v|).
#include <math.h>

#include "../../include/imex.h"
#include "common.cuh"
#include "kernels.h"

namespace imex {

__device__ void flow_velocity(int kind, const double* p, const double* X, double t, int d, double* out) {
  const double x = X[0], y = X[1], z = (d > 2) ? X[2] : 0.0;
  if (kind == IMEX_FLOW_TG2D) {
    const double F = exp(-2.0 * p[0] * t);
    out[0] = sin(x) * cos(y) * F;
    out[1] = -cos(x) * sin(y) * F;
    if (d > 2) out[2] = 0.0;
  } else if (kind == IMEX_FLOW_TG3D) {
    out[0] = sin(x) * cos(y) * cos(z);
    out[1] = -cos(x) * sin(y) * cos(z);
    if (d > 2) out[2] = 0.0;
  } else if (kind == IMEX_FLOW_TGTRAVEL) {
    const double tp = 2.0 * M_PI;
    const double a = tp * (x - t), b = tp * (y - 0.125 - t);
    const double F = exp(-8.0 * M_PI * M_PI * p[0] * t);
    out[0] = 1.0 + sin(a) * cos(b) * F;
    out[1] = 1.0 - cos(a) * sin(b) * F;
    if (d > 2) out[2] = 0.0;
  } else if (kind == IMEX_FLOW_VV && d == 3) {
    const double tp = 2.0 * M_PI;
    const double A = tp * (x + t), B = tp * (y + t), C = tp * (z + t);
    out[0] = (sin(A) + cos(B)) * sin(C);
    out[1] = (cos(A) + sin(B)) * sin(C);
    out[2] = (cos(A) + cos(B)) * cos(C);
  } else {
    for (int c = 0; c < d; ++c) out[c] = 0.0;
  }
}

__device__ double viscosity(int kind, const double* p, const double* X, double t, const double* v, int d) {
  if (kind == IMEX_NU_VARXYT) {
    const double tp = 2.0 * M_PI;
    return p[0] * (1.0 + 0.5 * sin(tp * X[0]) * sin(tp * X[1]) * cos(t));
  }
  if (kind == IMEX_NU_VELOCITY) {
    double m2 = 0.0;
    for (int c = 0; c < d; ++c) m2 += v[c] * v[c];
    return p[0] + p[1] * m2 / (p[2] * p[2]);
  }
  return p[0];
}

// f = (nu0 - nu) lap v - (grad v + grad v^T) grad nu for the traveling vortex, nu = nu(x, y, t)
__device__ void forcing_tgtravel_varnu(const double* p, const double* X, double t, double* f) {
  const double nu0 = p[0];
  const double tp = 2.0 * M_PI;
  const double x = X[0], y = X[1];
  const double a = tp * (x - t), b = tp * (y - 0.125 - t);
  const double F = exp(-8.0 * M_PI * M_PI * nu0 * t);
  const double sa = sin(a), ca = cos(a), sb = sin(b), cb = cos(b);
  const double vx = sa * cb * F, vy = -ca * sb * F;      // oscillating parts
  const double lapx = -8.0 * M_PI * M_PI * vx, lapy = -8.0 * M_PI * M_PI * vy;
  const double nu = nu0 * (1.0 + 0.5 * sin(tp * x) * sin(tp * y) * cos(t));
  const double cgn = 0.5 * nu0 * cos(t) * tp;
  const double gnx = cgn * cos(tp * x) * sin(tp * y), gny = cgn * sin(tp * x) * cos(tp * y);
  const double G00 = tp * ca * cb * F, G01 = -tp * sa * sb * F;
  const double G10 = tp * sa * sb * F, G11 = -tp * ca * cb * F;
  f[0] = (nu0 - nu) * lapx - (gnx * (G00 + G00) + gny * (G01 + G10));
  f[1] = (nu0 - nu) * lapy - (gnx * (G10 + G01) + gny * (G11 + G11));
}

// f = d_t v + (grad v) v - nu lap v - (grad v + grad v^T) grad nu + grad p for the vortex array
// of Sec. 4.2 (solenoidal, so div(v v) = (grad v) v and div(grad v^T) = 0), nu = nu(|v|):
// every argument is x_k + t, so d_t v_c = sum_k dv_c/dx_k, and lap v = -2 (2 pi)^2 v
__device__ void forcing_vv(const double* p, const double* X, double t, double* f) {
  const double nu0 = p[0], nu1 = p[1], vm = p[2];
  const double k = 2.0 * M_PI;
  const double A = k * (X[0] + t), B = k * (X[1] + t), C = k * (X[2] + t);
  const double sA = sin(A), cA = cos(A), sB = sin(B), cB = cos(B), sC = sin(C), cC = cos(C);
  const double v[3] = {(sA + cB) * sC, (cA + sB) * sC, (cA + cB) * cC};
  const double G[3][3] = {{k * cA * sC, -k * sB * sC, k * (sA + cB) * cC},
                          {-k * sA * sC, k * cB * sC, k * (cA + sB) * cC},
                          {-k * sA * cC, -k * sB * cC, -k * (cA + cB) * sC}};
  const double gp[3] = {k * cA * sB * sC, k * sA * cB * sC, k * sA * sB * cC};
  const double nu = nu0 + nu1 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) / (vm * vm);
  double gnu[3];
  for (int i = 0; i < 3; ++i) gnu[i] = 2.0 * nu1 / (vm * vm) * (v[0] * G[0][i] + v[1] * G[1][i] + v[2] * G[2][i]);
  for (int c = 0; c < 3; ++c) {
    double r = G[c][0] + G[c][1] + G[c][2] + 2.0 * k * k * nu * v[c] + gp[c];
    for (int i = 0; i < 3; ++i) r += v[i] * G[c][i] - (G[c][i] + G[i][c]) * gnu[i];
    f[c] = r;
  }
}

// nodal evaluation of a closed-form flow, viscosity law or forcing (Sec. 4)
template <int D, int N>
__global__ void field_kernel(Geom g, int what, FieldSpec fs, double t, const double* __restrict__ v,
                             long long stride, double* __restrict__ out) {
  constexpr int ND = ipow(N, D);
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= (size_t)g.ne * ND) return;
  const int e = (int)(idx / ND), node = (int)(idx % ND);
  int el = 0;
  const Geom gl = local_geom(g, e, el);
  int ec[3];
  elem_coords(gl, el, ec);
  int id[3] = {node % N, (D > 1) ? (node / N) % N : 0, (D > 2) ? node / (N * N) : 0};
  const double* xi = tab<double>(g).x[N];
  double X[3] = {0, 0, 0};
  for (int k = 0; k < D; ++k) X[k] = gl.lo[k] + (ec[k] + 0.5 * (xi[id[k]] + 1.0)) * gl.h[k];
  // batched meshes: the instance's own parameters, and t read as a fraction of its time step
  if (g.inst) {
    const InstGeom& I = g.inst[g.elem_inst[e]];
    const double* ip = what == 0 ? I.bc_p : (what == 1 ? I.nu_p : I.f_p);
    for (int j = 0; j < 8; ++j) fs.p[j] = ip[j];
    t = I.t + t * I.dt;
  }
  if (what == 0) {
    double u[3];
    flow_velocity(fs.kind, fs.p, X, t, D, u);
    for (int c = 0; c < D; ++c) out[(size_t)c * stride + idx] = u[c];
  } else if (what == 1) {
    double u[3] = {0, 0, 0};
    if (v) for (int c = 0; c < D; ++c) u[c] = v[(size_t)c * stride + idx];
    out[idx] = viscosity(fs.kind, fs.p, X, t, u, D);
  } else {
    double f[3] = {0, 0, 0};
    if (fs.kind == IMEX_FORCE_TGTRAVEL_VARNU && D == 2) forcing_tgtravel_varnu(fs.p, X, t, f);
    if (fs.kind == IMEX_FORCE_VV && D == 3) forcing_vv(fs.p, X, t, f);
    for (int c = 0; c < D; ++c) out[(size_t)c * stride + idx] = f[c];
  }
}

template <int D, int N>
static void launch_field(const Geom& g, int what, const FieldSpec& fs, double t, const double* v,
                         long long stride, double* out, cudaStream_t st) {
  const size_t n = (size_t)g.ne * ipow(N, D);
  IMEX_COUNTED(field_kernel<D, N><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, what, fs, t, v, stride, out));
}

int eval_field(const Geom& g, int N, int what, const FieldSpec& fs, double t, const double* v,
               long long stride, double* out, cudaStream_t st) {
#define IMEX_FIELD_CASE(DD, NN) \
  if (g.d == DD && N == NN) { launch_field<DD, NN>(g, what, fs, t, v, stride, out, st); return 0; }
  IMEX_FIELD_CASE(2, 3) IMEX_FIELD_CASE(2, 4) IMEX_FIELD_CASE(2, 5) IMEX_FIELD_CASE(2, 6)
  IMEX_FIELD_CASE(2, 7) IMEX_FIELD_CASE(2, 8) IMEX_FIELD_CASE(2, 9)
  IMEX_FIELD_CASE(3, 3) IMEX_FIELD_CASE(3, 4) IMEX_FIELD_CASE(3, 5) IMEX_FIELD_CASE(3, 6)
  IMEX_FIELD_CASE(3, 7) IMEX_FIELD_CASE(3, 8) IMEX_FIELD_CASE(3, 9)
#undef IMEX_FIELD_CASE
  return -1;
}

}  // namespace imex
