/*
 * imex.h -- C ABI of the GB300 IMEX Runge-Kutta / SDC incompressible-flow library.
 *
 * The library advances the incompressible Navier-Stokes equations with variable
 * viscosity (paper Sec. 3.1, Eqs. momentum / continuity / ic / bc) by the
 * projection-based IMEX Runge-Kutta method of Alg. 3 (Sec. 3.2.2) or the
 * semi-implicit SDC method of Alg. 4 (Sec. 3.2.3), on a DG spectral-element mesh
 * of a Cartesian box (Sec. 3.3): tensor-product GLL bases of degree P for the
 * velocity and P-1 for the pressure, over-integrated convection with local
 * Lax-Friedrichs fluxes, symmetric interior penalty (SIPG) operators for the
 * pressure and viscous problems, each solved by preconditioned CG (Jacobi, or p-multigrid
 * for the pressure).
 *
 * Conventions shared by every call
 *   - Layout: a scalar field is N_e * (P+1)^d doubles (pressure: N_e * P^d),
 *     element-major with elements numbered x fastest, nodes lexicographic with x
 *     fastest inside each element; a vector field is d such blocks, component-major.
 *   - Pointers: `on_device` = 1 means the pointer is CUDA device memory (e.g. a
 *     torch tensor's data_ptr()) usable on the context's stream; 0 means host memory.
 *     Caller buffers are only borrowed for the duration of the call.
 *   - Ownership: the context owns all of its device state; imex_destroy frees it.
 *   - Errors: every call returns an imex_status; no C++ exception crosses the ABI.
 *     imex_last_error() gives a human-readable message for the last failure.
 *   - Threads: one context must not be used from two host threads at once.
 *   - Environment switches (read once; none changes a result beyond rounding):
 *       IMEX_REFINE_DECADES=1..5  decades of FP32 residual decrease between FP64
 *                                 residual replacements (mixed forms; default 4 with the
 *                                 V-cycle, 2 with Jacobi)
 *       IMEX_PMG_CLUSTER=0        one launch per coarsest-level smoothing step instead of
 *                                 the single-cluster kernel
 *       IMEX_TUNE=0               default launch shapes, no timing of the alternatives
 *       IMEX_PERSIST=1            the persistent-kernel FP32 Jacobi pressure CG (measured
 *                                 slower than the graph-replayed iteration kernels)
 *       IMEX_PDL=1                CG loop kernels launched with programmatic dependent
 *                                 launch
 *       IMEX_BATCH_SERIAL=1       the groups of a batch stepped one after the other from the
 *                                 calling thread instead of one host thread per group
 *       IMEX_DEBUG=1              one stderr line per FP64 residual replacement
 */
#ifndef IMEX_GB300_H
#define IMEX_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct imex_ctx imex_ctx;

typedef enum {
  IMEX_OK = 0,
  IMEX_EINVAL = 1,     /* invalid argument: mesh, tableau (not CK-form), sizes, kinds */
  IMEX_ENOMEM = 2,     /* device allocation failed */
  IMEX_ENOTCONV = 3,   /* a linear solve reached maxit without meeting its tolerance */
  IMEX_EUNSTABLE = 4,  /* NaN/Inf or |v| above the instability threshold (Sec. 4.2.3) */
  IMEX_ECUDA = 5       /* a CUDA runtime call failed */
} imex_status;

/* arithmetic of the solves */
/* IMEX_FP64: every operator and solve in FP64.
   IMEX_MIXED: FP32 inner iterations of the Poisson and Helmholtz solves with FP64 refinement
     (true residual, iterate); stage storage and combinations in FP64, the convective
     operator on FP64 fields in float-float arithmetic (about 48 significant bits, on the
     FP32 pipes) -- the result matches IMEX_FP64 to the solver tolerance.
   IMEX_MIXED_FAST: IMEX_MIXED plus FP32 explicit operators (convection, F_d1) on FP32 copies
     of the state; adds an FP32 rounding error of about 1e-8 relative per step. */
enum { IMEX_FP64 = 0, IMEX_MIXED = 1, IMEX_MIXED_FAST = 2 };
/* pressure operator: SIPG on Q_{P-1} (Sec. 3.3), or B M^-1 B^T (discretely divergence-free) */
enum { IMEX_POISSON_SIPG = 0, IMEX_POISSON_CONSISTENT = 1 };
/* closed-form flows (initial / Dirichlet data); params[0] = nu_0.  IMEX_FLOW_VV: the
   travelling 3D vortex array of Sec. 4.2, Eq. (var-visc-test) (no parameters) */
enum { IMEX_FLOW_NONE = 0, IMEX_FLOW_TG2D = 1, IMEX_FLOW_TG3D = 2, IMEX_FLOW_TGTRAVEL = 3, IMEX_FLOW_VV = 4 };
/* viscosity laws: params {nu_0}; {nu_0} for nu0(1 + sin 2pi x sin 2pi y cos t / 2);
   {nu_0, nu_1, v_max} for nu_0 + nu_1 (|v|/v_max)^2 (Sec. 4.2); nodal field */
enum { IMEX_NU_CONST = 0, IMEX_NU_VARXYT = 1, IMEX_NU_VELOCITY = 2, IMEX_NU_FIELD = 3 };
/* forcing: none, the manufactured forcing of the traveling vortex under IMEX_NU_VARXYT, or
   the forcing of Eq. (var-visc-test:rhs) that makes the vortex array exact under the
   velocity-dependent viscosity (params {nu_0, nu_1, v_max}, 3D) */
enum { IMEX_FORCE_NONE = 0, IMEX_FORCE_TGTRAVEL_VARNU = 1, IMEX_FORCE_VV = 2 };
/* operator spaces of imex_op_sipg */
enum { IMEX_SPACE_VELOCITY = 0, IMEX_SPACE_PRESSURE = 1 };
/* arithmetic of the operator-level entry points (argument `arith`): FP64 kernels; FP32
   kernels on inputs rounded to FP32 (the inner CG iterations of IMEX_MIXED and the explicit
   operators of IMEX_MIXED_FAST); float-float kernels on FP64 fields (the FP64-class operators
   of IMEX_MIXED).  Results are always returned in FP64.  IMEX_ARITH_FP32 equals IMEX_MIXED. */
enum { IMEX_ARITH_FP64 = 0, IMEX_ARITH_FP32 = 1, IMEX_ARITH_FF = 3 };

typedef struct {
  int dim;              /* 2 or 3 */
  int P;                /* velocity degree, 2 <= P <= 8; pressure degree P-1 */
  int nelem[3];         /* elements per direction (nelem[2] ignored for dim 2) */
  double lo[3], hi[3];  /* box corners */
  int periodic[3];      /* 1 periodic; 0: Dirichlet velocity / Neumann pressure on both ends */
  int precision;        /* IMEX_FP64, IMEX_MIXED or IMEX_MIXED_FAST */
  int poisson;          /* IMEX_POISSON_SIPG or IMEX_POISSON_CONSISTENT */
  double tol;           /* relative residual tolerance of every solve, ||r|| <= tol ||b|| (Sec. 4 uses 1e-12) */
  int maxit;            /* CG iteration limit per (inner) solve */
  double inner_tol;     /* IMEX_MIXED: FP32 inner-solve tolerance (0: default 1e-5) */
  double vmax;          /* instability threshold on max |v| (0: no threshold, NaN still detected) */
  void* stream;         /* cudaStream_t to run on, or NULL for a private stream */
} imex_mesh_desc;

typedef struct {
  long long steps;           /* completed steps */
  long long stages;          /* nontrivial stages (substeps) completed */
  int poisson_solves, helmholtz_solves;   /* of the last imex_step call */
  long long poisson_iters, helmholtz_iters; /* CG iterations (inner iterations in IMEX_MIXED) */
  int refinements;           /* FP64 refinement sweeps (IMEX_MIXED) */
  double max_poisson_res;    /* largest final relative residual, last call */
  double max_helmholtz_res;
  double div_norm;           /* RMS of the weak divergence B v - (n.v_b) after the last projection */
  double max_velocity;       /* max |v_c| after the last step */
  double last_call_ms;       /* wall time of the last imex_step call (host clock, synchronised) */
} imex_stats;

/* Create a context: allocates the device state of one flow instance (Sec. 3.3 discretisation).
   Returns IMEX_EINVAL for an unsupported mesh (dim, P range, nelem < 1) and IMEX_ENOMEM if
   the device state does not fit.  The default method is RK-CB3e, nu = 0, no forcing. */
imex_status imex_create(const imex_mesh_desc* desc, imex_ctx** out);
/* frees every device and pinned host buffer of the context after its stream has finished
   (NULL: nothing) */
void imex_destroy(imex_ctx* ctx);
/* message of the context's last failed call; owned by the context, valid until its next
   call */
const char* imex_last_error(const imex_ctx* ctx);
/* velocity nodes per component, N_e (P+1)^d, and pressure nodes, N_e P^d (the Q_P / Q_{P-1}
   pair of Sec. 3.3) */
imex_status imex_sizes(const imex_ctx* ctx, long long* nvel, long long* npres);

/* IMEX RK tableau in the CK form of Eq. (imex-rk:butcher), row-major s x s arrays:
   requires c_1 = 0, a^IM_11 = 0, A^IM lower triangular, A^EX strictly lower triangular,
   row sums equal to c (to 1e-10).  Otherwise IMEX_EINVAL. */
imex_status imex_set_tableau(imex_ctx* ctx, int s, const double* c, const double* AI,
                             const double* bI, const double* AE, const double* bE);
/* The six tableaux of the paper's appendix by name: "TR", "CB2", "CB3c", "CB3e", "CB4",
   "ARS3", and "EULER" (IMEX Euler).  Selects RK stepping. */
imex_status imex_set_tableau_named(imex_ctx* ctx, const char* name);
/* SISDC of Sec. 3.2.3 with M subintervals on GLL nodes, K correction sweeps and the named
   predictor tableau ("EULER" for SDC-Eu).  Selects SDC stepping. */
imex_status imex_set_sdc(imex_ctx* ctx, int M, int K, const char* predictor);
/* IMEX BDF2 of Sec. 3.2.1 (Eq. (bdf2:variable-nu) with the splitting into extrapolation,
   projection, diffusion with the extrapolated viscosity and, for variable viscosity, an
   additional projection).  Not self-starting: the first step after this call, after
   imex_set_state / imex_init_flow, or after a change of dt is an IMEX Euler step.  Selects
   BDF2 stepping (one nontrivial substep per step); imex_set_tableau* / imex_set_sdc switch
   back.  Batches reject BDF2 contexts (IMEX_EINVAL). */
imex_status imex_set_bdf2(imex_ctx* ctx);

/* Divergence / mass-flux stabilisation after every stage projection (Sec. 3.3 adds one "for
   pressure robustness" without stating its form).  This library's reading, the penalised
   projection: the projected velocity v'' is replaced by v~ solving
     (M + A_D + A_C) v~ = M v'',
   A_D = sum_K tau_D,K B_K^T W_K B_K with tau_D,K = zeta_d |u_K| h_K / (P + 1) dt (B_K the
   element-local divergence at the GLL nodes, W_K the GLL weights, |u_K| the magnitude of the
   element's mean velocity, h_K the geometric mean element size, dt the step), and
   A_C = sum_F tau_C,F J_F^T W_F J_F with tau_C,F = zeta_c (|u_K-| + |u_K+|) / 2 dt (J_F the jump
   of the normal velocity component across an interior face).  Solved by CG to the context's
   tolerance.  zeta_d = zeta_c = 0 (the default) switches it off; batches reject it. */
imex_status imex_set_stabilization(imex_ctx* ctx, double zeta_d, double zeta_c);
/* out = v~ of the stabilisation above applied to the velocity v (d blocks) with time step dt;
   IMEX_EINVAL while the stabilisation is off */
imex_status imex_stabilize(imex_ctx* ctx, const double* v, double dt, double* out, int on_device);
/* The viscosity nu(x, t, v) of Eq. (momentum), Sec. 3.1.  Constant: nu >= 0 (IMEX_EINVAL
   otherwise).  Model: IMEX_NU_CONST {nu_0}; IMEX_NU_VARXYT {nu_0}, the nu(x, y, t) of the
   manufactured flow of Sec. 4.1; IMEX_NU_VELOCITY {nu_0, nu_1, v_max}, the law of Sec. 4.2,
   treated semi-implicitly as Alg. 2 / Alg. 3 prescribe (stage viscosities from the projected
   velocities).  IMEX_EINVAL for another kind, more than 8 parameters or v_max <= 0. */
imex_status imex_set_viscosity_const(imex_ctx* ctx, double nu);
imex_status imex_set_viscosity_model(imex_ctx* ctx, int kind, const double* params, int nparams);
/* nodal viscosity field (nvel doubles, used as a fixed nu(x) in Eq. (momentum)); copied into
   the context; IMEX_EINVAL for a NULL field */
imex_status imex_set_viscosity_field(imex_ctx* ctx, const double* nu, int on_device);
/* Dirichlet data v_b(x, t) of Eq. (bc) on non-periodic boundaries: a closed-form flow
   (IMEX_FLOW_*, at most 8 parameters), evaluated on the device at every stage time; a
   non-periodic mesh needs it before imex_step.  IMEX_EINVAL for an unknown kind. */
imex_status imex_set_boundary(imex_ctx* ctx, int kind, const double* params, int nparams);
/* forcing f of Eq. (momentum): IMEX_FORCE_* with its parameters, evaluated on the device at
   every stage time (F_s of Alg. 3).  IMEX_EINVAL for an unknown kind or a forcing of the
   other dimension (IMEX_FORCE_TGTRAVEL_VARNU is 2D, IMEX_FORCE_VV 3D). */
imex_status imex_set_forcing(imex_ctx* ctx, int kind, const double* params, int nparams);

/* the initial condition of Eq. (ic): velocity state (d * nvel doubles, layout above) at time
   t, copied into the context; restarts BDF2 with its Euler step */
imex_status imex_set_state(imex_ctx* ctx, double t, const double* v, int on_device);
/* the initial condition of Eq. (ic) from a closed-form flow of Sec. 4 evaluated on the device
   at time t (IMEX_FLOW_TG3D: Eq. (transition:v0) at the shifted point; IMEX_FLOW_VV: Eq.
   (var-visc-test)); IMEX_EINVAL for an unknown kind */
imex_status imex_init_flow(imex_ctx* ctx, int kind, const double* params, int nparams, double t);

/* Advance nsteps steps of size dt (Alg. 3 per step, or Alg. 4 after imex_set_sdc).
   IMEX_ENOTCONV: a solve hit maxit (state left at the failing stage, stats filled);
   IMEX_EUNSTABLE: NaN or max |v| > vmax after a step. */
imex_status imex_step(imex_ctx* ctx, double dt, int nsteps);

/* the velocity v of Eq. (momentum) at the context's time (d * nvel doubles, layout above) */
imex_status imex_get_velocity(imex_ctx* ctx, double* out, int on_device);
/* psi'' of the last stage projection (Alg. 3 / Alg. 4), mass-weighted mean removed */
imex_status imex_get_pressure(imex_ctx* ctx, double* out, int on_device);
/* the context's time t^n */
imex_status imex_get_time(const imex_ctx* ctx, double* t);
/* solver statistics of the last imex_step call (iterations, the final relative residuals
   ||r|| / ||b|| of Sec. 4's stopping rule) and counters since creation; every call returns
   IMEX_EINVAL for NULL arguments */
imex_status imex_get_stats(const imex_ctx* ctx, imex_stats* out);

/* ---- operator-level entry points (same discretisation, for composition and testing) ---- */

/* The SIPG operator of Sec. 3.3 (F_d1 = -M^{-1}(A(nu) v - r_b(v_b)) of Alg. 3, the Helmholtz
   operator of its implicit stage, the pressure operator of its projection):
   y = alpha M x + beta (A(nu) x - r_b(g)), optionally multiplied by M^{-1} (minv = 1).
   space: IMEX_SPACE_VELOCITY (degree P, Dirichlet faces on non-periodic sides, nsys
   components) or IMEX_SPACE_PRESSURE (degree P-1, nu = 1, Neumann faces, nsys = 1).
   nu: nodal viscosity (velocity space) or NULL for the context's constant viscosity.
   g: Dirichlet data, nsys blocks, or NULL for homogeneous data.  arith: IMEX_ARITH_* (the
   float-float kernel exists for the periodic 3D constant-viscosity operator only: IMEX_EINVAL
   for any other case). */
imex_status imex_op_sipg(imex_ctx* ctx, int space, const double* x, double* y, int nsys, double alpha,
                         double beta, const double* nu, const double* g, int minv, int arith,
                         int on_device);
/* diagonal of alpha M + beta A(nu) (the Jacobi preconditioner), one block */
imex_status imex_op_sipg_diag(imex_ctx* ctx, int space, double* y, double alpha, double beta,
                              const double* nu, int on_device);
/* The four operators below take `arith` = IMEX_ARITH_FP64 or IMEX_ARITH_FF (float-float on
   FP64 fields, the form IMEX_MIXED steps with); imex_op_conv also IMEX_ARITH_FP32 (the
   convection of IMEX_MIXED_FAST).  Other values: IMEX_EINVAL. */
/* the right-hand side of the projection's Poisson problem (Alg. 3, Sec. 3.3):
   b = B v - int_{dOmega} (n . w) q: mode 0 no boundary term, 1 w = wdata, 2 w = v (trace) */
imex_status imex_op_div(imex_ctx* ctx, const double* v, const double* wdata, int mode, double* b,
                        int arith, int on_device);
/* the projection's correction v'' = v' - grad psi of Alg. 3 uses out = M^{-1} B^T psi (DG
   gradient of a pressure field, d blocks) */
imex_status imex_op_grad(imex_ctx* ctx, const double* psi, double* out, int arith, int on_device);
/* the convective term of Eq. (momentum) as Sec. 3.3 discretises it: out = F_c(v) =
   -M^{-1} div(v v) with the local Lax-Friedrichs flux and over-integration on Gauss points;
   vb: Dirichlet data (d blocks) or NULL */
imex_status imex_op_conv(imex_ctx* ctx, const double* v, const double* vb, double* out, int arith,
                         int on_device);
/* the parts of the viscous term of Sec. 3.2 that Alg. 3 treats explicitly: out = F_d3 =
   -grad(nu div v) and, if out2 != NULL, out2 = F_d2 = div(nu (grad v)^T) */
imex_status imex_op_graddiv(imex_ctx* ctx, const double* v, const double* nu, double* out_fd3,
                            double* out_fd2, int arith, int on_device);
/* Preconditioner of the pressure Poisson solves (Sec. 3.3 solves them by preconditioned CG;
   its preconditioners are not described there): IMEX_PRECOND_JACOBI, or IMEX_PRECOND_PMG --
   one p-multigrid V-cycle per CG iteration over the pressure degrees P-1, halved down to 1
   on the same mesh, with the SIPG pressure operator rediscretised on every level,
   element-local GLL interpolation between levels (restriction: its transpose), Chebyshev-
   accelerated Jacobi smoothing before and after each coarse correction and a fixed
   Chebyshev polynomial on the degree-1 level.  params (nparams <= 4, optional): smoothing
   steps (default 3), steps on the coarsest level (10), smoothing range lmax / lmin (10),
   coarsest range (100).  Default: IMEX_PRECOND_PMG.  The IMEX_POISSON_CONSISTENT operator
   always uses Jacobi.  In the mixed forms the degree-1 level of a single 3D periodic mesh
   runs all its steps in one launch on one thread-block cluster (up to about 15,000
   elements); IMEX_PMG_CLUSTER=0 in the environment keeps one launch per step.  The mixed
   forms replace the FP32 recursion's residual by the FP64 one every four decades with the
   V-cycle, every two with Jacobi (IMEX_REFINE_DECADES=1..5 in the environment sets both).
   IMEX_EINVAL for an unknown kind or parameters out of range. */
enum { IMEX_PRECOND_JACOBI = 0, IMEX_PRECOND_PMG = 1 };
imex_status imex_set_pressure_precond(imex_ctx* ctx, int kind, const double* params, int nparams);
/* the V-cycle's levels (set up on first use): their number (<= 4), points per direction
   N[l] (finest first) and the upper ends lmax[l] of the Chebyshev intervals -- 1.15 times a
   40-step power-iteration estimate of the largest eigenvalue of D^{-1} A on the level.
   Output arrays of 4 entries; any pointer may be NULL. */
imex_status imex_pmg_info(imex_ctx* ctx, int* nlev, int* N, double* lmax);
/* z = one V-cycle applied to r (pressure space, np doubles each), in FP64 or FP32 arithmetic
   (arith IMEX_ARITH_FP64 / IMEX_ARITH_FP32); lmax: the upper ends of the Chebyshev intervals
   to use instead of the context's (nlev entries), or NULL. */
imex_status imex_op_pmg_vcycle(imex_ctx* ctx, const double* r, double* z, const double* lmax, int arith,
                               int on_device);
/* the projection's Poisson solve of Alg. 3: L psi = b - mean(b) with the context's pressure
   operator and preconditioner; psi mean-free; IMEX_ENOTCONV at maxit */
imex_status imex_solve_poisson(imex_ctx* ctx, const double* b, double* psi, int on_device);
/* the implicit viscous solve of an Alg. 3 stage: (M + gamma A(nu)) v = M g + gamma
   r_b(nu, vb) for all d components (gamma = dt a^IM_ii); IMEX_ENOTCONV at maxit */
imex_status imex_solve_helmholtz(imex_ctx* ctx, const double* g, const double* nu, double gamma,
                                 const double* vb, double* v, int on_device);
/* nodal evaluation: what 0 flow velocity (kind IMEX_FLOW_*), 1 viscosity law (IMEX_NU_*, v may
   be given), 2 forcing (IMEX_FORCE_*) at time t */
imex_status imex_eval_field(imex_ctx* ctx, int what, int kind, const double* params, int nparams,
                            double t, const double* v, double* out, int on_device);

/* ---- flow statistics of Sec. 4.3 (of the current velocity; single contexts only) ------ */
/* viscous dissipation rate eps = (1 / |Omega|) int nu grad v : grad v dOmega (the paper's
   nu / (8 pi^3) int grad v : grad v on [-pi, pi]^3), with the element-local gradient of the
   DG velocity and the GLL quadrature of its nodes; nu: the context's viscosity law at the
   current time and velocity */
imex_status imex_dissipation(imex_ctx* ctx, double* eps);
/* energy spectrum E[k], k = 0..kmax-1 (host array): the velocity interpolated to a regular
   grid of M points per direction (M a power of two, 2..1024; x_j = lo + j L / M, evaluated by
   the element containing it), a discrete Fourier transform normalised by M^-d, and
   E(k) = |Omega| / 2 sum |v^(n)|^2 over the integer wave vectors with k - 1/2 <= |n| < k + 1/2,
   so that the shells add up to the grid's kinetic energy ~ 1/2 int |v|^2.  The device
   scratch (d M^d complex values) is kept by the context. */
imex_status imex_energy_spectrum(imex_ctx* ctx, int M, int kmax, double* E);

/* ---- reductions (FP64 accumulation, deterministic two-level sums) -------------------- */
enum { IMEX_REDUCE_DOT = 0, IMEX_REDUCE_SUM = 1, IMEX_REDUCE_MAXABS = 2 };
/* *out (host) = sum_i x_i y_i (DOT), sum_i x_i (SUM) or max_i |x_i| (MAXABS; NaN if any x_i
   is NaN) over n doubles; y is used by DOT only.  With on_device = 0 the inputs are host
   arrays staged through the context, which needs n <= d * nvel (else IMEX_EINVAL).  These are
   the reductions behind the solver tolerances, the pressure mean and the instability check
   (Sec. 4: RMS residuals; Sec. 4.2.3: |v| threshold / NaN). */
imex_status imex_reduce(imex_ctx* ctx, int op, const double* x, const double* y, long long n,
                        double* out, int on_device);

/* Allocation-free form of imex_reduce, for callers that cannot allocate device memory
   at call time: code running while another framework's memory pool owns the device,
   hot loops where a cudaMalloc would synchronise the device, embedded or real-time
   hosts that forbid allocation after start-up.  There is no counterpart in the paper.
   x, y: device pointers (n doubles, FP64), out: host pointer to one double, stream: a
   cudaStream_t or NULL.  It needs no context and calls no cudaMalloc / cudaFree: its
   partial sums live in one fixed device array of 65,536 + 32 doubles (about 512 KB) that
   every GPU which loads this library holds until the process exits.
   Limit: n <= 16,777,216 (= 256 x 65,536); larger n returns IMEX_EINVAL without touching
   the GPU.  The first call on each device looks up the array's device address
   (cudaGetSymbolAddress); make that first call before any stream capture.  Every call
   rewrites the partial sums it reads before reading them, so nothing has to be cleared,
   and the array keeps the last call's contents.  All calls share the one array: calls
   that overlap on the GPU (different streams or threads) race on it and must be
   serialised by the caller.  The result is returned after a stream synchronisation. */
imex_status imex_reduce_noalloc(int op, const double* x, const double* y, long long n, double* out,
                                void* stream);

/* ---- instrumentation ---------------------------------------------------------------- */

/* kernel classes timed by imex_profile: the operator applies (CG applies of the pressure and
   Helmholtz solves, FP32 inner / FP64-class), the convection, the p-multigrid V-cycle (level
   applies; smoother vector updates and transfers), the CG vector kernels (step: x, r and the
   residual sums; direction: p and the preconditioned-residual scalars), and the projection's
   divergence and gradient and the grad-div derivatives */
enum {
  IMEX_PROF_PRESSURE_F32 = 0, IMEX_PROF_PRESSURE_F64 = 1, IMEX_PROF_HELMHOLTZ_F32 = 2,
  IMEX_PROF_HELMHOLTZ_F64 = 3, IMEX_PROF_CONV = 4,
  IMEX_PROF_PCG_PERSIST = 5,   /* persistent FP32 pressure CG launches (many iterations each) */
  IMEX_PROF_PMG_APPLY = 6, IMEX_PROF_PMG_VEC = 7, IMEX_PROF_CG_STEP = 8, IMEX_PROF_CG_DIR = 9,
  IMEX_PROF_DIV = 10, IMEX_PROF_GRAD = 11, IMEX_PROF_DERIV = 12,
  IMEX_PROF_PMG_APPLY_COARSE = 13,   /* the V-cycle's applies on the coarser levels (PMG_APPLY: finest) */
  IMEX_PROF_NCLASS = 14
};
/* enable (1) or disable (0) CUDA-event timing of the classes above on the context's
   stream; enabling resets the accumulated records */
imex_status imex_profile(imex_ctx* ctx, int enable);
/* launches and summed device time (ms) of one class since imex_profile(ctx, 1) */
imex_status imex_profile_read(imex_ctx* ctx, int cls, long long* launches, double* total_ms);
/* algorithmic work of those launches: bytes (every input read once, every output written
   once, in the arithmetic's storage type) and floating-point operations (FP64-equivalent for
   float-float), and the arithmetic (IMEX_ARITH_*) of the last launch (-1: none) */
imex_status imex_profile_work(imex_ctx* ctx, int cls, double* bytes, double* flops, int* arith);
/* Launch shapes chosen by the tuner of the periodic constant-viscosity SIPG applies (the CG
   and p-multigrid applies): on first use for a (d, N, precision, element count) each shape --
   the default elements per block (0), half (1), twice (2; not for 2D FP64), one more (3; 3D
   FP32 with N = 7 or 9) -- is timed with CUDA events and the fastest kept when it beats the default by
   more than 3% (IMEX_TUNE=0 in the environment: always the default).  Entry i: dimension,
   points per direction, FP32 (1) or FP64, elements, the chosen shape and the per-launch
   times (us) of the four shapes (us holds 4 values; 0: not timed).  Returns the number of
   entries (i < 0: just that), -1 for i out of range. */
int imex_tuning_info(int i, int* d, int* N, int* fp32, long long* ne, int* variant, double* us);
/* fix the launch shape for a (d, N, precision, element count) instead of the tuner's choice
   (also used by the operator entry points); IMEX_EINVAL for an unknown shape */
int imex_set_apply_variant(int d, int N, int fp32, long long ne, int variant);
/* kernels launched by this library so far, all contexts */
long long imex_launch_count(void);

/* ---- Batches of instances ---------------------------------------------------------------
 * Many independent instances advanced together (the ensemble and serving forms of the
 * per-stage work of Alg. 3).  imex_batch_create groups the given contexts by everything that
 * is not per-instance (d, P, periodicity, precision, solver settings, model kinds, tableau);
 * each group becomes one union mesh whose operators run as one launch over all its
 * instances and whose CG systems (each instance's pressure, each velocity component of
 * each instance) advance together with per-system step lengths and convergence tests.
 * Per instance: mesh box and element counts, viscosity and model parameters, time, time
 * step.  The batch copies the instances' current velocity, pressure and time at creation
 * and owns the stepped state from then on; the instance contexts are not modified and may
 * be destroyed.  RK tableaux only (SDC contexts and IMEX_NU_FIELD viscosity: IMEX_EINVAL).
 * Errors of a group (IMEX_ENOTCONV, IMEX_EUNSTABLE) are returned by imex_batch_step with the
 * group named in imex_batch_last_error; the other groups still complete their steps. */
typedef struct imex_batch imex_batch;
/* insts: n contexts (borrowed for the call); out: the new batch. */
imex_status imex_batch_create(imex_ctx* const* insts, int n, imex_batch** out);
void imex_batch_destroy(imex_batch* b);
const char* imex_batch_last_error(const imex_batch* b);
/* number of union-mesh groups the instances were sorted into */
int imex_batch_groups(const imex_batch* b);
/* nsteps steps of every instance; dt[i] > 0 is instance i's time step (host array of n) */
imex_status imex_batch_step(imex_batch* b, const double* dt, int nsteps);
/* instance i's velocity [d][its elements][nodes] / pressure / time, as for one context */
imex_status imex_batch_get_velocity(imex_batch* b, int i, double* out, int on_device);
imex_status imex_batch_get_pressure(imex_batch* b, int i, double* out, int on_device);
imex_status imex_batch_get_time(const imex_batch* b, int i, double* t);
/* totals of the last imex_batch_step over all groups (steps: per instance) */
imex_status imex_batch_get_stats(const imex_batch* b, imex_stats* out);
/* group q (0 <= q < imex_batch_groups): its instance count, degree P, velocity nodes per
   component of its union mesh, its stats and the wall time (ms) of its part of the last
   imex_batch_step; any output pointer may be NULL */
imex_status imex_batch_group_info(const imex_batch* b, int q, int* ninst, int* P, long long* nvel, imex_stats* st,
                                  double* last_ms);

/* ---- Serving: continuous batching ----------------------------------------------------
 * A server admits flow requests in arrival order while the estimated device footprint of
 * the active ones stays within an HBM budget, keeps every active request's fields and
 * solver state on the device in the union-mesh groups of the batched form, and advances all
 * active requests by one step per imex_server_tick; finished requests leave and queued ones
 * join between ticks (the groups' layouts are repacked on the device, no per-request
 * allocation).  Requests use RK-CB3e (Alg. 3). */
typedef struct imex_server imex_server;
typedef struct {
  double hbm_budget_bytes;  /* device bytes the active requests may occupy (<= 0: half the free memory) */
  int precision;            /* IMEX_FP64 | IMEX_MIXED | IMEX_MIXED_FAST */
  int poisson;              /* IMEX_POISSON_SIPG | IMEX_POISSON_CONSISTENT */
  double tol;               /* solver tolerance (<= 0: 1e-10) */
  int maxit;                /* (<= 0: 20000) */
  double vmax;              /* instability threshold on max |v| (0: none) */
  int keep_results;         /* 1: keep each finished request's velocity for imex_server_result */
} imex_server_desc;
typedef struct {
  int dim, P;
  int nelem[3];
  double lo[3], hi[3];
  int periodic[3];
  int flow; double flow_params[8];   /* initial field (IMEX_FLOW_*) at t0 */
  int nu_kind; double nu_params[8];  /* viscosity model (not IMEX_NU_FIELD) */
  int bc_kind; double bc_params[8];  /* Dirichlet data on non-periodic sides */
  int f_kind; double f_params[8];    /* forcing */
  double t0, dt;
  int nsteps;
} imex_request;
enum { IMEX_REQ_QUEUED = 0, IMEX_REQ_ACTIVE = 1, IMEX_REQ_DONE = 2, IMEX_REQ_FAILED = 3 };
typedef struct {
  long long submitted, completed, failed, active, queued, ticks;
  double p50_tick_ms, p99_tick_ms, mean_tick_ms;  /* wall time of a tick: admission, repack, one step */
  double dof_stages;                              /* velocity DOF x nontrivial stages advanced */
  double busy_s;                                  /* summed tick wall time */
  double footprint_bytes, max_footprint_bytes, budget_bytes;
  int groups;
} imex_server_stats;
imex_status imex_server_create(const imex_server_desc* desc, imex_server** out);
void imex_server_destroy(imex_server* sv);
const char* imex_server_last_error(const imex_server* sv);
/* queue a request (copied); id: its handle.  IMEX_EINVAL for an invalid mesh or model. */
imex_status imex_server_submit(imex_server* sv, const imex_request* r, long long* id);
/* device bytes a request occupies once admitted (the admission model of the HBM budget:
   fields, stage storage, CG work vectors and diagonals of its share of a union-mesh group,
   RK-CB3e); IMEX_EINVAL for an invalid mesh */
imex_status imex_request_footprint(const imex_request* r, double* bytes);
/* admit, repack, one step of every active request; active: requests still running after it.
   A group whose step fails marks its requests IMEX_REQ_FAILED (message: imex_server_last_error). */
imex_status imex_server_tick(imex_server* sv, int* active);
/* state (IMEX_REQ_*), steps done and time of a request */
imex_status imex_server_poll(const imex_server* sv, long long id, int* state, int* steps_done, double* t);
/* velocity of a finished request into host memory ([d][elements][nodes]); frees the copy */
imex_status imex_server_result(imex_server* sv, long long id, double* velocity);
imex_status imex_server_get_stats(const imex_server* sv, imex_server_stats* out);

#ifdef __cplusplus
}
#endif
#endif /* IMEX_GB300_H */
