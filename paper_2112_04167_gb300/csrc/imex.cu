// Host side of the library: context, solvers and the time steppers of Alg. 3
// (IMEX Runge-Kutta with projection splitting, Sec. 3.2.2) and Alg. 4 (SISDC,
// Sec. 3.2.3), behind the C ABI of include/imex.h.  Every arithmetic step runs in
// the device kernels; the host only sequences launches on the context's stream
// and reads back convergence flags once per chunk of CG iterations.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <string>
#include <thread>
#include <mutex>
#include <vector>

#include "../../include/imex.h"
#include "common.cuh"
#include "kernels.h"
#include "vec.h"

using namespace imex;

// helpers defined at the end of this file
void f2d(const float* in, double* out, size_t n, cudaStream_t st);

namespace {

struct Tab {
  int s = 0;
  double c[8] = {0};
  double AI[8][8] = {{0}};
  double bI[8] = {0};
  double AE[8][8] = {{0}};
  double bE[8] = {0};
};

// Butcher tableaux of the paper's appendix (RK-TR, RK-CB2, RK-CB3c, RK-CB3e, RK-CB4, RK-ARS3)
// and IMEX Euler, as doubles.
bool named_tableau(const std::string& name, Tab* t) {
  auto set = [&](int s, std::vector<double> c, std::vector<std::vector<double>> AI, std::vector<double> bI,
                 std::vector<std::vector<double>> AE, std::vector<double> bE) {
    *t = Tab();
    t->s = s;
    for (int i = 0; i < s; ++i) {
      t->c[i] = c[i];
      t->bI[i] = bI[i];
      t->bE[i] = bE[i];
      for (int j = 0; j < (int)AI[i].size(); ++j) t->AI[i][j] = AI[i][j];
      for (int j = 0; j < (int)AE[i].size(); ++j) t->AE[i][j] = AE[i][j];
    }
  };
  std::string n = name;
  for (auto& ch : n) ch = (char)toupper(ch);
  if (n.rfind("RK-", 0) == 0) n = n.substr(3);
  if (n == "EULER" || n == "EU") {
    set(2, {0, 1}, {{0}, {0, 1}}, {0, 1}, {{0}, {1}}, {1, 0});
  } else if (n == "TR") {
    set(3, {0, 1, 1}, {{0}, {0, 1}, {0.5, 0, 0.5}}, {0.5, 0, 0.5}, {{0}, {1}, {0.5, 0.5}}, {0.5, 0.5, 0});
  } else if (n == "CB2") {
    set(3, {0, 0.4, 1}, {{0}, {0, 0.4}, {0, 5.0 / 6, 1.0 / 6}}, {0, 5.0 / 6, 1.0 / 6}, {{0}, {0.4}, {0, 1}},
        {0, 5.0 / 6, 1.0 / 6});
  } else if (n == "CB3C") {
    const double c2 = 3375509829940.0 / 4525919076317.0, c3 = 272778623835.0 / 1039454778728.0;
    const double b2 = 673488652607.0 / 2334033219546.0, b3 = 493801219040.0 / 853653026979.0,
                 b4 = 184814777513.0 / 1389668723319.0;
    const double a32 = -11712383888607531889907.0 / 32694570495602105556248.0;
    const double a33 = 566138307881.0 / 912153721139.0;
    set(4, {0, c2, c3, 1}, {{0}, {0, c2}, {0, a32, a33}, {0, b2, b3, b4}}, {0, b2, b3, b4},
        {{0}, {c2}, {0, c3}, {0, b2, 1660544566939.0 / 2334033219546.0}}, {0, b2, b3, b4});
  } else if (n == "CB3E") {
    set(4, {0, 1.0 / 3, 1, 1}, {{0}, {0, 1.0 / 3}, {0, 0.5, 0.5}, {0, 0.75, -0.25, 0.5}}, {0, 0.75, -0.25, 0.5},
        {{0}, {1.0 / 3}, {0, 1}, {0, 0.75, 0.25}}, {0, 0.75, -0.25, 0.5});
  } else if (n == "CB4") {
    const double a1 = 232049084587.0 / 1377130630063.0, a2 = 322009889509.0 / 2243393849156.0,
                 a3 = -195109672787.0 / 1233165545817.0, b4 = -340582416761.0 / 705418832319.0,
                 b5 = 463396075661.0 / 409972144477.0, b6 = 323177943294.0 / 1626646580633.0;
    set(6, {0, 0.25, 0.75, 0.375, 0.5, 1},
        {{0},
         {0.125, 0.125},
         {216145252607.0 / 961230882893.0, 257479850128.0 / 1143310606989.0, 30481561667.0 / 101628412017.0},
         {a1, -381180097479.0 / 1276440792700.0, -54660926949.0 / 461115766612.0, 344309628413.0 / 552073727558.0},
         {a1, a2, -100836174740.0 / 861952129159.0, -250423827953.0 / 1283875864443.0, 0.5},
         {a1, a2, a3, b4, b5, b6}},
        {a1, a2, a3, b4, b5, b6},
        {{0},
         {0.25},
         {153985248130.0 / 1004999853329.0, 902825336800.0 / 1512825644809.0},
         {a1, 99316866929.0 / 820744730663.0, 82888780751.0 / 969573940619.0},
         {a1, a2, 57501241309.0 / 765040883867.0, 76345938311.0 / 676824576433.0},
         {a1, a2, a3, -4099309936455.0 / 6310162971841.0, 1395992540491.0 / 933264948679.0}},
        {a1, a2, a3, b4, b5, b6});
  } else if (n == "ARS3") {
    set(5, {0, 0.5, 2.0 / 3, 0.5, 1},
        {{0}, {0, 0.5}, {0, 1.0 / 6, 0.5}, {0, -0.5, 0.5, 0.5}, {0, 1.5, -1.5, 0.5, 0.5}}, {0, 1.5, -1.5, 0.5, 0.5},
        {{0}, {0.5}, {11.0 / 18, 1.0 / 18}, {5.0 / 6, -5.0 / 6, 0.5}, {0.25, 1.75, 0.75, -1.75}},
        {0.25, 1.75, 0.75, -1.75, 0});
  } else {
    return false;
  }
  return true;
}

bool valid_tableau(const Tab& t) {
  if (t.s < 2 || t.s > 8) return false;
  if (t.c[0] != 0.0 || t.AI[0][0] != 0.0) return false;
  for (int i = 0; i < t.s; ++i) {
    double si = 0, se = 0;
    for (int j = 0; j < t.s; ++j) {
      if (j > i && t.AI[i][j] != 0.0) return false;
      if (j >= i && t.AE[i][j] != 0.0) return false;
      si += t.AI[i][j];
      se += t.AE[i][j];
    }
    if (std::fabs(si - t.c[i]) > 1e-10 || std::fabs(se - t.c[i]) > 1e-10) return false;
  }
  return true;
}

// GLL points on [-1, 1] by Newton's method on L_M' (sub-nodes of the SDC step)
void gll_points(int n, double* x) {
  const int P = n - 1;
  x[0] = -1.0;
  x[P] = 1.0;
  for (int i = 1; i < P; ++i) {
    double z = -std::cos(M_PI * i / P);
    for (int it = 0; it < 100; ++it) {
      double p0 = 1, p1 = z, d0 = 0, d1 = 1;
      for (int k = 2; k <= P; ++k) {
        double p2 = ((2.0 * k - 1) * z * p1 - (k - 1.0) * p0) / k;
        double d2 = d0 + (2.0 * k - 1) * p1;
        p0 = p1; p1 = p2; d0 = d1; d1 = d2;
      }
      const double d2L = (2.0 * z * d1 - P * (P + 1.0) * p1) / (1.0 - z * z);
      const double dz = d1 / d2L;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
  }
}

}  // namespace

struct imex_ctx {
  imex_mesh_desc desc{};
  Geom gv{}, gp{};
  int d = 0, Nv = 0, Np = 0;
  size_t nv = 0, np = 0;        // nodes per velocity component / pressure nodes
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::string err;
  Tab tab;
  bool use_sdc = false;
  // IMEX BDF2 (Sec. 3.2.1): steps taken since its start (the first is IMEX Euler), the step
  // size of the history, and the history itself (v^{n-1}, nu^{n-1}; its right-hand sides are
  // E[1], Fd1[1], Fd3[1]) plus the extrapolated viscosity of the diffusion step
  bool use_bdf2 = false;
  long long bdf_n = 0;
  double bdf_dt = 0.0;
  double *bdf_vprev = nullptr, *bdf_nuprev = nullptr, *bdf_nustar = nullptr;
  int sdc_M = 0, sdc_K = 0;
  Tab sdc_pred;
  // models
  int nu_kind = IMEX_NU_CONST;
  double nu_p[8] = {0};
  int bc_kind = IMEX_FLOW_NONE;
  double bc_p[8] = {0};
  int f_kind = IMEX_FORCE_NONE;
  double f_p[8] = {0};
  double t = 0.0;
  // device memory
  Tables<double>* dtab64 = nullptr;
  Tables<float>* dtab32 = nullptr;
  // constant-viscosity line operators of the velocity (v) and pressure (p) spaces
  LineOps<double>* ops64_v = nullptr;
  LineOps<float>* ops32_v = nullptr;
  LineOps<double>* ops64_p = nullptr;
  LineOps<float>* ops32_p = nullptr;
  std::vector<void*> allocs;
  double *v = nullptr, *vp = nullptr, *vpp = nullptr, *g = nullptr, *tmp = nullptr, *vb = nullptr;
  double *nu = nullptr, *nu_fixed = nullptr, *phi = nullptr, *jac = nullptr, *fsbuf = nullptr;
  double *psi = nullptr, *bp = nullptr, *mass_v = nullptr, *mass_p = nullptr;
  // time scale tau of the stage potential held in psi (0: none): the stage projections
  // solve for psi'' ~ tau p, so the next solve starts from psi scaled to its own tau
  double psi_tau = 0.0;
  double* psi_f = nullptr;     // potential of the final projection (zero initial guess)
  std::vector<double*> E, Fd1, Fd3, Fs;         // stage storage (RK)
  // SDC storage
  std::vector<double*> sv, snu, sFEX, sFIM, sFq;
  // CG (FP64 and FP32)
  double *cx = nullptr, *cr = nullptr, *cz = nullptr, *cp = nullptr, *cAp = nullptr, *cdiag = nullptr;
  double* ffx = nullptr;     // float-float pairs of a float-float apply's input (same size as FP64)
  float *fx = nullptr, *fr = nullptr, *fp = nullptr, *fAp = nullptr, *fdiag = nullptr;
  float *fnu = nullptr, *fvtmp = nullptr;
  double* partial = nullptr;
  double* apartial = nullptr;   // per-block partials of the fused apply + dot
  size_t apartial_cap = 0;      // its length in doubles
  unsigned int* counters = nullptr;
  int nblocks = 0;
  double* dscal = nullptr;      // 16 x 4 doubles of scalars
  int* iscal = nullptr;
  double* hscal = nullptr;      // pinned host mirror
  int* hiscal = nullptr;
  // segmented CG: the systems of the pressure space and of the velocity space (one per
  // component), their per-system scalars (device, and a pinned host mirror) and partials
  struct Seg {
    SegTable t{};
    size_t total = 0;
    int nseg_cap = 0, nblk_cap = 0;       // capacity of the device arrays below
    long long *off_d = nullptr, *doff_d = nullptr;
    int *len_d = nullptr, *bs_d = nullptr, *bl_d = nullptr, *b0_d = nullptr;
    SegBlock* blk_d = nullptr;
  };
  Seg segp, segv;
  int maxsys = 0;
  double* cg_d = nullptr;       // 12 x maxsys
  float* cg_f = nullptr;        // 4 x maxsys
  int* cg_i = nullptr;          // 2 x maxsys
  double* cg_hd = nullptr;
  int* cg_hi = nullptr;
  double* seg_partial = nullptr;
  bool diag_valid_p = false;
  // diagonal of the velocity SIPG operator with unit factor for a viscosity that is constant
  // per element (the Helmholtz diagonals are M + gamma dt_e times it), valid for kdiag_nu
  double* kdiag = nullptr;
  bool kdiag_valid = false;
  double kdiag_nu = 0.0;
  // K v_i of the last Helmholtz solution (in cz, from its final residual check), valid for
  // the stage right-hand side that follows the solve without Dirichlet data (F_d1 = -M^-1 K v)
  bool kx_ready = false;
  const double* kx_for = nullptr;
  // instances of the mesh: one for a plain context; several for the union mesh of a batch
  // group, whose kernels see per-element geometry, viscosity, time step and time
  bool batched = false;
  long long ne_cap = 0;         // element and instance capacity of the buffers (>= current)
  int ninst_cap = 0;
  std::vector<InstGeom> inst;
  InstGeom* inst_d = nullptr;
  int* elem_inst_d = nullptr;
  int* nbr_d = nullptr;       // element neighbour table of the layout (Geom::nbr)
  double* edt = nullptr;        // per-element time step (batched)
  // CUDA graphs of CG iteration chunks, keyed by everything their launches depend on
  struct GraphEntry {
    std::vector<unsigned long long> key;
    cudaGraphExec_t exec;
    long long nkern;
  };
  std::vector<GraphEntry> graphs;
  bool use_graphs = true;
  // persistent FP32 CG of the periodic 3D pressure solves: partial sums, barrier, error flag
  bool use_persist = false;
  double* persist_partial = nullptr;   // 5 x 4096
  unsigned int* persist_bar = nullptr; // [2] barrier + [1] error flag (as int)
  // p-multigrid preconditioner of the pressure solves: levels of degree P-1 halved down to 1
  // on the same mesh, the SIPG pressure operator rediscretised on each, Chebyshev-Jacobi
  // smoothing, element-local GLL interpolation between levels
  struct Pmg {
    int kind = IMEX_PRECOND_PMG;   // IMEX_PRECOND_JACOBI / IMEX_PRECOND_PMG
    int pre = 3, coarse = 10;      // smoothing steps (before and after), steps of the coarsest level
    double ratio = 10.0, cratio = 100.0;
    bool alloc64 = false, alloc32 = false, ready = false;
    int nlev = 0;
    int N[4] = {0, 0, 0, 0};
    size_t cap[4] = {0, 0, 0, 0};  // nodes per level at the element capacity
    double lmax[4] = {0, 0, 0, 0};
    Interp1D I[4];                 // I[l]: level l+1 -> level l
    LineOps<double>* ops64[4] = {nullptr, nullptr, nullptr, nullptr};
    LineOps<float>* ops32[4] = {nullptr, nullptr, nullptr, nullptr};
    double* dinv64[4] = {nullptr, nullptr, nullptr, nullptr};
    float* dinv32[4] = {nullptr, nullptr, nullptr, nullptr};
    // per level: right-hand side, iterate, residual, Chebyshev direction, operator output (level
    // 0's right-hand side and iterate are the CG residual and z)
    double *b64[4] = {}, *x64[4] = {}, *r64[4] = {}, *d64[4] = {}, *ad64[4] = {};
    float *b32[4] = {}, *x32[4] = {}, *r32[4] = {}, *d32[4] = {}, *ad32[4] = {};
    double *z64 = nullptr, *ones64 = nullptr;
    float *z32 = nullptr, *ones32 = nullptr;
    // the FP32 coarsest level (N = 2, 3D periodic) smoothed by one cluster launch
    bool cluster = false;
  } pmg;
  // divergence / mass-flux stabilisation after each stage projection (zeta_D, zeta_C; both
  // 0: off), the time step of the step in progress, the element speeds, the inverse mass of
  // the d components and the single CG system spanning them
  double stab_zd = 0.0, stab_zc = 0.0;
  double cur_dt = 0.0;
  double* stab_speed = nullptr;
  double* stab_minv = nullptr;
  Seg segs;
  long long stab_iters = 0;
  // scratch of the flow statistics (grown on demand)
  double2* diag_grid = nullptr;
  size_t diag_grid_cap = 0;
  double* diag_part = nullptr;
  size_t diag_part_cap = 0;
  imex_stats stats{};
  double last_res = 0.0;
  // CUDA-event timing of kernel classes
  struct Prof {
    std::vector<cudaEvent_t> ev;   // pairs
    int used = 0;
    long long n = 0;
    double ms = 0.0;
    double bytes = 0.0, flops = 0.0;   // algorithmic work of the launches (see prof_end)
    int arith = -1;                    // IMEX_ARITH_* of the last launch
  };
  bool prof = false;
  Prof profc[IMEX_PROF_NCLASS];
};

namespace {

imex_status fail(imex_ctx* c, imex_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

imex_status cuda_check(imex_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return IMEX_OK;
  return fail(c, e == cudaErrorMemoryAllocation ? IMEX_ENOMEM : IMEX_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

// drain the recorded event pairs of one class into its totals
void prof_flush(imex_ctx* c, int cls) {
  auto& P = c->profc[cls];
  if (P.used == 0) return;
  cudaEventSynchronize(P.ev[2 * (P.used - 1) + 1]);
  for (int i = 0; i < P.used; ++i) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, P.ev[2 * i], P.ev[2 * i + 1]);
    P.ms += ms;
  }
  P.n += P.used;
  P.used = 0;
}

// record the start (begin = true) or end of one launch of a timed class
void prof_mark(imex_ctx* c, int cls, bool begin) {
  if (!c->prof) return;
  auto& P = c->profc[cls];
  const int cap = 4096;
  if (P.ev.empty()) {
    P.ev.resize(2 * cap);
    for (auto& e : P.ev) cudaEventCreate(&e);
  }
  if (begin && P.used == cap) prof_flush(c, cls);
  cudaEventRecord(P.ev[2 * P.used + (begin ? 0 : 1)], c->st);
  if (!begin) P.used++;
}

// end of one launch of a timed class with its algorithmic work: the bytes the operation must
// move (each input read once, each output written once) and its floating-point operations
void prof_end(imex_ctx* c, int cls, double bytes, double flops, int arith) {
  if (!c->prof) return;
  prof_mark(c, cls, false);
  auto& P = c->profc[cls];
  P.bytes += bytes;
  P.flops += flops;
  P.arith = arith;
}

// flops per node of the constant-viscosity SIPG apply on N points per direction (line form):
// per direction N multiply-adds of the element's own line operator row, four of the two
// neighbours' trace and derivative terms and two (amortised) forming those derivatives; six
// more to weight and combine the directions
double sipg_flops_per_node(int d, int N) { return 2.0 * d * (N + 6) + 6.0; }

// flops per element of the over-integrated convection on N points (Q Gauss points per
// direction): the d components interpolated to the Q^d points and the d^2 flux components
// differentiated back, each a sum-factorised sequence of d 1D passes
double conv_flops_per_elem(int d, int N) {
  const int Q = over_q(N);
  double pass = 0.0;
  for (int j = 1; j <= d; ++j) pass += std::pow((double)Q, j) * std::pow((double)N, d + 1 - j);
  return 2.0 * (d + d * d) * pass;
}

template <typename T>
imex_status dalloc(imex_ctx* c, T** p, size_t n) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
  if (e != cudaSuccess) return cuda_check(c, e, "cudaMalloc");
  c->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return IMEX_OK;
}

#define TRY(x)                       \
  do {                               \
    imex_status _s = (x);            \
    if (_s != IMEX_OK) return _s;    \
  } while (0)
#define CK(x, what) TRY(cuda_check(c, (x), what))

// Segment table of nseg systems: system s occupies [off[s], off[s] + len[s]) of the CG
// vectors and starts at doff[s] in the Jacobi diagonal; blocks of SEG_CHUNK elements.  The
// device arrays are allocated once with capacity (nseg_cap systems, nblk_cap blocks) and
// refilled when the layout changes.
imex_status make_seg(imex_ctx* c, int nseg, const long long* off, const long long* doff, const long long* len,
                     imex_ctx::Seg* out, int nseg_cap, int nblk_cap) {
  std::vector<int> blen(nseg), blk_seg, blk_lo, blk0(nseg + 1);
  std::vector<SegBlock> blk;
  size_t total = 0;
  for (int s = 0; s < nseg; ++s) {
    if (len[s] <= 0 || len[s] > (long long)INT_MAX - SEG_CHUNK) return fail(c, IMEX_EINVAL, "segment size");
    blen[s] = (int)len[s];
    blk0[s] = (int)blk_seg.size();
    for (long long lo = 0; lo < len[s]; lo += SEG_CHUNK) {
      blk_seg.push_back(s);
      blk_lo.push_back((int)lo);
      SegBlock b{};
      b.off = off[s] + lo;
      b.doff = doff[s] + lo;
      b.n = (int)std::min<long long>(SEG_CHUNK, len[s] - lo);
      b.s = s;
      blk.push_back(b);
    }
    total = std::max(total, (size_t)(off[s] + len[s]));
  }
  blk0[nseg] = (int)blk_seg.size();
  const int nblk = (int)blk_seg.size();
  if (out->nseg_cap == 0) {
    out->nseg_cap = std::max(nseg, nseg_cap);
    out->nblk_cap = std::max(nblk, nblk_cap);
    TRY(dalloc(c, &out->off_d, out->nseg_cap));
    TRY(dalloc(c, &out->doff_d, out->nseg_cap));
    TRY(dalloc(c, &out->len_d, out->nseg_cap));
    TRY(dalloc(c, &out->b0_d, out->nseg_cap + 1));
    TRY(dalloc(c, &out->bs_d, out->nblk_cap));
    TRY(dalloc(c, &out->bl_d, out->nblk_cap));
    TRY(dalloc(c, &out->blk_d, out->nblk_cap));
  }
  if (nseg > out->nseg_cap || nblk > out->nblk_cap) return fail(c, IMEX_EINVAL, "segment table above capacity");
  CK(cudaMemcpy(out->blk_d, blk.data(), blk.size() * sizeof(SegBlock), cudaMemcpyHostToDevice), "cp seg");
  CK(cudaMemcpy(out->off_d, off, nseg * sizeof(long long), cudaMemcpyHostToDevice), "cp seg");
  CK(cudaMemcpy(out->doff_d, doff, nseg * sizeof(long long), cudaMemcpyHostToDevice), "cp seg");
  CK(cudaMemcpy(out->len_d, blen.data(), nseg * sizeof(int), cudaMemcpyHostToDevice), "cp seg");
  CK(cudaMemcpy(out->bs_d, blk_seg.data(), blk_seg.size() * sizeof(int), cudaMemcpyHostToDevice), "cp seg");
  CK(cudaMemcpy(out->bl_d, blk_lo.data(), blk_lo.size() * sizeof(int), cudaMemcpyHostToDevice), "cp seg");
  CK(cudaMemcpy(out->b0_d, blk0.data(), (nseg + 1) * sizeof(int), cudaMemcpyHostToDevice), "cp seg");
  out->t.nseg = nseg;
  out->t.nblk = nblk;
  out->t.off = out->off_d;
  out->t.doff = out->doff_d;
  out->t.len = out->len_d;
  out->t.blk_seg = out->bs_d;
  out->t.blk_lo = out->bl_d;
  out->t.seg_blk0 = out->b0_d;
  out->t.blk = out->blk_d;
  out->total = total;
  return IMEX_OK;
}


imex_status launch_check(imex_ctx* c, int rc, const char* what) {
  if (rc != 0) return fail(c, IMEX_EINVAL, std::string(what) + ": unsupported (dim, P)");
  return cuda_check(c, cudaGetLastError(), what);
}

// ---- basic operators on the context's buffers --------------------------------------
template <typename T>
SipgArgs<T> sipg_args(const T* x, T* y, int nsys, long long stride, const T* nu, double nu0, const T* gd,
                      double alpha, double beta, int minv) {
  SipgArgs<T> a;
  a.x = x; a.y = y; a.nsys = nsys; a.sys_stride = stride; a.nu = nu; a.nu0 = (T)nu0;
  a.gdata = gd; a.g_stride = stride; a.alpha = (T)alpha; a.beta = (T)beta; a.minv = minv;
  a.ops = nullptr;
  a.dot_partial = nullptr;
  a.dot_counter = nullptr;
  a.dot_out = nullptr;
  a.cg_rz = nullptr;
  a.cg_alpha = nullptr;
  a.cg_alpha_f = nullptr;
  a.cg_done = nullptr;
  a.dot_defer = 0;
  a.dot_nblk = nullptr;
  a.done_flags = nullptr;
  a.done_ninst = 0;
  a.inst_nu = 0;
  a.inst_dt = 0;
  a.variant = 0;
  a.cheb = 0;
  a.ch_last = 0;
  a.ch_addx = 0;
  a.ch_r = a.ch_dout = a.ch_s = nullptr;
  a.ch_dinv = nullptr;
  a.ch_b = nullptr;
  a.xff = nullptr;
  a.ch_c1 = a.ch_c2 = T(0);
  return a;
}

template <typename T> const LineOps<T>* line_ops(const imex_ctx* c, bool velocity);
template <> const LineOps<double>* line_ops<double>(const imex_ctx* c, bool velocity) {
  return velocity ? c->ops64_v : c->ops64_p;
}
template <> const LineOps<float>* line_ops<float>(const imex_ctx* c, bool velocity) {
  return velocity ? c->ops32_v : c->ops32_p;
}

double nu_const(const imex_ctx* c) { return c->nu_p[0]; }

bool variable_nu(const imex_ctx* c) { return c->nu_kind != IMEX_NU_CONST; }

// fused CG dot of an operator apply: (p, A p) into cg->pAp and the step length alpha
template <typename T>
void fuse_cg(imex_ctx* c, SipgArgs<T>& a, const CgScalars* cg) {
  if (!cg) return;
  a.dot_out = cg->pAp;
  a.dot_partial = c->apartial;
  a.dot_counter = c->counters;
  a.cg_rz = cg->rz;
  a.cg_alpha = cg->alpha;
  a.cg_alpha_f = cg->alpha_f;
  a.cg_done = cg->done;
  if (cg->apart) {                       // the step kernel adds the partials itself
    a.dot_defer = 1;
    a.dot_nblk = const_cast<unsigned int*>(cg->apart_n);
  }
}

// batch groups in a CG loop: the operator skips the elements whose system has stopped (the
// done flags of the CG scalars; the systems of a group are its instances, times d for the
// velocity components)
template <typename T>
void skip_stopped_elems(imex_ctx* c, SipgArgs<T>& a, bool on) {
  if (!on || !c->batched) return;
  a.done_flags = c->cg_i;
  a.done_ninst = (int)c->inst.size();
}

// batch groups: velocity operators take the constant viscosity of each element's instance
// and, where their scale is a multiple of the time step, the instance's step
template <typename T>
void vel_flags(const imex_ctx* c, SipgArgs<T>& a, bool dt_scaled) {
  if (!c->batched) return;
  a.inst_nu = a.nu == nullptr ? 1 : 0;
  a.inst_dt = dt_scaled ? 1 : 0;
}

// the mixed forms evaluate their FP64-class operators (residual checks, F_d1, projection,
// grad-div; IMEX_MIXED also the convection) in float-float arithmetic on FP64 fields
bool ff_class(const imex_ctx* c) {
  return c->desc.precision == IMEX_MIXED || c->desc.precision == IMEX_MIXED_FAST;
}

// ---- launch-shape tuner ----------------------------------------------------------------
// The periodic constant-viscosity SIPG kernels (the CG and V-cycle applies) exist in three
// launch shapes: the default elements per block, half and twice as many.  On first use for a
// (d, N, precision, element count) the tuner times each shape with CUDA events on the
// context's stream (outside any graph capture) and keeps the fastest, when it beats the
// default by more than 3%; the choice is cached for the process.  IMEX_TUNE=0 disables it.
struct TuneEntry {
  int d, N, f32;
  long long ne;
  int variant;
  double us[4];
};
std::mutex g_tune_mu;
std::vector<TuneEntry> g_tune;

int tuned_variant(const imex_ctx* c, int N, bool f32) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (const auto& t : g_tune)
    if (t.d == c->d && t.N == N && t.f32 == (int)f32 && t.ne == c->gp.ne) return t.variant;
  return 0;
}

// arithmetic of an operator apply of type T on this context (the FP64 applies of the mixed
// forms run in float-float)
template <typename T>
int arith_of(const imex_ctx* c);

// SIPG apply: the FP64 applies of the mixed form (residual replacements, explicit F_d1) use
// float-float arithmetic on FP64 fields where that kernel exists (periodic 3D, constant
// viscosity), plain FP64 otherwise; the FP64 form always uses FP64 arithmetic
template <typename T>
int apply_dispatch(imex_ctx* c, const Geom& g, int N, const SipgArgs<T>& a) {
  if (sizeof(T) == 8 && ff_class(c)) {
    const int rc = sipg_apply_ff(g, N, reinterpret_cast<const SipgArgs<double>&>(a), c->ffx, c->st);
    if (rc == 0) return 0;
  }
  return sipg_apply<T>(g, N, a, c->st);
}

template <typename T>
int arith_of(const imex_ctx* c) {
  if (sizeof(T) == 4) return IMEX_ARITH_FP32;
  return ff_class(c) ? IMEX_ARITH_FF : IMEX_ARITH_FP64;
}

// the pressure operator L psi (pressure space), T = double / float
template <typename T>
imex_status apply_pressure(imex_ctx* c, const T* x, T* y, T* vtmp, const CgScalars* cg = nullptr,
                           bool skip_stopped = false) {
  const int cls = sizeof(T) == 4 ? IMEX_PROF_PRESSURE_F32 : IMEX_PROF_PRESSURE_F64;
  if (c->desc.poisson == IMEX_POISSON_SIPG) {
    SipgArgs<T> a = sipg_args<T>(x, y, 1, (long long)c->np, nullptr, 1.0, nullptr, 0.0, 1.0, 0);
    a.ops = line_ops<T>(c, false);
    a.variant = tuned_variant(c, c->Np, sizeof(T) == 4);
    fuse_cg(c, a, cg);
    skip_stopped_elems(c, a, skip_stopped);
    prof_mark(c, cls, true);
    const int rc = apply_dispatch<T>(c, c->gp, c->Np, a);
    prof_end(c, cls, 2.0 * sizeof(T) * c->np, sipg_flops_per_node(c->d, c->Np) * c->np, arith_of<T>(c));
    return launch_check(c, rc, "sipg_apply(p)");
  }
  // consistent: L = B M^{-1} B^T
  GradArgs<T> ga{x, nullptr, (long long)c->nv, T(1), vtmp};
  TRY(launch_check(c, dg_grad<T>(c->gv, c->Nv, ga, c->st), "dg_grad"));
  DivArgs<T> da{vtmp, (long long)c->nv, nullptr, 0, T(1), y};
  return launch_check(c, dg_div<T>(c->gv, c->Nv, da, c->st), "dg_div");
}

// velocity Helmholtz operator (M + gamma A(nu)), nsys components
template <typename T>
imex_status apply_helm(imex_ctx* c, const T* x, T* y, int nsys, const T* nu, double gamma,
                       const CgScalars* cg = nullptr, bool skip_stopped = false) {
  const int cls = sizeof(T) == 4 ? IMEX_PROF_HELMHOLTZ_F32 : IMEX_PROF_HELMHOLTZ_F64;
  SipgArgs<T> a = sipg_args<T>(x, y, nsys, (long long)c->nv, nu, nu_const(c), nullptr, 1.0, gamma, 0);
  a.ops = line_ops<T>(c, true);
  if (!nu) a.variant = tuned_variant(c, c->Nv, sizeof(T) == 4);
  vel_flags(c, a, true);
  fuse_cg(c, a, cg);
  skip_stopped_elems(c, a, skip_stopped);
  prof_mark(c, cls, true);
  const int rc = apply_dispatch<T>(c, c->gv, c->Nv, a);
  prof_end(c, cls, sizeof(T) * (double)c->nv * (2.0 * nsys + (nu ? 1.0 : 0.0)),
           sipg_flops_per_node(c->d, c->Nv) * c->nv * nsys, arith_of<T>(c));
  return launch_check(c, rc, "sipg_apply(v)");
}

// CG vector kernels of the iteration loop, timed as the CG_STEP / CG_DIR classes (words per
// node: step reads r, A p, D^-1, x, p and writes x, r; direction reads r, D^-1, p and writes p,
// and r when projected; the p-multigrid iteration's projection of r 2, (r, z) 2, p = z + beta p 3)
template <typename T>
int arith_t() { return sizeof(T) == 4 ? IMEX_ARITH_FP32 : IMEX_ARITH_FP64; }
template <typename T>
void cg_step(imex_ctx* c, T* x, T* r, const T* p, const T* Ap, const T* dj, const imex_ctx::Seg& sg,
             const CgScalars& sc, int maxit) {
  prof_mark(c, IMEX_PROF_CG_STEP, true);
  seg_step_xr<T>(x, r, p, Ap, dj, sg.t, sc, maxit, c->seg_partial, c->counters + 1, c->st);
  prof_end(c, IMEX_PROF_CG_STEP, 7.0 * sizeof(T) * sg.total, 10.0 * sg.total, arith_t<T>());
}
template <typename T>
void cg_dir(imex_ctx* c, T* p, T* r, const T* dinv, const imex_ctx::Seg& sg, const CgScalars& sc, int restart) {
  prof_mark(c, IMEX_PROF_CG_DIR, true);
  seg_step_p<T>(p, r, dinv, sg.t, sc, restart, c->st);
  prof_end(c, IMEX_PROF_CG_DIR, (sc.project ? 5.0 : 4.0) * sizeof(T) * sg.total, 4.0 * sg.total, arith_t<T>());
}
template <typename T>
void cg_rproj(imex_ctx* c, T* r, const imex_ctx::Seg& sg, const CgScalars& sc) {
  prof_mark(c, IMEX_PROF_CG_DIR, true);
  seg_rproj<T>(r, sg.t, sc, c->st);
  prof_end(c, IMEX_PROF_CG_DIR, 2.0 * sizeof(T) * sg.total, 1.0 * sg.total, arith_t<T>());
}
template <typename T>
void cg_rz(imex_ctx* c, const T* r, const T* z, const imex_ctx::Seg& sg, const CgScalars& sc, int init) {
  prof_mark(c, IMEX_PROF_CG_DIR, true);
  seg_rz<T>(r, z, sg.t, sc, c->seg_partial, c->counters + 3, init, c->st);
  prof_end(c, IMEX_PROF_CG_DIR, 2.0 * sizeof(T) * sg.total, 3.0 * sg.total, arith_t<T>());
}
template <typename T>
void cg_pz(imex_ctx* c, T* p, const T* z, const imex_ctx::Seg& sg, const CgScalars& sc, int restart) {
  prof_mark(c, IMEX_PROF_CG_DIR, true);
  seg_pz<T>(p, z, sg.t, sc, restart, c->st);
  prof_end(c, IMEX_PROF_CG_DIR, 3.0 * sizeof(T) * sg.total, 3.0 * sg.total, arith_t<T>());
}

// z = one p-multigrid V-cycle applied to r (defined with the p-multigrid code below)
template <typename T>
imex_status pmg_vcycle(imex_ctx* c, const T* r, T* z, const double* lm, T* rproj = nullptr,
                       const T* rmean = nullptr, const int* rdone = nullptr);

// ---- PCG -------------------------------------------------------------------------
// per-system CG scalars: cg_d holds rz, rz_old, rr, bb, pAp, zmean, a mean scratch, the true
// residual norm (mixed form), rmean, dsum, alpha and beta, maxsys entries each; cg_f the FP32
// alpha, beta, zmean, rmean; cg_i holds done and iters
CgScalars scalars(imex_ctx* c, double tol, bool project) {
  const int m = c->maxsys;
  CgScalars s;
  s.rz = c->cg_d + 0 * m;
  s.rz_old = c->cg_d + 1 * m;
  s.rr = c->cg_d + 2 * m;
  s.bb = c->cg_d + 3 * m;
  s.pAp = c->cg_d + 4 * m;
  s.zmean = c->cg_d + 5 * m;
  s.rmean = c->cg_d + 8 * m;
  s.dsum = c->cg_d + 9 * m;
  s.alpha = c->cg_d + 10 * m;
  s.beta = c->cg_d + 11 * m;
  s.alpha_f = c->cg_f + 0 * m;
  s.beta_f = c->cg_f + 1 * m;
  s.zmean_f = c->cg_f + 2 * m;
  s.rmean_f = c->cg_f + 3 * m;
  s.done = c->cg_i + 0 * m;
  s.iters = c->cg_i + 1 * m;
  s.tol2 = tol * tol;
  s.project = project ? 1 : 0;
  s.apart = nullptr;
  s.apart_n = nullptr;
  s.apart_seg = 0;
  return s;
}

// The (p, A p) partials of the CG loop are left to the step kernel, which forms alpha itself:
// those of the fused apply, or else those of the dot kernel (one per segment block, when
// they fit the partials buffer)
void defer_dot(imex_ctx* c, CgScalars& s, bool fused, const SegTable& t) {
  if (fused) {
    s.apart = c->apartial;
    s.apart_n = c->counters + 4;
  } else if ((size_t)t.nblk <= c->apartial_cap) {
    s.apart = c->apartial;
    s.apart_seg = 1;
  }
}

// Enqueue body() -- kernel launches only, no host synchronisation -- as a CUDA graph cached
// under key: the first call captures it, later calls replay it with one launch.
template <typename F>
imex_status run_graph(imex_ctx* c, const std::vector<unsigned long long>& key, F body) {
  if (!c->use_graphs || c->prof) return body();
  for (auto& g : c->graphs)
    if (g.key == key) {
      CK(cudaGraphLaunch(g.exec, c->st), "graph launch");
      add_launches(g.nkern);
      return IMEX_OK;
    }
  const long long l0 = thread_launch_count();
  CK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal), "begin capture");
  const imex_status s = body();
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->st, &graph);
  const long long nk = thread_launch_count() - l0;
  add_launches(-nk);                                  // capturing launched nothing
  if (s != IMEX_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  CK(e, "end capture");
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  CK(ei, "graph instantiate");
  if (c->graphs.size() >= 16) {                       // bounded cache: drop the oldest graph
    CK(cudaStreamSynchronize(c->st), "sync");
    cudaGraphExecDestroy(c->graphs.front().exec);
    c->graphs.erase(c->graphs.begin());
  }
  c->graphs.push_back({key, exec, nk});
  CK(cudaGraphLaunch(exec, c->st), "graph launch");
  add_launches(nk);
  return IMEX_OK;
}

unsigned long long bits(double x) {
  unsigned long long u;
  std::memcpy(&u, &x, sizeof(u));
  return u;
}
unsigned long long addr(const void* p) { return (unsigned long long)(uintptr_t)p; }

// copy the per-system flags (done, iters) and the recursive rr, bb to the host mirrors
imex_status pull_scalars(imex_ctx* c, int nsys) {
  const int m = c->maxsys;
  CK(cudaMemcpyAsync(c->cg_hi, c->cg_i, 2 * m * sizeof(int), cudaMemcpyDeviceToHost, c->st), "cp flags");
  CK(cudaMemcpyAsync(c->cg_hd + 2 * m, c->cg_d + 2 * m, 2 * m * sizeof(double), cudaMemcpyDeviceToHost, c->st),
     "cp rr bb");
  CK(cudaStreamSynchronize(c->st), "sync");
  (void)nsys;
  return IMEX_OK;
}

// Jacobi PCG (FP64) on the systems of a segment table; x holds the initial guess.  `project`:
// the systems are singular with the constants as null space (the pressure problems): the
// residual is projected onto the range and the preconditioned residual kept mean-free.
// pm: preconditioned by one p-multigrid V-cycle per iteration (pressure systems) instead of
// the Jacobi diagonal dinv
template <typename Op, typename OpDot>
imex_status pcg(imex_ctx* c, const imex_ctx::Seg& sg, Op op, OpDot op_dot, bool fused, const double* b, double* x,
                const double* dinv, double tol, int maxit, bool project,
                const std::vector<unsigned long long>& opkey, long long* iters_out, double* res_out, bool pm = false) {
  const SegTable& t = sg.t;
  CgScalars sc = scalars(c, tol, project);
  defer_dot(c, sc, fused, t);
  const int nsys = t.nseg;
  const int m = c->maxsys;
  double* r = c->cr;
  double* p = c->cp;
  double* Ap = c->cAp;
  double* z = pm ? c->pmg.z64 : nullptr;
  const double* dj = pm ? c->pmg.ones64 : dinv;     // the step kernel's diagonal
  TRY(op(x, Ap));
  LinComb lc{};
  lc.nterms = 2;
  lc.x[0] = b; lc.c[0] = 1.0;
  lc.x[1] = Ap; lc.c[1] = -1.0;
  lincomb(r, lc, sg.total, c->st);        // r = b - A x (the segments tile [0, total))
  if (project) seg_remove_mean(r, t, c->cg_d + 6 * m, c->seg_partial, c->counters + 3, c->st);
  seg_dot<double>(b, b, t, sc.bb, c->seg_partial, c->counters + 3, c->st);
  seg_init<double>(r, dj, t, sc, c->seg_partial, c->counters + 2, 1, c->st);
  if (pm) {
    TRY(pmg_vcycle<double>(c, r, z, c->pmg.lmax));
    cg_rz<double>(c, r, z, sg, sc, 1);
    cg_pz<double>(c, p, z, sg, sc, 1);
  } else {
    cg_dir<double>(c, p, r, dinv, sg, sc, 1);
  }
  CK(cudaGetLastError(), "cg_init");
  // a V-cycle iteration costs many launches: shorter chunks waste less after convergence
  const int chunk = pm ? 4 : 16;
  std::vector<unsigned long long> key = {64,        addr(&sg), addr(x), addr(b), addr(dinv), (unsigned long long)fused,
                                         (unsigned long long)maxit, bits(tol), (unsigned long long)project,
                                         (unsigned long long)pm};
  key.insert(key.end(), opkey.begin(), opkey.end());
  auto body = [&]() -> imex_status {
    for (int k = 0; k < chunk; ++k) {
      if (fused) {
        TRY(op_dot(p, Ap, &sc));                    // A p, (p, A p) and alpha in one launch
      } else {
        TRY(op(p, Ap));
        seg_pap<double>(p, Ap, t, sc, c->seg_partial, c->counters + 3, c->st);
      }
      cg_step<double>(c, x, r, p, Ap, dj, sg, sc, maxit);
      if (pm) {
        if (project) cg_rproj<double>(c, r, sg, sc);
        TRY(pmg_vcycle<double>(c, r, z, c->pmg.lmax));
        cg_rz<double>(c, r, z, sg, sc, 0);
        cg_pz<double>(c, p, z, sg, sc, 0);
      } else {
        cg_dir<double>(c, p, r, dinv, sg, sc, 0);
      }
    }
    return IMEX_OK;
  };
  for (int it = 0; it < maxit + chunk; it += chunk) {
    TRY(run_graph(c, key, body));
    TRY(pull_scalars(c, nsys));
    bool all = true;
    for (int s = 0; s < nsys; ++s) all = all && c->cg_hi[s] != 0;
    if (all) break;
  }
  long long its = 0;
  double res = 0.0;
  imex_status st = IMEX_OK;
  for (int s = 0; s < nsys; ++s) {
    its += c->cg_hi[m + s];
    const double rr = c->cg_hd[2 * m + s], bb = c->cg_hd[3 * m + s];
    res = std::max(res, bb > 0 ? std::sqrt(rr / bb) : std::sqrt(rr));
    if (c->cg_hi[s] == 3 || c->cg_hi[s] == 0) st = IMEX_ENOTCONV;
    if (c->cg_hi[s] == 2) st = IMEX_EUNSTABLE;
  }
  if (iters_out) *iters_out += its;
  if (res_out) *res_out = res;
  if (st == IMEX_ENOTCONV) return fail(c, st, "CG did not converge within maxit");
  if (st == IMEX_EUNSTABLE) return fail(c, st, "NaN in CG residual");
  return IMEX_OK;
}

// Decrease of the recursive FP32 residual between two replacements by the true FP64
// residual (reliable updates of the mixed form): four decades with the V-cycle, whose
// preconditioned system is well conditioned (the FP32 recursion drifts by about eps32 times
// the condition number over a cycle), two with Jacobi; IMEX_REFINE_DECADES (1 to 5) in the
// environment sets both.  Measured on the 16^3, P = 7 headline: 18 replacements and 27
// V-cycle iterations per step with two decades, 15 and 33 with four, 3 % less time.
static double refine_delta(bool pm) {
  static const double env = [] {
    const char* ev = std::getenv("IMEX_REFINE_DECADES");
    const double k = ev ? std::atof(ev) : 0.0;
    return (k >= 1.0 && k <= 5.0) ? k : 0.0;
  }();
  return std::pow(10.0, -(env > 0.0 ? env : (pm ? 4.0 : 2.0)));
}

// Mixed-precision PCG (the IMEX_MIXED form).  The iteration itself runs entirely in FP32:
// operator and Jacobi preconditioner applies, the correction y, the recursive residual and
// the search directions (GB300's FP64 rate is a small fraction of its FP32 rate, so FP64
// stays out of the per-node inner loop; dot products accumulate in FP32 per thread and in
// FP64 across threads and blocks).  FP64 holds the iterate x and the true residual: when the
// recursive residual has dropped by `delta` since the last replacement, or meets the
// tolerance, the correction is flushed (x += y, y = 0) and the residual replaced by the
// true FP64 residual b - A64 x (reliable updates; the FP32 recursion drifts from the true
// residual by about eps32 times the condition number times the residual it started from,
// so a replacement after every two (Jacobi) or four (V-cycle) orders of magnitude keeps the
// drift small, refine_delta).  The search direction is kept across a replacement while the
// recursive residual still tracks the true one (within a factor sqrt 2) and restarts from
// the true residual otherwise.  Singular (pressure) systems keep the preconditioned
// residual and the search directions mean-free.  A system is finished only when its true
// FP64 residual meets the tolerance.
template <typename Op64, typename Op32, typename Op32Dot>
imex_status pcg_mixed(imex_ctx* c, const imex_ctx::Seg& sg, Op64 op64, Op32 op32, Op32Dot op32dot, bool fused,
                      const double* b, double* x, const float* dinv, double tol, int maxit, bool project,
                      const std::vector<unsigned long long>& opkey, long long* iters_out, double* res_out,
                      bool pm = false) {
  const SegTable& t = sg.t;
  const size_t ntot = sg.total;
  CgScalars sc = scalars(c, tol, project);
  defer_dot(c, sc, fused, t);
  const int nsys = t.nseg;
  const int m = c->maxsys;
  const double delta = refine_delta(pm);
  float* z = pm ? c->pmg.z32 : nullptr;
  const float* dj = pm ? c->pmg.ones32 : dinv;      // the step kernel's diagonal
  double* r64 = c->cr;
  float* y = c->fx;
  float* r = c->fr;
  float* p = c->fp;
  float* Ap = c->fAp;
  double* rrtrue = c->cg_d + 7 * m;
  seg_dot<double>(b, b, t, sc.bb, c->seg_partial, c->counters + 3, c->st);
  CK(cudaMemsetAsync(y, 0, ntot * sizeof(float), c->st), "memset");
  std::vector<double> rr_ref(nsys, 0.0);
  std::vector<int> done_h(nsys, 0);
  // stagnation of the true residual at its rounding floor: a system whose inner iteration
  // converged three times in a row without the true residual falling below a quarter of its
  // best value is accepted there (the FP64 form, which stops on its recursive residual, does
  // not see this floor; the achieved residual is reported in the statistics)
  std::vector<double> best_true(nsys, 0.0);
  std::vector<int> inner_conv(nsys, 0), stall(nsys, 0);
  std::vector<long long> its_ref(nsys, 0);        // iterations at the last replacement
  const long long cycle_cap = pm ? 64 : 2000;
  bool started = false, restart = true;
  int breakdowns = 0;
  auto replace = [&]() -> imex_status {
    if (started) {
      axpy_f2d(x, y, ntot, c->st);                                   // flush the correction
      CK(cudaMemsetAsync(y, 0, ntot * sizeof(float), c->st), "memset");
      // a constant in x is invisible to the exact operator but not to its rounding
      // (A 1 is only zero to machine precision): keep the iterate of singular systems mean-free
      if (project) seg_remove_mean(x, t, c->cg_d + 6 * m, c->seg_partial, c->counters + 3, c->st);
    }
    TRY(op64(x, c->cAp));
    LinComb lc{};
    lc.nterms = 2;
    lc.x[0] = b; lc.c[0] = 1.0;
    lc.x[1] = c->cAp; lc.c[1] = -1.0;
    lincomb(r64, lc, ntot, c->st);
    if (project) seg_remove_mean(r64, t, c->cg_d + 6 * m, c->seg_partial, c->counters + 3, c->st);
    seg_dot<double>(r64, r64, t, rrtrue, c->seg_partial, c->counters + 3, c->st);
    convert_d2f(r64, r, ntot, c->st);
    CK(cudaMemcpyAsync(c->cg_hd + 7 * m, rrtrue, nsys * sizeof(double), cudaMemcpyDeviceToHost, c->st), "cp");
    CK(cudaMemcpyAsync(c->cg_hd + 3 * m, sc.bb, nsys * sizeof(double), cudaMemcpyDeviceToHost, c->st), "cp");
    CK(cudaStreamSynchronize(c->st), "sync");
    const double* rt = c->cg_hd + 7 * m;
    const double* bbh = c->cg_hd + 3 * m;
    const double* rrec = c->cg_hd + 2 * m;
    for (int s = 0; s < nsys; ++s)
      if (started && done_h[s] == 0 && rt[s] > 2.0 * rrec[s]) restart = true;
    for (int s = 0; s < nsys; ++s) {
      if (rt[s] != rt[s]) return fail(c, IMEX_EUNSTABLE, "NaN in the residual");
      if (done_h[s] == 4) continue;
      if (started && inner_conv[s]) {
        stall[s] = (best_true[s] > 0.0 && rt[s] > 0.0625 * best_true[s]) ? stall[s] + 1 : 0;
        inner_conv[s] = 0;
      }
      if (best_true[s] == 0.0 || rt[s] < best_true[s]) best_true[s] = rt[s];
      its_ref[s] = started ? c->cg_hi[m + s] : 0;
      if (rt[s] <= tol * tol * bbh[s] || stall[s] >= 3) {
        done_h[s] = 4;
      } else {
        done_h[s] = 0;
        rr_ref[s] = rt[s];
      }
    }
    if (std::getenv("IMEX_DEBUG"))
      for (int s = 0; s < nsys && s < 4; ++s)
        std::fprintf(stderr, "[imex] replace sys %d its %d rec %.3e true %.3e bb %.3e done %d restart %d\n", s,
                     c->cg_hi[m + s], std::sqrt(rrec[s]), std::sqrt(rt[s]), std::sqrt(bbh[s]), done_h[s],
                     (int)restart);
    CK(cudaMemcpyAsync(sc.done, done_h.data(), nsys * sizeof(int), cudaMemcpyHostToDevice, c->st), "cp flags");
    const int keep = (started && !restart) ? 1 : 0;
    seg_init<float>(r, dj, t, sc, c->seg_partial, c->counters + 2, 0, c->st);
    if (pm) {
      TRY(pmg_vcycle<float>(c, r, z, c->pmg.lmax));
      cg_rz<float>(c, r, z, sg, sc, 1);
      if (!keep) cg_pz<float>(c, p, z, sg, sc, 1);
    } else if (!keep) {
      cg_dir<float>(c, p, r, dinv, sg, sc, 1);
    }
    started = true;
    restart = false;
    c->stats.refinements++;
    return cuda_check(c, cudaGetLastError(), "cg_init_mixed");
  };
  CK(cudaMemsetAsync(sc.iters, 0, nsys * sizeof(int), c->st), "memset");
  TRY(replace());
  const int chunk = pm ? 4 : 16;
  std::vector<unsigned long long> key = {32, addr(&sg), addr(dinv), (unsigned long long)fused,
                                         (unsigned long long)maxit, bits(tol), (unsigned long long)project,
                                         (unsigned long long)pm};
  key.insert(key.end(), opkey.begin(), opkey.end());
  auto body = [&]() -> imex_status {
    for (int k = 0; k < chunk; ++k) {
      if (fused) {
        TRY(op32dot(p, Ap, &sc));
      } else {
        TRY(op32(p, Ap));
        seg_pap<float>(p, Ap, t, sc, c->seg_partial, c->counters + 3, c->st);
      }
      cg_step<float>(c, y, r, p, Ap, dj, sg, sc, maxit);
      if (pm) {
        // one projected segment: the mean comes off r in the V-cycle's first kernel
        const bool fuse = project && t.nseg == 1 && c->pmg.nlev > 1;
        if (project && !fuse) cg_rproj<float>(c, r, sg, sc);
        if (fuse) TRY(pmg_vcycle<float>(c, r, z, c->pmg.lmax, r, sc.rmean_f, sc.done));
        else TRY(pmg_vcycle<float>(c, r, z, c->pmg.lmax));
        cg_rz<float>(c, r, z, sg, sc, 0);
        cg_pz<float>(c, p, z, sg, sc, 0);
      } else {
        cg_dir<float>(c, p, r, dinv, sg, sc, 0);
      }
    }
    return IMEX_OK;
  };
  // the periodic 3D pressure solve of one instance runs its inner iterations persistently
  bool persist = !pm && c->use_persist && !c->batched && project && nsys == 1 && fused && c->d == 3 &&
                 c->gp.bc[0] == 0 && c->gp.bc[1] == 0 && c->gp.bc[2] == 0;
  for (int round = 0;; ++round) {
    bool all = true;
    for (int s = 0; s < nsys; ++s) all = all && done_h[s] == 4;
    if (all) break;
    int rc = -1;
    if (persist) {
      CK(cudaMemsetAsync(c->persist_bar, 0, 4 * sizeof(unsigned int), c->st), "memset");
      SipgArgs<float> a = sipg_args<float>(p, Ap, 1, (long long)c->np, nullptr, 1.0, nullptr, 0.0, 1.0, 0);
      a.ops = line_ops<float>(c, false);
      prof_mark(c, IMEX_PROF_PCG_PERSIST, true);
      rc = pcg_persist_f32(c->gp, c->Np, a, y, r, p, Ap, dinv, (long long)ntot, sc, delta * delta * rr_ref[0], maxit,
                           c->persist_partial, c->persist_bar, (int*)(c->persist_bar + 2), c->st);
      prof_mark(c, IMEX_PROF_PCG_PERSIST, false);
      if (rc == 0) TRY(cuda_check(c, cudaGetLastError(), "pcg_persist"));
      else persist = false;
    }
    if (rc != 0) TRY(run_graph(c, key, body));
    TRY(pull_scalars(c, nsys));
    bool need = false;
    for (int s = 0; s < nsys; ++s) {
      int st = c->cg_hi[s];
      if (done_h[s] == 4) continue;
      if (st == 2) {
        // FP32 breakdown: restart from the FP64 residual (bounded number of times)
        if (++breakdowns > 2) return fail(c, IMEX_EUNSTABLE, "NaN in CG residual");
        st = 0;
        need = true;
        restart = true;
      }
      if (st == 3) {
        char msg[256];
        std::snprintf(msg, sizeof msg,
                      "CG did not converge within maxit (system %d of %d, %lld iterations, recursive residual "
                      "%.3e, last true residual %.3e, |b| %.3e)",
                      s, nsys, (long long)c->cg_hi[m + s], std::sqrt(c->cg_hd[2 * m + s]),
                      std::sqrt(c->cg_hd[7 * m + s]), std::sqrt(c->cg_hd[3 * m + s]));
        return fail(c, IMEX_ENOTCONV, msg);
      }
      if (st == 1) { need = true; restart = true; inner_conv[s] = 1; }  // recursive residual converged
      if (st == 0 && c->cg_hd[2 * m + s] < delta * delta * rr_ref[s]) need = true;
      // a cycle that has not reached its target after cycle_cap iterations (a V-cycle gains
      // about a decade per iteration, Jacobi a healthy two decades in a few hundred) has met
      // the FP32 floor of this system: replace, counted as an inner convergence for the
      // stagnation rule of the true residual
      if (st == 0 && c->cg_hi[m + s] - its_ref[s] > cycle_cap) {
        need = true;
        restart = true;
        inner_conv[s] = 1;
      }
      done_h[s] = st;
    }
    if (need) TRY(replace());
    if (round > 4 * (maxit / chunk + 4)) return fail(c, IMEX_ENOTCONV, "mixed CG did not converge");
  }
  long long its = 0;
  double res = 0.0;
  for (int s = 0; s < nsys; ++s) {
    its += c->cg_hi[m + s];
    const double bb = c->cg_hd[3 * m + s];
    res = std::max(res, bb > 0 ? std::sqrt(c->cg_hd[7 * m + s] / bb) : 0.0);
  }
  if (iters_out) *iters_out += its;
  if (res_out) *res_out = res;
  return IMEX_OK;
}

}  // namespace

// small helper kernels local to this file
namespace imex {
// y = m x per component (mass products of the stage combinations, Alg. 3)
__global__ void diag_mul_kernel(double* out, const double* x, const double* m, size_t n, int nsys) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n * nsys; i += (size_t)gridDim.x * blockDim.x)
    out[i] = x[i] * m[i % n];
}
}  // namespace imex

namespace {

void diag_mul(imex_ctx* c, double* out, const double* x, const double* m, size_t n, int nsys) {
  IMEX_COUNTED(imex::diag_mul_kernel<<<c->nblocks, 256, 0, c->st>>>(out, x, m, n, nsys));
}


// ---- p-multigrid -----------------------------------------------------------------------
template <typename T> struct PmgVecs;
template <> struct PmgVecs<double> {
  static double** b(imex_ctx::Pmg& m) { return m.b64; }
  static double** x(imex_ctx::Pmg& m) { return m.x64; }
  static double** r(imex_ctx::Pmg& m) { return m.r64; }
  static double** d(imex_ctx::Pmg& m) { return m.d64; }
  static double** ad(imex_ctx::Pmg& m) { return m.ad64; }
  static double** dinv(imex_ctx::Pmg& m) { return m.dinv64; }
  static LineOps<double>** ops(imex_ctx::Pmg& m) { return m.ops64; }
  static double* z(imex_ctx::Pmg& m) { return m.z64; }
  static double* ones(imex_ctx::Pmg& m) { return m.ones64; }
};
template <> struct PmgVecs<float> {
  static float** b(imex_ctx::Pmg& m) { return m.b32; }
  static float** x(imex_ctx::Pmg& m) { return m.x32; }
  static float** r(imex_ctx::Pmg& m) { return m.r32; }
  static float** d(imex_ctx::Pmg& m) { return m.d32; }
  static float** ad(imex_ctx::Pmg& m) { return m.ad32; }
  static float** dinv(imex_ctx::Pmg& m) { return m.dinv32; }
  static LineOps<float>** ops(imex_ctx::Pmg& m) { return m.ops32; }
  static float* z(imex_ctx::Pmg& m) { return m.z32; }
  static float* ones(imex_ctx::Pmg& m) { return m.ones32; }
};

// levels, line operators and interpolation matrices (once), and the vectors of precision T
template <typename T>
imex_status pmg_alloc(imex_ctx* c) {
  imex_ctx::Pmg& M = c->pmg;
  if (M.nlev == 0) {
    int N = c->Np;
    M.N[0] = N;
    M.nlev = 1;
    while (N > 2 && M.nlev < 4) {
      N = (N - 1) / 2 + 1;                      // degree halved: p -> floor(p / 2)
      M.N[M.nlev++] = N;
    }
    Tables<double>* h64 = new Tables<double>();
    Tables<float>* h32 = new Tables<float>();
    build_tables(h64, h32);
    const double hh[3] = {1.0, 1.0, 1.0};
    LineOps<double>* o64 = new LineOps<double>();
    LineOps<float>* o32 = new LineOps<float>();
    imex_status s = IMEX_OK;
    M.ops64[0] = c->ops64_p;
    M.ops32[0] = c->ops32_p;
    for (int l = 1; l < M.nlev && s == IMEX_OK; ++l) {
      build_line_ops(*h64, M.N[l], hh, c->d, o64, o32);
      s = dalloc(c, &M.ops64[l], 1);
      if (s == IMEX_OK) s = dalloc(c, &M.ops32[l], 1);
      if (s == IMEX_OK && cudaMemcpy(M.ops64[l], o64, sizeof(*o64), cudaMemcpyHostToDevice) != cudaSuccess)
        s = IMEX_ECUDA;
      if (s == IMEX_OK && cudaMemcpy(M.ops32[l], o32, sizeof(*o32), cudaMemcpyHostToDevice) != cudaSuccess)
        s = IMEX_ECUDA;
    }
    delete o64;
    delete o32;
    delete h64;
    delete h32;
    TRY(s);
    for (int l = 0; l + 1 < M.nlev; ++l) gll_interp(M.N[l + 1], M.N[l], M.I[l].m);
    for (int l = 0; l < M.nlev; ++l) {
      M.cap[l] = (size_t)c->ne_cap * ipow(M.N[l], c->d);
      TRY(dalloc(c, &M.dinv64[l], M.cap[l]));
    }
  }
  bool& done = sizeof(T) == 8 ? M.alloc64 : M.alloc32;
  if (done) return IMEX_OK;
  using V = PmgVecs<T>;
  for (int l = 0; l < M.nlev; ++l) {
    if (l > 0) {
      TRY(dalloc(c, &V::b(M)[l], M.cap[l]));
      TRY(dalloc(c, &V::x(M)[l], M.cap[l]));
    }
    TRY(dalloc(c, &V::r(M)[l], M.cap[l]));
    TRY(dalloc(c, &V::d(M)[l], M.cap[l]));
    TRY(dalloc(c, &V::ad(M)[l], M.cap[l]));
    if (sizeof(T) == 4) TRY(dalloc(c, &M.dinv32[l], M.cap[l]));
  }
  T* z = nullptr;
  T* ones = nullptr;
  TRY(dalloc(c, &z, M.cap[0]));
  TRY(dalloc(c, &ones, M.cap[0]));
  std::vector<T> h(M.cap[0], T(1));
  CK(cudaMemcpy(ones, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice), "cp ones");
  if (sizeof(T) == 8) { M.z64 = (double*)(void*)z; M.ones64 = (double*)(void*)ones; }
  else { M.z32 = (float*)(void*)z; M.ones32 = (float*)(void*)ones; }
  done = true;
  // FP32 diagonals added after the set-up: rounded from the FP64 ones
  if (sizeof(T) == 4 && M.ready)
    for (int l = 0; l < M.nlev; ++l)
      convert_d2f(M.dinv64[l], M.dinv32[l], (size_t)c->gp.ne * ipow(M.N[l], c->d), c->st);
  return IMEX_OK;
}

// A x on level l (pressure space, unit viscosity, homogeneous Neumann faces)
template <typename T>
imex_status pmg_apply(imex_ctx* c, int l, const T* x, T* y) {
  imex_ctx::Pmg& M = c->pmg;
  const size_t n = (size_t)c->gp.ne * ipow(M.N[l], c->d);
  SipgArgs<T> a = sipg_args<T>(x, y, 1, (long long)n, nullptr, 1.0, nullptr, 0.0, 1.0, 0);
  a.ops = PmgVecs<T>::ops(M)[l];
  a.variant = tuned_variant(c, M.N[l], sizeof(T) == 4);
  const int cls = l == 0 ? IMEX_PROF_PMG_APPLY : IMEX_PROF_PMG_APPLY_COARSE;
  prof_mark(c, cls, true);
  const int rc = sipg_apply<T>(c->gp, M.N[l], a, c->st);
  prof_end(c, cls, 2.0 * sizeof(T) * n, sipg_flops_per_node(c->d, M.N[l]) * n, arith_t<T>());
  return launch_check(c, rc, "sipg_apply(pmg)");
}

// Jacobi diagonals of every level and the Chebyshev upper bounds: 1.15 x the Rayleigh
// quotient (x, A x) / (x, D x) after 40 power steps x <- D^{-1} A x (FP64, from a fixed
// pseudo-random start), which reaches within a few percent of the largest eigenvalue of
// D^{-1} A on these operators
imex_status pmg_setup(imex_ctx* c) {
  imex_ctx::Pmg& M = c->pmg;
  if (M.ready) return IMEX_OK;
  TRY(pmg_alloc<double>(c));
  const int d = c->d;
  for (int l = 0; l < M.nlev; ++l) {
    const size_t n = (size_t)c->gp.ne * ipow(M.N[l], d);
    SipgArgs<double> a = sipg_args<double>(nullptr, M.dinv64[l], 1, (long long)n, nullptr, 1.0, nullptr, 0.0, 1.0, 0);
    TRY(launch_check(c, sipg_diag<double>(c->gp, M.N[l], a, c->st), "sipg_diag(pmg)"));
    reciprocal<double>(M.dinv64[l], n, c->st);
    if (M.alloc32) convert_d2f(M.dinv64[l], M.dinv32[l], n, c->st);
    // power iteration with (x, D x) carried along: x = D^{-1} y, D x = y
    double* x = M.r64[l];
    double* Dx = M.d64[l];
    double* ad = M.ad64[l];
    std::vector<double> y0(n);
    unsigned long long st = 0x9e3779b97f4a7c15ull;
    for (size_t i = 0; i < n; ++i) {
      st = st * 6364136223846793005ull + 1442695040888963407ull;
      y0[i] = (double)(st >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    }
    CK(cudaMemcpyAsync(Dx, y0.data(), n * sizeof(double), cudaMemcpyHostToDevice, c->st), "cp");
    vec_mul(x, M.dinv64[l], Dx, 1.0, n, c->st);
    double lam = 0.0;
    for (int it = 0; it < 40; ++it) {
      TRY(pmg_apply<double>(c, l, x, ad));
      dot_batched(x, ad, n, (long long)n, 1, c->partial, c->nblocks, c->dscal + 40, c->st);
      dot_batched(x, Dx, n, (long long)n, 1, c->partial, c->nblocks, c->dscal + 41, c->st);
      CK(cudaMemcpyAsync(c->hscal + 40, c->dscal + 40, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->st), "cp");
      CK(cudaStreamSynchronize(c->st), "sync");
      const double num = c->hscal[40], den = c->hscal[41];
      if (!(den > 0.0) || !std::isfinite(num)) return fail(c, IMEX_ECUDA, "p-multigrid eigenvalue estimate failed");
      lam = num / den;
      const double sc = 1.0 / std::sqrt(den);     // keep (x, D x) = 1
      vec_mul(x, M.dinv64[l], ad, sc, n, c->st);  // x <- D^{-1} A x
      std::swap(Dx, ad);                          // D x <- A x (scaled below)
      LinComb lc{};
      lc.nterms = 1; lc.x[0] = Dx; lc.c[0] = sc;
      lincomb(Dx, lc, n, c->st);
    }
    M.lmax[l] = 1.15 * lam;
  }
  CK(cudaStreamSynchronize(c->st), "sync");
  {
    const char* ev = std::getenv("IMEX_PMG_CLUSTER");          // "0": separate launches per step
    M.cluster = pmg_cluster_prepare(c->gp, M.N[M.nlev - 1]) && !(ev && ev[0] == '0');
  }
  M.ready = true;
  return IMEX_OK;
}

// Chebyshev steps on level l for A x = b, started from x = 0 (PMG_FROM_ZERO), from the
// current x (PMG_FROM_X), or with the first step from zero already taken by the restriction
// that produced b (PMG_PRESET: r = b, d = x = D^{-1} b / theta)
enum { PMG_FROM_ZERO = 0, PMG_FROM_X = 1, PMG_PRESET = 2 };
template <typename T>
imex_status pmg_smooth(imex_ctx* c, int l, int steps, double lmax, double ratio, int start, const T* b, T* x,
                       T* bproj = nullptr, const T* bmean = nullptr, const int* bdone = nullptr) {
  imex_ctx::Pmg& M = c->pmg;
  using V = PmgVecs<T>;
  const size_t n = (size_t)c->gp.ne * ipow(M.N[l], c->d);
  T* r = V::r(M)[l];
  T* dv = V::d(M)[l];
  T* ad = V::ad(M)[l];
  const T* dinv = V::dinv(M)[l];
  const double lmin = lmax / ratio;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
  const int cls = l == 0 ? IMEX_PROF_PMG_APPLY : IMEX_PROF_PMG_APPLY_COARSE;
  const double apply_flops = sipg_flops_per_node(c->d, M.N[l]) * (double)n;
  bool addx = false;
  if (start == PMG_FROM_X && steps >= 2) {
    // the first step from x in the apply of x: r = b - A x, d = D^{-1} r / theta; x itself
    // takes d in the next step (ch_addx)
    SipgArgs<T> a = sipg_args<T>(x, nullptr, 1, (long long)n, nullptr, 1.0, nullptr, 0.0, 1.0, 0);
    a.ops = V::ops(M)[l];
    a.variant = tuned_variant(c, M.N[l], sizeof(T) == 4);
    a.cheb = 2;
    a.ch_b = b;
    a.ch_r = r;
    a.ch_dout = dv;
    a.ch_dinv = dinv;
    a.ch_c1 = (T)(1.0 / theta);
    prof_mark(c, cls, true);
    const int rc = sipg_apply<T>(c->gp, M.N[l], a, c->st);
    prof_end(c, cls, 5.0 * sizeof(T) * n, apply_flops + 3.0 * n, arith_t<T>());
    TRY(launch_check(c, rc, "sipg_apply(chebyshev first)"));
    addx = true;
  } else if (start == PMG_FROM_ZERO && bproj) {
    // from zero for a projected CG residual: its mean taken off here (and written back)
    prof_mark(c, IMEX_PROF_PMG_VEC, true);
    cheb_first_proj<T>(x, dv, r, bproj, dinv, 1.0 / theta, bmean, bdone, n, c->st);
    prof_end(c, IMEX_PROF_PMG_VEC, 6.0 * sizeof(T) * n, 3.0 * n, arith_t<T>());
  } else if (start != PMG_PRESET) {
    const bool from_x = start == PMG_FROM_X;
    if (from_x) TRY(pmg_apply<T>(c, l, x, ad));
    prof_mark(c, IMEX_PROF_PMG_VEC, true);
    cheb_first<T>(x, dv, r, b, from_x ? ad : nullptr, dinv, 1.0 / theta, n, from_x ? 1 : 0, c->st);
    prof_end(c, IMEX_PROF_PMG_VEC, (from_x ? 7.0 : 5.0) * sizeof(T) * n, (from_x ? 4.0 : 2.0) * n, arith_t<T>());
  }
  double rho = 1.0 / sigma;
  // each further step is one apply whose output stage performs the update (the new direction
  // alternates between the two direction buffers, as neighbours still read the old one)
  T* dcur = dv;
  T* dnext = ad;
  for (int k = 1; k < steps; ++k) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    const int last = k == steps - 1 ? 1 : 0;
    SipgArgs<T> a = sipg_args<T>(dcur, nullptr, 1, (long long)n, nullptr, 1.0, nullptr, 0.0, 1.0, 0);
    a.ops = V::ops(M)[l];
    a.variant = tuned_variant(c, M.N[l], sizeof(T) == 4);
    a.cheb = 1;
    a.ch_last = last;
    a.ch_addx = (k == 1 && addx) ? 1 : 0;
    a.ch_r = r;
    a.ch_dout = dnext;
    a.ch_s = x;
    a.ch_dinv = dinv;
    a.ch_c1 = (T)(rn * rho);
    a.ch_c2 = (T)(2.0 * rn / delta);
    prof_mark(c, cls, true);
    const int rc = sipg_apply<T>(c->gp, M.N[l], a, c->st);
    prof_end(c, cls, (last ? 5.0 : 7.0) * sizeof(T) * n, apply_flops + (a.ch_addx ? 7.0 : 6.0) * n, arith_t<T>());
    TRY(launch_check(c, rc, "sipg_apply(chebyshev)"));
    std::swap(dcur, dnext);
    rho = rn;
  }
  return IMEX_OK;
}

// z = one V-cycle applied to r (level 0); lm: the Chebyshev upper bounds of the levels;
// rproj (== r, one-segment projected CG systems): the mean *rmean is taken off r in the
// first kernel and the projected r written back, unless *rdone
template <typename T>
imex_status pmg_vcycle(imex_ctx* c, const T* r, T* z, const double* lm, T* rproj, const T* rmean,
                       const int* rdone) {
  imex_ctx::Pmg& M = c->pmg;
  using V = PmgVecs<T>;
  const int L = M.nlev;
  const T* b[4];
  T* x[4];
  auto nodes = [&](int l) { return (double)c->gp.ne * ipow(M.N[l], c->d); };
  // a transfer between levels l and l+1: d passes of 1D contractions per element
  auto xfer_flops = [&](int l) {
    double f = 0.0;
    for (int j = 1; j <= c->d; ++j) f += std::pow((double)M.N[l + 1], j) * std::pow((double)M.N[l], c->d + 1 - j);
    return 2.0 * f * c->gp.ne;
  };
  for (int l = 0; l < L; ++l) {
    b[l] = l == 0 ? r : V::b(M)[l];
    x[l] = l == 0 ? z : V::x(M)[l];
  }
  // the coarsest level on one cluster (FP32): its restriction then writes b only
  const bool clus = sizeof(T) == 4 && M.cluster && L >= 2;
  for (int l = 0; l + 1 < L; ++l) {
    if (l == 0) TRY(pmg_smooth<T>(c, l, M.pre, lm[l], M.ratio, PMG_FROM_ZERO, b[l], x[l], rproj, rmean, rdone));
    else TRY(pmg_smooth<T>(c, l, M.pre, lm[l], M.ratio, PMG_PRESET, b[l], x[l]));
    TRY(pmg_apply<T>(c, l, x[l], V::ad(M)[l]));
    // restriction of the residual, with the first smoothing step (from zero) of level l + 1
    const bool first = !(clus && l + 2 == L);
    const double ratio1 = (l + 2 == L) ? M.cratio : M.ratio;
    const double theta1 = 0.5 * (lm[l + 1] + lm[l + 1] / ratio1);
    const ChebInit<T> ci = first ? ChebInit<T>{x[l + 1], V::d(M)[l + 1], V::r(M)[l + 1], V::dinv(M)[l + 1],
                                               (T)(1.0 / theta1)}
                                 : ChebInit<T>{nullptr, nullptr, nullptr, nullptr, T(0)};
    prof_mark(c, IMEX_PROF_PMG_VEC, true);
    if (pmg_restrict_cheb<T>(c->d, c->gp.ne, M.N[l], M.N[l + 1], b[l], V::ad(M)[l], V::b(M)[l + 1], M.I[l], ci,
                             c->st) != 0)
      return fail(c, IMEX_EINVAL, "p-multigrid: unsupported level pair");
    prof_end(c, IMEX_PROF_PMG_VEC, sizeof(T) * (2.0 * nodes(l) + (first ? 5.0 : 1.0) * nodes(l + 1)),
             xfer_flops(l) + (first ? 2.0 : 0.0) * nodes(l + 1), arith_t<T>());
  }
  int crc = -1;
  if constexpr (sizeof(T) == 4) {
    if (clus) {
      prof_mark(c, IMEX_PROF_PMG_APPLY_COARSE, true);
      crc = pmg_coarse_cluster(c->gp, M.N[L - 1], b[L - 1], V::dinv(M)[L - 1], x[L - 1], M.coarse, lm[L - 1], M.cratio,
                               c->st);
      // b and D^{-1} read once, x written once; per step one apply and the update
      prof_end(c, IMEX_PROF_PMG_APPLY_COARSE, 3.0 * sizeof(T) * nodes(L - 1),
               (M.coarse - 1) * (sipg_flops_per_node(c->d, M.N[L - 1]) + 6.0) * nodes(L - 1) + 2.0 * nodes(L - 1),
               arith_t<T>());
      TRY(cuda_check(c, cudaGetLastError(), "pmg_coarse_cluster"));
    }
  }
  if (crc != 0)
    TRY(pmg_smooth<T>(c, L - 1, M.coarse, lm[L - 1], M.cratio, (L > 1 && !clus) ? PMG_PRESET : PMG_FROM_ZERO,
                      b[L - 1], x[L - 1]));
  for (int l = L - 2; l >= 0; --l) {
    prof_mark(c, IMEX_PROF_PMG_VEC, true);
    if (pmg_prolong<T>(c->d, c->gp.ne, M.N[l], M.N[l + 1], x[l + 1], x[l], M.I[l], c->st) != 0)
      return fail(c, IMEX_EINVAL, "p-multigrid: unsupported level pair");
    prof_end(c, IMEX_PROF_PMG_VEC, sizeof(T) * (2.0 * nodes(l) + nodes(l + 1)), xfer_flops(l), arith_t<T>());
    TRY(pmg_smooth<T>(c, l, M.pre, lm[l], M.ratio, PMG_FROM_X, b[l], x[l]));
  }
  return cuda_check(c, cudaGetLastError(), "pmg_vcycle");
}

// Tune the launch shape of the periodic constant-viscosity apply on N points of type T
// (nsys systems of the space's size n, its line operators ops): times each shape on the
// work vectors x, y (contents irrelevant) and records the choice.
template <typename T>
imex_status tune_apply(imex_ctx* c, int N, int nsys, size_t n, const LineOps<T>* ops, const T* x, T* y) {
  for (int k = 0; k < c->d; ++k)
    if (c->gp.bc[k] != 0) return IMEX_OK;                 // the tuned kernels are the periodic ones
  const char* env = std::getenv("IMEX_TUNE");
  if (env && env[0] == '0') return IMEX_OK;
  const bool f32 = sizeof(T) == 4;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto& t : g_tune)
      if (t.d == c->d && t.N == N && t.f32 == (int)f32 && t.ne == c->gp.ne) return IMEX_OK;
  }
  // 2D FP64: no doubled block (static shared memory); one element more: 3D FP32, N = 7, 9
  const int nvar = (c->d == 2 && !f32) ? 2 : ((c->d == 3 && f32 && (N == 7 || N == 9)) ? 4 : 3);
  TuneEntry te{c->d, N, (int)f32, c->gp.ne, 0, {0, 0, 0, 0}};
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0), "event");
  CK(cudaEventCreate(&e1), "event");
  for (int v = 0; v < nvar; ++v) {
    SipgArgs<T> a = sipg_args<T>(x, y, nsys, (long long)n, nullptr, 1.0, nullptr, 0.0, 1.0, 0);
    a.ops = ops;
    a.variant = v;
    double best = 1e30;
    for (int it = 0; it < 7; ++it) {
      CK(cudaEventRecord(e0, c->st), "event");
      const int rc = sipg_apply<T>(c->gp, N, a, c->st);
      CK(cudaEventRecord(e1, c->st), "event");
      TRY(launch_check(c, rc, "sipg_apply(tune)"));
      CK(cudaEventSynchronize(e1), "event");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (it >= 2) best = std::min(best, 1e3 * (double)ms);
    }
    te.us[v] = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int pick = 0;
  for (int v = 1; v < nvar; ++v)
    if (te.us[v] < 0.97 * te.us[0] && te.us[v] < te.us[pick]) pick = v;
  te.variant = pick;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.push_back(te);
  return IMEX_OK;
}

// ---- solves ------------------------------------------------------------------------
// Poisson: L psi = b (b is overwritten by its mean-free part); psi: initial guess in, solution out
imex_status solve_poisson(imex_ctx* c, double* b, double* psi, long long* iters, double* res) {
  const size_t n = c->np;
  const int m = c->maxsys;
  seg_remove_mean(b, c->segp.t, c->cg_d + 6 * m, c->seg_partial, c->counters + 3, c->st);
  if (!c->diag_valid_p) {
    SipgArgs<double> a = sipg_args<double>(nullptr, c->cdiag, 1, (long long)n, nullptr, 1.0, nullptr, 0.0, 1.0, 0);
    TRY(launch_check(c, sipg_diag<double>(c->gp, c->Np, a, c->st), "sipg_diag(p)"));
    reciprocal<double>(c->cdiag, n, c->st);
    convert_d2f(c->cdiag, c->fdiag + 0, n, c->st);
    c->diag_valid_p = true;
  }
  // the diagonal buffers are shared with the Helmholtz solves: recompute if clobbered
  const double tol = c->desc.tol;
  const bool pm = c->pmg.kind == IMEX_PRECOND_PMG && c->desc.poisson == IMEX_POISSON_SIPG;
  if (pm) {
    if (c->desc.precision != IMEX_FP64) TRY(pmg_alloc<float>(c));
    TRY(pmg_setup(c));
  }
  if (c->desc.poisson == IMEX_POISSON_SIPG) {
    // launch shapes of the CG and V-cycle applies (first use only)
    if (c->desc.precision == IMEX_FP64) {
      TRY(tune_apply<double>(c, c->Np, 1, n, c->ops64_p, c->cx, c->cAp));
      for (int l = 1; pm && l < c->pmg.nlev; ++l)
        TRY(tune_apply<double>(c, c->pmg.N[l], 1, (size_t)c->gp.ne * ipow(c->pmg.N[l], c->d), c->pmg.ops64[l],
                               c->pmg.r64[l], c->pmg.ad64[l]));
    } else {
      TRY(tune_apply<float>(c, c->Np, 1, n, c->ops32_p, c->fx, c->fAp));
      for (int l = 1; pm && l < c->pmg.nlev; ++l)
        TRY(tune_apply<float>(c, c->pmg.N[l], 1, (size_t)c->gp.ne * ipow(c->pmg.N[l], c->d), c->pmg.ops32[l],
                              c->pmg.r32[l], c->pmg.ad32[l]));
    }
  }
  if (c->desc.precision == IMEX_FP64) {
    auto op = [&](const double* x, double* y) { return apply_pressure<double>(c, x, y, c->tmp); };
    auto opd = [&](const double* x, double* y, const CgScalars* d) {
      return apply_pressure<double>(c, x, y, c->tmp, d);
    };
    const bool fused = c->desc.poisson == IMEX_POISSON_SIPG && !c->batched;
    imex_status s = pcg(c, c->segp, op, opd, fused, b, psi, c->cdiag, tol, c->desc.maxit, true, {1}, iters, res, pm);
    seg_remove_wmean(psi, c->mass_p, c->segp.t, c->cg_d + 6 * m, c->seg_partial, c->counters + 3, c->st);
    return s;
  }
  // mixed: FP32 operator and preconditioner, FP64 iterate and residual with reliable updates
  auto op64 = [&](const double* x, double* y) { return apply_pressure<double>(c, x, y, c->tmp); };
  // (the FP32 operator runs in the CG loop only: a batch group skips its stopped instances)
  auto op32 = [&](const float* x, float* y) { return apply_pressure<float>(c, x, y, c->fvtmp, nullptr, true); };
  auto op32d = [&](const float* x, float* y, const CgScalars* d) {
    return apply_pressure<float>(c, x, y, c->fvtmp, d);
  };
  const bool fused = c->desc.poisson == IMEX_POISSON_SIPG && !c->batched;
  TRY(pcg_mixed(c, c->segp, op64, op32, op32d, fused, b, psi, c->fdiag, tol, c->desc.maxit, true, {1}, iters, res,
                pm));
  seg_remove_wmean(psi, c->mass_p, c->segp.t, c->cg_d + 6 * m, c->seg_partial, c->counters + 3, c->st);
  return IMEX_OK;
}

// Helmholtz: (M + gamma A(nu)) x = rhs, d components; x: initial guess in, solution out.
imex_status solve_helmholtz(imex_ctx* c, const double* rhs, double* x, const double* nu, double gamma,
                            long long* iters, double* res, bool keep_kx = false) {
  const size_t n = c->nv;
  const int d = c->d;
  // Jacobi diagonal of M + gamma A(nu)  (stored in cdiag + np region-free slot: use cdiag[np..])
  double* dg = c->cdiag + c->np;
  float* fdg = c->fdiag + c->np;
  if (nu == nullptr) {
    // viscosity constant per element: M and A(nu) do not change between stages
    if (!c->kdiag_valid || c->kdiag_nu != nu_const(c)) {
      SipgArgs<double> a = sipg_args<double>(nullptr, c->kdiag, 1, (long long)n, nullptr, nu_const(c), nullptr, 0.0,
                                             1.0, 0);
      vel_flags(c, a, false);
      TRY(launch_check(c, sipg_diag<double>(c->gv, c->Nv, a, c->st), "sipg_diag(v)"));
      c->kdiag_valid = true;
      c->kdiag_nu = nu_const(c);
    }
    helm_diag(dg, c->mass_v, c->kdiag, gamma, c->batched ? c->edt : nullptr, ipow(c->Nv, d), n, c->st);
  } else {
    SipgArgs<double> a = sipg_args<double>(nullptr, dg, 1, (long long)n, nu, nu_const(c), nullptr, 1.0, gamma, 0);
    vel_flags(c, a, true);
    TRY(launch_check(c, sipg_diag<double>(c->gv, c->Nv, a, c->st), "sipg_diag(v)"));
    reciprocal<double>(dg, n, c->st);
  }
  const double tol = c->desc.tol;
  // the chunk graphs depend on gamma, on whether the viscosity is a field and on its constant
  // value (captured into the kernels' arguments)
  const std::vector<unsigned long long> hkey = {2, bits(gamma), addr(nu), (unsigned long long)d, bits(nu_const(c))};
  if (!nu && !c->batched) {
    if (c->desc.precision == IMEX_FP64) TRY(tune_apply<double>(c, c->Nv, d, n, c->ops64_v, c->cx, c->cAp));
    else TRY(tune_apply<float>(c, c->Nv, d, n, c->ops32_v, c->fx, c->fAp));
  }
  if (c->desc.precision == IMEX_FP64) {
    auto op = [&](const double* xx, double* yy) { return apply_helm<double>(c, xx, yy, d, nu, gamma); };
    auto opd = [&](const double* xx, double* yy, const CgScalars* dd) {
      return apply_helm<double>(c, xx, yy, d, nu, gamma, dd);
    };
    return pcg(c, c->segv, op, opd, nu == nullptr && !c->batched, rhs, x, dg, tol, c->desc.maxit, false,
               hkey, iters, res);
  }
  convert_d2f(dg, fdg, n, c->st);
  const float* fnu = nullptr;
  if (nu) { convert_d2f(nu, c->fnu, n, c->st); fnu = c->fnu; }
  // keep_kx: the FP64-class residual apply computes K x into cz and forms (M + gamma dt_e K) x
  // elementwise, so that K of the solution is left for F_d1 of the same stage
  auto op64 = [&](const double* xx, double* yy) -> imex_status {
    if (!keep_kx) return apply_helm<double>(c, xx, yy, d, nu, gamma);
    SipgArgs<double> a = sipg_args<double>(xx, c->cz, d, (long long)n, nu, nu_const(c), nullptr, 0.0, 1.0, 0);
    a.ops = c->ops64_v;
    vel_flags(c, a, false);
    prof_mark(c, IMEX_PROF_HELMHOLTZ_F64, true);
    const int rc = apply_dispatch<double>(c, c->gv, c->Nv, a);
    prof_end(c, IMEX_PROF_HELMHOLTZ_F64, 8.0 * (double)n * (2.0 * d + (nu ? 1.0 : 0.0)),
             sipg_flops_per_node(d, c->Nv) * n * d, arith_of<double>(c));
    TRY(launch_check(c, rc, "sipg_apply(Kx)"));
    kx_combine(yy, xx, c->mass_v, c->cz, gamma, c->batched ? c->edt : nullptr, ipow(c->Nv, d), n, d, 0, c->st);
    return IMEX_OK;
  };
  auto op32 = [&](const float* xx, float* yy) { return apply_helm<float>(c, xx, yy, d, fnu, gamma, nullptr, true); };
  auto op32d = [&](const float* xx, float* yy, const CgScalars* dd) {
    return apply_helm<float>(c, xx, yy, d, fnu, gamma, dd);
  };
  TRY(pcg_mixed(c, c->segv, op64, op32, op32d, fnu == nullptr && !c->batched, rhs, x, fdg, tol, c->desc.maxit, false,
                hkey, iters, res));
  if (keep_kx) {
    c->kx_ready = true;            // the last residual check applied K to the solution x
    c->kx_for = x;
  }
  return IMEX_OK;
}

// ---- right-hand sides ---------------------------------------------------------------
FieldSpec spec(int kind, const double* p) {
  FieldSpec f;
  f.kind = kind;
  for (int i = 0; i < 8; ++i) f.p[i] = p[i];
  return f;
}

bool has_boundary(const imex_ctx* c) {
  for (int k = 0; k < c->d; ++k)
    if (!c->desc.periodic[k]) return true;
  return false;
}

// Dirichlet data at time t into c->vb (or nullptr if all periodic)
imex_status eval_vb(imex_ctx* c, double t, const double** out) {
  if (!has_boundary(c)) { *out = nullptr; return IMEX_OK; }
  TRY(launch_check(c, eval_field(c->gv, c->Nv, 0, spec(c->bc_kind, c->bc_p), t, nullptr, (long long)c->nv, c->vb,
                                 c->st), "eval_field(vb)"));
  *out = c->vb;
  return IMEX_OK;
}

imex_status eval_nu(imex_ctx* c, double t, const double* v, double* nu) {
  if (c->nu_kind == IMEX_NU_FIELD) {
    CK(cudaMemcpyAsync(nu, c->nu_fixed, c->nv * sizeof(double), cudaMemcpyDeviceToDevice, c->st), "cp nu");
    return IMEX_OK;
  }
  return launch_check(c, eval_field(c->gv, c->Nv, 1, spec(c->nu_kind, c->nu_p), t, v, (long long)c->nv, nu, c->st),
                      "eval_field(nu)");
}

// nu pointer for the operators: nullptr for constant viscosity
const double* nu_ptr(const imex_ctx* c, const double* nu) { return variable_nu(c) ? nu : nullptr; }

// F_d3 = -D(nu D.v) into out; if E != nullptr also E += F_d2 = sum_k D_k(nu D_c v_k) (variable nu)
imex_status graddiv(imex_ctx* c, const double* v, const double* nu, double* fd3, double* fd2_acc) {
  // the mixed form evaluates the derivatives in float-float
  // words per node moved by the four derivative forms (in, nu, out)
  auto deriv = [&](const DerivArgs<double>& x) {
    const double d = c->d;
    const double w[4] = {d + 1.0 + (x.nu ? 1.0 : 0.0), 1.0 + d, d + d * d + (x.nu ? 1.0 : 0.0), d * d + 2.0 * d};
    prof_mark(c, IMEX_PROF_DERIV, true);
    const int rc = ff_class(c) ? dg_deriv_ff(c->gv, c->Nv, x, c->st) : dg_deriv<double>(c->gv, c->Nv, x, c->st);
    prof_end(c, IMEX_PROF_DERIV, 8.0 * w[x.op] * c->nv, 0.0, ff_class(c) ? IMEX_ARITH_FF : IMEX_ARITH_FP64);
    return rc;
  };
  DerivArgs<double> a{};
  a.op = 0; a.in = v; a.stride = (long long)c->nv; a.nu = nu_ptr(c, nu); a.nu0 = nu_const(c); a.out = c->phi;
  a.inst_nu = c->batched && a.nu == nullptr;
  TRY(launch_check(c, deriv(a), "dg_deriv(div)"));
  DerivArgs<double> b{};
  b.op = 1; b.in = c->phi; b.stride = (long long)c->nv; b.coef = -1.0; b.out = fd3;
  TRY(launch_check(c, deriv(b), "dg_deriv(grad)"));
  if (fd2_acc) {
    DerivArgs<double> j{};
    j.op = 2; j.in = v; j.stride = (long long)c->nv; j.nu = nu_ptr(c, nu); j.nu0 = nu_const(c); j.out = c->jac;
    j.inst_nu = c->batched && j.nu == nullptr;
    TRY(launch_check(c, deriv(j), "dg_deriv(jac)"));
    DerivArgs<double> q{};
    q.op = 3; q.in = c->jac; q.stride = (long long)c->nv; q.coef = 1.0; q.out = fd2_acc;
    TRY(launch_check(c, deriv(q), "dg_deriv(divT)"));
  }
  return IMEX_OK;
}

// stage right-hand sides at (t, v, nu): E = F_c + F_d2 + F_d3, Fd1, Fd3, Fs (Fs may be nullptr)
imex_status stage_rhs(imex_ctx* c, double t, const double* v, const double* nu, const double* vb, double* E,
                      double* Fd1, double* Fd3, double* Fs) {
  const size_t nt = c->nv * c->d;
  // K v left by the Helmholtz solve that produced v (same viscosity, no Dirichlet data)
  const bool use_kx = c->kx_ready && c->kx_for == v && vb == nullptr;
  c->kx_ready = false;
  // IMEX_MIXED_FAST applies the explicit operators (convection, F_d1) in FP32 from FP32
  // copies of v and the boundary data; the stage storage and every combination stay FP64
  const bool f32 = c->desc.precision == IMEX_MIXED_FAST;
  if (f32) {
    convert_d2f(v, c->fx, nt, c->st);
    if (vb) convert_d2f(vb, c->fr, nt, c->st);
    ConvArgs<float> ca{c->fx, (long long)c->nv, vb ? c->fr : nullptr, 1.f, c->fp};
    prof_mark(c, IMEX_PROF_CONV, true);
    const int rc = dg_conv<float>(c->gv, c->Nv, ca, c->st);
    prof_end(c, IMEX_PROF_CONV, 4.0 * nt * (vb ? 3.0 : 2.0), conv_flops_per_elem(c->d, c->Nv) * c->gv.ne,
             IMEX_ARITH_FP32);
    TRY(launch_check(c, rc, "dg_conv(f32)"));
    f2d(c->fp, E, nt, c->st);
  } else {
    // IMEX_MIXED: FP64 fields, float-float arithmetic on the FP32 pipes (about 48 bits);
    // IMEX_FP64: FP64 arithmetic throughout
    ConvArgs<double> ca{v, (long long)c->nv, vb, 1.0, E};
    prof_mark(c, IMEX_PROF_CONV, true);
    const int rc = c->desc.precision == IMEX_MIXED ? dg_conv_ff(c->gv, c->Nv, ca, c->st)
                                                   : dg_conv<double>(c->gv, c->Nv, ca, c->st);
    prof_end(c, IMEX_PROF_CONV, 8.0 * nt * (vb ? 3.0 : 2.0), conv_flops_per_elem(c->d, c->Nv) * c->gv.ne,
             c->desc.precision == IMEX_MIXED ? IMEX_ARITH_FF : IMEX_ARITH_FP64);
    TRY(launch_check(c, rc, "dg_conv"));
  }
  const bool varnu = variable_nu(c);
  if (varnu) {
    // E += F_d2 + F_d3 (F_d2 accumulated by the kernel)
    TRY(graddiv(c, v, nu, Fd3, E));
    LinComb lc{};
    lc.nterms = 2; lc.x[0] = E; lc.c[0] = 1.0; lc.x[1] = Fd3; lc.c[1] = 1.0;
    lincomb(E, lc, nt, c->st);
  } else {
    // constant nu: F_d2 + F_d3 = 0 exactly for the discrete operators; E = F_c
    TRY(graddiv(c, v, nu, Fd3, nullptr));
  }
  if (f32) {
    const float* fnu = nullptr;
    if (nu_ptr(c, nu)) {
      convert_d2f(nu, c->fnu, c->nv, c->st);
      fnu = c->fnu;
    }
    SipgArgs<float> a = sipg_args<float>(c->fx, c->fp, c->d, (long long)c->nv, fnu, nu_const(c), vb ? c->fr : nullptr,
                                         0.0, -1.0, 1);
    a.ops = c->ops32_v;
    vel_flags(c, a, false);
    TRY(launch_check(c, sipg_apply<float>(c->gv, c->Nv, a, c->st), "sipg_apply(Fd1, f32)"));
    f2d(c->fp, Fd1, nt, c->st);
  } else if (use_kx) {
    kx_combine(Fd1, v, c->mass_v, c->cz, 0.0, nullptr, 1, c->nv, c->d, 1, c->st);
  } else {
    SipgArgs<double> a = sipg_args<double>(v, Fd1, c->d, (long long)c->nv, nu_ptr(c, nu), nu_const(c), vb, 0.0, -1.0,
                                           1);
    a.ops = c->ops64_v;
    vel_flags(c, a, false);
    TRY(launch_check(c, apply_dispatch<double>(c, c->gv, c->Nv, a), "sipg_apply(Fd1)"));
  }
  if (Fs) {
    TRY(launch_check(c, eval_field(c->gv, c->Nv, 2, spec(c->f_kind, c->f_p), t, nullptr, (long long)c->nv, Fs, c->st),
                     "eval_field(f)"));
  }
  return IMEX_OK;
}

// divergence / mass-flux stabilisation of the projected velocity v (in place):
// (M + A_D + A_C) v~ = M v by CG with the inverse mass as preconditioner, from v
imex_status stabilize(imex_ctx* c, double* v) {
  const size_t nt = c->nv * c->d;
  if (stab_speed(c->gv, c->Nv, v, (long long)c->nv, c->stab_speed, c->st) != 0)
    return fail(c, IMEX_EINVAL, "stabilisation: unsupported (d, P)");
  diag_mul(c, c->tmp, v, c->mass_v, c->nv, c->d);
  const double zd = c->stab_zd, zc = c->stab_zc, dt = c->cur_dt;
  auto op = [&](const double* x, double* y) -> imex_status {
    return launch_check(c, stab_apply(c->gv, c->Nv, x, y, (long long)c->nv, c->stab_speed, zd, zc, dt, c->st) == 0
                               ? 0 : -1, "stab_apply");
  };
  auto opd = [&](const double* x, double* y, const CgScalars*) { return op(x, y); };   // (no fused dot)
  double res = 0.0;
  (void)nt;
  return pcg(c, c->segs, op, opd, false, c->tmp, v, c->stab_minv, c->desc.tol, c->desc.maxit, false,
             {3, bits(zd), bits(zc), bits(dt)}, &c->stab_iters, &res);
}

// projection: psi from L psi = B v' - int (n.w) q, then v'' = v' - G psi (written to out).
// Stage projections (mode 1) solve for a potential of size about tau p (tau = dt c_i for an
// RK stage, the subinterval length for an SDC correction): the previous stage's potential,
// scaled by the ratio of the two tau, is the initial guess.  The final projection (mode 2,
// a small correction) starts from zero in its own buffer and leaves the stage potential.
imex_status project(imex_ctx* c, const double* vin, const double* wdata, int mode, double* out, double tau = 0.0) {
  c->kx_ready = false;
  // the mixed form evaluates the projection's divergence and gradient in float-float
  const bool ffa = ff_class(c);
  DivArgs<double> da{vin, (long long)c->nv, wdata, mode, 1.0, c->bp};
  const int ar = ffa ? IMEX_ARITH_FF : IMEX_ARITH_FP64;
  prof_mark(c, IMEX_PROF_DIV, true);
  const int rcd = ffa ? dg_div_ff(c->gv, c->Nv, da, c->st) : dg_div<double>(c->gv, c->Nv, da, c->st);
  prof_end(c, IMEX_PROF_DIV, 8.0 * ((mode == 1 ? 2.0 : 1.0) * c->d * c->nv + c->np), 0.0, ar);
  TRY(launch_check(c, rcd, "dg_div"));
  double* psi = c->psi;
  if (mode == 2) {
    psi = c->psi_f;
    CK(cudaMemsetAsync(psi, 0, c->np * sizeof(double), c->st), "memset psi_f");
  } else if (c->psi_tau > 0.0 && tau > 0.0 && tau != c->psi_tau) {
    LinComb lc{};
    lc.nterms = 1;
    lc.x[0] = psi; lc.c[0] = tau / c->psi_tau;
    lincomb(psi, lc, c->np, c->st);
  }
  double res = 0.0;
  TRY(solve_poisson(c, c->bp, psi, &c->stats.poisson_iters, &res));
  if (mode != 2) c->psi_tau = tau > 0.0 ? tau : 0.0;
  c->stats.poisson_solves++;
  c->stats.max_poisson_res = std::max(c->stats.max_poisson_res, res);
  GradArgs<double> ga{psi, vin, (long long)c->nv, -1.0, out};
  prof_mark(c, IMEX_PROF_GRAD, true);
  const int rcg = ffa ? dg_grad_ff(c->gv, c->Nv, ga, c->st) : dg_grad<double>(c->gv, c->Nv, ga, c->st);
  prof_end(c, IMEX_PROF_GRAD, 8.0 * (2.0 * c->d * c->nv + c->np), 0.0, ar);
  TRY(launch_check(c, rcg, "dg_grad"));
  if (mode == 1 && (c->stab_zd > 0.0 || c->stab_zc > 0.0)) TRY(stabilize(c, out));
  return IMEX_OK;
}

// Helmholtz stage solve: v_out = (M + gamma A(nu))^{-1} (M g + gamma r_b(nu, vb)), initial guess g
imex_status helmholtz_stage(imex_ctx* c, const double* gfield, const double* nu, double gamma, const double* vb,
                            double* vout) {
  const size_t nt = c->nv * c->d;
  c->kx_ready = false;
  // rhs = M g + gamma r_b : r_b = -(A 0 - r_b(vb))
  diag_mul(c, c->tmp, gfield, c->mass_v, c->nv, c->d);
  if (vb) {
    SipgArgs<double> a = sipg_args<double>(c->cz, c->cp, c->d, (long long)c->nv, nu_ptr(c, nu), nu_const(c), vb, 0.0,
                                           -gamma, 0);
    a.ops = c->ops64_v;
    vel_flags(c, a, true);
    CK(cudaMemsetAsync(c->cz, 0, nt * sizeof(double), c->st), "memset");
    TRY(launch_check(c, sipg_apply<double>(c->gv, c->Nv, a, c->st), "sipg_apply(rb)"));
    LinComb lc{};
    lc.nterms = 2; lc.x[0] = c->tmp; lc.c[0] = 1.0; lc.x[1] = c->cp; lc.c[1] = 1.0;
    lincomb(c->tmp, lc, nt, c->st);
  }
  if (vout != gfield) CK(cudaMemcpyAsync(vout, gfield, nt * sizeof(double), cudaMemcpyDeviceToDevice, c->st), "cp");
  double res = 0.0;
  // the rhs lives in c->tmp; pcg uses cr/cz/cp/cAp as work space
  // without Dirichlet data F_d1 of the solution is -M^-1 K v, which the mixed form's last
  // residual check computes anyway
  const bool keep_kx = vb == nullptr && c->desc.precision == IMEX_MIXED;
  TRY(solve_helmholtz(c, c->tmp, vout, nu_ptr(c, nu), gamma, &c->stats.helmholtz_iters, &res, keep_kx));
  c->stats.helmholtz_solves++;
  c->stats.max_helmholtz_res = std::max(c->stats.max_helmholtz_res, res);
  return IMEX_OK;
}

// ---- Alg. 3 -------------------------------------------------------------------------
// Time-step scaling of the stage combinations: plain contexts fold dt into the coefficients;
// batch groups leave it to the per-element time step applied by the linear combination.
double dtc(const imex_ctx* c, double dt) { return c->batched ? 1.0 : dt; }
// time at fraction f of the step [t, t + dt]; batch groups pass the fraction and the field
// kernels add it to each instance's own time and step
double tat(const imex_ctx* c, double t, double dt, double f) { return c->batched ? f : t + f * dt; }
// linear combination of velocity-space vectors whose terms after the first nfixed are
// proportional to the time step
void lcomb_dt(imex_ctx* c, double* out, LinComb& lc, int nfixed, size_t n) {
  if (c->batched) {
    lc.edt = c->edt;
    lc.cstride = (long long)c->nv;
    lc.nd = ipow(c->Nv, c->d);
    lc.nfixed = nfixed;
  }
  lincomb(out, lc, n, c->st);
}

imex_status rk_step(imex_ctx* c, const Tab& tb, double* v, double t, double dt, bool final_projection) {
  c->cur_dt = dt;
  const int s = tb.s;
  const size_t nt = c->nv * c->d;
  const bool forcing = c->f_kind != IMEX_FORCE_NONE;
  const double* vb = nullptr;
  TRY(eval_vb(c, tat(c, t, dt, 0.0), &vb));
  TRY(eval_nu(c, tat(c, t, dt, 0.0), v, c->nu));
  TRY(stage_rhs(c, tat(c, t, dt, 0.0), v, c->nu, vb, c->E[0], c->Fd1[0], c->Fd3[0], forcing ? c->Fs[0] : nullptr));
  const double* vi = v;
  for (int i = 1; i < s; ++i) {
    const double ti = tat(c, t, dt, tb.c[i]);
    TRY(eval_vb(c, ti, &vb));
    if (forcing)
      TRY(launch_check(c, eval_field(c->gv, c->Nv, 2, spec(c->f_kind, c->f_p), ti, nullptr, (long long)c->nv,
                                     c->Fs[i], c->st), "eval_field(f)"));
    // line 4: v' = v + dt [sum_j a^EX_ij (E_j + Fd1_j + Fd3_j) + sum_{j<=i} a^IM_ij Fs_j]
    LinComb lc{};
    int k = 0;
    lc.x[k] = v; lc.c[k++] = 1.0;
    for (int j = 0; j < i; ++j) {
      const double a = dtc(c, dt) * tb.AE[i][j];
      if (a == 0.0) continue;
      lc.x[k] = c->E[j]; lc.c[k++] = a;
      lc.x[k] = c->Fd1[j]; lc.c[k++] = a;
      lc.x[k] = c->Fd3[j]; lc.c[k++] = a;
    }
    lc.nterms = k;
    lcomb_dt(c, c->vp, lc, 1, nt);
    if (forcing) {
      LinComb lf{};
      int q = 0;
      lf.x[q] = c->vp; lf.c[q++] = 1.0;
      for (int j = 0; j <= i; ++j)
        if (tb.AI[i][j] != 0.0) { lf.x[q] = c->Fs[j]; lf.c[q++] = dtc(c, dt) * tb.AI[i][j]; }
      lf.nterms = q;
      lcomb_dt(c, c->vp, lf, 1, nt);
    }
    // lines 5-6: projection
    TRY(project(c, c->vp, vb, 1, c->vpp, dtc(c, dt) * tb.c[i]));
    // line 7: nu_i
    TRY(eval_nu(c, ti, c->vpp, c->nu));
    // line 8: g_i
    LinComb lg{};
    k = 0;
    lg.x[k] = c->vpp; lg.c[k++] = 1.0;
    for (int j = 0; j < i; ++j) {
      const double a1 = dtc(c, dt) * (tb.AI[i][j] - tb.AE[i][j]);
      const double a3 = -dtc(c, dt) * tb.AE[i][j];
      if (a1 != 0.0) { lg.x[k] = c->Fd1[j]; lg.c[k++] = a1; }
      if (a3 != 0.0) { lg.x[k] = c->Fd3[j]; lg.c[k++] = a3; }
    }
    lg.nterms = k;
    lcomb_dt(c, c->g, lg, 1, nt);
    // line 9: Helmholtz solve into the stage buffer (reuse c->vp as v_i storage)
    TRY(helmholtz_stage(c, c->g, c->nu, dtc(c, dt) * tb.AI[i][i], vb, c->vp));
    c->stats.stages++;
    vi = c->vp;
    TRY(stage_rhs(c, ti, vi, c->nu, vb, c->E[i], c->Fd1[i], c->Fd3[i], nullptr));
    if (i < s - 1) {
      // v_i is only needed through its right-hand sides; keep nothing else
    }
  }
  // line 11: v = v_s + dt sum_i [(bE_i - aE_si) E_i + (bI_i - aI_si)(Fd1_i + Fs_i)]
  LinComb lc{};
  int k = 0;
  lc.x[k] = vi; lc.c[k++] = 1.0;
  for (int i = 0; i < s; ++i) {
    const double fe = tb.bE[i] - tb.AE[s - 1][i];
    const double fi = tb.bI[i] - tb.AI[s - 1][i];
    if (fe != 0.0) { lc.x[k] = c->E[i]; lc.c[k++] = dtc(c, dt) * fe; }
    if (fi != 0.0) {
      lc.x[k] = c->Fd1[i]; lc.c[k++] = dtc(c, dt) * fi;
      if (forcing) { lc.x[k] = c->Fs[i]; lc.c[k++] = dtc(c, dt) * fi; }
    }
  }
  lc.nterms = k;
  lcomb_dt(c, v, lc, 1, nt);
  if (final_projection) {
    TRY(project(c, v, nullptr, 2, c->vpp));
    CK(cudaMemcpyAsync(v, c->vpp, nt * sizeof(double), cudaMemcpyDeviceToDevice, c->st), "cp");
  }
  return IMEX_OK;
}

// ---- Alg. 4 -------------------------------------------------------------------------
imex_status sdc_step(imex_ctx* c, double* v, double t, double dt) {
  c->cur_dt = dt;
  const int M = c->sdc_M, K = c->sdc_K, d = c->d;
  const size_t nt = c->nv * d;
  const bool varnu = variable_nu(c);
  const bool fproj = varnu;
  const bool forcing = c->f_kind != IMEX_FORCE_NONE;
  // sub-nodes and quadrature weights w_{q,m} = int_{t_{m-1}}^{t_m} l_q (unit step)
  double x[16], tau[16];
  gll_points(M + 1, x);
  for (int m = 0; m <= M; ++m) tau[m] = 0.5 * (x[m] + 1.0);
  double W[16][16] = {{0}};
  {
    // integrate the Lagrange basis exactly with a Gauss rule of M+1 points
    const int ng = M + 1;
    double gx[16], gw[16];
    for (int i = 0; i < ng; ++i) {
      double z = -std::cos(M_PI * (i + 0.75) / (ng + 0.5));
      for (int it = 0; it < 100; ++it) {
        double p0 = 1, p1 = z, d0 = 0, d1 = 1;
        for (int kk = 2; kk <= ng; ++kk) {
          double p2 = ((2.0 * kk - 1) * z * p1 - (kk - 1.0) * p0) / kk;
          double d2 = d0 + (2.0 * kk - 1) * p1;
          p0 = p1; p1 = p2; d0 = d1; d1 = d2;
        }
        const double dz = p1 / d1;
        z -= dz;
        if (std::fabs(dz) < 1e-16) break;
      }
      double p0 = 1, p1 = z, d0 = 0, d1 = 1;
      for (int kk = 2; kk <= ng; ++kk) {
        double p2 = ((2.0 * kk - 1) * z * p1 - (kk - 1.0) * p0) / kk;
        double d2 = d0 + (2.0 * kk - 1) * p1;
        p0 = p1; p1 = p2; d0 = d1; d1 = d2;
      }
      gx[i] = z;
      gw[i] = 2.0 / ((1.0 - z * z) * d1 * d1);
    }
    for (int m = 1; m <= M; ++m) {
      const double a = tau[m - 1], b = tau[m];
      for (int q = 0; q <= M; ++q) {
        double s = 0.0;
        for (int i = 0; i < ng; ++i) {
          const double z = a + 0.5 * (gx[i] + 1.0) * (b - a);
          double l = 1.0;
          for (int r = 0; r <= M; ++r)
            if (r != q) l *= (z - tau[r]) / (tau[q] - tau[r]);
          s += 0.5 * (b - a) * gw[i] * l;
        }
        W[m][q] = s;
      }
    }
  }
  double tm[16], dts[16];
  for (int m = 0; m <= M; ++m) tm[m] = t + dt * tau[m];
  for (int m = 1; m <= M; ++m) dts[m] = tm[m] - tm[m - 1];
  // predictor
  CK(cudaMemcpyAsync(c->sv[0], v, nt * sizeof(double), cudaMemcpyDeviceToDevice, c->st), "cp");
  for (int m = 1; m <= M; ++m) {
    CK(cudaMemcpyAsync(c->sv[m], c->sv[m - 1], nt * sizeof(double), cudaMemcpyDeviceToDevice, c->st), "cp");
    TRY(rk_step(c, c->sdc_pred, c->sv[m], tm[m - 1], dts[m], fproj));
  }
  c->cur_dt = dt;              // the stabilisation scales with the step, not the subinterval
  const double* vb = nullptr;
  // F^EX_m = F_c + F_d2 + F_d3 at (v_m, nu_m); F^IM_m = F_d1(nu_{m-1}, v_m)
  auto f_ex = [&](int m, double* out) -> imex_status {
    TRY(eval_vb(c, tm[m], &vb));
    ConvArgs<double> ca{c->sv[m], (long long)c->nv, vb, 1.0, out};
    TRY(launch_check(c, dg_conv<double>(c->gv, c->Nv, ca, c->st), "dg_conv"));
    if (varnu) {
      TRY(graddiv(c, c->sv[m], c->snu[m], c->tmp, out));
      LinComb lc{};
      lc.nterms = 2; lc.x[0] = out; lc.c[0] = 1.0; lc.x[1] = c->tmp; lc.c[1] = 1.0;
      lincomb(out, lc, nt, c->st);
    }
    return IMEX_OK;
  };
  auto f_d1 = [&](const double* vm, const double* num, double tt, double* out) -> imex_status {
    TRY(eval_vb(c, tt, &vb));
    SipgArgs<double> a = sipg_args<double>(vm, out, d, (long long)c->nv, nu_ptr(c, num), nu_const(c), vb, 0.0, -1.0, 1);
    a.ops = c->ops64_v;
    return launch_check(c, sipg_apply<double>(c->gv, c->Nv, a, c->st), "sipg_apply(Fd1)");
  };
  for (int m = 0; m <= M; ++m) TRY(eval_nu(c, tm[m], c->sv[m], c->snu[m]));
  for (int m = 0; m < M; ++m) TRY(f_ex(m, c->sFEX[m]));
  for (int m = 1; m <= M; ++m) TRY(f_d1(c->sv[m], c->snu[m - 1], tm[m], c->sFIM[m]));
  double* Fp1 = c->Fd1[0];        // F'_d1 of the current subinterval
  double* Fp3 = c->Fd3[0];        // F'_d3
  double* gbuf = c->Fd1[1];       // right-hand side of the Helmholtz solve / scratch
  double* stage = c->E[0];        // F^{EX,k+1}_{m-1} while subinterval m runs
  double* fsbuf = c->Fd3[1];
  for (int k = 0; k < K; ++k) {
    // full right-hand sides F(t_q, v^k_q) = F^EX + F_d1(nu^k_q, v^k_q) + F_s for the quadrature term
    for (int q = 0; q <= M; ++q) {
      if (q < M) {
        CK(cudaMemcpyAsync(c->sFq[q], c->sFEX[q], nt * sizeof(double), cudaMemcpyDeviceToDevice, c->st), "cp");
      } else {
        TRY(f_ex(q, c->sFq[q]));
      }
      TRY(f_d1(c->sv[q], c->snu[q], tm[q], gbuf));
      LinComb lc{};
      int n = 0;
      lc.x[n] = c->sFq[q]; lc.c[n++] = 1.0;
      lc.x[n] = gbuf; lc.c[n++] = 1.0;
      if (forcing) {
        TRY(launch_check(c, eval_field(c->gv, c->Nv, 2, spec(c->f_kind, c->f_p), tm[q], nullptr, (long long)c->nv,
                                       fsbuf, c->st), "eval_field(f)"));
        lc.x[n] = fsbuf; lc.c[n++] = 1.0;
      }
      lc.nterms = n;
      lincomb(c->sFq[q], lc, nt, c->st);
    }
    // sweep through the subintervals; v^{k+1}_0 = v^0_0, nu^{k+1}_0 = nu^0_0, F^{EX,k+1}_0 = F^{EX,0}_0
    for (int m = 1; m <= M; ++m) {
      const double* new_fex_prev = (m == 1) ? c->sFEX[0] : stage;
      const double* nu_prev = c->snu[m - 1];         // nu^{k+1}_{m-1}
      TRY(eval_vb(c, tm[m], &vb));
      TRY(f_d1(c->sv[m], nu_prev, tm[m], Fp1));       // F'_d1 = F_d1(nu^{k+1}_{m-1}, v^k_m)
      TRY(graddiv(c, c->sv[m], nu_prev, Fp3, nullptr)); // F'_d3 = F_d3(nu^{k+1}_{m-1}, v^k_m)
      // v' = v^{k+1}_{m-1} + dt_m [F^{EX,k+1}_{m-1} + F'_d1 + F'_d3 - (F^{EX,k}_{m-1} + F^{IM,k}_m)] + S^k_m
      LinComb lc{};
      int n = 0;
      lc.x[n] = c->sv[m - 1]; lc.c[n++] = 1.0;
      lc.x[n] = new_fex_prev; lc.c[n++] = dts[m];
      lc.x[n] = Fp1; lc.c[n++] = dts[m];
      lc.x[n] = Fp3; lc.c[n++] = dts[m];
      lc.x[n] = c->sFEX[m - 1]; lc.c[n++] = -dts[m];
      lc.x[n] = c->sFIM[m]; lc.c[n++] = -dts[m];
      for (int q = 0; q <= M; ++q) { lc.x[n] = c->sFq[q]; lc.c[n++] = dt * W[m][q]; }
      lc.nterms = n;
      lincomb(c->vp, lc, nt, c->st);
      TRY(project(c, c->vp, vb, 1, c->vpp, dts[m]));
      // v3 - dt_m div(nu^{k+1}_{m-1} grad v3) = v'' - dt_m (F'_d1 + F'_d3)
      LinComb lg{};
      lg.nterms = 3;
      lg.x[0] = c->vpp; lg.c[0] = 1.0;
      lg.x[1] = Fp1; lg.c[1] = -dts[m];
      lg.x[2] = Fp3; lg.c[2] = -dts[m];
      lincomb(gbuf, lg, nt, c->st);
      TRY(helmholtz_stage(c, gbuf, nu_prev, dts[m], vb, c->vp));
      c->stats.stages++;
      if (fproj) {
        TRY(project(c, c->vp, nullptr, 2, c->vpp));
        CK(cudaMemcpyAsync(c->vp, c->vpp, nt * sizeof(double), cudaMemcpyDeviceToDevice, c->st), "cp");
      }
      CK(cudaMemcpyAsync(c->sv[m], c->vp, nt * sizeof(double), cudaMemcpyDeviceToDevice, c->st), "cp");
      TRY(eval_nu(c, tm[m], c->sv[m], c->snu[m]));                    // nu^{k+1}_m
      // F^{IM,k+1}_m = F_d1(nu^{k+1}_{m-1}, v^{k+1}_m)  (same lag as the initialisation)
      TRY(f_d1(c->sv[m], nu_prev, tm[m], c->sFIM[m]));
      if (m >= 2)
        CK(cudaMemcpyAsync(c->sFEX[m - 1], stage, nt * sizeof(double), cudaMemcpyDeviceToDevice, c->st), "cp");
      if (m < M) TRY(f_ex(m, stage));                                 // F^{EX,k+1}_m
    }
  }
  CK(cudaMemcpyAsync(v, c->sv[M], nt * sizeof(double), cudaMemcpyDeviceToDevice, c->st), "cp");
  return IMEX_OK;
}

// ---- IMEX BDF2 (Sec. 3.2.1) ----------------------------------------------------------
// One step from v = v^n at t, with v1 the extrapolated, v2 the projected and v3 the
// diffused velocity:
//   (1) v1 = [a0 v^n + a1 v^{n-1} + dt (b0 (F_c + F_d + F_d3)^n + b1 (...)^{n-1} + F_s(t + dt))] / g0,
//       where F_c + F_d + F_d3 = E + F_d1 + F_d3 (E = F_c + F_d2 + F_d3);
//   (2) projection of v1 with the boundary flux of v_b(t + dt), psi = (dt / g0) p'';
//   (3) v3 - (dt / g0) div(nu* grad v3) = v2 - (dt / g0)[b0 (F_d1 + F_d3)^n + b1 (...)^{n-1}],
//       nu* = b0 nu^n + b1 nu^{n-1}, v3 = v_b(t + dt) on the boundary;
//   (4) the additional projection (homogeneous Neumann data) when the viscosity varies.
// The first step after a start, a new state or a change of dt uses the IMEX Euler
// coefficients (a0 = b0 = g0 = 1, a1 = b1 = 0).
imex_status bdf2_step(imex_ctx* c, double* v, double t, double dt) {
  c->cur_dt = dt;
  const size_t nt = c->nv * c->d;
  const bool first = c->bdf_n == 0 || dt != c->bdf_dt;
  const double a0 = first ? 1.0 : 2.0, a1 = first ? 0.0 : -0.5;
  const double b0 = first ? 1.0 : 2.0, b1 = first ? 0.0 : -1.0;
  const double g0 = first ? 1.0 : 1.5;
  const bool forcing = c->f_kind != IMEX_FORCE_NONE;
  const bool varnu = variable_nu(c);
  c->kx_ready = false;
  const double* vb = nullptr;
  TRY(eval_vb(c, t, &vb));
  TRY(eval_nu(c, t, v, c->nu));
  TRY(stage_rhs(c, t, v, c->nu, vb, c->E[0], c->Fd1[0], c->Fd3[0], nullptr));
  TRY(eval_vb(c, t + dt, &vb));
  if (forcing)
    TRY(launch_check(c, eval_field(c->gv, c->Nv, 2, spec(c->f_kind, c->f_p), t + dt, nullptr, (long long)c->nv,
                                   c->Fs[0], c->st), "eval_field(f)"));
  // (1) extrapolation
  LinComb lc{};
  int k = 0;
  lc.x[k] = v; lc.c[k++] = a0 / g0;
  if (a1 != 0.0) { lc.x[k] = c->bdf_vprev; lc.c[k++] = a1 / g0; }
  const double* cur[3] = {c->E[0], c->Fd1[0], c->Fd3[0]};
  const double* prev[3] = {c->E[1], c->Fd1[1], c->Fd3[1]};
  for (int q = 0; q < 3; ++q) {
    lc.x[k] = cur[q]; lc.c[k++] = dt * b0 / g0;
    if (b1 != 0.0) { lc.x[k] = prev[q]; lc.c[k++] = dt * b1 / g0; }
  }
  if (forcing) { lc.x[k] = c->Fs[0]; lc.c[k++] = dt / g0; }
  lc.nterms = k;
  lincomb(c->vp, lc, nt, c->st);
  // (2) projection
  TRY(project(c, c->vp, vb, 1, c->vpp, dt / g0));
  // (3) diffusion with the extrapolated viscosity
  const double* nus = c->nu;
  if (varnu && b1 != 0.0) {
    LinComb ln{};
    ln.nterms = 2; ln.x[0] = c->nu; ln.c[0] = b0; ln.x[1] = c->bdf_nuprev; ln.c[1] = b1;
    lincomb(c->bdf_nustar, ln, c->nv, c->st);
    nus = c->bdf_nustar;
  }
  LinComb lg{};
  k = 0;
  lg.x[k] = c->vpp; lg.c[k++] = 1.0;
  lg.x[k] = c->Fd1[0]; lg.c[k++] = -dt * b0 / g0;
  lg.x[k] = c->Fd3[0]; lg.c[k++] = -dt * b0 / g0;
  if (b1 != 0.0) {
    lg.x[k] = c->Fd1[1]; lg.c[k++] = -dt * b1 / g0;
    lg.x[k] = c->Fd3[1]; lg.c[k++] = -dt * b1 / g0;
  }
  lg.nterms = k;
  lincomb(c->g, lg, nt, c->st);
  imex_status hs = helmholtz_stage(c, c->g, nus, dt / g0, vb, c->vp);
  TRY(hs);
  c->kx_ready = false;
  c->stats.stages++;
  // history: v^n, its right-hand sides and viscosity become the previous step's
  CK(cudaMemcpyAsync(c->bdf_vprev, v, nt * sizeof(double), cudaMemcpyDeviceToDevice, c->st), "cp");
  std::swap(c->E[0], c->E[1]);
  std::swap(c->Fd1[0], c->Fd1[1]);
  std::swap(c->Fd3[0], c->Fd3[1]);
  std::swap(c->nu, c->bdf_nuprev);
  // (4) additional projection
  if (varnu) {
    TRY(project(c, c->vp, nullptr, 2, c->vpp));
    CK(cudaMemcpyAsync(v, c->vpp, nt * sizeof(double), cudaMemcpyDeviceToDevice, c->st), "cp");
  } else {
    CK(cudaMemcpyAsync(v, c->vp, nt * sizeof(double), cudaMemcpyDeviceToDevice, c->st), "cp");
  }
  c->bdf_n++;
  c->bdf_dt = dt;
  return IMEX_OK;
}

imex_status check_state(imex_ctx* c) {
  reduce_max_abs(c->v, c->nv * c->d, c->partial, c->nblocks, c->dscal + 60, c->st);
  CK(cudaMemcpyAsync(c->hscal + 60, c->dscal + 60, sizeof(double), cudaMemcpyDeviceToHost, c->st), "cp");
  CK(cudaStreamSynchronize(c->st), "sync");
  const double m = c->hscal[60];
  c->stats.max_velocity = m;
  if (m != m) return fail(c, IMEX_EUNSTABLE, "NaN in the velocity");
  if (c->desc.vmax > 0 && m > c->desc.vmax) return fail(c, IMEX_EUNSTABLE, "velocity above the threshold");
  return IMEX_OK;
}

imex_status copy_in(imex_ctx* c, double* dst, const double* src, size_t n, int on_device) {
  CK(cudaMemcpyAsync(dst, src, n * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     c->st), "copy in");
  return IMEX_OK;
}
imex_status copy_out(imex_ctx* c, double* dst, const double* src, size_t n, int on_device) {
  CK(cudaMemcpyAsync(dst, src, n * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     c->st), "copy out");
  CK(cudaStreamSynchronize(c->st), "sync");
  return IMEX_OK;
}

imex_status alloc_sdc(imex_ctx* c) {
  const size_t nt = c->nv * c->d;
  const int M = c->sdc_M;
  while ((int)c->sv.size() < M + 1) {
    double *a, *b, *f1, *f2, *f3;
    TRY(dalloc(c, &a, nt));
    TRY(dalloc(c, &b, c->nv));
    TRY(dalloc(c, &f1, nt));
    TRY(dalloc(c, &f2, nt));
    TRY(dalloc(c, &f3, nt));
    c->sv.push_back(a); c->snu.push_back(b); c->sFEX.push_back(f1); c->sFIM.push_back(f2); c->sFq.push_back(f3);
  }
  return IMEX_OK;
}

imex_status alloc_stages(imex_ctx* c, int s) {
  const size_t nt = (size_t)std::max<long long>(c->ne_cap, c->gv.ne) * ipow(c->Nv, c->d) * c->d;
  while ((int)c->E.size() < s) {
    double *e, *f1, *f3, *fs;
    TRY(dalloc(c, &e, nt));
    TRY(dalloc(c, &f1, nt));
    TRY(dalloc(c, &f3, nt));
    TRY(dalloc(c, &fs, nt));
    c->E.push_back(e); c->Fd1.push_back(f1); c->Fd3.push_back(f3); c->Fs.push_back(fs);
  }
  return IMEX_OK;
}

// Layout of the instances in a context's buffers (the instance list c->inst, e0 contiguous
// from 0): element count, vector sizes, the per-instance tables, the CG segment tables and the
// mass diagonals.  Cached CUDA graphs depend on the layout and are dropped.
imex_status set_layout(imex_ctx* c) {
  const int d = c->d;
  long long ne = 0;
  for (const auto& I : c->inst) ne += I.ne;
  const int ni = (int)c->inst.size();
  if (ne > c->ne_cap || ni > c->ninst_cap || ni < 1) return fail(c, IMEX_EINVAL, "layout above capacity");
  c->gv.ne = c->gp.ne = (int)ne;
  const long long ndv = ipow(c->Nv, d), ndp = ipow(c->Np, d);
  c->nv = (size_t)ne * ndv;
  c->np = (size_t)ne * ndp;
  if (c->batched) {
    std::vector<int> ei(ne);
    for (int i = 0; i < ni; ++i)
      for (int e = 0; e < c->inst[i].ne; ++e) ei[c->inst[i].e0 + e] = i;
    CK(cudaMemcpy(c->inst_d, c->inst.data(), ni * sizeof(InstGeom), cudaMemcpyHostToDevice), "cp inst");
    CK(cudaMemcpy(c->elem_inst_d, ei.data(), ei.size() * sizeof(int), cudaMemcpyHostToDevice), "cp inst");
  }
  // element neighbours across the faces, for the kernels that would otherwise recompute
  // them per thread (index arithmetic with run-time divisions)
  {
    std::vector<int> nb((size_t)ne * 2 * d);
    for (int i = 0; i < ni; ++i) {
      const InstGeom& I = c->inst[i];
      for (int el = 0; el < I.ne; ++el) {
        const int ec[3] = {el % I.n[0], (el / I.n[0]) % I.n[1], el / (I.n[0] * I.n[1])};
        for (int k = 0; k < d; ++k)
          for (int side = 0; side < 2; ++side) {
            int cc[3] = {ec[0], ec[1], ec[2]};
            int j = cc[k] + (side ? 1 : -1);
            int v = -1;
            if (j >= 0 && j < I.n[k]) {
              cc[k] = j;
              v = I.e0 + cc[0] + I.n[0] * (cc[1] + I.n[1] * cc[2]);
            } else if (c->gv.bc[k] == 0) {
              cc[k] = j < 0 ? j + I.n[k] : j - I.n[k];
              v = I.e0 + cc[0] + I.n[0] * (cc[1] + I.n[1] * cc[2]);
            }
            nb[((size_t)(I.e0 + el) * d + k) * 2 + side] = v;
          }
      }
    }
    if (!c->nbr_d) TRY(dalloc(c, &c->nbr_d, (size_t)std::max<long long>(c->ne_cap, ne) * 2 * d));
    CK(cudaMemcpy(c->nbr_d, nb.data(), nb.size() * sizeof(int), cudaMemcpyHostToDevice), "cp nbr");
    c->gv.nbr = c->gp.nbr = c->nbr_d;
  }
  // CG systems: the pressure of each instance, and each velocity component of each
  // instance (component-major); the Jacobi diagonal of the velocity is shared by the
  // components of an instance
  std::vector<long long> offp(ni), lenp(ni), offv(d * ni), doffv(d * ni), lenv(d * ni);
  for (int i = 0; i < ni; ++i) {
    offp[i] = c->inst[i].e0 * ndp;
    lenp[i] = c->inst[i].ne * ndp;
    for (int k = 0; k < d; ++k) {
      offv[k * ni + i] = (long long)(k * c->nv) + c->inst[i].e0 * ndv;
      doffv[k * ni + i] = c->inst[i].e0 * ndv;
      lenv[k * ni + i] = c->inst[i].ne * ndv;
    }
  }
  const int pcap = (int)((c->ne_cap * ndp) / SEG_CHUNK + c->ninst_cap + 1);
  const int vcap = d * (int)((c->ne_cap * ndv) / SEG_CHUNK + c->ninst_cap + 1);
  TRY(make_seg(c, ni, offp.data(), offp.data(), lenp.data(), &c->segp, c->ninst_cap, pcap));
  TRY(make_seg(c, d * ni, offv.data(), doffv.data(), lenv.data(), &c->segv, d * c->ninst_cap, vcap));
  // mass diagonals: the diag kernel with alpha = 1, beta = 0
  SipgArgs<double> a = sipg_args<double>(nullptr, c->mass_v, 1, (long long)c->nv, nullptr, 0.0, nullptr, 1.0, 0.0, 0);
  TRY(launch_check(c, sipg_diag<double>(c->gv, c->Nv, a, c->st), "mass(v)"));
  SipgArgs<double> b = sipg_args<double>(nullptr, c->mass_p, 1, (long long)c->np, nullptr, 0.0, nullptr, 1.0, 0.0, 0);
  TRY(launch_check(c, sipg_diag<double>(c->gp, c->Np, b, c->st), "mass(p)"));
  c->diag_valid_p = false;
  c->kdiag_valid = false;
  c->pmg.ready = false;
  CK(cudaStreamSynchronize(c->st), "sync");
  for (auto& gr : c->graphs) cudaGraphExecDestroy(gr.exec);
  c->graphs.clear();
  return IMEX_OK;
}

// Device state of a context whose geometry (gv, gp, nv, np, stream) and instance list are
// set: tables, line operators, work vectors, CG systems, mass diagonals, stage storage.
imex_status init_ctx(imex_ctx* c) {
  const int d = c->d;
  const Geom& g = c->gv;
  imex_status s = IMEX_OK;
  auto bail = [&](imex_status e) { return e; };
  // tables
  {
    Tables<double>* h64 = new Tables<double>();
    Tables<float>* h32 = new Tables<float>();
    build_tables(h64, h32);
    s = dalloc(c, &c->dtab64, 1);
    if (s == IMEX_OK) s = dalloc(c, &c->dtab32, 1);
    if (s == IMEX_OK && cudaMemcpy(c->dtab64, h64, sizeof(*h64), cudaMemcpyHostToDevice) != cudaSuccess) s = IMEX_ECUDA;
    if (s == IMEX_OK && cudaMemcpy(c->dtab32, h32, sizeof(*h32), cudaMemcpyHostToDevice) != cudaSuccess) s = IMEX_ECUDA;
    if (s == IMEX_OK) init_const_lines(*h64);
    if (s == IMEX_OK) {
      const double hh[3] = {1.0, 1.0, 1.0};      // unit-size line operators, scaled per element
      LineOps<double>* o64 = new LineOps<double>();
      LineOps<float>* o32 = new LineOps<float>();
      const int Ns[2] = {c->Nv, c->Np};
      for (int sp = 0; sp < 2 && s == IMEX_OK; ++sp) {
        build_line_ops(*h64, Ns[sp], hh, d, o64, o32);
        LineOps<double>** p64 = sp == 0 ? &c->ops64_v : &c->ops64_p;
        LineOps<float>** p32 = sp == 0 ? &c->ops32_v : &c->ops32_p;
        s = dalloc(c, p64, 1);
        if (s == IMEX_OK) s = dalloc(c, p32, 1);
        if (s == IMEX_OK && cudaMemcpy(*p64, o64, sizeof(*o64), cudaMemcpyHostToDevice) != cudaSuccess) s = IMEX_ECUDA;
        if (s == IMEX_OK && cudaMemcpy(*p32, o32, sizeof(*o32), cudaMemcpyHostToDevice) != cudaSuccess) s = IMEX_ECUDA;
      }
      delete o64;
      delete o32;
    }
    delete h64;
    delete h32;
    if (s != IMEX_OK) return bail(s);
    c->gv.tab64 = c->gp.tab64 = c->dtab64;
    c->gv.tab32 = c->gp.tab32 = c->dtab32;
  }
  // buffers sized for the capacity: ne_cap elements, ninst_cap instances
  if (c->ne_cap < g.ne) c->ne_cap = g.ne;
  if (c->ninst_cap < (int)c->inst.size()) c->ninst_cap = (int)c->inst.size();
  const long long ndv = ipow(c->Nv, d), ndp = ipow(c->Np, d);
  const size_t nvc = (size_t)c->ne_cap * ndv, npc = (size_t)c->ne_cap * ndp;
  if (c->batched) {
    if ((s = dalloc(c, &c->inst_d, (size_t)c->ninst_cap)) != IMEX_OK) return bail(s);
    if ((s = dalloc(c, &c->elem_inst_d, (size_t)c->ne_cap)) != IMEX_OK) return bail(s);
    if ((s = dalloc(c, &c->edt, (size_t)c->ne_cap)) != IMEX_OK) return bail(s);
    c->gv.inst = c->gp.inst = c->inst_d;
    c->gv.elem_inst = c->gp.elem_inst = c->elem_inst_d;
  }
  const size_t nt = nvc * d;
  const size_t big = std::max(nt, npc);
  double** f64[] = {&c->v, &c->vp, &c->vpp, &c->g, &c->tmp, &c->vb, &c->cx, &c->cr, &c->cz, &c->cp, &c->cAp,
                     &c->ffx};
  for (double** p : f64) if ((s = dalloc(c, p, big)) != IMEX_OK) return bail(s);
  if ((s = dalloc(c, &c->nu, nvc)) != IMEX_OK) return bail(s);
  if ((s = dalloc(c, &c->nu_fixed, nvc)) != IMEX_OK) return bail(s);
  if ((s = dalloc(c, &c->phi, nvc)) != IMEX_OK) return bail(s);
  if ((s = dalloc(c, &c->jac, nvc * d * d)) != IMEX_OK) return bail(s);
  if ((s = dalloc(c, &c->psi, npc)) != IMEX_OK) return bail(s);
  if ((s = dalloc(c, &c->psi_f, npc)) != IMEX_OK) return bail(s);
  if ((s = dalloc(c, &c->bp, npc)) != IMEX_OK) return bail(s);
  if ((s = dalloc(c, &c->mass_v, nvc)) != IMEX_OK) return bail(s);
  if ((s = dalloc(c, &c->kdiag, nvc)) != IMEX_OK) return bail(s);
  if ((s = dalloc(c, &c->mass_p, npc)) != IMEX_OK) return bail(s);
  if ((s = dalloc(c, &c->cdiag, npc + nvc)) != IMEX_OK) return bail(s);
  float** f32[] = {&c->fx, &c->fr, &c->fp, &c->fAp};
  for (float** p : f32) if ((s = dalloc(c, p, big)) != IMEX_OK) return bail(s);
  if ((s = dalloc(c, &c->fdiag, npc + nvc)) != IMEX_OK) return bail(s);
  if ((s = dalloc(c, &c->fnu, nvc)) != IMEX_OK) return bail(s);
  if ((s = dalloc(c, &c->fvtmp, nt + npc)) != IMEX_OK) return bail(s);
  c->nblocks = 152 * 4;
  if ((s = dalloc(c, &c->partial, (size_t)c->nblocks * 8)) != IMEX_OK) return bail(s);
  c->apartial_cap = (size_t)(c->ne_cap + 64) * 3;
  if ((s = dalloc(c, &c->apartial, c->apartial_cap)) != IMEX_OK) return bail(s);
  if ((s = dalloc(c, &c->counters, 8)) != IMEX_OK) return bail(s);
  cudaMemsetAsync(c->counters, 0, 8 * sizeof(unsigned int), c->st);
  if ((s = dalloc(c, &c->persist_partial, 5 * 4096)) != IMEX_OK) return bail(s);
  if ((s = dalloc(c, &c->persist_bar, 4)) != IMEX_OK) return bail(s);
  c->use_persist = false;      // measured slower than the graph-replayed kernels; opt in with IMEX_PERSIST=1
  if (const char* e = std::getenv("IMEX_PERSIST")) c->use_persist = std::atoi(e) != 0;
  if ((s = dalloc(c, &c->dscal, 128)) != IMEX_OK) return bail(s);
  if ((s = dalloc(c, &c->iscal, 64)) != IMEX_OK) return bail(s);
  if (cudaMallocHost((void**)&c->hscal, 128 * sizeof(double)) != cudaSuccess) return bail(IMEX_ENOMEM);
  if (cudaMallocHost((void**)&c->hiscal, 64 * sizeof(int)) != cudaSuccess) return bail(IMEX_ENOMEM);
  {
    // CG systems: each instance's pressure, each velocity component of each instance
    c->maxsys = d * c->ninst_cap;
    const int nblk = d * (int)((c->ne_cap * ndv) / SEG_CHUNK + c->ninst_cap + 1) + 1;
    if ((s = dalloc(c, &c->seg_partial, (size_t)5 * nblk + 64)) != IMEX_OK) return bail(s);
    if ((s = dalloc(c, &c->cg_d, (size_t)12 * c->maxsys)) != IMEX_OK) return bail(s);
    if ((s = dalloc(c, &c->cg_i, (size_t)2 * c->maxsys)) != IMEX_OK) return bail(s);
    cudaMemsetAsync(c->cg_d, 0, 12 * c->maxsys * sizeof(double), c->st);
    if ((s = dalloc(c, &c->cg_f, (size_t)4 * c->maxsys)) != IMEX_OK) return bail(s);
    cudaMemsetAsync(c->cg_f, 0, 4 * c->maxsys * sizeof(float), c->st);
    cudaMemsetAsync(c->cg_i, 0, 2 * c->maxsys * sizeof(int), c->st);
    if (cudaMallocHost((void**)&c->cg_hd, 12 * c->maxsys * sizeof(double)) != cudaSuccess) return bail(IMEX_ENOMEM);
    if (cudaMallocHost((void**)&c->cg_hi, 2 * c->maxsys * sizeof(int)) != cudaSuccess) return bail(IMEX_ENOMEM);
  }
  cudaMemsetAsync(c->psi, 0, npc * sizeof(double), c->st);
  cudaMemsetAsync(c->v, 0, big * sizeof(double), c->st);
  if ((s = set_layout(c)) != IMEX_OK) return bail(s);
  if ((s = alloc_stages(c, 4)) != IMEX_OK) return bail(s);
  if (cudaStreamSynchronize(c->st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return bail(IMEX_ECUDA);
  return IMEX_OK;
}


// ---- batches ------------------------------------------------------------------------
// Two instances can share a batch group when every setting that is not per-instance matches:
// space (d, P, periodicity), precision, solvers, model kinds and the time integrator.
bool same_group(const imex_ctx* a, const imex_ctx* b) {
  if (a->d != b->d || a->Nv != b->Nv) return false;
  for (int k = 0; k < a->d; ++k)
    if ((a->desc.periodic[k] != 0) != (b->desc.periodic[k] != 0)) return false;
  if (a->desc.precision != b->desc.precision || a->desc.poisson != b->desc.poisson) return false;
  if (a->desc.tol != b->desc.tol || a->desc.maxit != b->desc.maxit || a->desc.vmax != b->desc.vmax) return false;
  if (a->nu_kind != b->nu_kind || a->bc_kind != b->bc_kind || a->f_kind != b->f_kind) return false;
  if (a->use_sdc || b->use_sdc || a->use_bdf2 || b->use_bdf2) return false;
  if (a->stab_zd > 0.0 || a->stab_zc > 0.0 || b->stab_zd > 0.0 || b->stab_zc > 0.0) return false;
  if (a->pmg.kind != b->pmg.kind || a->pmg.pre != b->pmg.pre || a->pmg.coarse != b->pmg.coarse ||
      a->pmg.ratio != b->pmg.ratio || a->pmg.cratio != b->pmg.cratio)
    return false;
  return std::memcmp(&a->tab, &b->tab, sizeof(Tab)) == 0;
}

// The union-mesh context of a batch group: the instances' elements concatenated in the
// given order, each vector field stored [component][union element][node], so that every
// operator is one launch over all instances and each CG system (an instance's pressure, or
// one velocity component of an instance) a segment of the union vectors.
imex_status create_union(const std::vector<imex_ctx*>& src, imex_ctx** out) {
  const imex_ctx* s0 = src[0];
  imex_ctx* c = new imex_ctx();
  c->desc = s0->desc;
  c->desc.stream = nullptr;
  c->d = s0->d;
  c->Nv = s0->Nv;
  c->Np = s0->Np;
  c->batched = true;
  c->tab = s0->tab;
  c->pmg.kind = s0->pmg.kind;
  c->pmg.pre = s0->pmg.pre;
  c->pmg.coarse = s0->pmg.coarse;
  c->pmg.ratio = s0->pmg.ratio;
  c->pmg.cratio = s0->pmg.cratio;
  c->nu_kind = s0->nu_kind;
  c->bc_kind = s0->bc_kind;
  c->f_kind = s0->f_kind;
  std::memcpy(c->nu_p, s0->nu_p, sizeof(c->nu_p));
  std::memcpy(c->bc_p, s0->bc_p, sizeof(c->bc_p));
  std::memcpy(c->f_p, s0->f_p, sizeof(c->f_p));
  long long ne = 0;
  for (const imex_ctx* x : src) {
    InstGeom I{};
    I.e0 = (int)ne;
    I.ne = x->gv.ne;
    for (int k = 0; k < 3; ++k) {
      I.n[k] = x->gv.n[k];
      I.lo[k] = x->gv.lo[k];
      I.h[k] = x->gv.h[k];
      I.hf[k] = x->gv.hf[k];
    }
    I.nu0 = x->nu_p[0];
    I.nu0f = (float)x->nu_p[0];
    I.dt = 0.0;
    I.t = x->t;
    std::memcpy(I.nu_p, x->nu_p, sizeof(I.nu_p));
    std::memcpy(I.bc_p, x->bc_p, sizeof(I.bc_p));
    std::memcpy(I.f_p, x->f_p, sizeof(I.f_p));
    c->inst.push_back(I);
    ne += x->gv.ne;
  }
  if (ne > (1LL << 30)) {
    delete c;
    return IMEX_EINVAL;
  }
  c->gv = s0->gv;
  c->gp = s0->gp;
  c->gv.ne = c->gp.ne = (int)ne;
  c->nv = (size_t)ne * ipow(c->Nv, c->d);
  c->np = (size_t)ne * ipow(c->Np, c->d);
  if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess) {
    delete c;
    return IMEX_ECUDA;
  }
  c->own_stream = true;
  imex_status s = init_ctx(c);
  if (s == IMEX_OK) s = alloc_stages(c, c->tab.s);
  // the instances' current fields, re-laid out per component
  const size_t ndv = ipow(c->Nv, c->d), ndp = ipow(c->Np, c->d);
  for (size_t i = 0; i < src.size() && s == IMEX_OK; ++i) {
    imex_ctx* x = src[i];
    if (cudaStreamSynchronize(x->st) != cudaSuccess) s = IMEX_ECUDA;
    for (int k = 0; k < c->d && s == IMEX_OK; ++k)
      if (cudaMemcpyAsync(c->v + k * c->nv + c->inst[i].e0 * ndv, x->v + k * x->nv, x->nv * sizeof(double),
                          cudaMemcpyDeviceToDevice, c->st) != cudaSuccess)
        s = IMEX_ECUDA;
    if (s == IMEX_OK && cudaMemcpyAsync(c->psi + c->inst[i].e0 * ndp, x->psi, x->np * sizeof(double),
                                        cudaMemcpyDeviceToDevice, c->st) != cudaSuccess)
      s = IMEX_ECUDA;
  }
  if (s == IMEX_OK && cudaStreamSynchronize(c->st) != cudaSuccess) s = IMEX_ECUDA;
  if (s != IMEX_OK) {
    imex_destroy(c);
    return s;
  }
  *out = c;
  return IMEX_OK;
}

// per-instance time steps of a group: the instance table and the per-element step
imex_status set_group_dt(imex_ctx* c, const std::vector<double>& dt) {
  std::vector<double> edt(c->gv.ne);
  for (size_t i = 0; i < c->inst.size(); ++i) {
    c->inst[i].dt = dt[i];
    c->inst[i].dtf = (float)dt[i];
    for (int e = 0; e < c->inst[i].ne; ++e) edt[c->inst[i].e0 + e] = dt[i];
  }
  CK(cudaMemcpyAsync(c->edt, edt.data(), edt.size() * sizeof(double), cudaMemcpyHostToDevice, c->st), "cp dt");
  CK(cudaMemcpyAsync(c->inst_d, c->inst.data(), c->inst.size() * sizeof(InstGeom), cudaMemcpyHostToDevice, c->st),
     "cp inst");
  CK(cudaStreamSynchronize(c->st), "sync");
  return IMEX_OK;
}

// one step of every instance of a group, each with its own time step
imex_status group_step(imex_ctx* c) {
  TRY(rk_step(c, c->tab, c->v, 0.0, 1.0, variable_nu(c)));
  for (auto& I : c->inst) I.t += I.dt;
  CK(cudaMemcpyAsync(c->inst_d, c->inst.data(), c->inst.size() * sizeof(InstGeom), cudaMemcpyHostToDevice, c->st),
     "cp inst");
  c->stats.steps++;
  TRY(check_state(c));
  return IMEX_OK;
}


// ---- continuous batching ---------------------------------------------------------------
// A member of a server group: its geometry and parameters (InstGeom), and for a member that
// joins at the next regroup the initial field to set.
struct JoinSpec {
  InstGeom g;
  int flow;
  double flow_p[8];
  double t0;
};

// New member list of a group: the surviving members (by their current index, in order) and
// the joining ones; their fields are repacked into the new contiguous layout (survivors'
// velocity and pressure copied, joiners' velocity from their initial flow, pressure zero).
// dst may be c itself or a larger group taking over c's members (c then keeps its state).
imex_status regroup(imex_ctx* c, imex_ctx* dst, const std::vector<int>& keep, const std::vector<JoinSpec>& join) {
  const int d = c->d;
  const size_t ndv = ipow(c->Nv, d), ndp = ipow(c->Np, d);
  std::vector<InstGeom> ni;
  long long e0 = 0;
  for (int i : keep) {
    InstGeom I = c->inst[i];
    I.e0 = (int)e0;
    e0 += I.ne;
    ni.push_back(I);
  }
  for (const auto& j : join) {
    InstGeom I = j.g;
    I.e0 = (int)e0;
    e0 += I.ne;
    ni.push_back(I);
  }
  if (e0 > dst->ne_cap || (long long)ni.size() > dst->ninst_cap) return fail(c, IMEX_EINVAL, "group capacity");
  if (ni.empty()) {
    c->inst.clear();
    return IMEX_OK;
  }
  const size_t nv_new = (size_t)e0 * ndv, np_new = (size_t)e0 * ndp;
  // survivors: old layout of c -> new layout in dst's scratch (tmp, bp)
  CK(cudaStreamSynchronize(c->st), "sync");
  for (size_t q = 0; q < keep.size(); ++q) {
    const InstGeom& O = c->inst[keep[q]];
    const InstGeom& N = ni[q];
    for (int k = 0; k < d; ++k)
      CK(cudaMemcpyAsync(dst->tmp + k * nv_new + N.e0 * ndv, c->v + k * c->nv + O.e0 * ndv,
                         (size_t)O.ne * ndv * sizeof(double), cudaMemcpyDeviceToDevice, dst->st), "cp v");
    CK(cudaMemcpyAsync(dst->bp + N.e0 * ndp, c->psi + O.e0 * ndp, (size_t)O.ne * ndp * sizeof(double),
                       cudaMemcpyDeviceToDevice, dst->st), "cp psi");
  }
  // joiners: initial velocity from the analytic flow on the instance's own mesh
  for (size_t q = 0; q < join.size(); ++q) {
    const InstGeom& N = ni[keep.size() + q];
    Geom g1 = dst->gv;
    g1.inst = nullptr;
    g1.elem_inst = nullptr;
    g1.ne = N.ne;
    for (int k = 0; k < 3; ++k) {
      g1.n[k] = N.n[k];
      g1.lo[k] = N.lo[k];
      g1.h[k] = N.h[k];
      g1.hf[k] = N.hf[k];
    }
    double pp[8];
    std::memcpy(pp, join[q].flow_p, sizeof(pp));
    TRY(launch_check(dst, eval_field(g1, dst->Nv, 0, spec(join[q].flow, pp), join[q].t0, nullptr, (long long)nv_new,
                                     dst->tmp + N.e0 * ndv, dst->st), "eval_field(join)"));
    CK(cudaMemsetAsync(dst->bp + N.e0 * ndp, 0, (size_t)N.ne * ndp * sizeof(double), dst->st), "memset psi");
  }
  CK(cudaMemcpyAsync(dst->v, dst->tmp, d * nv_new * sizeof(double), cudaMemcpyDeviceToDevice, dst->st), "cp v");
  CK(cudaMemcpyAsync(dst->psi, dst->bp, np_new * sizeof(double), cudaMemcpyDeviceToDevice, dst->st), "cp psi");
  dst->psi_tau = keep.empty() ? 0.0 : c->psi_tau;    // groups count tau in units of their members' steps
  dst->inst = ni;
  return set_layout(dst);
}

// An empty server group with the settings of the given mesh and models and room for
// ne_cap elements and ninst_cap instances; its first member joins through regroup.
imex_status create_group(const imex_mesh_desc& desc, int nu_kind, int bc_kind, int f_kind, const InstGeom& first,
                         long long ne_cap, int ninst_cap, imex_ctx** out) {
  imex_ctx* c = new imex_ctx();
  c->desc = desc;
  c->desc.stream = nullptr;
  c->d = desc.dim;
  c->Nv = desc.P + 1;
  c->Np = desc.P;
  c->batched = true;
  named_tableau("CB3e", &c->tab);
  c->nu_kind = nu_kind;
  c->bc_kind = bc_kind;
  c->f_kind = f_kind;
  Geom g{};
  g.d = c->d;
  g.idt = 1.0;
  g.idtf = 1.f;
  for (int k = 0; k < 3; ++k) {
    g.n[k] = first.n[k];
    g.lo[k] = first.lo[k];
    g.h[k] = first.h[k];
    g.hf[k] = first.hf[k];
  }
  g.ne = first.ne;
  c->gv = g;
  c->gp = g;
  for (int k = 0; k < 3; ++k) {
    const bool per = (k >= c->d) || desc.periodic[k];
    c->gv.bc[k] = per ? 0 : 1;
    c->gp.bc[k] = per ? 0 : 2;
  }
  c->inst.push_back(first);
  c->inst[0].e0 = 0;
  c->ne_cap = std::max<long long>(ne_cap, first.ne);
  c->ninst_cap = std::max(ninst_cap, 1);
  if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess) {
    delete c;
    return IMEX_ECUDA;
  }
  c->own_stream = true;
  imex_status s = init_ctx(c);
  if (s == IMEX_OK) s = alloc_stages(c, c->tab.s);
  if (s != IMEX_OK) {
    imex_destroy(c);
    return s;
  }
  *out = c;
  return IMEX_OK;
}

// device bytes of one instance's share of a group's buffers (velocity nodes nv per
// component, pressure nodes np, s stages)
double footprint_bytes(int d, long long nv, long long np, int s) {
  const double f64v = 11.0 * d + 4.0 + d * d + 2.0 + 4.0 * s * d;    // work vectors, fields, stages, diagonals
  const double f32v = 5.0 * d + 2.0;
  return (double)nv * (8.0 * f64v + 4.0 * f32v) + (double)np * (8.0 * 6.0 + 4.0 * 2.0) + 256.0;
}

}  // namespace

// =====================================================================================
// C ABI
// =====================================================================================
extern "C" {

imex_status imex_create(const imex_mesh_desc* desc, imex_ctx** out) {
  if (!desc || !out) return IMEX_EINVAL;
  *out = nullptr;
  const int d = desc->dim;
  if (d != 2 && d != 3) return IMEX_EINVAL;
  if (desc->P < 2 || desc->P > IMEX_MAXN - 1) return IMEX_EINVAL;
  for (int k = 0; k < d; ++k) {
    if (desc->nelem[k] < 1) return IMEX_EINVAL;
    if (!(desc->hi[k] > desc->lo[k])) return IMEX_EINVAL;
  }
  if (desc->precision != IMEX_FP64 && desc->precision != IMEX_MIXED && desc->precision != IMEX_MIXED_FAST)
    return IMEX_EINVAL;
  if (desc->poisson != IMEX_POISSON_SIPG && desc->poisson != IMEX_POISSON_CONSISTENT) return IMEX_EINVAL;
  imex_ctx* c = new imex_ctx();
  c->desc = *desc;
  if (c->desc.tol <= 0) c->desc.tol = 1e-12;
  if (c->desc.maxit <= 0) c->desc.maxit = 5000;
  c->d = d;
  c->Nv = desc->P + 1;
  c->Np = desc->P;
  long long ne = 1;
  Geom g{};
  g.idt = 1.0;
  g.idtf = 1.f;
  g.d = d;
  for (int k = 0; k < 3; ++k) {
    g.n[k] = (k < d) ? desc->nelem[k] : 1;
    g.lo[k] = (k < d) ? desc->lo[k] : 0.0;
    g.h[k] = (k < d) ? (desc->hi[k] - desc->lo[k]) / desc->nelem[k] : 1.0;
    g.hf[k] = (float)g.h[k];
    ne *= g.n[k];
  }
  if (ne > (1LL << 30)) { delete c; return IMEX_EINVAL; }
  g.ne = (int)ne;
  c->gv = g;
  c->gp = g;
  for (int k = 0; k < 3; ++k) {
    const bool per = (k >= d) || desc->periodic[k];
    c->gv.bc[k] = per ? 0 : 1;
    c->gp.bc[k] = per ? 0 : 2;
  }
  c->nv = (size_t)ne * ipow(c->Nv, d);
  c->np = (size_t)ne * ipow(c->Np, d);
  if (desc->stream) {
    c->st = (cudaStream_t)desc->stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess) { delete c; return IMEX_ECUDA; }
    c->own_stream = true;
  }
  InstGeom I{};
  I.e0 = 0;
  I.ne = g.ne;
  for (int k = 0; k < 3; ++k) {
    I.n[k] = g.n[k];
    I.lo[k] = g.lo[k];
    I.h[k] = g.h[k];
    I.hf[k] = g.hf[k];
  }
  I.dt = 1.0;
  I.dtf = 1.f;
  c->inst.push_back(I);
  const imex_status s = init_ctx(c);
  if (s != IMEX_OK) {
    imex_destroy(c);
    return s;
  }
  named_tableau("CB3e", &c->tab);
  *out = c;
  return IMEX_OK;
}

void imex_destroy(imex_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  for (auto& P : c->profc)
    for (auto& e : P.ev) cudaEventDestroy(e);
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  for (void* p : c->allocs) cudaFree(p);
  if (c->hscal) cudaFreeHost(c->hscal);
  if (c->hiscal) cudaFreeHost(c->hiscal);
  if (c->cg_hd) cudaFreeHost(c->cg_hd);
  if (c->cg_hi) cudaFreeHost(c->cg_hi);
  if (c->own_stream && c->st) cudaStreamDestroy(c->st);
  delete c;
}

const char* imex_last_error(const imex_ctx* c) { return c ? c->err.c_str() : "null context"; }

imex_status imex_sizes(const imex_ctx* c, long long* nvel, long long* npres) {
  if (!c) return IMEX_EINVAL;
  if (nvel) *nvel = (long long)c->nv;
  if (npres) *npres = (long long)c->np;
  return IMEX_OK;
}

imex_status imex_set_tableau(imex_ctx* c, int s, const double* cc, const double* AI, const double* bI,
                             const double* AE, const double* bE) {
  if (!c || !cc || !AI || !bI || !AE || !bE || s < 2 || s > 8) return fail(c, IMEX_EINVAL, "bad tableau arguments");
  Tab t;
  t.s = s;
  for (int i = 0; i < s; ++i) {
    t.c[i] = cc[i]; t.bI[i] = bI[i]; t.bE[i] = bE[i];
    for (int j = 0; j < s; ++j) { t.AI[i][j] = AI[i * s + j]; t.AE[i][j] = AE[i * s + j]; }
  }
  if (!valid_tableau(t)) return fail(c, IMEX_EINVAL, "tableau is not of CK form");
  TRY(alloc_stages(c, s));
  c->tab = t;
  c->use_sdc = false;
  c->use_bdf2 = false;
  return IMEX_OK;
}

imex_status imex_set_tableau_named(imex_ctx* c, const char* name) {
  if (!c || !name) return IMEX_EINVAL;
  Tab t;
  if (!named_tableau(name, &t)) return fail(c, IMEX_EINVAL, std::string("unknown tableau ") + name);
  TRY(alloc_stages(c, t.s));
  c->tab = t;
  c->use_sdc = false;
  c->use_bdf2 = false;
  return IMEX_OK;
}

imex_status imex_set_sdc(imex_ctx* c, int M, int K, const char* predictor) {
  if (!c || M < 1 || M > 8 || K < 0 || K > 200) return fail(c, IMEX_EINVAL, "bad SDC parameters");
  Tab t;
  if (!named_tableau(predictor ? predictor : "EULER", &t)) return fail(c, IMEX_EINVAL, "unknown predictor");
  TRY(alloc_stages(c, t.s));
  c->sdc_M = M; c->sdc_K = K; c->sdc_pred = t;
  TRY(alloc_sdc(c));
  c->use_sdc = true;
  c->use_bdf2 = false;
  return IMEX_OK;
}

imex_status imex_set_stabilization(imex_ctx* c, double zeta_d, double zeta_c) {
  if (!c || !(zeta_d >= 0.0) || !(zeta_c >= 0.0)) return IMEX_EINVAL;
  if (c->batched) return fail(c, IMEX_EINVAL, "stabilisation of batched instances is not supported");
  if ((zeta_d > 0.0 || zeta_c > 0.0) && !c->stab_speed) {
    const size_t nt = c->nv * c->d;
    TRY(dalloc(c, &c->stab_speed, (size_t)c->gv.ne));
    TRY(dalloc(c, &c->stab_minv, nt));
    for (int k = 0; k < c->d; ++k)
      CK(cudaMemcpyAsync(c->stab_minv + k * c->nv, c->mass_v, c->nv * sizeof(double), cudaMemcpyDeviceToDevice,
                         c->st), "cp");
    reciprocal<double>(c->stab_minv, nt, c->st);
    const long long off = 0, len = (long long)nt;
    TRY(make_seg(c, 1, &off, &off, &len, &c->segs, 1, (int)(nt / SEG_CHUNK) + 2));
  }
  c->stab_zd = zeta_d;
  c->stab_zc = zeta_c;
  return IMEX_OK;
}

imex_status imex_stabilize(imex_ctx* c, const double* v, double dt, double* out, int on_device) {
  if (!c || !v || !out || !(dt > 0.0)) return IMEX_EINVAL;
  if (!(c->stab_zd > 0.0 || c->stab_zc > 0.0)) return fail(c, IMEX_EINVAL, "stabilisation is off");
  const size_t nt = c->nv * c->d;
  TRY(copy_in(c, c->vpp, v, nt, on_device));
  const double saved = c->cur_dt;
  c->cur_dt = dt;
  c->stab_iters = 0;
  imex_status s = stabilize(c, c->vpp);
  c->cur_dt = saved;
  TRY(s);
  return copy_out(c, out, c->vpp, nt, on_device);
}

imex_status imex_set_bdf2(imex_ctx* c) {
  if (!c) return IMEX_EINVAL;
  TRY(alloc_stages(c, 2));
  if (!c->bdf_vprev) {
    TRY(dalloc(c, &c->bdf_vprev, c->nv * c->d));
    TRY(dalloc(c, &c->bdf_nuprev, c->nv));
    TRY(dalloc(c, &c->bdf_nustar, c->nv));
  }
  c->use_bdf2 = true;
  c->use_sdc = false;
  c->bdf_n = 0;
  return IMEX_OK;
}

imex_status imex_set_viscosity_const(imex_ctx* c, double nu) {
  if (!c || !(nu >= 0)) return fail(c, IMEX_EINVAL, "bad viscosity");
  c->nu_kind = IMEX_NU_CONST;
  c->nu_p[0] = nu;
  return IMEX_OK;
}

imex_status imex_set_viscosity_model(imex_ctx* c, int kind, const double* p, int np) {
  if (!c || kind < IMEX_NU_CONST || kind > IMEX_NU_VELOCITY || np < 0 || np > 8 || (np > 0 && !p))
    return fail(c, IMEX_EINVAL, "bad viscosity model");
  if (kind == IMEX_NU_VELOCITY && (np < 3 || !(p[2] > 0))) return fail(c, IMEX_EINVAL, "nu(v) needs nu0, nu1, vmax");
  c->nu_kind = kind;
  std::memset(c->nu_p, 0, sizeof(c->nu_p));
  for (int i = 0; i < np; ++i) c->nu_p[i] = p[i];
  return IMEX_OK;
}

imex_status imex_set_viscosity_field(imex_ctx* c, const double* nu, int on_device) {
  if (!c || !nu) return IMEX_EINVAL;
  TRY(copy_in(c, c->nu_fixed, nu, c->nv, on_device));
  c->nu_kind = IMEX_NU_FIELD;
  return IMEX_OK;
}

imex_status imex_set_boundary(imex_ctx* c, int kind, const double* p, int np) {
  if (!c || kind < IMEX_FLOW_NONE || kind > IMEX_FLOW_VV || np < 0 || np > 8 || (np > 0 && !p))
    return fail(c, IMEX_EINVAL, "bad boundary kind");
  c->bc_kind = kind;
  std::memset(c->bc_p, 0, sizeof(c->bc_p));
  for (int i = 0; i < np; ++i) c->bc_p[i] = p[i];
  return IMEX_OK;
}

imex_status imex_set_forcing(imex_ctx* c, int kind, const double* p, int np) {
  if (!c || kind < IMEX_FORCE_NONE || kind > IMEX_FORCE_VV || np < 0 || np > 8 || (np > 0 && !p))
    return fail(c, IMEX_EINVAL, "bad forcing kind");
  if (kind == IMEX_FORCE_TGTRAVEL_VARNU && c->d != 2) return fail(c, IMEX_EINVAL, "forcing is 2D only");
  if (kind == IMEX_FORCE_VV && c->d != 3) return fail(c, IMEX_EINVAL, "forcing is 3D only");
  c->f_kind = kind;
  std::memset(c->f_p, 0, sizeof(c->f_p));
  for (int i = 0; i < np; ++i) c->f_p[i] = p[i];
  return IMEX_OK;
}

imex_status imex_set_state(imex_ctx* c, double t, const double* v, int on_device) {
  if (!c || !v) return IMEX_EINVAL;
  TRY(copy_in(c, c->v, v, c->nv * c->d, on_device));
  c->t = t;
  c->bdf_n = 0;                 // a new state restarts IMEX BDF2 with an Euler step
  return IMEX_OK;
}

imex_status imex_init_flow(imex_ctx* c, int kind, const double* p, int np, double t) {
  if (!c || kind < IMEX_FLOW_NONE || kind > IMEX_FLOW_VV || np < 0 || np > 8 || (np > 0 && !p))
    return fail(c, IMEX_EINVAL, "bad flow kind");
  double pp[8] = {0};
  for (int i = 0; i < np; ++i) pp[i] = p[i];
  TRY(launch_check(c, eval_field(c->gv, c->Nv, 0, spec(kind, pp), t, nullptr, (long long)c->nv, c->v, c->st),
                   "eval_field"));
  c->t = t;
  c->bdf_n = 0;
  return IMEX_OK;
}

imex_status imex_step(imex_ctx* c, double dt, int nsteps) {
  if (!c || !(dt > 0) || nsteps < 0) return fail(c, IMEX_EINVAL, "bad step arguments");
  if (has_boundary(c) && c->bc_kind == IMEX_FLOW_NONE)
    return fail(c, IMEX_EINVAL, "non-periodic mesh needs boundary data (imex_set_boundary)");
  auto t0 = std::chrono::steady_clock::now();
  c->stats.poisson_solves = c->stats.helmholtz_solves = 0;
  c->stats.poisson_iters = c->stats.helmholtz_iters = 0;
  c->stats.refinements = 0;
  c->stats.max_poisson_res = c->stats.max_helmholtz_res = 0.0;
  for (int n = 0; n < nsteps; ++n) {
    imex_status s = c->use_bdf2 ? bdf2_step(c, c->v, c->t, dt)
                    : c->use_sdc ? sdc_step(c, c->v, c->t, dt)
                                 : rk_step(c, c->tab, c->v, c->t, dt, variable_nu(c));
    if (s != IMEX_OK) return s;
    c->t += dt;
    c->stats.steps++;
    TRY(check_state(c));
  }
  CK(cudaStreamSynchronize(c->st), "sync");
  c->stats.last_call_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return IMEX_OK;
}

imex_status imex_get_velocity(imex_ctx* c, double* out, int on_device) {
  if (!c || !out) return IMEX_EINVAL;
  return copy_out(c, out, c->v, c->nv * c->d, on_device);
}
imex_status imex_get_pressure(imex_ctx* c, double* out, int on_device) {
  if (!c || !out) return IMEX_EINVAL;
  return copy_out(c, out, c->psi, c->np, on_device);
}
imex_status imex_get_time(const imex_ctx* c, double* t) {
  if (!c || !t) return IMEX_EINVAL;
  *t = c->t;
  return IMEX_OK;
}
imex_status imex_get_stats(const imex_ctx* c, imex_stats* out) {
  if (!c || !out) return IMEX_EINVAL;
  *out = c->stats;
  return IMEX_OK;
}

imex_status imex_op_sipg(imex_ctx* c, int space, const double* x, double* y, int nsys, double alpha, double beta,
                         const double* nu, const double* gd, int minv, int arith, int on_device) {
  if (!c || !x || !y) return IMEX_EINVAL;
  const bool vel = space == IMEX_SPACE_VELOCITY;
  if (!vel && space != IMEX_SPACE_PRESSURE) return fail(c, IMEX_EINVAL, "bad space");
  if (nsys < 1 || nsys > 3 || (!vel && nsys != 1)) return fail(c, IMEX_EINVAL, "bad nsys");
  const size_t n = vel ? c->nv : c->np;
  const Geom& g = vel ? c->gv : c->gp;
  const int N = vel ? c->Nv : c->Np;
  TRY(copy_in(c, c->cx, x, n * nsys, on_device));
  const double* dnu = nullptr;
  if (nu && vel) { TRY(copy_in(c, c->nu, nu, c->nv, on_device)); dnu = c->nu; }
  const double* dg = nullptr;
  if (gd) { TRY(copy_in(c, c->vb, gd, n * nsys, on_device)); dg = c->vb; }
  const double nu0 = vel ? nu_const(c) : 1.0;
  if (arith != IMEX_ARITH_FP64 && arith != IMEX_ARITH_FP32 && arith != IMEX_ARITH_FF)
    return fail(c, IMEX_EINVAL, "bad arith");
  // timed as the pressure / Helmholtz classes: read x (and nu, g), write y
  const int cls64 = vel ? IMEX_PROF_HELMHOLTZ_F64 : IMEX_PROF_PRESSURE_F64;
  const int cls32 = vel ? IMEX_PROF_HELMHOLTZ_F32 : IMEX_PROF_PRESSURE_F32;
  const double words = (double)n * (2.0 * nsys + (dnu ? 1.0 : 0.0) + (dg ? nsys : 0.0));
  const double flops = sipg_flops_per_node(c->d, N) * n * nsys;
  if (arith == IMEX_ARITH_FF) {
    SipgArgs<double> a = sipg_args<double>(c->cx, c->cAp, nsys, (long long)n, dnu, nu0, dg, alpha, beta, minv);
    a.ops = line_ops<double>(c, vel);
    prof_mark(c, cls64, true);
    const int rc = sipg_apply_ff(g, N, a, c->ffx, c->st);
    prof_end(c, cls64, 8.0 * words, flops, IMEX_ARITH_FF);
    if (rc != 0) return fail(c, IMEX_EINVAL, "no float-float kernel for this operator");
    TRY(cuda_check(c, cudaGetLastError(), "sipg_apply_ff"));
  } else if (arith == IMEX_ARITH_FP64) {
    SipgArgs<double> a = sipg_args<double>(c->cx, c->cAp, nsys, (long long)n, dnu, nu0, dg, alpha, beta, minv);
    a.ops = line_ops<double>(c, vel);
    a.variant = tuned_variant(c, N, false);
    prof_mark(c, cls64, true);
    const int rc = sipg_apply<double>(g, N, a, c->st);
    prof_end(c, cls64, 8.0 * words, flops, IMEX_ARITH_FP64);
    TRY(launch_check(c, rc, "sipg_apply"));
  } else {
    convert_d2f(c->cx, c->fx, n * nsys, c->st);
    const float* fnu = nullptr;
    if (dnu) { convert_d2f(dnu, c->fnu, c->nv, c->st); fnu = c->fnu; }
    const float* fg = nullptr;
    if (dg) { convert_d2f(dg, c->fr, n * nsys, c->st); fg = c->fr; }
    SipgArgs<float> a = sipg_args<float>(c->fx, c->fAp, nsys, (long long)n, fnu, nu0, fg, alpha, beta, minv);
    a.ops = line_ops<float>(c, vel);
    a.variant = tuned_variant(c, N, true);
    prof_mark(c, cls32, true);
    const int rc = sipg_apply<float>(g, N, a, c->st);
    prof_end(c, cls32, 4.0 * words, flops, IMEX_ARITH_FP32);
    TRY(launch_check(c, rc, "sipg_apply(f32)"));
    f2d(c->fAp, c->cAp, n * nsys, c->st);
  }
  return copy_out(c, y, c->cAp, n * nsys, on_device);
}

imex_status imex_op_sipg_diag(imex_ctx* c, int space, double* y, double alpha, double beta, const double* nu,
                              int on_device) {
  if (!c || !y) return IMEX_EINVAL;
  const bool vel = space == IMEX_SPACE_VELOCITY;
  const size_t n = vel ? c->nv : c->np;
  const double* dnu = nullptr;
  if (nu && vel) { TRY(copy_in(c, c->nu, nu, c->nv, on_device)); dnu = c->nu; }
  SipgArgs<double> a = sipg_args<double>(nullptr, c->cAp, 1, (long long)n, dnu, vel ? nu_const(c) : 1.0, nullptr,
                                         alpha, beta, 0);
  TRY(launch_check(c, sipg_diag<double>(vel ? c->gv : c->gp, vel ? c->Nv : c->Np, a, c->st), "sipg_diag"));
  return copy_out(c, y, c->cAp, n, on_device);
}

// arith of the divergence, gradient and grad-div entry points: FP64 or float-float
static bool ff_arith(int arith, bool* ff) {
  *ff = arith == IMEX_ARITH_FF;
  return arith == IMEX_ARITH_FP64 || arith == IMEX_ARITH_FF;
}

imex_status imex_op_div(imex_ctx* c, const double* v, const double* w, int mode, double* b, int arith,
                        int on_device) {
  if (!c || !v || !b || mode < 0 || mode > 2 || (mode == 1 && !w)) return IMEX_EINVAL;
  bool ff = false;
  if (!ff_arith(arith, &ff)) return fail(c, IMEX_EINVAL, "bad arith");
  TRY(copy_in(c, c->cx, v, c->nv * c->d, on_device));
  if (mode == 1) TRY(copy_in(c, c->vb, w, c->nv * c->d, on_device));
  DivArgs<double> da{c->cx, (long long)c->nv, c->vb, mode, 1.0, c->bp};
  prof_mark(c, IMEX_PROF_DIV, true);
  const int rc = ff ? dg_div_ff(c->gv, c->Nv, da, c->st) : dg_div<double>(c->gv, c->Nv, da, c->st);
  prof_end(c, IMEX_PROF_DIV, 8.0 * ((mode == 1 ? 2.0 : 1.0) * c->d * c->nv + c->np), 0.0,
           ff ? IMEX_ARITH_FF : IMEX_ARITH_FP64);
  TRY(launch_check(c, rc, "dg_div"));
  return copy_out(c, b, c->bp, c->np, on_device);
}

imex_status imex_op_grad(imex_ctx* c, const double* psi, double* out, int arith, int on_device) {
  if (!c || !psi || !out) return IMEX_EINVAL;
  bool ff = false;
  if (!ff_arith(arith, &ff)) return fail(c, IMEX_EINVAL, "bad arith");
  TRY(copy_in(c, c->bp, psi, c->np, on_device));
  GradArgs<double> ga{c->bp, nullptr, (long long)c->nv, 1.0, c->cAp};
  prof_mark(c, IMEX_PROF_GRAD, true);
  const int rc = ff ? dg_grad_ff(c->gv, c->Nv, ga, c->st) : dg_grad<double>(c->gv, c->Nv, ga, c->st);
  prof_end(c, IMEX_PROF_GRAD, 8.0 * ((double)c->d * c->nv + c->np), 0.0, ff ? IMEX_ARITH_FF : IMEX_ARITH_FP64);
  TRY(launch_check(c, rc, "dg_grad"));
  return copy_out(c, out, c->cAp, c->nv * c->d, on_device);
}

imex_status imex_op_conv(imex_ctx* c, const double* v, const double* vb, double* out, int arith, int on_device) {
  if (!c || !v || !out) return IMEX_EINVAL;
  if (arith != IMEX_ARITH_FP64 && arith != IMEX_ARITH_FP32 && arith != IMEX_ARITH_FF)
    return fail(c, IMEX_EINVAL, "bad arith");
  const size_t nt = c->nv * c->d;
  TRY(copy_in(c, c->cx, v, nt, on_device));
  const double* dvb = nullptr;
  if (vb) { TRY(copy_in(c, c->vb, vb, nt, on_device)); dvb = c->vb; }
  if (arith == IMEX_ARITH_FP32) {
    convert_d2f(c->cx, c->fx, nt, c->st);
    if (dvb) convert_d2f(dvb, c->fr, nt, c->st);
    ConvArgs<float> ca{c->fx, (long long)c->nv, dvb ? c->fr : nullptr, 1.f, c->fp};
    prof_mark(c, IMEX_PROF_CONV, true);
    const int rc = dg_conv<float>(c->gv, c->Nv, ca, c->st);
    prof_end(c, IMEX_PROF_CONV, 4.0 * nt * (dvb ? 3.0 : 2.0), conv_flops_per_elem(c->d, c->Nv) * c->gv.ne,
             IMEX_ARITH_FP32);
    TRY(launch_check(c, rc, "dg_conv(f32)"));
    f2d(c->fp, c->cAp, nt, c->st);
  } else {
    ConvArgs<double> ca{c->cx, (long long)c->nv, dvb, 1.0, c->cAp};
    prof_mark(c, IMEX_PROF_CONV, true);
    const int rc = arith == IMEX_ARITH_FF ? dg_conv_ff(c->gv, c->Nv, ca, c->st)
                                          : dg_conv<double>(c->gv, c->Nv, ca, c->st);
    prof_end(c, IMEX_PROF_CONV, 8.0 * nt * (dvb ? 3.0 : 2.0), conv_flops_per_elem(c->d, c->Nv) * c->gv.ne, arith);
    TRY(launch_check(c, rc, "dg_conv"));
  }
  return copy_out(c, out, c->cAp, nt, on_device);
}

imex_status imex_op_graddiv(imex_ctx* c, const double* v, const double* nu, double* fd3, double* fd2, int arith,
                            int on_device) {
  if (!c || !v || !fd3) return IMEX_EINVAL;
  bool ff = false;
  if (!ff_arith(arith, &ff)) return fail(c, IMEX_EINVAL, "bad arith");
  const size_t nt = c->nv * c->d;
  TRY(copy_in(c, c->cx, v, nt, on_device));
  const int saved = c->nu_kind;
  const int saved_prec = c->desc.precision;
  const double* dnu = nullptr;
  if (nu) { TRY(copy_in(c, c->nu, nu, c->nv, on_device)); dnu = c->nu; c->nu_kind = IMEX_NU_FIELD; }
  CK(cudaMemsetAsync(c->cz, 0, nt * sizeof(double), c->st), "memset");
  c->desc.precision = ff ? IMEX_MIXED : IMEX_FP64;     // graddiv() picks float-float for the mixed form
  imex_status s = graddiv(c, c->cx, dnu, c->cAp, fd2 ? c->cz : nullptr);
  c->nu_kind = saved;
  c->desc.precision = saved_prec;
  TRY(s);
  TRY(copy_out(c, fd3, c->cAp, nt, on_device));
  if (fd2) TRY(copy_out(c, fd2, c->cz, nt, on_device));
  return IMEX_OK;
}

imex_status imex_solve_poisson(imex_ctx* c, const double* b, double* psi, int on_device) {
  if (!c || !b || !psi) return IMEX_EINVAL;
  TRY(copy_in(c, c->bp, b, c->np, on_device));
  CK(cudaMemsetAsync(c->psi, 0, c->np * sizeof(double), c->st), "memset");
  double res = 0.0;
  long long its = 0;
  TRY(solve_poisson(c, c->bp, c->psi, &its, &res));
  c->psi_tau = 0.0;
  c->stats.poisson_iters = its;
  c->stats.max_poisson_res = res;
  return copy_out(c, psi, c->psi, c->np, on_device);
}

imex_status imex_solve_helmholtz(imex_ctx* c, const double* gf, const double* nu, double gamma, const double* vb,
                                 double* v, int on_device) {
  if (!c || !gf || !v || !(gamma >= 0)) return IMEX_EINVAL;
  const size_t nt = c->nv * c->d;
  TRY(copy_in(c, c->g, gf, nt, on_device));
  const int saved = c->nu_kind;
  if (nu) { TRY(copy_in(c, c->nu, nu, c->nv, on_device)); c->nu_kind = IMEX_NU_FIELD; }
  const double* dvb = nullptr;
  if (vb) { TRY(copy_in(c, c->vb, vb, nt, on_device)); dvb = c->vb; }
  c->stats.helmholtz_iters = 0;
  imex_status s = helmholtz_stage(c, c->g, nu ? c->nu : nullptr, gamma, dvb, c->vpp);
  c->nu_kind = saved;
  TRY(s);
  return copy_out(c, v, c->vpp, nt, on_device);
}

imex_status imex_eval_field(imex_ctx* c, int what, int kind, const double* p, int np, double t, const double* v,
                            double* out, int on_device) {
  if (!c || !out || what < 0 || what > 2 || np < 0 || np > 8 || (np > 0 && !p)) return IMEX_EINVAL;
  double pp[8] = {0};
  for (int i = 0; i < np; ++i) pp[i] = p[i];
  const double* dv = nullptr;
  if (v) { TRY(copy_in(c, c->cx, v, c->nv * c->d, on_device)); dv = c->cx; }
  TRY(launch_check(c, eval_field(c->gv, c->Nv, what, spec(kind, pp), t, dv, (long long)c->nv, c->cAp, c->st),
                   "eval_field"));
  return copy_out(c, out, c->cAp, (what == 1 ? 1 : c->d) * c->nv, on_device);
}

imex_status imex_reduce(imex_ctx* c, int op, const double* x, const double* y, long long n, double* out,
                        int on_device) {
  if (!c || !x || !out || n < 0 || op < IMEX_REDUCE_DOT || op > IMEX_REDUCE_MAXABS || (op == IMEX_REDUCE_DOT && !y))
    return fail(c, IMEX_EINVAL, "bad reduction arguments");
  const size_t cap = std::max(c->nv * c->d, c->np);
  if (!on_device && (size_t)n > cap) return fail(c, IMEX_EINVAL, "host reduction larger than the context buffers");
  const double* dx = x;
  const double* dy = y;
  if (!on_device) {
    TRY(copy_in(c, c->cx, x, (size_t)n, 0));
    dx = c->cx;
    if (op == IMEX_REDUCE_DOT) { TRY(copy_in(c, c->cz, y, (size_t)n, 0)); dy = c->cz; }
  }
  double* res = c->dscal + 64;
  if (n == 0) {
    *out = 0.0;
    return IMEX_OK;
  }
  if (op == IMEX_REDUCE_DOT)
    dot_batched(dx, dy, (size_t)n, (long long)n, 1, c->partial, c->nblocks, res, c->st);
  else if (op == IMEX_REDUCE_SUM)
    reduce_sum(dx, (size_t)n, c->partial, c->nblocks, res, c->st);
  else
    reduce_max_abs(dx, (size_t)n, c->partial, c->nblocks, res, c->st);
  CK(cudaGetLastError(), "reduction");
  CK(cudaMemcpyAsync(c->hscal + 64, res, sizeof(double), cudaMemcpyDeviceToHost, c->st), "copy result");
  CK(cudaStreamSynchronize(c->st), "sync");
  *out = c->hscal[64];
  return IMEX_OK;
}

imex_status imex_set_pressure_precond(imex_ctx* c, int kind, const double* p, int np) {
  if (!c || (kind != IMEX_PRECOND_JACOBI && kind != IMEX_PRECOND_PMG) || np < 0 || np > 4 || (np > 0 && !p))
    return IMEX_EINVAL;
  imex_ctx::Pmg& M = c->pmg;
  int pre = M.pre, coarse = M.coarse;
  double ratio = M.ratio, cratio = M.cratio;
  if (np > 0) pre = (int)p[0];
  if (np > 1) coarse = (int)p[1];
  if (np > 2) ratio = p[2];
  if (np > 3) cratio = p[3];
  if (pre < 1 || pre > 16 || coarse < 1 || coarse > 64 || !(ratio > 1.0) || !(cratio > 1.0))
    return fail(c, IMEX_EINVAL, "bad p-multigrid parameters");
  M.kind = kind;
  M.pre = pre;
  M.coarse = coarse;
  M.ratio = ratio;
  M.cratio = cratio;
  for (auto& gr : c->graphs) cudaGraphExecDestroy(gr.exec);      // captured V-cycles change
  c->graphs.clear();
  return IMEX_OK;
}

imex_status imex_pmg_info(imex_ctx* c, int* nlev, int* N, double* lmax) {
  if (!c) return IMEX_EINVAL;
  TRY(pmg_setup(c));
  if (nlev) *nlev = c->pmg.nlev;
  for (int l = 0; l < c->pmg.nlev; ++l) {
    if (N) N[l] = c->pmg.N[l];
    if (lmax) lmax[l] = c->pmg.lmax[l];
  }
  return IMEX_OK;
}

imex_status imex_op_pmg_vcycle(imex_ctx* c, const double* r, double* z, const double* lmax, int arith,
                               int on_device) {
  if (!c || !r || !z || (arith != IMEX_ARITH_FP64 && arith != IMEX_ARITH_FP32)) return IMEX_EINVAL;
  TRY(pmg_setup(c));
  imex_ctx::Pmg& M = c->pmg;
  double lm[4];
  for (int l = 0; l < M.nlev; ++l) {
    lm[l] = lmax ? lmax[l] : M.lmax[l];
    if (!(lm[l] > 0.0)) return fail(c, IMEX_EINVAL, "bad lmax");
  }
  TRY(copy_in(c, c->bp, r, c->np, on_device));
  if (arith == IMEX_ARITH_FP64) {
    TRY(pmg_vcycle<double>(c, c->bp, c->psi_f, lm));
  } else {
    TRY(pmg_alloc<float>(c));
    for (int l = 0; l < M.nlev; ++l)
      convert_d2f(M.dinv64[l], M.dinv32[l], (size_t)c->gp.ne * ipow(M.N[l], c->d), c->st);
    convert_d2f(c->bp, c->fr, c->np, c->st);
    TRY(pmg_vcycle<float>(c, c->fr, c->fx, lm));
    f2d(c->fx, c->psi_f, c->np, c->st);
  }
  return copy_out(c, z, c->psi_f, c->np, on_device);
}

static double box_volume(const imex_ctx* c) {
  double vol = 1.0;
  for (int k = 0; k < c->d; ++k) vol *= c->desc.hi[k] - c->desc.lo[k];
  return vol;
}

imex_status imex_dissipation(imex_ctx* c, double* eps) {
  if (!c || !eps) return IMEX_EINVAL;
  if (c->batched) return fail(c, IMEX_EINVAL, "statistics of a single instance only");
  const double* nu = nullptr;
  if (variable_nu(c)) {
    TRY(eval_nu(c, c->t, c->v, c->nu));
    nu = c->nu;
  }
  if (dissipation_elems(c->gv, c->Nv, c->v, (long long)c->nv, nu, nu_const(c), c->tmp, c->st) != 0)
    return fail(c, IMEX_EINVAL, "dissipation: unsupported (d, P)");
  reduce_sum(c->tmp, (size_t)c->gv.ne, c->partial, c->nblocks, c->dscal + 42, c->st);
  CK(cudaMemcpyAsync(c->hscal + 42, c->dscal + 42, sizeof(double), cudaMemcpyDeviceToHost, c->st), "cp");
  CK(cudaStreamSynchronize(c->st), "sync");
  *eps = c->hscal[42] / box_volume(c);
  return IMEX_OK;
}

imex_status imex_energy_spectrum(imex_ctx* c, int M, int kmax, double* E) {
  if (!c || !E || kmax < 1 || kmax > 4096 || M < 2 || M > 1024 || (M & (M - 1))) return IMEX_EINVAL;
  if (c->batched) return fail(c, IMEX_EINVAL, "statistics of a single instance only");
  size_t npts = 1;
  for (int k = 0; k < c->d; ++k) npts *= (size_t)M;
  const size_t ng = npts * c->d;
  if (ng > ((size_t)1 << 31)) return fail(c, IMEX_EINVAL, "grid too large");
  if (ng > c->diag_grid_cap) {
    TRY(dalloc(c, &c->diag_grid, ng));
    c->diag_grid_cap = ng;
  }
  const int nb = 152 * 4;
  if ((size_t)nb * kmax + kmax > c->diag_part_cap) {
    TRY(dalloc(c, &c->diag_part, (size_t)nb * kmax + kmax));
    c->diag_part_cap = (size_t)nb * kmax + kmax;
  }
  double* dE = c->diag_part + (size_t)nb * kmax;
  if (energy_spectrum(c->gv, c->Nv, c->v, (long long)c->nv, M, kmax, box_volume(c), c->diag_grid, c->diag_part, nb,
                      dE, c->st) != 0)
    return fail(c, IMEX_EINVAL, "energy spectrum: unsupported arguments");
  TRY(cuda_check(c, cudaGetLastError(), "energy_spectrum"));
  CK(cudaMemcpyAsync(E, dE, kmax * sizeof(double), cudaMemcpyDeviceToHost, c->st), "cp");
  CK(cudaStreamSynchronize(c->st), "sync");
  return IMEX_OK;
}

imex_status imex_profile(imex_ctx* c, int enable) {
  if (!c) return IMEX_EINVAL;
  for (int k = 0; k < IMEX_PROF_NCLASS; ++k) {
    prof_flush(c, k);
    c->profc[k].n = 0;
    c->profc[k].ms = 0.0;
    c->profc[k].bytes = 0.0;
    c->profc[k].flops = 0.0;
    c->profc[k].arith = -1;
  }
  c->prof = enable != 0;
  return IMEX_OK;
}

imex_status imex_profile_read(imex_ctx* c, int cls, long long* launches, double* total_ms) {
  if (!c || cls < 0 || cls >= IMEX_PROF_NCLASS) return IMEX_EINVAL;
  CK(cudaStreamSynchronize(c->st), "sync");
  prof_flush(c, cls);
  if (launches) *launches = c->profc[cls].n;
  if (total_ms) *total_ms = c->profc[cls].ms;
  return IMEX_OK;
}

imex_status imex_profile_work(imex_ctx* c, int cls, double* bytes, double* flops, int* arith) {
  if (!c || cls < 0 || cls >= IMEX_PROF_NCLASS) return IMEX_EINVAL;
  if (bytes) *bytes = c->profc[cls].bytes;
  if (flops) *flops = c->profc[cls].flops;
  if (arith) *arith = c->profc[cls].arith;
  return IMEX_OK;
}

int imex_set_apply_variant(int d, int N, int fp32, long long ne, int variant) {
  if ((d != 2 && d != 3) || N < 2 || N > IMEX_MAXN || ne < 1 || variant < 0 || variant > 3 ||
      (d == 2 && !fp32 && variant == 2) || (variant == 3 && (d != 3 || !fp32 || (N != 7 && N != 9))))
    return IMEX_EINVAL;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (auto& t : g_tune)
    if (t.d == d && t.N == N && t.f32 == (fp32 ? 1 : 0) && t.ne == ne) {
      t.variant = variant;
      return IMEX_OK;
    }
  g_tune.push_back(TuneEntry{d, N, fp32 ? 1 : 0, ne, variant, {0, 0, 0, 0}});
  return IMEX_OK;
}

int imex_tuning_info(int i, int* d, int* N, int* fp32, long long* ne, int* variant, double* us) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (i < 0) return (int)g_tune.size();
  if (i >= (int)g_tune.size()) return -1;
  const TuneEntry& t = g_tune[i];
  if (d) *d = t.d;
  if (N) *N = t.N;
  if (fp32) *fp32 = t.f32;
  if (ne) *ne = t.ne;
  if (variant) *variant = t.variant;
  if (us) for (int k = 0; k < 4; ++k) us[k] = t.us[k];
  return (int)g_tune.size();
}

long long imex_launch_count(void) { return imex::launch_count(); }


// ---- batches of instances --------------------------------------------------------------
struct imex_batch {
  std::vector<imex_ctx*> groups;
  std::vector<std::vector<int>> members;   // per group: the caller's instance indices
  std::vector<int> grp, loc;               // per instance: group and position in it
  std::vector<double> group_ms;            // per group: wall time of the last imex_batch_step
  std::string err;
  imex_stats stats{};
};

imex_status imex_batch_create(imex_ctx* const* insts, int n, imex_batch** out) {
  if (!insts || n <= 0 || !out) return IMEX_EINVAL;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!insts[i] || insts[i]->batched) return IMEX_EINVAL;
    if (insts[i]->use_sdc || insts[i]->use_bdf2 || insts[i]->nu_kind == IMEX_NU_FIELD || insts[i]->stab_zd > 0.0 ||
        insts[i]->stab_zc > 0.0)
      return IMEX_EINVAL;
    if (has_boundary(insts[i]) && insts[i]->bc_kind == IMEX_FLOW_NONE) return IMEX_EINVAL;
  }
  imex_batch* b = new imex_batch();
  b->grp.assign(n, -1);
  b->loc.assign(n, -1);
  for (int i = 0; i < n; ++i) {
    int g = -1;
    for (size_t q = 0; q < b->members.size() && g < 0; ++q)
      if (same_group(insts[b->members[q][0]], insts[i])) g = (int)q;
    if (g < 0) {
      g = (int)b->members.size();
      b->members.emplace_back();
    }
    b->grp[i] = g;
    b->loc[i] = (int)b->members[g].size();
    b->members[g].push_back(i);
  }
  for (auto& m : b->members) {
    std::vector<imex_ctx*> src;
    for (int i : m) src.push_back(insts[i]);
    imex_ctx* c = nullptr;
    const imex_status s = create_union(src, &c);
    if (s != IMEX_OK) {
      imex_batch_destroy(b);
      return s;
    }
    b->groups.push_back(c);
  }
  *out = b;
  return IMEX_OK;
}

void imex_batch_destroy(imex_batch* b) {
  if (!b) return;
  for (imex_ctx* c : b->groups) imex_destroy(c);
  delete b;
}

const char* imex_batch_last_error(const imex_batch* b) { return b ? b->err.c_str() : "null batch"; }

int imex_batch_groups(const imex_batch* b) { return b ? (int)b->groups.size() : 0; }

imex_status imex_batch_step(imex_batch* b, const double* dt, int nsteps) {
  if (!b || !dt || nsteps < 0) return IMEX_EINVAL;
  const int n = (int)b->grp.size();
  for (int i = 0; i < n; ++i)
    if (!(dt[i] > 0)) return IMEX_EINVAL;
  auto t0 = std::chrono::steady_clock::now();
  // the groups run concurrently, each from its own host thread on its own stream
  std::vector<imex_status> st(b->groups.size(), IMEX_OK);
  b->group_ms.assign(b->groups.size(), 0.0);
  auto run = [&](size_t q) {
    const auto g0 = std::chrono::steady_clock::now();
    imex_ctx* c = b->groups[q];
    std::vector<double> gdt;
    for (int i : b->members[q]) gdt.push_back(dt[i]);
    c->stats.poisson_solves = c->stats.helmholtz_solves = 0;
    c->stats.poisson_iters = c->stats.helmholtz_iters = 0;
    c->stats.refinements = 0;
    c->stats.max_poisson_res = c->stats.max_helmholtz_res = 0.0;
    imex_status s = set_group_dt(c, gdt);
    for (int k = 0; k < nsteps && s == IMEX_OK; ++k) s = group_step(c);
    if (s == IMEX_OK && cudaStreamSynchronize(c->st) != cudaSuccess) s = IMEX_ECUDA;
    st[q] = s;
    b->group_ms[q] = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - g0).count();
  };
  // IMEX_BATCH_SERIAL=1 steps the groups one after the other from the calling thread
  const char* ser = std::getenv("IMEX_BATCH_SERIAL");
  if (b->groups.size() == 1 || (ser && std::atoi(ser) != 0)) {
    for (size_t q = 0; q < b->groups.size(); ++q) run(q);
  } else {
    std::vector<std::thread> th;
    for (size_t q = 0; q < b->groups.size(); ++q) th.emplace_back(run, q);
    for (auto& t : th) t.join();
  }
  imex_stats tot{};
  imex_status res = IMEX_OK;
  for (size_t q = 0; q < b->groups.size(); ++q) {
    const imex_stats& g = b->groups[q]->stats;
    tot.steps = std::max(tot.steps, g.steps);
    tot.stages += g.stages;
    tot.poisson_solves += g.poisson_solves;
    tot.helmholtz_solves += g.helmholtz_solves;
    tot.poisson_iters += g.poisson_iters;
    tot.helmholtz_iters += g.helmholtz_iters;
    tot.refinements += g.refinements;
    tot.max_poisson_res = std::max(tot.max_poisson_res, g.max_poisson_res);
    tot.max_helmholtz_res = std::max(tot.max_helmholtz_res, g.max_helmholtz_res);
    tot.max_velocity = std::max(tot.max_velocity, g.max_velocity);
    if (st[q] != IMEX_OK && res == IMEX_OK) {
      res = st[q];
      b->err = "group " + std::to_string(q) + ": " + b->groups[q]->err;
    }
  }
  tot.last_call_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  b->stats = tot;
  return res;
}

imex_status imex_batch_get_velocity(imex_batch* b, int i, double* out, int on_device) {
  if (!b || !out || i < 0 || i >= (int)b->grp.size()) return IMEX_EINVAL;
  imex_ctx* c = b->groups[b->grp[i]];
  const InstGeom& I = c->inst[b->loc[i]];
  const size_t ndv = ipow(c->Nv, c->d);
  const size_t n = (size_t)I.ne * ndv;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  for (int k = 0; k < c->d; ++k)
    if (cudaMemcpyAsync(out + k * n, c->v + k * c->nv + I.e0 * ndv, n * sizeof(double), kind, c->st) != cudaSuccess)
      return IMEX_ECUDA;
  return cudaStreamSynchronize(c->st) == cudaSuccess ? IMEX_OK : IMEX_ECUDA;
}

imex_status imex_batch_get_pressure(imex_batch* b, int i, double* out, int on_device) {
  if (!b || !out || i < 0 || i >= (int)b->grp.size()) return IMEX_EINVAL;
  imex_ctx* c = b->groups[b->grp[i]];
  const InstGeom& I = c->inst[b->loc[i]];
  const size_t ndp = ipow(c->Np, c->d);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (cudaMemcpyAsync(out, c->psi + I.e0 * ndp, (size_t)I.ne * ndp * sizeof(double), kind, c->st) != cudaSuccess)
    return IMEX_ECUDA;
  return cudaStreamSynchronize(c->st) == cudaSuccess ? IMEX_OK : IMEX_ECUDA;
}

imex_status imex_batch_get_time(const imex_batch* b, int i, double* t) {
  if (!b || !t || i < 0 || i >= (int)b->grp.size()) return IMEX_EINVAL;
  *t = b->groups[b->grp[i]]->inst[b->loc[i]].t;
  return IMEX_OK;
}

imex_status imex_batch_get_stats(const imex_batch* b, imex_stats* out) {
  if (!b || !out) return IMEX_EINVAL;
  *out = b->stats;
  return IMEX_OK;
}

imex_status imex_batch_group_info(const imex_batch* b, int q, int* ninst, int* P, long long* nvel, imex_stats* st,
                                  double* last_ms) {
  if (!b || q < 0 || q >= (int)b->groups.size()) return IMEX_EINVAL;
  const imex_ctx* c = b->groups[q];
  if (ninst) *ninst = (int)c->inst.size();
  if (P) *P = c->Nv - 1;
  if (nvel) *nvel = (long long)c->nv;
  if (st) *st = c->stats;
  if (last_ms) *last_ms = q < (int)b->group_ms.size() ? b->group_ms[q] : 0.0;
  return IMEX_OK;
}


// ---- serving: continuous batching ------------------------------------------------------
struct imex_server {
  imex_server_desc desc{};
  double budget = 0.0;
  struct Req {
    imex_request r{};
    int state = IMEX_REQ_QUEUED;
    int steps_done = 0;
    double t = 0.0;
    double footprint = 0.0;
    long long dof = 0;
    int group = -1;
    std::vector<double> result;
    std::string err;
  };
  std::vector<Req> reqs;
  std::deque<long long> queue;
  struct Group {
    imex_ctx* c = nullptr;
    std::vector<long long> members;   // request ids, in the group's instance order
    std::vector<long long> joining;   // admitted, not yet in the layout
    bool leaving = false;             // a member finished or failed: regroup before the next step
  };
  std::vector<Group> groups;
  double active_fp = 0.0, max_fp = 0.0;
  std::vector<double> tick_ms;
  double dof_stages = 0.0, busy_s = 0.0;
  long long completed = 0, failed = 0;
  std::string err;
};

namespace {

// settings that must agree within a group (the rest is per instance)
bool same_server_group(const imex_request& a, const imex_request& b) {
  if (a.dim != b.dim || a.P != b.P || a.nu_kind != b.nu_kind || a.bc_kind != b.bc_kind || a.f_kind != b.f_kind)
    return false;
  for (int k = 0; k < a.dim; ++k)
    if ((a.periodic[k] != 0) != (b.periodic[k] != 0)) return false;
  return true;
}

InstGeom req_geom(const imex_request& r) {
  InstGeom I{};
  I.ne = 1;
  for (int k = 0; k < 3; ++k) {
    const int n = k < r.dim ? r.nelem[k] : 1;
    I.n[k] = n;
    I.lo[k] = k < r.dim ? r.lo[k] : 0.0;
    I.h[k] = k < r.dim ? (r.hi[k] - r.lo[k]) / n : 1.0;
    I.hf[k] = (float)I.h[k];
    I.ne *= n;
  }
  I.nu0 = r.nu_params[0];
  I.nu0f = (float)r.nu_params[0];
  I.dt = r.dt;
  I.dtf = (float)r.dt;
  I.t = r.t0;
  std::memcpy(I.nu_p, r.nu_params, sizeof(I.nu_p));
  std::memcpy(I.bc_p, r.bc_params, sizeof(I.bc_p));
  std::memcpy(I.f_p, r.f_params, sizeof(I.f_p));
  return I;
}

imex_mesh_desc req_desc(const imex_server* sv, const imex_request& r) {
  imex_mesh_desc d{};
  d.dim = r.dim;
  d.P = r.P;
  for (int k = 0; k < 3; ++k) {
    d.nelem[k] = k < r.dim ? r.nelem[k] : 1;
    d.lo[k] = r.lo[k];
    d.hi[k] = r.hi[k];
    d.periodic[k] = k < r.dim ? r.periodic[k] : 1;
  }
  d.precision = sv->desc.precision;
  d.poisson = sv->desc.poisson;
  d.tol = sv->desc.tol > 0 ? sv->desc.tol : 1e-10;
  d.maxit = sv->desc.maxit > 0 ? sv->desc.maxit : 20000;
  d.vmax = sv->desc.vmax;
  return d;
}

// apply the pending joins and departures of a server group (growing it when needed)
imex_status server_regroup(imex_server* sv, imex_server::Group& G) {
  imex_ctx* c = G.c;
  std::vector<int> keep;
  std::vector<long long> kept_ids;
  for (size_t i = 0; i < G.members.size(); ++i) {
    const auto& R = sv->reqs[G.members[i]];
    if (R.state == IMEX_REQ_ACTIVE) {
      keep.push_back((int)i);
      kept_ids.push_back(G.members[i]);
    }
  }
  std::vector<JoinSpec> join;
  long long ne = 0;
  for (int i : keep) ne += c->inst[i].ne;
  for (long long id : G.joining) {
    const auto& R = sv->reqs[id];
    JoinSpec j{};
    j.g = req_geom(R.r);
    j.flow = R.r.flow;
    std::memcpy(j.flow_p, R.r.flow_params, sizeof(j.flow_p));
    j.t0 = R.r.t0;
    join.push_back(j);
    ne += j.g.ne;
  }
  const int ni = (int)(keep.size() + join.size());
  imex_ctx* dst = c;
  if (ni > 0 && (ne > c->ne_cap || ni > c->ninst_cap)) {
    // grow: a new group with twice the needed room takes the members over
    const imex_request& r0 = sv->reqs[kept_ids.empty() ? G.joining[0] : kept_ids[0]].r;
    TRY(create_group(req_desc(sv, r0), r0.nu_kind, r0.bc_kind, r0.f_kind, req_geom(r0), 2 * ne, 2 * ni, &dst));
  }
  const imex_status s = regroup(c, dst, keep, join);
  if (dst != c) {
    imex_destroy(c);
    G.c = dst;
  }
  if (s != IMEX_OK) return s;
  G.members = kept_ids;
  G.members.insert(G.members.end(), G.joining.begin(), G.joining.end());
  G.joining.clear();
  G.leaving = false;
  return IMEX_OK;
}

}  // namespace

imex_status imex_server_create(const imex_server_desc* desc, imex_server** out) {
  if (!desc || !out) return IMEX_EINVAL;
  if (desc->precision != IMEX_FP64 && desc->precision != IMEX_MIXED && desc->precision != IMEX_MIXED_FAST)
    return IMEX_EINVAL;
  imex_server* sv = new imex_server();
  sv->desc = *desc;
  sv->budget = desc->hbm_budget_bytes;
  if (!(sv->budget > 0)) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete sv;
      return IMEX_ECUDA;
    }
    sv->budget = 0.5 * (double)fr;
  }
  *out = sv;
  return IMEX_OK;
}

void imex_server_destroy(imex_server* sv) {
  if (!sv) return;
  for (auto& G : sv->groups) imex_destroy(G.c);
  delete sv;
}

const char* imex_server_last_error(const imex_server* sv) { return sv ? sv->err.c_str() : "null server"; }

imex_status imex_server_submit(imex_server* sv, const imex_request* r, long long* id) {
  if (!sv || !r || !id) return IMEX_EINVAL;
  if ((r->dim != 2 && r->dim != 3) || r->P < 2 || r->P > IMEX_MAXN - 1 || !(r->dt > 0) || r->nsteps < 1)
    return IMEX_EINVAL;
  bool bnd = false;
  for (int k = 0; k < r->dim; ++k) {
    if (r->nelem[k] < 1 || !(r->hi[k] > r->lo[k])) return IMEX_EINVAL;
    bnd = bnd || !r->periodic[k];
  }
  if (bnd && r->bc_kind == IMEX_FLOW_NONE) return IMEX_EINVAL;
  if (r->nu_kind == IMEX_NU_FIELD) return IMEX_EINVAL;
  imex_server::Req R;
  R.r = *r;
  R.t = r->t0;
  const InstGeom I = req_geom(*r);
  const long long nv = (long long)I.ne * ipow(r->P + 1, r->dim), np = (long long)I.ne * ipow(r->P, r->dim);
  R.footprint = footprint_bytes(r->dim, nv, np, 4);
  R.dof = r->dim * nv;
  *id = (long long)sv->reqs.size();
  sv->reqs.push_back(std::move(R));
  sv->queue.push_back(*id);
  return IMEX_OK;
}

imex_status imex_request_footprint(const imex_request* r, double* bytes) {
  if (!r || !bytes || (r->dim != 2 && r->dim != 3) || r->P < 2 || r->P > IMEX_MAXN - 1) return IMEX_EINVAL;
  for (int k = 0; k < r->dim; ++k)
    if (r->nelem[k] < 1) return IMEX_EINVAL;
  const InstGeom I = req_geom(*r);
  const long long nv = (long long)I.ne * ipow(r->P + 1, r->dim), np = (long long)I.ne * ipow(r->P, r->dim);
  *bytes = footprint_bytes(r->dim, nv, np, 4);
  return IMEX_OK;
}

imex_status imex_server_tick(imex_server* sv, int* active) {
  if (!sv) return IMEX_EINVAL;
  const auto t0 = std::chrono::steady_clock::now();
  // 1. admission in arrival order while the active footprint stays within the budget
  while (!sv->queue.empty()) {
    const long long id = sv->queue.front();
    auto& R = sv->reqs[id];
    if (sv->active_fp + R.footprint > sv->budget) {
      if (sv->active_fp > 0) break;                 // wait for room
      R.state = IMEX_REQ_FAILED;                    // would not fit even alone
      R.err = "request footprint above the HBM budget";
      sv->failed++;
      sv->queue.pop_front();
      continue;
    }
    sv->queue.pop_front();
    int g = -1;
    for (size_t q = 0; q < sv->groups.size() && g < 0; ++q) {
      const auto& G = sv->groups[q];
      const long long any = !G.members.empty() ? G.members[0] : G.joining[0];
      if (same_server_group(sv->reqs[any].r, R.r)) g = (int)q;
    }
    if (g < 0) {
      imex_ctx* c = nullptr;
      const InstGeom I = req_geom(R.r);
      const imex_status s = create_group(req_desc(sv, R.r), R.r.nu_kind, R.r.bc_kind, R.r.f_kind, I,
                                         2 * (long long)I.ne, 16, &c);
      if (s != IMEX_OK) {
        R.state = IMEX_REQ_FAILED;
        R.err = "group creation failed";
        sv->failed++;
        continue;
      }
      imex_server::Group G;
      G.c = c;
      sv->groups.push_back(G);
      g = (int)sv->groups.size() - 1;
    }
    sv->groups[g].joining.push_back(id);
    R.group = g;
    R.state = IMEX_REQ_ACTIVE;
    sv->active_fp += R.footprint;
    sv->max_fp = std::max(sv->max_fp, sv->active_fp);
  }
  // 2. layout changes, then drop empty groups
  for (auto& G : sv->groups)
    if (!G.joining.empty() || G.leaving) {
      const imex_status s = server_regroup(sv, G);
      if (s != IMEX_OK) {
        for (long long id : G.joining) {
          sv->reqs[id].state = IMEX_REQ_FAILED;
          sv->reqs[id].err = "regroup failed";
          sv->failed++;
          sv->active_fp -= sv->reqs[id].footprint;
        }
        G.joining.clear();
        sv->err = G.c ? G.c->err : "regroup failed";
      }
    }
  for (size_t q = 0; q < sv->groups.size();)
    if (sv->groups[q].members.empty() && sv->groups[q].joining.empty()) {
      imex_destroy(sv->groups[q].c);
      sv->groups.erase(sv->groups.begin() + q);
      for (auto& R : sv->reqs)
        if (R.state == IMEX_REQ_ACTIVE && R.group > (int)q) R.group--;
    } else {
      ++q;
    }
  // 3. one step of every active request, the groups concurrently
  std::vector<imex_status> st(sv->groups.size(), IMEX_OK);
  auto run = [&](size_t q) {
    imex_ctx* c = sv->groups[q].c;
    std::vector<double> dt;
    for (long long id : sv->groups[q].members) dt.push_back(sv->reqs[id].r.dt);
    imex_status s = set_group_dt(c, dt);
    if (s == IMEX_OK) s = group_step(c);
    if (s == IMEX_OK && cudaStreamSynchronize(c->st) != cudaSuccess) s = IMEX_ECUDA;
    st[q] = s;
  };
  if (sv->groups.size() == 1) {
    run(0);
  } else if (!sv->groups.empty()) {
    std::vector<std::thread> th;
    for (size_t q = 0; q < sv->groups.size(); ++q) th.emplace_back(run, q);
    for (auto& t : th) t.join();
  }
  // 4. bookkeeping: finished and failed requests leave at the next tick
  int nact = 0;
  for (size_t q = 0; q < sv->groups.size(); ++q) {
    auto& G = sv->groups[q];
    imex_ctx* c = G.c;
    for (size_t i = 0; i < G.members.size(); ++i) {
      auto& R = sv->reqs[G.members[i]];
      if (R.state != IMEX_REQ_ACTIVE) continue;
      if (st[q] != IMEX_OK) {
        R.state = IMEX_REQ_FAILED;
        R.err = c->err;
        sv->failed++;
        sv->active_fp -= R.footprint;
        G.leaving = true;
        continue;
      }
      R.steps_done++;
      R.t = c->inst[i].t;
      sv->dof_stages += (double)R.dof * (c->tab.s - 1);
      if (R.steps_done >= R.r.nsteps) {
        if (sv->desc.keep_results) {
          const InstGeom& I = c->inst[i];
          const size_t ndv = ipow(c->Nv, c->d), n = (size_t)I.ne * ndv;
          R.result.resize(c->d * n);
          for (int k = 0; k < c->d; ++k)
            cudaMemcpy(R.result.data() + k * n, c->v + k * c->nv + I.e0 * ndv, n * sizeof(double),
                       cudaMemcpyDeviceToHost);
        }
        R.state = IMEX_REQ_DONE;
        sv->completed++;
        sv->active_fp -= R.footprint;
        G.leaving = true;
      } else {
        nact++;
      }
    }
    if (st[q] != IMEX_OK) sv->err = "group " + std::to_string(q) + ": " + c->err;
  }
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (!sv->groups.empty()) {
    sv->tick_ms.push_back(ms);
    sv->busy_s += ms * 1e-3;
  }
  if (active) *active = nact;
  return IMEX_OK;
}

imex_status imex_server_poll(const imex_server* sv, long long id, int* state, int* steps_done, double* t) {
  if (!sv || id < 0 || id >= (long long)sv->reqs.size()) return IMEX_EINVAL;
  const auto& R = sv->reqs[id];
  if (state) *state = R.state;
  if (steps_done) *steps_done = R.steps_done;
  if (t) *t = R.t;
  return IMEX_OK;
}

imex_status imex_server_result(imex_server* sv, long long id, double* velocity) {
  if (!sv || !velocity || id < 0 || id >= (long long)sv->reqs.size()) return IMEX_EINVAL;
  auto& R = sv->reqs[id];
  if (R.state != IMEX_REQ_DONE || R.result.empty()) return IMEX_EINVAL;
  std::memcpy(velocity, R.result.data(), R.result.size() * sizeof(double));
  std::vector<double>().swap(R.result);
  return IMEX_OK;
}

imex_status imex_server_get_stats(const imex_server* sv, imex_server_stats* out) {
  if (!sv || !out) return IMEX_EINVAL;
  imex_server_stats s{};
  s.submitted = (long long)sv->reqs.size();
  s.completed = sv->completed;
  s.failed = sv->failed;
  s.queued = (long long)sv->queue.size();
  for (const auto& R : sv->reqs) s.active += R.state == IMEX_REQ_ACTIVE ? 1 : 0;
  s.ticks = (long long)sv->tick_ms.size();
  if (!sv->tick_ms.empty()) {
    std::vector<double> t = sv->tick_ms;
    std::sort(t.begin(), t.end());
    s.p50_tick_ms = t[t.size() / 2];
    s.p99_tick_ms = t[std::min(t.size() - 1, (size_t)(0.99 * (double)t.size()))];
    double sum = 0.0;
    for (double x : t) sum += x;
    s.mean_tick_ms = sum / (double)t.size();
  }
  s.dof_stages = sv->dof_stages;
  s.busy_s = sv->busy_s;
  s.footprint_bytes = sv->active_fp;
  s.max_footprint_bytes = sv->max_fp;
  s.budget_bytes = sv->budget;
  s.groups = (int)sv->groups.size();
  *out = s;
  return IMEX_OK;
}

}  // extern "C"

namespace imex {
// FP32 -> FP64 copy (the FP64 refinement of the mixed-precision solves)
__global__ void f2d_kernel(const float* in, double* out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}
}  // namespace imex
void f2d(const float* in, double* out, size_t n, cudaStream_t st) {
  IMEX_COUNTED(imex::f2d_kernel<<<(unsigned)std::min<size_t>((n + 255) / 256, 1216), 256, 0, st>>>(in, out, n));
}
