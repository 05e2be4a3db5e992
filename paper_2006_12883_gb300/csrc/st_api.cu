// C ABI of the space-time multigrid / SDC library: handle, level hierarchy,
// workspace, the V-cycle / SDC / adjoint drivers and CUDA-graph replay.
// See include/st.h for the contract of every entry point.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "st_kernels.cuh"
#include "st_setup.h"

using namespace st;

namespace st {
thread_local int tl_pdl = 1;
thread_local int tl_tma = 1;
}

namespace {

thread_local char g_err[512] = "";

void set_err(cudaError_t e, const char* what) {
  snprintf(g_err, sizeof(g_err), "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define CK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) {                    \
      set_err(e_, #x);                          \
      return ST_ERR_CUDA;                       \
    }                                           \
  } while (0)
#define CKL() CK(cudaGetLastError())
#define TRY(x)                \
  do {                        \
    int s_ = (x);             \
    if (s_ != ST_OK) return s_; \
  } while (0)

struct InnerLev {
  GridP g;
  void* y = nullptr;
  void* z = nullptr;
  void* t = nullptr;
  void* cbar = nullptr;
};

// The collocation data of one node count: Q and its eigenbasis, the real
// forward / back transforms of the Q-diagonalised slab solve (forward and
// adjoint), the shift groups, and the slab-bisection transfers.
struct NodeSet {
  int M = 0;
  Colloc col;
  int ngroups = 0;
  int gplane[MAXM], gcplx[MAXM];
  std::complex<double> glam[MAXM];
  double Ff[MAXM][MAXM], Bf[MAXM][MAXM], Fa[MAXM][MAXM], Ba[MAXM][MAXM];
  double RtT[MAXM][2 * MAXM];  // P_t^T (adjoint restriction)
  double PtT[2 * MAXM][MAXM];  // R_t^T (adjoint prolongation)
};

struct Level {
  GridP g;
  int Nt = 0;
  int M = 1;                    // collocation nodes per slab on this level
  const NodeSet* ns = nullptr;  // their collocation data
  double dt = 0, mu = 0, omega = 1;
  int next = 0;  // 0 coarsest, 1 space, 2 slabs, 3 space and nodes (M -> M-1)
  // next == 3: node-set transfers to the coarser level (P: M x Mc, R: Mc x M)
  // and their transposes (adjoint), and a buffer of M planes on the coarse grid
  double Pn[MAXM][MAXM], Rn[MAXM][MAXM], PnT[MAXM][MAXM], RnT[MAXM][MAXM];
  void* tmp = nullptr;
  int bottom_sweeps = 2;
  // depth of the inner multigrid the block-Jacobi smoother uses, and the
  // Jacobi sweeps at its bottom
  int smooth_depth = 1;
  int smooth_sweeps = 2;
  void* e = nullptr;
  void* r = nullptr;
  void* cbar = nullptr;
  std::vector<InnerLev> in;
  // a small level whose forward smoothing steps run as one launch each (one
  // block per slab): the post-smoothing step writes its e into e2, which the
  // finer level's prolongation then reads
  bool fused = false;
  void* e2 = nullptr;
};

struct Alloc {
  void* p;
  size_t bytes;
};

// One PFASST level above the finest (FP64 state; the grid and the inner
// spatial multigrid are those of the space-bisected cycle level of the same
// index).
struct PfLevel {
  int M = 1;
  double* U = nullptr;     // iterate [Nt][M][Ns]
  double* Ubar = nullptr;  // the restricted iterate before the coarse sweeps
  double* tau = nullptr;   // FAS correction
  double* W = nullptr;     // work: dt Q F(U) + tau
  double* tmp = nullptr;   // transfers: the finer level's node count on this grid
  double* u0 = nullptr;    // restricted initial value
  double Rv[MAXM][MAXM];   // node values, finer -> this (M x M_finer)
  double Pv[MAXM][MAXM];   // node values, this -> finer (M_finer x M)
};

template <typename T>
StencilC<T> stencil_of(const GridP& g, double nu) {
  StencilC<T> c;
  c.cx = (T)(nu * g.ih2[0]);
  c.cy = (T)(nu * g.ih2[1]);
  c.cz = (T)(nu * g.ih2[2]);
  c.k2 = (T)(-2.0 * nu * (g.ih2[0] + g.ih2[1] + g.ih2[2]));
  return c;
}

bool can_coarsen_axis(int bc, int n) {
  if (bc == ST_BC_DIRICHLET) return n >= 3 && (n & 1);
  if (bc == ST_BC_PERIODIC) return n >= 2 && !(n & 1);
  return n >= 3 && !((n - 1) & 1);
}

int coarse_axis(int bc, int n) {
  if (bc == ST_BC_DIRICHLET) return (n - 1) / 2;
  if (bc == ST_BC_PERIODIC) return n / 2;
  return (n - 1) / 2 + 1;
}

bool can_coarsen(int d, const GridP& g) {
  const int nn[3] = {g.n0, g.n1, g.n2};
  for (int a = 0; a < d; ++a)
    if (!can_coarsen_axis(g.bc, nn[a])) return false;
  return true;
}

GridP coarsen(int d, const GridP& g, double X) {
  int n[3] = {g.n0, g.n1, g.n2};
  for (int a = 0; a < d; ++a) n[a] = coarse_axis(g.bc, n[a]);
  return make_grid(d, n, g.bc, X);
}

const int kInnerCoarseMax = 8;     // stop inner coarsening at <= this many points
const int kInnerCoarseLimit = 256; // largest grid the single-block kernel takes
const int kCoarseKMax = 96;        // largest dense slab block M*Nc

struct PlanLevel {
  GridP g;
  int Nt;
  int M;
  double dt, mu, omega;
  int next;
  std::vector<GridP> inner;
  int bottom_sweeps;  // Jacobi sweeps on the bottom inner grid when it does not fit one block
};

// Largest |shift| per unit dt of the slab systems: max |lambda(Q)| and the
// SDC diagonal entries.
double max_shift(int M) {
  Colloc c;
  if (colloc_setup(M, &c) != 0) return 1.0;
  double m = 0;
  for (int q = 0; q < M; ++q) {
    m = std::max(m, std::abs(c.lam[q]));
    m = std::max(m, std::max(c.QI_ie[q][q], c.QI_lu[q][q]));
  }
  return m;
}

// max |lambda(Q)|.
double max_eig(int M) {
  Colloc c;
  if (colloc_setup(M, &c) != 0) return 1.0;
  double m = 0;
  for (int q = 0; q < M; ++q) m = std::max(m, std::abs(c.lam[q]));
  return m;
}

// Diffusion number of the shifted slab operator on grid g: |s| nu 2 sum 1/h^2.
double stiffness(const GridP& g, double nu, double dt, double lam) {
  return lam * dt * nu * 2.0 * (g.ih2[0] + g.ih2[1] + g.ih2[2]);
}

const double kSigmaStop = 0.25;
const double kMinStep = 1.0 / (1 << 20);  // smallest line-search step before DIVERGED  // below this Jacobi alone solves the slab systems

double default_omega(const st_solver_opts& o, double mu) {
  if (o.omega > 0) return o.omega;
  if (mu >= 16.0) return 1.0;
  if (mu >= o.mu_crit) return 0.8;
  return 0.5;
}

int validate(const st_problem* p, const st_solver_opts* o) {
  if (!p) return ST_ERR_INVALID_ARG;
  if (p->d < 1 || p->d > 3) return ST_ERR_INVALID_ARG;
  for (int a = 0; a < p->d; ++a) {
    if (p->n[a] < 1) return ST_ERR_INVALID_ARG;
    if (p->bc == ST_BC_NEUMANN && p->n[a] < 2) return ST_ERR_INVALID_ARG;
  }
  if (p->bc < 0 || p->bc > 2) return ST_ERR_INVALID_ARG;
  if (p->reaction < 0 || p->reaction > 2) return ST_ERR_INVALID_ARG;
  if (!(p->X > 0) || !(p->T > 0) || !(p->nu > 0) || !std::isfinite(p->rho)) return ST_ERR_INVALID_ARG;
  if (p->Nt < 1 || p->M < 1 || p->M > ST_MAX_M) return ST_ERR_INVALID_ARG;
  {
    long long ns = 1;
    for (int a = 0; a < p->d; ++a) ns *= p->n[a];
    // kernels index (slab, point) pairs with 32-bit integers
    if (ns * (long long)p->Nt >= 0x7fffffffLL) return ST_ERR_UNSUPPORTED;
  }
  if (o) {
    if (o->precision != ST_PREC_FP64 && o->precision != ST_PREC_FP32_REFINE) return ST_ERR_INVALID_ARG;
    if (o->coarsening != ST_COARSEN_SPACE && o->coarsening != ST_COARSEN_AUTO_MU &&
        o->coarsening != ST_COARSEN_SPACE_NODES && o->coarsening != ST_COARSEN_SPACE_TIME)
      return ST_ERR_INVALID_ARG;
    if (o->nu1 < 0 || o->nu2 < 0 || o->nu1 + o->nu2 < 1 || o->nu1 > 8 || o->nu2 > 8) return ST_ERR_INVALID_ARG;
    if (o->inner_cycles < 1 || o->inner_smooth < 1 || o->inner_coarse_iters < 1) return ST_ERR_INVALID_ARG;
    if (o->smooth_inner_levels < 0 || o->smooth_sweeps < 2) return ST_ERR_INVALID_ARG;
    if (o->krylov < 0 || o->krylov > 30 || !(o->krylov_rtol > 0.0)) return ST_ERR_INVALID_ARG;
    if (o->krylov_fallback < 0 || o->krylov_fallback > 30) return ST_ERR_INVALID_ARG;
    if (o->pfasst_levels < 1 || o->pfasst_coarse_M < 1 || o->pfasst_sweeps < 1) return ST_ERR_INVALID_ARG;
    if (o->sdc_inner_cycles < 1 || o->max_iters < 0 || !(o->tol >= 0)) return ST_ERR_INVALID_ARG;
    if (o->max_levels < 1 || o->coarse_max_points < 1 || o->coarse_max_slabs < 1) return ST_ERR_INVALID_ARG;
    if (o->sdc_qdelta != ST_SDC_IE && o->sdc_qdelta != ST_SDC_LU) return ST_ERR_INVALID_ARG;
  }
  return ST_OK;
}

int plan_levels(const st_problem* p, const st_solver_opts& o, std::vector<PlanLevel>& out) {
  out.clear();
  const int d = p->d;
  PlanLevel L0;
  L0.g = make_grid(d, p->n, p->bc, p->X);
  L0.Nt = p->Nt;
  L0.M = p->M;
  L0.dt = p->T / p->Nt;
  out.push_back(L0);
  const int maxl = std::min(o.max_levels, ST_MAX_LEVELS);
  const double lam_q = max_eig(p->M);
  while ((int)out.size() < maxl) {
    PlanLevel& cur = out.back();
    const bool cs = can_coarsen(d, cur.g);
    // Slab bisection doubles dt; with a growing reaction (R' up to |rho|) the
    // coarse slab systems stay well conditioned only while 2 dt |rho| max|lambda(Q)|
    // stays below 1/2.
    const bool ct = (cur.Nt % 2 == 0) && cur.Nt >= 2 &&
                    (p->reaction == ST_REACTION_NONE || 2.0 * cur.dt * std::fabs(p->rho) * lam_q <= 0.5);
    const double mu = p->nu * cur.dt * cur.g.ih2[0];
    int kind = 0;
    if (o.coarsening == ST_COARSEN_SPACE) {
      if (cs && cur.g.Ns > o.coarse_max_points) kind = 1;
    } else if (o.coarsening == ST_COARSEN_SPACE_NODES) {
      if (cs && cur.g.Ns > o.coarse_max_points) kind = cur.M > 1 ? 3 : 1;
    } else if (o.coarsening == ST_COARSEN_SPACE_TIME) {
      const bool ss = cs && cur.g.Ns > o.coarse_max_points;
      const bool tt = ct && cur.Nt > o.coarse_max_slabs;
      kind = (ss && tt) ? 4 : (ss ? 1 : (tt ? 2 : 0));
    } else {
      const bool small_s = cur.g.Ns <= o.coarse_max_points;
      const bool small_t = cur.Nt <= o.coarse_max_slabs;
      if (small_s && (small_t || !ct)) kind = 0;
      else if (cs && !small_s && mu >= o.mu_crit) kind = 1;
      else if (ct && !small_t) kind = 2;
      else if (cs && !small_s) kind = 1;
    }
    if (kind == 0) break;
    PlanLevel nx;
    nx.Nt = cur.Nt;
    nx.dt = cur.dt;
    nx.M = kind == 3 ? cur.M - 1 : cur.M;
    if (kind == 4) {
      nx.g = coarsen(d, cur.g, p->X);
      nx.Nt = cur.Nt / 2;
      nx.dt = cur.dt * 2;
    } else if (kind == 1 || kind == 3) {
      nx.g = coarsen(d, cur.g, p->X);
    } else {
      nx.g = cur.g;
      nx.Nt = cur.Nt / 2;
      nx.dt = cur.dt * 2;
    }
    cur.next = kind;
    out.push_back(nx);
  }
  out.back().next = 0;
  const double wj = d == 1 ? 2.0 / 3.0 : (d == 2 ? 0.8 : 6.0 / 7.0);
  for (auto& L : out) {
    const double lmax = max_shift(L.M);
    L.mu = p->nu * L.dt * L.g.ih2[0];
    L.omega = default_omega(o, L.mu);
    L.inner.clear();
    L.inner.push_back(L.g);
    while (L.inner.back().Ns > kInnerCoarseMax && can_coarsen(d, L.inner.back()) &&
           stiffness(L.inner.back(), p->nu, L.dt, lmax) > kSigmaStop)
      L.inner.push_back(coarsen(d, L.inner.back(), p->X));
    // sweeps for a 0.05 reduction of the smoothest mode, factor 1 - wj/(1+sigma)
    const double sig = stiffness(L.inner.back(), p->nu, L.dt, lmax);
    const double rho = std::max(1e-3, 1.0 - wj / (1.0 + sig));
    L.bottom_sweeps = std::max(2, std::min(o.inner_coarse_iters, (int)std::ceil(std::log(0.05) / std::log(rho))));
  }
  if (out.back().g.Ns * out.back().M > kCoarseKMax) return ST_ERR_UNSUPPORTED;
  return ST_OK;
}

// Depth of the inner multigrid the slab solves of level l use (the smoother
// policy): capped to o.smooth_inner_levels while a coarser level of the
// hierarchy is coarser in space and the next level keeps the node count.
int smooth_depth_of(const std::vector<PlanLevel>& pl, size_t l, const st_solver_opts& o) {
  bool space_below = false;
  for (size_t q = l; q < pl.size(); ++q)
    space_below = space_below || pl[q].next == 1 || pl[q].next == 3 || pl[q].next == 4;
  const int full = (int)pl[l].inner.size();
  const int cap = o.smooth_inner_levels;
  return (cap > 0 && cap < full && space_below && pl[l].next != 3) ? cap : full;
}

// Whether level l's forward smoothing steps run as one launch each (one
// block per slab, planes in shared memory; see k_slab_smooth): a level
// between the finest and the coarsest whose slab solves are plain Jacobi
// sweeps from the zero-start iterate, V(1,1), and whose grid is small enough
// (kFusedSmoothMaxNs) that the separate launches are latency bound; on larger
// grids N_t blocks are too few to occupy the GPU.
const long long kFusedSmoothMaxNs = 1024;
bool fused_smoothing(const std::vector<PlanLevel>& pl, size_t l, const st_solver_opts& o, size_t esz) {
  const bool multi = !(pl[l].inner.size() == 1 && pl[l].inner[0].Ns <= kInnerCoarseLimit);
  return l >= 1 && l + 1 < pl.size() && smooth_depth_of(pl, l, o) == 1 && multi && o.nu1 == 1 && o.nu2 == 1 &&
         o.inner_cycles == 1 && pl[l].g.Ns <= kFusedSmoothMaxNs &&
         (size_t)(4 * pl[l].M + 1) * (size_t)pl[l].g.Ns * esz <= 220 * 1024;
}

size_t round_up(size_t b) { return (b + 255) / 256 * 256; }

// pinned host doubles: [0, 8) scalars read back after reductions, [16, 80)
// Krylov dot products
const int kHostScalars = 80;
const int kHostKrylov = 16;
const int kHostFlag = 8;          // an int: the count of expired TMA waits, read synchronously
const int kHostFlagDeferred = 9;  // an int: the same count, copied behind an asynchronous cycle

}  // namespace

// ---------------------------------------------------------------------------
struct st_handle {
  st_problem p;
  st_solver_opts o;
  st_runtime rt;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  int D = 1, fp64 = 0;
  size_t esz = 4;
  // collocation data per node count (index M); the finest level's is `fine`
  NodeSet ns[MAXM + 1];
  const NodeSet* fine = nullptr;
  std::vector<Level> L;
  // coarsest level
  int Nc = 0, K = 0;
  double* Lc = nullptr;
  void *Ainv = nullptr, *Wf = nullptr, *Wt = nullptr, *Wfrow = nullptr, *Wtrow = nullptr, *cin = nullptr;
  bool coarse_ready = false;
  bool linearized = false;
  // fine-level FP64 data
  std::vector<double> u0_host;
  double* u0 = nullptr;
  double* partial = nullptr;
  double* partial2 = nullptr;
  long long npartial = 0;
  double* scal = nullptr;   // device scalars
  double* hscal = nullptr;  // pinned host scalars
  double* Ustage = nullptr;
  double* Rstage = nullptr;  // FP64 residual staging for host output on an FP32 handle
  double* lam = nullptr;
  void* cnode = nullptr;  // R'(U) per node (exact finest-level Jacobian), layout of U
  // Krylov-accelerated Newton step: bases V (m+1 vectors) and Z (m vectors)
  void* kV = nullptr;
  void* kZ = nullptr;
  double* kpart = nullptr;  // dot-product partial sums
  double* kdots = nullptr;  // 64 device doubles
  int kdim = 0;             // Krylov steps the bases hold
  double* plane = nullptr;  // staging for one plane (gT / target / du0)
  double* plane2 = nullptr;
  std::vector<Alloc> allocs;
  // graphs: 0 forward cycle, 1 adjoint cycle, 2 linearisation, 3 linearisation + cycle, 4 PFASST iteration,
  // 5 and 6: 0 and 3 after a fine residual that did the first smoothing step
  // 7 and 8: 5 and 6 whose last level-0 smoothing step also updates U
  static constexpr int kGraphs = 9;
  cudaGraphExec_t gexec[kGraphs] = {};
  size_t gnodes[kGraphs] = {};
  // second capture stream and events of the linearise + cycle graph: the
  // cbar chain and the coarse setup run beside the cycle's finest levels
  cudaStream_t cap2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_lvl[ST_MAX_LEVELS + 1] = {};
  bool split_lin = false;  // set while that graph's cycle is enqueued
  // set while a forward cycle is enqueued whose first level-0 smoothing
  // starts from the y and z the fine residual wrote (SmoothStart)
  bool start_ready = false;
  // bit l (l >= 1): the kernel that restricted onto level l also did the
  // first step of its first smoothing (set and used while a cycle is enqueued)
  unsigned start_mask = 0;
  // the update U += e fused into the cycle's last level-0 smoothing step:
  // device slot holding U's address, set before each such cycle; set while
  // such a cycle is enqueued / its last level-0 smoothing step is; set by
  // the step that did the update; per graph, whether its capture did
  double** Uslot = nullptr;
  bool upd_capture = false, upd_target = false, upd_applied = false;
  bool gupd[kGraphs] = {};
  bool last_update_in_cycle = false;  // for st_stats
  int nt_override = 0;     // > 0: inner solves act on this many slabs from the first
  int* tma_err = nullptr;   // device count of expired TMA waits (this device's copy)
  int tma_seen = 0;         // the count this handle has reported
  cudaEvent_t ev_norm = nullptr;  // the residual norm of an asynchronous st_vcycle is on the host
  std::vector<PfLevel> pf;  // PFASST levels 1.. (allocated at first use)
  double* pfW0 = nullptr;   // PFASST work on the finest level
  double* pfU = nullptr;    // PFASST: the finest iterate (fixed address for the iteration graph)
  long long D_total = 0;
  int chunk = 1;
};

namespace {

// Launch mode of the calling thread for the duration of one API call.
struct PdlScope {
  int saved, saved_tma;
  explicit PdlScope(const st_handle* h) : saved(tl_pdl), saved_tma(tl_tma) {
    if (h) {
      tl_pdl = h->o.use_pdl ? 1 : 0;
      tl_tma = h->o.use_tma ? 1 : 0;
    }
  }
  ~PdlScope() {
    tl_pdl = saved;
    tl_tma = saved_tma;
  }
};

void* dev_alloc(st_handle* h, size_t bytes) {
  bytes = round_up(std::max<size_t>(bytes, 256));
  void* p = nullptr;
  if (h->rt.alloc) {
    p = h->rt.alloc(bytes, (void*)h->stream, h->rt.ctx);
  } else {
    if (cudaMallocAsync(&p, bytes, h->stream) != cudaSuccess) p = nullptr;
  }
  if (p) h->allocs.push_back({p, bytes});
  return p;
}

int alloc_into(st_handle* h, void** dst, size_t bytes) {
  *dst = dev_alloc(h, bytes);
  if (!*dst) {
    cudaGetLastError();
    return ST_ERR_OOM;
  }
  return ST_OK;
}

template <typename P>
int alloc_typed(st_handle* h, P** dst, size_t bytes) {
  void* v = nullptr;
  int s = alloc_into(h, &v, bytes);
  *dst = (P*)v;
  return s;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void build_nodeset(NodeSet& s, int M) {
  s.M = M;
  const Colloc& c = s.col;
  // groups
  s.ngroups = 0;
  for (int q = 0; q < M;) {
    s.gplane[s.ngroups] = q;
    s.glam[s.ngroups] = c.lam[q];
    if (c.lam[q].imag() == 0.0) {
      s.gcplx[s.ngroups] = 0;
      ++q;
    } else {
      s.gcplx[s.ngroups] = 1;
      q += 2;
    }
    ++s.ngroups;
  }
  // forward (Q = V L V^-1): y = Vinv res, e += Re(V z);
  // adjoint (Q^T = W L W^-1 with W = V^{-T}, W^{-1} = V^T)
  for (int a = 0; a < MAXM; ++a)
    for (int b = 0; b < MAXM; ++b) s.Ff[a][b] = s.Bf[a][b] = s.Fa[a][b] = s.Ba[a][b] = 0;
  for (int gq = 0; gq < s.ngroups; ++gq) {
    const int p = s.gplane[gq];
    for (int j = 0; j < M; ++j) {
      const std::complex<double> fi = c.Vinv[p][j];   // forward row p of V^-1
      const std::complex<double> ai = c.V[j][p];      // adjoint row p of V^T
      const std::complex<double> fb = c.V[j][p];      // forward back-transform
      const std::complex<double> ab = c.Vinv[p][j];   // adjoint back: (V^{-T})[j][p] = Vinv[p][j]
      if (!s.gcplx[gq]) {
        s.Ff[p][j] = fi.real();
        s.Fa[p][j] = ai.real();
        s.Bf[j][p] = fb.real();
        s.Ba[j][p] = ab.real();
      } else {
        s.Ff[p][j] = fi.real();
        s.Ff[p + 1][j] = fi.imag();
        s.Fa[p][j] = ai.real();
        s.Fa[p + 1][j] = ai.imag();
        s.Bf[j][p] = 2 * fb.real();
        s.Bf[j][p + 1] = -2 * fb.imag();
        s.Ba[j][p] = 2 * ab.real();
        s.Ba[j][p + 1] = -2 * ab.imag();
      }
    }
  }
  for (int m = 0; m < MAXM; ++m)
    for (int kk = 0; kk < 2 * MAXM; ++kk) {
      s.RtT[m][kk] = (m < M && kk < 2 * M) ? c.Pt[kk][m] : 0.0;
      s.PtT[kk][m] = (m < M && kk < 2 * M) ? c.Rt[m][kk] : 0.0;
    }
}

template <typename T>
Shifts<T> level_shifts(const NodeSet& h, double dt) {
  Shifts<T> s;
  for (int p = 0; p < MAXM; ++p) {
    s.kind[p] = SH_NONE;
    s.sr[p] = s.si[p] = (T)0;
  }
  for (int q = 0; q < h.ngroups; ++q) {
    const int p = h.gplane[q];
    s.kind[p] = h.gcplx[q] ? SH_RE : SH_REAL;
    if (h.gcplx[q]) s.kind[p + 1] = SH_IM;
    s.sr[p] = (T)(dt * h.glam[q].real());
    s.si[p] = (T)(dt * h.glam[q].imag());
  }
  return s;
}

template <typename T>
Shifts<T> real_shift(T s0) {
  Shifts<T> s;
  for (int p = 0; p < MAXM; ++p) {
    s.kind[p] = SH_NONE;
    s.sr[p] = s.si[p] = (T)0;
  }
  s.kind[0] = SH_REAL;
  s.sr[0] = s0;
  return s;
}

double jacobi_weight(int d) { return d == 1 ? 2.0 / 3.0 : (d == 2 ? 0.8 : 6.0 / 7.0); }

// ---------------------------------------------------------------------------
// Inner spatial multigrid on the shifted slab systems of level l.
// ---------------------------------------------------------------------------
template <typename T>
InnerParams<T> inner_params(st_handle* h, Level& Lv, int k, int P, const Shifts<T>& sh, bool use_cbar) {
  InnerParams<T> ip;
  InnerLev& I = Lv.in[k];
  ip.g = I.g;
  ip.gc = (k + 1 < (int)Lv.in.size()) ? Lv.in[k + 1].g : I.g;
  ip.Nt = h->nt_override > 0 ? h->nt_override : Lv.Nt;
  ip.P = P;
  ip.sh = sh;
  ip.sc = stencil_of<T>(I.g, h->p.nu);
  ip.k2c = stencil_of<T>(ip.gc, h->p.nu).k2;
  ip.omega = (T)jacobi_weight(h->D);
  ip.fuse_bt = 0;
  ip.e_zero = 0;
  ip.omega_bt = (T)0;
  ip.e = nullptr;
  ip.Uslot = nullptr;
  ip.write_e = 1;
  for (int a2 = 0; a2 < MAXM; ++a2)
    for (int b = 0; b < MAXM; ++b) ip.B[a2][b] = (T)0;
  ip.cbar = use_cbar ? (const T*)I.cbar : nullptr;
  ip.cbarc = (use_cbar && k + 1 < (int)Lv.in.size()) ? (const T*)Lv.in[k + 1].cbar : nullptr;
  ip.y = (const T*)I.y;
  ip.z = (const T*)I.z;
  ip.zout = (T*)I.t;
  ip.res = (const T*)I.t;
  ip.yc = (k + 1 < (int)Lv.in.size()) ? (T*)Lv.in[k + 1].y : nullptr;
  ip.zc = (k + 1 < (int)Lv.in.size()) ? (T*)Lv.in[k + 1].z : nullptr;
  ip.iters = h->o.inner_coarse_iters;
  return ip;
}

// Fused epilogue of the last sweep at inner level 0: e = (e_zero ? 0 : e) + omega B z.
template <typename T>
struct BtFuse {
  bool on = false;
  int e_zero = 0;
  T omega = 0;
  T B[MAXM][MAXM];
  T* e = nullptr;
  // the two-sweep kernel also adds e' to U (*Uslot) and leaves e unwritten
  double* const* Uslot = nullptr;
};

template <typename T>
void apply_fuse(InnerParams<T>& ip, const BtFuse<T>& f) {
  ip.fuse_bt = 1;
  ip.e_zero = f.e_zero;
  ip.omega_bt = f.omega;
  ip.e = f.e;
  ip.Uslot = f.Uslot;
  ip.write_e = f.Uslot ? 0 : 1;
  for (int a = 0; a < MAXM; ++a)
    for (int b = 0; b < MAXM; ++b) ip.B[a][b] = f.B[a][b];
}

template <typename T>
InnerParams<T> inner_params_fused(st_handle* h, Level& Lv, int k, int P, const Shifts<T>& sh, bool use_cbar,
                                  const BtFuse<T>& f) {
  InnerParams<T> ip = inner_params<T>(h, Lv, k, P, sh, use_cbar);
  apply_fuse(ip, f);
  return ip;
}

template <typename T>
int inner_vcycle(st_handle* h, Level& Lv, int k, int depth, int sweeps, int P, const Shifts<T>& sh, bool use_cbar,
                 bool presmoothed, const BtFuse<T>* fuse, cudaStream_t st) {
  InnerLev& I = Lv.in[k];
  const int last = depth - 1;
  if (k == last) {
    if (k == (int)Lv.in.size() - 1 && I.g.Ns <= kInnerCoarseLimit) {
      // one block per slab, all sweeps in shared memory
      InnerParams<T> ip = inner_params<T>(h, Lv, k, P, sh, use_cbar);
      ip.zout = (T*)I.z;
      if (fuse) apply_fuse(ip, *fuse);
      launch_inner_coarse<T>(h->D, ip, st);
      CKL();
      return ST_OK;
    }
    // non-stiff bottom grid: Jacobi sweeps continuing from z (which holds
    // the zero-start iterate when `presmoothed`)
    const int todo = presmoothed ? sweeps - 1 : sweeps;
    if constexpr (std::is_same<T, float>::value) {
      // the last two sweeps as one kernel, the middle iterate kept on chip
      if (fuse && todo >= 2 && h->o.fuse_sweeps) {
        for (int it = 0; it < todo - 2; ++it) {
          InnerParams<T> ip = inner_params<T>(h, Lv, k, P, sh, use_cbar);
          launch_inner_jacobi<T>(h->D, 0, ip, st);
          CKL();
          std::swap(I.z, I.t);
        }
        InnerParams<T> ip = inner_params<T>(h, Lv, k, P, sh, use_cbar);
        apply_fuse(ip, *fuse);
        if (launch_sweep2(h->D, ip, st)) {
          CKL();
          if (ip.Uslot) h->upd_applied = true;
          return ST_OK;
        }
        // not applicable here: the two sweeps run as separate launches
        InnerParams<T> ip1 = inner_params<T>(h, Lv, k, P, sh, use_cbar);
        launch_inner_jacobi<T>(h->D, 0, ip1, st);
        CKL();
        std::swap(I.z, I.t);
        launch_inner_jacobi<T>(h->D, 0, inner_params_fused<T>(h, Lv, k, P, sh, use_cbar, *fuse), st);
        CKL();
        return ST_OK;
      }
    }
    for (int it = 0; it < todo; ++it) {
      InnerParams<T> ip = inner_params<T>(h, Lv, k, P, sh, use_cbar);
      if (fuse && it == todo - 1) {
        apply_fuse(ip, *fuse);
        launch_inner_jacobi<T>(h->D, 0, ip, st);
        CKL();
      } else {
        launch_inner_jacobi<T>(h->D, 0, ip, st);
        CKL();
        std::swap(I.z, I.t);
      }
    }
    return ST_OK;
  }
  const int ns = h->o.inner_smooth;
  for (int it = 0; it < ns; ++it) {
    if (it == 0 && presmoothed) continue;
    InnerParams<T> ip = inner_params<T>(h, Lv, k, P, sh, use_cbar);
    launch_inner_jacobi<T>(h->D, 0, ip, st);
    CKL();
    std::swap(I.z, I.t);
  }
  {
    // residual of the shifted systems into t, then full weighting to the
    // coarser grid (with the coarse zero-start Jacobi iterate)
    InnerParams<T> ip = inner_params<T>(h, Lv, k, P, sh, use_cbar);
    launch_shifted_residual<T>(h->D, ip, st);
    CKL();
    launch_inner_restrict<T>(h->D, ip, st);
    CKL();
  }
  TRY(inner_vcycle<T>(h, Lv, k + 1, depth, sweeps, P, sh, use_cbar, true, nullptr, st));
  const int nt_in = h->nt_override > 0 ? h->nt_override : Lv.Nt;
  launch_prolong_space_add<T>(h->D, I.g, Lv.in[k + 1].g, (long long)nt_in * P, (const T*)Lv.in[k + 1].z,
                              (T*)I.z, st);
  CKL();
  for (int it = 0; it < ns; ++it) {
    InnerParams<T> ip = inner_params<T>(h, Lv, k, P, sh, use_cbar);
    if (fuse && it == ns - 1) {
      apply_fuse(ip, *fuse);
      launch_inner_jacobi<T>(h->D, 0, ip, st);
      CKL();
    } else {
      launch_inner_jacobi<T>(h->D, 0, ip, st);
      CKL();
      std::swap(I.z, I.t);
    }
  }
  return ST_OK;
}

// Solve the shifted systems with rhs in[0].y into in[0].z (zero start; when
// `zero_done`, in[0].z already holds the zero-start Jacobi iterate).  With
// `fuse` the last sweep applies the back-transform update instead.
template <typename T>
int inner_solve(st_handle* h, Level& Lv, int depth, int sweeps, int P, const Shifts<T>& sh, bool use_cbar,
                int cycles, bool zero_done, const BtFuse<T>* fuse, cudaStream_t st) {
  const bool smem_bottom_only = Lv.in.size() == 1 && Lv.in[0].g.Ns <= kInnerCoarseLimit;
  if (smem_bottom_only) cycles = 1;  // the shared-memory solve restarts from zero
  for (int c = 0; c < cycles; ++c) {
    const BtFuse<T>* f = (c == cycles - 1) ? fuse : nullptr;
    bool pre = false;
    if (c == 0 && !smem_bottom_only) {
      if (!zero_done) {
        InnerParams<T> ip = inner_params<T>(h, Lv, 0, P, sh, use_cbar);
        ip.zout = (T*)Lv.in[0].z;
        launch_inner_jacobi<T>(h->D, 1, ip, st);  // zero start
        CKL();
      }
      pre = true;
    }
    TRY(inner_vcycle<T>(h, Lv, 0, depth, sweeps, P, sh, use_cbar, pre, f, st));
  }
  return ST_OK;
}

// ---------------------------------------------------------------------------
// Level operations of the space-time cycle
// ---------------------------------------------------------------------------
template <typename T>
LinParams<T> lin_params(st_handle* h, const Level& Lv, int adj) {
  LinParams<T> lp;
  lp.g = Lv.g;
  lp.Nt = Lv.Nt;
  lp.M = Lv.M;
  lp.chunk = (Lv.g.Ns >= 4096 && Lv.Nt >= 8) ? 4 : 1;
  lp.transpose = adj;
  for (int a = 0; a < MAXM; ++a)
    for (int b = 0; b < MAXM; ++b) {
      const double q = (a < Lv.M && b < Lv.M) ? (adj ? Lv.ns->col.Q[b][a] : Lv.ns->col.Q[a][b]) : 0.0;
      lp.W[a][b] = (T)(Lv.dt * q);
      lp.F[a][b] = (T)(adj ? Lv.ns->Fa[a][b] : Lv.ns->Ff[a][b]);
    }
  lp.sc = stencil_of<T>(Lv.g, h->p.nu);
  lp.nchunks = (Lv.Nt + lp.chunk - 1) / lp.chunk;
  lp.zout = nullptr;
  lp.sh = level_shifts<T>(*Lv.ns, Lv.dt);
  lp.omega_j = (T)jacobi_weight(h->D);
  lp.e = nullptr;
  lp.r = nullptr;
  lp.cbar = (h->p.reaction != ST_REACTION_NONE) ? (const T*)Lv.cbar : nullptr;
  // the finest level's operator is the exact Jacobian (R' per node) when kept
  lp.cnode = (&Lv == &h->L[0] && !adj) ? (const T*)h->cnode : nullptr;
  lp.out = nullptr;
  lp.transform = 0;
  return lp;
}

template <typename T>
int level_residual(st_handle* h, int l, int adj, const void* e, const void* r, void* out, int transform,
                   cudaStream_t st) {
  Level& Lv = h->L[l];
  LinParams<T> lp = lin_params<T>(h, Lv, adj);
  lp.e = (const T*)e;
  lp.r = (const T*)r;
  lp.out = (T*)out;
  lp.transform = transform;
  launch_lin_residual<T>(h->D, lp, st);
  CKL();
  return ST_OK;
}

template <typename T>
int smooth(st_handle* h, int l, int adj, bool e_zero, cudaStream_t st) {
  Level& Lv = h->L[l];
  const int M = Lv.M;
  if (!adj && Lv.fused) {
    LinParams<T> lp = lin_params<T>(h, Lv, 0);
    lp.e = e_zero ? nullptr : (const T*)Lv.e;
    lp.r = (const T*)Lv.r;
    InnerParams<T> ip = inner_params<T>(h, Lv, 0, M, level_shifts<T>(*Lv.ns, Lv.dt),
                                        h->p.reaction != ST_REACTION_NONE);
    ip.omega_bt = (T)Lv.omega;
    for (int a = 0; a < MAXM; ++a)
      for (int b = 0; b < MAXM; ++b) ip.B[a][b] = (T)Lv.ns->Bf[a][b];
    launch_slab_smooth<T>(h->D, lp, ip, Lv.smooth_sweeps, (T*)(e_zero ? Lv.e : Lv.e2), st);
    CKL();
    return ST_OK;
  }
  const bool multi = !(Lv.in.size() == 1 && Lv.in[0].g.Ns <= kInnerCoarseLimit);
  const bool started = !adj && e_zero && (l == 0 ? h->start_ready : ((h->start_mask >> l) & 1u) != 0);
  if (l > 0) h->start_mask &= ~(1u << l);
  if (started) {
    // the fine residual (level 0) or the residual-restriction kernel (the
    // levels below) wrote this step's y = F r and zero-start z
  } else {
    // residual + Q-eigenbasis transform (+ zero-start Jacobi of the slab systems)
    LinParams<T> lp = lin_params<T>(h, Lv, adj);
    lp.e = e_zero ? nullptr : (const T*)Lv.e;
    lp.r = (const T*)Lv.r;
    lp.out = (T*)Lv.in[0].y;
    lp.transform = 1;
    lp.zout = multi ? (T*)Lv.in[0].z : nullptr;
    launch_lin_residual<T>(h->D, lp, st);
    CKL();
  }
  const bool use_cbar = h->p.reaction != ST_REACTION_NONE;
  BtFuse<T> f;
  f.on = true;
  f.e_zero = e_zero ? 1 : 0;
  f.omega = (T)Lv.omega;
  f.e = (T*)Lv.e;
  for (int a = 0; a < MAXM; ++a)
    for (int b = 0; b < MAXM; ++b) f.B[a][b] = (T)(adj ? Lv.ns->Ba[a][b] : Lv.ns->Bf[a][b]);
  // the cycle's last level-0 smoothing step may also do the update of U
  if (l == 0 && !adj && !e_zero && h->upd_target) f.Uslot = h->Uslot;
  TRY(inner_solve<T>(h, Lv, Lv.smooth_depth, Lv.smooth_sweeps, M, level_shifts<T>(*Lv.ns, Lv.dt), use_cbar,
                     h->o.inner_cycles, multi, &f, st));
  return ST_OK;
}

template <typename T>
int restrict_level(st_handle* h, int l, int adj, const void* fine, void* coarse, cudaStream_t st) {
  Level& Lv = h->L[l];
  Level& Lc = h->L[l + 1];
  const int M = Lv.M;
  if (Lv.next == 1) {
    launch_restrict_space<T>(h->D, Lv.g, Lc.g, (long long)Lv.Nt * M, (const T*)fine, (T*)coarse, st);
  } else if (Lv.next == 3) {
    // full weighting of every node plane, then the node-set restriction
    launch_restrict_space<T>(h->D, Lv.g, Lc.g, (long long)Lv.Nt * M, (const T*)fine, (T*)Lv.tmp, st);
    CKL();
    launch_node_transfer<T>(Lc.g.Ns, Lc.Nt, M, Lc.M, adj ? Lv.PnT : Lv.Rn, (const T*)Lv.tmp, (T*)coarse, 0, st);
  } else if (Lv.next == 4) {
    // full weighting in space (every slab), then the slab restriction on the coarse grid
    launch_restrict_space<T>(h->D, Lv.g, Lc.g, (long long)Lv.Nt * M, (const T*)fine, (T*)Lv.tmp, st);
    CKL();
    launch_restrict_time<T>(Lc.g, Lc.Nt, M, adj ? Lv.ns->RtT : Lv.ns->col.Rt, (const T*)Lv.tmp, (T*)coarse, st);
  } else {
    launch_restrict_time<T>(Lv.g, Lc.Nt, M, adj ? Lv.ns->RtT : Lv.ns->col.Rt, (const T*)fine, (T*)coarse, st);
  }
  CKL();
  return ST_OK;
}

template <typename T>
int prolong_level(st_handle* h, int l, int adj, const void* coarse, void* fine, cudaStream_t st) {
  Level& Lv = h->L[l];
  Level& Lc = h->L[l + 1];
  const int M = Lv.M;
  if (Lv.next == 1) {
    launch_prolong_space_add<T>(h->D, Lv.g, Lc.g, (long long)Lv.Nt * M, (const T*)coarse, (T*)fine, st);
  } else if (Lv.next == 3) {
    // node-set interpolation on the coarse grid, then linear interpolation
    launch_node_transfer<T>(Lc.g.Ns, Lc.Nt, Lc.M, M, adj ? Lv.RnT : Lv.Pn, (const T*)coarse, (T*)Lv.tmp, 0, st);
    CKL();
    launch_prolong_space_add<T>(h->D, Lv.g, Lc.g, (long long)Lv.Nt * M, (const T*)Lv.tmp, (T*)fine, st);
  } else if (Lv.next == 4) {
    // slab interpolation on the coarse grid, then linear interpolation in space
    CK(cudaMemsetAsync(Lv.tmp, 0, (size_t)Lc.g.Ns * Lv.Nt * M * h->esz, st));
    launch_prolong_time_add<T>(Lc.g, Lc.Nt, M, adj ? Lv.ns->PtT : Lv.ns->col.Pt, (const T*)coarse, (T*)Lv.tmp, st);
    CKL();
    launch_prolong_space_add<T>(h->D, Lv.g, Lc.g, (long long)Lv.Nt * M, (const T*)Lv.tmp, (T*)fine, st);
  } else {
    launch_prolong_time_add<T>(Lv.g, Lc.Nt, M, adj ? Lv.ns->PtT : Lv.ns->col.Pt, (const T*)coarse, (T*)fine, st);
  }
  CKL();
  return ST_OK;
}

template <typename T>
CoarseParams<T> coarse_params(st_handle* h) {
  Level& Lv = h->L.back();
  CoarseParams<T> cp;
  cp.Nt = Lv.Nt;
  cp.M = Lv.M;
  cp.Nc = h->Nc;
  cp.K = h->K;
  for (int a = 0; a < MAXM; ++a)
    for (int b = 0; b < MAXM; ++b)
      cp.dtq[a][b] = (a < Lv.M && b < Lv.M) ? Lv.dt * Lv.ns->col.Q[a][b] : 0.0;
  cp.nu = h->p.nu;
  cp.Lc = h->Lc;
  cp.cbar = (h->p.reaction != ST_REACTION_NONE) ? (const T*)Lv.cbar : nullptr;
  cp.Ainv = (T*)h->Ainv;
  cp.Wf = (T*)h->Wf;
  cp.Wt = (T*)h->Wt;
  cp.Wfrow = (T*)h->Wfrow;
  cp.Wtrow = (T*)h->Wtrow;
  return cp;
}

template <typename T>
int coarse_solve(st_handle* h, int adj, const void* r, void* e, cudaStream_t st) {
  CoarseParams<T> cp = coarse_params<T>(h);
  launch_coarse_solve<T>(cp, adj, (const T*)r, (T*)e, (T*)h->cin, st);
  CKL();
  return ST_OK;
}

SmoothStart smooth_start(st_handle* h, int l);

// The level residual and its restriction onto level l + 1 as one kernel
// (launch_linres_restrict) where it applies; false: the caller runs both.
// Where level l + 1 smooths with its inner multigrid from e = 0 (fuse_start)
// the kernel also does that smoothing's first step (start_mask).
template <typename T>
bool residual_restrict_fused(st_handle* h, int l, int adj, cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value) {
    Level& Lv = h->L[l];
    if (adj || !h->o.fuse_restrict || Lv.next != 1) return false;
    LinParams<float> lp = lin_params<float>(h, Lv, 0);
    lp.e = (const float*)Lv.e;
    lp.r = (const float*)Lv.r;
    Level& Lc = h->L[l + 1];
    const bool want = h->o.fuse_start && h->o.nu1 >= 1 && l + 2 < (int)h->L.size() && !Lc.fused &&
                      !(Lc.in.size() == 1 && Lc.in[0].g.Ns <= kInnerCoarseLimit);
    SmoothStart ss{};
    if (want) {
      ss = smooth_start(h, l + 1);
      // the coarse level's cbar is written by the linearisation branch
      if (h->split_lin && cudaStreamWaitEvent(st, h->ev_lvl[l + 1], 0) != cudaSuccess) {
        cudaGetLastError();
        return false;
      }
    }
    const float* cbc = h->p.reaction != ST_REACTION_NONE ? (const float*)Lc.cbar : nullptr;
    bool started = false;
    if (!launch_linres_restrict(h->D, lp, Lc.g, (float*)Lc.r, st, want ? &ss : nullptr, cbc, &started))
      return false;
    if (started) h->start_mask |= 1u << (l + 1);
    return true;
  }
  return false;
}

template <typename T>
int vcycle_level(st_handle* h, int l, int adj, cudaStream_t st) {
  Level& Lv = h->L[l];
  const int last = (int)h->L.size() - 1;
  if (l == 0) h->start_mask = 0;
  if (h->split_lin) CK(cudaStreamWaitEvent(st, h->ev_lvl[l == last ? last + 1 : l], 0));
  if (l == last) return coarse_solve<T>(h, adj, Lv.r, Lv.e, st);
  const int nu1 = h->o.nu1, nu2 = h->o.nu2;
  const long long n = Lv.g.Ns * Lv.Nt * Lv.M;
  if (nu1 == 0) CK(cudaMemsetAsync(Lv.e, 0, n * h->esz, st));
  for (int i = 0; i < nu1; ++i) TRY(smooth<T>(h, l, adj, i == 0, st));
  if (!residual_restrict_fused<T>(h, l, adj, st)) {
    TRY(level_residual<T>(h, l, adj, Lv.e, Lv.r, Lv.in[0].y, 0, st));
    TRY(restrict_level<T>(h, l, adj, Lv.in[0].y, h->L[l + 1].r, st));
  }
  TRY(vcycle_level<T>(h, l + 1, adj, st));
  const Level& Lc = h->L[l + 1];
  TRY(prolong_level<T>(h, l, adj, (!adj && Lc.fused) ? Lc.e2 : Lc.e, Lv.e, st));
  for (int i = 0; i < nu2; ++i) {
    h->upd_target = l == 0 && !adj && h->upd_capture && i == nu2 - 1;
    const int s = smooth<T>(h, l, adj, false, st);
    h->upd_target = false;
    TRY(s);
  }
  return ST_OK;
}

// cbar of every level and of its inner levels, restricted from level 0's,
// then the coarsest blocks' inverses.  With `ev` (the linearise + cycle
// graph) only the inner levels the smoothers use are restricted, ev[l] is
// recorded once level l's coefficients are ready and ev[L] after the coarse
// setup.
template <typename T>
int enqueue_linearize(st_handle* h, cudaStream_t st, cudaEvent_t* ev = nullptr) {
  const bool rx = h->p.reaction != ST_REACTION_NONE;
  const size_t L = h->L.size();
  for (size_t l = 0; l < L; ++l) {
    Level& Lv = h->L[l];
    if (rx) {
      const size_t kin = ev ? (size_t)Lv.smooth_depth : Lv.in.size();
      for (size_t k = 1; k < kin; ++k) {
        launch_restrict_space<T>(h->D, Lv.in[k - 1].g, Lv.in[k].g, Lv.Nt, (const T*)Lv.in[k - 1].cbar,
                                 (T*)Lv.in[k].cbar, st);
        CKL();
      }
    }
    if (ev) CK(cudaEventRecord(ev[l], st));
    if (rx && l + 1 < L) {
      Level& Lc = h->L[l + 1];
      if (Lv.next == 1 || Lv.next == 3) {
        launch_restrict_space<T>(h->D, Lv.g, Lc.g, Lv.Nt, (const T*)Lv.cbar, (T*)Lc.cbar, st);
      } else if (Lv.next == 4) {
        launch_restrict_space<T>(h->D, Lv.g, Lc.g, Lv.Nt, (const T*)Lv.cbar, (T*)Lv.tmp, st);
        CKL();
        launch_cbar_time<T>(Lc.g, Lc.Nt, (const T*)Lv.tmp, (T*)Lc.cbar, st);
      } else {
        launch_cbar_time<T>(Lv.g, Lc.Nt, (const T*)Lv.cbar, (T*)Lc.cbar, st);
      }
      CKL();
    }
  }
  if (rx || !h->coarse_ready) {
    CoarseParams<T> cp = coarse_params<T>(h);
    launch_coarse_setup<T>(cp, st);
    CKL();
  }
  if (ev) CK(cudaEventRecord(ev[L], st));
  return ST_OK;
}

int run_graph(st_handle* h, int which, int (*enq)(st_handle*, cudaStream_t)) {
  h->upd_applied = false;
  if (!h->o.use_graphs) return enq(h, h->stream);
  if (h->gexec[which]) h->upd_applied = h->gupd[which];
  if (!h->gexec[which]) {
    // make sure the capture stream sees all prior work of the user stream
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    int s = enq(h, h->cap);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap, &g);
    if (s != ST_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) {
      set_err(e, "cudaStreamEndCapture");
      return ST_ERR_CUDA;
    }
    size_t nn = 0;
    if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess) h->gnodes[which] = nn;
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      set_err(e, "cudaGraphInstantiate");
      return ST_ERR_CUDA;
    }
    h->gexec[which] = ex;
    h->gupd[which] = h->upd_applied;
  }
  CK(cudaGraphLaunch(h->gexec[which], h->stream));
  return ST_OK;
}

template <typename T>
int enq_cycle_fwd(st_handle* h, cudaStream_t st) { return vcycle_level<T>(h, 0, 0, st); }
template <typename T>
int enq_cycle_adj(st_handle* h, cudaStream_t st) { return vcycle_level<T>(h, 0, 1, st); }
template <typename T>
int enq_lin(st_handle* h, cudaStream_t st) { return enqueue_linearize<T>(h, st); }
// linearise on a forked branch, cycle on the main one, joined at the end
template <typename T>
int enq_lin_cycle(st_handle* h, cudaStream_t st) {
  CK(cudaEventRecord(h->ev_fork, st));
  CK(cudaStreamWaitEvent(h->cap2, h->ev_fork, 0));
  TRY(enqueue_linearize<T>(h, h->cap2, h->ev_lvl));
  h->split_lin = true;
  const int s = vcycle_level<T>(h, 0, 0, st);
  h->split_lin = false;
  CK(cudaEventRecord(h->ev_join, h->cap2));
  CK(cudaStreamWaitEvent(st, h->ev_join, 0));
  return s;
}

// the forward cycle (and linearise + cycle) whose first level-0 smoothing
// step the fine residual did (FP32 cycles only)
int enq_cycle_started(st_handle* h, cudaStream_t st) {
  h->start_ready = true;
  const int s = vcycle_level<float>(h, 0, 0, st);
  h->start_ready = false;
  return s;
}
int enq_lin_cycle_started(st_handle* h, cudaStream_t st) {
  h->start_ready = true;
  const int s = enq_lin_cycle<float>(h, st);
  h->start_ready = false;
  return s;
}

// ... whose last level-0 smoothing step also adds e to U (*h->Uslot)
int enq_cycle_started_upd(st_handle* h, cudaStream_t st) {
  h->upd_capture = true;
  const int s = enq_cycle_started(h, st);
  h->upd_capture = false;
  return s;
}
int enq_lin_cycle_started_upd(st_handle* h, cudaStream_t st) {
  h->upd_capture = true;
  const int s = enq_lin_cycle_started(h, st);
  h->upd_capture = false;
  return s;
}

// `started`: the fine residual just did the first smoothing step
// (fine_residual); `upd`: the cycle may also do the update U += e, with U's
// address in h->Uslot (launch_set_uslot before it): h->upd_applied then says
// whether it did (else the caller updates U)
int cycle(st_handle* h, int adj, bool started = false, bool upd = false) {
  if (h->fp64) return run_graph(h, adj, adj ? enq_cycle_adj<double> : enq_cycle_fwd<double>);
  if (started && !adj) return run_graph(h, upd ? 7 : 5, upd ? enq_cycle_started_upd : enq_cycle_started);
  return run_graph(h, adj, adj ? enq_cycle_adj<float> : enq_cycle_fwd<float>);
}

// relinearise and run one forward cycle as one graph
int lin_cycle(st_handle* h, bool started = false, bool upd = false) {
  if (!h->o.use_graphs || !h->cap2) {
    TRY(h->fp64 ? run_graph(h, 2, enq_lin<double>) : run_graph(h, 2, enq_lin<float>));
    h->coarse_ready = true;
    return cycle(h, 0, started, upd);
  }
  if (h->fp64) TRY(run_graph(h, 3, enq_lin_cycle<double>));
  else if (started) TRY(run_graph(h, upd ? 8 : 6, upd ? enq_lin_cycle_started_upd : enq_lin_cycle_started));
  else TRY(run_graph(h, 3, enq_lin_cycle<float>));
  h->coarse_ready = true;
  return ST_OK;
}

int linearize_levels(st_handle* h) {
  int s = h->fp64 ? run_graph(h, 2, enq_lin<double>) : run_graph(h, 2, enq_lin<float>);
  if (s == ST_OK) h->coarse_ready = true;
  return s;
}

void invalidate_graphs(st_handle* h) {
  for (int i = 0; i < st_handle::kGraphs; ++i)
    if (h->gexec[i]) {
      cudaGraphExecDestroy(h->gexec[i]);
      h->gexec[i] = nullptr;
    }
}

// ---------------------------------------------------------------------------
// Fine FP64 steps
// ---------------------------------------------------------------------------
ResidParams fine_params(st_handle* h, const double* U, int adj) {
  ResidParams rp;
  const Level& L0 = h->L[0];
  rp.g = L0.g;
  rp.Nt = h->p.Nt;
  rp.M = h->p.M;
  rp.chunk = h->chunk;
  for (int a = 0; a < MAXM; ++a)
    for (int b = 0; b < MAXM; ++b)
      rp.dtq[a][b] = (a < h->p.M && b < h->p.M) ? L0.dt * (adj ? h->fine->col.Q[b][a] : h->fine->col.Q[a][b]) : 0.0;
  rp.nu = h->p.nu;
  rp.sc = stencil_of<double>(L0.g, h->p.nu);
  rp.nchunks = (rp.Nt + rp.chunk - 1) / rp.chunk;
  rp.rho = h->p.rho;
  rp.reaction = h->p.reaction;
  rp.U = U;
  rp.u0 = h->u0;
  rp.lam = nullptr;
  rp.gT = nullptr;
  rp.R = nullptr;
  rp.cbar = nullptr;
  rp.cnode = nullptr;
  rp.tau = nullptr;
  rp.partial = h->partial;
  return rp;
}

// r = G(U) into R (type per r_fp64), cbar optional, ||G||^2 into scal[slot].
// The first step of the forward cycle's first level-0 smoothing (from
// e = 0: y = F r and the zero-start iterate z) as the fine residual's second
// output, where the cycle is FP32 and level 0 is smoothed by its inner
// multigrid with at least one pre-smoothing step.
bool start_possible(const st_handle* h) {
  if (!h->o.fuse_start || h->fp64 || h->L.size() < 2 || h->o.nu1 < 1) return false;
  const Level& L0 = h->L[0];
  return !L0.fused && !(L0.in.size() == 1 && L0.in[0].g.Ns <= kInnerCoarseLimit);
}

SmoothStart smooth_start(st_handle* h, int l = 0) {
  Level& L0 = h->L[l];
  const LinParams<float> lp = lin_params<float>(h, L0, 0);
  SmoothStart ss;
  ss.y = (float*)L0.in[0].y;
  ss.z = (float*)L0.in[0].z;
  for (int a = 0; a < MAXM; ++a)
    for (int b = 0; b < MAXM; ++b) ss.F[a][b] = lp.F[a][b];
  ss.sh = lp.sh;
  ss.k2 = lp.sc.k2;
  ss.omega = lp.omega_j;
  return ss;
}

// With `started`, the residual also does the cycle's first smoothing step
// where it can and reports whether it did: the forward cycle that follows is
// then run as cycle(h, 0, true) / lin_cycle(h, true).
int fine_residual(st_handle* h, const double* U, void* R, int r_fp64, bool want_cbar, int slot,
                  bool* started = nullptr) {
  ResidParams rp = fine_params(h, U, 0);
  rp.R = R;
  rp.cbar = (want_cbar && h->p.reaction != ST_REACTION_NONE) ? h->L[0].cbar : nullptr;
  rp.cnode = rp.cbar ? h->cnode : nullptr;
  long long nparts = residual_blocks(rp);
  if (started) *started = false;
  if (!r_fp64 && !h->fp64) {  // FP32 output: double-float kernel
    SmoothStart ss{};
    const bool st = started && start_possible(h) && ((ss = smooth_start(h)), residual_start_ok(h->D, rp, &ss));
    launch_residual_ff(h->D, rp, h->stream, st ? &ss : nullptr);
    if (started) *started = st;
    nparts = residual_ff_blocks(h->D, rp);
  } else {
    launch_residual(h->D, r_fp64, h->fp64, rp, h->stream);
  }
  CKL();
  launch_sum_partials(h->partial, nparts, h->scal + slot, h->stream);
  CKL();
  return ST_OK;
}

// A TMA-staged kernel gave up waiting for its copies since this handle last
// looked: report it once.
int tma_report(st_handle* h, int count) {
  if (count > h->tma_seen) {
    h->tma_seen = count;
    return ST_ERR_TIMEOUT;
  }
  return ST_OK;
}

int read_scalars(st_handle* h, int n) {
  CK(cudaMemcpyAsync(h->hscal, h->scal, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  int* hflag = reinterpret_cast<int*>(h->hscal + kHostFlag);
  *hflag = 0;
  if (h->tma_err) CK(cudaMemcpyAsync(hflag, h->tma_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return tma_report(h, *hflag);
}

int stage_in(st_handle* h, const double* U, double** Ud, bool copy) {
  if (!U) return ST_ERR_INVALID_ARG;
  if (is_device_ptr(U)) {
    *Ud = (double*)U;
    return ST_OK;
  }
  if (!h->Ustage) TRY(alloc_typed(h, &h->Ustage, h->D_total * sizeof(double)));
  if (copy)
    CK(cudaMemcpyAsync(h->Ustage, U, h->D_total * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  *Ud = h->Ustage;
  return ST_OK;
}

int stage_out(st_handle* h, double* U, const double* Ud) {
  if (U != Ud) CK(cudaMemcpyAsync(U, Ud, h->D_total * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  return ST_OK;
}

int stage_plane(st_handle* h, const double* p, double* buf, const double** out) {
  if (is_device_ptr(p)) {
    *out = p;
    return ST_OK;
  }
  CK(cudaMemcpyAsync(buf, p, h->L[0].g.Ns * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  *out = buf;
  return ST_OK;
}

double ref_norm(const st_handle* h) {
  double s = 0;
  for (double v : h->u0_host) s += v * v;
  const double r = std::sqrt((double)h->p.M * s);
  return r > 0 ? r : 1.0;
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

void fill_info(st_solve_info* info, int it, int status, double rel, double abs_, double ref, double secs,
               const std::vector<double>& hist) {
  if (!info) return;
  info->iterations = it;
  info->status = status;
  info->rel_residual = rel;
  info->abs_residual = abs_;
  info->ref_norm = ref;
  info->seconds = secs;
  info->cycles = it;
  info->history_len = (int)std::min<size_t>(hist.size(), ST_MAX_HISTORY);
  const size_t off = hist.size() > ST_MAX_HISTORY ? hist.size() - ST_MAX_HISTORY : 0;
  for (int i = 0; i < info->history_len; ++i) info->history[i] = hist[off + i];
}

// The (linearise +) cycle and the update U += e of one outer iteration after
// the fine residual.  Where the fine residual did the first smoothing step
// and U is 16-byte aligned, the cycle's last level-0 step does the update
// (fuse_update; e is then not written: nothing reads it before the next
// cycle overwrites it); otherwise the update is its own launch.
int cycle_and_update(st_handle* h, double* Ud, bool started, bool relin) {
  const bool upd = started && h->o.fuse_update && aligned16(Ud);
  if (upd) {
    launch_set_uslot(h->Uslot, Ud, h->stream);
    CKL();
  }
  if (relin) {
    TRY(lin_cycle(h, started, upd));
    h->linearized = true;
  } else {
    TRY(cycle(h, 0, started, upd));
  }
  h->last_update_in_cycle = upd && h->upd_applied;
  if (!h->last_update_in_cycle) {
    launch_update(h->fp64, Ud, h->L[0].e, h->D_total, h->stream);
    CKL();
  }
  return ST_OK;
}

// One outer iteration on device U: residual + cbar, linearise, cycle, update.
// The squared norm of G(U) is left in scal[0].
int outer_step(st_handle* h, double* Ud, bool do_cycle) {
  const bool rx = h->p.reaction != ST_REACTION_NONE;
  const bool relin = rx && (h->o.newton || !h->linearized);
  bool started = false;
  TRY(fine_residual(h, Ud, h->L[0].r, h->fp64, relin, 0, do_cycle ? &started : nullptr));
  if (!do_cycle) return ST_OK;
  TRY(cycle_and_update(h, Ud, started, relin || !h->coarse_ready));
  return ST_OK;
}

// One outer iteration on a device iterate that returns as soon as ||G(U)||
// is known: the norm is copied to the host behind the residual and the call
// waits for that copy only, while the linearisation, the cycle and the
// update of U stay queued on the stream (stream order covers every later use
// of U).  Repeated calls thus keep the device busy: the next residual is
// queued while this cycle runs.  An expired TMA wait inside the cycle is
// reported by the next call that synchronises.
int outer_step_async(st_handle* h, double* Ud, double* norm) {
  const bool rx = h->p.reaction != ST_REACTION_NONE;
  const bool relin = rx && (h->o.newton || !h->linearized);
  int* deferred = reinterpret_cast<int*>(h->hscal + kHostFlagDeferred);
  bool started = false;
  TRY(fine_residual(h, Ud, h->L[0].r, h->fp64, relin, 0, &started));
  CK(cudaMemcpyAsync(h->hscal, h->scal, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaEventRecord(h->ev_norm, h->stream));
  TRY(cycle_and_update(h, Ud, started, relin || !h->coarse_ready));
  CK(cudaEventSynchronize(h->ev_norm));
  *norm = std::sqrt(h->hscal[0]);
  // the count copied behind the previous call's cycle has landed (it precedes
  // this call's residual on the stream); the next copy goes behind this cycle
  const int seen = *deferred;
  if (h->tma_err) CK(cudaMemcpyAsync(deferred, h->tma_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  return tma_report(h, seen);
}

// Switch the finest level's operator to the exact Jacobian (allocates R'
// per node; the captured cycle graphs hold the old operator).
int enable_exact_jacobian(st_handle* h) {
  if (h->cnode || h->p.reaction == ST_REACTION_NONE) return ST_OK;
  TRY(alloc_into(h, &h->cnode, (size_t)h->D_total * h->esz));
  invalidate_graphs(h);
  return ST_OK;
}

// Right-preconditioned flexible GMRES (Saad 1993) on the finest level's
// linear system (A - C) d = r with r = G(U) in L0.r, one V-cycle as the
// preconditioner; at most o.krylov iterations or until the preconditioned
// residual estimate drops by o.krylov_rtol.  The correction is left in L0.e.
int krylov_step(st_handle* h, int m, int* its) {
  Level& L0 = h->L[0];
  const long long n = h->D_total;
  const size_t es = h->esz;
  const int f64 = h->fp64 ? 1 : 0;
  cudaStream_t st = h->stream;
  double* hk = h->hscal + kHostKrylov;
  if (h->kdim < m) {  // bases for m steps (earlier, smaller ones stay with the handle)
    TRY(alloc_into(h, &h->kV, (size_t)(m + 1) * n * es));
    TRY(alloc_into(h, &h->kZ, (size_t)m * n * es));
    if (!h->kpart) TRY(alloc_typed(h, &h->kpart, (size_t)krylov_partials(n) * sizeof(double)));
    if (!h->kdots) TRY(alloc_typed(h, &h->kdots, 64 * sizeof(double)));
    h->kdim = m;
  }
  auto V = [&](int i) { return (void*)((char*)h->kV + (size_t)i * n * es); };
  auto Z = [&](int i) { return (void*)((char*)h->kZ + (size_t)i * n * es); };
  // hk[0..k) = <w, B_i>, B_i = B + i n
  auto dots = [&](const void* w, const void* B, int k) -> int {
    launch_mdot(f64, w, B, n, k, n, h->kpart, h->kdots, st);
    CKL();
    CK(cudaMemcpyAsync(hk, h->kdots, k * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return ST_OK;
  };
  auto apply = [&](const void* z, void* out) -> int {  // out = -(A - C) z
    if (f64) return level_residual<double>(h, 0, 0, z, nullptr, out, 0, st);
    return level_residual<float>(h, 0, 0, z, nullptr, out, 0, st);
  };
  TRY(dots(L0.r, L0.r, 1));
  const double beta = std::sqrt(hk[0]);
  *its = 0;
  if (!(beta > 0.0) || !std::isfinite(beta)) {
    CK(cudaMemsetAsync(L0.e, 0, n * es, st));
    return std::isfinite(beta) ? ST_OK : ST_ERR_DIVERGED;
  }
  launch_axpby(f64, V(0), L0.r, 1.0 / beta, 0.0, n, st);
  CKL();
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m, 0.0), sn(m, 0.0), g(m + 1, 0.0);
  auto Hc = [&](int i, int j) -> double& { return H[(size_t)j * (m + 1) + i]; };
  g[0] = beta;
  int j = 0;
  while (j < m) {
    CK(cudaMemcpyAsync(L0.r, V(j), n * es, cudaMemcpyDeviceToDevice, st));
    TRY(cycle(h, 0));
    CK(cudaMemcpyAsync(Z(j), L0.e, n * es, cudaMemcpyDeviceToDevice, st));
    TRY(apply(Z(j), V(j + 1)));  // w = -(A - C) z_j
    // classical Gram-Schmidt, twice; H(i, j) = <(A - C) z_j, v_i> = -<w, v_i>
    for (int pass = 0; pass < 2; ++pass) {
      TRY(dots(V(j + 1), h->kV, j + 1));
      KrylovCoef c;
      c.k = j + 1;
      for (int i = 0; i <= j; ++i) {
        c.c[i] = hk[i];
        Hc(i, j) -= hk[i];
      }
      launch_maxpy(f64, V(j + 1), h->kV, n, c, n, st);
      CKL();
    }
    TRY(dots(V(j + 1), V(j + 1), 1));
    const double nrm = std::sqrt(hk[0]);
    if (!std::isfinite(nrm)) return ST_ERR_DIVERGED;
    Hc(j + 1, j) = nrm;
    if (nrm > 0.0) {
      launch_axpby(f64, V(j + 1), V(j + 1), -1.0 / nrm, 0.0, n, st);
      CKL();
    }
    for (int i = 0; i < j; ++i) {
      const double a0 = Hc(i, j), a1 = Hc(i + 1, j);
      Hc(i, j) = cs[i] * a0 + sn[i] * a1;
      Hc(i + 1, j) = -sn[i] * a0 + cs[i] * a1;
    }
    const double den = std::hypot(Hc(j, j), Hc(j + 1, j));
    cs[j] = den > 0.0 ? Hc(j, j) / den : 1.0;
    sn[j] = den > 0.0 ? Hc(j + 1, j) / den : 0.0;
    Hc(j, j) = den;
    Hc(j + 1, j) = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    ++j;
    if (std::fabs(g[j]) <= h->o.krylov_rtol * beta || nrm == 0.0) break;
  }
  std::vector<double> y(j, 0.0);
  for (int i = j - 1; i >= 0; --i) {
    double s = g[i];
    for (int q = i + 1; q < j; ++q) s -= Hc(i, q) * y[q];
    y[i] = Hc(i, i) != 0.0 ? s / Hc(i, i) : 0.0;
  }
  CK(cudaMemsetAsync(L0.e, 0, n * es, st));
  KrylovCoef c;
  c.k = j;
  for (int i = 0; i < j; ++i) c.c[i] = -y[i];
  launch_maxpy(f64, L0.e, h->kZ, n, c, n, st);
  CKL();
  *its = j;
  return ST_OK;
}

// ---------------------------------------------------------------------------
// PFASST (Section 4.1): IMEX SDC sweeps on a hierarchy of space-bisected
// levels with fewer nodes, FAS corrections, serial sweeps on the coarsest.
// ---------------------------------------------------------------------------
// Residual parameters of nt slabs of PFASST level data (FP64 arithmetic).
ResidParams pf_params(st_handle* h, const Level& Lv, int M, const double* U, const double* u0, const double* tau,
                      int nt) {
  ResidParams rp = fine_params(h, U, 0);
  rp.g = Lv.g;
  rp.Nt = nt;
  rp.M = M;
  rp.chunk = 1;
  rp.nchunks = nt;
  for (int a = 0; a < MAXM; ++a)
    for (int b = 0; b < MAXM; ++b) rp.dtq[a][b] = (a < M && b < M) ? Lv.dt * h->ns[M].col.Q[a][b] : 0.0;
  rp.sc = stencil_of<double>(Lv.g, h->p.nu);
  rp.u0 = u0;
  rp.tau = tau;
  rp.partial = nullptr;
  return rp;
}

// One IMEX SDC sweep (correction form) of slabs [n0, n0 + nt) of level l
// with M nodes; slab n0 starts from u0 if n0 == 0, else from the current
// last node of slab n0 - 1.  Spatial solves: the level's inner multigrid.
int pf_sweep(st_handle* h, int l, int M, double* U, const double* u0, const double* tau, int n0, int nt) {
  Level& Lv = h->L[l];
  const long long Ns = Lv.g.Ns;
  double* Un = U + (long long)n0 * M * Ns;
  const double* prev = n0 == 0 ? u0 : U + ((long long)(n0 - 1) * M + (M - 1)) * Ns;
  ResidParams rp = pf_params(h, Lv, M, Un, prev, tau ? tau + (long long)n0 * M * Ns : nullptr, nt);
  rp.R = Lv.r;
  launch_residual(h->D, h->fp64, h->fp64, rp, h->stream);
  CKL();
  const Colloc& c = h->ns[M].col;
  const double(*QI)[MAXM] = (h->o.sdc_qdelta == ST_SDC_LU) ? c.QI_lu : c.QI_ie;
  h->nt_override = nt;
  int s = ST_OK;
  for (int m = 0; m < M && s == ST_OK; ++m) {
    SdcCoef cf;
    for (int q = 0; q < MAXM; ++q) {
      cf.qi[q] = (q < m) ? Lv.dt * QI[m][q] : 0.0;
      cf.qe[q] = (q < m) ? Lv.dt * c.QE[m][q] : 0.0;
    }
    launch_sdc_rhs(h->D, h->fp64, Lv.g, nt, M, m, h->p.nu, h->p.reaction, h->p.rho, cf, Lv.r, Lv.e, Un,
                   Lv.in[0].y, h->stream);
    if (cudaGetLastError() != cudaSuccess) { s = ST_ERR_CUDA; break; }
    if (h->fp64)
      s = inner_solve<double>(h, Lv, (int)Lv.in.size(), Lv.bottom_sweeps, 1, real_shift<double>(Lv.dt * QI[m][m]),
                              false, h->o.sdc_inner_cycles, false, nullptr, h->stream);
    else
      s = inner_solve<float>(h, Lv, (int)Lv.in.size(), Lv.bottom_sweeps, 1,
                             real_shift<float>((float)(Lv.dt * QI[m][m])), false, h->o.sdc_inner_cycles, false,
                             nullptr, h->stream);
    if (s != ST_OK) break;
    launch_scatter_plane(h->fp64, Lv.in[0].z, Lv.e, Ns, nt, M, m, h->stream);
  }
  h->nt_override = 0;
  TRY(s);
  CKL();
  launch_update(h->fp64, Un, Lv.e, (long long)nt * M * Ns, h->stream);
  CKL();
  return ST_OK;
}

// W = dt Q F(U) + tau on every slab of level l (M nodes)
int pf_integrals(st_handle* h, int l, int M, const double* U, const double* u0, const double* tau, double* W) {
  Level& Lv = h->L[l];
  ResidParams rp = pf_params(h, Lv, M, U, u0, tau, Lv.Nt);
  rp.R = W;
  launch_residual(h->D, 1, h->fp64, rp, h->stream);
  CKL();
  launch_add_state(W, U, u0, Lv.g.Ns, Lv.Nt, M, h->stream);
  CKL();
  return ST_OK;
}

// out (level l + 1) = value restriction of in (level l, Mf nodes)
int pf_restrict(st_handle* h, int l, int Mf, const double* in, double* out) {
  Level& Lf = h->L[l];
  Level& Lc = h->L[l + 1];
  PfLevel& P = h->pf[l + 1];
  launch_restrict_space<double>(h->D, Lf.g, Lc.g, (long long)Lf.Nt * Mf, in, P.tmp, h->stream);
  CKL();
  launch_node_transfer<double>(Lc.g.Ns, Lc.Nt, Mf, P.M, P.Rv, P.tmp, out, 0, h->stream);
  CKL();
  return ST_OK;
}

// fine (level l, Mf nodes) += interpolation of d (level l + 1)
int pf_prolong_add(st_handle* h, int l, int Mf, const double* d, double* fine) {
  Level& Lf = h->L[l];
  Level& Lc = h->L[l + 1];
  PfLevel& P = h->pf[l + 1];
  launch_node_transfer<double>(Lc.g.Ns, Lc.Nt, P.M, Mf, P.Pv, d, P.tmp, 0, h->stream);
  CKL();
  launch_prolong_space_add<double>(h->D, Lf.g, Lc.g, (long long)Lf.Nt * Mf, P.tmp, fine, h->stream);
  CKL();
  return ST_OK;
}

int pf_setup(st_handle* h, int nl) {
  if ((int)h->pf.size() == nl) {
    for (int l = 1; l < nl; ++l) {  // the initial value may have changed
      const double* src = l == 1 ? h->u0 : h->pf[l - 1].u0;
      launch_restrict_space<double>(h->D, h->L[l - 1].g, h->L[l].g, 1, src, h->pf[l].u0, h->stream);
      CKL();
    }
    return ST_OK;
  }
  if (!h->pf.empty()) return ST_ERR_INVALID_ARG;  // the hierarchy is fixed per handle
  h->pf.resize(nl);
  TRY(alloc_typed(h, &h->pfW0, (size_t)h->D_total * sizeof(double)));
  TRY(alloc_typed(h, &h->pfU, (size_t)h->D_total * sizeof(double)));
  for (int l = 1; l < nl; ++l) {
    PfLevel& P = h->pf[l];
    const int Mf = l == 1 ? h->p.M : h->pf[l - 1].M;
    P.M = std::min(h->o.pfasst_coarse_M, Mf);
    const Level& Lv = h->L[l];
    const size_t n = (size_t)Lv.g.Ns * Lv.Nt * P.M;
    TRY(alloc_typed(h, &P.U, n * sizeof(double)));
    TRY(alloc_typed(h, &P.Ubar, n * sizeof(double)));
    TRY(alloc_typed(h, &P.tau, n * sizeof(double)));
    TRY(alloc_typed(h, &P.W, n * sizeof(double)));
    TRY(alloc_typed(h, &P.tmp, (size_t)Lv.g.Ns * Lv.Nt * Mf * sizeof(double)));
    TRY(alloc_typed(h, &P.u0, (size_t)Lv.g.Ns * sizeof(double)));
    if (node_eval_setup(Mf, P.M, P.Rv) != 0 || node_eval_setup(P.M, Mf, P.Pv) != 0) return ST_ERR_UNSUPPORTED;
    // the restricted initial value
    const double* src = l == 1 ? h->u0 : h->pf[l - 1].u0;
    launch_restrict_space<double>(h->D, h->L[l - 1].g, Lv.g, 1, src, P.u0, h->stream);
    CKL();
  }
  return ST_OK;
}

// One PFASST iteration on the finest iterate Ud.
int pf_iteration(st_handle* h, double* Ud) {
  const int nl = (int)h->pf.size();
  const int ns = h->o.pfasst_sweeps;
  const int Nt = h->p.Nt;
  auto lvU = [&](int l) { return l == 0 ? Ud : h->pf[l].U; };
  auto lvM = [&](int l) { return l == 0 ? h->p.M : h->pf[l].M; };
  auto lvu0 = [&](int l) { return l == 0 ? (const double*)h->u0 : (const double*)h->pf[l].u0; };
  auto lvtau = [&](int l) { return l == 0 ? (const double*)nullptr : (const double*)h->pf[l].tau; };
  auto lvW = [&](int l) { return l == 0 ? h->pfW0 : h->pf[l].W; };
  if (nl == 1) {
    for (int s = 0; s < ns; ++s) TRY(pf_sweep(h, 0, lvM(0), Ud, lvu0(0), nullptr, 0, Nt));
    return ST_OK;
  }
  for (int l = 0; l + 1 < nl; ++l) {
    for (int s = 0; s < ns; ++s) TRY(pf_sweep(h, l, lvM(l), lvU(l), lvu0(l), lvtau(l), 0, Nt));
    PfLevel& C = h->pf[l + 1];
    // tau_{l+1} = R(dt Q F(U_l) + tau_l) - dt Q F(R U_l)
    TRY(pf_integrals(h, l, lvM(l), lvU(l), lvu0(l), lvtau(l), lvW(l)));
    TRY(pf_restrict(h, l, lvM(l), lvW(l), C.tau));
    TRY(pf_restrict(h, l, lvM(l), lvU(l), C.U));
    TRY(pf_integrals(h, l + 1, C.M, C.U, C.u0, nullptr, C.W));
    launch_axpby(1, C.tau, C.W, -1.0, 1.0, (long long)h->L[l + 1].g.Ns * Nt * C.M, h->stream);
    CKL();
    CK(cudaMemcpyAsync(C.Ubar, C.U, (size_t)h->L[l + 1].g.Ns * Nt * C.M * sizeof(double),
                       cudaMemcpyDeviceToDevice, h->stream));
  }
  // the coarsest level, slab after slab
  const int c = nl - 1;
  for (int n = 0; n < Nt; ++n)
    for (int s = 0; s < ns; ++s) TRY(pf_sweep(h, c, lvM(c), lvU(c), lvu0(c), lvtau(c), n, 1));
  // back up: U_l += P(U_{l+1} - Ubar_{l+1}), sweeps on the levels in between
  for (int l = nl - 2; l >= 0; --l) {
    PfLevel& C = h->pf[l + 1];
    launch_axpby(1, C.Ubar, C.U, 1.0, -1.0, (long long)h->L[l + 1].g.Ns * Nt * C.M, h->stream);
    CKL();
    TRY(pf_prolong_add(h, l, lvM(l), C.Ubar, lvU(l)));
    if (l > 0)
      for (int s = 0; s < ns; ++s) TRY(pf_sweep(h, l, lvM(l), lvU(l), lvu0(l), lvtau(l), 0, Nt));
  }
  return ST_OK;
}

// The PFASST iteration on the handle's copy of the iterate, captured once as
// a graph (its launch sequence is fixed by the hierarchy: the serial coarsest
// sweep alone is N_t slab sweeps of some twenty launches each).
int enq_pf_iteration(st_handle* h, cudaStream_t st) {
  const cudaStream_t saved = h->stream;
  h->stream = st;
  const int s = pf_iteration(h, h->pfU);
  h->stream = saved;
  return s;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void st_default_opts(st_solver_opts* o) {
  if (!o) return;
  o->precision = ST_PREC_FP32_REFINE;
  o->coarsening = ST_COARSEN_AUTO_MU;
  o->max_levels = ST_MAX_LEVELS;
  o->nu1 = 1;
  o->nu2 = 1;
  o->omega = 0.0;
  o->mu_crit = 1.0;
  o->inner_cycles = 1;
  o->inner_smooth = 1;
  o->inner_coarse_iters = 8;
  o->coarse_max_points = 16;
  o->coarse_max_slabs = 4;
  o->sdc_qdelta = ST_SDC_IE;
  o->sdc_inner_cycles = 2;
  o->tol = 1e-8;
  o->max_iters = 1000;
  o->newton = 1;
  o->use_graphs = 1;
  o->use_pdl = 1;
  o->smooth_inner_levels = 1;
  o->smooth_sweeps = 3;
  o->line_search = 1;
  o->exact_jacobian = 0;
  o->krylov = 0;
  o->krylov_rtol = 1e-2;
  o->krylov_fallback = 10;
  o->pfasst_levels = 3;
  o->pfasst_coarse_M = 1;
  o->pfasst_sweeps = 1;
  o->use_tma = 1;
  o->recompute_slabs = 0;
  o->fuse_sweeps = 1;
  o->fuse_start = 1;
  o->fuse_restrict = 1;
  o->fuse_update = 1;
}

const char* st_status_str(int s) {
  switch (s) {
    case ST_OK: return "ok";
    case ST_ERR_INVALID_ARG: return "invalid argument";
    case ST_ERR_OOM: return "out of device memory";
    case ST_ERR_CUDA: return "CUDA error";
    case ST_ERR_NOT_CONVERGED: return "not converged";
    case ST_ERR_DIVERGED: return "diverged";
    case ST_ERR_TIMEOUT: return "timeout";
    case ST_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
  }
}

const char* st_last_error(void) { return g_err; }

int st_plan(const st_problem* p, const st_solver_opts* oin, st_plan_info* out) {
  st_solver_opts o;
  st_default_opts(&o);
  if (oin) o = *oin;
  TRY(validate(p, &o));
  std::vector<PlanLevel> pl;
  TRY(plan_levels(p, o, pl));
  if (!out) return ST_OK;
  memset(out, 0, sizeof(*out));
  out->levels = (int)pl.size();
  const size_t esz = o.precision == ST_PREC_FP64 ? 8 : 4;
  const bool rx = p->reaction != ST_REACTION_NONE;
  size_t bytes = 0;
  for (size_t l = 0; l < pl.size(); ++l) {
    const PlanLevel& L = pl[l];
    st_level_info& li = out->level[l];
    li.n[0] = L.g.n0; li.n[1] = L.g.n1; li.n[2] = L.g.n2;
    li.Ns = L.g.Ns;
    li.Nt = L.Nt;
    li.dt = L.dt;
    for (int a = 0; a < 3; ++a) li.h[a] = L.g.ih2[a] > 0 ? 1.0 / std::sqrt(L.g.ih2[a]) : 0.0;
    li.mu = L.mu;
    li.next_kind = L.next;
    li.omega = L.omega;
    li.inner_levels = (int)L.inner.size();
    li.M = L.M;
    const size_t D = (size_t)L.g.Ns * L.Nt * L.M;
    bytes += 5 * round_up(D * esz) + (rx ? round_up((size_t)L.g.Ns * L.Nt * esz) : 0);
    if (L.next == 3 || L.next == 4) bytes += round_up((size_t)pl[l + 1].g.Ns * L.Nt * L.M * esz);
    if (fused_smoothing(pl, l, o, esz)) bytes += round_up(D * esz);
    for (size_t k = 1; k < L.inner.size(); ++k) {
      const size_t Dk = (size_t)L.inner[k].Ns * L.Nt * L.M;
      bytes += 3 * round_up(Dk * esz) + (rx ? round_up((size_t)L.inner[k].Ns * L.Nt * esz) : 0);
    }
  }
  const PlanLevel& C = pl.back();
  const size_t Kc = (size_t)C.g.Ns * C.M;
  bytes += round_up(C.Nt * Kc * Kc * esz) + 2 * round_up(C.Nt * Kc * C.g.Ns * esz) +
           2 * round_up(C.Nt * C.g.Ns * C.g.Ns * esz) + round_up(C.Nt * C.g.Ns * esz);
  if (rx && o.exact_jacobian) bytes += round_up((size_t)pl[0].g.Ns * p->Nt * p->M * esz);
  out->workspace_bytes = bytes;
  out->coarse_points = (int)C.g.Ns;
  return ST_OK;
}

int st_create(const st_problem* pin, const st_solver_opts* oin, const st_runtime* rtin, st_handle** out) {
  if (!out) return ST_ERR_INVALID_ARG;
  *out = nullptr;
  st_solver_opts o;
  st_default_opts(&o);
  if (oin) o = *oin;
  TRY(validate(pin, &o));
  if (!pin->u0) return ST_ERR_INVALID_ARG;
  std::vector<PlanLevel> pl;
  TRY(plan_levels(pin, o, pl));
  st_handle* h = new st_handle();
  h->p = *pin;
  h->p.u0 = nullptr;
  h->o = o;
  if (rtin) h->rt = *rtin;
  else memset(&h->rt, 0, sizeof(h->rt));
  h->stream = (cudaStream_t)h->rt.stream;
  h->D = pin->d;
  h->fp64 = o.precision == ST_PREC_FP64;
  h->esz = h->fp64 ? 8 : 4;
  auto fail = [&](int s) {
    st_destroy(h);
    return s;
  };
  for (int m = 1; m <= pin->M; ++m) {
    if (colloc_setup(m, &h->ns[m].col) != 0) return fail(ST_ERR_UNSUPPORTED);
    build_nodeset(h->ns[m], m);
  }
  h->fine = &h->ns[pin->M];
  if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->cap2, cudaStreamNonBlocking) != cudaSuccess) {
    set_err(cudaGetLastError(), "cudaStreamCreate");
    return fail(ST_ERR_CUDA);
  }
  {
    bool ok = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&h->ev_norm, cudaEventDisableTiming) == cudaSuccess;
    for (int l = 0; l <= ST_MAX_LEVELS && ok; ++l)
      ok = cudaEventCreateWithFlags(&h->ev_lvl[l], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      set_err(cudaGetLastError(), "cudaEventCreate");
      return fail(ST_ERR_CUDA);
    }
  }
  const int M = pin->M;
  const bool rx = pin->reaction != ST_REACTION_NONE;
  // levels and buffers
  slab_smooth_prepare();
  sweep2_prepare();
  linres_restrict_prepare();
  h->L.resize(pl.size());
  for (size_t l = 0; l < pl.size(); ++l) {
    Level& Lv = h->L[l];
    Lv.g = pl[l].g;
    Lv.Nt = pl[l].Nt;
    Lv.dt = pl[l].dt;
    Lv.mu = pl[l].mu;
    Lv.omega = pl[l].omega;
    Lv.next = pl[l].next;
    Lv.M = pl[l].M;
    Lv.ns = &h->ns[Lv.M];
    Lv.bottom_sweeps = pl[l].bottom_sweeps;
    {
      // While some coarser level of the hierarchy is coarser in space, the
      // smooth spatial error is left to it, so the slab solves need only damp
      // the oscillatory part; below the last space bisection (only slab
      // bisection or the coarsest level follows) they keep the full spatial
      // multigrid.  So does a level whose next coarser one has fewer nodes:
      // the error modes of its time polynomial that the coarse node set does
      // not represent are left to the smoother at every spatial frequency.
      const int full = (int)pl[l].inner.size();
      Lv.smooth_depth = smooth_depth_of(pl, l, h->o);
      Lv.smooth_sweeps = Lv.smooth_depth < full ? h->o.smooth_sweeps : Lv.bottom_sweeps;
      Lv.fused = fused_smoothing(pl, l, h->o, h->esz) &&
                 (h->fp64 ? slab_smooth_fits<double>(Lv.M, Lv.g.Ns) : slab_smooth_fits<float>(Lv.M, Lv.g.Ns));
    }
    const size_t D = (size_t)Lv.g.Ns * Lv.Nt * Lv.M;
    int s = ST_OK;
    if (Lv.next == 3) {
      double P[MAXM][MAXM], R[MAXM][MAXM];
      if (node_transfer_setup(Lv.M, pl[l + 1].M, P, R) != 0) return fail(ST_ERR_UNSUPPORTED);
      for (int i = 0; i < MAXM; ++i)
        for (int j = 0; j < MAXM; ++j) {
          Lv.Pn[i][j] = P[i][j];
          Lv.Rn[i][j] = R[i][j];
          Lv.PnT[i][j] = P[j][i];
          Lv.RnT[i][j] = R[j][i];
        }
      s |= alloc_into(h, &Lv.tmp, (size_t)pl[l + 1].g.Ns * Lv.Nt * Lv.M * h->esz);
    }
    if (Lv.next == 4) s |= alloc_into(h, &Lv.tmp, (size_t)pl[l + 1].g.Ns * Lv.Nt * Lv.M * h->esz);
    s |= alloc_into(h, &Lv.e, D * h->esz);
    if (Lv.fused) s |= alloc_into(h, &Lv.e2, D * h->esz);
    s |= alloc_into(h, &Lv.r, D * h->esz);
    if (rx) s |= alloc_into(h, &Lv.cbar, (size_t)Lv.g.Ns * Lv.Nt * h->esz);
    Lv.in.resize(pl[l].inner.size());
    for (size_t k = 0; k < Lv.in.size(); ++k) {
      InnerLev& I = Lv.in[k];
      I.g = pl[l].inner[k];
      const size_t Dk = (size_t)I.g.Ns * Lv.Nt * Lv.M;
      s |= alloc_into(h, &I.y, Dk * h->esz);
      s |= alloc_into(h, &I.z, Dk * h->esz);
      s |= alloc_into(h, &I.t, Dk * h->esz);
      if (k == 0) I.cbar = Lv.cbar;
      else if (rx) s |= alloc_into(h, &I.cbar, (size_t)I.g.Ns * Lv.Nt * h->esz);
    }
    if (s != ST_OK) return fail(ST_ERR_OOM);
  }
  h->D_total = (long long)h->L[0].g.Ns * pin->Nt * M;
  h->chunk = (h->L[0].g.Ns >= 4096 && pin->Nt >= 8) ? 4 : 1;
  if (rx && h->o.exact_jacobian) {
    if (alloc_into(h, &h->cnode, (size_t)h->D_total * h->esz) != ST_OK) return fail(ST_ERR_OOM);
  }
  // coarsest level
  {
    Level& C = h->L.back();
    h->Nc = (int)C.g.Ns;
    h->K = h->Nc * C.M;
    // dense Laplacian of the coarsest grid by applying the stencil to unit vectors
    std::vector<double> Lc((size_t)h->Nc * h->Nc, 0.0);
    const int nn[3] = {C.g.n0, C.g.n1, C.g.n2};
    const long long st3[3] = {1, C.g.n0, (long long)C.g.n0 * C.g.n1};
    for (long long s = 0; s < C.g.Ns; ++s) {
      long long r = s;
      int ij[3];
      ij[0] = (int)(r % nn[0]); r /= nn[0];
      ij[1] = (int)(r % nn[1]);
      ij[2] = (int)(r / nn[1]);
      for (int a = 0; a < h->D; ++a) {
        const double w = C.g.ih2[a];
        Lc[s * h->Nc + s] += -2.0 * w;
        for (int dir = -1; dir <= 1; dir += 2) {
          int q = ij[a] + dir;
          bool zero = false;
          if (q < 0 || q >= nn[a]) {
            if (C.g.bc == ST_BC_PERIODIC) q = (q + nn[a]) % nn[a];
            else if (C.g.bc == ST_BC_NEUMANN) q = (q < 0) ? 1 : nn[a] - 2;
            else zero = true;
          }
          if (!zero) Lc[s * h->Nc + (s + (long long)(q - ij[a]) * st3[a])] += w;
        }
      }
    }
    int s = ST_OK;
    s |= alloc_typed(h, &h->Lc, Lc.size() * sizeof(double));
    const size_t Kc = h->K;
    s |= alloc_into(h, &h->Ainv, (size_t)C.Nt * Kc * Kc * h->esz);
    s |= alloc_into(h, &h->Wf, (size_t)C.Nt * Kc * h->Nc * h->esz);
    s |= alloc_into(h, &h->Wt, (size_t)C.Nt * Kc * h->Nc * h->esz);
    s |= alloc_into(h, &h->Wfrow, (size_t)C.Nt * h->Nc * h->Nc * h->esz);
    s |= alloc_into(h, &h->Wtrow, (size_t)C.Nt * h->Nc * h->Nc * h->esz);
    s |= alloc_into(h, &h->cin, (size_t)C.Nt * h->Nc * h->esz);
    if (s != ST_OK) return fail(ST_ERR_OOM);
    if (cudaMemcpyAsync(h->Lc, Lc.data(), Lc.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream) !=
        cudaSuccess) {
      set_err(cudaGetLastError(), "copy Lc");
      return fail(ST_ERR_CUDA);
    }
    cudaError_t e = h->fp64 ? prepare_coarse_setup<double>(coarse_params<double>(h))
                            : prepare_coarse_setup<float>(coarse_params<float>(h));
    if (e != cudaSuccess) {
      set_err(e, "cudaFuncSetAttribute");
      return fail(ST_ERR_CUDA);
    }
  }
  // fine-level buffers
  {
    const long long Ns = h->L[0].g.Ns;
    ResidParams rp = fine_params(h, nullptr, 0);
    h->npartial = std::max(residual_blocks(rp), gradient_blocks(rp));
    int s = ST_OK;
    s |= alloc_typed(h, &h->partial, h->npartial * sizeof(double));
    s |= alloc_typed(h, &h->partial2, h->npartial * sizeof(double));
    s |= alloc_typed(h, &h->scal, 8 * sizeof(double));
    s |= alloc_typed(h, &h->Uslot, sizeof(double*));
    s |= alloc_typed(h, &h->u0, Ns * sizeof(double));
    s |= alloc_typed(h, &h->plane, Ns * sizeof(double));
    s |= alloc_typed(h, &h->plane2, Ns * sizeof(double));
    if (s != ST_OK) return fail(ST_ERR_OOM);
    if (cudaMallocHost(&h->hscal, kHostScalars * sizeof(double)) != cudaSuccess) {
      set_err(cudaGetLastError(), "cudaMallocHost");
      return fail(ST_ERR_CUDA);
    }
    std::memset(h->hscal, 0, kHostScalars * sizeof(double));
  }
  h->tma_err = tma_error_flag();
  if (h->tma_err) {  // expiries before this handle existed are not its own
    int c = 0;
    if (cudaMemcpy(&c, h->tma_err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess) h->tma_seen = c;
  }
  tma_prepare();
  int s = st_set_u0(h, pin->u0);
  if (s != ST_OK) return fail(s);
  // zero the cycle buffers once (cbar stays 0 for linear problems)
  for (auto& Lv : h->L) {
    const size_t D = (size_t)Lv.g.Ns * Lv.Nt * Lv.M;
    const cudaError_t e = cudaMemsetAsync(Lv.e, 0, D * h->esz, h->stream);
    if (e != cudaSuccess) {
      set_err(e, "cudaMemsetAsync");
      return fail(ST_ERR_CUDA);
    }
  }
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
    set_err(cudaGetLastError(), "st_create sync");
    return fail(ST_ERR_CUDA);
  }
  *out = h;
  return ST_OK;
}

void st_destroy(st_handle* h) {
  if (!h) return;
  invalidate_graphs(h);
  cudaStreamSynchronize(h->stream);
  for (auto it = h->allocs.rbegin(); it != h->allocs.rend(); ++it) {
    if (h->rt.alloc) {
      if (h->rt.free) h->rt.free(it->p, it->bytes, (void*)h->stream, h->rt.ctx);
    } else {
      cudaFreeAsync(it->p, h->stream);
    }
  }
  cudaStreamSynchronize(h->stream);
  if (h->hscal) cudaFreeHost(h->hscal);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->cap2) cudaStreamDestroy(h->cap2);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_norm) cudaEventDestroy(h->ev_norm);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  for (int l = 0; l <= ST_MAX_LEVELS; ++l)
    if (h->ev_lvl[l]) cudaEventDestroy(h->ev_lvl[l]);
  cudaGetLastError();
  delete h;
}

int st_set_params(st_handle* h, double nu, double rho) {
  PdlScope pdl_scope(h);
  if (!h || !(nu > 0) || !std::isfinite(rho)) return ST_ERR_INVALID_ARG;
  h->p.nu = nu;
  h->p.rho = rho;
  for (auto& Lv : h->L) {
    Lv.mu = nu * Lv.dt * Lv.g.ih2[0];
    Lv.omega = default_omega(h->o, Lv.mu);
  }
  invalidate_graphs(h);
  h->coarse_ready = false;
  h->linearized = false;
  return ST_OK;
}

int st_set_u0(st_handle* h, const double* u0) {
  PdlScope pdl_scope(h);
  if (!h || !u0) return ST_ERR_INVALID_ARG;
  const long long Ns = h->L[0].g.Ns;
  h->u0_host.assign(Ns, 0.0);
  const cudaMemcpyKind k = is_device_ptr(u0) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
  CK(cudaMemcpy(h->u0_host.data(), u0, Ns * sizeof(double), k));
  CK(cudaMemcpyAsync(h->u0, h->u0_host.data(), Ns * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return ST_OK;
}

int st_residual(st_handle* h, const double* U, void* R, int R_is_fp64, double* norm_out) {
  PdlScope pdl_scope(h);
  if (!h || !U) return ST_ERR_INVALID_ARG;
  double* Ud = nullptr;
  TRY(stage_in(h, U, &Ud, true));
  const int r64 = (R_is_fp64 || h->fp64) ? 1 : 0;
  void* Rd = R;
  const bool host_R = R && !is_device_ptr(R);
  if (host_R) Rd = h->L[0].r;  // device staging (may need a double-size buffer)
  if (host_R && r64 && !h->fp64) {
    // FP64 output for an FP32 handle on the host: level 0's residual buffer
    // holds floats, so stage through a buffer of its own
    if (!h->Rstage) TRY(alloc_typed(h, &h->Rstage, h->D_total * sizeof(double)));
    Rd = h->Rstage;
  }
  TRY(fine_residual(h, Ud, Rd, r64, false, 0));
  if (host_R)
    CK(cudaMemcpyAsync(R, Rd, h->D_total * (r64 ? 8 : 4), cudaMemcpyDeviceToHost, h->stream));
  TRY(read_scalars(h, 1));
  if (norm_out) *norm_out = std::sqrt(h->hscal[0]);
  return ST_OK;
}

int st_vcycle(st_handle* h, double* U, double* norm_out) {
  PdlScope pdl_scope(h);
  if (!h || !U) return ST_ERR_INVALID_ARG;
  if (is_device_ptr(U)) {
    double nrm = 0.0;
    TRY(outer_step_async(h, U, &nrm));
    if (norm_out) *norm_out = nrm;
    return ST_OK;
  }
  double* Ud = nullptr;
  TRY(stage_in(h, U, &Ud, true));
  TRY(outer_step(h, Ud, true));
  TRY(stage_out(h, U, Ud));
  TRY(read_scalars(h, 1));
  if (norm_out) *norm_out = std::sqrt(h->hscal[0]);
  return ST_OK;
}

int st_solve(st_handle* h, double* U, st_solve_info* info) {
  PdlScope pdl_scope(h);
  if (!h || !U) return ST_ERR_INVALID_ARG;
  const double t0 = now_s();
  double* Ud = nullptr;
  TRY(stage_in(h, U, &Ud, true));
  const double ref = ref_norm(h);
  std::vector<double> hist;
  int status = ST_ERR_NOT_CONVERGED;
  double rel = 0, nrm = 0;
  int it = 0;
  // Backtracking on ||G|| (non-linear problems): the step U += alpha e of an
  // iteration is halved until ||G|| drops by the factor 1 - 1e-4 alpha.
  const bool ls = h->o.line_search && h->p.reaction != ST_REACTION_NONE;
  double alpha = 0.0, prev = 0.0;
  int cycles = 0;
  int kry = h->o.krylov;
  for (;;) {
    bool started = false;
    TRY(fine_residual(h, Ud, h->L[0].r, h->fp64,
                      h->p.reaction != ST_REACTION_NONE && (h->o.newton || !h->linearized), 0,
                      kry == 0 ? &started : nullptr));
    TRY(read_scalars(h, 1));
    nrm = std::sqrt(h->hscal[0]);
    rel = nrm / ref;
    if (ls && alpha > 0.0 && !(nrm <= (1.0 - 1e-4 * alpha) * prev)) {
      if (alpha < kMinStep) {
        if (kry == 0 && h->o.krylov_fallback > 0) {
          // the cycle's correction is no descent direction here: continue
          // with Newton steps on the exact Jacobian solved by FGMRES
          kry = h->o.krylov_fallback;
          TRY(enable_exact_jacobian(h));
          alpha = 0.0;
          continue;
        }
        status = ST_ERR_DIVERGED;
        break;
      }
      launch_update(h->fp64, Ud, h->L[0].e, h->D_total, h->stream, -0.5 * alpha);
      CKL();
      alpha *= 0.5;
      continue;
    }
    hist.push_back(rel);
    if (!std::isfinite(rel) || rel > 1e8) { status = ST_ERR_DIVERGED; break; }
    if (rel <= h->o.tol) { status = ST_OK; break; }
    if (it >= h->o.max_iters) { status = ST_ERR_NOT_CONVERGED; break; }
    const bool relin = h->p.reaction != ST_REACTION_NONE && (h->o.newton || !h->linearized);
    bool did_cycle = false;
    if (kry == 0 && (relin || !h->coarse_ready)) {
      TRY(lin_cycle(h, started));
      h->linearized = true;
      did_cycle = true;
      ++cycles;
    } else if (relin || !h->coarse_ready) {
      TRY(linearize_levels(h));
      h->linearized = true;
    }
    if (kry > 0) {
      int lits = 0;
      const int s = krylov_step(h, kry, &lits);
      cycles += lits;
      if (s != ST_OK) {
        status = s;
        break;
      }
    } else if (!did_cycle) {
      TRY(cycle(h, 0, started));
      ++cycles;
    }
    launch_update(h->fp64, Ud, h->L[0].e, h->D_total, h->stream);
    CKL();
    prev = nrm;
    alpha = 1.0;
    ++it;
  }
  TRY(stage_out(h, U, Ud));
  CK(cudaStreamSynchronize(h->stream));
  fill_info(info, it, status, rel, nrm, ref, now_s() - t0, hist);
  if (info) info->cycles = cycles;
  return status;
}

int st_pfasst(st_handle* h, double* U, st_solve_info* info) {
  PdlScope pdl_scope(h);
  if (!h || !U) return ST_ERR_INVALID_ARG;
  for (size_t l = 0; l + 1 < h->L.size(); ++l)
    if ((int)l + 1 < h->o.pfasst_levels && h->L[l].next != 1) return ST_ERR_UNSUPPORTED;
  const int nl = std::min(h->o.pfasst_levels, (int)h->L.size());
  const double t0 = now_s();
  double* Ud = nullptr;
  TRY(stage_in(h, U, &Ud, true));
  TRY(pf_setup(h, nl));
  CK(cudaMemcpyAsync(h->pfU, Ud, (size_t)h->D_total * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  const double ref = ref_norm(h);
  std::vector<double> hist;
  int status = ST_ERR_NOT_CONVERGED;
  double rel = 0, nrm = 0;
  int it = 0;
  for (;;) {
    TRY(fine_residual(h, h->pfU, nullptr, 1, false, 0));
    TRY(read_scalars(h, 1));
    nrm = std::sqrt(h->hscal[0]);
    rel = nrm / ref;
    hist.push_back(rel);
    if (!std::isfinite(rel) || rel > 1e8) { status = ST_ERR_DIVERGED; break; }
    if (rel <= h->o.tol) { status = ST_OK; break; }
    if (it >= h->o.max_iters) { status = ST_ERR_NOT_CONVERGED; break; }
    TRY(run_graph(h, 4, enq_pf_iteration));
    ++it;
  }
  CK(cudaMemcpyAsync(Ud, h->pfU, (size_t)h->D_total * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  TRY(stage_out(h, U, Ud));
  CK(cudaStreamSynchronize(h->stream));
  fill_info(info, it, status, rel, nrm, ref, now_s() - t0, hist);
  return status;
}

int st_sdc_sweep(st_handle* h, double* U, int nsweeps, double* norm_out) {
  PdlScope pdl_scope(h);
  if (!h || !U || nsweeps < 1) return ST_ERR_INVALID_ARG;
  double* Ud = nullptr;
  TRY(stage_in(h, U, &Ud, true));
  Level& L0 = h->L[0];
  const int M = h->p.M;
  const double(*QI)[MAXM] = (h->o.sdc_qdelta == ST_SDC_LU) ? h->fine->col.QI_lu : h->fine->col.QI_ie;
  for (int sw = 0; sw < nsweeps; ++sw) {
    TRY(fine_residual(h, Ud, L0.r, h->fp64, false, 0));
    for (int m = 0; m < M; ++m) {
      SdcCoef cf;
      for (int q = 0; q < MAXM; ++q) {
        cf.qi[q] = (q < m) ? L0.dt * QI[m][q] : 0.0;
        cf.qe[q] = (q < m) ? L0.dt * h->fine->col.QE[m][q] : 0.0;
      }
      launch_sdc_rhs(h->D, h->fp64, L0.g, L0.Nt, M, m, h->p.nu, h->p.reaction, h->p.rho, cf, L0.r, L0.e, Ud,
                     L0.in[0].y, h->stream);
      CKL();
      if (h->fp64) {
        Shifts<double> sh = real_shift<double>(L0.dt * QI[m][m]);
        TRY(inner_solve<double>(h, L0, (int)L0.in.size(), L0.bottom_sweeps, 1, sh, false, h->o.sdc_inner_cycles,
                                false, nullptr, h->stream));
      } else {
        Shifts<float> sh = real_shift<float>((float)(L0.dt * QI[m][m]));
        TRY(inner_solve<float>(h, L0, (int)L0.in.size(), L0.bottom_sweeps, 1, sh, false, h->o.sdc_inner_cycles,
                                false, nullptr, h->stream));
      }
      launch_scatter_plane(h->fp64, L0.in[0].z, L0.e, L0.g.Ns, L0.Nt, M, m, h->stream);
      CKL();
    }
    launch_update(h->fp64, Ud, L0.e, h->D_total, h->stream);
    CKL();
  }
  TRY(stage_out(h, U, Ud));
  TRY(read_scalars(h, 1));
  if (norm_out) *norm_out = std::sqrt(h->hscal[0]);
  return ST_OK;
}

int st_adjoint_solve_terminal(st_handle* h, const double* U, const double* gT, double* dnu, double* drho,
                              double* du0, st_solve_info* info) {
  PdlScope pdl_scope(h);
  if (!h || !U || !gT) return ST_ERR_INVALID_ARG;
  const double t0 = now_s();
  double* Ud = nullptr;
  TRY(stage_in(h, U, &Ud, true));
  const double* gd = nullptr;
  TRY(stage_plane(h, gT, h->plane, &gd));
  // Neumann: the mirrored-ghost Laplacian is not symmetric, L^T = W L W^-1
  // with W the lumped mass weights (L = -M_h^-1 K_h, K_h symmetric), so
  // J^T = W J^ W^-1, J^ being J^T with L in place of L^T - the operator the
  // transposed kernels apply.  Solve J^ mu = -W^-1 g, then lambda = W mu.
  const bool neumann = h->p.bc == ST_BC_NEUMANN;
  if (neumann) {
    if (gd != h->plane)
      CK(cudaMemcpyAsync(h->plane, gd, h->L[0].g.Ns * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    launch_mass_weight(h->plane, h->L[0].g, 1, 1, h->stream);
    CKL();
    gd = h->plane;
  }
  if (!h->lam) TRY(alloc_typed(h, &h->lam, h->D_total * sizeof(double)));
  CK(cudaMemsetAsync(h->lam, 0, h->D_total * sizeof(double), h->stream));
  // linearise at U (cbar of every level, coarsest blocks)
  TRY(fine_residual(h, Ud, nullptr, h->fp64, true, 0));
  TRY(linearize_levels(h));
  h->linearized = true;
  std::vector<double> hist;
  int status = ST_ERR_NOT_CONVERGED;
  double rel = 0, nrm = 0, ref = 1;
  int it = 0;
  for (;; ++it) {
    ResidParams rp = fine_params(h, Ud, 1);
    rp.lam = h->lam;
    rp.gT = gd;
    rp.R = h->L[0].r;
    launch_adj_residual(h->D, h->fp64, rp, h->stream);
    CKL();
    launch_sum_partials(h->partial, residual_blocks(rp), h->scal, h->stream);
    CKL();
    TRY(read_scalars(h, 1));
    nrm = std::sqrt(h->hscal[0]);
    if (it == 0) ref = nrm > 0 ? nrm : 1.0;
    rel = nrm / ref;
    hist.push_back(rel);
    if (!std::isfinite(rel) || rel > 1e8) { status = ST_ERR_DIVERGED; break; }
    if (rel <= h->o.tol || nrm == 0) { status = ST_OK; break; }
    if (it >= h->o.max_iters) { status = ST_ERR_NOT_CONVERGED; break; }
    TRY(cycle(h, 1));
    launch_update(h->fp64, h->lam, h->L[0].e, h->D_total, h->stream);
    CKL();
  }
  if (neumann) {
    launch_mass_weight(h->lam, h->L[0].g, (long long)h->L[0].Nt * h->p.M, 0, h->stream);
    CKL();
  }
  // gradients
  {
    ResidParams rp = fine_params(h, Ud, 1);
    rp.lam = h->lam;
    const bool host_du0 = du0 && !is_device_ptr(du0);
    double* du0d = du0 ? (host_du0 ? h->plane2 : du0) : nullptr;
    // dnu partials go to rp.partial (= h->partial), drho partials to partial2
    launch_gradients(h->D, rp, h->partial2, du0d, h->stream);
    CKL();
    const long long nb = gradient_blocks(rp);
    launch_sum_partials(h->partial, nb, h->scal + 1, h->stream);
    launch_sum_partials(h->partial2, nb, h->scal + 2, h->stream);
    CKL();
    if (host_du0)
      CK(cudaMemcpyAsync(du0, h->plane2, h->L[0].g.Ns * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    TRY(read_scalars(h, 3));
    if (dnu) *dnu = h->hscal[1];
    if (drho) *drho = h->hscal[2];
  }
  fill_info(info, it, status, rel, nrm, ref, now_s() - t0, hist);
  return status;
}

int st_adjoint_lambda(st_handle* h, double* out) {
  PdlScope pdl_scope(h);
  if (!h || !out || !h->lam) return ST_ERR_INVALID_ARG;
  CK(cudaMemcpyAsync(out, h->lam, h->D_total * sizeof(double), cudaMemcpyDefault, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return ST_OK;
}

int st_adjoint_solve(st_handle* h, const double* U, const double* u_target, double* dnu, double* drho,
                     double* du0, st_solve_info* info) {
  PdlScope pdl_scope(h);
  if (!h || !U || !u_target) return ST_ERR_INVALID_ARG;
  // gT = h^d (u_{Nt,M} - target), formed on the host from the last plane
  const long long Ns = h->L[0].g.Ns;
  std::vector<double> last(Ns), tgt(Ns);
  const double* lastp = U + (h->D_total - Ns);
  CK(cudaMemcpy(last.data(), lastp, Ns * sizeof(double), cudaMemcpyDefault));
  CK(cudaMemcpy(tgt.data(), u_target, Ns * sizeof(double), cudaMemcpyDefault));
  double hd = 1.0;
  for (int a = 0; a < h->D; ++a) hd /= std::sqrt(h->L[0].g.ih2[a]);
  for (long long s = 0; s < Ns; ++s) last[s] = hd * (last[s] - tgt[s]);
  return st_adjoint_solve_terminal(h, U, last.data(), dnu, drho, du0, info);
}

int st_collocation(int M, double* tau, double* Q, double* lam, double* V, double* Vinv) {
  Colloc c;
  if (colloc_setup(M, &c) != 0) return ST_ERR_INVALID_ARG;
  for (int m = 0; m < M; ++m) {
    if (tau) tau[m] = c.tau[m];
    if (lam) { lam[2 * m] = c.lam[m].real(); lam[2 * m + 1] = c.lam[m].imag(); }
    for (int j = 0; j < M; ++j) {
      if (Q) Q[m * M + j] = c.Q[m][j];
      if (V) { V[2 * (m * M + j)] = c.V[m][j].real(); V[2 * (m * M + j) + 1] = c.V[m][j].imag(); }
      if (Vinv) {
        Vinv[2 * (m * M + j)] = c.Vinv[m][j].real();
        Vinv[2 * (m * M + j) + 1] = c.Vinv[m][j].imag();
      }
    }
  }
  return ST_OK;
}

int st_node_transfer(int Mf, int Mc, double* P, double* R) {
  double Pm[MAXM][MAXM], Rm[MAXM][MAXM];
  if (node_transfer_setup(Mf, Mc, Pm, Rm) != 0) return ST_ERR_INVALID_ARG;
  for (int j = 0; j < Mf; ++j)
    for (int m = 0; m < Mc; ++m) {
      if (P) P[j * Mc + m] = Pm[j][m];
      if (R) R[m * Mf + j] = Rm[m][j];
    }
  return ST_OK;
}

int st_time_transfer(int M, double* Pt, double* Rt) {
  Colloc c;
  if (colloc_setup(M, &c) != 0) return ST_ERR_INVALID_ARG;
  for (int kk = 0; kk < 2 * M; ++kk)
    for (int m = 0; m < M; ++m) {
      if (Pt) Pt[kk * M + m] = c.Pt[kk][m];
      if (Rt) Rt[m * 2 * M + kk] = c.Rt[m][kk];
    }
  return ST_OK;
}

int st_num_levels(const st_handle* h) { return h ? (int)h->L.size() : 0; }

int st_level_info_get(const st_handle* h, int level, st_level_info* out) {
  if (!h || !out || level < 0 || level >= (int)h->L.size()) return ST_ERR_INVALID_ARG;
  const Level& Lv = h->L[level];
  memset(out, 0, sizeof(*out));
  out->n[0] = Lv.g.n0; out->n[1] = Lv.g.n1; out->n[2] = Lv.g.n2;
  out->Ns = Lv.g.Ns;
  out->Nt = Lv.Nt;
  out->dt = Lv.dt;
  for (int a = 0; a < 3; ++a) out->h[a] = Lv.g.ih2[a] > 0 ? 1.0 / std::sqrt(Lv.g.ih2[a]) : 0.0;
  out->mu = Lv.mu;
  out->next_kind = Lv.next;
  out->omega = Lv.omega;
  out->inner_levels = (int)Lv.in.size();
  out->M = Lv.M;
  return ST_OK;
}

int st_linearize(st_handle* h, const double* U) {
  PdlScope pdl_scope(h);
  if (!h || !U) return ST_ERR_INVALID_ARG;
  double* Ud = nullptr;
  TRY(stage_in(h, U, &Ud, true));
  TRY(fine_residual(h, Ud, nullptr, h->fp64, true, 0));
  TRY(linearize_levels(h));
  h->linearized = true;
  CK(cudaStreamSynchronize(h->stream));
  return ST_OK;
}

static size_t level_elems(const st_handle* h, int l) {
  return (size_t)h->L[l].g.Ns * h->L[l].Nt * h->L[l].M;
}

int st_level_cbar(st_handle* h, int level, void* out) {
  PdlScope pdl_scope(h);
  if (!h || !out || level < 0 || level >= (int)h->L.size()) return ST_ERR_INVALID_ARG;
  const Level& Lv = h->L[level];
  const size_t n = (size_t)Lv.g.Ns * Lv.Nt * h->esz;
  if (Lv.cbar) CK(cudaMemcpyAsync(out, Lv.cbar, n, cudaMemcpyDeviceToDevice, h->stream));
  else CK(cudaMemsetAsync(out, 0, n, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return ST_OK;
}

int st_level_residual(st_handle* h, int level, int transpose, const void* e, const void* r, void* out) {
  PdlScope pdl_scope(h);
  if (!h || !r || !out || level < 0 || level >= (int)h->L.size()) return ST_ERR_INVALID_ARG;
  if (h->fp64) TRY(level_residual<double>(h, level, transpose, e, r, out, 0, h->stream));
  else TRY(level_residual<float>(h, level, transpose, e, r, out, 0, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return ST_OK;
}

int st_level_smooth(st_handle* h, int level, int transpose, void* e, const void* r) {
  PdlScope pdl_scope(h);
  if (!h || !e || !r || level < 0 || level >= (int)h->L.size()) return ST_ERR_INVALID_ARG;
  Level& Lv = h->L[level];
  const size_t n = level_elems(h, level) * h->esz;
  CK(cudaMemcpyAsync(Lv.e, e, n, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpyAsync(Lv.r, r, n, cudaMemcpyDeviceToDevice, h->stream));
  if (h->fp64) TRY(smooth<double>(h, level, transpose, false, h->stream));
  else TRY(smooth<float>(h, level, transpose, false, h->stream));
  CK(cudaMemcpyAsync(e, Lv.e, n, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return ST_OK;
}

int st_level_restrict(st_handle* h, int level, int transpose, const void* fine, void* coarse) {
  PdlScope pdl_scope(h);
  if (!h || !fine || !coarse || level < 0 || level + 1 >= (int)h->L.size()) return ST_ERR_INVALID_ARG;
  if (h->fp64) TRY(restrict_level<double>(h, level, transpose, fine, coarse, h->stream));
  else TRY(restrict_level<float>(h, level, transpose, fine, coarse, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return ST_OK;
}

int st_level_prolong(st_handle* h, int level, int transpose, const void* coarse, void* fine) {
  PdlScope pdl_scope(h);
  if (!h || !fine || !coarse || level < 0 || level + 1 >= (int)h->L.size()) return ST_ERR_INVALID_ARG;
  if (h->fp64) TRY(prolong_level<double>(h, level, transpose, coarse, fine, h->stream));
  else TRY(prolong_level<float>(h, level, transpose, coarse, fine, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return ST_OK;
}

int st_coarse_solve(st_handle* h, int transpose, const void* r, void* e) {
  PdlScope pdl_scope(h);
  if (!h || !r || !e) return ST_ERR_INVALID_ARG;
  if (!h->coarse_ready) TRY(linearize_levels(h));
  if (h->fp64) TRY(coarse_solve<double>(h, transpose, r, e, h->stream));
  else TRY(coarse_solve<float>(h, transpose, r, e, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return ST_OK;
}

int st_level_vcycle(st_handle* h, int transpose, const void* r, void* e) {
  PdlScope pdl_scope(h);
  if (!h || !r || !e) return ST_ERR_INVALID_ARG;
  if (!h->coarse_ready) TRY(linearize_levels(h));
  const size_t n = level_elems(h, 0) * h->esz;
  CK(cudaMemcpyAsync(h->L[0].r, r, n, cudaMemcpyDeviceToDevice, h->stream));
  TRY(cycle(h, transpose ? 1 : 0));
  CK(cudaMemcpyAsync(e, h->L[0].e, n, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return ST_OK;
}

int st_time_kernel(st_handle* h, int which, const double* U, int iters, double* ms_per_launch,
                   double* bytes_per_launch) {
  PdlScope pdl_scope(h);
  if (!h || iters < 1 || which < 0 || which > ST_KERNEL_SWEEP2_UPDATE) return ST_ERR_INVALID_ARG;
  if (which >= ST_KERNEL_SHIFTED_RESIDUAL && which <= ST_KERNEL_PROLONG && h->L[0].in.size() < 2)
    return ST_ERR_UNSUPPORTED;
  if ((which == ST_KERNEL_FINE_RESIDUAL || which == ST_KERNEL_UPDATE || which == ST_KERNEL_SWEEP2_UPDATE) &&
      (!U || !is_device_ptr(U)))
    return ST_ERR_INVALID_ARG;
  if (which == ST_KERNEL_SWEEP2_UPDATE && !aligned16(U)) return ST_ERR_UNSUPPORTED;
  Level& L0 = h->L[0];
  const bool rx = h->p.reaction != ST_REACTION_NONE;
  const double D = (double)h->D_total;
  const double planes = (double)L0.g.Ns * L0.Nt;
  const double es = (double)h->esz;
  double bytes = 0;
  if (!h->coarse_ready) TRY(linearize_levels(h));
  auto one = [&](cudaStream_t st) -> int {
    switch (which) {
      case ST_KERNEL_FINE_RESIDUAL: {
        ResidParams rp = fine_params(h, U, 0);
        rp.R = L0.r;
        rp.cbar = rx ? L0.cbar : nullptr;
        rp.cnode = rx ? h->cnode : nullptr;
        if (h->fp64) {
          launch_residual(h->D, 1, 1, rp, st);
        } else {
          // as the step runs it: with the first smoothing step where it applies
          SmoothStart ss{};
          const bool stt = start_possible(h) && ((ss = smooth_start(h)), residual_start_ok(h->D, rp, &ss));
          launch_residual_ff(h->D, rp, st, stt ? &ss : nullptr);
        }
        CKL();
        return ST_OK;
      }
      case ST_KERNEL_LEVEL_RESIDUAL:
        return h->fp64 ? level_residual<double>(h, 0, 0, L0.e, L0.r, L0.in[0].y, 1, st)
                       : level_residual<float>(h, 0, 0, L0.e, L0.r, L0.in[0].y, 1, st);
      case ST_KERNEL_JACOBI: {
        // the fine-level sweep as the cycle runs it last: fused with the
        // back-transform and the damped block-Jacobi update of e
        auto go = [&](auto tag) -> int {
          using TT = decltype(tag);
          InnerParams<TT> ip = inner_params<TT>(h, L0, 0, h->p.M, level_shifts<TT>(*L0.ns, L0.dt), rx);
          BtFuse<TT> f;
          f.on = true;
          f.e_zero = 0;
          f.omega = (TT)L0.omega;
          f.e = (TT*)L0.e;
          for (int a2 = 0; a2 < MAXM; ++a2)
            for (int b = 0; b < MAXM; ++b) f.B[a2][b] = (TT)h->fine->Bf[a2][b];
          apply_fuse(ip, f);
          launch_inner_jacobi<TT>(h->D, 0, ip, st);
          CKL();
          return ST_OK;
        };
        return h->fp64 ? go(double(0)) : go(float(0));
      }
      case ST_KERNEL_JACOBI_PLAIN: {  // z -> t with the level-0 shifts
        auto go = [&](auto tag) -> int {
          using TT = decltype(tag);
          InnerParams<TT> ip = inner_params<TT>(h, L0, 0, h->p.M, level_shifts<TT>(*L0.ns, L0.dt), rx);
          launch_inner_jacobi<TT>(h->D, 0, ip, st);
          CKL();
          return ST_OK;
        };
        return h->fp64 ? go(double(0)) : go(float(0));
      }
      case ST_KERNEL_BACKTRANSFORM: {
        if (h->fp64) {
          double B[MAXM][MAXM];
          for (int a2 = 0; a2 < MAXM; ++a2)
            for (int b = 0; b < MAXM; ++b) B[a2][b] = h->fine->Bf[a2][b];
          launch_backtransform<double>(L0.g, L0.Nt, h->p.M, B, L0.omega, 0, (const double*)L0.in[0].z,
                                       (double*)L0.e, st);
        } else {
          float B[MAXM][MAXM];
          for (int a2 = 0; a2 < MAXM; ++a2)
            for (int b = 0; b < MAXM; ++b) B[a2][b] = (float)h->fine->Bf[a2][b];
          launch_backtransform<float>(L0.g, L0.Nt, h->p.M, B, (float)L0.omega, 0, (const float*)L0.in[0].z,
                                      (float*)L0.e, st);
        }
        CKL();
        return ST_OK;
      }
      case ST_KERNEL_SHIFTED_RESIDUAL:
      case ST_KERNEL_INNER_RESTRICT:
      case ST_KERNEL_PROLONG: {
        auto go = [&](auto tag) -> int {
          using TT = decltype(tag);
          InnerParams<TT> ip = inner_params<TT>(h, L0, 0, h->p.M, level_shifts<TT>(*L0.ns, L0.dt), rx);
          if (which == ST_KERNEL_SHIFTED_RESIDUAL) launch_shifted_residual<TT>(h->D, ip, st);
          else if (which == ST_KERNEL_INNER_RESTRICT) launch_inner_restrict<TT>(h->D, ip, st);
          else
            launch_prolong_space_add<TT>(h->D, L0.in[0].g, L0.in[1].g, (long long)L0.Nt * h->p.M,
                                         (const TT*)L0.in[1].z, (TT*)L0.in[0].z, st);
          CKL();
          return ST_OK;
        };
        return h->fp64 ? go(double(0)) : go(float(0));
      }
      case ST_KERNEL_SWEEP2:
      case ST_KERNEL_SWEEP2_UPDATE: {
        if (h->fp64) return ST_ERR_UNSUPPORTED;
        InnerParams<float> ip = inner_params<float>(h, L0, 0, h->p.M, level_shifts<float>(*L0.ns, L0.dt), rx);
        BtFuse<float> f;
        f.on = true;
        f.e_zero = 0;
        f.omega = (float)L0.omega;
        f.e = (float*)L0.e;
        for (int a2 = 0; a2 < MAXM; ++a2)
          for (int b = 0; b < MAXM; ++b) f.B[a2][b] = (float)h->fine->Bf[a2][b];
        if (which == ST_KERNEL_SWEEP2_UPDATE) f.Uslot = h->Uslot;  // set to U before the timing
        apply_fuse(ip, f);
        if (!launch_sweep2(h->D, ip, st)) return ST_ERR_UNSUPPORTED;
        CKL();
        return ST_OK;
      }
      case ST_KERNEL_RESID_RESTRICT:
        if (h->fp64 || h->L.size() < 2 || !residual_restrict_fused<float>(h, 0, 0, st)) return ST_ERR_UNSUPPORTED;
        CKL();
        return ST_OK;
      case ST_KERNEL_UPDATE:
        // U + 0 * e with e zeroed above: the loads and stores of the cycle's
        // update, U's values unchanged
        launch_update(h->fp64, const_cast<double*>(U), L0.e, h->D_total, st, 0.0);
        CKL();
        return ST_OK;
      default:
        return cycle(h, 0);
    }
  };
  switch (which) {
    case ST_KERNEL_FINE_RESIDUAL: {
      bytes = D * (8 + es) + (rx ? planes * es : 0);
      if (!h->fp64 && start_possible(h)) {
        ResidParams rp = fine_params(h, U, 0);
        rp.R = L0.r;
        rp.cbar = rx ? L0.cbar : nullptr;
        const SmoothStart ss = smooth_start(h);
        if (residual_start_ok(h->D, rp, &ss)) bytes += 2 * D * es;  // y and z
      }
      break;
    }
    case ST_KERNEL_LEVEL_RESIDUAL: bytes = D * 3 * es + (rx ? planes * es : 0); break;
    case ST_KERNEL_JACOBI: bytes = D * 4 * es + (rx ? planes * es : 0); break;
    case ST_KERNEL_JACOBI_PLAIN: bytes = D * 3 * es + (rx ? planes * es : 0); break;
    case ST_KERNEL_BACKTRANSFORM: bytes = D * 3 * es; break;
    case ST_KERNEL_UPDATE: bytes = D * (8 + es + 8); break;
    case ST_KERNEL_SWEEP2: bytes = D * 4 * es + (rx ? planes * es : 0); break;
    case ST_KERNEL_SWEEP2_UPDATE: bytes = D * (3 * es + 16) + (rx ? planes * es : 0); break;  // e not written
    case ST_KERNEL_RESID_RESTRICT:  // e and r read, the coarse residual written
      bytes = 2 * D * es + (rx ? planes * es : 0) +
              (h->L.size() > 1 ? (double)h->L[1].g.Ns * h->L[1].Nt * h->L[1].M * es : 0);
      break;
    case ST_KERNEL_SHIFTED_RESIDUAL: bytes = D * 3 * es + (rx ? planes * es : 0); break;
    case ST_KERNEL_INNER_RESTRICT: {
      const double Dc = (double)L0.in[1].g.Ns * L0.Nt * h->p.M;
      bytes = D * es + 2 * Dc * es + (rx ? (double)L0.in[1].g.Ns * L0.Nt * es : 0);
      break;
    }
    case ST_KERNEL_PROLONG: {
      const double Dc = (double)L0.in[1].g.Ns * L0.Nt * h->p.M;
      bytes = 2 * D * es + Dc * es;
      break;
    }
    default: bytes = 0;
  }
  // the update runs on a zeroed e, so U + 0 * e == U whatever e held before
  if (which == ST_KERNEL_UPDATE) CK(cudaMemsetAsync(L0.e, 0, (size_t)h->D_total * h->esz, h->stream));
  if (which == ST_KERNEL_SWEEP2_UPDATE) {
    launch_set_uslot(h->Uslot, const_cast<double*>(U), h->stream);
    CKL();
  }
  TRY(one(h->stream));  // warm (and capture, for the cycle)
  if (which == ST_KERNEL_RESID_RESTRICT && (h->start_mask & 2u)) {
    // as in the cycle, the kernel also wrote level 1's smoothing start (y, z)
    bytes += 2.0 * (double)h->L[1].g.Ns * h->L[1].Nt * h->L[1].M * es;
  }
  h->start_mask = 0;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, h->stream));
  for (int i = 0; i < iters; ++i) {
    int s = one(h->stream);
    if (s != ST_OK) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return s;
    }
  }
  CK(cudaEventRecord(e1, h->stream));
  CK(cudaEventSynchronize(e1));
  h->start_mask = 0;  // set by the residual-restriction probe, consumed by no cycle
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ms_per_launch) *ms_per_launch = ms / iters;
  if (bytes_per_launch) *bytes_per_launch = bytes;
  return ST_OK;
}

int st_wait_selftest(st_handle* h) {
  if (!h) return ST_ERR_INVALID_ARG;
  if (!h->tma_err) return ST_ERR_UNSUPPORTED;
  const int s0 = read_scalars(h, 1);  // earlier expiries are not this call's
  if (s0 != ST_OK && s0 != ST_ERR_TIMEOUT) return s0;
  launch_wait_expiry(h->stream);
  CKL();
  return read_scalars(h, 1);
}

int st_stats(st_handle* h, st_stats_info* out) {
  PdlScope pdl_scope(h);
  if (!h || !out) return ST_ERR_INVALID_ARG;
  out->levels = (int)h->L.size();
  // the relinearise + cycle graph replaces both when it has been built; the
  // variants after a fine residual that did the first smoothing step (5, 6;
  // 7, 8 with the update) replace the plain ones (0, 3) when built
  const int gc = h->gexec[7] ? 7 : (h->gexec[5] ? 5 : 0), glc = h->gexec[8] ? 8 : (h->gexec[6] ? 6 : 3);
  out->update_in_cycle = h->last_update_in_cycle ? 1 : 0;
  out->cycle_graph_nodes = (int)(h->gexec[glc] ? h->gnodes[glc] : h->gnodes[gc]);
  out->linearize_graph_nodes = (int)(h->gexec[glc] ? 0 : h->gnodes[2]);
  const bool rx = h->p.reaction != ST_REACTION_NONE;
  // fine residual + partial sum + update, plus the graph(s) of one st_vcycle
  // (the linearise + cycle graph holds a few event nodes besides its kernels)
  if (rx && h->o.newton && h->gexec[glc])
    out->launches_per_vcycle = 3 + (int)h->gnodes[glc];
  else
    out->launches_per_vcycle = 3 + (int)h->gnodes[gc] + ((rx && h->o.newton) ? (int)h->gnodes[2] : 0);
  return ST_OK;
}

}  // extern "C"
