/*
 * st.h - C ABI of the GB300 space-time multigrid / SDC library (libst.so).
 *
 * Problem (Benedusi, Minion, Krause, "An experimental comparison of a
 * space-time multigrid method with PFASST for a reaction-diffusion problem",
 * Sections 2-4): the reaction-diffusion equation u_t = nu*Delta u + R(u)
 * (Eq. 3.1 with nu and the reaction generalised) on a d-dimensional box,
 * second-order finite differences in space (the lumped P1 FEM of Section 3
 * for NEUMANN), right-Radau collocation in time on Nt slabs of M nodes
 * (Eq. 2.3; equivalently DG in time, Eq. 2.8-2.11).  All slabs are solved at
 * once: the unknown U is the space-time vector of Eq. (3.6),
 *
 *     U[n][m][z][y][x]   n < Nt (slab), m < M (Radau node), x fastest,
 *
 * stored as doubles, and the discrete system is, for every slab n,
 *
 *     G_n(U) = 1 (x) u_{n-1,M} + dt (Q (x) I) F(U_n) - U_n = 0,
 *     F(u) = nu*Delta_h u + R(u),  u_{-1,M} := u0,                      (*)
 *
 * the collocation form (2.3) chained through the slab coupling of Eq. (3.4).
 *
 * Grids (per axis, domain [0, X)): DIRICHLET n interior points, h = X/(n+1);
 * PERIODIC n points, h = X/n; NEUMANN n vertices, h = X/(n-1).
 *
 * Pointers.  Every double* argument named U, u0, u_target, gT, du0 or R may be
 * a device pointer (on the handle's device) or a host pointer; host data is
 * staged through library-owned device buffers inside the call.  The caller
 * owns all these arrays; the library never keeps a pointer across calls.
 * The st_level_* diagnostic calls take device pointers only.
 *
 * Streams.  All work is ordered on the stream given in st_runtime (0 = the
 * legacy default stream).  Calls that return a host value (a norm, a
 * gradient, an info struct) synchronise that stream once per iteration.
 *
 * Errors.  Every int-returning call returns an st_status.  No call aborts,
 * exits or traps; on a CUDA error the handle should be destroyed.
 */
#ifndef ST_H
#define ST_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ST_OK = 0,
  ST_ERR_INVALID_ARG = 1,   /* bad size, pointer or option */
  ST_ERR_OOM = 2,           /* the allocator returned NULL */
  ST_ERR_CUDA = 3,          /* a CUDA runtime error (see st_last_error) */
  ST_ERR_NOT_CONVERGED = 4, /* max_iters reached ("n.c." of Section 5.2) */
  ST_ERR_DIVERGED = 5,      /* non-finite or growing residual ("n.c.") */
  ST_ERR_TIMEOUT = 6,       /* a bounded device wait (TMA-staged kernels) expired */
  ST_ERR_UNSUPPORTED = 7    /* valid input the library does not handle */
} st_status;

enum { ST_BC_DIRICHLET = 0, ST_BC_PERIODIC = 1, ST_BC_NEUMANN = 2 };
/* R(u): NONE 0; LOGISTIC rho*u*(1-u); CUBIC rho*u*(1-u^2), which is the
 * paper's -gamma*(u^3 - u) of Eq. (3.1)/(3.7) with gamma = rho. */
enum { ST_REACTION_NONE = 0, ST_REACTION_LOGISTIC = 1, ST_REACTION_CUBIC = 2 };
/* FP64: every level in double.  FP32_REFINE: the multigrid cycle, smoother,
 * transfers and coarse solve in float inside an FP64 residual / update. */
enum { ST_PREC_FP64 = 0, ST_PREC_FP32_REFINE = 1 };
/* Level hierarchy of Eq. (4.1): SPACE = SMG (space bisection only, Section
 * 5.2); AUTO_MU = per level, bisect space if mu_l = nu*dt_l/h_l^2 >= mu_crit,
 * else bisect the slabs (the mu rule of Section 4.2). */
/* SPACE: space bisection only (the paper's SMG); AUTO_MU: space bisection while
 * mu_l = nu dt_l / h_l^2 >= mu_crit, slab bisection otherwise (STMG with the mu
 * rule); SPACE_NODES: space bisection with one collocation node fewer per
 * level until M = 1 (the paper's SMMG, Section 5.2); SPACE_TIME: space and
 * slab bisection on every level at once, M fixed (the paper's STMG, Section
 * 5.2), continuing in the one direction left once the other reaches its
 * coarse limit (coarse_max_points, coarse_max_slabs). */
enum { ST_COARSEN_SPACE = 0, ST_COARSEN_AUTO_MU = 1, ST_COARSEN_SPACE_NODES = 2, ST_COARSEN_SPACE_TIME = 3 };
/* SDC lower-triangular preconditioner: implicit Euler node to node, or the
 * LU trick (Q^T = L U, QI = U^T). */
enum { ST_SDC_IE = 0, ST_SDC_LU = 1 };

#define ST_MAX_M 5
#define ST_MAX_LEVELS 32
#define ST_MAX_HISTORY 64

typedef struct {
  int d;            /* 1, 2 or 3 */
  int n[3];         /* points per axis, n[0] = x (fastest); unused axes 1 */
  int bc;           /* ST_BC_* (same on every face) */
  double X;         /* domain length per axis */
  double nu;        /* diffusion coefficient (> 0) */
  int reaction;     /* ST_REACTION_* */
  double rho;       /* reaction rate */
  double T;         /* final time */
  int Nt;           /* slabs */
  int M;            /* right-Radau nodes per slab, 1..5 */
  const double* u0; /* initial value, n[0]*n[1]*n[2] doubles (host or device);
                       copied at st_create */
} st_problem;

typedef struct {
  int precision;        /* ST_PREC_*, default FP32_REFINE */
  int coarsening;       /* ST_COARSEN_*, default AUTO_MU */
  int max_levels;       /* default ST_MAX_LEVELS */
  int nu1, nu2;         /* pre/post smoothing steps, default 1, 1 */
  double omega;         /* block-Jacobi damping; <= 0: per level from mu_l
                           (1.0 if mu_l >= 16, 0.8 if mu_l >= mu_crit, else 0.5) */
  double mu_crit;       /* default 1.0 */
  int inner_cycles;     /* spatial multigrid cycles per slab solve, default 1 */
  int inner_smooth;     /* Jacobi sweeps per inner level and side, default 1 */
  int inner_coarse_iters; /* Jacobi sweeps on the coarsest inner grid, default 8 */
  int coarse_max_points;  /* stop space coarsening at <= this many points, default 16 */
  int coarse_max_slabs;   /* AUTO_MU: stop time coarsening at <= this many slabs, default 4 */
  int sdc_qdelta;       /* ST_SDC_*, default IE */
  int sdc_inner_cycles; /* spatial multigrid cycles per SDC node solve, default 2 */
  double tol;           /* relative residual ||G(U)|| / ||G(0)|| target, default 1e-8 */
  int max_iters;        /* default 1000 (Section 5.2) */
  int newton;           /* 1: relinearise (cbar from the current U) every
                           iteration; 0: keep the first linearisation */
  int use_graphs;       /* 1 (default): replay the cycle as a CUDA graph */
  int use_pdl;          /* 1 (default): programmatic dependent launch, so each
                           kernel is scheduled while its predecessor drains */
  int smooth_inner_levels; /* depth of the spatial multigrid inside the
                           block-Jacobi smoother's slab solves on levels above
                           the last space bisection: 1 (default) = Jacobi
                           sweeps on the level's own grid, 0 = the full
                           hierarchy (coarsened until non-stiff).  Levels below
                           the last space bisection and SDC node solves always
                           use the full hierarchy. */
  int smooth_sweeps;    /* Jacobi sweeps of a depth-capped smoother slab solve
                           (>= 2, default 3; the first is the zero-start one) */
  int line_search;      /* 1 (default): st_solve halves the step of a Newton
                           iteration (reaction != NONE) until ||G|| decreases
                           by the factor 1 - 1e-4 * step; DIVERGED below 2^-20 */
  int exact_jacobian;   /* 1: the finest level's linear operator uses R'(U) at
                           every node (the exact Jacobian of G; one more array
                           of the size of U), so a cycle that reduces the
                           linear residual gives a descent direction for
                           ||G||; the smoother and coarser levels keep the
                           node average.  0 (default): node average
                           everywhere (quasi-Newton; same rate per cycle on
                           the bench workloads, about 2.5 % less traffic). */
  int krylov;           /* 0 (default): one V-cycle per outer iteration.
                           m in 1..30: each st_solve iteration solves the
                           finest-level linear system by right-preconditioned
                           flexible GMRES with one V-cycle per Krylov step, at
                           most m steps (2m + 1 extra vectors of the size of U
                           in the cycle precision, allocated at first use);
                           use with exact_jacobian = 1 for a Newton method */
  double krylov_rtol;   /* GMRES stops when its residual estimate falls by
                           this factor (default 1e-2) */
  int krylov_fallback;  /* with krylov = 0: when the line search finds no
                           decrease along a cycle's correction, st_solve
                           continues with the exact Jacobian and FGMRES of
                           this many steps (default 10; 0 = report DIVERGED) */
  int pfasst_levels;    /* st_pfasst: levels of the hierarchy (default 3; the
                           handle must coarsen in space only, ST_COARSEN_SPACE) */
  int pfasst_coarse_M;  /* st_pfasst: nodes per slab on the levels above the
                           finest (default 1) */
  int pfasst_sweeps;    /* st_pfasst: SDC sweeps per level and visit (default 1) */
  int use_tma;          /* 1 (default): the Jacobi sweep that also updates e
                           (the last of a slab solve) on 2D periodic grids with
                           x % 64 == 0, y % 16 == 0 and M = 3 or 5 stages its
                           tiles through TMA copies (persistent, two stages); a
                           wait that expires makes the call report
                           ST_ERR_TIMEOUT.  0: direct float4 loads. */
  int recompute_slabs;  /* slab recomputation checkpointing (st_ckpt_*): slabs
                           per block, a divisor of Nt; 0 (default) = off.
                           st_create ignores it. */
  int fuse_sweeps;      /* 1 (default): the last two Jacobi sweeps of a slab
                           solve on 2D periodic grids in whole 64 x 8 tiles,
                           M = 3 or 5, FP32, run as one kernel with the middle
                           iterate in shared memory (same arithmetic); 0: two
                           launches */
  int fuse_start;       /* 1 (default): where the FP64-accurate fine residual
                           runs tiled (2D periodic, 64 x 16 tiles, M = 3 or 5)
                           and the cycle is FP32, it also writes the first
                           step of the cycle's first level-0 smoothing (from
                           e = 0: y = F r and the zero-start Jacobi iterate),
                           which the cycle then skips (same arithmetic); 0:
                           the cycle does that step itself */
  int fuse_restrict;    /* 1 (default): the forward level residual of the
                           coarse-grid correction and its full weighting onto
                           the next grid run as one kernel where both space
                           axes are halved (2D periodic, whole 64 x 16 fine
                           tiles, M = 3 or 5, FP32, cbar operator): the fine
                           residual stays in shared memory (same arithmetic);
                           0: two launches */
  int fuse_update;      /* 1 (default): in st_vcycle, where the smoothing
                           start applies, the last two-sweep kernel of the
                           cycle's level-0 post-smoothing also does the update
                           U += e (same arithmetic; U 16-byte aligned), and the
                           separate update launch is skipped; 0: the update
                           is its own launch.  st_solve keeps its own launch
                           (its line search reuses e). */
} st_solver_opts;

/* Device allocator hooks (e.g. a framework's caching allocator).  alloc must
 * return memory usable on `stream`, aligned to 256 bytes, or NULL.  With
 * alloc == NULL the library uses cudaMallocAsync / cudaFreeAsync. */
typedef void* (*st_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*st_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);
typedef struct {
  void* stream;     /* cudaStream_t; NULL = legacy default stream */
  st_alloc_fn alloc;
  st_free_fn free;
  void* ctx;
} st_runtime;

typedef struct {
  int iterations;          /* outer iterations performed */
  int status;              /* st_status of the call */
  double rel_residual;     /* final ||G(U)|| / ||G(0)|| (adjoint: / ||g||) */
  double abs_residual;     /* final ||G(U)||_2 */
  double ref_norm;         /* ||G(0)||_2 = sqrt(M) ||u0||_2 (adjoint: ||g||) */
  double seconds;          /* wall time of the call */
  int history_len;
  double history[ST_MAX_HISTORY]; /* relative residual per iteration */
  int cycles;              /* V-cycles applied (= iterations unless krylov > 0) */
} st_solve_info;

typedef struct {
  int n[3];
  long long Ns;       /* points per plane */
  int Nt;             /* slabs */
  double dt, h[3], mu;
  int next_kind;      /* 0 coarsest, 1 space bisection, 2 slab bisection,
                         3 space bisection and one node fewer, 4 space and
                         slab bisection */
  double omega;       /* damping used on this level */
  int inner_levels;   /* spatial multigrid depth of the slab solves */
  int M;              /* collocation nodes per slab on this level */
} st_level_info;

typedef struct {
  int levels;
  st_level_info level[ST_MAX_LEVELS];
  size_t workspace_bytes;   /* device bytes st_create allocates */
  int coarse_points;        /* points of the coarsest grid */
} st_plan_info;

typedef struct st_handle st_handle;

/* Fill *o with the defaults listed above. */
void st_default_opts(st_solver_opts* o);

/* Level hierarchy and workspace size for (p, o) without touching a GPU.
 * Errors: ST_ERR_INVALID_ARG for an invalid problem or options;
 * ST_ERR_UNSUPPORTED if the grid does not coarsen to a small coarsest grid. */
int st_plan(const st_problem* p, const st_solver_opts* o, st_plan_info* out);

/* Create a handle: collocation setup (right-Radau nodes, Q, eigen-
 * decomposition of Q; Section 2.1), level hierarchy, workspace allocation,
 * copy of u0.  o may be NULL (defaults), rt may be NULL (default stream,
 * cudaMallocAsync).  *out is NULL on failure. */
int st_create(const st_problem* p, const st_solver_opts* o, const st_runtime* rt,
              st_handle** out);

/* Release the workspace (stream-ordered) and the handle.  NULL is allowed. */
void st_destroy(st_handle* h);

/* Replace nu and rho (e.g. for finite differences or a new parameter point);
 * the next call relinearises. */
int st_set_params(st_handle* h, double nu, double rho);

/* Replace the initial value u0 (Ns doubles, host or device). */
int st_set_u0(st_handle* h, const double* u0);

/* Collocation residual (*) in FP64 at U (Eq. 2.3 on every slab, Eq. 3.4
 * coupling).  R receives G(U) in the handle's cycle precision (float for
 * FP32_REFINE, double for FP64) unless R_is_fp64 = 1 (always double); R may
 * be NULL.  norm_out (may be NULL) receives ||G(U)||_2 computed in FP64 with
 * a fixed reduction order. */
int st_residual(st_handle* h, const double* U, void* R, int R_is_fp64, double* norm_out);

/* One outer iteration: r = G(U) (FP64), linearise (cbar_n = mean_m R'(U_n,m)
 * on every level), one space-time V-cycle on A e - C e = r (damped block
 * Jacobi in time with Q-diagonalised spatial multigrid slab solves, space /
 * slab bisection transfers, exact forward substitution on the coarsest
 * level; Section 4.2), then U += e.  norm_out receives ||G(U)|| before the
 * update.  With a device U the call returns as soon as that norm is known:
 * the linearisation, the cycle and the update of U stay queued on the
 * handle's stream, so work queued on that stream afterwards (or following a
 * synchronisation of it) sees the updated U, and back-to-back calls keep the
 * device busy.  An expired wait of a TMA-staged kernel in that cycle is
 * reported (ST_ERR_TIMEOUT) by the next call that synchronises.  With a host
 * U the call returns after U has been copied back. */
int st_vcycle(st_handle* h, double* U, double* norm_out);

/* nsweeps IMEX SDC sweeps on all slabs at once (Section 4.1; reaction
 * explicit, diffusion implicit as in Section 5.4), in correction form on
 * top of the FP64 residual: slab n starts from the previous iterate's last
 * node of slab n-1.  norm_out receives ||G(U)|| before the last sweep. */
int st_sdc_sweep(st_handle* h, double* U, int nsweeps, double* norm_out);

/* PFASST (Section 4.1; Emmett and Minion 2012): iterate on U (Nt*M*Ns
 * doubles in the layout of st_solve, host or device; its content is the
 * start iterate, e.g. u0 spread over every node) until the collocation
 * residual ||G(U)|| / ||G(0)|| <= o.tol or o.max_iters iterations.  One
 * iteration: IMEX SDC sweeps on all slabs at once on each level from the
 * finest down (each slab starting from the last node of the slab before),
 * the restriction of the iterate with the FAS correction
 * tau_{l+1} = R(dt Q F(U_l) + tau_l) - dt Q F(R U_l), serial sweeps slab
 * after slab on the coarsest level, then the interpolated coarse corrections
 * back up with sweeps on the levels in between.  Level l is the handle's
 * l-th space-bisected level with o.pfasst_coarse_M nodes (l >= 1); transfers
 * are full weighting / linear interpolation in space and nodal-polynomial
 * evaluation between node sets; spatial solves use the level's inner
 * multigrid (o.sdc_inner_cycles cycles).  The state of the levels above the
 * finest is FP64; sweep corrections use the cycle precision.
 * Errors: ST_ERR_UNSUPPORTED unless the first o.pfasst_levels - 1 levels
 * bisect space only; otherwise as st_solve (info->history: residual per
 * iteration). */
int st_pfasst(st_handle* h, double* U, st_solve_info* info);

/* Solve G(U) = 0 from the given U (zero initial guess in the paper, Section
 * 5.2) by V-cycles inside FP64 defect correction (Newton with the averaged
 * reaction derivative for R != 0) until ||G(U)||/||G(0)|| <= tol.
 * Returns ST_ERR_NOT_CONVERGED / ST_ERR_DIVERGED with info filled. */
int st_solve(st_handle* h, double* U, st_solve_info* info);

/* Discrete adjoint at a converged U (not in the paper; derived from (*)).
 * Objective Phi = 1/2 h^d sum_x (u_{Nt,M} - u_target)^2.  Solves
 * J^T lambda = -dPhi/dU backward in time with the transposed V-cycle and
 * FP64 refinement, then returns dPhi/dnu, dPhi/drho (host doubles, may be
 * NULL) and dPhi/du0 (Ns doubles, host or device, may be NULL).
 * NEUMANN: the mirrored-ghost Delta_h is not symmetric; the solve uses
 * Delta_h^T = W Delta_h W^-1 (W the lumped mass weights of the vertex grid,
 * 1/2 per boundary axis) and solves for W^-1 lambda with the same kernels. */
int st_adjoint_solve(st_handle* h, const double* U, const double* u_target,
                     double* dnu, double* drho, double* du0, st_solve_info* info);

/* Same with an arbitrary terminal gradient gT = dPhi/du_{Nt,M} (Ns doubles). */
int st_adjoint_solve_terminal(st_handle* h, const double* U, const double* gT,
                              double* dnu, double* drho, double* du0,
                              st_solve_info* info);

/* Copy the adjoint state lambda of the last st_adjoint_solve* call (layout
 * of U, Nt*M*Ns doubles, host or device) into out.  ST_ERR_INVALID_ARG if no
 * adjoint solve has run on this handle. */
int st_adjoint_lambda(st_handle* h, double* out);

/* ---------------------------------------------------------------------
 * Slab recomputation checkpointing (not in the paper; the adjoint is
 * derived from (*)).  The system (*) is block lower bidiagonal in time, so
 * the slabs can be solved block after block, each block (K = recompute_slabs
 * slabs) taking as initial value the last node plane of the block before it;
 * J^T is block upper bidiagonal, so the adjoint runs block after block
 * backward, each block's terminal data being dPhi/d(initial value) of the
 * block after it (the du0 of that block's adjoint solve).  An st_ckpt keeps
 * only the initial planes of the Nt/K blocks and a K-slab workspace; the
 * adjoint pass recomputes each block's U from its initial plane.  Device
 * memory: a K-slab handle, K*M*Ns doubles for the block iterate and
 * (Nt/K + 2)*Ns doubles, instead of the Nt-slab handle and U.
 * ------------------------------------------------------------------- */
typedef struct st_ckpt st_ckpt;

/* Create: o->recompute_slabs = K >= 1 must divide p->Nt (else
 * ST_ERR_INVALID_ARG); the block handle is st_create of p with Nt = K and
 * T = K dt (same dt), so every option of o applies to the block solves. */
int st_ckpt_create(const st_problem* p, const st_solver_opts* o, const st_runtime* rt, st_ckpt** out);

/* Forward pass: solve the Nt slabs block after block (st_solve from the zero
 * guess on each block, to o->tol relative to the block's own ||G(0)||),
 * keeping each block's initial plane; uT (Ns doubles, host or device, may
 * be NULL) receives u_{Nt,M}.  info sums iterations and cycles over the
 * blocks and reports the largest block residual; the first block that fails
 * ends the pass with its status. */
int st_ckpt_forward(st_ckpt* c, double* uT, st_solve_info* info);

/* Adjoint pass after st_ckpt_forward: for the blocks from the last to the
 * first, recompute U of the block from its initial plane, then
 * st_adjoint_solve_terminal on the block with the terminal data gT (last
 * block) or the previous result's du0.  dnu, drho (host, may be NULL) sum
 * the blocks' contributions; du0 (Ns doubles, host or device, may be NULL)
 * is the first block's.  ST_ERR_INVALID_ARG without a forward pass since the
 * last st_ckpt_set_params / st_ckpt_set_u0. */
int st_ckpt_adjoint(st_ckpt* c, const double* gT, double* dnu, double* drho, double* du0,
                    st_solve_info* info);

/* Replace nu, rho / the initial value (Ns doubles, host or device); the next
 * st_ckpt_adjoint needs a new forward pass. */
int st_ckpt_set_params(st_ckpt* c, double nu, double rho);
int st_ckpt_set_u0(st_ckpt* c, const double* u0);

/* Release everything (stream-ordered); NULL is allowed. */
void st_ckpt_destroy(st_ckpt* c);

const char* st_status_str(int status);

/* Text of the last CUDA error seen by this thread ("" if none). */
const char* st_last_error(void);

/* ---------------------------------------------------------------------
 * Setup values and level-wise diagnostics (device pointers only).  They
 * expose the individual hot-path steps for testing against a reference.
 * Vectors at level l have Nt_l * M * Ns_l elements in the cycle precision
 * (float for FP32_REFINE, double for FP64).
 * ------------------------------------------------------------------- */

/* Right-Radau nodes tau[M] and Q[M*M] (row major) on the unit interval
 * (Section 2.1), eigenvalues lam[M] (re, im pairs: 2M doubles), eigenvector
 * matrix V and its inverse (row major, complex as re/im pairs: 2M*M doubles
 * each), ordered: real eigenvalues first, then each complex eigenvalue with
 * Im > 0 followed by its conjugate.  Any output may be NULL. */
int st_collocation(int M, double* tau, double* Q, double* lam, double* V, double* Vinv);

/* Time transfer matrices used for slab bisection: P_t (2M x M) and R_t
 * (M x 2M), row major (Eq. 4.1; the restriction acts through the DG form,
 * R_t = K^{-1} P_t^T blockdiag(K, K)). */
int st_time_transfer(int M, double* Pt, double* Rt);

/* M-coarsening transfers between the node sets of one slab (SMMG of Section
 * 5.2): P_M (Mf x Mc) evaluates the coarse nodal polynomial at the fine
 * nodes, R_M (Mc x Mf) = K_c^{-1} P_M^T K_f restricts collocation-form
 * residuals; row major.  ST_ERR_INVALID_ARG unless 1 <= Mc <= Mf <= 5. */
int st_node_transfer(int Mf, int Mc, double* P, double* R);

int st_num_levels(const st_handle* h);
int st_level_info_get(const st_handle* h, int level, st_level_info* out);

/* Linearise at U: cbar_0 = mean_m R'(U_{n,m}) and its restrictions to every
 * level, plus the coarsest-level factorisation. */
int st_linearize(st_handle* h, const double* U);

/* cbar of level l into out (Nt_l * Ns_l floats/doubles per precision). */
int st_level_cbar(st_handle* h, int level, void* out);

/* out = r - A_l e + C e at level l (transpose = 1: r - A_l^T e + C^T e). */
int st_level_residual(st_handle* h, int level, int transpose, const void* e,
                      const void* r, void* out);

/* One damped block-Jacobi-in-time smoothing step at level l, in place on e. */
int st_level_smooth(st_handle* h, int level, int transpose, void* e, const void* r);

/* coarse = restriction of fine (level l -> l+1). */
int st_level_restrict(st_handle* h, int level, int transpose, const void* fine, void* coarse);

/* fine += prolongation of coarse (level l+1 -> l). */
int st_level_prolong(st_handle* h, int level, int transpose, const void* coarse, void* fine);

/* Exact solve of A_L e - C e = r on the coarsest level (transpose = 1:
 * A_L^T e - C^T e = r, backward in time). */
int st_coarse_solve(st_handle* h, int transpose, const void* r, void* e);

/* One V-cycle on the linear level-0 problem A e - C e = r with zero start
 * (e overwritten). */
int st_level_vcycle(st_handle* h, int transpose, const void* r, void* e);

/* ---------------------------------------------------------------------
 * Measurement
 * ------------------------------------------------------------------- */

enum {
  ST_KERNEL_FINE_RESIDUAL = 0, /* FP64 residual G(U) -> cycle precision + cbar (+ the cycle's
                                  first smoothing step where fuse_start applies, as st_vcycle) */
  ST_KERNEL_LEVEL_RESIDUAL = 1,/* level-0 residual r - A e + C e with the Q-eigenbasis transform */
  ST_KERNEL_JACOBI = 2,        /* level-0 Jacobi sweep of the shifted slab systems fused with the
                                  back-transform and damped update of e (the cycle's last sweep) */
  ST_KERNEL_BACKTRANSFORM = 3, /* level-0 back-transform + damped block-Jacobi update */
  ST_KERNEL_VCYCLE = 4,        /* one whole V-cycle (graph replay), not a single kernel */
  ST_KERNEL_SHIFTED_RESIDUAL = 5, /* residual of the level-0 shifted slab systems */
  ST_KERNEL_INNER_RESTRICT = 6,   /* full weighting of that residual to the next inner grid */
  ST_KERNEL_PROLONG = 7,          /* linear interpolation + correction, inner grid 1 -> 0 */
  ST_KERNEL_JACOBI_PLAIN = 8,     /* level-0 Jacobi sweep of the shifted slab systems that only
                                     updates z (the sweeps before the cycle's last) */
  ST_KERNEL_UPDATE = 9,           /* the defect-correction update U += alpha e in FP64, run with
                                     alpha = 0: the update's traffic (U and e read, U written)
                                     with U's values left unchanged */
  ST_KERNEL_SWEEP2 = 10,          /* the last two level-0 Jacobi sweeps of a slab solve as one
                                     kernel, the second fused with the back-transform and update
                                     of e (ST_ERR_UNSUPPORTED where that kernel does not apply) */
  ST_KERNEL_RESID_RESTRICT = 11,  /* the level-0 residual r - A e + C e fused with its full
                                     weighting onto level 1 (ST_ERR_UNSUPPORTED where that kernel
                                     does not apply) */
  ST_KERNEL_SWEEP2_UPDATE = 12    /* ST_KERNEL_SWEEP2 as st_vcycle's last launch (fuse_update):
                                     its epilogue also adds e' to U and does not write e.  U
                                     (device) is modified: U += e' per launch (ST_ERR_UNSUPPORTED
                                     where that kernel does not apply) */
};

/* Launch kernel `which` `iters` times back to back on the handle's stream
 * between two CUDA events (after one untimed launch) and return the mean
 * duration per launch in milliseconds, plus the algorithmic bytes one launch
 * must move (each input read once, each output written once).  U (device,
 * Nt*M*Ns doubles) is the input of ST_KERNEL_FINE_RESIDUAL, the buffer
 * ST_KERNEL_UPDATE rewrites in place (with its own values) and the iterate
 * ST_KERNEL_SWEEP2_UPDATE adds its correction to; the other kernels
 * run on the handle's level-0 work buffers (contents unspecified). */
int st_time_kernel(st_handle* h, int which, const double* U, int iters, double* ms_per_launch,
                   double* bytes_per_launch);

/* Self-check of the bounded device waits: launches, on the handle's stream,
 * one block that waits on an mbarrier nothing will complete, with the limit
 * the TMA-staged kernels use (about a second).  The wait expires, the block
 * counts the expiry and returns, and the following synchronisation reports
 * it: the call returns ST_ERR_TIMEOUT when that chain works (and leaves the
 * handle usable, the expiry reported once), ST_ERR_CUDA on a CUDA error. */
int st_wait_selftest(st_handle* h);

typedef struct {
  int levels;
  int cycle_graph_nodes;        /* kernel + memset nodes of one V-cycle */
  int linearize_graph_nodes;    /* nodes of one relinearisation */
  int launches_per_vcycle;      /* all launches of one st_vcycle call */
  int update_in_cycle;          /* 1: the last st_vcycle's update of U ran inside
                                   its cycle (fuse_update), 0: as its own launch */
} st_stats_info;

/* Launch counts of the captured graphs (0 before the first st_vcycle). */
int st_stats(st_handle* h, st_stats_info* out);

/* ---------------------------------------------------------------------
 * Allocation-free residual norm (no counterpart in the paper: it exists for
 * callers that cannot allocate device memory where they need a residual
 * norm - code running under another framework's fixed-budget memory pool,
 * code called from inside an allocator callback, or a latency-critical loop
 * that must not pay cudaMalloc's implicit synchronisation).
 *
 * Computes G(U) of (*) in FP64 exactly like st_residual, without a handle
 * and without allocating: the per-block partial sums of the norm live in a
 * fixed file-scope device array of 2^18 + 1 doubles (2 MiB) that every GPU
 * loading the library keeps until process exit.
 *   p       problem; p->u0 must be a DEVICE pointer (Ns doubles)
 *   U       device, Nt*M*Ns doubles
 *   R       device, Nt*M*Ns doubles receiving G(U), or NULL
 *   norm_out host double receiving ||G(U)||_2, or NULL (then the call does
 *           not synchronise)
 *   stream  cudaStream_t (NULL = legacy default stream)
 * Every call looks up the array's device address in the current device's
 * context (the caller's device must be current).  Under lazy module loading
 * (the CUDA default) the first call on a device may load the library's
 * module, and that load allocates device memory for the module's code and
 * this array: make one warm-up call on each device at start-up, outside any
 * stream capture and outside any allocator callback or fixed-budget pool.
 * All calls share the one array and it keeps the last call's contents:
 * calls that overlap on the GPU (different streams or devices' host
 * threads racing on the same device) race on it - serialise them.
 * Errors: ST_ERR_INVALID_ARG for bad sizes or host pointers;
 * ST_ERR_UNSUPPORTED when a spatial plane has more than 2^26 points (the
 * partial sums would not fit) or Ns*Nt >= 2^31; ST_ERR_CUDA on a CUDA error.
 * Apart from that first module load, it calls no cudaMalloc, cudaFree or
 * other allocating routine. */
int st_residual_noalloc(const st_problem* p, const double* U, double* R, double* norm_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ST_H */
