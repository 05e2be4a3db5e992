// Launcher declarations of the CUDA kernels (one translation unit per group).
#pragma once

#include <algorithm>
#include <utility>

#include "st_internal.cuh"

namespace st {

// 1 (default): launches carry the programmatic-stream-serialisation attribute,
// which hides most of the launch latency of the many small kernels of a cycle;
// set per call from the handle's options.
extern thread_local int tl_pdl;
constexpr unsigned long long kPdlMaxBlocks = 152ull * 32;  // about 4 waves of 8 blocks per SM

// Kernel launch used by every launcher: the kernel's first instruction is
// grid_dep_wait(), so ordering against the previous launch on `st` holds with or
// without the attribute.  Errors surface through cudaGetLastError.
template <typename... KArgs, typename... Args>
inline void st_launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                      Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  // only launches of a few waves: their blocks' early residency hides the
  // launch latency, which is a large part of a short kernel; a grid of many
  // waves gains nothing from it, and its waiting blocks held SM slots while a
  // long predecessor drained (a V-cycle at 5.4e9 dofs ran 10 % slower with it)
  const unsigned long long nblk = (unsigned long long)grid.x * grid.y * grid.z;
  cfg.numAttrs = (tl_pdl && nblk <= kPdlMaxBlocks) ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// SDC node coefficients: qi[q] = dt*QI[m][q], qe[q] = dt*QE[m][q] for q < m.
struct SdcCoef {
  double qi[MAXM];
  double qe[MAXM];
};

// Coarsest-level data (one dense block per slab, K = M*Nc).
template <typename T>
struct CoarseParams {
  int Nt, M, Nc, K;
  double dtq[MAXM][MAXM];  // dt * Q of the coarsest level
  double nu;
  const double* Lc;        // dense Laplacian of the coarsest grid [Nc][Nc] (no nu)
  const T* cbar;           // [Nt][Nc] or null
  T* Ainv;                 // [Nt][K][K]
  T* Wf;                   // [Nt][K][Nc]   A^{-1} (1 (x) I)
  T* Wt;                   // [Nt][K][Nc]   A^{-T} (e_M (x) I)
  T* Wfrow;                // [Nt][Nc][Nc]  rows of Wf at node M
  T* Wtrow;                // [Nt][Nc][Nc]  sum over nodes of Wt
};

// Coefficients of a multi-axpy (at most 32 vectors).
struct KrylovCoef {
  int k;
  double c[32];
};

// k_tma.cu: the Jacobi sweep with TMA-staged tiles (2D periodic, x % 64, y % 16,
// M = 3 or 5, FP32); false when the shape does not qualify (nothing launched)
extern thread_local int tl_tma;
bool jacobi_tma_ok(int D, const InnerParams<float>& p);
bool launch_jacobi_tma(int D, const InnerParams<float>& p, cudaStream_t st);
// the level residual with e (forward, node-averaged cbar), same shapes
bool launch_linres_tma(int D, const LinParams<float>& p, cudaStream_t st);
// device address of the count of expired waits of the TMA-staged kernels
int* tma_error_flag();
// one block whose bounded mbarrier wait expires (nothing completes it); the
// expiry is counted like a staged kernel's
void launch_wait_expiry(cudaStream_t st);
// once per handle, outside any stream capture: the tensor-map encoder and the
// kernels' shared-memory limits and residency
void tma_prepare();

// k_krylov.cu
// number of doubles the partial-sum buffer of launch_mdot needs for n values
long long krylov_partials(long long n);
// out[i] = <w, V_i> for i < k (device doubles), V_i = V + i*stride
void launch_mdot(int fp64, const void* w, const void* V, long long stride, int k, long long n, double* partial,
                 double* out, cudaStream_t st);
// w -= sum_i c.c[i] V_i
void launch_maxpy(int fp64, void* w, const void* V, long long stride, const KrylovCoef& c, long long n,
                  cudaStream_t st);
// y = a x + b y
void launch_axpby(int fp64, void* y, const void* x, double a, double b, long long n, cudaStream_t st);

// k_fine.cu
long long residual_blocks(const ResidParams& p);
// blocks (= partial sums) the FP32-output residual launches for this problem
long long residual_ff_blocks(int D, const ResidParams& p);
long long gradient_blocks(const ResidParams& p);
void launch_residual(int D, int r_fp64, int c_fp64, const ResidParams& p, cudaStream_t st);
// double-float variant (float residual and cbar outputs); with ss it also
// writes the cycle's smoothing start where the tiled kernel applies
// (residual_start_ok) and ignores ss elsewhere
void launch_residual_ff(int D, const ResidParams& p, cudaStream_t st, const SmoothStart* ss = nullptr);
bool residual_start_ok(int D, const ResidParams& p, const SmoothStart* ss);
void launch_adj_residual(int D, int r_fp64, const ResidParams& p, cudaStream_t st);
void launch_gradients(int D, const ResidParams& p, double* partial2, double* du0, cudaStream_t st);
void launch_sum_partials(const double* part, long long n, double* out, cudaStream_t st);
// W += U - prev (the slab's initial value on every node): G(U) -> dt Q F(U) + tau
void launch_add_state(double* W, const double* U, const double* u0, long long Ns, int Nt, int M, cudaStream_t st);
// U += alpha * e (n values)
void launch_update(int fp64, double* U, const void* e, long long n, cudaStream_t st, double alpha = 1.0);
void launch_mass_weight(double* v, const GridP& g, long long planes, int inverse, cudaStream_t st);
void launch_sdc_rhs(int D, int fp64, const GridP& g, int Nt, int M, int m, double nu, int reaction,
                    double rho, const SdcCoef& cf, const void* G, const void* delta, const double* U,
                    void* y, cudaStream_t st);
void launch_scatter_plane(int fp64, const void* src, void* dst, long long Ns, int Nt, int M, int m,
                          cudaStream_t st);

// k_level.cu
template <typename T> void launch_lin_residual(int D, const LinParams<T>& p, cudaStream_t st);
template <typename T>
void launch_backtransform(const GridP& g, int Nt, int M, const T B[MAXM][MAXM], T omega, int e_zero,
                          const T* z, T* e, cudaStream_t st);
template <typename T> void launch_inner_jacobi(int D, int zero, const InnerParams<T>& p, cudaStream_t st);
// a whole forward smoothing step of a small level, one block per slab, planes
// in shared memory (k_level.cu); eout must not alias lp.e
void slab_smooth_prepare();
// k_sweep2.cu: the last two Jacobi sweeps of a depth-capped slab solve (the
// second fused with the back-transform and update of e, p.fuse_bt) as one
// kernel on 2D periodic grids in whole 64 x 8 tiles, M = 3 or 5; false where
// it does not apply.  p is the first sweep's parameter block (z in).
void sweep2_prepare();
// k_linres_restrict.cu: the forward level residual r - A e + C e (FP32,
// cbar, no exact Jacobian) fused with the full weighting onto gc (2D
// periodic, both axes halved, whole 64 x 16 fine tiles, M = 3 or 5) into
// coarse; false where it does not apply.  With ss (and the coarse level's
// cbar, or null without a reaction term) it also writes the first step of
// the coarse level's first smoothing into ss->y, ss->z (*started: whether it did).
void linres_restrict_prepare();
bool launch_linres_restrict(int D, const LinParams<float>& p, const GridP& gc, float* coarse, cudaStream_t st,
                            const SmoothStart* ss = nullptr, const float* cbarc = nullptr, bool* started = nullptr);
bool launch_sweep2(int D, const InnerParams<float>& p, cudaStream_t st);
// *slot = U on the stream (the address the two-sweep kernel's fused update reads)
void launch_set_uslot(double** slot, double* U, cudaStream_t st);
template <typename T> bool slab_smooth_fits(int M, long long Ns);
template <typename T>
void launch_slab_smooth(int D, const LinParams<T>& lp, const InnerParams<T>& ip, int sweeps, T* eout,
                        cudaStream_t st);
template <typename T> void launch_inner_restrict(int D, const InnerParams<T>& p, cudaStream_t st);
template <typename T> void launch_shifted_residual(int D, const InnerParams<T>& p, cudaStream_t st);
template <typename T> size_t inner_coarse_smem(const InnerParams<T>& p);
template <typename T> void launch_inner_coarse(int D, const InnerParams<T>& p, cudaStream_t st);
template <typename T>
void launch_restrict_space(int D, const GridP& gf, const GridP& gc, long long planes, const T* f, T* c,
                           cudaStream_t st);
template <typename T>
void launch_prolong_space_add(int D, const GridP& gf, const GridP& gc, long long planes, const T* c, T* f,
                              cudaStream_t st);
template <typename T>
void launch_restrict_time(const GridP& g, int Ntc, int M, const double R[MAXM][2 * MAXM], const T* f, T* c,
                          cudaStream_t st);
template <typename T>
void launch_prolong_time_add(const GridP& g, int Ntc, int M, const double P[2 * MAXM][MAXM], const T* c, T* f,
                             cudaStream_t st);
template <typename T> void launch_cbar_time(const GridP& g, int Ntc, const T* f, T* c, cudaStream_t st);
// out[n][a][s] (+)= sum_b X[a][b] in[n][b][s], X Mo x Mi (node-set transfer)
template <typename T>
void launch_node_transfer(long long Ns, int Nt, int Mi, int Mo, const double X[MAXM][MAXM], const T* in, T* out,
                          int add, cudaStream_t st);

// k_level4.cu: float4 variants (return false when they do not apply)
bool launch_lin_residual4(int D, const LinParams<float>& p, cudaStream_t st);
bool launch_inner4(int D, int mode, const InnerParams<float>& p, cudaStream_t st);  // 0 residual, 1 Jacobi
bool launch_prolong4(int D, const GridP& gf, const GridP& gc, long long planes, const float* c, float* f,
                     cudaStream_t st);
bool launch_restrict4(int D, const GridP& gf, const GridP& gc, long long planes, const float* f, float* c,
                      cudaStream_t st);
bool launch_inner_restrict4(int D, const InnerParams<float>& p, cudaStream_t st);

// k_coarse.cu
template <typename T> size_t coarse_setup_smem(const CoarseParams<T>& p);
template <typename T> cudaError_t prepare_coarse_setup(const CoarseParams<T>& p);
template <typename T> void launch_coarse_setup(const CoarseParams<T>& p, cudaStream_t st);
template <typename T>
void launch_coarse_solve(const CoarseParams<T>& p, int transpose, const T* r, T* e, T* in, cudaStream_t st);

}  // namespace st
