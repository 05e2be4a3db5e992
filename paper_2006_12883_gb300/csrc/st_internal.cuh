// Internal declarations of the space-time multigrid library: kernel
// parameter blocks, stencil and transfer index helpers, launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/st.h"

#define MAXM ST_MAX_M

namespace st {

enum { BC_DIR = ST_BC_DIRICHLET, BC_PER = ST_BC_PERIODIC, BC_NEU = ST_BC_NEUMANN };

// A spatial grid as the kernels see it (x fastest, unused axes have n = 1).
struct GridP {
  int n0, n1, n2;
  int bc;
  long long Ns;
  double ih2[3];  // 1/h^2 per axis (0 for unused axes)
};

// Index helpers --------------------------------------------------------------

__host__ __device__ inline void decompose(long long s, const GridP& g, int& i, int& j, int& k) {
  i = (int)(s % g.n0);
  long long r = s / g.n0;
  j = (int)(r % g.n1);
  k = (int)(r / g.n1);
}

// Laplacian (without the diffusion coefficient) of the plane p at point s,
// with the boundary rule of g.bc: zero ghosts (DIRICHLET), wrap-around
// (PERIODIC) or mirrored ghosts (NEUMANN).  c is p[s] already loaded.
template <int D, typename T, typename AT>
__device__ __forceinline__ AT lap_at(const T* __restrict__ p, long long s, int i, int j, int k,
                                     const GridP& g, AT c, AT ihx, AT ihy, AT ihz) {
  AT acc;
  {
    const int n = g.n0;
    AT a, b;
    if (i > 0) a = (AT)p[s - 1];
    else a = (g.bc == BC_PER) ? (AT)p[s + (n - 1)] : (g.bc == BC_NEU ? (AT)p[s + 1] : (AT)0);
    if (i < n - 1) b = (AT)p[s + 1];
    else b = (g.bc == BC_PER) ? (AT)p[s - (n - 1)] : (g.bc == BC_NEU ? (AT)p[s - 1] : (AT)0);
    acc = ihx * (a + b - (AT)2 * c);
  }
  if (D >= 2) {
    const int n = g.n1;
    const long long st = g.n0;
    AT a, b;
    if (j > 0) a = (AT)p[s - st];
    else a = (g.bc == BC_PER) ? (AT)p[s + (long long)(n - 1) * st] : (g.bc == BC_NEU ? (AT)p[s + st] : (AT)0);
    if (j < n - 1) b = (AT)p[s + st];
    else b = (g.bc == BC_PER) ? (AT)p[s - (long long)(n - 1) * st] : (g.bc == BC_NEU ? (AT)p[s - st] : (AT)0);
    acc += ihy * (a + b - (AT)2 * c);
  }
  if (D >= 3) {
    const int n = g.n2;
    const long long st = (long long)g.n0 * g.n1;
    AT a, b;
    if (k > 0) a = (AT)p[s - st];
    else a = (g.bc == BC_PER) ? (AT)p[s + (long long)(n - 1) * st] : (g.bc == BC_NEU ? (AT)p[s + st] : (AT)0);
    if (k < n - 1) b = (AT)p[s + st];
    else b = (g.bc == BC_PER) ? (AT)p[s - (long long)(n - 1) * st] : (g.bc == BC_NEU ? (AT)p[s - st] : (AT)0);
    acc += ihz * (a + b - (AT)2 * c);
  }
  return acc;
}

// Diagonal of the Laplacian stencil (as used by Jacobi): -2 sum_axes 1/h^2.
template <int D>
__host__ __device__ inline double lap_diag(const GridP& g) {
  double d = -2.0 * g.ih2[0];
  if (D >= 2) d += -2.0 * g.ih2[1];
  if (D >= 3) d += -2.0 * g.ih2[2];
  return d;
}

// Full weighting [1 2 1]/4 along one axis: the fine indices feeding coarse
// index I (fine size nf) and their weights.  Always three entries.
__device__ __forceinline__ void restr_1d(int I, int nf, int bc, int idx[3], float w[3]) {
  int c = (bc == BC_DIR) ? 2 * I + 1 : 2 * I;
  int a = c - 1, b = c + 1;
  if (bc == BC_PER) {
    if (a < 0) a += nf;
    if (b >= nf) b -= nf;
  } else if (bc == BC_NEU) {
    if (a < 0) a = 1;
    if (b >= nf) b = nf - 2;
  }
  idx[0] = a; idx[1] = c; idx[2] = b;
  w[0] = 0.25f; w[1] = 0.5f; w[2] = 0.25f;
}

// Linear interpolation along one axis: coarse indices (coarse size nc)
// contributing to fine index i and their weights; returns the count (1 or 2;
// a zero Dirichlet boundary value contributes nothing).
__device__ __forceinline__ int prol_1d(int i, int nc, int bc, int idx[2], float w[2]) {
  if (bc == BC_DIR) {
    if (i & 1) { idx[0] = (i - 1) >> 1; w[0] = 1.f; return 1; }
    int I = i >> 1;  // fine point between coarse I-1 and I
    int c = 0;
    if (I - 1 >= 0) { idx[c] = I - 1; w[c] = 0.5f; ++c; }
    if (I < nc) { idx[c] = I; w[c] = 0.5f; ++c; }
    return c;
  }
  if (!(i & 1)) { idx[0] = i >> 1; w[0] = 1.f; return 1; }
  int I = i >> 1;
  int J = I + 1;
  if (bc == BC_PER && J >= nc) J -= nc;
  idx[0] = I; w[0] = 0.5f;
  idx[1] = J; w[1] = 0.5f;
  return 2;
}

// Reaction terms -------------------------------------------------------------

template <typename AT>
__device__ __forceinline__ AT react(int kind, AT rho, AT u) {
  if (kind == ST_REACTION_LOGISTIC) return rho * u * ((AT)1 - u);
  if (kind == ST_REACTION_CUBIC) return rho * u * ((AT)1 - u * u);
  return (AT)0;
}
template <typename AT>
__device__ __forceinline__ AT dreact(int kind, AT rho, AT u) {
  if (kind == ST_REACTION_LOGISTIC) return rho * ((AT)1 - (AT)2 * u);
  if (kind == ST_REACTION_CUBIC) return rho * ((AT)1 - (AT)3 * u * u);
  return (AT)0;
}
template <typename AT>
__device__ __forceinline__ AT rshape(int kind, AT u) {
  if (kind == ST_REACTION_LOGISTIC) return u * ((AT)1 - u);
  if (kind == ST_REACTION_CUBIC) return u * ((AT)1 - u * u);
  return (AT)0;
}

// Deterministic block sum of a double (thread 0 gets the result).
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double ws[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) ws[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? ws[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Parameter blocks -----------------------------------------------------------

// Fine FP64 residual (*) and its adjoint; also the SDC right-hand side.
struct ResidParams {
  GridP g;
  int Nt, M, chunk;
  double dtq[MAXM][MAXM];  // dt*Q (forward) or dt*Q^T (adjoint: row = output node)
  double nu, rho;
  int reaction;
  const double* U;
  const double* u0;    // forward: slab coupling of the first slab
  const double* lam;   // adjoint: lambda
  const double* gT;    // adjoint: terminal gradient on node M of slab Nt (may be null)
  void* R;             // output residual (float or double, may be null)
  void* cbar;          // output mean_m R'(U) (may be null)
  double* partial;     // per-block sums of squares (may be null)
};

// Level operator A_l e - C e of the cycle (cycle precision T).
template <typename T>
struct LinParams {
  GridP g;
  int Nt, M, chunk;
  int transpose;       // 0: forward operator, 1: A^T and C^T
  T W[MAXM][MAXM];     // dt_l*Q (forward) or dt_l*Q^T (transpose)
  T nu;
  const T* e;          // may be null (= 0)
  const T* r;
  const T* cbar;       // may be null (= 0)
  T* out;
  int transform;       // 1: out = F * res (per point, over the M nodes)
  T F[MAXM][MAXM];
};

// Shift groups of the Q-diagonalised slab solve: group q occupies plane
// plane[q] (real) or planes plane[q], plane[q]+1 (re, im) and solves
// (I - s_q (nu*Delta + cbar)) z = y with s_q = dt_l * lambda_q.
template <typename T>
struct Shifts {
  int ngroups;
  int plane[MAXM];
  int cplx[MAXM];
  T sr[MAXM], si[MAXM];
};

template <typename T>
struct InnerParams {
  GridP g;            // grid of this inner level
  GridP gc;           // next coarser grid (restriction)
  int Nt, P;          // slabs, planes per slab
  Shifts<T> sh;
  T nu, omega;        // diffusion, Jacobi weight
  const T* cbar;      // [Nt][Ns] (may be null)
  const T* cbarc;     // coarse cbar (may be null)
  const T* y;
  const T* z;
  T* zout;
  T* yc;              // coarse rhs (restriction)
  T* zc;              // coarse initial guess (restriction) - set to omega*D^-1*yc
  int iters;          // coarse kernel sweeps
};

}  // namespace st
