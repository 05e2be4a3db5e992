// Internal declarations of the space-time multigrid library: kernel
// parameter blocks, stencil and transfer index helpers, launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/st.h"

#define MAXM ST_MAX_M

namespace st {

// Every kernel is launched with programmatic stream serialisation (see
// st_launch): its blocks may become resident while the previous kernel on the
// stream drains, so each kernel begins by waiting for that kernel's completion
// and memory flush, and then lets its own successor be scheduled.  Without the
// launch attribute both instructions are no-ops.
__device__ __forceinline__ void grid_dep_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

enum { BC_DIR = ST_BC_DIRICHLET, BC_PER = ST_BC_PERIODIC, BC_NEU = ST_BC_NEUMANN };

// Division of 0 <= n < 2^31 by a fixed divisor d with a multiply-high and a
// shift: with l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
// n / d = (umulhi(m, n) + n) >> l (Granlund and Montgomery, PLDI 1994).
struct FastDiv {
  unsigned d, m, l;
  __host__ __device__ FastDiv() : d(1), m(1), l(0) {}
  __host__ explicit FastDiv(unsigned dv) : d(dv ? dv : 1) {
    l = 0;
    while ((1ull << l) < d) ++l;
    m = (unsigned)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
  }
  __device__ __forceinline__ unsigned div(unsigned n) const { return (__umulhi(m, n) + n) >> l; }
};

// A spatial grid as the kernels see it (x fastest, unused axes have n = 1).
struct GridP {
  int n0, n1, n2;
  int bc;
  long long Ns;
  double ih2[3];  // 1/h^2 per axis (0 for unused axes)
  FastDiv f0, f1, fNs;  // division by n0, n1 and Ns
};

// True when p sits on a 16-byte boundary (float4 / double2 and TMA access; a
// null pointer counts as aligned).
inline bool aligned16(const void* p) { return ((unsigned long long)(size_t)p & 15ull) == 0; }

// Grid construction (host) ---------------------------------------------------

inline double spacing(int bc, int n, double X) {
  if (bc == BC_DIR) return X / (n + 1);
  if (bc == BC_PER) return X / n;
  return X / (n - 1);
}

inline GridP make_grid(int d, const int n[3], int bc, double X) {
  GridP g;
  g.n0 = n[0];
  g.n1 = d >= 2 ? n[1] : 1;
  g.n2 = d >= 3 ? n[2] : 1;
  g.bc = bc;
  g.Ns = (long long)g.n0 * g.n1 * g.n2;
  const int nn[3] = {g.n0, g.n1, g.n2};
  for (int a = 0; a < 3; ++a) {
    if (a < d) {
      const double h = spacing(bc, nn[a], X);
      g.ih2[a] = 1.0 / (h * h);
    } else {
      g.ih2[a] = 0.0;
    }
  }
  g.f0 = FastDiv((unsigned)g.n0);
  g.f1 = FastDiv((unsigned)g.n1);
  g.fNs = FastDiv((unsigned)(g.Ns < 0x7fffffffLL ? g.Ns : 0x7fffffffLL));
  return g;
}

// Index helpers --------------------------------------------------------------

__host__ __device__ inline void decompose(long long s, const GridP& g, int& i, int& j, int& k) {
  i = (int)(s % g.n0);
  long long r = s / g.n0;
  j = (int)(r % g.n1);
  k = (int)(r / g.n1);
}

// Flattened (block, point) index -> block number b, point s and its (i,j,k).
// idx < 2^31 is guaranteed by the host (Ns * slabs < 2^31).
__device__ __forceinline__ void split_index(unsigned idx, const GridP& g, int& b, int& s, int& i, int& j,
                                            int& k) {
  b = (int)g.fNs.div(idx);
  s = (int)(idx - (unsigned)b * (unsigned)g.Ns);
  const int r = (int)g.f0.div((unsigned)s);
  i = s - r * g.n0;
  k = (int)g.f1.div((unsigned)r);
  j = r - k * g.n1;
}

__device__ __forceinline__ void point_ijk(int s, const GridP& g, int& i, int& j, int& k) {
  const int r = (int)g.f0.div((unsigned)s);
  i = s - r * g.n0;
  k = (int)g.f1.div((unsigned)r);
  j = r - k * g.n1;
}

// Sum of the two neighbours of point s along one axis (index q of n, stride
// st) under the boundary rule: zero (DIRICHLET), wrap (PERIODIC), mirror
// (NEUMANN).
template <typename T, typename AT>
__device__ __forceinline__ AT nbr_sum(const T* __restrict__ p, long long s, int q, int n, long long st, int bc) {
  AT a, b;
  if (q > 0) a = (AT)p[s - st];
  else a = (bc == BC_PER) ? (AT)p[s + (long long)(n - 1) * st] : (bc == BC_NEU ? (AT)p[s + st] : (AT)0);
  if (q < n - 1) b = (AT)p[s + st];
  else b = (bc == BC_PER) ? (AT)p[s - (long long)(n - 1) * st] : (bc == BC_NEU ? (AT)p[s - st] : (AT)0);
  return a + b;
}

// Neighbour offsets of one point (relative to it) and a validity mask (a
// cleared bit is a zero DIRICHLET ghost), computed once per point and shared
// by all planes of a slab.
struct Nbr {
  long long o[6];
  unsigned mask;
};

template <int D>
__device__ __forceinline__ Nbr make_nbr(int i, int j, int k, const GridP& g) {
  Nbr nb;
  nb.mask = 0x3f;
  const int q[3] = {i, j, k};
  const int n[3] = {g.n0, g.n1, g.n2};
  const long long st[3] = {1, g.n0, (long long)g.n0 * g.n1};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a < D) {
      long long lo = -st[a], hi = st[a];
      if (q[a] == 0) {
        if (g.bc == BC_PER) lo = (long long)(n[a] - 1) * st[a];
        else if (g.bc == BC_NEU) lo = st[a];
        else { lo = 0; nb.mask &= ~(1u << (2 * a)); }
      }
      if (q[a] == n[a] - 1) {
        if (g.bc == BC_PER) hi = -(long long)(n[a] - 1) * st[a];
        else if (g.bc == BC_NEU) hi = -st[a];
        else { hi = 0; nb.mask &= ~(1u << (2 * a + 1)); }
      }
      nb.o[2 * a] = lo;
      nb.o[2 * a + 1] = hi;
    } else {
      nb.o[2 * a] = nb.o[2 * a + 1] = 0;
    }
  }
  return nb;
}

// nu * Lap u + acc from precomputed neighbours (c = nu/h^2 per axis,
// k2 = -2 (c_x + c_y + c_z)).
template <int D, typename T, typename AT>
__device__ __forceinline__ AT lap_nb(const T* __restrict__ p, long long s, const Nbr& nb, AT u, AT cx, AT cy,
                                     AT cz, AT k2, AT acc) {
  acc = fma(k2, u, acc);
  const AT c[3] = {cx, cy, cz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a < D) {
      AT lo = (AT)p[s + nb.o[2 * a]];
      AT hi = (AT)p[s + nb.o[2 * a + 1]];
      lo = (nb.mask & (1u << (2 * a))) ? lo : (AT)0;
      hi = (nb.mask & (1u << (2 * a + 1))) ? hi : (AT)0;
      acc = fma(c[a], lo + hi, acc);
    }
  }
  return acc;
}

// c_x (a+b)_x + c_y (a+b)_y + c_z (a+b)_z + k2 u with c = nu/h^2 per axis and
// k2 = -2 (c_x + c_y + c_z): nu * Lap u, accumulated onto acc.
template <int D, typename T, typename AT>
__device__ __forceinline__ AT lap_acc(const T* __restrict__ p, long long s, int i, int j, int k, const GridP& g,
                                      AT u, AT cx, AT cy, AT cz, AT k2, AT acc) {
  acc = fma(k2, u, acc);
  acc = fma(cx, nbr_sum<T, AT>(p, s, i, g.n0, 1, g.bc), acc);
  if (D >= 2) acc = fma(cy, nbr_sum<T, AT>(p, s, j, g.n1, g.n0, g.bc), acc);
  if (D >= 3) acc = fma(cz, nbr_sum<T, AT>(p, s, k, g.n2, (long long)g.n0 * g.n1, g.bc), acc);
  return acc;
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

// R(u) = rho u (1 - u) = u * (rho - rho u);  rho u (1 - u^2) = u * (rho - rho u u)
template <typename AT>
__device__ __forceinline__ AT react(int kind, AT rho, AT u) {
  if (kind == ST_REACTION_LOGISTIC) return u * fma(-rho, u, rho);
  if (kind == ST_REACTION_CUBIC) return u * fma(-rho * u, u, rho);
  return (AT)0;
}
// R'(u) = rho - 2 rho u;  rho - 3 rho u^2
template <typename AT>
__device__ __forceinline__ AT dreact(int kind, AT rho, AT u) {
  if (kind == ST_REACTION_LOGISTIC) return fma((AT)-2 * rho, u, rho);
  if (kind == ST_REACTION_CUBIC) return fma((AT)-3 * rho * u, u, rho);
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

// Stencil coefficients nu/h^2 per axis and the diagonal -2 sum of them.
template <typename AT>
struct StencilC {
  AT cx, cy, cz, k2;
};

// Fine FP64 residual (*) and its adjoint; also the SDC right-hand side.
// Quotient by the diagonal of a shifted slab system in the Jacobi updates:
// the fast reciprocal-based division in FP32 (error about 2 ulp; a damped
// Jacobi smoother needs the diagonal inverse only approximately, and every
// FP32 smoothing kernel uses this same form), the IEEE one in FP64.
template <typename T>
__device__ __forceinline__ T jdiv(T a, T b) {
  return a / b;
}
template <>
__device__ __forceinline__ float jdiv<float>(float a, float b) {
  return __fdividef(a, b);
}

// Damped Jacobi update of the shifted slab systems at one point in FP32,
// with every rounding spelt out (explicit FMAs and rounded products, so no
// kernel's contraction choices differ): the real system
//   z' = z + omega (y - (z - s L)) / (1 - s dg),
// and a complex pair s = sr + i si,
//   z' = z + omega conj(d) (y - (z - s L)) / |d|^2,  d = 1 - s dg,
// with L = (nu Lap + cbar) z at the point and dg = its diagonal coefficient.
// The sweep kernels that must agree to the bit (direct, TMA-staged, two
// sweeps in one) all use these.
__device__ __forceinline__ float jac_real(float y, float z, float L, float sr, float omega, float dg) {
  const float r = __fsub_rn(y, fmaf(-sr, L, z));
  return __fadd_rn(z, jdiv(__fmul_rn(omega, r), fmaf(-sr, dg, 1.f)));
}
__device__ __forceinline__ void jac_cplx(float yr, float yi, float zr, float zi, float Lr, float Li, float sr,
                                         float si, float omega, float dg, float& outr, float& outi) {
  const float rr = __fsub_rn(yr, fmaf(si, Li, fmaf(-sr, Lr, zr)));
  const float ri = __fsub_rn(yi, fmaf(-si, Lr, fmaf(-sr, Li, zi)));
  const float dr = fmaf(-sr, dg, 1.f), di = __fmul_rn(-si, dg);
  const float inv = jdiv(omega, fmaf(dr, dr, __fmul_rn(di, di)));
  outr = fmaf(fmaf(rr, dr, __fmul_rn(ri, di)), inv, zr);
  outi = fmaf(fmaf(ri, dr, __fmul_rn(-rr, di)), inv, zi);
}

// The zero-start damped Jacobi iterate z = omega D^-1 y of the shifted slab
// systems at one point (the first sweep from e = 0), roundings spelt out as
// in jac_real / jac_cplx: every kernel that forms it (the level residuals and
// the fine residual's smoothing start) gives the same bits.
__device__ __forceinline__ void jac_zero(float yr, float yi, bool cplx, float sr, float si, float dg, float omega,
                                         float& zr, float& zi) {
  if (!cplx) {
    zr = jdiv(__fmul_rn(omega, yr), fmaf(-sr, dg, 1.f));
    zi = 0.f;
  } else {
    const float dr = fmaf(-sr, dg, 1.f), di = __fmul_rn(-si, dg);
    const float inv = jdiv(omega, fmaf(dr, dr, __fmul_rn(di, di)));
    zr = __fmul_rn(fmaf(yr, dr, __fmul_rn(yi, di)), inv);
    zi = __fmul_rn(fmaf(yi, dr, __fmul_rn(-yr, di)), inv);
  }
}

struct ResidParams {
  GridP g;
  int Nt, M, chunk, nchunks;
  double dtq[MAXM][MAXM];  // dt*Q (forward) or dt*Q^T (adjoint: row = output node)
  double nu, rho;
  StencilC<double> sc;
  int reaction;
  const double* U;
  const double* u0;    // forward: slab coupling of the first slab
  const double* lam;   // adjoint: lambda
  const double* gT;    // adjoint: terminal gradient on node M of slab Nt (may be null)
  void* R;             // output residual (float or double, may be null)
  void* cbar;          // output mean_m R'(U) (may be null)
  void* cnode;         // output R'(U) at every node, layout of U (may be null)
  const double* tau;   // added to G (FAS correction of a coarse PFASST level; may be null;
                       // honoured by the FP64-arithmetic kernel only)
  double* partial;     // per-block sums of squares (may be null)
};

// Shifted slab systems of the Q-diagonalised solve, one entry per plane:
// kind[p] = SH_REAL (a real eigenvalue), SH_RE / SH_IM (real and imaginary
// part of a complex eigenvalue, planes p and p+1) or SH_NONE.  Plane p with
// kind SH_REAL or SH_RE solves (I - s (nu*Delta + cbar)) z = y with
// s = sr[p] + i si[p] = dt_l * lambda.
enum { SH_REAL = 0, SH_RE = 1, SH_IM = 2, SH_NONE = 3 };
template <typename T>
struct Shifts {
  int kind[MAXM];
  T sr[MAXM], si[MAXM];
};

// Optional second output of the FP32 fine residual: the first step of the
// cycle's first level-0 smoothing, which starts from e = 0 (so its level
// residual is r itself): the Q-eigenbasis transform y = F r per point and
// the zero-start Jacobi iterate z of the shifted slab systems, with the
// same arithmetic as the level-residual kernels.
struct SmoothStart {
  float* y;             // [Nt][M][Ns]
  float* z;             // [Nt][M][Ns]
  float F[MAXM][MAXM];  // forward transform to the Q eigenbasis
  Shifts<float> sh;
  float k2;             // diagonal coefficient of the level-0 stencil
  float omega;          // Jacobi weight
};

// Level operator A_l e - C e of the cycle (cycle precision T).
template <typename T>
struct LinParams {
  GridP g;
  int Nt, M, chunk, nchunks;
  int transpose;       // 0: forward operator, 1: A^T and C^T
  T W[MAXM][MAXM];     // dt_l*Q (forward) or dt_l*Q^T (transpose)
  StencilC<T> sc;
  const T* e;          // may be null (= 0)
  const T* r;          // may be null (= 0)
  const T* cbar;       // may be null (= 0)
  const T* cnode;      // forward only: R'(U) per node replacing cbar in A e (exact Jacobian; may be null)
  T* out;
  int transform;       // 1: out = F * res (per point, over the M nodes)
  T F[MAXM][MAXM];
  // optional zero-start Jacobi of the shifted slab systems on out (transform = 1)
  T* zout;
  Shifts<T> sh;
  T omega_j;
};

template <typename T>
struct InnerParams {
  GridP g;            // grid of this inner level
  GridP gc;           // next coarser grid (restriction)
  int Nt, P;          // slabs, planes per slab
  Shifts<T> sh;
  StencilC<T> sc;     // this grid
  T k2c;              // diagonal coefficient of the coarser grid
  T omega;            // Jacobi weight
  const T* cbar;      // [Nt][Ns] (may be null)
  const T* cbarc;     // coarse cbar (may be null)
  const T* y;
  const T* z;
  T* zout;
  const T* res;       // fine residual of the shifted systems (restriction input)
  T* yc;              // coarse rhs (restriction)
  T* zc;              // coarse start omega*D^-1*yc (restriction)
  int iters;          // coarse kernel sweeps
  // optional fused epilogue of a Jacobi sweep: e = (e_zero ? 0 : e) + omega_bt B z'
  int fuse_bt, e_zero;
  T B[MAXM][MAXM];
  T omega_bt;
  T* e;
  // two-sweep kernel only: with Uslot (device memory holding the FP64
  // iterate's address) the fused epilogue also adds e' to U; write_e = 0
  // then leaves e itself unwritten
  double* const* Uslot;
  int write_e;
};

}  // namespace st
