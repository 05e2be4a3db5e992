// Cycle-precision kernels of the space-time V-cycle (templated on T = float
// or double): the level operator residual with the Q-eigenbasis transform,
// the spatial multigrid of the shifted slab systems (with the back-transform
// and damped block-Jacobi update fused into its last sweep), a whole
// smoothing step of a small level in one launch (k_slab_smooth), and the
// space / slab transfers (Eq. 4.1).
//
// Indexing: one thread per (slab or slab chunk, point), flattened into a
// 32-bit index (the host guarantees Ns * slabs < 2^31); divisions by the grid
// sizes use precomputed multiply-shift constants.
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "st_kernels.cuh"

namespace st {

static inline unsigned nblk(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// One group's zero-start Jacobi value  omega D^{-1} y  (D = 1 - s d').
template <typename T>
__device__ __forceinline__ void zero_jacobi(T yr, T yi, int cplx, T sr, T si, T dprime, T omega, T& zr, T& zi) {
  if (!cplx) {
    zr = jdiv(omega * yr, (T)1 - sr * dprime);
    zi = (T)0;
  } else {
    const T dr = (T)1 - sr * dprime, di = -si * dprime;
    const T inv = jdiv(omega, dr * dr + di * di);
    zr = (yr * dr + yi * di) * inv;
    zi = (yi * dr - yr * di) * inv;
  }
}

// ---------------------------------------------------------------------------
// Level residual  res = r - A_l e + C e   (transpose: r - A_l^T e + C^T e)
//   forward:   res_a = r_a - e_a + sum_b W[a][b] (nu Lap e_b + cbar e_b) + e_{n-1,M}
//   transpose: res_a = r_a - e_a + sum_b W[a][b] (nu Lap e_b + cbar e_b)
//                      + [a = M-1] sum_b e_{n+1,b}
// (W = dt_l Q or dt_l Q^T).  With transform = 1 the output is F * res, and
// with zout set also the zero-start Jacobi iterate of the shifted systems.
// ---------------------------------------------------------------------------
template <int D, typename T>
__global__ void __launch_bounds__(256) k_lin_residual(LinParams<T> p) {
  grid_dep_wait();
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (unsigned)p.nchunks * (unsigned)p.g.Ns) return;
  int c, s, i, j, k;
  split_index(idx, p.g, c, s, i, j, k);
  const Nbr nb = make_nbr<D>(i, j, k, p.g);
  const long long Ns = p.g.Ns;
  const int M = p.M;
  const int n0 = c * p.chunk;
  const int n1 = min(n0 + p.chunk, p.Nt);
  const bool hase = (p.e != nullptr);
  T carry = (T)0;
  if (hase) {
    if (!p.transpose) {
      if (n0 > 0) carry = p.e[((long long)(n0 - 1) * M + (M - 1)) * Ns + s];
    } else if (n1 < p.Nt) {
      for (int b = 0; b < M; ++b) carry += p.e[((long long)n1 * M + b) * Ns + s];
    }
  }
  const T dlap = p.sc.k2;
  for (int t = 0; t < n1 - n0; ++t) {
    const int n = p.transpose ? (n1 - 1 - t) : (n0 + t);
    const long long base = (long long)n * M * Ns + s;
    T res[MAXM];
    const T cb = p.cbar ? p.cbar[(long long)n * Ns + s] : (T)0;
    if (hase) {
      T ev[MAXM], Fe[MAXM];
      T sum = (T)0, last = (T)0;
#pragma unroll
      for (int b = 0; b < MAXM; ++b) {
        if (b < M) {
          const T* pl = p.e + (long long)n * M * Ns + (long long)b * Ns;
          const T eb = pl[s];
          ev[b] = eb;
          const T cr = p.cnode ? p.cnode[base + (long long)b * Ns] : cb;
          Fe[b] = lap_nb<D, T, T>(pl, s, nb, eb, p.sc.cx, p.sc.cy, p.sc.cz, p.sc.k2, cr * eb);
          sum += eb;
          if (b == M - 1) last = eb;
        }
      }
#pragma unroll
      for (int a = 0; a < MAXM; ++a) {
        if (a < M) {
          T acc = (p.r ? p.r[base + (long long)a * Ns] : (T)0) - ev[a];
#pragma unroll
          for (int b = 0; b < MAXM; ++b)
            if (b < M) acc = fma(p.W[a][b], Fe[b], acc);
          if (!p.transpose || a == M - 1) acc += carry;
          res[a] = acc;
        }
      }
      carry = p.transpose ? sum : last;
    } else {
#pragma unroll
      for (int a = 0; a < MAXM; ++a)
        if (a < M) res[a] = p.r ? p.r[base + (long long)a * Ns] : (T)0;
    }
    if (p.transform) {
      T y[MAXM];
#pragma unroll
      for (int a = 0; a < MAXM; ++a) {
        if (a < M) {
          T acc = (T)0;
#pragma unroll
          for (int b = 0; b < MAXM; ++b)
            if (b < M) acc = fma(p.F[a][b], res[b], acc);
          y[a] = acc;
          p.out[base + (long long)a * Ns] = acc;
        }
      }
      if (p.zout) {
        const T dprime = dlap + cb;
#pragma unroll
        for (int pl = 0; pl < MAXM; ++pl) {
          const int kd = p.sh.kind[pl];
          if (kd == SH_REAL || kd == SH_RE) {
            T zr, zi;
            const T yi = (pl + 1 < MAXM && kd == SH_RE) ? y[pl + 1 < MAXM ? pl + 1 : pl] : (T)0;
            zero_jacobi<T>(y[pl], yi, kd == SH_RE, p.sh.sr[pl], p.sh.si[pl], dprime, p.omega_j, zr, zi);
            p.zout[base + (long long)pl * Ns] = zr;
            if (kd == SH_RE) p.zout[base + (long long)(pl + 1) * Ns] = zi;
          }
        }
      }
    } else {
#pragma unroll
      for (int a = 0; a < MAXM; ++a)
        if (a < M) p.out[base + (long long)a * Ns] = res[a];
    }
  }
}

// e = (e_zero ? 0 : e) + omega * B z   (pointwise over the M planes)
template <typename T>
struct BackParams {
  GridP g;
  int Nt, M, e_zero;
  T B[MAXM][MAXM];
  T omega;
  const T* z;
  T* e;
};

template <typename T>
__global__ void __launch_bounds__(256) k_backtransform(BackParams<T> p) {
  grid_dep_wait();
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (unsigned)p.Nt * (unsigned)p.g.Ns) return;
  const int n = (int)p.g.fNs.div(idx);
  const int s = (int)(idx - (unsigned)n * (unsigned)p.g.Ns);
  const long long Ns = p.g.Ns;
  const int M = p.M;
  const long long base = (long long)n * M * Ns + s;
  T z[MAXM];
#pragma unroll
  for (int b = 0; b < MAXM; ++b)
    if (b < M) z[b] = p.z[base + (long long)b * Ns];
#pragma unroll
  for (int a = 0; a < MAXM; ++a) {
    if (a < M) {
      T acc = (T)0;
#pragma unroll
      for (int b = 0; b < MAXM; ++b)
        if (b < M) acc = fma(p.B[a][b], z[b], acc);
      const long long o = base + (long long)a * Ns;
      p.e[o] = (p.e_zero ? (T)0 : p.e[o]) + p.omega * acc;
    }
  }
}

// ---------------------------------------------------------------------------
// Shifted slab operators (I - s (nu Lap + cbar)) on every group.  For a
// complex group (zr, zi) with s = sr + i si and L' = nu Lap + cbar:
//   out_r = zr - sr L'zr + si L'zi,   out_i = zi - sr L'zi - si L'zr.
// ---------------------------------------------------------------------------

// The Jacobi update at point s of one slab's shifted systems: zn = z + omega
// D^{-1} (y - A z), with zs / ys the slab's planes (plane pl at + pl * Ns)
// and cb the node-averaged reaction coefficient at s.
template <int D, typename T>
__device__ __forceinline__ void jacobi_core(const InnerParams<T>& p, const T* zs, const T* ys, long long Ns, int s,
                                            const Nbr& nb, T cb, T zn[MAXM]) {
  const T dprime = p.sc.k2 + cb;  // diagonal of L'
#pragma unroll
  for (int pl = 0; pl < MAXM; ++pl) {
    const int kd = p.sh.kind[pl];
    if (kd == SH_REAL || kd == SH_RE) {
      const T sr = p.sh.sr[pl], si = p.sh.si[pl];
      const T* zpr = zs + (long long)pl * Ns;
      const T zr = zpr[s];
      const T Lr = lap_nb<D, T, T>(zpr, s, nb, zr, p.sc.cx, p.sc.cy, p.sc.cz, p.sc.k2, cb * zr);
      const long long o = (long long)pl * Ns + s;
      if (kd == SH_REAL) {
        const T dg = (T)1 - sr * dprime;
        zn[pl] = zr + jdiv(p.omega * (ys[o] - (zr - sr * Lr)), dg);
      } else if (pl + 1 < MAXM) {
        const T* zpi = zpr + Ns;
        const T zi = zpi[s];
        const T Li = lap_nb<D, T, T>(zpi, s, nb, zi, p.sc.cx, p.sc.cy, p.sc.cz, p.sc.k2, cb * zi);
        const T rr = ys[o] - (zr - sr * Lr + si * Li);
        const T ri = ys[o + Ns] - (zi - sr * Li - si * Lr);
        const T dr = (T)1 - sr * dprime, di = -si * dprime;
        const T inv = jdiv(p.omega, dr * dr + di * di);
        zn[pl] = zr + (rr * dr + ri * di) * inv;
        zn[pl + 1 < MAXM ? pl + 1 : pl] = zi + (ri * dr - rr * di) * inv;
      }
    }
  }
}

// One Jacobi sweep at point s of slab n: zout = z + omega D^{-1} (y - A z);
// with fuse_bt the result is not stored but applied as
// e = (e_zero ? 0 : e) + omega_bt B zout.
template <int D, typename T>
__device__ __forceinline__ void jacobi_point(const InnerParams<T>& p, int s, int n, const Nbr& nb) {
  const long long Ns = p.g.Ns;
  const T cb = p.cbar ? p.cbar[(long long)n * Ns + s] : (T)0;
  const long long base = (long long)n * p.P * Ns + s;
  T zn[MAXM];
  jacobi_core<D, T>(p, p.z + (long long)n * p.P * Ns, p.y + (long long)n * p.P * Ns, Ns, s, nb, cb, zn);
  if (!p.fuse_bt) {
#pragma unroll
    for (int q = 0; q < MAXM; ++q)
      if (q < p.P) p.zout[base + (long long)q * Ns] = zn[q];
  } else {
#pragma unroll
    for (int a = 0; a < MAXM; ++a) {
      if (a < p.P) {
        T acc = (T)0;
#pragma unroll
        for (int b = 0; b < MAXM; ++b)
          if (b < p.P) acc = fma(p.B[a][b], zn[b], acc);
        const long long o = base + (long long)a * Ns;
        p.e[o] = (p.e_zero ? (T)0 : p.e[o]) + p.omega_bt * acc;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// A whole smoothing step of a small level in one launch, one block per slab
// (forward operator): the level residual r - A e + C e with the slab coupling
// (e = 0 when lp.e is null), its Q-eigenbasis transform y, the zero-start
// Jacobi iterate of the shifted systems, `sweeps - 1` more sweeps and the
// back-transform with the damped block-Jacobi update, e_out = e + omega_bt B z
// -- the work of the launches k_lin_residual, k_inner_jacobi make, on the
// slab's planes held in shared memory.  e_out is another buffer than lp.e:
// a block reads the previous slab's last node of lp.e while that slab's block
// may already be writing its update.
// ---------------------------------------------------------------------------
template <int D, typename T>
__global__ void __launch_bounds__(1024) k_slab_smooth(LinParams<T> lp, InnerParams<T> ip, int sweeps, T* eout) {
  grid_dep_wait();
  extern __shared__ __align__(16) unsigned char sraw[];
  const int n = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
  const int M = lp.M;
  const long long Ns = lp.g.Ns;
  T* E = reinterpret_cast<T*>(sraw);  // [M][Ns]
  T* Y = E + (long long)M * Ns;
  T* Z = Y + (long long)M * Ns;
  T* Z2 = Z + (long long)M * Ns;
  T* CB = Z2 + (long long)M * Ns;    // [Ns]
  const bool hase = lp.e != nullptr;
  const long long slab = (long long)n * M * Ns;
  for (int s = tid; s < Ns; s += nth) {
    CB[s] = lp.cbar ? lp.cbar[(long long)n * Ns + s] : (T)0;
    for (int b = 0; b < M; ++b) E[(long long)b * Ns + s] = hase ? lp.e[slab + (long long)b * Ns + s] : (T)0;
  }
  __syncthreads();
  for (int s = tid; s < Ns; s += nth) {
    int i, j, k;
    point_ijk(s, lp.g, i, j, k);
    const Nbr nb = make_nbr<D>(i, j, k, lp.g);
    const T cb = CB[s];
    T res[MAXM];
    if (hase) {
      const T carry = n > 0 ? lp.e[((long long)(n - 1) * M + (M - 1)) * Ns + s] : (T)0;
      T Fe[MAXM];
#pragma unroll
      for (int b = 0; b < MAXM; ++b)
        if (b < M) {
          const T* pl = E + (long long)b * Ns;
          const T eb = pl[s];
          Fe[b] = lap_nb<D, T, T>(pl, s, nb, eb, lp.sc.cx, lp.sc.cy, lp.sc.cz, lp.sc.k2, cb * eb);
        }
#pragma unroll
      for (int a = 0; a < MAXM; ++a)
        if (a < M) {
          T acc = lp.r[slab + (long long)a * Ns + s] - E[(long long)a * Ns + s];
#pragma unroll
          for (int b = 0; b < MAXM; ++b)
            if (b < M) acc = fma(lp.W[a][b], Fe[b], acc);
          res[a] = acc + carry;
        }
    } else {
#pragma unroll
      for (int a = 0; a < MAXM; ++a)
        if (a < M) res[a] = lp.r[slab + (long long)a * Ns + s];
    }
    T y[MAXM];
#pragma unroll
    for (int a = 0; a < MAXM; ++a)
      if (a < M) {
        T acc = (T)0;
#pragma unroll
        for (int b = 0; b < MAXM; ++b)
          if (b < M) acc = fma(lp.F[a][b], res[b], acc);
        y[a] = acc;
        Y[(long long)a * Ns + s] = acc;
      }
    const T dprime = lp.sc.k2 + cb;
#pragma unroll
    for (int pl = 0; pl < MAXM; ++pl) {
      const int kd = lp.sh.kind[pl];
      if (kd == SH_REAL || kd == SH_RE) {
        T zr, zi;
        const T yi = (pl + 1 < MAXM && kd == SH_RE) ? y[pl + 1 < MAXM ? pl + 1 : pl] : (T)0;
        zero_jacobi<T>(y[pl], yi, kd == SH_RE, lp.sh.sr[pl], lp.sh.si[pl], dprime, lp.omega_j, zr, zi);
        Z[(long long)pl * Ns + s] = zr;
        if (kd == SH_RE) Z[(long long)(pl + 1) * Ns + s] = zi;
      }
    }
  }
  __syncthreads();
  for (int it = 1; it <= sweeps; ++it) {
    const bool last = it == sweeps;
    for (int s = tid; s < Ns; s += nth) {
      T zn[MAXM];
      if (it == 1 && sweeps == 1) {
        // the zero-start iterate is the slab solve
#pragma unroll
        for (int q = 0; q < MAXM; ++q) zn[q] = q < M ? Z[(long long)q * Ns + s] : (T)0;
      } else if (it == 1) {
        continue;  // (the zero-start iterate is in Z)
      } else {
        int i, j, k;
        point_ijk(s, lp.g, i, j, k);
        jacobi_core<D, T>(ip, Z, Y, Ns, s, make_nbr<D>(i, j, k, lp.g), CB[s], zn);
      }
      if (!last) {
#pragma unroll
        for (int q = 0; q < MAXM; ++q)
          if (q < M) Z2[(long long)q * Ns + s] = zn[q];
      } else {
#pragma unroll
        for (int a = 0; a < MAXM; ++a)
          if (a < M) {
            T acc = (T)0;
#pragma unroll
            for (int b = 0; b < MAXM; ++b)
              if (b < M) acc = fma(ip.B[a][b], zn[b], acc);
            eout[slab + (long long)a * Ns + s] = E[(long long)a * Ns + s] + ip.omega_bt * acc;
          }
      }
    }
    __syncthreads();
    if (it > 1 && !last) {
      T* t = Z;
      Z = Z2;
      Z2 = t;
    }
  }
}

template <int D, typename T>
__global__ void __launch_bounds__(256) k_inner_jacobi(InnerParams<T> p) {
  grid_dep_wait();
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (unsigned)p.Nt * (unsigned)p.g.Ns) return;
  int n, s, i, j, k;
  split_index(idx, p.g, n, s, i, j, k);
  jacobi_point<D, T>(p, s, n, make_nbr<D>(i, j, k, p.g));
}

// Zero-start Jacobi z = omega D^{-1} y (pointwise).
template <typename T>
__global__ void __launch_bounds__(256) k_inner_jacobi_zero(InnerParams<T> p) {
  grid_dep_wait();
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (unsigned)p.Nt * (unsigned)p.g.Ns) return;
  const int n = (int)p.g.fNs.div(idx);
  const int s = (int)(idx - (unsigned)n * (unsigned)p.g.Ns);
  const long long Ns = p.g.Ns;
  const T cb = p.cbar ? p.cbar[(long long)n * Ns + s] : (T)0;
  const T dprime = p.sc.k2 + cb;
  const long long base = (long long)n * p.P * Ns + s;
#pragma unroll
  for (int pl = 0; pl < MAXM; ++pl) {
    const int kd = p.sh.kind[pl];
    if (kd == SH_REAL || kd == SH_RE) {
      const long long o = base + (long long)pl * Ns;
      T zr, zi;
      zero_jacobi<T>(p.y[o], kd == SH_RE ? p.y[o + Ns] : (T)0, kd == SH_RE, p.sh.sr[pl], p.sh.si[pl], dprime,
                     p.omega, zr, zi);
      p.zout[o] = zr;
      if (kd == SH_RE) p.zout[o + Ns] = zi;
    }
  }
}

// Residual y - A z of the shifted systems at every (slab, point), all planes,
// into zout.
template <int D, typename T>
__global__ void __launch_bounds__(256) k_shifted_residual(InnerParams<T> p) {
  grid_dep_wait();
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (unsigned)p.Nt * (unsigned)p.g.Ns) return;
  int n, s, i, j, k;
  split_index(idx, p.g, n, s, i, j, k);
  const Nbr nb = make_nbr<D>(i, j, k, p.g);
  const long long Ns = p.g.Ns;
  const T cb = p.cbar ? p.cbar[(long long)n * Ns + s] : (T)0;
#pragma unroll
  for (int pl = 0; pl < MAXM; ++pl) {
    const int kd = p.sh.kind[pl];
    if (kd == SH_REAL || kd == SH_RE) {
      const T sr = p.sh.sr[pl], si = p.sh.si[pl];
      const T* zr_p = p.z + (long long)(n * p.P + pl) * Ns;
      const T zr = zr_p[s];
      const T Lr = lap_nb<D, T, T>(zr_p, s, nb, zr, p.sc.cx, p.sc.cy, p.sc.cz, p.sc.k2, cb * zr);
      const long long o = (long long)(n * p.P + pl) * Ns + s;
      if (kd == SH_REAL) {
        p.zout[o] = p.y[o] - (zr - sr * Lr);
      } else if (pl + 1 < MAXM) {
        const T* zi_p = zr_p + Ns;
        const T zi = zi_p[s];
        const T Li = lap_nb<D, T, T>(zi_p, s, nb, zi, p.sc.cx, p.sc.cy, p.sc.cz, p.sc.k2, cb * zi);
        p.zout[o] = p.y[o] - (zr - sr * Lr + si * Li);
        p.zout[o + Ns] = p.y[o + Ns] - (zi - sr * Li - si * Lr);
      }
    }
  }
}

// Coarse rhs yc = full weighting of the fine residual res; coarse start
// zc = omega Dc^{-1} yc.
template <int D, typename T>
__global__ void __launch_bounds__(256) k_inner_restrict(InnerParams<T> p) {
  grid_dep_wait();
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (unsigned)p.Nt * (unsigned)p.gc.Ns) return;
  int n, sc, I, J, K;
  split_index(idx, p.gc, n, sc, I, J, K);
  const long long Nc = p.gc.Ns;
  const long long Ns = p.g.Ns;
  int ix[3], iy[3], iz[3];
  float wx[3], wy[3], wz[3];
  restr_1d(I, p.g.n0, p.g.bc, ix, wx);
  if (D >= 2) restr_1d(J, p.g.n1, p.g.bc, iy, wy);
  if (D >= 3) restr_1d(K, p.g.n2, p.g.bc, iz, wz);
  constexpr int NY = D >= 2 ? 3 : 1, NZ = D >= 3 ? 3 : 1;
  T acc[MAXM];
#pragma unroll
  for (int a = 0; a < MAXM; ++a) acc[a] = (T)0;
  const T* rb = p.res + (long long)n * p.P * Ns;
#pragma unroll
  for (int cc = 0; cc < NZ; ++cc)
#pragma unroll
    for (int b = 0; b < NY; ++b)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int zz = D >= 3 ? iz[cc] : 0, yy = D >= 2 ? iy[b] : 0;
        const T w = (T)(wx[a] * (D >= 2 ? wy[b] : 1.f) * (D >= 3 ? wz[cc] : 1.f));
        const long long s = ((long long)zz * p.g.n1 + yy) * p.g.n0 + ix[a];
#pragma unroll
        for (int q = 0; q < MAXM; ++q)
          if (q < p.P) acc[q] = fma(w, rb[(long long)q * Ns + s], acc[q]);
      }
  const T cb = p.cbarc ? p.cbarc[(long long)n * Nc + sc] : (T)0;
  const T dprime = p.k2c + cb;
  const long long base = (long long)n * p.P * Nc + sc;
#pragma unroll
  for (int pl = 0; pl < MAXM; ++pl) {
    const int kd = p.sh.kind[pl];
    if (kd == SH_REAL || kd == SH_RE) {
      const long long o = base + (long long)pl * Nc;
      const T ai = (kd == SH_RE) ? acc[pl + 1 < MAXM ? pl + 1 : pl] : (T)0;
      T zr, zi;
      zero_jacobi<T>(acc[pl], ai, kd == SH_RE, p.sh.sr[pl], p.sh.si[pl], dprime, p.omega, zr, zi);
      p.yc[o] = acc[pl];
      p.zc[o] = zr;
      if (kd == SH_RE) {
        p.yc[o + Nc] = ai;
        p.zc[o + Nc] = zi;
      }
    }
  }
}

// Coarsest inner grid: one block per slab runs `iters` Jacobi sweeps on all
// groups in shared memory, starting from z = 0; with fuse_bt the last sweep
// applies the back-transform update instead of storing z.
template <int D, typename T>
__global__ void __launch_bounds__(256) k_inner_coarse(InnerParams<T> p) {
  grid_dep_wait();
  extern __shared__ unsigned char smem_raw[];
  T* sz = reinterpret_cast<T*>(smem_raw);      // [P][Ns]
  T* sz2 = sz + (long long)p.P * p.g.Ns;      // [P][Ns]
  const int Ns = (int)p.g.Ns;
  const int n = blockIdx.x;
  for (int t = threadIdx.x; t < p.P * Ns; t += blockDim.x) sz[t] = (T)0;
  __syncthreads();
  InnerParams<T> q = p;
  q.Nt = 1;
  q.fuse_bt = 0;
  q.cbar = p.cbar ? p.cbar + (long long)n * Ns : nullptr;
  q.y = p.y + (long long)n * p.P * Ns;
  for (int it = 0; it < p.iters; ++it) {
    const bool last = (it == p.iters - 1);
    q.z = sz;
    q.zout = sz2;
    if (last && p.fuse_bt) {
      q.fuse_bt = 1;
      q.e = p.e + (long long)n * p.P * Ns;
    }
    for (int s = threadIdx.x; s < Ns; s += blockDim.x) {
      int i, j, k;
      point_ijk(s, p.g, i, j, k);
      jacobi_point<D, T>(q, s, 0, make_nbr<D>(i, j, k, p.g));
    }
    __syncthreads();
    T* tmp = sz;
    sz = sz2;
    sz2 = tmp;
  }
  if (!p.fuse_bt)
    for (int t = threadIdx.x; t < p.P * Ns; t += blockDim.x) p.zout[(long long)n * p.P * Ns + t] = sz[t];
}

// ---------------------------------------------------------------------------
// Spatial transfers of [planes][Ns] fields.
// ---------------------------------------------------------------------------
template <int D, typename T>
__global__ void __launch_bounds__(256) k_restrict_space(GridP gf, GridP gc, int planes,
                                                        const T* __restrict__ fine, T* __restrict__ coarse) {
  grid_dep_wait();
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (unsigned)planes * (unsigned)gc.Ns) return;
  int pl, sc, I, J, K;
  split_index(idx, gc, pl, sc, I, J, K);
  int ix[3], iy[3], iz[3];
  float wx[3], wy[3], wz[3];
  restr_1d(I, gf.n0, gf.bc, ix, wx);
  if (D >= 2) restr_1d(J, gf.n1, gf.bc, iy, wy);
  if (D >= 3) restr_1d(K, gf.n2, gf.bc, iz, wz);
  constexpr int NY = D >= 2 ? 3 : 1, NZ = D >= 3 ? 3 : 1;
  const T* f = fine + (long long)pl * gf.Ns;
  T acc = (T)0;
#pragma unroll
  for (int c = 0; c < NZ; ++c)
#pragma unroll
    for (int b = 0; b < NY; ++b)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int zz = D >= 3 ? iz[c] : 0, yy = D >= 2 ? iy[b] : 0;
        const float w3 = wx[a] * (D >= 2 ? wy[b] : 1.f) * (D >= 3 ? wz[c] : 1.f);
        acc = fma((T)w3, f[(zz * gf.n1 + yy) * gf.n0 + ix[a]], acc);
      }
  coarse[(long long)pl * gc.Ns + sc] = acc;
}

template <int D, typename T>
__global__ void __launch_bounds__(256) k_prolong_space_add(GridP gf, GridP gc, int planes,
                                                           const T* __restrict__ coarse, T* __restrict__ fine) {
  grid_dep_wait();
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (unsigned)planes * (unsigned)gf.Ns) return;
  int pl, s, i, j, k;
  split_index(idx, gf, pl, s, i, j, k);
  int ix[2], iy[2], iz[2];
  float wx[2], wy[2], wz[2];
  const int cx = prol_1d(i, gc.n0, gf.bc, ix, wx);
  int cy = 1, cz = 1;
  if (D >= 2) cy = prol_1d(j, gc.n1, gf.bc, iy, wy);
  if (D >= 3) cz = prol_1d(k, gc.n2, gf.bc, iz, wz);
  constexpr int NY = D >= 2 ? 2 : 1, NZ = D >= 3 ? 2 : 1;
  const T* c = coarse + (long long)pl * gc.Ns;
  T acc = (T)0;
#pragma unroll
  for (int cc = 0; cc < NZ; ++cc)
#pragma unroll
    for (int b = 0; b < NY; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        if (a < cx && (D < 2 || b < cy) && (D < 3 || cc < cz)) {
          const int zz = D >= 3 ? iz[cc] : 0, yy = D >= 2 ? iy[b] : 0;
          const float w3 = wx[a] * (D >= 2 ? wy[b] : 1.f) * (D >= 3 ? wz[cc] : 1.f);
          acc = fma((T)w3, c[(zz * gc.n1 + yy) * gc.n0 + ix[a]], acc);
        }
      }
  fine[(long long)pl * gf.Ns + s] += acc;
}

// Slab bisection: coarse[N][m] = sum_k R[m][k] fine[2N + k/M][k%M]
template <typename T>
struct TimeXfer {
  T A[MAXM][2 * MAXM];  // restriction R (M x 2M)
  T B[2 * MAXM][MAXM];  // prolongation P (2M x M)
};

template <typename T>
__global__ void __launch_bounds__(256) k_restrict_time(GridP g, int Ntc, int M, TimeXfer<T> X,
                                                       const T* __restrict__ fine, T* __restrict__ coarse) {
  grid_dep_wait();
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (unsigned)Ntc * (unsigned)g.Ns) return;
  const int N = (int)g.fNs.div(idx);
  const long long s = idx - (unsigned)N * (unsigned)g.Ns;
  const long long Ns = g.Ns;
  T f[2 * MAXM];
  for (int kk = 0; kk < 2 * M; ++kk) f[kk] = fine[((long long)(2 * N + kk / M) * M + (kk % M)) * Ns + s];
  for (int m = 0; m < M; ++m) {
    T acc = (T)0;
    for (int kk = 0; kk < 2 * M; ++kk) acc = fma(X.A[m][kk], f[kk], acc);
    coarse[((long long)N * M + m) * Ns + s] = acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_prolong_time_add(GridP g, int Ntc, int M, TimeXfer<T> X,
                                                          const T* __restrict__ coarse, T* __restrict__ fine) {
  grid_dep_wait();
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (unsigned)Ntc * (unsigned)g.Ns) return;
  const int N = (int)g.fNs.div(idx);
  const long long s = idx - (unsigned)N * (unsigned)g.Ns;
  const long long Ns = g.Ns;
  T cv[MAXM];
  for (int m = 0; m < M; ++m) cv[m] = coarse[((long long)N * M + m) * Ns + s];
  for (int kk = 0; kk < 2 * M; ++kk) {
    T acc = (T)0;
    for (int m = 0; m < M; ++m) acc = fma(X.B[kk][m], cv[m], acc);
    fine[((long long)(2 * N + kk / M) * M + (kk % M)) * Ns + s] += acc;
  }
}

// cbar of two fine slabs averaged onto the coarse slab.
template <typename T>
__global__ void __launch_bounds__(256) k_cbar_time(GridP g, int Ntc, const T* __restrict__ fine,
                                                   T* __restrict__ coarse) {
  grid_dep_wait();
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (unsigned)Ntc * (unsigned)g.Ns) return;
  const int N = (int)g.fNs.div(idx);
  const long long s = idx - (unsigned)N * (unsigned)g.Ns;
  coarse[idx] = (T)0.5 * (fine[(2LL * N) * g.Ns + s] + fine[(2LL * N + 1) * g.Ns + s]);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
#define DISPATCH_D(D, CALL) \
  do {                      \
    if ((D) == 1) { constexpr int DD = 1; CALL; } \
    else if ((D) == 2) { constexpr int DD = 2; CALL; } \
    else { constexpr int DD = 3; CALL; } \
  } while (0)

template <typename T>
void launch_lin_residual(int D, const LinParams<T>& p, cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value) {
    if (tl_tma && launch_linres_tma(D, p, st)) return;
    if (launch_lin_residual4(D, p, st)) return;
  }
  const unsigned nb = nblk((long long)p.g.Ns * p.nchunks, 256);
  DISPATCH_D(D, (st_launch(k_lin_residual<DD, T>, nb, 256, 0, st, p)));
}

template <typename T>
void launch_backtransform(const GridP& g, int Nt, int M, const T B[MAXM][MAXM], T omega, int e_zero, const T* z,
                          T* e, cudaStream_t st) {
  BackParams<T> p;
  p.g = g; p.Nt = Nt; p.M = M; p.e_zero = e_zero; p.omega = omega; p.z = z; p.e = e;
  for (int a = 0; a < MAXM; ++a)
    for (int b = 0; b < MAXM; ++b) p.B[a][b] = B[a][b];
  st_launch(k_backtransform<T>, nblk(g.Ns * Nt, 256), 256, 0, st, p);
}

template <typename T>
void launch_inner_jacobi(int D, int zero, const InnerParams<T>& p, cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value) {
    if (!zero && tl_tma && launch_jacobi_tma(D, p, st)) return;
    if (!zero && launch_inner4(D, 1, p, st)) return;
  }
  const unsigned nb = nblk(p.g.Ns * p.Nt, 256);
  if (zero) st_launch(k_inner_jacobi_zero<T>, nb, 256, 0, st, p);
  else DISPATCH_D(D, (st_launch(k_inner_jacobi<DD, T>, nb, 256, 0, st, p)));
}

// shared memory one slab-smoothing block may take (the opt-in is set once)
constexpr size_t kSlabSmoothSmem = 220 * 1024;
static int g_slab_smooth_ready = 0;

void slab_smooth_prepare() {
  static std::once_flag once;
  std::call_once(once, [] {
    bool ok = true;
    auto set = [&](auto kern) {
      ok = ok && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSlabSmoothSmem) ==
                     cudaSuccess;
    };
    set(k_slab_smooth<1, float>); set(k_slab_smooth<2, float>); set(k_slab_smooth<3, float>);
    set(k_slab_smooth<1, double>); set(k_slab_smooth<2, double>); set(k_slab_smooth<3, double>);
    g_slab_smooth_ready = ok ? 1 : 0;
    (void)cudaGetLastError();
  });
}

template <typename T>
size_t slab_smooth_smem(int M, long long Ns) {
  return (size_t)(4 * M + 1) * (size_t)Ns * sizeof(T);
}

template <typename T>
bool slab_smooth_fits(int M, long long Ns) {
  return g_slab_smooth_ready && slab_smooth_smem<T>(M, Ns) <= kSlabSmoothSmem;
}

template <typename T>
void launch_slab_smooth(int D, const LinParams<T>& lp, const InnerParams<T>& ip, int sweeps, T* eout,
                        cudaStream_t st) {
  const size_t smem = slab_smooth_smem<T>(lp.M, lp.g.Ns);
  const int threads = (int)std::min<long long>(1024, (lp.g.Ns + 31) / 32 * 32);
  DISPATCH_D(D, (st_launch(k_slab_smooth<DD, T>, (unsigned)lp.Nt, threads, smem, st, lp, ip, sweeps, eout)));
}

template <typename T>
void launch_inner_restrict(int D, const InnerParams<T>& p, cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value)
    if (launch_inner_restrict4(D, p, st)) return;
  const unsigned nb = nblk(p.gc.Ns * p.Nt, 256);
  DISPATCH_D(D, (st_launch(k_inner_restrict<DD, T>, nb, 256, 0, st, p)));
}

template <typename T>
void launch_shifted_residual(int D, const InnerParams<T>& p, cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value)
    if (launch_inner4(D, 0, p, st)) return;
  const unsigned nb = nblk(p.g.Ns * p.Nt, 256);
  DISPATCH_D(D, (st_launch(k_shifted_residual<DD, T>, nb, 256, 0, st, p)));
}

template <typename T>
size_t inner_coarse_smem(const InnerParams<T>& p) {
  return (size_t)2 * p.P * p.g.Ns * sizeof(T);
}

template <typename T>
void launch_inner_coarse(int D, const InnerParams<T>& p, cudaStream_t st) {
  const size_t sm = inner_coarse_smem(p);
  int bs = (int)((p.g.Ns + 31) / 32 * 32);
  if (bs > 256) bs = 256;
  DISPATCH_D(D, (st_launch(k_inner_coarse<DD, T>, p.Nt, bs, sm, st, p)));
}

template <typename T>
void launch_restrict_space(int D, const GridP& gf, const GridP& gc, long long planes, const T* f, T* c,
                           cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value)
    if (launch_restrict4(D, gf, gc, planes, f, c, st)) return;
  const unsigned nb = nblk(gc.Ns * planes, 256);
  DISPATCH_D(D, (st_launch(k_restrict_space<DD, T>, nb, 256, 0, st, gf, gc, (int)planes, f, c)));
}

template <typename T>
void launch_prolong_space_add(int D, const GridP& gf, const GridP& gc, long long planes, const T* c, T* f,
                              cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value)
    if (launch_prolong4(D, gf, gc, planes, c, f, st)) return;
  const unsigned nb = nblk(gf.Ns * planes, 256);
  DISPATCH_D(D, (st_launch(k_prolong_space_add<DD, T>, nb, 256, 0, st, gf, gc, (int)planes, c, f)));
}

template <typename T>
void launch_restrict_time(const GridP& g, int Ntc, int M, const double R[MAXM][2 * MAXM], const T* f, T* c,
                          cudaStream_t st) {
  TimeXfer<T> X;
  for (int m = 0; m < MAXM; ++m)
    for (int kk = 0; kk < 2 * MAXM; ++kk) X.A[m][kk] = (T)R[m][kk];
  st_launch(k_restrict_time<T>, nblk(g.Ns * Ntc, 256), 256, 0, st, g, Ntc, M, X, f, c);
}

template <typename T>
void launch_prolong_time_add(const GridP& g, int Ntc, int M, const double P[2 * MAXM][MAXM], const T* c, T* f,
                             cudaStream_t st) {
  TimeXfer<T> X;
  for (int kk = 0; kk < 2 * MAXM; ++kk)
    for (int m = 0; m < MAXM; ++m) X.B[kk][m] = (T)P[kk][m];
  st_launch(k_prolong_time_add<T>, nblk(g.Ns * Ntc, 256), 256, 0, st, g, Ntc, M, X, c, f);
}

template <typename T>
void launch_cbar_time(const GridP& g, int Ntc, const T* f, T* c, cudaStream_t st) {
  st_launch(k_cbar_time<T>, nblk(g.Ns * Ntc, 256), 256, 0, st, g, Ntc, f, c);
}

// Node-set transfer of every (slab, point): out[n][a][s] = sum_b X[a][b] in[n][b][s]
// (X: Mo x Mi), optionally added to out (M-coarsening of SMMG).
template <typename T>
struct NodeX {
  T x[MAXM][MAXM];
};

template <typename T>
__global__ void __launch_bounds__(256) k_node_transfer(long long Ns, int Nt, int Mi, int Mo, NodeX<T> X,
                                                       const T* __restrict__ in, T* __restrict__ out, int add) {
  grid_dep_wait();
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Ns * Nt) return;
  const long long n = idx / Ns, s = idx - n * Ns;
  T v[MAXM];
#pragma unroll
  for (int b = 0; b < MAXM; ++b) v[b] = (b < Mi) ? in[(n * Mi + b) * Ns + s] : (T)0;
#pragma unroll
  for (int a = 0; a < MAXM; ++a) {
    if (a < Mo) {
      T acc = add ? out[(n * Mo + a) * Ns + s] : (T)0;
#pragma unroll
      for (int b = 0; b < MAXM; ++b) acc = fma(X.x[a][b], v[b], acc);
      out[(n * Mo + a) * Ns + s] = acc;
    }
  }
}

template <typename T>
void launch_node_transfer(long long Ns, int Nt, int Mi, int Mo, const double X[MAXM][MAXM], const T* in, T* out,
                          int add, cudaStream_t st) {
  NodeX<T> x;
  for (int a = 0; a < MAXM; ++a)
    for (int b = 0; b < MAXM; ++b) x.x[a][b] = (a < Mo && b < Mi) ? (T)X[a][b] : (T)0;
  st_launch(k_node_transfer<T>, nblk(Ns * Nt, 256), 256, 0, st, Ns, Nt, Mi, Mo, x, in, out, add);
}

#define INST(T)                                                                                     \
  template void launch_lin_residual<T>(int, const LinParams<T>&, cudaStream_t);                    \
  template void launch_backtransform<T>(const GridP&, int, int, const T[MAXM][MAXM], T, int, const T*, \
                                        T*, cudaStream_t);                                         \
  template void launch_inner_jacobi<T>(int, int, const InnerParams<T>&, cudaStream_t);             \
  template void launch_inner_restrict<T>(int, const InnerParams<T>&, cudaStream_t);                \
  template void launch_shifted_residual<T>(int, const InnerParams<T>&, cudaStream_t);              \
  template size_t inner_coarse_smem<T>(const InnerParams<T>&);                                     \
  template void launch_inner_coarse<T>(int, const InnerParams<T>&, cudaStream_t);                  \
  template void launch_restrict_space<T>(int, const GridP&, const GridP&, long long, const T*, T*, \
                                         cudaStream_t);                                            \
  template void launch_prolong_space_add<T>(int, const GridP&, const GridP&, long long, const T*,  \
                                            T*, cudaStream_t);                                     \
  template void launch_restrict_time<T>(const GridP&, int, int, const double[MAXM][2 * MAXM],      \
                                        const T*, T*, cudaStream_t);                               \
  template void launch_prolong_time_add<T>(const GridP&, int, int, const double[2 * MAXM][MAXM],   \
                                           const T*, T*, cudaStream_t);                            \
  template void launch_cbar_time<T>(const GridP&, int, const T*, T*, cudaStream_t);                \
  template void launch_node_transfer<T>(long long, int, int, int, const double[MAXM][MAXM], const T*, T*, \
                                        int, cudaStream_t);                                        \
  template bool slab_smooth_fits<T>(int, long long);                                               \
  template void launch_slab_smooth<T>(int, const LinParams<T>&, const InnerParams<T>&, int, T*, cudaStream_t);

INST(float)
INST(double)

}  // namespace st
