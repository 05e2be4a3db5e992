// Cycle-precision kernels of the space-time V-cycle (templated on T = float
// or double): the level operator residual with the Q-eigenbasis transform,
// the back-transform with damped block-Jacobi update, the spatial multigrid
// of the shifted slab systems, and the space / slab transfers (Eq. 4.1).
#include "st_kernels.cuh"

namespace st {

static inline unsigned nblk(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// ---------------------------------------------------------------------------
// Level residual  res = r - A_l e + C e   (transpose: r - A_l^T e + C^T e)
//   forward:   res_a = r_a - e_a + sum_b W[a][b] (nu Lap e_b + cbar e_b) + e_{n-1,M}
//   transpose: res_a = r_a - e_a + sum_b W[a][b] (nu Lap e_b + cbar e_b)
//                      + [a = M-1] sum_b e_{n+1,b}
// (W = dt_l Q or dt_l Q^T).  With transform = 1 the output is F * res.
// ---------------------------------------------------------------------------
template <int D, typename T>
__global__ void __launch_bounds__(256) k_lin_residual(LinParams<T> p) {
  const long long Ns = p.g.Ns;
  const int M = p.M;
  const long long nchunks = (p.Nt + p.chunk - 1) / p.chunk;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Ns * nchunks) return;
  const long long s = idx % Ns;
  const int c = (int)(idx / Ns);
  const int n0 = c * p.chunk;
  const int n1 = min(n0 + p.chunk, p.Nt);
  int i, j, k;
  decompose(s, p.g, i, j, k);
  const T ihx = (T)p.g.ih2[0], ihy = (T)p.g.ih2[1], ihz = (T)p.g.ih2[2];
  const bool hase = (p.e != nullptr);
  T carry = (T)0;
  if (hase) {
    if (!p.transpose) {
      if (n0 > 0) carry = p.e[((long long)(n0 - 1) * M + (M - 1)) * Ns + s];
    } else if (n1 < p.Nt) {
      for (int b = 0; b < M; ++b) carry += p.e[((long long)n1 * M + b) * Ns + s];
    }
  }
  for (int t = 0; t < n1 - n0; ++t) {
    const int n = p.transpose ? (n1 - 1 - t) : (n0 + t);
    T res[MAXM];
    const T cb = p.cbar ? p.cbar[(long long)n * Ns + s] : (T)0;
    if (hase) {
      T ev[MAXM], Fe[MAXM];
      T sum = (T)0;
#pragma unroll
      for (int b = 0; b < MAXM; ++b) {
        if (b < M) {
          const T* pl = p.e + ((long long)n * M + b) * Ns;
          const T eb = pl[s];
          ev[b] = eb;
          Fe[b] = p.nu * lap_at<D, T, T>(pl, s, i, j, k, p.g, eb, ihx, ihy, ihz) + cb * eb;
          sum += eb;
        }
      }
#pragma unroll
      for (int a = 0; a < MAXM; ++a) {
        if (a < M) {
          T acc = p.r[((long long)n * M + a) * Ns + s] - ev[a];
#pragma unroll
          for (int b = 0; b < MAXM; ++b)
            if (b < M) acc += p.W[a][b] * Fe[b];
          if (!p.transpose) acc += carry;
          else if (a == M - 1) acc += carry;
          res[a] = acc;
        }
      }
      carry = p.transpose ? sum : ev[M - 1];
    } else {
#pragma unroll
      for (int a = 0; a < MAXM; ++a)
        if (a < M) res[a] = p.r[((long long)n * M + a) * Ns + s];
    }
    if (p.transform) {
#pragma unroll
      for (int a = 0; a < MAXM; ++a) {
        if (a < M) {
          T acc = (T)0;
#pragma unroll
          for (int b = 0; b < MAXM; ++b)
            if (b < M) acc += p.F[a][b] * res[b];
          p.out[((long long)n * M + a) * Ns + s] = acc;
        }
      }
    } else {
#pragma unroll
      for (int a = 0; a < MAXM; ++a)
        if (a < M) p.out[((long long)n * M + a) * Ns + s] = res[a];
    }
  }
}

// e = (e_zero ? 0 : e) + omega * B z   (pointwise over the M planes)
template <typename T>
struct BackParams {
  long long Ns;
  int Nt, M, e_zero;
  T B[MAXM][MAXM];
  T omega;
  const T* z;
  T* e;
};

template <typename T>
__global__ void __launch_bounds__(256) k_backtransform(BackParams<T> p) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= p.Ns * p.Nt) return;
  const long long s = idx % p.Ns;
  const long long n = idx / p.Ns;
  const int M = p.M;
  T z[MAXM];
#pragma unroll
  for (int b = 0; b < MAXM; ++b)
    if (b < M) z[b] = p.z[(n * M + b) * p.Ns + s];
#pragma unroll
  for (int a = 0; a < MAXM; ++a) {
    if (a < M) {
      T acc = (T)0;
#pragma unroll
      for (int b = 0; b < MAXM; ++b)
        if (b < M) acc += p.B[a][b] * z[b];
      const long long o = (n * M + a) * p.Ns + s;
      p.e[o] = (p.e_zero ? (T)0 : p.e[o]) + p.omega * acc;
    }
  }
}

// ---------------------------------------------------------------------------
// Shifted slab operator (I - s (nu Lap + cbar)) on one group, and its
// diagonal.  For a complex group (zr, zi) with s = sr + i si:
//   out_r = zr - sr L'zr + si L'zi,  out_i = zi - sr L'zi - si L'zr,
// L' = nu Lap + cbar.
// ---------------------------------------------------------------------------

// Jacobi update for all groups at one point of one slab.
//   zero_init: z = omega D^{-1} y ; else zout = z + omega D^{-1} (y - A z)
template <int D, typename T, bool ZERO>
__device__ __forceinline__ void jacobi_point(const InnerParams<T>& p, long long s, int n, int i, int j,
                                             int k, T dlap) {
  const long long Ns = p.g.Ns;
  const T ihx = (T)p.g.ih2[0], ihy = (T)p.g.ih2[1], ihz = (T)p.g.ih2[2];
  const T cb = p.cbar ? p.cbar[(long long)n * Ns + s] : (T)0;
  const T dprime = p.nu * dlap + cb;  // diagonal of L'
  const long long base = (long long)n * p.P * Ns + s;
#pragma unroll
  for (int q = 0; q < MAXM; ++q) {
    if (q < p.sh.ngroups) {
      const int pl = p.sh.plane[q];
      const T sr = p.sh.sr[q], si = p.sh.si[q];
      if (!p.sh.cplx[q]) {
        const T dg = (T)1 - sr * dprime;
        const long long o = base + (long long)pl * Ns;
        if (ZERO) {
          p.zout[o] = p.omega * p.y[o] / dg;
        } else {
          const T* zp = p.z + (long long)(n * p.P + pl) * Ns;
          const T zc = zp[s];
          const T Lz = p.nu * lap_at<D, T, T>(zp, s, i, j, k, p.g, zc, ihx, ihy, ihz) + cb * zc;
          const T Az = zc - sr * Lz;
          p.zout[o] = zc + p.omega * (p.y[o] - Az) / dg;
        }
      } else {
        // D = (1 - sr d') - i si d';  1/D = conj(D)/|D|^2
        const T dr = (T)1 - sr * dprime, di = -si * dprime;
        const T inv = (T)1 / (dr * dr + di * di);
        const long long o_r = base + (long long)pl * Ns, o_i = o_r + Ns;
        T rr, ri;
        T zr = (T)0, zi = (T)0;
        if (ZERO) {
          rr = p.y[o_r];
          ri = p.y[o_i];
        } else {
          const T* zpr = p.z + (long long)(n * p.P + pl) * Ns;
          const T* zpi = zpr + Ns;
          zr = zpr[s];
          zi = zpi[s];
          const T Lr = p.nu * lap_at<D, T, T>(zpr, s, i, j, k, p.g, zr, ihx, ihy, ihz) + cb * zr;
          const T Li = p.nu * lap_at<D, T, T>(zpi, s, i, j, k, p.g, zi, ihx, ihy, ihz) + cb * zi;
          rr = p.y[o_r] - (zr - sr * Lr + si * Li);
          ri = p.y[o_i] - (zi - sr * Li - si * Lr);
        }
        // (rr + i ri) * (dr - i di) * inv
        const T qr = (rr * dr + ri * di) * inv;
        const T qi = (ri * dr - rr * di) * inv;
        p.zout[o_r] = zr + p.omega * qr;
        p.zout[o_i] = zi + p.omega * qi;
      }
    }
  }
}

template <int D, typename T, bool ZERO>
__global__ void __launch_bounds__(256) k_inner_jacobi(InnerParams<T> p) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= p.g.Ns * p.Nt) return;
  const long long s = idx % p.g.Ns;
  const int n = (int)(idx / p.g.Ns);
  int i, j, k;
  decompose(s, p.g, i, j, k);
  jacobi_point<D, T, ZERO>(p, s, n, i, j, k, (T)lap_diag<D>(p.g));
}

// Residual of the shifted systems at one fine point, all groups, into res[P].
template <int D, typename T>
__device__ __forceinline__ void shifted_residual(const InnerParams<T>& p, long long s, int n, T* res) {
  const long long Ns = p.g.Ns;
  int i, j, k;
  decompose(s, p.g, i, j, k);
  const T ihx = (T)p.g.ih2[0], ihy = (T)p.g.ih2[1], ihz = (T)p.g.ih2[2];
  const T cb = p.cbar ? p.cbar[(long long)n * Ns + s] : (T)0;
#pragma unroll
  for (int q = 0; q < MAXM; ++q) {
    if (q < p.sh.ngroups) {
      const int pl = p.sh.plane[q];
      const T sr = p.sh.sr[q], si = p.sh.si[q];
      const T* zr_p = p.z + (long long)(n * p.P + pl) * Ns;
      const T zr = zr_p[s];
      const T Lr = p.nu * lap_at<D, T, T>(zr_p, s, i, j, k, p.g, zr, ihx, ihy, ihz) + cb * zr;
      const long long o = (long long)(n * p.P + pl) * Ns + s;
      if (!p.sh.cplx[q]) {
        res[pl] = p.y[o] - (zr - sr * Lr);
      } else {
        const T* zi_p = zr_p + Ns;
        const T zi = zi_p[s];
        const T Li = p.nu * lap_at<D, T, T>(zi_p, s, i, j, k, p.g, zi, ihx, ihy, ihz) + cb * zi;
        res[pl] = p.y[o] - (zr - sr * Lr + si * Li);
        res[pl + 1] = p.y[o + Ns] - (zi - sr * Li - si * Lr);
      }
    }
  }
}

// Coarse rhs yc = full weighting of (y - A z); coarse start zc = omega Dc^{-1} yc.
template <int D, typename T>
__global__ void __launch_bounds__(256) k_inner_restrict(InnerParams<T> p) {
  const long long Nc = p.gc.Ns;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Nc * p.Nt) return;
  const long long sc = idx % Nc;
  const int n = (int)(idx / Nc);
  int I, J, K;
  decompose(sc, p.gc, I, J, K);
  int ix[3], iy[3], iz[3];
  float wx[3], wy[3], wz[3];
  restr_1d(I, p.g.n0, p.g.bc, ix, wx);
  int ny = 1, nz = 1;
  if (D >= 2) { restr_1d(J, p.g.n1, p.g.bc, iy, wy); ny = 3; } else { iy[0] = 0; wy[0] = 1.f; }
  if (D >= 3) { restr_1d(K, p.g.n2, p.g.bc, iz, wz); nz = 3; } else { iz[0] = 0; wz[0] = 1.f; }
  T acc[MAXM];
#pragma unroll
  for (int a = 0; a < MAXM; ++a) acc[a] = (T)0;
  for (int c = 0; c < nz; ++c)
    for (int b = 0; b < ny; ++b)
      for (int a = 0; a < 3; ++a) {
        const long long s = ((long long)iz[c] * p.g.n1 + iy[b]) * p.g.n0 + ix[a];
        const T w = (T)(wx[a] * wy[b] * wz[c]);
        T res[MAXM];
        shifted_residual<D, T>(p, s, n, res);
#pragma unroll
        for (int q = 0; q < MAXM; ++q)
          if (q < p.P) acc[q] += w * res[q];
      }
  // write yc and the zero-start Jacobi iterate zc
  const T cb = p.cbarc ? p.cbarc[(long long)n * Nc + sc] : (T)0;
  const T dprime = p.nu * (T)lap_diag<D>(p.gc) + cb;
  const long long base = (long long)n * p.P * Nc + sc;
#pragma unroll
  for (int q = 0; q < MAXM; ++q) {
    if (q < p.sh.ngroups) {
      const int pl = p.sh.plane[q];
      const T sr = p.sh.sr[q], si = p.sh.si[q];
      const long long o = base + (long long)pl * Nc;
      if (!p.sh.cplx[q]) {
        p.yc[o] = acc[pl];
        p.zc[o] = p.omega * acc[pl] / ((T)1 - sr * dprime);
      } else {
        const T dr = (T)1 - sr * dprime, di = -si * dprime;
        const T inv = (T)1 / (dr * dr + di * di);
        const T rr = acc[pl], ri = acc[pl + 1];
        p.yc[o] = rr;
        p.yc[o + Nc] = ri;
        p.zc[o] = p.omega * (rr * dr + ri * di) * inv;
        p.zc[o + Nc] = p.omega * (ri * dr - rr * di) * inv;
      }
    }
  }
}

// Coarsest inner grid: one block per slab runs `iters` Jacobi sweeps on all
// groups in shared memory, starting from z = 0.
template <int D, typename T>
__global__ void __launch_bounds__(256) k_inner_coarse(InnerParams<T> p) {
  extern __shared__ unsigned char smem_raw[];
  T* sz = reinterpret_cast<T*>(smem_raw);          // [P][Ns]
  T* sz2 = sz + (long long)p.P * p.g.Ns;          // [P][Ns]
  const long long Ns = p.g.Ns;
  const int n = blockIdx.x;
  for (long long t = threadIdx.x; t < p.P * Ns; t += blockDim.x) sz[t] = (T)0;
  __syncthreads();
  InnerParams<T> q = p;
  q.Nt = 1;
  q.cbar = p.cbar ? p.cbar + (long long)n * Ns : nullptr;
  q.y = p.y + (long long)n * p.P * Ns;
  const T dl = (T)lap_diag<D>(p.g);
  for (int it = 0; it < p.iters; ++it) {
    q.z = sz;
    q.zout = sz2;
    for (long long s = threadIdx.x; s < Ns; s += blockDim.x) {
      int i, j, k;
      decompose(s, p.g, i, j, k);
      jacobi_point<D, T, false>(q, s, 0, i, j, k, dl);
    }
    __syncthreads();
    T* tmp = sz;
    sz = sz2;
    sz2 = tmp;
  }
  for (long long t = threadIdx.x; t < p.P * Ns; t += blockDim.x) p.zout[(long long)n * p.P * Ns + t] = sz[t];
}

// ---------------------------------------------------------------------------
// Spatial transfers of [planes][Ns] fields.
// ---------------------------------------------------------------------------
template <int D, typename T>
__global__ void __launch_bounds__(256) k_restrict_space(GridP gf, GridP gc, long long planes,
                                                        const T* __restrict__ fine, T* __restrict__ coarse) {
  const long long Nc = gc.Ns;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Nc * planes) return;
  const long long sc = idx % Nc;
  const long long pl = idx / Nc;
  int I, J, K;
  decompose(sc, gc, I, J, K);
  int ix[3], iy[3], iz[3];
  float wx[3], wy[3], wz[3];
  restr_1d(I, gf.n0, gf.bc, ix, wx);
  int ny = 1, nz = 1;
  if (D >= 2) { restr_1d(J, gf.n1, gf.bc, iy, wy); ny = 3; } else { iy[0] = 0; wy[0] = 1.f; }
  if (D >= 3) { restr_1d(K, gf.n2, gf.bc, iz, wz); nz = 3; } else { iz[0] = 0; wz[0] = 1.f; }
  const T* f = fine + pl * gf.Ns;
  T acc = (T)0;
  for (int c = 0; c < nz; ++c)
    for (int b = 0; b < ny; ++b)
      for (int a = 0; a < 3; ++a)
        acc += (T)(wx[a] * wy[b] * wz[c]) * f[((long long)iz[c] * gf.n1 + iy[b]) * gf.n0 + ix[a]];
  coarse[idx] = acc;
}

template <int D, typename T>
__global__ void __launch_bounds__(256) k_prolong_space_add(GridP gf, GridP gc, long long planes,
                                                           const T* __restrict__ coarse, T* __restrict__ fine) {
  const long long Nf = gf.Ns;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Nf * planes) return;
  const long long s = idx % Nf;
  const long long pl = idx / Nf;
  int i, j, k;
  decompose(s, gf, i, j, k);
  int ix[2], iy[2], iz[2];
  float wx[2], wy[2], wz[2];
  const int cx = prol_1d(i, gc.n0, gf.bc, ix, wx);
  int cy = 1, cz = 1;
  if (D >= 2) cy = prol_1d(j, gc.n1, gf.bc, iy, wy); else { iy[0] = 0; wy[0] = 1.f; }
  if (D >= 3) cz = prol_1d(k, gc.n2, gf.bc, iz, wz); else { iz[0] = 0; wz[0] = 1.f; }
  const T* c = coarse + pl * gc.Ns;
  T acc = (T)0;
  for (int cc = 0; cc < cz; ++cc)
    for (int b = 0; b < cy; ++b)
      for (int a = 0; a < cx; ++a)
        acc += (T)(wx[a] * wy[b] * wz[cc]) * c[((long long)iz[cc] * gc.n1 + iy[b]) * gc.n0 + ix[a]];
  fine[idx] += acc;
}

// Slab bisection: coarse[N][m] = sum_k R[m][k] fine[2N + k/M][k%M]
template <typename T>
struct TimeXfer {
  T A[MAXM][2 * MAXM];  // restriction R (M x 2M)
  T B[2 * MAXM][MAXM];  // prolongation P (2M x M)
};

template <typename T>
__global__ void __launch_bounds__(256) k_restrict_time(long long Ns, int Ntc, int M, TimeXfer<T> X,
                                                       const T* __restrict__ fine, T* __restrict__ coarse) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Ns * Ntc) return;
  const long long s = idx % Ns;
  const long long N = idx / Ns;
  T f[2 * MAXM];
  for (int kk = 0; kk < 2 * M; ++kk) f[kk] = fine[((2 * N + kk / M) * M + (kk % M)) * Ns + s];
  for (int m = 0; m < M; ++m) {
    T acc = (T)0;
    for (int kk = 0; kk < 2 * M; ++kk) acc += X.A[m][kk] * f[kk];
    coarse[(N * M + m) * Ns + s] = acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_prolong_time_add(long long Ns, int Ntc, int M, TimeXfer<T> X,
                                                          const T* __restrict__ coarse, T* __restrict__ fine) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Ns * Ntc) return;
  const long long s = idx % Ns;
  const long long N = idx / Ns;
  T cv[MAXM];
  for (int m = 0; m < M; ++m) cv[m] = coarse[(N * M + m) * Ns + s];
  for (int kk = 0; kk < 2 * M; ++kk) {
    T acc = (T)0;
    for (int m = 0; m < M; ++m) acc += X.B[kk][m] * cv[m];
    fine[((2 * N + kk / M) * M + (kk % M)) * Ns + s] += acc;
  }
}

// cbar of two fine slabs averaged onto the coarse slab.
template <typename T>
__global__ void __launch_bounds__(256) k_cbar_time(long long Ns, int Ntc, const T* __restrict__ fine,
                                                   T* __restrict__ coarse) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Ns * Ntc) return;
  const long long s = idx % Ns;
  const long long N = idx / Ns;
  coarse[idx] = (T)0.5 * (fine[(2 * N) * Ns + s] + fine[(2 * N + 1) * Ns + s]);
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
  const long long nchunks = (p.Nt + p.chunk - 1) / p.chunk;
  const unsigned nb = nblk(p.g.Ns * nchunks, 256);
  DISPATCH_D(D, (k_lin_residual<DD, T><<<nb, 256, 0, st>>>(p)));
}

template <typename T>
void launch_backtransform(long long Ns, int Nt, int M, const T B[MAXM][MAXM], T omega, int e_zero,
                          const T* z, T* e, cudaStream_t st) {
  BackParams<T> p;
  p.Ns = Ns; p.Nt = Nt; p.M = M; p.e_zero = e_zero; p.omega = omega; p.z = z; p.e = e;
  for (int a = 0; a < MAXM; ++a)
    for (int b = 0; b < MAXM; ++b) p.B[a][b] = B[a][b];
  k_backtransform<T><<<nblk(Ns * Nt, 256), 256, 0, st>>>(p);
}

template <typename T>
void launch_inner_jacobi(int D, int zero, const InnerParams<T>& p, cudaStream_t st) {
  const unsigned nb = nblk(p.g.Ns * p.Nt, 256);
  if (zero) DISPATCH_D(D, (k_inner_jacobi<DD, T, true><<<nb, 256, 0, st>>>(p)));
  else DISPATCH_D(D, (k_inner_jacobi<DD, T, false><<<nb, 256, 0, st>>>(p)));
}

template <typename T>
void launch_inner_restrict(int D, const InnerParams<T>& p, cudaStream_t st) {
  const unsigned nb = nblk(p.gc.Ns * p.Nt, 256);
  DISPATCH_D(D, (k_inner_restrict<DD, T><<<nb, 256, 0, st>>>(p)));
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
  DISPATCH_D(D, (k_inner_coarse<DD, T><<<p.Nt, bs, sm, st>>>(p)));
}

template <typename T>
void launch_restrict_space(int D, const GridP& gf, const GridP& gc, long long planes, const T* f, T* c,
                           cudaStream_t st) {
  const unsigned nb = nblk(gc.Ns * planes, 256);
  DISPATCH_D(D, (k_restrict_space<DD, T><<<nb, 256, 0, st>>>(gf, gc, planes, f, c)));
}

template <typename T>
void launch_prolong_space_add(int D, const GridP& gf, const GridP& gc, long long planes, const T* c, T* f,
                              cudaStream_t st) {
  const unsigned nb = nblk(gf.Ns * planes, 256);
  DISPATCH_D(D, (k_prolong_space_add<DD, T><<<nb, 256, 0, st>>>(gf, gc, planes, c, f)));
}

template <typename T>
void launch_restrict_time(long long Ns, int Ntc, int M, const double R[MAXM][2 * MAXM], const T* f, T* c,
                          cudaStream_t st) {
  TimeXfer<T> X;
  for (int m = 0; m < MAXM; ++m)
    for (int kk = 0; kk < 2 * MAXM; ++kk) X.A[m][kk] = (T)R[m][kk];
  k_restrict_time<T><<<nblk(Ns * Ntc, 256), 256, 0, st>>>(Ns, Ntc, M, X, f, c);
}

template <typename T>
void launch_prolong_time_add(long long Ns, int Ntc, int M, const double P[2 * MAXM][MAXM], const T* c, T* f,
                             cudaStream_t st) {
  TimeXfer<T> X;
  for (int kk = 0; kk < 2 * MAXM; ++kk)
    for (int m = 0; m < MAXM; ++m) X.B[kk][m] = (T)P[kk][m];
  k_prolong_time_add<T><<<nblk(Ns * Ntc, 256), 256, 0, st>>>(Ns, Ntc, M, X, c, f);
}

template <typename T>
void launch_cbar_time(long long Ns, int Ntc, const T* f, T* c, cudaStream_t st) {
  k_cbar_time<T><<<nblk(Ns * Ntc, 256), 256, 0, st>>>(Ns, Ntc, f, c);
}

#define INST(T)                                                                                     \
  template void launch_lin_residual<T>(int, const LinParams<T>&, cudaStream_t);                    \
  template void launch_backtransform<T>(long long, int, int, const T[MAXM][MAXM], T, int, const T*, \
                                        T*, cudaStream_t);                                         \
  template void launch_inner_jacobi<T>(int, int, const InnerParams<T>&, cudaStream_t);             \
  template void launch_inner_restrict<T>(int, const InnerParams<T>&, cudaStream_t);                \
  template size_t inner_coarse_smem<T>(const InnerParams<T>&);                                     \
  template void launch_inner_coarse<T>(int, const InnerParams<T>&, cudaStream_t);                  \
  template void launch_restrict_space<T>(int, const GridP&, const GridP&, long long, const T*, T*, \
                                         cudaStream_t);                                            \
  template void launch_prolong_space_add<T>(int, const GridP&, const GridP&, long long, const T*,  \
                                            T*, cudaStream_t);                                     \
  template void launch_restrict_time<T>(long long, int, int, const double[MAXM][2 * MAXM], const T*, \
                                        T*, cudaStream_t);                                         \
  template void launch_prolong_time_add<T>(long long, int, int, const double[2 * MAXM][MAXM],      \
                                           const T*, T*, cudaStream_t);                            \
  template void launch_cbar_time<T>(long long, int, const T*, T*, cudaStream_t);

INST(float)
INST(double)

}  // namespace st
