// Four-points-per-thread (float4) variants of the largest FP32 cycle kernels:
// the level residual with the Q-eigenbasis transform, the residual of the
// shifted slab systems, the Jacobi sweep with the fused back-transform, and
// spatial prolongation.  A thread owns 4 consecutive x points of one row
// (x size a multiple of 4, so every float4 access is 16-byte aligned); the
// row neighbours (y, z) are float4 loads and the two x neighbours outside the
// group two scalar loads.  The node count M is a template parameter so the
// per-thread arrays are exactly sized.  The arithmetic per point is the same
// as in the one-point kernels of k_level.cu.
#include "st_kernels.cuh"

namespace st {

namespace {

__device__ __forceinline__ float4 ld4(const float* __restrict__ p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, const float v[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void to4(const float4 a, float v[4]) {
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}

// Neighbour offsets of the group of 4 points starting at x index i0 (relative
// to its first point): o[0] left of point 0, o[1] right of point 3, o[2..5]
// the y and z rows; cleared mask bits are zero (Dirichlet) ghosts.
template <int D>
__device__ __forceinline__ Nbr make_nbr4(int i0, int j, int k, const GridP& g) {
  Nbr nb = make_nbr<D>(i0, j, k, g);  // y, z and the left x neighbour
  long long hi = 4;
  if (i0 + 3 == g.n0 - 1) {
    if (g.bc == BC_PER) hi = 4 - g.n0;
    else if (g.bc == BC_NEU) hi = 2;
    else { hi = 3; nb.mask &= ~2u; }
  }
  nb.o[1] = hi;
  if (i0 != 0) nb.mask |= 1u;
  return nb;
}

// acc[q] += nu Lap at the 4 points (c = the group's own values).
template <int D>
__device__ __forceinline__ void lap4(const float* __restrict__ p, long long s0, const Nbr& nb, const float c[4],
                                     const StencilC<float>& sc, float acc[4]) {
  const float xl = (nb.mask & 1u) ? p[s0 + nb.o[0]] : 0.f;
  const float xr = (nb.mask & 2u) ? p[s0 + nb.o[1]] : 0.f;
  const float v[6] = {xl, c[0], c[1], c[2], c[3], xr};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    acc[q] = fmaf(sc.k2, c[q], acc[q]);
    acc[q] = fmaf(sc.cx, v[q] + v[q + 2], acc[q]);
  }
  if (D >= 2) {
    float lo[4] = {0.f, 0.f, 0.f, 0.f}, hi[4] = {0.f, 0.f, 0.f, 0.f};
    if (nb.mask & 4u) to4(ld4(p + s0 + nb.o[2]), lo);
    if (nb.mask & 8u) to4(ld4(p + s0 + nb.o[3]), hi);
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = fmaf(sc.cy, lo[q] + hi[q], acc[q]);
  }
  if (D >= 3) {
    float lo[4] = {0.f, 0.f, 0.f, 0.f}, hi[4] = {0.f, 0.f, 0.f, 0.f};
    if (nb.mask & 16u) to4(ld4(p + s0 + nb.o[4]), lo);
    if (nb.mask & 32u) to4(ld4(p + s0 + nb.o[5]), hi);
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = fmaf(sc.cz, lo[q] + hi[q], acc[q]);
  }
}

// flattened (block, group) index -> block b, first point s0 and its (i, j, k)
__device__ __forceinline__ void split4(unsigned idx, const GridP& g, const FastDiv& fG, int& b, int& s0, int& i0,
                                       int& j, int& k) {
  const unsigned G = (unsigned)(g.Ns >> 2);
  b = (int)fG.div(idx);
  s0 = (int)(idx - (unsigned)b * G) << 2;
  point_ijk(s0, g, i0, j, k);
}

__device__ __forceinline__ void zero_jacobi(float yr, float yi, bool cplx, float sr, float si, float dprime,
                                            float omega, float& zr, float& zi) {
  jac_zero(yr, yi, cplx, sr, si, dprime, omega, zr, zi);
}

}  // namespace

// ---------------------------------------------------------------------------
// One plane (the SDC node solves) fits 64 registers (8 blocks of 128 per SM);
// with every plane's z and y loaded up front, 2D instances take up to 128
// (4 blocks of 128: the loads in flight, not the warps, hide the latency);
// 3D instances keep their registers rather than spill.
template <int D, int M, int MODE>
constexpr int inner4_min_blocks() { return M == 1 ? 4 : (D == 2 ? 2 : 1); }

// With e (E = true) the level residual keeps M planes of e and r (all loaded
// up front) and their stencil sums live: at most 128 registers (2 blocks of
// 256 per SM).  Without e (the zero start of a pre-smoothing step) only r is
// read: M = 3 fits 64 registers (4 blocks), M = 5 85 (3 blocks).
template <int D, int M, bool E>
constexpr int lin4_min_blocks() { return E ? 2 : (M == 3 ? 4 : 3); }

template <int D, int M, bool E>
__global__ void __launch_bounds__(256, lin4_min_blocks<D, M, E>()) k_lin_residual4(LinParams<float> p, FastDiv fG) {
  grid_dep_wait();
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (unsigned)p.nchunks * (unsigned)(p.g.Ns >> 2)) return;
  int c, s0, i0, j, k;
  split4(idx, p.g, fG, c, s0, i0, j, k);
  const Nbr nb = make_nbr4<D>(i0, j, k, p.g);
  const long long Ns = p.g.Ns;
  const int n0 = c * p.chunk;
  const int n1 = min(n0 + p.chunk, p.Nt);
  constexpr bool hase = E;  // the launcher picks E = (p.e != nullptr)
  float carry[4] = {0.f, 0.f, 0.f, 0.f};
  if (hase) {
    if (!p.transpose) {
      if (n0 > 0) to4(ld4(p.e + ((long long)(n0 - 1) * M + (M - 1)) * Ns + s0), carry);
    } else if (n1 < p.Nt) {
#pragma unroll
      for (int b = 0; b < M; ++b) {
        float t[4];
        to4(ld4(p.e + ((long long)n1 * M + b) * Ns + s0), t);
#pragma unroll
        for (int q = 0; q < 4; ++q) carry[q] += t[q];
      }
    }
  }
  for (int t = 0; t < n1 - n0; ++t) {
    const int n = p.transpose ? (n1 - 1 - t) : (n0 + t);
    const long long base = (long long)n * M * Ns + s0;
    float cb[4] = {0.f, 0.f, 0.f, 0.f};
    if (p.cbar) to4(ld4(p.cbar + (long long)n * Ns + s0), cb);
    float res[M][4];
    if (hase) {
      float ev[M][4], Fe[M][4];
      float sum[4] = {0.f, 0.f, 0.f, 0.f};
      // every plane of e and r of this slab in flight before any arithmetic
      float4 r4v[M];
#pragma unroll
      for (int b = 0; b < M; ++b) {
        to4(ld4(p.e + base + (long long)b * Ns), ev[b]);
        r4v[b] = p.r ? ld4(p.r + base + (long long)b * Ns) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int b = 0; b < M; ++b) {
        const float* pl = p.e + base + (long long)b * Ns - s0;
        float cr[4] = {cb[0], cb[1], cb[2], cb[3]};
        if (p.cnode) to4(ld4(p.cnode + base + (long long)b * Ns), cr);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          Fe[b][q] = cr[q] * ev[b][q];
          sum[q] += ev[b][q];
        }
        lap4<D>(pl, s0, nb, ev[b], p.sc, Fe[b]);
      }
#pragma unroll
      for (int a = 0; a < M; ++a) {
        float r4[4];
        to4(r4v[a], r4);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float acc = r4[q] - ev[a][q];
#pragma unroll
          for (int b = 0; b < M; ++b) acc = fmaf(p.W[a][b], Fe[b][q], acc);
          if (!p.transpose || a == M - 1) acc += carry[q];
          res[a][q] = acc;
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) carry[q] = p.transpose ? sum[q] : ev[M - 1][q];
    } else {
#pragma unroll
      for (int a = 0; a < M; ++a) {
        if (p.r) to4(ld4(p.r + base + (long long)a * Ns), res[a]);
        else res[a][0] = res[a][1] = res[a][2] = res[a][3] = 0.f;
      }
    }
    if (p.transform) {
      float y[M][4];
#pragma unroll
      for (int a = 0; a < M; ++a) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float acc = 0.f;
#pragma unroll
          for (int b = 0; b < M; ++b) acc = fmaf(p.F[a][b], res[b][q], acc);
          y[a][q] = acc;
        }
        st4(p.out + base + (long long)a * Ns, y[a]);
      }
      if (p.zout) {
#pragma unroll
        for (int pl = 0; pl < M; ++pl) {
          const int kd = p.sh.kind[pl];
          if (kd == SH_REAL || kd == SH_RE) {
            float zr[4], zi[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
              zero_jacobi(y[pl][q], (kd == SH_RE && pl + 1 < M) ? y[pl + 1 < M ? pl + 1 : pl][q] : 0.f,
                          kd == SH_RE, p.sh.sr[pl], p.sh.si[pl], p.sc.k2 + cb[q], p.omega_j, zr[q], zi[q]);
            st4(p.zout + base + (long long)pl * Ns, zr);
            if (kd == SH_RE && pl + 1 < M) st4(p.zout + base + (long long)(pl + 1) * Ns, zi);
          }
        }
      }
    } else {
#pragma unroll
      for (int a = 0; a < M; ++a) st4(p.out + base + (long long)a * Ns, res[a]);
    }
  }
}

// Shifted-system operator at 4 points of all planes: out[pl][q] = y - A z
// (mode 0: residual into zout), a Jacobi sweep into zout (mode 1), or a
// Jacobi sweep fused with the back-transform and the damped update of e
// (mode 2, p.fuse_bt).

template <int D, int M, int MODE>
__global__ void __launch_bounds__(128, 2 * inner4_min_blocks<D, M, MODE>()) k_inner4(InnerParams<float> p, FastDiv fG) {
  grid_dep_wait();
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (unsigned)p.Nt * (unsigned)(p.g.Ns >> 2)) return;
  int n, s0, i0, j, k;
  split4(idx, p.g, fG, n, s0, i0, j, k);
  const Nbr nb = make_nbr4<D>(i0, j, k, p.g);
  const long long Ns = p.g.Ns;
  const long long base = (long long)n * M * Ns + s0;
  float cb[4] = {0.f, 0.f, 0.f, 0.f};
  if (p.cbar) to4(ld4(p.cbar + (long long)n * Ns + s0), cb);
  // every plane's z and y streamed in before any arithmetic: all of the
  // thread's DRAM loads in flight at once (the neighbour rows and columns
  // that follow mostly hit L2)
  float4 zv[M], yv[M];
#pragma unroll
  for (int pl = 0; pl < M; ++pl) {
    zv[pl] = ld4(p.z + base + (long long)pl * Ns);
    yv[pl] = ld4(p.y + base + (long long)pl * Ns);
  }
  // the sweep fused with the damped update of e (MODE 2) reads e too
  constexpr int ME = MODE == 2 ? M : 1;
  float4 ev0[ME];
  const bool pre_e = MODE == 2 && !p.e_zero;
#pragma unroll
  for (int a = 0; a < ME; ++a) ev0[a] = pre_e ? ld4(p.e + base + (long long)a * Ns) : make_float4(0.f, 0.f, 0.f, 0.f);
  float out[M][4];
#pragma unroll
  for (int pl = 0; pl < M; ++pl) {
    const int kd = p.sh.kind[pl];
    if (kd == SH_REAL || kd == SH_RE) {
      const float sr = p.sh.sr[pl], si = p.sh.si[pl];
      const float* zrp = p.z + base - s0 + (long long)pl * Ns;
      float zr[4], Lr[4], yr[4];
      to4(zv[pl], zr);
      to4(yv[pl], yr);
#pragma unroll
      for (int q = 0; q < 4; ++q) Lr[q] = cb[q] * zr[q];
      lap4<D>(zrp, s0, nb, zr, p.sc, Lr);
      if (kd == SH_REAL) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (MODE == 0) out[pl][q] = yr[q] - (zr[q] - sr * Lr[q]);
          else out[pl][q] = jac_real(yr[q], zr[q], Lr[q], sr, p.omega, p.sc.k2 + cb[q]);
        }
      } else if (pl + 1 < M) {
        const float* zip = zrp + Ns;
        float zi[4], Li[4], yi[4];
        to4(zv[pl + 1 < M ? pl + 1 : pl], zi);
        to4(yv[pl + 1 < M ? pl + 1 : pl], yi);
#pragma unroll
        for (int q = 0; q < 4; ++q) Li[q] = cb[q] * zi[q];
        lap4<D>(zip, s0, nb, zi, p.sc, Li);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (MODE == 0) {
            out[pl][q] = yr[q] - (zr[q] - sr * Lr[q] + si * Li[q]);
            out[pl + 1 < M ? pl + 1 : pl][q] = yi[q] - (zi[q] - sr * Li[q] - si * Lr[q]);
          } else {
            jac_cplx(yr[q], yi[q], zr[q], zi[q], Lr[q], Li[q], sr, si, p.omega, p.sc.k2 + cb[q], out[pl][q],
                     out[pl + 1 < M ? pl + 1 : pl][q]);
          }
        }
      }
    }
  }
  if (MODE != 2) {
#pragma unroll
    for (int pl = 0; pl < M; ++pl) st4(p.zout + base + (long long)pl * Ns, out[pl]);
  } else {
#pragma unroll
    for (int a = 0; a < M; ++a) {
      float ev[4];
      to4(ev0[a < ME ? a : 0], ev);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float acc = 0.f;
#pragma unroll
        for (int b = 0; b < M; ++b) acc = fmaf(p.B[a][b], out[b][q], acc);
        ev[q] = fmaf(p.omega_bt, acc, ev[q]);
      }
      st4(p.e + base + (long long)a * Ns, ev);
    }
  }
}

// Linear interpolation + correction on a periodic grid whose fine x size is
// a multiple of 4: fine x 4m..4m+3 take coarse x 2m, 2m+1, 2m+2 (wrapped).
template <int D>
__global__ void __launch_bounds__(256) k_prolong4(GridP gf, GridP gc, int planes, FastDiv fG,
                                                  const float* __restrict__ coarse, float* __restrict__ fine) {
  grid_dep_wait();
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (unsigned)planes * (unsigned)(gf.Ns >> 2)) return;
  int pl, s0, i0, j, k;
  split4(idx, gf, fG, pl, s0, i0, j, k);
  int iy[2], iz[2];
  float wy[2], wz[2];
  int cy = 1, cz = 1;
  if (D >= 2) cy = prol_1d(j, gc.n1, gf.bc, iy, wy);
  if (D >= 3) cz = prol_1d(k, gc.n2, gf.bc, iz, wz);
  const int I0 = i0 >> 1;
  const int I2 = (I0 + 2 >= gc.n0) ? I0 + 2 - gc.n0 : I0 + 2;
  const float* cp = coarse + (long long)pl * gc.Ns;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  constexpr int NY = D >= 2 ? 2 : 1, NZ = D >= 3 ? 2 : 1;
#pragma unroll
  for (int cc = 0; cc < NZ; ++cc)
#pragma unroll
    for (int b = 0; b < NY; ++b) {
      if ((D < 2 || b < cy) && (D < 3 || cc < cz)) {
        const int zz = D >= 3 ? iz[cc] : 0, yy = D >= 2 ? iy[b] : 0;
        const float w = (D >= 2 ? wy[b] : 1.f) * (D >= 3 ? wz[cc] : 1.f);
        const float* row = cp + ((long long)zz * gc.n1 + yy) * gc.n0;
        const float2 ab = *reinterpret_cast<const float2*>(row + I0);
        const float cnext = row[I2];
        acc[0] = fmaf(w, ab.x, acc[0]);
        acc[1] = fmaf(w, 0.5f * (ab.x + ab.y), acc[1]);
        acc[2] = fmaf(w, ab.y, acc[2]);
        acc[3] = fmaf(w, 0.5f * (ab.y + cnext), acc[3]);
      }
    }
  float* fp = fine + (long long)pl * gf.Ns + s0;
  float4 f = *reinterpret_cast<float4*>(fp);
  f.x += acc[0];
  f.y += acc[1];
  f.z += acc[2];
  f.w += acc[3];
  *reinterpret_cast<float4*>(fp) = f;
}

// Full weighting onto 4 consecutive coarse x points of one coarse row
// (periodic, coarse x size a multiple of 4): coarse I takes
// 1/4 f[2I-1] + 1/2 f[2I] + 1/4 f[2I+1]; the 9 fine values 8m-1 .. 8m+7 of a
// fine row are one scalar and two float4 loads.
__device__ __forceinline__ void restrict_row4(const float* __restrict__ row, int I0, int nf, float w, float acc[4]) {
  const int f0 = 2 * I0;
  const float l = row[f0 == 0 ? nf - 1 : f0 - 1];
  float a[4], b[4];
  to4(ld4(row + f0), a);
  to4(ld4(row + f0 + 4), b);
  const float v[9] = {l, a[0], a[1], a[2], a[3], b[0], b[1], b[2], b[3]};
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q] = fmaf(w, 0.25f * (v[2 * q] + v[2 * q + 2]) + 0.5f * v[2 * q + 1], acc[q]);
}

template <int D>
__device__ __forceinline__ void restrict4_point(const float* __restrict__ f, const GridP& gf, int I0, int J, int K,
                                                float acc[4]) {
  int iy[3], iz[3];
  float wy[3], wz[3];
  if (D >= 2) restr_1d(J, gf.n1, gf.bc, iy, wy);
  if (D >= 3) restr_1d(K, gf.n2, gf.bc, iz, wz);
  constexpr int NY = D >= 2 ? 3 : 1, NZ = D >= 3 ? 3 : 1;
#pragma unroll
  for (int c = 0; c < NZ; ++c)
#pragma unroll
    for (int b = 0; b < NY; ++b) {
      const int zz = D >= 3 ? iz[c] : 0, yy = D >= 2 ? iy[b] : 0;
      const float w = (D >= 2 ? wy[b] : 1.f) * (D >= 3 ? wz[c] : 1.f);
      restrict_row4(f + ((long long)zz * gf.n1 + yy) * gf.n0, I0, gf.n0, w, acc);
    }
}

// Outer restriction of [planes][Ns] fields.
template <int D>
__global__ void __launch_bounds__(256) k_restrict4(GridP gf, GridP gc, int planes, FastDiv fG,
                                                   const float* __restrict__ fine, float* __restrict__ coarse) {
  grid_dep_wait();
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (unsigned)planes * (unsigned)(gc.Ns >> 2)) return;
  int pl, s0, I0, J, K;
  split4(idx, gc, fG, pl, s0, I0, J, K);
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  restrict4_point<D>(fine + (long long)pl * gf.Ns, gf, I0, J, K, acc);
  st4(coarse + (long long)pl * gc.Ns + s0, acc);
}

// Inner restriction of the shifted-system residual (all planes of a slab)
// with the coarse zero-start Jacobi iterate.
template <int D, int M>
__global__ void __launch_bounds__(256) k_inner_restrict4(InnerParams<float> p, FastDiv fG) {
  grid_dep_wait();
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (unsigned)p.Nt * (unsigned)(p.gc.Ns >> 2)) return;
  int n, s0, I0, J, K;
  split4(idx, p.gc, fG, n, s0, I0, J, K);
  const long long Ns = p.g.Ns, Nc = p.gc.Ns;
  float acc[M][4];
#pragma unroll
  for (int q = 0; q < M; ++q) {
#pragma unroll
    for (int t = 0; t < 4; ++t) acc[q][t] = 0.f;
    restrict4_point<D>(p.res + ((long long)n * M + q) * Ns, p.g, I0, J, K, acc[q]);
  }
  float cb[4] = {0.f, 0.f, 0.f, 0.f};
  if (p.cbarc) to4(ld4(p.cbarc + (long long)n * Nc + s0), cb);
  const long long base = (long long)n * M * Nc + s0;
#pragma unroll
  for (int pl = 0; pl < M; ++pl) {
    const int kd = p.sh.kind[pl];
    if (kd == SH_REAL || kd == SH_RE) {
      float zr[4], zi[4];
#pragma unroll
      for (int t = 0; t < 4; ++t)
        zero_jacobi(acc[pl][t], (kd == SH_RE && pl + 1 < M) ? acc[pl + 1 < M ? pl + 1 : pl][t] : 0.f, kd == SH_RE,
                    p.sh.sr[pl], p.sh.si[pl], p.k2c + cb[t], p.omega, zr[t], zi[t]);
      st4(p.yc + base + (long long)pl * Nc, acc[pl]);
      st4(p.zc + base + (long long)pl * Nc, zr);
      if (kd == SH_RE && pl + 1 < M) {
        st4(p.yc + base + (long long)(pl + 1) * Nc, acc[pl + 1 < M ? pl + 1 : pl]);
        st4(p.zc + base + (long long)(pl + 1) * Nc, zi);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Dispatch: returns false when the 4-wide path does not apply.
// ---------------------------------------------------------------------------
static inline unsigned nblk4(long long n) { return (unsigned)((n + 255) / 256); }

bool vec4_ok(const GridP& g, int D, int M) {
  return D >= 2 && (M == 3 || M == 5) && g.n0 >= 4 && (g.n0 % 4) == 0 && g.bc == BC_PER;
}

bool launch_lin_residual4(int D, const LinParams<float>& p, cudaStream_t st) {
  if (!vec4_ok(p.g, D, p.M)) return false;
  const FastDiv fG((unsigned)(p.g.Ns >> 2));
  const unsigned nb = nblk4((p.g.Ns >> 2) * p.nchunks);
#define L4(DD, MM)                                                                      \
  do {                                                                                  \
    if (p.e) st_launch(k_lin_residual4<DD, MM, true>, nb, 256, 0, st, p, fG);           \
    else st_launch(k_lin_residual4<DD, MM, false>, nb, 256, 0, st, p, fG);              \
  } while (0)
  if (D == 2 && p.M == 3) L4(2, 3);
  else if (D == 2 && p.M == 5) L4(2, 5);
  else if (D == 3 && p.M == 3) L4(3, 3);
  else L4(3, 5);
#undef L4
  return true;
}

// the shifted systems of the slab solves (P = M planes) and of the SDC node
// solves (P = 1)
static bool inner4_ok(const GridP& g, int D, int P) {
  return D >= 2 && (P == 1 || P == 3 || P == 5) && g.n0 >= 4 && (g.n0 % 4) == 0 && g.bc == BC_PER;
}

bool launch_inner4(int D, int mode, const InnerParams<float>& p, cudaStream_t st) {
  if (!inner4_ok(p.g, D, p.P)) return false;
  const FastDiv fG((unsigned)(p.g.Ns >> 2));
  // 128-thread blocks: measured faster than 256 for the sweeps (finer-grained
  // scheduling at the same registers per thread)
  const unsigned nb = (unsigned)(((p.g.Ns >> 2) * p.Nt + 127) / 128);
#define K4(DD, MM)                                                         \
  do {                                                                     \
    if (mode == 0) st_launch(k_inner4<DD, MM, 0>, nb, 128, 0, st, p, fG);         \
    else if (p.fuse_bt) st_launch(k_inner4<DD, MM, 2>, nb, 128, 0, st, p, fG);    \
    else st_launch(k_inner4<DD, MM, 1>, nb, 128, 0, st, p, fG);                   \
  } while (0)
  if (D == 2 && p.P == 3) K4(2, 3);
  else if (D == 2 && p.P == 5) K4(2, 5);
  else if (D == 2) K4(2, 1);
  else if (p.P == 3) K4(3, 3);
  else if (p.P == 5) K4(3, 5);
  else K4(3, 1);
#undef K4
  return true;
}

static bool restrict4_ok(int D, const GridP& gf, const GridP& gc) {
  return D >= 2 && gf.bc == BC_PER && gc.n0 >= 4 && gc.n0 % 4 == 0 && gf.n0 == 2 * gc.n0;
}

bool launch_restrict4(int D, const GridP& gf, const GridP& gc, long long planes, const float* f, float* c,
                      cudaStream_t st) {
  if (!restrict4_ok(D, gf, gc)) return false;
  const FastDiv fG((unsigned)(gc.Ns >> 2));
  const unsigned nb = nblk4((gc.Ns >> 2) * planes);
  if (D == 2) st_launch(k_restrict4<2>, nb, 256, 0, st, gf, gc, (int)planes, fG, f, c);
  else st_launch(k_restrict4<3>, nb, 256, 0, st, gf, gc, (int)planes, fG, f, c);
  return true;
}

bool launch_inner_restrict4(int D, const InnerParams<float>& p, cudaStream_t st) {
  if (!restrict4_ok(D, p.g, p.gc) || !(p.P == 1 || p.P == 3 || p.P == 5)) return false;
  const FastDiv fG((unsigned)(p.gc.Ns >> 2));
  const unsigned nb = nblk4((p.gc.Ns >> 2) * p.Nt);
  if (D == 2 && p.P == 3) st_launch(k_inner_restrict4<2, 3>, nb, 256, 0, st, p, fG);
  else if (D == 2 && p.P == 5) st_launch(k_inner_restrict4<2, 5>, nb, 256, 0, st, p, fG);
  else if (D == 2) st_launch(k_inner_restrict4<2, 1>, nb, 256, 0, st, p, fG);
  else if (p.P == 3) st_launch(k_inner_restrict4<3, 3>, nb, 256, 0, st, p, fG);
  else if (p.P == 5) st_launch(k_inner_restrict4<3, 5>, nb, 256, 0, st, p, fG);
  else st_launch(k_inner_restrict4<3, 1>, nb, 256, 0, st, p, fG);
  return true;
}

bool launch_prolong4(int D, const GridP& gf, const GridP& gc, long long planes, const float* c, float* f,
                     cudaStream_t st) {
  if (!(D >= 2 && gf.bc == BC_PER && gf.n0 >= 4 && gf.n0 % 4 == 0 && gc.n0 * 2 == gf.n0)) return false;
  const FastDiv fG((unsigned)(gf.Ns >> 2));
  const unsigned nb = nblk4((gf.Ns >> 2) * planes);
  if (D == 2) st_launch(k_prolong4<2>, nb, 256, 0, st, gf, gc, (int)planes, fG, c, f);
  else st_launch(k_prolong4<3>, nb, 256, 0, st, gf, gc, (int)planes, fG, c, f);
  return true;
}

}  // namespace st
