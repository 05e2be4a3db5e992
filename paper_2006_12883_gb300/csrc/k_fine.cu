// FP64 fine-level kernels: the collocation residual G(U) (Eq. 2.3 chained by
// the slab coupling of Eq. 3.4), its adjoint, parameter gradients, FP64
// reductions, the U update and the SDC right-hand side.
//
// Thread mapping: one thread owns one spatial point s for a run of `chunk`
// consecutive slabs, so the coupling plane u_{n-1,M} is carried in a
// register from one slab to the next; consecutive threads own consecutive
// points (coalesced along x).  The per-block partial sums depend only on this
// fixed mapping, so norms are bitwise reproducible.
#include "ff_arith.cuh"
#include "st_kernels.cuh"

namespace st {

long long residual_blocks(const ResidParams& p);
long long residual_blocks4(const ResidParams& p);

// ---------------------------------------------------------------------------
// K1: r = G(U),  cbar_n = mean_m R'(U_{n,m}),  partial sums of G^2.
// ---------------------------------------------------------------------------
template <int D, typename TR, typename TC>
__global__ void __launch_bounds__(256) k_residual(ResidParams p) {
  grid_dep_wait();
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  double sq = 0.0;
  if (idx < (unsigned)p.nchunks * (unsigned)p.g.Ns) {
    int c, s, i, j, k;
    split_index(idx, p.g, c, s, i, j, k);
    const Nbr nb = make_nbr<D>(i, j, k, p.g);
    const long long Ns = p.g.Ns;
    const int M = p.M;
    const int n0 = c * p.chunk;
    const int n1 = min(n0 + p.chunk, p.Nt);
    double prev = (n0 == 0) ? p.u0[s] : p.U[((long long)(n0 - 1) * M + (M - 1)) * Ns + s];
    TR* R = (TR*)p.R;
    TC* cb = (TC*)p.cbar;
    TC* cn = (TC*)p.cnode;
    const double invM = 1.0 / M;
    for (int n = n0; n < n1; ++n) {
      const long long base = (long long)n * M * Ns + s;
      double u[MAXM], F[MAXM];
      double cbs = 0.0, ulast = 0.0;
#pragma unroll
      for (int m = 0; m < MAXM; ++m) {
        if (m < M) {
          const double* pl = p.U + (long long)n * M * Ns + (long long)m * Ns;
          const double um = pl[s];
          u[m] = um;
          if (m == M - 1) ulast = um;
          F[m] = lap_nb<D, double, double>(pl, s, nb, um, p.sc.cx, p.sc.cy, p.sc.cz, p.sc.k2,
                                            react<double>(p.reaction, p.rho, um));
          if (cb || cn) {
            const double dr = dreact<double>(p.reaction, p.rho, um);
            cbs += dr;
            if (cn) cn[base + (long long)m * Ns] = (TC)dr;
          }
        }
      }
#pragma unroll
      for (int m = 0; m < MAXM; ++m) {
        if (m < M) {
          double g = prev - u[m];
#pragma unroll
          for (int q = 0; q < MAXM; ++q)
            if (q < M) g = fma(p.dtq[m][q], F[q], g);
          if (p.tau) g += p.tau[base + (long long)m * Ns];
          sq = fma(g, g, sq);
          if (R) R[base + (long long)m * Ns] = (TR)g;
        }
      }
      if (cb) cb[(long long)n * Ns + s] = (TC)(cbs * invM);
      prev = ulast;
    }
  }
  if (p.partial) {
    const double t = block_sum(sq);
    if (threadIdx.x == 0) p.partial[blockIdx.x] = t;
  }
}

// ---------------------------------------------------------------------------
// The same residual in double-float arithmetic (ff_arith.cuh) for the FP32
// cycle, output rounded to float.
// ---------------------------------------------------------------------------
__device__ __forceinline__ ff nb_ff(const double* __restrict__ p, long long s, long long o, bool valid) {
  return valid ? split_double(p[s + o]) : ff{0.0f, 0.0f};
}

template <int D>
__global__ void __launch_bounds__(256) k_residual_ff(ResidParams p, ResidFF c) {
  grid_dep_wait();
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  float sq = 0.0f;
  if (idx < (unsigned)p.nchunks * (unsigned)p.g.Ns) {
    int ch, s, i, j, k;
    split_index(idx, p.g, ch, s, i, j, k);
    const Nbr nb = make_nbr<D>(i, j, k, p.g);
    const long long Ns = p.g.Ns;
    const int M = p.M;
    const int n0 = ch * p.chunk;
    const int n1 = min(n0 + p.chunk, p.Nt);
    ff prev = split_double((n0 == 0) ? p.u0[s] : p.U[((long long)(n0 - 1) * M + (M - 1)) * Ns + s]);
    float* R = (float*)p.R;
    float* cb = (float*)p.cbar;
    float* cn = (float*)p.cnode;
    const float invM = 1.0f / M;
    for (int n = n0; n < n1; ++n) {
      const long long base = (long long)n * M * Ns + s;
      ff u[MAXM], F[MAXM];
      float cbs = 0.0f;
      ff ulast = {0.0f, 0.0f};
#pragma unroll
      for (int m = 0; m < MAXM; ++m) {
        if (m < M) {
          const double* pl = p.U + (long long)n * M * Ns + (long long)m * Ns;
          const ff um = split_double(pl[s]);
          u[m] = um;
          if (m == M - 1) ulast = um;
          ff acc = ff_mul_c(um, c.k2.hi, c.k2.lo);
          {
            const ff a = nb_ff(pl, s, nb.o[0], nb.mask & 1u), b = nb_ff(pl, s, nb.o[1], nb.mask & 2u);
            acc = ff_madd_c(acc, ff_add(a, b), c.cx.hi, c.cx.lo);
          }
          if (D >= 2) {
            const ff a = nb_ff(pl, s, nb.o[2], nb.mask & 4u), b = nb_ff(pl, s, nb.o[3], nb.mask & 8u);
            acc = ff_madd_c(acc, ff_add(a, b), c.cy.hi, c.cy.lo);
          }
          if (D >= 3) {
            const ff a = nb_ff(pl, s, nb.o[4], nb.mask & 16u), b = nb_ff(pl, s, nb.o[5], nb.mask & 32u);
            acc = ff_madd_c(acc, ff_add(a, b), c.cz.hi, c.cz.lo);
          }
          if (p.reaction == ST_REACTION_LOGISTIC) {
            // rho u (1 - u) = u * (rho - rho u)
            const ff t = ff_add({c.rho.hi, c.rho.lo}, ff_neg(ff_mul_c(um, c.rho.hi, c.rho.lo)));
            acc = ff_add(acc, ff_mul(um, t));
            const float dr = fmaf(-2.0f * c.rho32, um.hi, c.rho32);
            cbs += dr;
            if (cn) cn[base + (long long)m * Ns] = dr;
          } else if (p.reaction == ST_REACTION_CUBIC) {
            // rho u (1 - u^2) = u * (rho - rho u u)
            const ff ru = ff_mul_c(um, c.rho.hi, c.rho.lo);
            const ff t = ff_add({c.rho.hi, c.rho.lo}, ff_neg(ff_mul(ru, um)));
            acc = ff_add(acc, ff_mul(um, t));
            const float dr = fmaf(-3.0f * c.rho32 * um.hi, um.hi, c.rho32);
            cbs += dr;
            if (cn) cn[base + (long long)m * Ns] = dr;
          }
          F[m] = acc;
        }
      }
#pragma unroll
      for (int m = 0; m < MAXM; ++m) {
        if (m < M) {
          ff g = ff_add(prev, ff_neg(u[m]));
#pragma unroll
          for (int q = 0; q < MAXM; ++q)
            if (q < M) g = ff_madd_c(g, F[q], c.w[m][q].hi, c.w[m][q].lo);
          const float gf = g.hi + g.lo;
          sq = fmaf(gf, gf, sq);
          if (R) R[base + (long long)m * Ns] = gf;
        }
      }
      if (cb) cb[(long long)n * Ns + s] = cbs * invM;
      prev = ulast;
    }
  }
  if (p.partial) {
    const double t = block_sum((double)sq);
    if (threadIdx.x == 0) p.partial[blockIdx.x] = t;
  }
}

// Four consecutive x points per thread (periodic, x size a multiple of 4,
// M = 3 or 5): the centre and row values are double2 loads and each loaded
// value is split once for the 4 points.
template <int D, int M>
__global__ void __launch_bounds__(256) k_residual_ff4(ResidParams p, ResidFF c, FastDiv fG) {
  grid_dep_wait();
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  float sq = 0.0f;
  const unsigned G = (unsigned)(p.g.Ns >> 2);
  if (idx < (unsigned)p.nchunks * G) {
    const int ch = (int)fG.div(idx);
    const int s0 = (int)(idx - (unsigned)ch * G) << 2;
    int i0, j, k;
    point_ijk(s0, p.g, i0, j, k);
    Nbr nb = make_nbr<D>(i0, j, k, p.g);  // periodic: every mask bit set
    const long long xl = (i0 == 0) ? (long long)(p.g.n0 - 1) : -1;
    const long long xr = (i0 + 4 == p.g.n0) ? (long long)(4 - p.g.n0) : 4;
    const long long Ns = p.g.Ns;
    const int n0 = ch * p.chunk;
    const int n1 = min(n0 + p.chunk, p.Nt);
    ff prev[4];
    {
      const double* pp = (n0 == 0) ? p.u0 + s0 : p.U + ((long long)(n0 - 1) * M + (M - 1)) * Ns + s0;
      const double2 a = *reinterpret_cast<const double2*>(pp), b = *reinterpret_cast<const double2*>(pp + 2);
      prev[0] = split_double(a.x); prev[1] = split_double(a.y);
      prev[2] = split_double(b.x); prev[3] = split_double(b.y);
    }
    float* R = (float*)p.R;
    float* cb = (float*)p.cbar;
    float* cn = (float*)p.cnode;
    for (int n = n0; n < n1; ++n) {
      const long long base = (long long)n * M * Ns + s0;
      ff u[M][4], F[M][4];
      float cbs[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const double* pl = p.U + base + (long long)m * Ns;
        {
          const double2 a = *reinterpret_cast<const double2*>(pl), b = *reinterpret_cast<const double2*>(pl + 2);
          u[m][0] = split_double(a.x); u[m][1] = split_double(a.y);
          u[m][2] = split_double(b.x); u[m][3] = split_double(b.y);
        }
        const ff vl = split_double(pl[xl]), vr = split_double(pl[xr]);
        const ff v[6] = {vl, u[m][0], u[m][1], u[m][2], u[m][3], vr};
        ff acc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc[q] = ff_mul_c(u[m][q], c.k2.hi, c.k2.lo);
          acc[q] = ff_madd_c(acc[q], ff_add(v[q], v[q + 2]), c.cx.hi, c.cx.lo);
        }
#pragma unroll
        for (int ax = 1; ax < D; ++ax) {
          const double* lo = pl + nb.o[2 * ax];
          const double* hi = pl + nb.o[2 * ax + 1];
          const double2 la = *reinterpret_cast<const double2*>(lo), lb = *reinterpret_cast<const double2*>(lo + 2);
          const double2 ha = *reinterpret_cast<const double2*>(hi), hb = *reinterpret_cast<const double2*>(hi + 2);
          const double lv[4] = {la.x, la.y, lb.x, lb.y}, hv[4] = {ha.x, ha.y, hb.x, hb.y};
          const FFC cc = (ax == 1) ? c.cy : c.cz;
#pragma unroll
          for (int q = 0; q < 4; ++q)
            acc[q] = ff_madd_c(acc[q], ff_add(split_double(lv[q]), split_double(hv[q])), cc.hi, cc.lo);
        }
        float dr[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const ff um = u[m][q];
          if (p.reaction == ST_REACTION_LOGISTIC) {
            const ff t = ff_add({c.rho.hi, c.rho.lo}, ff_neg(ff_mul_c(um, c.rho.hi, c.rho.lo)));
            acc[q] = ff_add(acc[q], ff_mul(um, t));
            dr[q] = fmaf(-2.0f * c.rho32, um.hi, c.rho32);
          } else if (p.reaction == ST_REACTION_CUBIC) {
            const ff ru = ff_mul_c(um, c.rho.hi, c.rho.lo);
            const ff t = ff_add({c.rho.hi, c.rho.lo}, ff_neg(ff_mul(ru, um)));
            acc[q] = ff_add(acc[q], ff_mul(um, t));
            dr[q] = fmaf(-3.0f * c.rho32 * um.hi, um.hi, c.rho32);
          }
          cbs[q] += dr[q];
          F[m][q] = acc[q];
        }
        if (cn) *reinterpret_cast<float4*>(cn + base + (long long)m * Ns) = make_float4(dr[0], dr[1], dr[2], dr[3]);
      }
#pragma unroll
      for (int m = 0; m < M; ++m) {
        float out[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          ff g = ff_add(prev[q], ff_neg(u[m][q]));
#pragma unroll
          for (int b = 0; b < M; ++b) g = ff_madd_c(g, F[b][q], c.w[m][b].hi, c.w[m][b].lo);
          out[q] = g.hi + g.lo;
          sq = fmaf(out[q], out[q], sq);
        }
        if (R) *reinterpret_cast<float4*>(R + base + (long long)m * Ns) = make_float4(out[0], out[1], out[2], out[3]);
      }
      if (cb) {
        const float invM = 1.0f / M;
        *reinterpret_cast<float4*>(cb + (long long)n * Ns + s0) =
            make_float4(cbs[0] * invM, cbs[1] * invM, cbs[2] * invM, cbs[3] * invM);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) prev[q] = u[M - 1][q];
    }
  }
  if (p.partial) {
    const double t = block_sum((double)sq);
    if (threadIdx.x == 0) p.partial[blockIdx.x] = t;
  }
}

static FFC split_const(double v) {
  FFC c;
  c.hi = (float)v;
  c.lo = (float)(v - (double)c.hi);
  return c;
}

static bool ff4_ok(int D, const ResidParams& p) {
  return D >= 2 && (p.M == 3 || p.M == 5) && p.g.bc == BC_PER && p.g.n0 >= 4 && p.g.n0 % 4 == 0 &&
         aligned16(p.U) && aligned16(p.u0) && aligned16(p.R) && aligned16(p.cbar) && aligned16(p.cnode);
}

long long residual_ff_blocks(int D, const ResidParams& p) {
  const long long nt = residual_tile_blocks(D, p);
  if (nt > 0) return nt;
  return ff4_ok(D, p) ? residual_blocks4(p) : residual_blocks(p);
}

bool residual_start_ok(int D, const ResidParams& p, const SmoothStart* ss) {
  return residual_tile_start_ok(D, p, ss);
}

void launch_residual_ff(int D, const ResidParams& p, cudaStream_t st, const SmoothStart* ss) {
  ResidFF c;
  c.cx = split_const(p.sc.cx);
  c.cy = split_const(p.sc.cy);
  c.cz = split_const(p.sc.cz);
  c.k2 = split_const(p.sc.k2);
  c.rho = split_const(p.rho);
  c.rho32 = (float)p.rho;
  for (int a = 0; a < MAXM; ++a)
    for (int b = 0; b < MAXM; ++b) c.w[a][b] = split_const(p.dtq[a][b]);
  if (launch_residual_tile(D, p, c, st, ss)) return;
  if (ff4_ok(D, p)) {
    const FastDiv fG((unsigned)(p.g.Ns >> 2));
    const unsigned nb4 = (unsigned)residual_blocks4(p);
    if (D == 2 && p.M == 3) st_launch(k_residual_ff4<2, 3>, nb4, 256, 0, st, p, c, fG);
    else if (D == 2) st_launch(k_residual_ff4<2, 5>, nb4, 256, 0, st, p, c, fG);
    else if (p.M == 3) st_launch(k_residual_ff4<3, 3>, nb4, 256, 0, st, p, c, fG);
    else st_launch(k_residual_ff4<3, 5>, nb4, 256, 0, st, p, c, fG);
    return;
  }
  const unsigned nb = (unsigned)residual_blocks(p);
  if (D == 1) st_launch(k_residual_ff<1>, nb, 256, 0, st, p, c);
  else if (D == 2) st_launch(k_residual_ff<2>, nb, 256, 0, st, p, c);
  else st_launch(k_residual_ff<3>, nb, 256, 0, st, p, c);
}

// blocks of the 4-point double-float residual (one partial sum per block)
long long residual_blocks4(const ResidParams& p) { return ((p.g.Ns >> 2) * p.nchunks + 255) / 256; }

// ---------------------------------------------------------------------------
// Adjoint residual rho = g - A^T lambda + C^T lambda with the exact Jacobian:
//   rho_{n,j} = g_{n,j} - lambda_{n,j}
//             + sum_m dtq[j][m] (nu*Lap lambda_{n,m}) + R'(U_{n,j}) sum_m dtq[j][m] lambda_{n,m}
//             + [j = M-1] sum_m lambda_{n+1,m}
// (dtq holds dt*Q^T).  Marches backward through its chunk of slabs.
// ---------------------------------------------------------------------------
template <int D, typename TR>
__global__ void __launch_bounds__(256) k_adj_residual(ResidParams p) {
  grid_dep_wait();
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  double sq = 0.0;
  if (idx < (unsigned)p.nchunks * (unsigned)p.g.Ns) {
    int c, s, i, j, k;
    split_index(idx, p.g, c, s, i, j, k);
    const Nbr nb = make_nbr<D>(i, j, k, p.g);
    const long long Ns = p.g.Ns;
    const int M = p.M;
    const int n0 = c * p.chunk;
    const int n1 = min(n0 + p.chunk, p.Nt);
    double next = 0.0;  // sum_m lambda_{n+1,m}
    if (n1 < p.Nt) {
      for (int m = 0; m < M; ++m) next += p.lam[((long long)n1 * M + m) * Ns + s];
    }
    TR* R = (TR*)p.R;
    for (int n = n1 - 1; n >= n0; --n) {
      const long long base = (long long)n * M * Ns + s;
      double l[MAXM], Ll[MAXM];
      double sum = 0.0;
#pragma unroll
      for (int m = 0; m < MAXM; ++m) {
        if (m < M) {
          const double* pl = p.lam + (long long)n * M * Ns + (long long)m * Ns;
          const double lm = pl[s];
          l[m] = lm;
          Ll[m] = lap_nb<D, double, double>(pl, s, nb, lm, p.sc.cx, p.sc.cy, p.sc.cz, p.sc.k2, 0.0);
          sum += lm;
        }
      }
#pragma unroll
      for (int a = 0; a < MAXM; ++a) {
        if (a < M) {
          double accL = 0.0, accl = 0.0;
#pragma unroll
          for (int m = 0; m < MAXM; ++m)
            if (m < M) {
              accL = fma(p.dtq[a][m], Ll[m], accL);
              accl = fma(p.dtq[a][m], l[m], accl);
            }
          double rp = 0.0;
          if (p.reaction != ST_REACTION_NONE) rp = dreact<double>(p.reaction, p.rho, p.U[base + (long long)a * Ns]);
          double g = fma(rp, accl, accL) - l[a];
          if (a == M - 1) {
            g += next;
            if (n == p.Nt - 1 && p.gT) g += p.gT[s];
          }
          sq = fma(g, g, sq);
          if (R) R[base + (long long)a * Ns] = (TR)g;
        }
      }
      next = sum;
    }
  }
  if (p.partial) {
    const double t = block_sum(sq);
    if (threadIdx.x == 0) p.partial[blockIdx.x] = t;
  }
}

// ---------------------------------------------------------------------------
// Gradients lambda^T dG/dtheta: per block partial sums of
//   dnu:  sum_j (dt Q^T lambda_n)_j * Lap U_{n,j}
//   drho: sum_j (dt Q^T lambda_n)_j * r(U_{n,j})
// and du0 = sum_m lambda_{0,m} (written by the threads of slab 0).
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(256) k_gradients(ResidParams p, double* partial2, double* du0) {
  grid_dep_wait();
  const long long Ns = p.g.Ns;
  const int M = p.M;
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  double gnu = 0.0, grho = 0.0;
  if (idx < (unsigned)p.Nt * (unsigned)p.g.Ns) {
    int n, s, i, j, k;
    split_index(idx, p.g, n, s, i, j, k);
    const double ihx = p.g.ih2[0], ihy = p.g.ih2[1], ihz = p.g.ih2[2];
    double l[MAXM];
    double sum = 0.0;
#pragma unroll
    for (int m = 0; m < MAXM; ++m)
      if (m < M) {
        l[m] = p.lam[((long long)n * M + m) * Ns + s];
        sum += l[m];
      }
#pragma unroll
    for (int a = 0; a < MAXM; ++a) {
      if (a < M) {
        double qt = 0.0;
#pragma unroll
        for (int m = 0; m < MAXM; ++m)
          if (m < M) qt += p.dtq[a][m] * l[m];
        const double* pl = p.U + ((long long)n * M + a) * Ns;
        const double ua = pl[s];
        gnu += qt * lap_at<D, double, double>(pl, s, i, j, k, p.g, ua, ihx, ihy, ihz);
        grho += qt * rshape<double>(p.reaction, ua);
      }
    }
    if (n == 0 && du0) du0[s] = sum;
  }
  const double t1 = block_sum(gnu);
  if (threadIdx.x == 0) p.partial[blockIdx.x] = t1;
  const double t2 = block_sum(grho);
  if (threadIdx.x == 0) partial2[blockIdx.x] = t2;
}

// Sum n partials in a fixed order into out[0] (single block of 1024).
__global__ void __launch_bounds__(1024) k_sum_partials(const double* __restrict__ part, long long n,
                                                       double* out) {
  grid_dep_wait();
  double v = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) v += part[i];
  v = block_sum(v);
  if (threadIdx.x == 0) out[0] = v;
}

// U += e (e in the cycle precision), optionally scaled.
template <typename T>
__global__ void __launch_bounds__(256) k_update(double* __restrict__ U, const T* __restrict__ e, long long n,
                                                double alpha) {
  grid_dep_wait();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) U[i] += alpha * (double)e[i];
}

// Exact float -> double by bit manipulation: the conversion instruction runs
// on the FP64 pipe, 1/64 of the FP32 rate on this GPU, and with the FP64 add
// it made the update bound by that pipe rather than by memory.  Normal
// floats and zeros convert exactly, infinities and NaNs stay so; subnormal
// floats (|e| < 2^-126) become a zero of the same sign.
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned sign = b & 0x80000000u, ex = (b >> 23) & 0xffu, man = b & 0x7fffffu;
  const unsigned hi = (ex == 0u) ? sign : sign | ((ex == 0xffu ? 0x7ffu : ex + 896u) << 20) | (man >> 3);
  const unsigned lo = (ex == 0u) ? 0u : (man << 29);
  return __hiloint2double((int)hi, (int)lo);
}

// Four values per thread; U and e 16-byte aligned (checked by the launcher).
template <typename T>
__global__ void __launch_bounds__(256) k_update4(double* __restrict__ U, const T* __restrict__ e, long long n,
                                                 double alpha) {
  grid_dep_wait();
  const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (i + 4 <= n) {
    double2 a = *reinterpret_cast<const double2*>(U + i);
    double2 b = *reinterpret_cast<const double2*>(U + i + 2);
    double e0, e1, e2, e3;
    if constexpr (sizeof(T) == 4) {
      const float4 v = *reinterpret_cast<const float4*>(e + i);
      e0 = f2d_bits(v.x); e1 = f2d_bits(v.y); e2 = f2d_bits(v.z); e3 = f2d_bits(v.w);
    } else {
      const double2 v0 = *reinterpret_cast<const double2*>(e + i);
      const double2 v1 = *reinterpret_cast<const double2*>(e + i + 2);
      e0 = v0.x; e1 = v0.y; e2 = v1.x; e3 = v1.y;
    }
    a.x += alpha * e0; a.y += alpha * e1; b.x += alpha * e2; b.y += alpha * e3;
    *reinterpret_cast<double2*>(U + i) = a;
    *reinterpret_cast<double2*>(U + i + 2) = b;
  } else {
    for (long long q = i; q < n; ++q) U[q] += alpha * (double)e[q];
  }
}

// ---------------------------------------------------------------------------
// SDC right-hand side for node m (correction form):
//   y = g_m + sum_{j<m} [ dt*QI_mj*nu*Lap delta_j + dt*QE_mj*(R(U_j + delta_j) - R(U_j)) ]
// g is G(U^k) (cycle precision), delta holds the corrections of nodes < m.
// Arithmetic in the cycle precision T; the reaction difference is taken in
// closed form, rho d (1 - 2u - d) (logistic) or rho d (1 - 3u^2 - 3ud - d^2)
// (cubic), so a small correction d loses no digits to cancellation.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T react_diff(int reaction, T rho, T u, T d) {
  if (reaction == ST_REACTION_LOGISTIC) return rho * d * ((T)1 - (T)2 * u - d);
  if (reaction == ST_REACTION_CUBIC) return rho * d * ((T)1 - (T)3 * u * u - (T)3 * u * d - d * d);
  return (T)0;
}

template <int D, typename T>
__global__ void __launch_bounds__(256) k_sdc_rhs(GridP g, int Nt, int M, int m, double nu, int reaction,
                                                 double rho, SdcCoef cf,
                                                 const T* __restrict__ G, const T* __restrict__ delta,
                                                 const double* __restrict__ U, T* __restrict__ y) {
  grid_dep_wait();
  const long long Ns = g.Ns;
  const unsigned idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (unsigned)Nt * (unsigned)g.Ns) return;
  int n, s, i, j, k;
  split_index(idx, g, n, s, i, j, k);
  const T ihx = (T)g.ih2[0], ihy = (T)g.ih2[1], ihz = (T)g.ih2[2];
  const T nuT = (T)nu, rhoT = (T)rho;
  T acc = G[((long long)n * M + m) * Ns + s];
  for (int q = 0; q < m; ++q) {
    const T* pl = delta + ((long long)n * M + q) * Ns;
    const T dq = pl[s];
    acc += (T)cf.qi[q] * nuT * lap_at<D, T, T>(pl, s, i, j, k, g, dq, ihx, ihy, ihz);
    if (reaction != ST_REACTION_NONE)
      acc += (T)cf.qe[q] * react_diff<T>(reaction, rhoT, (T)U[((long long)n * M + q) * Ns + s], dq);
  }
  y[(long long)n * Ns + s] = acc;
}

// Copy a [Nt][Ns] field into plane m of a [Nt][M][Ns] field.
template <typename T>
__global__ void __launch_bounds__(256) k_scatter_plane(const T* __restrict__ src, T* __restrict__ dst,
                                                       long long Ns, int Nt, int M, int m) {
  grid_dep_wait();
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Ns * Nt) return;
  const long long s = idx % Ns;
  const long long n = idx / Ns;
  dst[(n * M + m) * Ns + s] = src[idx];
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
static inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

long long residual_blocks(const ResidParams& p) { return (p.g.Ns * p.nchunks + 255) / 256; }

template <typename TR, typename TC>
static void launch_res_t(int D, const ResidParams& p, cudaStream_t st) {
  const unsigned nb = (unsigned)residual_blocks(p);
  if (D == 1) st_launch(k_residual<1, TR, TC>, nb, 256, 0, st, p);
  else if (D == 2) st_launch(k_residual<2, TR, TC>, nb, 256, 0, st, p);
  else st_launch(k_residual<3, TR, TC>, nb, 256, 0, st, p);
}

void launch_residual(int D, int r_fp64, int c_fp64, const ResidParams& p, cudaStream_t st) {
  if (r_fp64 && c_fp64) launch_res_t<double, double>(D, p, st);
  else if (r_fp64) launch_res_t<double, float>(D, p, st);
  else launch_res_t<float, float>(D, p, st);
}

void launch_adj_residual(int D, int r_fp64, const ResidParams& p, cudaStream_t st) {
  const unsigned nb = (unsigned)residual_blocks(p);
  if (r_fp64) {
    if (D == 1) st_launch(k_adj_residual<1, double>, nb, 256, 0, st, p);
    else if (D == 2) st_launch(k_adj_residual<2, double>, nb, 256, 0, st, p);
    else st_launch(k_adj_residual<3, double>, nb, 256, 0, st, p);
  } else {
    if (D == 1) st_launch(k_adj_residual<1, float>, nb, 256, 0, st, p);
    else if (D == 2) st_launch(k_adj_residual<2, float>, nb, 256, 0, st, p);
    else st_launch(k_adj_residual<3, float>, nb, 256, 0, st, p);
  }
}

long long gradient_blocks(const ResidParams& p) { return (p.g.Ns * p.Nt + 255) / 256; }

void launch_gradients(int D, const ResidParams& p, double* partial2, double* du0, cudaStream_t st) {
  const unsigned nb = (unsigned)gradient_blocks(p);
  if (D == 1) st_launch(k_gradients<1>, nb, 256, 0, st, p, partial2, du0);
  else if (D == 2) st_launch(k_gradients<2>, nb, 256, 0, st, p, partial2, du0);
  else st_launch(k_gradients<3>, nb, 256, 0, st, p, partial2, du0);
}

void launch_sum_partials(const double* part, long long n, double* out, cudaStream_t st) {
  st_launch(k_sum_partials, 1, 1024, 0, st, part, n, out);
}

// W[n][m][s] += U[n][m][s] - prev_n(s), prev_n = u0 (n = 0) or U[n-1][M-1]:
// turns a residual G(U) (with its tau) into dt Q F(U) + tau.
__global__ void __launch_bounds__(256) k_add_state(double* __restrict__ W, const double* __restrict__ U,
                                                   const double* __restrict__ u0, long long Ns, int Nt, int M) {
  grid_dep_wait();
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Ns * Nt * M) return;
  const long long s = idx % Ns;
  const long long nm = idx / Ns;
  const long long n = nm / M;
  const double prev = (n == 0) ? u0[s] : U[((n - 1) * M + (M - 1)) * Ns + s];
  W[idx] += U[idx] - prev;
}

void launch_add_state(double* W, const double* U, const double* u0, long long Ns, int Nt, int M, cudaStream_t st) {
  st_launch(k_add_state, blocks_for(Ns * Nt * M, 256), 256, 0, st, W, U, u0, Ns, Nt, M);
}

// v <- W v (inverse = 0) or W^-1 v (inverse = 1) on every plane, W the lumped
// mass weights of a Neumann vertex grid relative to h^d: a factor 1/2 for
// each axis on which the point is a boundary vertex.  Exact (powers of two).
__global__ void __launch_bounds__(256) k_mass_weight(double* __restrict__ v, GridP g, long long planes,
                                                     int inverse) {
  grid_dep_wait();
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= planes * g.Ns) return;
  int i, j, k;
  decompose(idx % g.Ns, g, i, j, k);
  int nb = (i == 0 || i == g.n0 - 1) ? 1 : 0;
  if (g.n1 > 1 && (j == 0 || j == g.n1 - 1)) ++nb;
  if (g.n2 > 1 && (k == 0 || k == g.n2 - 1)) ++nb;
  if (nb) v[idx] = inverse ? ldexp(v[idx], nb) : ldexp(v[idx], -nb);
}

void launch_mass_weight(double* v, const GridP& g, long long planes, int inverse, cudaStream_t st) {
  st_launch(k_mass_weight, blocks_for(planes * g.Ns, 256), 256, 0, st, v, g, planes, inverse);
}

void launch_update(int fp64, double* U, const void* e, long long n, cudaStream_t st, double alpha) {
  if (((uintptr_t)U & 15) == 0 && ((uintptr_t)e & 15) == 0) {
    const unsigned nb = blocks_for((n + 3) / 4, 256);
    if (fp64) st_launch(k_update4<double>, nb, 256, 0, st, U, (const double*)e, n, alpha);
    else st_launch(k_update4<float>, nb, 256, 0, st, U, (const float*)e, n, alpha);
    return;
  }
  if (fp64) st_launch(k_update<double>, blocks_for(n, 256), 256, 0, st, U, (const double*)e, n, alpha);
  else st_launch(k_update<float>, blocks_for(n, 256), 256, 0, st, U, (const float*)e, n, alpha);
}

void launch_sdc_rhs(int D, int fp64, const GridP& g, int Nt, int M, int m, double nu, int reaction,
                    double rho, const SdcCoef& cf, const void* G, const void* delta,
                    const double* U, void* y, cudaStream_t st) {
  const unsigned nb = blocks_for(g.Ns * Nt, 256);
#define SDC_L(DD, TT)                                                                              \
  st_launch(k_sdc_rhs<DD, TT>, nb, 256, 0, st, g, Nt, M, m, nu, reaction, rho, cf, (const TT*)G,     \
                                        (const TT*)delta, U, (TT*)y)
  if (fp64) {
    if (D == 1) SDC_L(1, double); else if (D == 2) SDC_L(2, double); else SDC_L(3, double);
  } else {
    if (D == 1) SDC_L(1, float); else if (D == 2) SDC_L(2, float); else SDC_L(3, float);
  }
#undef SDC_L
}

void launch_scatter_plane(int fp64, const void* src, void* dst, long long Ns, int Nt, int M, int m,
                          cudaStream_t st) {
  const unsigned nb = blocks_for(Ns * Nt, 256);
  if (fp64) st_launch(k_scatter_plane<double>, nb, 256, 0, st, (const double*)src, (double*)dst, Ns, Nt, M, m);
  else st_launch(k_scatter_plane<float>, nb, 256, 0, st, (const float*)src, (float*)dst, Ns, Nt, M, m);
}

}  // namespace st
