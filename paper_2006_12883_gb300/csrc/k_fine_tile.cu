// Fine residual G(U) (Eq. 2.3 with the slab coupling of Eq. 3.4) on 2D
// periodic grids in 64 x 16 tiles: FP64-accurate arithmetic on the FP32
// pipes, FP32 output, as the double-float kernels of k_fine.cu, with every
// value split once instead of at each of its five uses and with a split that
// makes the 5-point second differences exact.
//
// A block owns one tile for a run of `chunk` slabs and walks its node planes
// in order.  The doubles of one plane (tile and one-point halo, periodic
// wrap) are loaded and the block takes E, the largest binary exponent among
// them.  Each value u is then held as hq + l, with hq = u rounded to a
// multiple of 2^(E-20) (at most 22 significant bits) and l = u - hq rounded
// to float (|l| <= 2^(E-21)), in a double-buffered shared-memory plane.  Sums
// of a few hq are exact in FP32, so the second differences
//     Sx = hq(i-1) + hq(i+1) - 2 hq(i)      (and Sy along y)
// carry no rounding; the low parts enter in plain FP32 (they are 2^-21 of
// the data).  The products with nu/h^2, the reaction term and the mixing
// with dt*Q use error-free products and TwoSums with the errors summed in
// FP32 and one final rounding, the compensated sum and dot product of Ogita,
// Rump and Oishi (2005).  The representation error of u is at most 2^(E-45),
// about 3e-14 of the tile's largest value, and the arithmetic rounds at a few
// 2^-48 of the terms, so G carries an absolute error of a few 1e-14 times
// its largest term, the accuracy of the double-float kernels.
//
// The next plane's doubles are loaded while the current plane is computed.
// The M residual rows of a slab are accumulated as the planes arrive:
// G_m starts from u_{n-1,M}, plane b subtracts u_b from G_b and adds
// dt q_{mb} F(u_b) to every G_m.  Tiles with a value of magnitude 2^100 or
// more (or not finite) give NaN residuals; magnitudes below 2^-126 count as 0.
#include "ff_arith.cuh"
#include "st_kernels.cuh"

namespace st {

namespace {

constexpr int kRW = 64, kRH = 16;
constexpr int kRS = 72;                 // shared row stride: halo column 3, interior 4..67, halo column 68
constexpr unsigned kEmaxLimit = 1123;   // biased exponent of 2^100
constexpr int kQmin = -100;             // smallest grid spacing 2^kQmin of the high parts

struct RPlane {
  float hi[kRH + 2][kRS];  // row 0: the row above the tile, rows 1..16 the tile, row 17 the row below
  float lo[kRH + 2][kRS];
};
struct RSmem {
  RPlane pl[2];
  unsigned emax[2];
};

// Knuth's TwoSum: s + e == a + b exactly
__device__ __forceinline__ float tsum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}

// a * (chi + clo) as an unevaluated pair p + e (exact product of a and chi
// by FMA, the small cross term added)
__device__ __forceinline__ float tprod(float a, float chi, float clo, float& e) {
  const float p = __fmul_rn(a, chi);
  e = fmaf(a, clo, fmaf(a, chi, -p));
  return p;
}

// ISO: h_x = h_y (cx == cy), so the two exact second differences add exactly
// (|Sx + Sy| <= 2^24 grid steps) and take one error-free product with nu/h^2.
// START: also write the first step of the cycle's first smoothing from the
// float residual (y = F r and the zero-start Jacobi iterate z, SmoothStart).
template <int M, bool ISO, bool START>
__global__ void __launch_bounds__(256, M == 3 ? 3 : 2) k_residual_tile(ResidParams p, ResidFF c, SmoothStart ss) {
  grid_dep_wait();
  __shared__ __align__(16) RSmem S;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4, lane = tid & 31;
  const int nx = p.g.n0, ny = p.g.n1;
  const long long Ns = p.g.Ns;
  const int ntx = nx / kRW;
  const int per_slab = ntx * (ny / kRH);
  const int tile = (int)(blockIdx.x % (unsigned)per_slab), ch = (int)(blockIdx.x / (unsigned)per_slab);
  const int j0 = (tile / ntx) * kRH, i0 = (tile % ntx) * kRW;
  const int sA = ch * p.chunk, sB = min(sA + p.chunk, p.Nt);
  // this thread's four points: row j0 + ty, columns i0 + 4 tx .. i0 + 4 tx + 3
  const long long own = (long long)(j0 + ty) * nx + i0 + 4 * tx;
  // this thread's halo values: threads 0..63 a pair of the rows above (0..31)
  // or below (32..63), threads 64..95 one value of the left / right column
  int hkind = 0, hrow = 0, hcol = 0;
  long long hoff = 0;
  if (tid < 64) {
    const int side = tid >> 5, x = 2 * (tid & 31);
    const int row = side ? (j0 + kRH == ny ? 0 : j0 + kRH) : (j0 == 0 ? ny - 1 : j0 - 1);
    hkind = 1;
    hoff = (long long)row * nx + i0 + x;
    hrow = side ? kRH + 1 : 0;
    hcol = 4 + x;
  } else if (tid < 96) {
    const int q = tid - 64, side = q & 1, row = q >> 1;
    const int col = side ? (i0 + kRW == nx ? 0 : i0 + kRW) : (i0 == 0 ? nx - 1 : i0 - 1);
    hkind = 2;
    hoff = (long long)(j0 + row) * nx + col;
    hrow = 1 + row;
    hcol = side ? 4 + kRW : 3;
  }
  auto load = [&](long long plane, double raw[6]) {
    const double* base = p.U + plane * Ns;
    const double2 a = *reinterpret_cast<const double2*>(base + own);
    const double2 b = *reinterpret_cast<const double2*>(base + own + 2);
    raw[0] = a.x; raw[1] = a.y; raw[2] = b.x; raw[3] = b.y;
    raw[4] = 0.0; raw[5] = 0.0;
    if (hkind == 1) {
      const double2 h = *reinterpret_cast<const double2*>(base + hoff);
      raw[4] = h.x; raw[5] = h.y;
    } else if (hkind == 2) {
      raw[4] = base[hoff];
    }
  };

  if (tid == 0) { S.emax[0] = 0u; S.emax[1] = 0u; }
  // the coupling value u_{n-1,M} at this thread's points
  float ph[4], pl[4];
  {
    const double* pp = (sA == 0) ? p.u0 + own : p.U + ((long long)(sA - 1) * M + (M - 1)) * Ns + own;
    const double2 a = *reinterpret_cast<const double2*>(pp), b = *reinterpret_cast<const double2*>(pp + 2);
    const double v[4] = {a.x, a.y, b.x, b.y};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const ff s = split_double(v[q]);
      ph[q] = s.hi; pl[q] = s.lo;
    }
  }
  double raw[6];
  load((long long)sA * M, raw);
  __syncthreads();

  float* R = (float*)p.R;
  float* cb = (float*)p.cbar;
  float* cn = (float*)p.cnode;
  const int rx = p.reaction;
  float sq = 0.0f;
  int k = 0;  // planes done by this block (selects the shared buffer)
  for (int n = sA; n < sB; ++n) {
    float g[M][4], ge[M][4];
#pragma unroll
    for (int m = 0; m < M; ++m)
#pragma unroll
      for (int q = 0; q < 4; ++q) { g[m][q] = ph[q]; ge[m][q] = pl[q]; }
    float cbs[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int b = 0; b < M; ++b, ++k) {
      const int buf = k & 1;
      // the block's largest exponent of this plane
      unsigned ex = 0u;
#pragma unroll
      for (int i = 0; i < 6; ++i) ex = max(ex, ((unsigned)__double2hiint(raw[i]) >> 20) & 0x7ffu);
      ex = __reduce_max_sync(0xffffffffu, ex);
      if (lane == 0) atomicMax(&S.emax[buf], ex);
      __syncthreads();
      const unsigned E = S.emax[buf];
      const bool bad = E >= kEmaxLimit;
      const int Q = bad ? 0 : max((int)E - 1023 - 20, kQmin);
      const float C = __int_as_float(((Q + 150) << 23) | 0x400000);  // 1.5 * 2^(Q+23)
      float chh[4], cll[4];
      auto qsplit = [&](double v, float& h, float& l) {
        const ff s = split_double(v);
        h = __fsub_rn(__fadd_rn(s.hi, C), C);      // s.hi rounded to a multiple of 2^Q
        l = __fadd_rn(__fsub_rn(s.hi, h), s.lo);   // s.hi - h is exact
      };
#pragma unroll
      for (int q = 0; q < 4; ++q) qsplit(raw[q], chh[q], cll[q]);
      RPlane& P = S.pl[buf];
      *reinterpret_cast<float4*>(&P.hi[ty + 1][4 + 4 * tx]) = make_float4(chh[0], chh[1], chh[2], chh[3]);
      *reinterpret_cast<float4*>(&P.lo[ty + 1][4 + 4 * tx]) = make_float4(cll[0], cll[1], cll[2], cll[3]);
      if (hkind == 1) {
        float h0, l0, h1, l1;
        qsplit(raw[4], h0, l0);
        qsplit(raw[5], h1, l1);
        *reinterpret_cast<float2*>(&P.hi[hrow][hcol]) = make_float2(h0, h1);
        *reinterpret_cast<float2*>(&P.lo[hrow][hcol]) = make_float2(l0, l1);
      } else if (hkind == 2) {
        float h0, l0;
        qsplit(raw[4], h0, l0);
        P.hi[hrow][hcol] = h0;
        P.lo[hrow][hcol] = l0;
      }
      // the next plane of this block, in flight while this one is computed
      if (b + 1 < M) load((long long)n * M + b + 1, raw);
      else if (n + 1 < sB) load((long long)(n + 1) * M, raw);
      __syncthreads();
      if (tid == 0) S.emax[buf] = 0u;  // every thread has read it; reused two planes on
      const float4 ah = *reinterpret_cast<const float4*>(&P.hi[ty][4 + 4 * tx]);
      const float4 bh = *reinterpret_cast<const float4*>(&P.hi[ty + 2][4 + 4 * tx]);
      const float4 al = *reinterpret_cast<const float4*>(&P.lo[ty][4 + 4 * tx]);
      const float4 bl = *reinterpret_cast<const float4*>(&P.lo[ty + 2][4 + 4 * tx]);
      const float xh[6] = {P.hi[ty + 1][3 + 4 * tx], chh[0], chh[1], chh[2], chh[3], P.hi[ty + 1][8 + 4 * tx]};
      const float xl[6] = {P.lo[ty + 1][3 + 4 * tx], cll[0], cll[1], cll[2], cll[3], P.lo[ty + 1][8 + 4 * tx]};
      const float ahv[4] = {ah.x, ah.y, ah.z, ah.w}, bhv[4] = {bh.x, bh.y, bh.z, bh.w};
      const float alv[4] = {al.x, al.y, al.z, al.w}, blv[4] = {bl.x, bl.y, bl.z, bl.w};
      float dr[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float h = chh[q], l = cll[q];
        // nu * Laplacian: exact second differences of the high parts
        const float sx = fmaf(-2.0f, h, __fadd_rn(xh[q], xh[q + 2]));
        const float sy = fmaf(-2.0f, h, __fadd_rn(ahv[q], bhv[q]));
        const float lx = fmaf(-2.0f, l, xl[q] + xl[q + 2]);
        const float ly = fmaf(-2.0f, l, alv[q] + blv[q]);
        float s, t;
        if constexpr (ISO) {
          s = tprod(__fadd_rn(sx, sy), c.cx.hi, c.cx.lo, t);
          t = fmaf(c.cx.hi, lx + ly, t);
        } else {
          float e1, e2;
          const float p1 = tprod(sx, c.cx.hi, c.cx.lo, e1);
          const float p2 = tprod(sy, c.cy.hi, c.cy.lo, e2);
          s = tsum(p1, p2, t);
          t = fmaf(c.cy.hi, ly, fmaf(c.cx.hi, lx, t + (e1 + e2)));
        }
        // the reaction term R(u) = rho (u - u^2) or rho (u - u^3)
        float rs = 0.0f, re = 0.0f;
        const float u32 = h + l;
        dr[q] = 0.0f;
        if (rx == ST_REACTION_LOGISTIC || rx == ST_REACTION_CUBIC) {
          const float pu = __fmul_rn(h, h);
          float eu = fmaf(h, h, -pu);
          eu = fmaf(h + h, l, eu);
          eu = fmaf(l, l, eu);  // u^2 = pu + eu
          float pw = pu, ew = eu;
          if (rx == ST_REACTION_CUBIC) {  // u^3 = (pu + eu) u
            pw = __fmul_rn(pu, h);
            ew = fmaf(eu, h, fmaf(pu, l, fmaf(pu, h, -pw)));
          }
          float tt;
          const float ss = tsum(h, -pw, tt);
          tt += l - ew;
          float er;
          rs = tprod(ss, c.rho.hi, c.rho.lo, er);
          re = fmaf(tt, c.rho.hi, er);
          dr[q] = (rx == ST_REACTION_LOGISTIC) ? fmaf(-2.0f * c.rho32, u32, c.rho32)
                                               : fmaf(-3.0f * c.rho32 * u32, u32, c.rho32);
        }
        float fe;
        float fh = tsum(s, rs, fe);
        fe += t + re;
        if (bad) fh = __int_as_float(0x7fffffff);
        // G_b -= u_b; G_m += dt q_{mb} F(u_b)
        {
          float x;
          g[b][q] = tsum(g[b][q], -h, x);
          ge[b][q] += x - l;
        }
#pragma unroll
        for (int m = 0; m < M; ++m) {
          float pe, x;
          const float pw = tprod(fh, c.w[m][b].hi, c.w[m][b].lo, pe);
          pe = fmaf(fe, c.w[m][b].hi, pe);
          g[m][q] = tsum(g[m][q], pw, x);
          ge[m][q] += x + pe;
        }
        cbs[q] += dr[q];
      }
      if (cn)
        *reinterpret_cast<float4*>(cn + ((long long)n * M + b) * Ns + own) = make_float4(dr[0], dr[1], dr[2], dr[3]);
      if (b == M - 1) {
#pragma unroll
        for (int q = 0; q < 4; ++q) { ph[q] = chh[q]; pl[q] = cll[q]; }
      }
    }
    float out[M][4];
#pragma unroll
    for (int m = 0; m < M; ++m) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        out[m][q] = g[m][q] + ge[m][q];
        sq = fmaf(out[m][q], out[m][q], sq);
      }
      if (R)
        *reinterpret_cast<float4*>(R + ((long long)n * M + m) * Ns + own) =
            make_float4(out[m][0], out[m][1], out[m][2], out[m][3]);
    }
    float cbv[4] = {0.f, 0.f, 0.f, 0.f};
    if (cb) {
      const float invM = 1.0f / M;
#pragma unroll
      for (int q = 0; q < 4; ++q) cbv[q] = cbs[q] * invM;
      *reinterpret_cast<float4*>(cb + (long long)n * Ns + own) = make_float4(cbv[0], cbv[1], cbv[2], cbv[3]);
    }
    if constexpr (START) {
      // y = F r per point (the level residual of e = 0 is r), then the
      // zero-start iterate of each real plane and complex pair
      const long long base = (long long)n * M * Ns + own;
      float y[M][4];
#pragma unroll
      for (int a = 0; a < M; ++a) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float acc = 0.f;
#pragma unroll
          for (int b = 0; b < M; ++b) acc = fmaf(ss.F[a][b], out[b][q], acc);
          y[a][q] = acc;
        }
        *reinterpret_cast<float4*>(ss.y + base + (long long)a * Ns) = make_float4(y[a][0], y[a][1], y[a][2], y[a][3]);
      }
#pragma unroll
      for (int pl = 0; pl < M; ++pl) {
        const int kd = ss.sh.kind[pl];
        if (kd == SH_REAL || kd == SH_RE) {
          const int pi = pl + 1 < M ? pl + 1 : pl;
          float zr[4], zi[4];
#pragma unroll
          for (int q = 0; q < 4; ++q)
            jac_zero(y[pl][q], kd == SH_REAL ? 0.f : y[pi][q], kd != SH_REAL, ss.sh.sr[pl], ss.sh.si[pl],
                     ss.k2 + cbv[q], ss.omega, zr[q], zi[q]);
          *reinterpret_cast<float4*>(ss.z + base + (long long)pl * Ns) = make_float4(zr[0], zr[1], zr[2], zr[3]);
          if (kd == SH_RE && pl + 1 < M)
            *reinterpret_cast<float4*>(ss.z + base + (long long)pi * Ns) = make_float4(zi[0], zi[1], zi[2], zi[3]);
        }
      }
    }
  }
  if (p.partial) {
    const double t = block_sum((double)sq);
    if (tid == 0) p.partial[blockIdx.x] = t;
  }
}

bool tile_ok(int D, const ResidParams& p) {
  return D == 2 && (p.M == 3 || p.M == 5) && p.g.bc == BC_PER && p.g.n0 >= kRW && p.g.n0 % kRW == 0 &&
         p.g.n1 >= kRH && p.g.n1 % kRH == 0 && p.tau == nullptr && aligned16(p.U) && aligned16(p.u0) &&
         aligned16(p.R) && aligned16(p.cbar) && aligned16(p.cnode);
}

// the smoothing start needs the float residual it transforms and, with a
// reaction term, the cbar this call writes
bool start_ok(const ResidParams& p, const SmoothStart* ss) {
  return ss && ss->y && ss->z && p.R && aligned16(ss->y) && aligned16(ss->z) &&
         (p.reaction == ST_REACTION_NONE || p.cbar);
}

}  // namespace

long long residual_tile_blocks(int D, const ResidParams& p) {
  if (!tile_ok(D, p)) return 0;
  return (long long)(p.g.n0 / kRW) * (p.g.n1 / kRH) * p.nchunks;
}

bool residual_tile_start_ok(int D, const ResidParams& p, const SmoothStart* ss) {
  return tile_ok(D, p) && start_ok(p, ss);
}

bool launch_residual_tile(int D, const ResidParams& p, const ResidFF& c, cudaStream_t st, const SmoothStart* ss) {
  if (!tile_ok(D, p)) return false;
  const unsigned nb = (unsigned)residual_tile_blocks(D, p);
  const bool iso = p.sc.cx == p.sc.cy;
  const bool start = start_ok(p, ss);
  SmoothStart s{};
  if (start) s = *ss;
#define RT(MM, II)                                                                  \
  do {                                                                              \
    if (start) st_launch(k_residual_tile<MM, II, true>, nb, 256, 0, st, p, c, s);   \
    else st_launch(k_residual_tile<MM, II, false>, nb, 256, 0, st, p, c, s);        \
  } while (0)
  if (p.M == 3 && iso) RT(3, true);
  else if (p.M == 3) RT(3, false);
  else if (iso) RT(5, true);
  else RT(5, false);
#undef RT
  return true;
}

}  // namespace st
