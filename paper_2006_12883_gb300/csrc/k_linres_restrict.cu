// The level residual of the V-cycle's coarse-grid correction (Eq. 4.1 with
// the level operator of Eq. 3.4), res = r - (A e - C e), fused with its full
// weighting onto the next grid (2D periodic, every axis halved, M = 3 or 5,
// FP32, forward operator with cbar).  The two-kernel sequence writes res to
// HBM and reads it back for the restriction (17.8 bytes per fine dof at
// M = 5); here a block stages e with a two-point ring, r, cbar and the slab
// coupling plane with a one-point ring in shared memory (cp.async), computes
// res on its 64 x 16 fine tile and the one-point ring the weighting needs,
// in place of r (one 4-point group or ring point per thread), and writes the
// 32 x 8 coarse tile: 9.8 bytes per fine dof (the coupling plane and the
// halos come from L2).  The arithmetic is term for term that of k_lin_residual4 and
// k_restrict4 (k_level4.cu), so the coarse values equal the two-launch
// sequence's to the bit.  With START the kernel also does the first step of
// the coarse level's first smoothing, which starts from e = 0 (so its level
// residual is the restricted residual itself): y = F r and the zero-start
// Jacobi iterate z on the coarse tile, as the coarse level's residual kernel
// would.
#include <mutex>

#include "st_kernels.cuh"

namespace st {

namespace {

constexpr int kFW = 64, kFH = 16;  // fine tile
constexpr int kS = 72;             // shared row stride: fine columns -4..67, the tile's at 4..67
constexpr int kThreads = 320;     // one residual item (and at M = 5 one coarse group) per thread

// e rows -2..16 of the tile (shared row = tile row + 2), r, cbar and the
// coupling plane rows -1..15 (shared row = tile row + 1)
template <int M>
struct LRSmem {
  static constexpr int kER = kFH + 3, kRR = kFH + 1;
  float e[M][kER][kS];
  float r[M][kRR][kS];  // r, then res in place
  float cb[kRR][kS];
  float carry[kRR][kS];
};

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(__cvta_generic_to_global(src))
               : "memory");
}

__device__ __forceinline__ void ld4s(const float* s, float (&v)[4]) {
  const float4 a = *reinterpret_cast<const float4*>(s);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}

// NQ consecutive shared values from s (a 16-byte aligned float4 for NQ = 4)
template <int NQ>
__device__ __forceinline__ void ldq(const float* s, float (&v)[NQ]) {
  if constexpr (NQ == 4) {
    ld4s(s, v);
  } else {
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] = s[q];
  }
}

// res at NQ consecutive points of one row (shared column c0 of the first;
// shared e row re, r row rr): k_lin_residual4's arithmetic, in its order.
template <int M, int NQ>
__device__ __forceinline__ void residual_points(const LinParams<float>& p, LRSmem<M>& S, int re, int rr, int c0,
                                                bool has_cb) {
  float cb[NQ], acc[M][NQ], ec[M][NQ], t[NQ];
  if (has_cb) ldq<NQ>(&S.cb[rr][c0], cb);
  else
#pragma unroll
    for (int q = 0; q < NQ; ++q) cb[q] = 0.f;
#pragma unroll
  for (int a = 0; a < M; ++a) {
    ldq<NQ>(&S.r[a][rr][c0], acc[a]);
    ldq<NQ>(&S.e[a][re][c0], ec[a]);
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[a][q] = acc[a][q] - ec[a][q];
  }
#pragma unroll
  for (int b = 0; b < M; ++b) {
    float up[NQ], dn[NQ], Fe[NQ];
    const float (&c)[NQ] = ec[b];
    ldq<NQ>(&S.e[b][re - 1][c0], up);
    ldq<NQ>(&S.e[b][re + 1][c0], dn);
    float v[NQ + 2];
    v[0] = S.e[b][re][c0 - 1];
    v[NQ + 1] = S.e[b][re][c0 + NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q + 1] = c[q];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      Fe[q] = cb[q] * c[q];
      Fe[q] = fmaf(p.sc.k2, c[q], Fe[q]);
      Fe[q] = fmaf(p.sc.cx, v[q] + v[q + 2], Fe[q]);
      Fe[q] = fmaf(p.sc.cy, up[q] + dn[q], Fe[q]);
    }
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
      for (int q = 0; q < NQ; ++q) acc[a][q] = fmaf(p.W[a][b], Fe[q], acc[a][q]);
  }
  ldq<NQ>(&S.carry[rr][c0], t);
#pragma unroll
  for (int a = 0; a < M; ++a) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[a][q] = acc[a][q] + t[q];
    if constexpr (NQ == 4)
      *reinterpret_cast<float4*>(&S.r[a][rr][c0]) = make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
    else
#pragma unroll
      for (int q = 0; q < NQ; ++q) S.r[a][rr][c0 + q] = acc[a][q];
  }
}

template <int M, bool START>
__global__ void __launch_bounds__(kThreads, M == 3 ? 4 : 3) k_linres_restrict(LinParams<float> p, GridP gc,
                                                                              float* __restrict__ coarse,
                                                                              SmoothStart ss,
                                                                              const float* __restrict__ cbarc) {
  grid_dep_wait();
  constexpr int kER = LRSmem<M>::kER, kRR = LRSmem<M>::kRR;
  extern __shared__ __align__(16) unsigned char smraw[];
  LRSmem<M>& S = *reinterpret_cast<LRSmem<M>*>(smraw);
  const int tid = threadIdx.x;
  const int nx = p.g.n0, ny = p.g.n1;
  const long long Ns = p.g.Ns, Nc = gc.Ns;
  const int ntx = nx / kFW;
  const int per_slab = ntx * (ny / kFH);
  const int tile = (int)(blockIdx.x % (unsigned)per_slab), n = (int)(blockIdx.x / (unsigned)per_slab);
  const int j0 = (tile / ntx) * kFH, i0 = (tile % ntx) * kFW;
  const long long base = (long long)n * M * Ns;
  auto row = [&](int r) -> long long {  // periodic row r of the tile (-2..kFH + 1)
    int j = j0 + r;
    j = j < 0 ? j + ny : (j >= ny ? j - ny : j);
    return (long long)j * nx;
  };
  const bool has_cb = p.cbar != nullptr;
  const int cl = i0 == 0 ? nx - 4 : i0 - 4, cr = i0 + kFW == nx ? 0 : i0 + kFW;
  auto gcol = [&](int g) { return g == 0 ? cl : (g == 17 ? cr : i0 + 4 * (g - 1)); };
  for (int sl = tid; sl < kER * 18; sl += kThreads) {  // e: rows -2..16, column groups -1..16
    const int r = sl / 18, g = sl - r * 18;
    const float* src = p.e + base + row(r - 2) + gcol(g);
    float* dst = &S.e[0][r][4 * g];
#pragma unroll
    for (int b = 0; b < M; ++b) cp_async16(dst + b * (kER * kS), src + b * Ns);
  }
  // the coupling plane e_{n-1,M} (zero on the first slab)
  const float* prev = n > 0 ? p.e + ((long long)(n - 1) * M + (M - 1)) * Ns : nullptr;
  for (int sl = tid; sl < kRR * 18; sl += kThreads) {  // r, cbar, coupling: rows -1..15
    const int r = sl / 18, g = sl - r * 18;
    const long long off = row(r - 1) + gcol(g);
    float* dst = &S.r[0][r][4 * g];
#pragma unroll
    for (int a = 0; a < M; ++a) cp_async16(dst + a * (kRR * kS), p.r + base + off + a * Ns);
    if (has_cb) cp_async16(&S.cb[r][4 * g], p.cbar + (long long)n * Ns + off);
    if (prev) cp_async16(&S.carry[r][4 * g], prev + off);
    else *reinterpret_cast<float4*>(&S.carry[r][4 * g]) = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();

  // res on tile rows -1..15: columns 0..63 in groups of 4, and column -1
  // (one item per thread: 17 x 16 groups and 17 single points)
  for (int it = tid; it < kRR * 17; it += kThreads) {
    if (it < kRR * 16) {
      const int r = it >> 4, c0 = 4 + 4 * (it & 15);
      residual_points<M, 4>(p, S, r + 1, r, c0, has_cb);
    } else {
      const int r = it - kRR * 16;
      residual_points<M, 1>(p, S, r + 1, r, 3, has_cb);
    }
  }
  __syncthreads();

  // full weighting: coarse rows J of the tile take fine rows 2J-1, 2J, 2J+1
  // (weights 1/4, 1/2, 1/4), each row k_restrict4's 9-value combination
  const int I0 = i0 >> 1, J0 = j0 >> 1;
  for (int it = tid; it < M * (kFH / 2) * (kFW / 8); it += kThreads) {
    const int a = it / ((kFH / 2) * (kFW / 8)), rem = it - a * ((kFH / 2) * (kFW / 8));
    const int J = rem >> 3, G = rem & 7;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float w = k == 1 ? 0.5f : 0.25f;
      const float* f = &S.r[a][2 * J + k][0];  // fine row 2J - 1 + k
      float x[4], y[4];
      ld4s(f + 8 * G + 4, x);
      ld4s(f + 8 * G + 8, y);
      const float v[9] = {f[8 * G + 3], x[0], x[1], x[2], x[3], y[0], y[1], y[2], y[3]};
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fmaf(w, 0.25f * (v[2 * q] + v[2 * q + 2]) + 0.5f * v[2 * q + 1], acc[q]);
    }
    *reinterpret_cast<float4*>(coarse + ((long long)n * M + a) * Nc + (long long)(J0 + J) * gc.n0 + I0 + 4 * G) =
        make_float4(acc[0], acc[1], acc[2], acc[3]);
    if constexpr (START)  // the coarse tile, all planes, for the smoothing start (over cbar and the coupling plane)
      *reinterpret_cast<float4*>(&S.cb[0][0] + (a * (kFH / 2) + J) * (kFW / 2) + 4 * G) =
          make_float4(acc[0], acc[1], acc[2], acc[3]);
  }
  if constexpr (START) {
    __syncthreads();
    // y = F r per coarse point, then the zero-start iterate of each real
    // plane and complex pair (k_lin_residual4's arithmetic without e); four
    // coarse points per item
    const float* rc = &S.cb[0][0];
    for (int it = tid; it < (kFH / 2) * (kFW / 8); it += kThreads) {
      const int J = it >> 3, G = it & 7;
      const long long pt = (long long)(J0 + J) * gc.n0 + I0 + 4 * G, base_c = (long long)n * M * Nc + pt;
      float r[M][4], y[M][4], cb[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int b = 0; b < M; ++b) ld4s(rc + (b * (kFH / 2) + J) * (kFW / 2) + 4 * G, r[b]);
      if (cbarc) {
        const float4 c = *reinterpret_cast<const float4*>(cbarc + (long long)n * Nc + pt);
        cb[0] = c.x; cb[1] = c.y; cb[2] = c.z; cb[3] = c.w;
      }
#pragma unroll
      for (int a = 0; a < M; ++a) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float t = 0.f;
#pragma unroll
          for (int b = 0; b < M; ++b) t = fmaf(ss.F[a][b], r[b][q], t);
          y[a][q] = t;
        }
        *reinterpret_cast<float4*>(ss.y + base_c + (long long)a * Nc) = make_float4(y[a][0], y[a][1], y[a][2], y[a][3]);
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
                     ss.k2 + cb[q], ss.omega, zr[q], zi[q]);
          *reinterpret_cast<float4*>(ss.z + base_c + (long long)pl * Nc) = make_float4(zr[0], zr[1], zr[2], zr[3]);
          if (kd == SH_RE && pl + 1 < M)
            *reinterpret_cast<float4*>(ss.z + base_c + (long long)pi * Nc) = make_float4(zi[0], zi[1], zi[2], zi[3]);
        }
      }
    }
  }
}

int g_lr_ready = 0;  // 1 once the shared-memory opt-in is set

}  // namespace

void linres_restrict_prepare() {
  static std::once_flag once;
  std::call_once(once, [] {
    bool ok = true;
    auto opt_in = [&ok](auto kernel, size_t bytes) {
      ok = ok && cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess;
    };
    opt_in(k_linres_restrict<3, false>, sizeof(LRSmem<3>));
    opt_in(k_linres_restrict<3, true>, sizeof(LRSmem<3>));
    opt_in(k_linres_restrict<5, false>, sizeof(LRSmem<5>));
    opt_in(k_linres_restrict<5, true>, sizeof(LRSmem<5>));
    cudaGetLastError();  // without the opt-in the two steps stay separate launches
    g_lr_ready = ok ? 1 : 0;
  });
}

bool launch_linres_restrict(int D, const LinParams<float>& p, const GridP& gc, float* coarse, cudaStream_t st,
                            const SmoothStart* ss, const float* cbarc, bool* started) {
  if (started) *started = false;
  if (g_lr_ready != 1) return false;
  if (!(D == 2 && (p.M == 3 || p.M == 5) && !p.transpose && !p.transform && p.e && p.r && !p.cnode &&
        p.g.bc == BC_PER && p.g.n0 >= kFW && p.g.n0 % kFW == 0 && p.g.n1 >= kFH && p.g.n1 % kFH == 0 &&
        gc.bc == BC_PER && gc.n0 * 2 == p.g.n0 && gc.n1 * 2 == p.g.n1 && aligned16(p.e) && aligned16(p.r) &&
        aligned16(p.cbar) && aligned16(coarse)))
    return false;
  const long long nb = (long long)(p.g.n0 / kFW) * (p.g.n1 / kFH) * p.Nt;
  if (nb >= 0x7fffffffLL) return false;
  const bool start = ss && ss->y && ss->z && aligned16(ss->y) && aligned16(ss->z) && aligned16(cbarc);
  SmoothStart s{};
  if (start) s = *ss;
#define LR(MM)                                                                                            \
  do {                                                                                                    \
    if (start)                                                                                            \
      st_launch(k_linres_restrict<MM, true>, (unsigned)nb, kThreads, sizeof(LRSmem<MM>), st, p, gc, coarse, s, \
                cbarc);                                                                                   \
    else                                                                                                  \
      st_launch(k_linres_restrict<MM, false>, (unsigned)nb, kThreads, sizeof(LRSmem<MM>), st, p, gc, coarse, s, \
                cbarc);                                                                                   \
  } while (0)
  if (p.M == 3) LR(3);
  else LR(5);
#undef LR
  if (started) *started = start;
  return true;
}

}  // namespace st
