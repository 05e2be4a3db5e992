// TMA-staged level kernels on 2D periodic grids (x size a multiple of 64, y
// size a multiple of 16, M = 3, FP32; at M = 5 two stages of a tile take a
// block's shared memory, and the direct float4 kernels that issue all of a
// thread's loads up front are faster):
//  * k_jacobi_tma (M = 3): the Jacobi sweep of the Q-diagonalised slab
//    systems that also updates e (the last of a slab solve), the same
//    arithmetic as k_inner4<2, 3, 2> in k_level4.cu, with the operands of a 64 x 16 tile
//    (z, y, e of every plane and cbar) brought into shared memory by
//    cp.async.bulk.tensor copies and the one-point halo of z by plain loads;
//  * k_linres_tma: the level residual with e (and the eigenbasis transform),
//    e, r, cbar and the previous slab's last node plane staged the same way.
// A persistent grid (two blocks per SM) walks the tiles with two stages: the
// copies of the next tile are in flight while the current one is computed.
// Every wait on a stage's mbarrier is bounded; on expiry the block counts the
// event in a device counter (read back with the norms), stops computing and
// returns after waiting, again bounded, for its copies in flight.
// k_wait_expiry exercises that path on purpose (a wait nothing completes)
// for the self-check st_wait_selftest.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "st_kernels.cuh"

namespace st {

__device__ int g_tma_error = 0;  // count of expired waits (never reset)

namespace {

constexpr int kTW = 64;           // tile width (x points)
constexpr int kTH = 16;           // tile height (rows)
constexpr int kStages = 2;
constexpr int kMinTilesPerBlock = 1;
constexpr int kSpinLimit = 1 << 24;  // mbarrier polls (about a second with the back-off) before giving up

struct TmaMaps {
  CUtensorMap z, y, e, cb;
};

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// non-blocking test of the phase with the given parity
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait; false on expiry
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  for (int i = 0; i < kSpinLimit; ++i) {
    if (mbar_test(bar, parity)) return true;
    if (i > 256) __nanosleep(64);
  }
  return false;
}

__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* map, int x, int y, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_addr(dst)), "l"(map), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

template <int M>
struct TileSmem {
  float z[kStages][M][kTH][kTW];
  float y[kStages][M][kTH][kTW];
  float e[kStages][M][kTH][kTW];
  float cb[kStages][kTH][kTW];
  float zrow[kStages][M][2][kTW];   // rows above and below the tile
  float zcol[kStages][M][kTH][2];   // columns left and right of the tile
  unsigned long long bar[kStages];
};

template <int M>
__global__ void __launch_bounds__(256, 2) k_jacobi_tma(const __grid_constant__ TmaMaps maps, InnerParams<float> p) {
  grid_dep_wait();
  extern __shared__ __align__(128) unsigned char smraw[];
  TileSmem<M>& S = *reinterpret_cast<TileSmem<M>*>(smraw);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int n0 = p.g.n0, n1 = p.g.n1;
  const long long Ns = p.g.Ns;
  const int ntx = n0 / kTW, nty = n1 / kTH;
  const int per_slab = ntx * nty;
  const int ntiles = per_slab * p.Nt;
  const bool has_e = p.fuse_bt && !p.e_zero;
  const bool has_cb = p.cbar != nullptr;
  const unsigned bytes = (unsigned)(kTH * kTW * 4) * (2 * M + (has_e ? M : 0) + (has_cb ? 1 : 0));
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&S.bar[s]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int t, int s) {  // one thread: the copies of tile t into stage s
    const int n = t / per_slab, r = t - n * per_slab;
    const int j0 = (r / ntx) * kTH, i0 = (r % ntx) * kTW;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect(&S.bar[s], bytes);
    for (int pl = 0; pl < M; ++pl) {
      const int row = (n * M + pl) * n1 + j0;
      tma_2d(&S.z[s][pl][0][0], &maps.z, i0, row, &S.bar[s]);
      tma_2d(&S.y[s][pl][0][0], &maps.y, i0, row, &S.bar[s]);
      if (has_e) tma_2d(&S.e[s][pl][0][0], &maps.e, i0, row, &S.bar[s]);
    }
    if (has_cb) tma_2d(&S.cb[s][0][0], &maps.cb, i0, n * n1 + j0, &S.bar[s]);
  };
  // the one-point halo of z of tile t (periodic wrap): this thread's values
  constexpr int kHaloRow = M * 2 * kTW, kHalo = kHaloRow + M * kTH * 2;
  constexpr int kPer = (kHalo + 255) / 256;
  auto halo_load = [&](int t, float v[kPer]) {
    const int n = t / per_slab, r = t - n * per_slab;
    const int j0 = (r / ntx) * kTH, i0 = (r % ntx) * kTW;
    const int jn = (j0 == 0 ? n1 : j0) - 1, js = (j0 + kTH == n1) ? 0 : j0 + kTH;
    const int il = (i0 == 0 ? n0 : i0) - 1, ir = (i0 + kTW == n0) ? 0 : i0 + kTW;
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int q = threadIdx.x + 256 * u;
      if (q < kHaloRow) {
        const int pl = q / (2 * kTW), side = (q / kTW) & 1, x = q % kTW;
        v[u] = p.z[((long long)n * M + pl) * Ns + (long long)(side ? js : jn) * n0 + i0 + x];
      } else if (q < kHalo) {
        const int qq = q - kHaloRow;
        const int pl = qq / (2 * kTH), row = (qq >> 1) % kTH, side = qq & 1;
        v[u] = p.z[((long long)n * M + pl) * Ns + (long long)(j0 + row) * n0 + (side ? ir : il)];
      }
    }
  };
  auto halo_store = [&](int s, const float v[kPer]) {
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int q = threadIdx.x + 256 * u;
      if (q < kHaloRow) {
        const int pl = q / (2 * kTW), side = (q / kTW) & 1, x = q % kTW;
        S.zrow[s][pl][side][x] = v[u];
      } else if (q < kHalo) {
        const int qq = q - kHaloRow;
        const int pl = qq / (2 * kTH), row = (qq >> 1) % kTH, side = qq & 1;
        S.zcol[s][pl][row][side] = v[u];
      }
    }
  };
  float hv[kPer];
  if (threadIdx.x == 0 && (int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
  if ((int)blockIdx.x < ntiles) {
    halo_load(blockIdx.x, hv);
    halo_store(0, hv);
  }
  bool failed = false;
  int it = 0;
  int t = blockIdx.x;
  for (; t < ntiles; t += gridDim.x, ++it) {
    const int s = it & 1;
    const int tn = t + gridDim.x;
    if (threadIdx.x == 0 && tn < ntiles) issue(tn, s ^ 1);
    if (tn < ntiles) halo_load(tn, hv);  // in flight while this tile is computed
    const int n = t / per_slab, r = t - n * per_slab;
    const int j0 = (r / ntx) * kTH, i0 = (r % ntx) * kTW;
    if (!mbar_wait(&S.bar[s], (unsigned)((it >> 1) & 1))) {
      failed = true;
      if (threadIdx.x == 0) atomicAdd(&g_tma_error, 1);
    }
    __syncthreads();
    if (__syncthreads_or(failed)) break;
    const int c0 = 4 * tx;
    float cb[4] = {0.f, 0.f, 0.f, 0.f};
    if (has_cb) {
      const float4 v = *reinterpret_cast<const float4*>(&S.cb[s][ty][c0]);
      cb[0] = v.x; cb[1] = v.y; cb[2] = v.z; cb[3] = v.w;
    }
    float out[M][4];
    auto lap = [&](int pl, const float zc[4], float acc[4]) {
      const float xl = tx == 0 ? S.zcol[s][pl][ty][0] : S.z[s][pl][ty][c0 - 1];
      const float xr = tx == 15 ? S.zcol[s][pl][ty][1] : S.z[s][pl][ty][c0 + 4];
      const float v[6] = {xl, zc[0], zc[1], zc[2], zc[3], xr};
      const float4 lo = ty == 0 ? *reinterpret_cast<const float4*>(&S.zrow[s][pl][0][c0])
                                : *reinterpret_cast<const float4*>(&S.z[s][pl][ty - 1][c0]);
      const float4 hi = ty == kTH - 1 ? *reinterpret_cast<const float4*>(&S.zrow[s][pl][1][c0])
                                      : *reinterpret_cast<const float4*>(&S.z[s][pl][ty + 1][c0]);
      const float lv[4] = {lo.x, lo.y, lo.z, lo.w}, hv[4] = {hi.x, hi.y, hi.z, hi.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[q] = fmaf(p.sc.k2, zc[q], acc[q]);
        acc[q] = fmaf(p.sc.cx, v[q] + v[q + 2], acc[q]);
        acc[q] = fmaf(p.sc.cy, lv[q] + hv[q], acc[q]);
      }
    };
#pragma unroll
    for (int pl = 0; pl < M; ++pl) {
      const int kd = p.sh.kind[pl];
      if (kd == SH_REAL || kd == SH_RE) {
        const float sr = p.sh.sr[pl], si = p.sh.si[pl];
        float zr[4], yr[4], Lr[4];
        {
          const float4 a = *reinterpret_cast<const float4*>(&S.z[s][pl][ty][c0]);
          const float4 b = *reinterpret_cast<const float4*>(&S.y[s][pl][ty][c0]);
          zr[0] = a.x; zr[1] = a.y; zr[2] = a.z; zr[3] = a.w;
          yr[0] = b.x; yr[1] = b.y; yr[2] = b.z; yr[3] = b.w;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) Lr[q] = cb[q] * zr[q];
        lap(pl, zr, Lr);
        if (kd == SH_REAL) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            out[pl][q] = jac_real(yr[q], zr[q], Lr[q], sr, p.omega, p.sc.k2 + cb[q]);
          }
        } else if (pl + 1 < M) {
          const int pi = pl + 1 < M ? pl + 1 : pl;
          float zi[4], yi[4], Li[4];
          {
            const float4 a = *reinterpret_cast<const float4*>(&S.z[s][pi][ty][c0]);
            const float4 b = *reinterpret_cast<const float4*>(&S.y[s][pi][ty][c0]);
            zi[0] = a.x; zi[1] = a.y; zi[2] = a.z; zi[3] = a.w;
            yi[0] = b.x; yi[1] = b.y; yi[2] = b.z; yi[3] = b.w;
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) Li[q] = cb[q] * zi[q];
          lap(pi, zi, Li);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            jac_cplx(yr[q], yi[q], zr[q], zi[q], Lr[q], Li[q], sr, si, p.omega, p.sc.k2 + cb[q], out[pl][q],
                     out[pi][q]);
          }
        }
      }
    }
    const long long base = (long long)n * M * Ns + (long long)(j0 + ty) * n0 + i0 + c0;
    if (!p.fuse_bt) {
#pragma unroll
      for (int pl = 0; pl < M; ++pl)
        *reinterpret_cast<float4*>(p.zout + base + (long long)pl * Ns) =
            make_float4(out[pl][0], out[pl][1], out[pl][2], out[pl][3]);
    } else {
#pragma unroll
      for (int a = 0; a < M; ++a) {
        float ev[4] = {0.f, 0.f, 0.f, 0.f};
        if (has_e) {
          const float4 v = *reinterpret_cast<const float4*>(&S.e[s][a][ty][c0]);
          ev[0] = v.x; ev[1] = v.y; ev[2] = v.z; ev[3] = v.w;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float acc = 0.f;
#pragma unroll
          for (int b = 0; b < M; ++b) acc = fmaf(p.B[a][b], out[b][q], acc);
          ev[q] = fmaf(p.omega_bt, acc, ev[q]);
        }
        *reinterpret_cast<float4*>(p.e + base + (long long)a * Ns) = make_float4(ev[0], ev[1], ev[2], ev[3]);
      }
    }
    if (tn < ntiles) halo_store(s ^ 1, hv);
    __syncthreads();  // stage s is free again, the next halo is in place
  }
  if (failed && threadIdx.x == 0) {
    // let the copies still in flight (this tile's and, if issued, the next
    // one's) land before the block exits; bounded
    mbar_wait(&S.bar[it & 1], (unsigned)((it >> 1) & 1));
    if (t + (int)gridDim.x < ntiles) mbar_wait(&S.bar[(it + 1) & 1], (unsigned)(((it + 1) >> 1) & 1));
  }
}

// ---------------------------------------------------------------------------
// The level residual r - A e + C e (forward) with the Q-eigenbasis transform
// and the optional zero-start Jacobi iterate (or without the transform), as
// k_lin_residual4<2, M> computes it, with e, r, cbar and the previous slab's
// last node plane of e staged by TMA copies and the halo of e prefetched.
// ---------------------------------------------------------------------------
struct LinMaps {
  CUtensorMap e, r, cb, out;
};

template <int M>
struct LinSmem {
  float e[kStages][M][kTH][kTW];
  float r[kStages][M][kTH][kTW];
  float ep[kStages][kTH][kTW];     // last node of the previous slab (coupling)
  float cb[kStages][kTH][kTW];
  float erow[kStages][M][2][kTW];
  float ecol[kStages][M][kTH][2];
  unsigned long long bar[kStages];
};

template <int M>
__global__ void __launch_bounds__(256, 2) k_linres_tma(const __grid_constant__ LinMaps maps, LinParams<float> p) {
  grid_dep_wait();
  extern __shared__ __align__(128) unsigned char smraw[];
  LinSmem<M>& S = *reinterpret_cast<LinSmem<M>*>(smraw);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int n0 = p.g.n0, n1 = p.g.n1;
  const long long Ns = p.g.Ns;
  const int ntx = n0 / kTW, nty = n1 / kTH;
  const int per_slab = ntx * nty;
  const int ntiles = per_slab * p.Nt;
  const bool has_cb = p.cbar != nullptr;
  auto tile_bytes = [&](int n) {
    return (unsigned)(kTH * kTW * 4) * (2 * M + (n > 0 ? 1 : 0) + (has_cb ? 1 : 0));
  };
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&S.bar[s]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int t, int s) {
    const int n = t / per_slab, r = t - n * per_slab;
    const int j0 = (r / ntx) * kTH, i0 = (r % ntx) * kTW;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect(&S.bar[s], tile_bytes(n));
    for (int pl = 0; pl < M; ++pl) {
      const int row = (n * M + pl) * n1 + j0;
      tma_2d(&S.e[s][pl][0][0], &maps.e, i0, row, &S.bar[s]);
      tma_2d(&S.r[s][pl][0][0], &maps.r, i0, row, &S.bar[s]);
    }
    if (n > 0) tma_2d(&S.ep[s][0][0], &maps.e, i0, ((n - 1) * M + (M - 1)) * n1 + j0, &S.bar[s]);
    if (has_cb) tma_2d(&S.cb[s][0][0], &maps.cb, i0, n * n1 + j0, &S.bar[s]);
  };
  constexpr int kHaloRow = M * 2 * kTW, kHalo = kHaloRow + M * kTH * 2;
  constexpr int kPer = (kHalo + 255) / 256;
  auto halo_load = [&](int t, float v[kPer]) {
    const int n = t / per_slab, r = t - n * per_slab;
    const int j0 = (r / ntx) * kTH, i0 = (r % ntx) * kTW;
    const int jn = (j0 == 0 ? n1 : j0) - 1, js = (j0 + kTH == n1) ? 0 : j0 + kTH;
    const int il = (i0 == 0 ? n0 : i0) - 1, ir = (i0 + kTW == n0) ? 0 : i0 + kTW;
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int q = threadIdx.x + 256 * u;
      if (q < kHaloRow) {
        const int pl = q / (2 * kTW), side = (q / kTW) & 1, x = q % kTW;
        v[u] = p.e[((long long)n * M + pl) * Ns + (long long)(side ? js : jn) * n0 + i0 + x];
      } else if (q < kHalo) {
        const int qq = q - kHaloRow;
        const int pl = qq / (2 * kTH), row = (qq >> 1) % kTH, side = qq & 1;
        v[u] = p.e[((long long)n * M + pl) * Ns + (long long)(j0 + row) * n0 + (side ? ir : il)];
      }
    }
  };
  auto halo_store = [&](int s, const float v[kPer]) {
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int q = threadIdx.x + 256 * u;
      if (q < kHaloRow) {
        const int pl = q / (2 * kTW), side = (q / kTW) & 1, x = q % kTW;
        S.erow[s][pl][side][x] = v[u];
      } else if (q < kHalo) {
        const int qq = q - kHaloRow;
        const int pl = qq / (2 * kTH), row = (qq >> 1) % kTH, side = qq & 1;
        S.ecol[s][pl][row][side] = v[u];
      }
    }
  };
  float hv[kPer];
  if (threadIdx.x == 0 && (int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
  if ((int)blockIdx.x < ntiles) {
    halo_load(blockIdx.x, hv);
    halo_store(0, hv);
  }
  bool failed = false;
  int it = 0;
  int t = blockIdx.x;
  for (; t < ntiles; t += gridDim.x, ++it) {
    const int s = it & 1;
    const int tn = t + gridDim.x;
    if (threadIdx.x == 0 && tn < ntiles) issue(tn, s ^ 1);
    if (tn < ntiles) halo_load(tn, hv);
    const int n = t / per_slab, r = t - n * per_slab;
    const int j0 = (r / ntx) * kTH, i0 = (r % ntx) * kTW;
    if (!mbar_wait(&S.bar[s], (unsigned)((it >> 1) & 1))) {
      failed = true;
      if (threadIdx.x == 0) atomicAdd(&g_tma_error, 1);
    }
    __syncthreads();
    if (__syncthreads_or(failed)) break;
    const int c0 = 4 * tx;
    auto ld = [](const float* a, float v[4]) {
      const float4 x = *reinterpret_cast<const float4*>(a);
      v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    };
    float cb[4] = {0.f, 0.f, 0.f, 0.f}, carry[4] = {0.f, 0.f, 0.f, 0.f};
    if (has_cb) ld(&S.cb[s][ty][c0], cb);
    if (n > 0) ld(&S.ep[s][ty][c0], carry);
    float ev[M][4], Fe[M][4];
#pragma unroll
    for (int b = 0; b < M; ++b) {
      ld(&S.e[s][b][ty][c0], ev[b]);
      const float xl = tx == 0 ? S.ecol[s][b][ty][0] : S.e[s][b][ty][c0 - 1];
      const float xr = tx == 15 ? S.ecol[s][b][ty][1] : S.e[s][b][ty][c0 + 4];
      const float v[6] = {xl, ev[b][0], ev[b][1], ev[b][2], ev[b][3], xr};
      float lo[4], hi[4];
      ld(ty == 0 ? &S.erow[s][b][0][c0] : &S.e[s][b][ty - 1][c0], lo);
      ld(ty == kTH - 1 ? &S.erow[s][b][1][c0] : &S.e[s][b][ty + 1][c0], hi);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        Fe[b][q] = cb[q] * ev[b][q];
        Fe[b][q] = fmaf(p.sc.k2, ev[b][q], Fe[b][q]);
        Fe[b][q] = fmaf(p.sc.cx, v[q] + v[q + 2], Fe[b][q]);
        Fe[b][q] = fmaf(p.sc.cy, lo[q] + hi[q], Fe[b][q]);
      }
    }
    float res[M][4];
#pragma unroll
    for (int a = 0; a < M; ++a) {
      float r4[4];
      ld(&S.r[s][a][ty][c0], r4);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float acc = r4[q] - ev[a][q];
#pragma unroll
        for (int b = 0; b < M; ++b) acc = fmaf(p.W[a][b], Fe[b][q], acc);
        res[a][q] = acc + carry[q];
      }
    }
    const long long base = (long long)n * M * Ns + (long long)(j0 + ty) * n0 + i0 + c0;
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
        *reinterpret_cast<float4*>(p.out + base + (long long)a * Ns) = make_float4(y[a][0], y[a][1], y[a][2], y[a][3]);
      }
      if (p.zout) {
#pragma unroll
        for (int pl = 0; pl < M; ++pl) {
          const int kd = p.sh.kind[pl];
          if (kd == SH_REAL || kd == SH_RE) {
            const int pi = pl + 1 < M ? pl + 1 : pl;
            float zr[4], zi[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
              jac_zero(y[pl][q], kd == SH_REAL ? 0.f : y[pi][q], kd != SH_REAL, p.sh.sr[pl], p.sh.si[pl],
                       p.sc.k2 + cb[q], p.omega_j, zr[q], zi[q]);
            *reinterpret_cast<float4*>(p.zout + base + (long long)pl * Ns) = make_float4(zr[0], zr[1], zr[2], zr[3]);
            if (kd == SH_RE && pl + 1 < M)
              *reinterpret_cast<float4*>(p.zout + base + (long long)pi * Ns) =
                  make_float4(zi[0], zi[1], zi[2], zi[3]);
          }
        }
      }
    } else {
#pragma unroll
      for (int a = 0; a < M; ++a)
        *reinterpret_cast<float4*>(p.out + base + (long long)a * Ns) =
            make_float4(res[a][0], res[a][1], res[a][2], res[a][3]);
    }
    if (tn < ntiles) halo_store(s ^ 1, hv);
    __syncthreads();
  }
  if (failed && threadIdx.x == 0) {
    mbar_wait(&S.bar[it & 1], (unsigned)((it >> 1) & 1));
    if (t + (int)gridDim.x < ntiles) mbar_wait(&S.bar[(it + 1) & 1], (unsigned)(((it + 1) >> 1) & 1));
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
int g_resident[1] = {0};  // resident blocks of k_jacobi_tma<3> on the device
int g_resident_lin[1] = {0};  // resident blocks of k_linres_tma<3> on the device
std::mutex g_prepare_mu;

bool encode(CUtensorMap* map, const float* base, int n0, long long rows) {
  if (!g_encode || !base || rows >= (1ll << 31)) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)n0, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)n0 * sizeof(float)};
  const cuuint32_t box[2] = {kTW, kTH};
  const cuuint32_t estr[2] = {1, 1};
  return g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool jacobi_tma_ok(int D, const InnerParams<float>& p) {
  return D == 2 && p.P == 3 && p.g.bc == BC_PER && p.g.n0 % kTW == 0 && p.g.n1 % kTH == 0 &&
         aligned16(p.z) && aligned16(p.y) && (!p.fuse_bt || aligned16(p.e)) && (p.fuse_bt || aligned16(p.zout)) &&
         (!p.cbar || aligned16(p.cbar));
}

bool launch_jacobi_tma(int D, const InnerParams<float>& p, cudaStream_t st) {
  if (!jacobi_tma_ok(D, p)) return false;
  // measured: staging pays for the sweep that also reads and updates e (ten
  // tiles per stage); with seven the direct float4 loads are as fast.  At
  // M = 5 a block's two stages take 130 KB, one block per SM, and the direct
  // kernel with every load issued up front is faster (14.8 against 17.2 ms
  // on 1024^2 x 1024 slabs), so only M = 3 stages its tiles.
  if (!(p.fuse_bt && !p.e_zero) || p.P != 3) return false;
  TmaMaps m;
  memset(&m, 0, sizeof(m));
  const long long rows = (long long)p.Nt * p.P * p.g.n1;
  if (!encode(&m.z, p.z, p.g.n0, rows) || !encode(&m.y, p.y, p.g.n0, rows)) return false;
  if (p.fuse_bt && !p.e_zero && !encode(&m.e, p.e, p.g.n0, rows)) return false;
  if (p.cbar && !encode(&m.cb, p.cbar, p.g.n0, (long long)p.Nt * p.g.n1)) return false;
  if (g_resident[0] < 1) return false;  // tma_prepare not run or no room
  const long long ntiles = (long long)(p.g.n0 / kTW) * (p.g.n1 / kTH) * p.Nt;
  // the two-stage pipeline pays only when every block walks enough tiles
  if (ntiles < (long long)kMinTilesPerBlock * g_resident[0]) return false;
  // persistent grid: the resident blocks of every SM, no more than tiles
  const unsigned grid = (unsigned)std::min<long long>(ntiles, (long long)g_resident[0]);
  st_launch(k_jacobi_tma<3>, grid, 256, sizeof(TileSmem<3>), st, m, p);
  return true;
}

bool launch_linres_tma(int D, const LinParams<float>& p, cudaStream_t st) {
  // forward operator with e (the stencil variants), node-averaged cbar only;
  // M = 3 only: at M = 5 the direct float4 kernel with every load of a slab
  // issued up front is faster (11.2 against 12.2 ms on 1024^2 x 1024 slabs)
  if (!(D == 2 && p.M == 3 && p.g.bc == BC_PER && p.g.n0 % kTW == 0 && p.g.n1 % kTH == 0 &&
        p.e && !p.transpose && !p.cnode && aligned16(p.e) && aligned16(p.r) && aligned16(p.out) &&
        (!p.zout || aligned16(p.zout)) && (!p.cbar || aligned16(p.cbar))))
    return false;
  if (g_resident_lin[0] < 1) return false;
  const long long ntiles = (long long)(p.g.n0 / kTW) * (p.g.n1 / kTH) * p.Nt;
  if (ntiles < (long long)kMinTilesPerBlock * g_resident_lin[0]) return false;
  LinMaps m;
  memset(&m, 0, sizeof(m));
  const long long rows = (long long)p.Nt * p.M * p.g.n1;
  if (!encode(&m.e, p.e, p.g.n0, rows) || !encode(&m.r, p.r, p.g.n0, rows)) return false;
  if (p.cbar && !encode(&m.cb, p.cbar, p.g.n0, (long long)p.Nt * p.g.n1)) return false;
  const unsigned grid = (unsigned)std::min<long long>(ntiles, (long long)g_resident_lin[0]);
  st_launch(k_linres_tma<3>, grid, 256, sizeof(LinSmem<3>), st, m, p);
  return true;
}

void tma_prepare() {
  std::lock_guard<std::mutex> lock(g_prepare_mu);
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  auto setup = [&](auto kern, size_t sm) {
    int per_sm = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, sm) != cudaSuccess)
      per_sm = 0;
    return per_sm * sms;
  };
  g_resident[0] = setup(k_jacobi_tma<3>, sizeof(TileSmem<3>));
  g_resident_lin[0] = setup(k_linres_tma<3>, sizeof(LinSmem<3>));
  cudaGetLastError();  // a failed query leaves the TMA path off, not an error
}

// One block waiting on an mbarrier that no copy and no thread will complete:
// the bounded wait of the staged kernels expires, the expiry is counted as
// theirs are, and the block returns (nothing is in flight).
__global__ void k_wait_expiry() {
  __shared__ unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0u)) atomicAdd(&g_tma_error, 1);
}

void launch_wait_expiry(cudaStream_t st) { k_wait_expiry<<<1, 32, 0, st>>>(); }

int* tma_error_flag() {
  void* a = nullptr;
  if (cudaGetSymbolAddress(&a, g_tma_error) != cudaSuccess) return nullptr;
  return (int*)a;
}

}  // namespace st
