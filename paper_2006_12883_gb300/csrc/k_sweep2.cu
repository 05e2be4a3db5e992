// The last two Jacobi sweeps of a depth-capped slab solve in one kernel
// (2D periodic grids in whole 64 x 8 tiles, M = 3 or 5, FP32): the sweep
// z -> z' and the sweep z' -> z'' fused with the back-transform and the
// damped block-Jacobi update of e, e = (e_zero ? 0 : e) + omega_bt B z''.
// The separate kernels stream z, y and cbar twice and z' out and back in;
// here a block brings z with a two-point halo, y and cbar with a one-point
// halo into shared memory (cp.async copies, all of a thread's copies in
// flight at once), computes z' on the tile and its one-point ring into
// registers, writes it over z once every thread has read z, and computes the
// second sweep on the tile: 16.8 instead of 29.6 bytes per dof at M = 5.
// Tiles of 64 x 8 with z' over z take 35 KB of shared memory at M = 5 (five
// blocks per SM) and 22 KB at M = 3 (seven); a separate z' buffer (four
// blocks) and 64 x 16 tiles (two blocks) measured slower.  The arithmetic is
// that of k_inner4's sweep (k_level4.cu), term for term, so the result
// equals the two-launch sequence.
#include <mutex>

#include "st_kernels.cuh"

namespace st {

namespace {

constexpr int kW = 64;            // tile width (x points)
// Plane pattern of the Q eigenbasis at odd M (the setup orders the real
// eigenvalue first, then the conjugate pairs): plane 0 real, planes 1-2 and
// 3-4 complex pairs.  The launcher checks it.
__host__ __device__ constexpr bool lead_plane(int q) { return q == 0 || (q & 1); }
__host__ __device__ constexpr int plane_kind(int q) { return q == 0 ? SH_REAL : ((q & 1) ? SH_RE : SH_IM); }
constexpr int kTH = 8;            // tile height (rows)
constexpr int kS = 72;            // shared row stride: columns -4..67, the tile's at 4..67

// shared planes of a tile of kH rows: z rows -2..kH+1, y and cbar rows
// -1..kH (the first sweep's result z' replaces z in place, rows -1..kH, once
// every thread has read z)
template <int M, int kH>
struct Sweep2Smem {
  static constexpr int kZR = kH + 4, kYR = kH + 2;
  float z[M][kZR][kS];
  float y[M][kYR][kS];
  float cb[kYR][kS];
};

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(__cvta_generic_to_global(src))
               : "memory");
}

// One damped Jacobi update at NQ points of one real plane (kd == SH_REAL:
// the r-arrays) or of one complex pair (kd == SH_RE: planes r and i), from
// the centre values z, the right-hand sides y, the sums of the two x and the
// two y neighbours and cbar: k_inner4's arithmetic, in its order, with the
// update itself in jac_real / jac_cplx as there.
template <int NQ>
__device__ __forceinline__ void jacobi_pair(const InnerParams<float>& p, int kd, float sr, float si,
                                            const float (&zr)[NQ], const float (&yr)[NQ], const float (&sxr)[NQ],
                                            const float (&syr)[NQ], const float (&zi)[NQ], const float (&yi)[NQ],
                                            const float (&sxi)[NQ], const float (&syi)[NQ], const float (&cb)[NQ],
                                            float (&outr)[NQ], float (&outi)[NQ]) {
  float Lr[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    Lr[q] = cb[q] * zr[q];
    Lr[q] = fmaf(p.sc.k2, zr[q], Lr[q]);
    Lr[q] = fmaf(p.sc.cx, sxr[q], Lr[q]);
    Lr[q] = fmaf(p.sc.cy, syr[q], Lr[q]);
  }
  if (kd == SH_REAL) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) outr[q] = jac_real(yr[q], zr[q], Lr[q], sr, p.omega, p.sc.k2 + cb[q]);
    return;
  }
  float Li[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    Li[q] = cb[q] * zi[q];
    Li[q] = fmaf(p.sc.k2, zi[q], Li[q]);
    Li[q] = fmaf(p.sc.cx, sxi[q], Li[q]);
    Li[q] = fmaf(p.sc.cy, syi[q], Li[q]);
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q)
    jac_cplx(yr[q], yi[q], zr[q], zi[q], Lr[q], Li[q], sr, si, p.omega, p.sc.k2 + cb[q], outr[q], outi[q]);
}

__device__ __forceinline__ void ld4s(const float* s, float (&v)[4]) {
  const float4 a = *reinterpret_cast<const float4*>(s);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}

// The operands of one plane at a group of 4 points (shared column c0, a
// multiple of 4): centre, y, x-neighbour sums, y-neighbour sums; zc is the
// centre row of the plane's z (or z') in shared memory, zu / zd the rows
// above and below, yrow the plane's y row.
__device__ __forceinline__ void group_operands(const float* zc, const float* zu, const float* zd,
                                               const float* yrow, int c0, float (&z)[4], float (&y)[4],
                                               float (&sx)[4], float (&sy)[4]) {
  ld4s(zc + c0, z);
  ld4s(yrow + c0, y);
  float u[4], d[4];
  ld4s(zu + c0, u);
  ld4s(zd + c0, d);
  const float v[6] = {zc[c0 - 1], z[0], z[1], z[2], z[3], zc[c0 + 4]};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    sx[q] = v[q] + v[q + 2];
    sy[q] = u[q] + d[q];
  }
}

// one thread per group of 4 points of the first sweep's region (rows -1..kH)
template <int kH>
__host__ __device__ constexpr int sweep2_threads() { return (kH + 2) * 16; }

// The update U += e' of the defect correction from the float e' of the
// tile's points, as k_update4 does it (float to double by bit
// manipulation, one FP64 add).
__device__ __forceinline__ double f2d(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned sign = b & 0x80000000u, ex = (b >> 23) & 0xffu, man = b & 0x7fffffu;
  const unsigned hi = (ex == 0u) ? sign : sign | ((ex == 0xffu ? 0x7ffu : ex + 896u) << 20) | (man >> 3);
  const unsigned lo = (ex == 0u) ? 0u : (man << 29);
  return __hiloint2double((int)hi, (int)lo);
}

// UPD: the epilogue also adds e' to the FP64 iterate (*p.Uslot) and writes e
// only if p.write_e: the step's update of U done by the cycle's last kernel.
template <int M, int kH, bool UPD>
__global__ void __launch_bounds__(sweep2_threads<kH>(), M == 3 ? 7 : 5) k_sweep2(InnerParams<float> p) {
  grid_dep_wait();
  constexpr int kZR = kH + 4, kYR = kH + 2, kThreads = sweep2_threads<kH>();
  extern __shared__ __align__(16) unsigned char smraw[];
  Sweep2Smem<M, kH>& S = *reinterpret_cast<Sweep2Smem<M, kH>*>(smraw);
  const int tid = threadIdx.x;
  const int nx = p.g.n0, ny = p.g.n1;
  const long long Ns = p.g.Ns;
  const int ntx = nx / kW;
  const int per_slab = ntx * (ny / kH);
  const int tile = (int)(blockIdx.x % (unsigned)per_slab), n = (int)(blockIdx.x / (unsigned)per_slab);
  const int j0 = (tile / ntx) * kH, i0 = (tile % ntx) * kW;
  const long long base = (long long)n * M * Ns;
  auto row = [&](int r) -> long long {  // periodic row r of the tile (r may be -2..kH+1)
    int j = j0 + r;
    j = j < 0 ? j + ny : (j >= ny ? j - ny : j);
    return (long long)j * nx;
  };
  const bool has_cb = p.cbar != nullptr;
  // every copy of the block in flight at once; a thread takes fixed (row,
  // column group) slots and walks the planes.  The halo columns come in the
  // aligned 16-byte groups that hold them (columns -4..-1 and 64..67).
  const int cl = i0 == 0 ? nx - 4 : i0 - 4, cr = i0 + kW == nx ? 0 : i0 + kW;
  for (int sl = tid; sl < kZR * 18; sl += kThreads) {  // z: rows -2..kH+1, groups -1..16
    const int r = sl / 18, g = sl - r * 18;
    const int gc = g == 0 ? cl : (g == 17 ? cr : i0 + 4 * (g - 1));
    const float* src = p.z + base + row(r - 2) + gc;
    float* dst = &S.z[0][r][4 * g];
#pragma unroll
    for (int pl = 0; pl < M; ++pl) cp_async16(dst + pl * (kZR * kS), src + pl * Ns);
  }
  for (int sl = tid; sl < kYR * 18; sl += kThreads) {  // y: rows -1..kH, groups -1..16
    const int r = sl / 18, g = sl - r * 18;
    const int gc = g == 0 ? cl : (g == 17 ? cr : i0 + 4 * (g - 1));
    const float* src = p.y + base + row(r - 1) + gc;
    float* dst = &S.y[0][r][4 * g];
#pragma unroll
    for (int pl = 0; pl < M; ++pl) cp_async16(dst + pl * (kYR * kS), src + pl * Ns);
    if (has_cb) cp_async16(&S.cb[r][4 * g], p.cbar + (long long)n * Ns + row(r - 1) + gc);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  // the e of the tile's thread (4 points of tile row ty, every plane), for the epilogue
  const bool in_tile = tid < kH * 16;
  const int ty = tid >> 4, tx = tid & 15;
  const long long own = base + (in_tile ? row(ty) : 0) + i0 + 4 * tx;
  float4 e0[M];
#pragma unroll
  for (int a = 0; a < M; ++a)
    e0[a] = (p.e_zero || !in_tile) ? make_float4(0.f, 0.f, 0.f, 0.f)
                                   : *reinterpret_cast<const float4*>(p.e + own + a * Ns);
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();

  // first sweep on rows -1..kH: thread tid takes the group of 4 points at
  // shared row r (tile row r - 1) and columns c0..c0+3
  // (held in registers until every thread has read z)
  const int r1 = tid >> 4, c1 = 4 + 4 * (tid & 15);
  float z1g[M][4];
  {
    const int r = r1, c0 = c1;
    float cb[4] = {0.f, 0.f, 0.f, 0.f};
    if (has_cb) ld4s(&S.cb[r][c0], cb);
#pragma unroll
    for (int pl = 0; pl < M; ++pl) {
      if (!lead_plane(pl)) continue;
      const int kd = plane_kind(pl);
      const int pi = pl + 1 < M ? pl + 1 : pl;
      float zr[4], yr[4], sxr[4], syr[4], zi[4], yi[4], sxi[4], syi[4];
      group_operands(S.z[pl][r + 1], S.z[pl][r], S.z[pl][r + 2], S.y[pl][r], c0, zr, yr, sxr, syr);
      if (kd == SH_RE) group_operands(S.z[pi][r + 1], S.z[pi][r], S.z[pi][r + 2], S.y[pi][r], c0, zi, yi, sxi, syi);
      jacobi_pair<4>(p, kd, p.sh.sr[pl], p.sh.si[pl], zr, yr, sxr, syr, zi, yi, sxi, syi, cb, z1g[pl], z1g[pi]);
    }
  }
  // first sweep at the ring's columns -1 and 64 of rows -1..kH: one item per
  // (point, real plane or complex pair), spread over the block
  constexpr int np = (M + 1) / 2;  // the real plane and the pairs
  static_assert(kYR * 2 * np <= kThreads, "one ring item per thread at most");
  const bool ring = tid < kYR * 2 * np;
  float ring_r = 0.f, ring_i = 0.f;
  int ring_pl = 0, ring_pi = 0, ring_row = 0, ring_col = 0;
  {
    for (int item = tid; item < kYR * 2 * np; item += kThreads) {
      const int pt = item % (kYR * 2), k = item / (kYR * 2);
      const int r = pt >> 1, c = 4 + ((pt & 1) ? kW : -1);
      const int pl = k == 0 ? 0 : 2 * k - 1;  // the k-th leading plane
      const int kd = pl == 0 ? SH_REAL : SH_RE;
      const int pi = pl + 1 < M ? pl + 1 : pl;
      float cb[1] = {has_cb ? S.cb[r][c] : 0.f};
      float zr[1] = {S.z[pl][r + 1][c]}, yr[1] = {S.y[pl][r][c]};
      float sxr[1] = {S.z[pl][r + 1][c - 1] + S.z[pl][r + 1][c + 1]}, syr[1] = {S.z[pl][r][c] + S.z[pl][r + 2][c]};
      float zi[1] = {S.z[pi][r + 1][c]}, yi[1] = {S.y[pi][r][c]};
      float sxi[1] = {S.z[pi][r + 1][c - 1] + S.z[pi][r + 1][c + 1]}, syi[1] = {S.z[pi][r][c] + S.z[pi][r + 2][c]};
      float outr[1], outi[1];
      jacobi_pair<1>(p, kd, p.sh.sr[pl], p.sh.si[pl], zr, yr, sxr, syr, zi, yi, sxi, syi, cb, outr, outi);
      ring_r = outr[0];
      ring_i = outi[0];
      ring_pl = pl;
      ring_pi = kd == SH_RE ? pi : -1;
      ring_row = r;
      ring_col = c;
    }
  }
  __syncthreads();
  // z' over z: z' row r (tile row r - 1) at z row r + 1, same columns
#pragma unroll
  for (int pl = 0; pl < M; ++pl)
    *reinterpret_cast<float4*>(&S.z[pl][r1 + 1][c1]) = make_float4(z1g[pl][0], z1g[pl][1], z1g[pl][2], z1g[pl][3]);
  if (ring) {
    S.z[ring_pl][ring_row + 1][ring_col] = ring_r;
    if (ring_pi >= 0) S.z[ring_pi][ring_row + 1][ring_col] = ring_i;
  }
  __syncthreads();

  // second sweep on the tile, fused with the back-transform and the update of e
  float evs[UPD ? M : 1][4];
  if (in_tile) {
    const int r = ty + 1, c0 = 4 + 4 * tx;
    float cb[4] = {0.f, 0.f, 0.f, 0.f};
    if (has_cb) ld4s(&S.cb[r][c0], cb);
    float out[M][4];
#pragma unroll
    for (int pl = 0; pl < M; ++pl) {
      if (!lead_plane(pl)) continue;
      const int kd = plane_kind(pl);
      const int pi = pl + 1 < M ? pl + 1 : pl;
      float zr[4], yr[4], sxr[4], syr[4], zi[4], yi[4], sxi[4], syi[4];
      group_operands(S.z[pl][r + 1], S.z[pl][r], S.z[pl][r + 2], S.y[pl][r], c0, zr, yr, sxr, syr);
      if (kd == SH_RE) group_operands(S.z[pi][r + 1], S.z[pi][r], S.z[pi][r + 2], S.y[pi][r], c0, zi, yi, sxi, syi);
      jacobi_pair<4>(p, kd, p.sh.sr[pl], p.sh.si[pl], zr, yr, sxr, syr, zi, yi, sxi, syi, cb, out[pl], out[pi]);
    }
#pragma unroll
    for (int a = 0; a < M; ++a) {
      float ev[4] = {e0[a].x, e0[a].y, e0[a].z, e0[a].w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float acc = 0.f;
#pragma unroll
        for (int b = 0; b < M; ++b) acc = fmaf(p.B[a][b], out[b][q], acc);
        ev[q] = fmaf(p.omega_bt, acc, ev[q]);
      }
      if constexpr (UPD) {
#pragma unroll
        for (int q = 0; q < 4; ++q) evs[a][q] = ev[q];
      } else {
        *reinterpret_cast<float4*>(p.e + own + a * Ns) = make_float4(ev[0], ev[1], ev[2], ev[3]);
      }
    }
  }
  if constexpr (UPD) {
    // e' to shared memory over z (once every thread has read z'), then
    // U += e' on the tile: every thread, two points per item, the loads of U
    // of all its items issued first
    __syncthreads();
    if (in_tile) {
#pragma unroll
      for (int a = 0; a < M; ++a)
        *reinterpret_cast<float4*>(&S.z[0][0][0] + (a * kH + ty) * kW + 4 * tx) =
            make_float4(evs[a][0], evs[a][1], evs[a][2], evs[a][3]);
    }
    __syncthreads();
    double* __restrict__ U = *p.Uslot;
    constexpr int kItems = M * kH * (kW / 2), kPer = (kItems + kThreads - 1) / kThreads;
    double2 u[kPer];
    long long off[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int it = tid + j * kThreads;
      off[j] = 0;
      if (it < kItems) {
        const int a = it / (kH * (kW / 2)), rem = it - a * (kH * (kW / 2)), r = rem / (kW / 2), c2 = rem - r * (kW / 2);
        off[j] = base + (long long)a * Ns + row(r) + i0 + 2 * c2;
        u[j] = *reinterpret_cast<const double2*>(U + off[j]);
      }
    }
    const float* et = &S.z[0][0][0];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int it = tid + j * kThreads;
      if (it < kItems) {
        const float2 ev = *reinterpret_cast<const float2*>(et + 2 * it);
        u[j].x += f2d(ev.x);
        u[j].y += f2d(ev.y);
        *reinterpret_cast<double2*>(U + off[j]) = u[j];
        if (p.write_e) *reinterpret_cast<float2*>(p.e + off[j]) = ev;
      }
    }
  }
}

__global__ void k_set_uslot(double** slot, double* U) { *slot = U; }

int g_sweep2_ready = 0;  // 1 once the shared-memory opt-in is set

}  // namespace

void sweep2_prepare() {
  static std::once_flag once;
  std::call_once(once, [] {
    bool ok = true;
    auto opt_in = [&ok](auto kernel, size_t bytes) {
      ok = ok && cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess;
    };
    opt_in(k_sweep2<3, kTH, false>, sizeof(Sweep2Smem<3, kTH>));
    opt_in(k_sweep2<3, kTH, true>, sizeof(Sweep2Smem<3, kTH>));
    opt_in(k_sweep2<5, kTH, false>, sizeof(Sweep2Smem<5, kTH>));
    opt_in(k_sweep2<5, kTH, true>, sizeof(Sweep2Smem<5, kTH>));
    cudaGetLastError();  // without the opt-in the two sweeps stay separate launches
    g_sweep2_ready = ok ? 1 : 0;
  });
}

bool launch_sweep2(int D, const InnerParams<float>& p, cudaStream_t st) {
  if (g_sweep2_ready != 1) return false;
  for (int q = 0; q < p.P; ++q)
    if (p.sh.kind[q] != plane_kind(q)) return false;  // the compiled plane pattern
  if (!(D == 2 && (p.P == 3 || p.P == 5) && p.g.bc == BC_PER && p.g.n0 >= kW && p.g.n0 % kW == 0 &&
        p.g.n1 >= kTH && p.g.n1 % kTH == 0 && p.fuse_bt && p.e && aligned16(p.z) && aligned16(p.y) &&
        aligned16(p.e) && aligned16(p.cbar)))
    return false;
  const long long nb = (long long)(p.g.n0 / kW) * (p.g.n1 / kTH) * p.Nt;
  if (nb >= 0x7fffffffLL) return false;
  constexpr int nt = sweep2_threads<kTH>();
  const bool upd = p.Uslot != nullptr;
  if (p.P == 3) {
    if (upd) st_launch(k_sweep2<3, kTH, true>, (unsigned)nb, nt, sizeof(Sweep2Smem<3, kTH>), st, p);
    else st_launch(k_sweep2<3, kTH, false>, (unsigned)nb, nt, sizeof(Sweep2Smem<3, kTH>), st, p);
  } else {
    if (upd) st_launch(k_sweep2<5, kTH, true>, (unsigned)nb, nt, sizeof(Sweep2Smem<5, kTH>), st, p);
    else st_launch(k_sweep2<5, kTH, false>, (unsigned)nb, nt, sizeof(Sweep2Smem<5, kTH>), st, p);
  }
  return true;
}

// a plain launch (no programmatic serialisation): the cycle that reads the
// slot follows it in stream order
void launch_set_uslot(double** slot, double* U, cudaStream_t st) { k_set_uslot<<<1, 1, 0, st>>>(slot, U); }

}  // namespace st
