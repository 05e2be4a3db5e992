// Double-float arithmetic on the FP32 pipes for the FP64-accurate fine
// residual: error-free transformations and the split of a double into two
// floats.  Shared by the kernels of k_fine.cu and k_fine_tile.cu.
#pragma once

#include "st_kernels.cuh"

namespace st {

// A value is an unevaluated sum hi + lo of two floats (about 48 significant
// bits).  Error-free transformations: Knuth's TwoSum, Dekker's FastTwoSum and
// the FMA-based exact product error (Dekker 1971); additions use the "sloppy"
// double-float add whose error is bounded by a few 2^-48 times the operands'
// magnitudes, which is the scale the residual tolerance is stated in.
struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
// a * c with c = chi + clo
__device__ __forceinline__ ff ff_mul_c(ff a, float chi, float clo) {
  const float p = a.hi * chi;
  float e = fmaf(a.hi, chi, -p);
  e = fmaf(a.hi, clo, e);
  e = fmaf(a.lo, chi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) { return ff_mul_c(a, b.hi, b.lo); }
// acc + a * c
__device__ __forceinline__ ff ff_madd_c(ff acc, ff a, float chi, float clo) {
  const float p = a.hi * chi;
  float e = fmaf(a.hi, chi, -p);
  e = fmaf(a.hi, clo, e);
  e = fmaf(a.lo, chi, e);
  const ff s = two_sum(acc.hi, p);
  return fast_two_sum(s.hi, s.lo + (acc.lo + e));
}

// Split a double into hi + lo floats with integer operations only: hi keeps
// the leading 24 significant bits (truncated), lo the next 29 bits rounded to
// 24.  Magnitudes below 2^-126 become 0 and lo is dropped below 2^-74; both
// are far below the residual's rounding level for O(1) data; infinities and
// NaNs stay infinities and NaNs.
__device__ __forceinline__ ff split_double(double u) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(u);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const int e = (int)((hw >> 20) & 0x7ffu);
  const unsigned sign = hw & 0x80000000u;
  const unsigned hb = sign | ((unsigned)(e - 896) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29);
  float hi = (e >= 897) ? __uint_as_float(hb) : 0.0f;
  if (e > 1150) {  // beyond the float range: infinity, or NaN for a NaN input
    const bool nan = (e == 2047) && (((hw & 0xfffffu) | lw) != 0u);
    return {__uint_as_float(nan ? 0x7fc00000u : (sign | 0x7f800000u)), 0.0f};
  }
  const float scale = __uint_as_float((unsigned)max(e - 948, 0) << 23);  // 2^(e-1075), 0 if subnormal
  float lo = __uint2float_rn(lw & 0x1fffffffu) * scale;
  lo = (e >= 949) ? lo : 0.0f;
  return {hi, sign ? -lo : lo};
}

struct FFC {
  float hi, lo;
};
struct ResidFF {
  FFC cx, cy, cz, k2, rho, w[MAXM][MAXM];
  float rho32;
};

// k_fine_tile.cu: the variant for 2D periodic grids in whole 64 x 16 tiles
// (M = 3 or 5, 16-byte aligned arrays); false / 0 where it does not apply.
// With ss (float residual written, cbar written when there is a reaction
// term) it also writes the smoothing start.
bool launch_residual_tile(int D, const ResidParams& p, const ResidFF& c, cudaStream_t st, const SmoothStart* ss);
long long residual_tile_blocks(int D, const ResidParams& p);
bool residual_tile_start_ok(int D, const ResidParams& p, const SmoothStart* ss);

}  // namespace st
