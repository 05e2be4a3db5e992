// Vector kernels of the Krylov-accelerated Newton step: batched dot products
// with a fixed block-to-data mapping (deterministic FP64 sums of FP32 or FP64
// vectors), multi-axpy and scaled copies.  All vectors are contiguous, n
// values each; a basis of k vectors is one allocation with stride n.
#include "st_kernels.cuh"

namespace st {

namespace {

constexpr int kDotThreads = 256;
constexpr int kDotGroup = 8;  // vectors per dot launch

// partial[i * nblocks + b] = sum over block b's slice of w * V_i (i < g).
template <typename T, int G>
__global__ void __launch_bounds__(kDotThreads) k_mdot(const T* __restrict__ w, const T* __restrict__ V,
                                                      long long stride, int g, long long n, double* partial) {
  grid_dep_wait();
  double acc[G];
#pragma unroll
  for (int i = 0; i < G; ++i) acc[i] = 0.0;
  const long long step = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += step) {
    const double we = (double)w[e];
#pragma unroll
    for (int i = 0; i < G; ++i)
      if (i < g) acc[i] = fma(we, (double)V[i * stride + e], acc[i]);
  }
  __shared__ double red[kDotThreads / 32][G];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < G; ++i) {
    double v = acc[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[wid][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < G && threadIdx.x < g) {
    double s = 0.0;
    for (int q = 0; q < kDotThreads / 32; ++q) s += red[q][threadIdx.x];
    partial[(long long)threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
}

// out[i] = sum_b partial[i * nb + b], one block per row, fixed order.
__global__ void __launch_bounds__(256) k_sum_rows(const double* __restrict__ partial, int nb, double* out) {
  grid_dep_wait();
  __shared__ double red[256];
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += partial[(long long)blockIdx.x * nb + b];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// w -= sum_i c_i V_i
template <typename T>
__global__ void __launch_bounds__(256) k_maxpy(T* __restrict__ w, const T* __restrict__ V, long long stride,
                                               KrylovCoef c, long long n) {
  grid_dep_wait();
  const long long step = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += step) {
    double s = (double)w[e];
    for (int i = 0; i < c.k; ++i) s = fma(-c.c[i], (double)V[i * stride + e], s);
    w[e] = (T)s;
  }
}

// y = a x + b y  (b == 0: y = a x, y not read)
template <typename T>
__global__ void __launch_bounds__(256) k_axpby(T* __restrict__ y, const T* __restrict__ x, double a, double b,
                                               long long n) {
  grid_dep_wait();
  const long long step = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += step) {
    const double v = a * (double)x[e];
    y[e] = (T)(b == 0.0 ? v : fma(b, (double)y[e], v));
  }
}

unsigned stream_blocks(long long n) {
  // a fixed count (a multiple of the SM count), so the dot-product partition
  // and hence the rounding of the sums depend on n only
  const long long want = (n + 255) / 256;
  return (unsigned)std::max<long long>(1, std::min<long long>(want, 152 * 8));
}

}  // namespace

long long krylov_partials(long long n) { return (long long)stream_blocks(n) * kDotGroup; }

void launch_mdot(int fp64, const void* w, const void* V, long long stride, int k, long long n, double* partial,
                 double* out, cudaStream_t st) {
  const unsigned nb = stream_blocks(n);
  for (int i0 = 0; i0 < k; i0 += kDotGroup) {
    const int g = std::min(kDotGroup, k - i0);
    if (fp64)
      st_launch(k_mdot<double, kDotGroup>, nb, kDotThreads, 0, st, (const double*)w,
                (const double*)V + i0 * stride, stride, g, n, partial);
    else
      st_launch(k_mdot<float, kDotGroup>, nb, kDotThreads, 0, st, (const float*)w, (const float*)V + i0 * stride,
                stride, g, n, partial);
    st_launch(k_sum_rows, (unsigned)g, 256, 0, st, (const double*)partial, (int)nb, out + i0);
  }
}

void launch_maxpy(int fp64, void* w, const void* V, long long stride, const KrylovCoef& c, long long n,
                  cudaStream_t st) {
  const unsigned nb = stream_blocks(n);
  if (fp64) st_launch(k_maxpy<double>, nb, 256, 0, st, (double*)w, (const double*)V, stride, c, n);
  else st_launch(k_maxpy<float>, nb, 256, 0, st, (float*)w, (const float*)V, stride, c, n);
}

void launch_axpby(int fp64, void* y, const void* x, double a, double b, long long n, cudaStream_t st) {
  const unsigned nb = stream_blocks(n);
  if (fp64) st_launch(k_axpby<double>, nb, 256, 0, st, (double*)y, (const double*)x, a, b, n);
  else st_launch(k_axpby<float>, nb, 256, 0, st, (float*)y, (const float*)x, a, b, n);
}

}  // namespace st
