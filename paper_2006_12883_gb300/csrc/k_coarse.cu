// Exact solve on the coarsest space-time level (replaces the LU of Section
// 4.2): the system A_n e_n - 1 (x) e_{n-1,M} = r_n is block lower
// bidiagonal, so it is solved by forward substitution over the slabs.  Each
// slab block A_n = I - dt Q (x) (nu Lap_c + diag cbar_n) is tiny (K = M*Nc
// unknowns) and is inverted once per linearisation.  The substitution only
// couples slabs through Nc values, so it runs in three launches:
//   (a) f_n = A_n^{-1} r_n                     all slabs in parallel
//   (b) in_{n+1} = f_{n,M} + W_{n,M} in_n      sequential, Nc values per step
//   (c) e_n = f_n + W_n in_n                   all slabs in parallel
// with W_n = A_n^{-1} (1 (x) I).  The transposed system (adjoint) runs the
// same scheme backward with A_n^{-T} and the coupling C^T.
#include "st_kernels.cuh"

namespace st {

// One block per slab: Gauss-Jordan with partial pivoting on [A | I] in
// shared memory (cycle precision T; the pivot search is a warp argmax), then
// the inverse and the coupling matrices.
template <typename T>
__global__ void __launch_bounds__(256) k_coarse_setup(CoarseParams<T> p) {
  grid_dep_wait();
  extern __shared__ unsigned char smraw[];
  T* A = reinterpret_cast<T*>(smraw);  // [K][2K]
  const int K = p.K, Nc = p.Nc, M = p.M;
  const int W2 = 2 * K;
  __shared__ int piv;
  const int n = blockIdx.x;
  for (int t = threadIdx.x; t < K * W2; t += blockDim.x) {
    const int r = t / W2, c = t % W2;
    double v;
    if (c < K) {
      const int m = r / Nc, pp = r % Nc, j = c / Nc, q = c % Nc;
      double lv = p.nu * p.Lc[pp * Nc + q];
      if (pp == q && p.cbar) lv += (double)p.cbar[(long long)n * Nc + pp];
      v = (r == c ? 1.0 : 0.0) - p.dtq[m][j] * lv;
    } else {
      v = (c - K == r) ? 1.0 : 0.0;
    }
    A[t] = (T)v;
  }
  __syncthreads();
  for (int col = 0; col < K; ++col) {
    if (threadIdx.x < 32) {
      int best = -1;
      T bv = (T)-1;
      for (int r = col + (int)threadIdx.x; r < K; r += 32) {
        const T v = fabs(A[r * W2 + col]);
        if (v > bv) { bv = v; best = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_down_sync(0xffffffffu, bv, o);
        const int ob = __shfl_down_sync(0xffffffffu, best, o);
        if (ov > bv || (ov == bv && ob >= 0 && (best < 0 || ob < best))) { bv = ov; best = ob; }
      }
      if (threadIdx.x == 0) piv = best < 0 ? col : best;
    }
    __syncthreads();
    const int pr = piv;
    if (pr != col) {
      for (int c = threadIdx.x; c < W2; c += blockDim.x) {
        const T t0 = A[col * W2 + c];
        A[col * W2 + c] = A[pr * W2 + c];
        A[pr * W2 + c] = t0;
      }
      __syncthreads();
    }
    const T inv = (T)1 / A[col * W2 + col];
    __syncthreads();
    for (int c = threadIdx.x; c < W2; c += blockDim.x) A[col * W2 + c] *= inv;
    __syncthreads();
    {
      // rows by warp, columns by lane: no per-element index division
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
      for (int r = warp; r < K; r += nw) {
        if (r == col) continue;
        const T f = A[r * W2 + col];
        for (int c = lane; c < W2; c += 32)
          if (c != col) A[r * W2 + c] -= f * A[col * W2 + c];
      }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < K; r += blockDim.x)
      if (r != col) A[r * W2 + col] = (T)0;
    __syncthreads();
  }
  // inverse is A[:, K:2K]
  T* Ai = p.Ainv + (long long)n * K * K;
  for (int t = threadIdx.x; t < K * K; t += blockDim.x) {
    const int r = t / K, c = t % K;
    Ai[t] = A[r * W2 + K + c];
  }
  // forward coupling W = Ainv (1 (x) I): W[r][q] = sum_m Ainv[r][m Nc + q]
  T* W = p.Wf + (long long)n * K * Nc;
  T* Wt = p.Wt + (long long)n * K * Nc;
  for (int t = threadIdx.x; t < K * Nc; t += blockDim.x) {
    const int r = t / Nc, q = t % Nc;
    T acc = (T)0;
    for (int m = 0; m < M; ++m) acc += A[r * W2 + K + m * Nc + q];
    W[t] = acc;
    // transposed coupling Wt = Ainv^T (e_M (x) I): Wt[r][q] = Ainv[(M-1)Nc+q][r]
    Wt[t] = A[((M - 1) * Nc + q) * W2 + K + r];
  }
  T* Wr = p.Wfrow + (long long)n * Nc * Nc;
  T* Wtr = p.Wtrow + (long long)n * Nc * Nc;
  for (int t = threadIdx.x; t < Nc * Nc; t += blockDim.x) {
    const int pp = t / Nc, q = t % Nc;
    T accf = (T)0, acct = (T)0;
    for (int m = 0; m < M; ++m) {
      accf += A[((M - 1) * Nc + pp) * W2 + K + m * Nc + q];  // W[(M-1)Nc+pp][q]
      acct += A[((M - 1) * Nc + q) * W2 + K + m * Nc + pp];  // sum_m Wt[m Nc+pp][q]
    }
    Wr[t] = accf;
    Wtr[t] = acct;
  }
}

// (a) e_n = A_n^{-1} r_n (or A_n^{-T} r_n)
template <typename T>
__global__ void __launch_bounds__(128) k_coarse_apply(CoarseParams<T> p, int transpose, const T* __restrict__ r,
                                                      T* __restrict__ e) {
  grid_dep_wait();
  const int n = blockIdx.x, K = p.K;
  const T* Ai = p.Ainv + (long long)n * K * K;
  const T* rn = r + (long long)n * K;
  for (int row = threadIdx.x; row < K; row += blockDim.x) {
    T acc = (T)0;
    if (!transpose)
      for (int c = 0; c < K; ++c) acc += Ai[row * K + c] * rn[c];
    else
      for (int c = 0; c < K; ++c) acc += Ai[c * K + row] * rn[c];
    e[(long long)n * K + row] = acc;
  }
}

// (b) sequential recurrence of the incoming coupling vectors in[n][Nc]
template <typename T>
__global__ void __launch_bounds__(128) k_coarse_recur(CoarseParams<T> p, int transpose, const T* __restrict__ f,
                                                      T* __restrict__ in) {
  grid_dep_wait();
  const int K = p.K, Nc = p.Nc, M = p.M, Nt = p.Nt;
  const int q = threadIdx.x;
  if (!transpose) {
    if (q < Nc) in[q] = (T)0;
    __syncthreads();
    for (int n = 0; n + 1 < Nt; ++n) {
      T v = (T)0;
      if (q < Nc) {
        const T* Wr = p.Wfrow + (long long)n * Nc * Nc;
        v = f[(long long)n * K + (M - 1) * Nc + q];
        for (int c = 0; c < Nc; ++c) v += Wr[q * Nc + c] * in[(long long)n * Nc + c];
      }
      __syncthreads();
      if (q < Nc) in[(long long)(n + 1) * Nc + q] = v;
      __syncthreads();
    }
  } else {
    if (q < Nc) in[(long long)(Nt - 1) * Nc + q] = (T)0;
    __syncthreads();
    for (int n = Nt - 1; n >= 1; --n) {
      T v = (T)0;
      if (q < Nc) {
        const T* Wr = p.Wtrow + (long long)n * Nc * Nc;
        for (int m = 0; m < M; ++m) v += f[(long long)n * K + m * Nc + q];
        for (int c = 0; c < Nc; ++c) v += Wr[q * Nc + c] * in[(long long)n * Nc + c];
      }
      __syncthreads();
      if (q < Nc) in[(long long)(n - 1) * Nc + q] = v;
      __syncthreads();
    }
  }
}

// (c) e_n += W_n in_n
template <typename T>
__global__ void __launch_bounds__(128) k_coarse_finish(CoarseParams<T> p, int transpose, const T* __restrict__ in,
                                                       T* __restrict__ e) {
  grid_dep_wait();
  const int n = blockIdx.x, K = p.K, Nc = p.Nc;
  const T* W = (transpose ? p.Wt : p.Wf) + (long long)n * K * Nc;
  const T* v = in + (long long)n * Nc;
  for (int row = threadIdx.x; row < K; row += blockDim.x) {
    T acc = (T)0;
    for (int c = 0; c < Nc; ++c) acc += W[row * Nc + c] * v[c];
    e[(long long)n * K + row] += acc;
  }
}

template <typename T>
size_t coarse_setup_smem(const CoarseParams<T>& p) {
  return (size_t)p.K * 2 * p.K * sizeof(T);
}

template <typename T>
cudaError_t prepare_coarse_setup(const CoarseParams<T>& p) {
  return cudaFuncSetAttribute(k_coarse_setup<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)coarse_setup_smem(p));
}

template <typename T>
void launch_coarse_setup(const CoarseParams<T>& p, cudaStream_t st) {
  st_launch(k_coarse_setup<T>, p.Nt, 256, coarse_setup_smem(p), st, p);
}

template <typename T>
void launch_coarse_solve(const CoarseParams<T>& p, int transpose, const T* r, T* e, T* in, cudaStream_t st) {
  st_launch(k_coarse_apply<T>, p.Nt, 128, 0, st, p, transpose, r, e);
  st_launch(k_coarse_recur<T>, 1, 128, 0, st, p, transpose, e, in);
  st_launch(k_coarse_finish<T>, p.Nt, 128, 0, st, p, transpose, in, e);
}

#define INSTC(T)                                                                       \
  template size_t coarse_setup_smem<T>(const CoarseParams<T>&);                        \
  template cudaError_t prepare_coarse_setup<T>(const CoarseParams<T>&);                \
  template void launch_coarse_setup<T>(const CoarseParams<T>&, cudaStream_t);          \
  template void launch_coarse_solve<T>(const CoarseParams<T>&, int, const T*, T*, T*, cudaStream_t);
INSTC(float)
INSTC(double)

}  // namespace st
