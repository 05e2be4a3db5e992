// Allocation-free variant of the FP64 residual-and-norm computation.
//
// st_residual normally runs inside a handle whose workspace st_create
// allocates; its norm needs a scratch buffer for the per-block partial sums.
// Some callers cannot allocate device memory at the point where they want a
// residual norm: code that runs inside another framework's memory manager
// with a fixed budget (every byte already owned by its pool), code called
// from within an allocator callback, or latency-critical loops that must not
// hit cudaMalloc's implicit synchronisation.  st_residual_noalloc serves
// them: its scratch is a fixed file-scope device array, so the call itself
// allocates nothing.
#include <cmath>

#include "st_kernels.cuh"
#include "st_setup.h"

namespace {

// Scratch: up to kMaxBlocks per-block partial sums plus one result slot
// (2 MiB + 8 bytes).  Every GPU that loads the library holds it until exit.
constexpr long long kMaxBlocks = 1LL << 18;
static __device__ __align__(256) double g_scratch[kMaxBlocks + 1];

// Device address of the scratch array in the current device's context.  In
// host code the array's name is only a host-side stand-in, so the address is
// looked up on every call with the caller's device current: the lookup is
// cheap, and an address cached across calls would go stale if the context
// were torn down and the module loaded again at another address.
int scratch_address(double** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return ST_ERR_CUDA;
  }
  *out = (double*)p;
  return ST_OK;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int st_residual_noalloc(const st_problem* p, const double* U, double* R, double* norm_out,
                                   void* stream) {
  using namespace st;
  if (!p || !U || !p->u0) return ST_ERR_INVALID_ARG;
  if (p->d < 1 || p->d > 3 || p->bc < 0 || p->bc > 2 || p->reaction < 0 || p->reaction > 2) return ST_ERR_INVALID_ARG;
  if (p->Nt < 1 || p->M < 1 || p->M > ST_MAX_M || !(p->nu > 0) || !(p->T > 0) || !(p->X > 0))
    return ST_ERR_INVALID_ARG;
  long long Ns = 1;
  for (int a = 0; a < p->d; ++a) {
    if (p->n[a] < 1 || (p->bc == ST_BC_NEUMANN && p->n[a] < 2)) return ST_ERR_INVALID_ARG;
    Ns *= p->n[a];
  }
  if (Ns * (long long)p->Nt >= 0x7fffffffLL) return ST_ERR_UNSUPPORTED;
  if (!on_device(U) || !on_device(p->u0) || (R && !on_device(R))) return ST_ERR_INVALID_ARG;
  Colloc col;
  if (colloc_setup(p->M, &col) != 0) return ST_ERR_UNSUPPORTED;

  ResidParams rp;
  rp.g = make_grid(p->d, p->n, p->bc, p->X);
  rp.Nt = p->Nt;
  rp.M = p->M;
  // one partial sum per block of 256 (point, slab-run) pairs: lengthen the
  // slab runs until the partial sums fit the scratch array
  rp.chunk = 1;
  while ((Ns * ((p->Nt + rp.chunk - 1) / rp.chunk) + 255) / 256 > kMaxBlocks && rp.chunk < p->Nt) rp.chunk *= 2;
  rp.nchunks = (p->Nt + rp.chunk - 1) / rp.chunk;
  const long long nblocks = residual_blocks(rp);
  if (nblocks > kMaxBlocks) return ST_ERR_UNSUPPORTED;  // a plane of more than 2^26 points
  const double dt = p->T / p->Nt;
  for (int a = 0; a < MAXM; ++a)
    for (int b = 0; b < MAXM; ++b) rp.dtq[a][b] = (a < p->M && b < p->M) ? dt * col.Q[a][b] : 0.0;
  rp.nu = p->nu;
  rp.rho = p->rho;
  rp.reaction = p->reaction;
  rp.sc.cx = p->nu * rp.g.ih2[0];
  rp.sc.cy = p->nu * rp.g.ih2[1];
  rp.sc.cz = p->nu * rp.g.ih2[2];
  rp.sc.k2 = -2.0 * p->nu * (rp.g.ih2[0] + rp.g.ih2[1] + rp.g.ih2[2]);
  rp.U = U;
  rp.u0 = p->u0;
  rp.lam = nullptr;
  rp.gT = nullptr;
  rp.R = R;
  rp.cbar = nullptr;
  rp.cnode = nullptr;
  rp.tau = nullptr;
  double* scratch = nullptr;
  int s = scratch_address(&scratch);
  if (s != ST_OK) return s;
  rp.partial = scratch;
  cudaStream_t st = (cudaStream_t)stream;
  launch_residual(p->d, 1, 1, rp, st);
  // every one of the nblocks partial slots is rewritten above, and the sum
  // kernel overwrites the result slot: nothing left from an earlier call is read
  launch_sum_partials(scratch, nblocks, scratch + kMaxBlocks, st);
  if (cudaGetLastError() != cudaSuccess) return ST_ERR_CUDA;
  if (norm_out) {
    double sq = 0.0;
    if (cudaMemcpyAsync(&sq, scratch + kMaxBlocks, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      return ST_ERR_CUDA;
    }
    *norm_out = std::sqrt(sq);
  }
  return ST_OK;
}
