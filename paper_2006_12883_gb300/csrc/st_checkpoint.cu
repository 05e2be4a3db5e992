// Slab recomputation checkpointing for the adjoint (st_ckpt_* in st.h).
//
// The all-at-once system (Eq. 3.4) is block lower bidiagonal in time: slabs
// 1..K of the solution depend on u0 only, slabs K+1..2K on slab K's last
// node plane, and so on.  The forward pass therefore solves the Nt slabs in
// blocks of K with one K-slab handle, keeping only each block's initial
// plane.  The transposed system is block upper bidiagonal: a block's adjoint
// needs only its own U and the terminal data sum_m lambda_{first slab of the
// next block, m}, which is the derivative of the objective with respect to
// the next block's initial value - the du0 that block's adjoint solve
// returns.  The adjoint pass walks the blocks backward, recomputing each
// block's U from its initial plane before its adjoint solve; the parameter
// gradients are sums over the blocks.  Host code only: every step runs
// through the library's own entry points on the block handle.
#include <cmath>
#include <vector>

#include <cuda_runtime.h>

#include "st.h"

struct st_ckpt {
  st_handle* blk = nullptr;
  st_runtime rt{};
  cudaStream_t stream = nullptr;
  int Nt = 0, K = 0, B = 0, M = 0;
  long long Ns = 0;
  double* starts = nullptr;  // B planes: the initial value of each block (block 0: u0)
  double* Ublk = nullptr;    // K*M*Ns: the block iterate
  double* g = nullptr;       // Ns: terminal data of the block being solved backward
  double* du0 = nullptr;     // Ns: dPhi/d(initial value) of the last block solved
  bool forward_done = false;
  struct Buf {
    void* p;
    size_t bytes;
  };
  std::vector<Buf> bufs;
};

namespace {

int ck_alloc(st_ckpt* c, double** out, size_t bytes) {
  void* p = nullptr;
  if (c->rt.alloc) {
    p = c->rt.alloc(bytes, (void*)c->stream, c->rt.ctx);
  } else if (cudaMallocAsync(&p, bytes, c->stream) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (!p) return ST_ERR_OOM;
  c->bufs.push_back({p, bytes});
  *out = (double*)p;
  return ST_OK;
}

int copy(st_ckpt* c, void* dst, const void* src, size_t bytes) {
  if (cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream) != cudaSuccess) {
    cudaGetLastError();
    return ST_ERR_CUDA;
  }
  return ST_OK;
}

// U of block b from its initial plane (zero initial guess, as every solve)
int solve_block(st_ckpt* c, int b, st_solve_info* info) {
  // the plane may still be in flight on the stream; st_set_u0 reads it
  // with a synchronous copy
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaGetLastError();
    return ST_ERR_CUDA;
  }
  int s = st_set_u0(c->blk, c->starts + (long long)b * c->Ns);
  if (s != ST_OK) return s;
  if (cudaMemsetAsync(c->Ublk, 0, (size_t)c->K * c->M * c->Ns * sizeof(double), c->stream) != cudaSuccess) {
    cudaGetLastError();
    return ST_ERR_CUDA;
  }
  return st_solve(c->blk, c->Ublk, info);
}

void merge(st_solve_info* acc, const st_solve_info& b, bool first) {
  if (first) {
    *acc = b;
    return;
  }
  acc->iterations += b.iterations;
  acc->cycles += b.cycles;
  acc->seconds += b.seconds;
  acc->status = b.status;
  if (b.rel_residual > acc->rel_residual || !std::isfinite(b.rel_residual)) {
    acc->rel_residual = b.rel_residual;
    acc->abs_residual = b.abs_residual;
    acc->ref_norm = b.ref_norm;
  }
}

}  // namespace

extern "C" {

int st_ckpt_create(const st_problem* p, const st_solver_opts* o, const st_runtime* rt, st_ckpt** out) {
  if (!out) return ST_ERR_INVALID_ARG;
  *out = nullptr;
  if (!p || !o || !p->u0 || p->Nt < 1 || o->recompute_slabs < 1 || p->Nt % o->recompute_slabs != 0)
    return ST_ERR_INVALID_ARG;
  st_ckpt* c = new st_ckpt();
  if (rt) c->rt = *rt;
  c->stream = (cudaStream_t)c->rt.stream;
  c->Nt = p->Nt;
  c->K = o->recompute_slabs;
  c->B = p->Nt / c->K;
  c->M = p->M;
  c->Ns = 1;
  for (int a = 0; a < p->d && a < 3; ++a) c->Ns *= p->n[a];
  st_problem pb = *p;
  pb.Nt = c->K;
  pb.T = p->T * (double)c->K / (double)p->Nt;
  int s = st_create(&pb, o, rt, &c->blk);
  if (s == ST_OK) s = ck_alloc(c, &c->starts, (size_t)c->B * c->Ns * sizeof(double));
  if (s == ST_OK) s = ck_alloc(c, &c->Ublk, (size_t)c->K * c->M * c->Ns * sizeof(double));
  if (s == ST_OK) s = ck_alloc(c, &c->g, (size_t)c->Ns * sizeof(double));
  if (s == ST_OK) s = ck_alloc(c, &c->du0, (size_t)c->Ns * sizeof(double));
  if (s == ST_OK) s = copy(c, c->starts, p->u0, (size_t)c->Ns * sizeof(double));
  if (s == ST_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaGetLastError();
    s = ST_ERR_CUDA;
  }
  if (s != ST_OK) {
    st_ckpt_destroy(c);
    return s;
  }
  *out = c;
  return ST_OK;
}

int st_ckpt_set_params(st_ckpt* c, double nu, double rho) {
  if (!c) return ST_ERR_INVALID_ARG;
  c->forward_done = false;
  return st_set_params(c->blk, nu, rho);
}

int st_ckpt_set_u0(st_ckpt* c, const double* u0) {
  if (!c || !u0) return ST_ERR_INVALID_ARG;
  c->forward_done = false;
  int s = copy(c, c->starts, u0, (size_t)c->Ns * sizeof(double));
  if (s == ST_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaGetLastError();
    s = ST_ERR_CUDA;
  }
  return s;
}

int st_ckpt_forward(st_ckpt* c, double* uT, st_solve_info* info) {
  if (!c) return ST_ERR_INVALID_ARG;
  c->forward_done = false;
  st_solve_info acc{}, ib{};
  const long long last = ((long long)(c->K - 1) * c->M + (c->M - 1)) * c->Ns;
  int s = ST_OK;
  for (int b = 0; b < c->B; ++b) {
    s = solve_block(c, b, &ib);
    merge(&acc, ib, b == 0);
    if (s != ST_OK) break;
    double* dst = (b + 1 < c->B) ? c->starts + (long long)(b + 1) * c->Ns : uT;
    if (dst && (s = copy(c, dst, c->Ublk + last, (size_t)c->Ns * sizeof(double))) != ST_OK) break;
  }
  if (s == ST_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaGetLastError();
    s = ST_ERR_CUDA;
  }
  acc.status = s;
  if (info) *info = acc;
  c->forward_done = (s == ST_OK);
  return s;
}

int st_ckpt_adjoint(st_ckpt* c, const double* gT, double* dnu, double* drho, double* du0, st_solve_info* info) {
  if (!c || !gT || !c->forward_done) return ST_ERR_INVALID_ARG;
  int s = copy(c, c->g, gT, (size_t)c->Ns * sizeof(double));
  double snu = 0.0, srho = 0.0;
  st_solve_info acc{}, ib{};
  bool first = true;
  for (int b = c->B - 1; b >= 0 && s == ST_OK; --b) {
    s = solve_block(c, b, &ib);  // recompute the block's U
    if (s != ST_OK) {
      merge(&acc, ib, first);
      break;
    }
    double bn = 0.0, br = 0.0;
    s = st_adjoint_solve_terminal(c->blk, c->Ublk, c->g, &bn, &br, c->du0, &ib);
    merge(&acc, ib, first);
    first = false;
    if (s != ST_OK) break;
    snu += bn;
    srho += br;
    // the terminal data of the block before: dPhi/d(this block's initial value)
    if (b > 0) s = copy(c, c->g, c->du0, (size_t)c->Ns * sizeof(double));
  }
  if (s == ST_OK && du0) s = copy(c, du0, c->du0, (size_t)c->Ns * sizeof(double));
  if (s == ST_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaGetLastError();
    s = ST_ERR_CUDA;
  }
  acc.status = s;
  if (info) *info = acc;
  if (s == ST_OK) {
    if (dnu) *dnu = snu;
    if (drho) *drho = srho;
  }
  return s;
}

void st_ckpt_destroy(st_ckpt* c) {
  if (!c) return;
  for (const auto& b : c->bufs) {
    if (c->rt.free) c->rt.free(b.p, b.bytes, (void*)c->stream, c->rt.ctx);
    else cudaFreeAsync(b.p, c->stream);
  }
  c->bufs.clear();
  st_destroy(c->blk);
  delete c;
}

}  // extern "C"
