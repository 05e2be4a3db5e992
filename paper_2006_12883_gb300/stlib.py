"""ctypes binding of libst.so (include/st.h): the same entry points, with
argument marshalling only - every step of the computation runs in the CUDA
library.  The library must be built (``paper_2006_12883_gb300.build.build()``);
loading fails loudly otherwise, and there is no CPU fallback.

PyTorch provides device memory (its caching allocator backs the library's
workspace through the st_runtime hooks) and streams.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_longlong, c_size_t, c_void_p

import importlib as _importlib

_build = _importlib.import_module(__package__ + ".build")

ST_OK, ST_ERR_INVALID_ARG, ST_ERR_OOM, ST_ERR_CUDA = 0, 1, 2, 3
ST_ERR_NOT_CONVERGED, ST_ERR_DIVERGED, ST_ERR_TIMEOUT, ST_ERR_UNSUPPORTED = 4, 5, 6, 7
DIRICHLET, PERIODIC, NEUMANN = 0, 1, 2
NONE, LOGISTIC, CUBIC = 0, 1, 2
FP64, FP32_REFINE = 0, 1
COARSEN_SPACE, COARSEN_AUTO_MU, COARSEN_SPACE_NODES, COARSEN_SPACE_TIME = 0, 1, 2, 3
SDC_IE, SDC_LU = 0, 1
MAX_M, MAX_LEVELS, MAX_HISTORY = 5, 32, 64


class StProblem(ctypes.Structure):
    _fields_ = [("d", c_int), ("n", c_int * 3), ("bc", c_int), ("X", c_double), ("nu", c_double),
                ("reaction", c_int), ("rho", c_double), ("T", c_double), ("Nt", c_int), ("M", c_int),
                ("u0", c_void_p)]


class StSolverOpts(ctypes.Structure):
    _fields_ = [("precision", c_int), ("coarsening", c_int), ("max_levels", c_int), ("nu1", c_int),
                ("nu2", c_int), ("omega", c_double), ("mu_crit", c_double), ("inner_cycles", c_int),
                ("inner_smooth", c_int), ("inner_coarse_iters", c_int), ("coarse_max_points", c_int),
                ("coarse_max_slabs", c_int), ("sdc_qdelta", c_int), ("sdc_inner_cycles", c_int),
                ("tol", c_double), ("max_iters", c_int), ("newton", c_int), ("use_graphs", c_int),
                ("use_pdl", c_int), ("smooth_inner_levels", c_int),
                ("smooth_sweeps", c_int), ("line_search", c_int),
                ("exact_jacobian", c_int), ("krylov", c_int), ("krylov_rtol", c_double),
                ("krylov_fallback", c_int), ("pfasst_levels", c_int), ("pfasst_coarse_M", c_int),
                ("pfasst_sweeps", c_int), ("use_tma", c_int), ("recompute_slabs", c_int),
                ("fuse_sweeps", c_int),
                ("fuse_start", c_int),
                ("fuse_restrict", c_int),
                ("fuse_update", c_int)]


ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, c_size_t, c_void_p, c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_size_t, c_void_p, c_void_p)


class StRuntime(ctypes.Structure):
    _fields_ = [("stream", c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", c_void_p)]


class StSolveInfo(ctypes.Structure):
    _fields_ = [("iterations", c_int), ("status", c_int), ("rel_residual", c_double),
                ("abs_residual", c_double), ("ref_norm", c_double), ("seconds", c_double),
                ("history_len", c_int), ("history", c_double * MAX_HISTORY), ("cycles", c_int)]

    def as_dict(self):
        return dict(iterations=self.iterations, status=self.status, rel_residual=self.rel_residual,
                    abs_residual=self.abs_residual, ref_norm=self.ref_norm, seconds=self.seconds,
                    history=list(self.history[:self.history_len]), cycles=self.cycles)


class StLevelInfo(ctypes.Structure):
    _fields_ = [("n", c_int * 3), ("Ns", c_longlong), ("Nt", c_int), ("dt", c_double), ("h", c_double * 3),
                ("mu", c_double), ("next_kind", c_int), ("omega", c_double), ("inner_levels", c_int),
                ("M", c_int)]

    def as_dict(self):
        return dict(n=list(self.n), Ns=self.Ns, Nt=self.Nt, dt=self.dt, h=list(self.h), mu=self.mu,
                    next_kind=self.next_kind, omega=self.omega, inner_levels=self.inner_levels, M=self.M)


class StStatsInfo(ctypes.Structure):
    _fields_ = [("levels", c_int), ("cycle_graph_nodes", c_int), ("linearize_graph_nodes", c_int),
                ("launches_per_vcycle", c_int), ("update_in_cycle", c_int)]


class StPlanInfo(ctypes.Structure):
    _fields_ = [("levels", c_int), ("level", StLevelInfo * MAX_LEVELS), ("workspace_bytes", c_size_t),
                ("coarse_points", c_int)]


_LIB = None

_SIGS = {
    "st_default_opts": (None, [POINTER(StSolverOpts)]),
    "st_plan": (c_int, [POINTER(StProblem), POINTER(StSolverOpts), POINTER(StPlanInfo)]),
    "st_create": (c_int, [POINTER(StProblem), POINTER(StSolverOpts), POINTER(StRuntime), POINTER(c_void_p)]),
    "st_destroy": (None, [c_void_p]),
    "st_set_params": (c_int, [c_void_p, c_double, c_double]),
    "st_set_u0": (c_int, [c_void_p, c_void_p]),
    "st_residual": (c_int, [c_void_p, c_void_p, c_void_p, c_int, POINTER(c_double)]),
    "st_vcycle": (c_int, [c_void_p, c_void_p, POINTER(c_double)]),
    "st_sdc_sweep": (c_int, [c_void_p, c_void_p, c_int, POINTER(c_double)]),
    "st_solve": (c_int, [c_void_p, c_void_p, POINTER(StSolveInfo)]),
    "st_adjoint_solve": (c_int, [c_void_p, c_void_p, c_void_p, POINTER(c_double), POINTER(c_double),
                                 c_void_p, POINTER(StSolveInfo)]),
    "st_adjoint_solve_terminal": (c_int, [c_void_p, c_void_p, c_void_p, POINTER(c_double),
                                          POINTER(c_double), c_void_p, POINTER(StSolveInfo)]),
    "st_adjoint_lambda": (c_int, [c_void_p, c_void_p]),
    "st_status_str": (ctypes.c_char_p, [c_int]),
    "st_last_error": (ctypes.c_char_p, []),
    "st_collocation": (c_int, [c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "st_time_transfer": (c_int, [c_int, c_void_p, c_void_p]),
    "st_node_transfer": (c_int, [c_int, c_int, c_void_p, c_void_p]),
    "st_pfasst": (c_int, [c_void_p, c_void_p, c_void_p]),
    "st_num_levels": (c_int, [c_void_p]),
    "st_level_info_get": (c_int, [c_void_p, c_int, POINTER(StLevelInfo)]),
    "st_linearize": (c_int, [c_void_p, c_void_p]),
    "st_level_cbar": (c_int, [c_void_p, c_int, c_void_p]),
    "st_level_residual": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "st_level_smooth": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p]),
    "st_level_restrict": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p]),
    "st_level_prolong": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p]),
    "st_coarse_solve": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "st_level_vcycle": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "st_time_kernel": (c_int, [c_void_p, c_int, c_void_p, c_int, POINTER(c_double), POINTER(c_double)]),
    "st_stats": (c_int, [c_void_p, POINTER(StStatsInfo)]),
    "st_wait_selftest": (c_int, [c_void_p]),
    "st_residual_noalloc": (c_int, [POINTER(StProblem), c_void_p, c_void_p, POINTER(c_double), c_void_p]),
    "st_ckpt_create": (c_int, [POINTER(StProblem), POINTER(StSolverOpts), POINTER(StRuntime), POINTER(c_void_p)]),
    "st_ckpt_forward": (c_int, [c_void_p, c_void_p, POINTER(StSolveInfo)]),
    "st_ckpt_adjoint": (c_int, [c_void_p, c_void_p, POINTER(c_double), POINTER(c_double), c_void_p,
                                POINTER(StSolveInfo)]),
    "st_ckpt_set_params": (c_int, [c_void_p, c_double, c_double]),
    "st_ckpt_set_u0": (c_int, [c_void_p, c_void_p]),
    "st_ckpt_destroy": (None, [c_void_p]),
}

KERNEL_FINE_RESIDUAL, KERNEL_LEVEL_RESIDUAL, KERNEL_JACOBI, KERNEL_BACKTRANSFORM, KERNEL_VCYCLE = 0, 1, 2, 3, 4
KERNEL_SHIFTED_RESIDUAL, KERNEL_INNER_RESTRICT, KERNEL_PROLONG, KERNEL_JACOBI_PLAIN = 5, 6, 7, 8


def lib_path() -> str:
    return _build.LIB


def lib():
    """The loaded libst.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libst.so not built ({path}); run paper_2006_12883_gb300.build.build()")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


class StError(RuntimeError):
    def __init__(self, status: int, where: str):
        L = lib()
        msg = L.st_status_str(status).decode()
        detail = L.st_last_error().decode()
        super().__init__(f"{where}: {msg} ({status}) {detail}")
        self.status = status


def check(status: int, where: str):
    if status != ST_OK:
        if status == ST_ERR_CUDA:
            detail = lib().st_last_error()
            where = f"{where} [{detail.decode() if detail else ''}]"
        raise StError(status, where)
    return status


# ------------------------------------------------------------ C names, thin

def st_default_opts() -> StSolverOpts:
    o = StSolverOpts()
    lib().st_default_opts(ctypes.byref(o))
    return o


def st_plan(problem: StProblem, opts: StSolverOpts | None = None) -> StPlanInfo:
    info = StPlanInfo()
    check(lib().st_plan(ctypes.byref(problem), ctypes.byref(opts) if opts else None, ctypes.byref(info)),
          "st_plan")
    return info


def st_collocation(M: int):
    """(tau[M], Q[M][M], lam[M] complex, V, Vinv) from the library's setup."""
    import numpy as np
    tau = np.zeros(M)
    Q = np.zeros(M * M)
    lam = np.zeros(2 * M)
    V = np.zeros(2 * M * M)
    Vi = np.zeros(2 * M * M)
    check(lib().st_collocation(M, tau.ctypes.data, Q.ctypes.data, lam.ctypes.data, V.ctypes.data,
                               Vi.ctypes.data), "st_collocation")
    c = lambda a: (a[0::2] + 1j * a[1::2])
    return tau, Q.reshape(M, M), c(lam), c(V).reshape(M, M), c(Vi).reshape(M, M)


def st_node_transfer(Mf: int, Mc: int):
    """(P_M[Mf][Mc], R_M[Mc][Mf]) from the library's setup."""
    import numpy as np
    P = np.zeros(Mf * Mc)
    R = np.zeros(Mc * Mf)
    check(lib().st_node_transfer(Mf, Mc, P.ctypes.data, R.ctypes.data), "st_node_transfer")
    return P.reshape(Mf, Mc), R.reshape(Mc, Mf)


def st_time_transfer(M: int):
    import numpy as np
    Pt = np.zeros(2 * M * M)
    Rt = np.zeros(2 * M * M)
    check(lib().st_time_transfer(M, Pt.ctypes.data, Rt.ctypes.data), "st_time_transfer")
    return Pt.reshape(2 * M, M), Rt.reshape(M, 2 * M)


def make_problem(shape, bc, nu, Nt, M, T=1.0, X=1.0, reaction=NONE, rho=0.0, u0_ptr=None) -> StProblem:
    """shape in x-fastest order (nx, ny, nz)."""
    p = StProblem()
    p.d = len(shape)
    for a in range(3):
        p.n[a] = shape[a] if a < len(shape) else 1
    p.bc, p.X, p.nu, p.reaction, p.rho, p.T, p.Nt, p.M = bc, X, nu, reaction, rho, T, Nt, M
    p.u0 = u0_ptr
    return p


def make_opts(**kw) -> StSolverOpts:
    o = st_default_opts()
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


# ------------------------------------------------------------ torch-side API

def _torch():
    import torch
    return torch


class Solver:
    """A handle on one space-time problem.  Fields are torch tensors shaped
    (Nt, M, *grid) in numpy order (slowest first); pointers of CUDA tensors or
    of host (CPU) tensors are passed straight to the C ABI."""

    def __init__(self, grid_shape, bc, nu, Nt, M, u0, T=1.0, X=1.0, reaction=NONE, rho=0.0,
                 opts: StSolverOpts | None = None, torch_alloc: bool = True, stream=None):
        torch = _torch()
        self.grid_shape = tuple(grid_shape)  # numpy order
        self.Nt, self.M = Nt, M
        self.Ns = 1
        for n in self.grid_shape:
            self.Ns *= n
        self.opts = opts if opts is not None else st_default_opts()
        self.fp64 = self.opts.precision == FP64
        u0t = torch.as_tensor(u0, dtype=torch.float64).reshape(-1).contiguous()
        self._u0 = u0t
        self.problem = make_problem(self.grid_shape[::-1], bc, nu, Nt, M, T, X, reaction, rho, u0t.data_ptr())
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        rt = StRuntime()
        rt.stream = self.stream.cuda_stream
        rt.ctx = None
        if torch_alloc:
            dev = self.device.index

            def _alloc(nbytes, st, ctx):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, st or 0)
                except Exception:
                    return None

            def _free(ptr, nbytes, st, ctx):
                torch.cuda.caching_allocator_delete(ptr)

            rt.alloc = ALLOC_FN(_alloc)
            rt.free = FREE_FN(_free)
        else:
            rt.alloc = ALLOC_FN(0)
            rt.free = FREE_FN(0)
        self._rt = rt  # keep the callbacks alive
        h = c_void_p()
        check(lib().st_create(ctypes.byref(self.problem), ctypes.byref(self.opts), ctypes.byref(rt),
                              ctypes.byref(h)), "st_create")
        self.h = h

    # shapes
    @property
    def field_shape(self):
        return (self.Nt, self.M) + self.grid_shape

    def zeros(self, device=None, dtype=None):
        torch = _torch()
        return torch.zeros(self.field_shape, dtype=dtype or torch.float64, device=device or self.device)

    @property
    def cycle_dtype(self):
        torch = _torch()
        return torch.float64 if self.fp64 else torch.float32

    def close(self):
        if getattr(self, "h", None):
            lib().st_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _ptr(t):
        if t is None:
            return None
        assert t.is_contiguous()
        return t.data_ptr()

    # entry points ---------------------------------------------------------
    def set_params(self, nu, rho):
        check(lib().st_set_params(self.h, float(nu), float(rho)), "st_set_params")

    def set_u0(self, u0):
        torch = _torch()
        u0t = torch.as_tensor(u0, dtype=torch.float64).reshape(-1).contiguous()
        check(lib().st_set_u0(self.h, self._ptr(u0t)), "st_set_u0")

    def residual(self, U, R=None, fp64=True):
        nrm = c_double()
        check(lib().st_residual(self.h, self._ptr(U), self._ptr(R), 1 if fp64 else 0, ctypes.byref(nrm)),
              "st_residual")
        return nrm.value

    def vcycle(self, U):
        nrm = c_double()
        check(lib().st_vcycle(self.h, self._ptr(U), ctypes.byref(nrm)), "st_vcycle")
        return nrm.value

    def sdc_sweep(self, U, nsweeps=1):
        nrm = c_double()
        check(lib().st_sdc_sweep(self.h, self._ptr(U), int(nsweeps), ctypes.byref(nrm)), "st_sdc_sweep")
        return nrm.value

    def solve(self, U, raise_on_error=True):
        info = StSolveInfo()
        s = lib().st_solve(self.h, self._ptr(U), ctypes.byref(info))
        if raise_on_error and s not in (ST_OK,):
            raise StError(s, "st_solve")
        d = info.as_dict()
        d["status"] = s
        return d

    def pfasst(self, U, raise_on_error=True):
        """PFASST iterations on U (start iterate in, solution out)."""
        info = StSolveInfo()
        s = lib().st_pfasst(self.h, self._ptr(U), ctypes.byref(info))
        if raise_on_error and s != ST_OK:
            raise StError(s, "st_pfasst")
        d = info.as_dict()
        d["status"] = s
        return d

    def adjoint(self, U, target=None, gT=None, du0=None, raise_on_error=True):
        dnu, drho = c_double(), c_double()
        info = StSolveInfo()
        if gT is not None:
            s = lib().st_adjoint_solve_terminal(self.h, self._ptr(U), self._ptr(gT), ctypes.byref(dnu),
                                                ctypes.byref(drho), self._ptr(du0), ctypes.byref(info))
        else:
            s = lib().st_adjoint_solve(self.h, self._ptr(U), self._ptr(target), ctypes.byref(dnu),
                                       ctypes.byref(drho), self._ptr(du0), ctypes.byref(info))
        if raise_on_error and s != ST_OK:
            raise StError(s, "st_adjoint_solve")
        d = info.as_dict()
        d["status"] = s
        return dnu.value, drho.value, d

    def time_kernel(self, which, U=None, iters=20):
        ms, nb = c_double(), c_double()
        check(lib().st_time_kernel(self.h, int(which), self._ptr(U), int(iters), ctypes.byref(ms),
                                   ctypes.byref(nb)), "st_time_kernel")
        return ms.value, nb.value

    def stats(self):
        st = StStatsInfo()
        check(lib().st_stats(self.h, ctypes.byref(st)), "st_stats")
        return dict(levels=st.levels, cycle_graph_nodes=st.cycle_graph_nodes,
                    linearize_graph_nodes=st.linearize_graph_nodes, launches_per_vcycle=st.launches_per_vcycle,
                    update_in_cycle=st.update_in_cycle)

    def wait_selftest(self):
        """Status of st_wait_selftest (ST_ERR_TIMEOUT when a bounded device wait
        expires, is counted and is reported as it should)."""
        return lib().st_wait_selftest(self.h)

    def adjoint_lambda(self, out=None):
        out = self.zeros() if out is None else out
        check(lib().st_adjoint_lambda(self.h, self._ptr(out)), "st_adjoint_lambda")
        return out

    # level diagnostics ----------------------------------------------------
    def num_levels(self):
        return lib().st_num_levels(self.h)

    def level_info(self, l):
        li = StLevelInfo()
        check(lib().st_level_info_get(self.h, l, ctypes.byref(li)), "st_level_info_get")
        return li.as_dict()

    def level_shape(self, l):
        li = self.level_info(l)
        d = len(self.grid_shape)
        return (li["Nt"], li["M"]) + tuple(li["n"][:d][::-1])

    def linearize(self, U):
        check(lib().st_linearize(self.h, self._ptr(U)), "st_linearize")

    def level_cbar(self, l):
        torch = _torch()
        li = self.level_info(l)
        d = len(self.grid_shape)
        out = torch.empty((li["Nt"],) + tuple(li["n"][:d][::-1]), dtype=self.cycle_dtype, device=self.device)
        check(lib().st_level_cbar(self.h, l, self._ptr(out)), "st_level_cbar")
        return out

    def level_residual(self, l, e, r, transpose=False):
        out = _torch().empty_like(r)
        check(lib().st_level_residual(self.h, l, int(transpose), self._ptr(e), self._ptr(r), self._ptr(out)),
              "st_level_residual")
        return out

    def level_smooth(self, l, e, r, transpose=False):
        check(lib().st_level_smooth(self.h, l, int(transpose), self._ptr(e), self._ptr(r)), "st_level_smooth")
        return e

    def level_restrict(self, l, fine, transpose=False):
        out = _torch().empty(self.level_shape(l + 1), dtype=fine.dtype, device=fine.device)
        check(lib().st_level_restrict(self.h, l, int(transpose), self._ptr(fine), self._ptr(out)),
              "st_level_restrict")
        return out

    def level_prolong(self, l, coarse, fine, transpose=False):
        check(lib().st_level_prolong(self.h, l, int(transpose), self._ptr(coarse), self._ptr(fine)),
              "st_level_prolong")
        return fine

    def coarse_solve(self, r, transpose=False):
        e = _torch().empty_like(r)
        check(lib().st_coarse_solve(self.h, int(transpose), self._ptr(r), self._ptr(e)), "st_coarse_solve")
        return e

    def level_vcycle(self, r, transpose=False):
        e = _torch().empty_like(r)
        check(lib().st_level_vcycle(self.h, int(transpose), self._ptr(r), self._ptr(e)), "st_level_vcycle")
        return e


# ------------------------------------------------------- differentiable solve

_STSOLVE = None


def _stsolve_function():
    global _STSOLVE
    if _STSOLVE is not None:
        return _STSOLVE
    torch = _torch()

    class _STSolve(torch.autograd.Function):
        @staticmethod
        def forward(ctx, solver, nu, rho, u0):
            solver.set_params(float(nu), float(rho))
            solver.set_u0(u0.detach().to(solver.device))
            ctx.solver = solver
            ctx.theta = (float(nu), float(rho))
            ctx.u0 = u0.detach()
            if isinstance(solver, CheckpointSolver):
                # only the blocks' initial planes are kept; backward recomputes
                uT, _ = solver.forward()
                return uT
            U = solver.zeros()
            solver.solve(U)
            ctx.save_for_backward(U)
            return U[-1, -1].clone()

        @staticmethod
        def backward(ctx, g):
            S = ctx.solver
            gT = g.detach().to(device=S.device, dtype=torch.float64).contiguous().reshape(-1)
            du0 = torch.empty(S.Ns, dtype=torch.float64, device=S.device)
            if isinstance(S, CheckpointSolver):
                dnu, drho, _ = S.adjoint(gT, du0=du0)
            else:
                (U,) = ctx.saved_tensors
                S.set_params(*ctx.theta)
                S.set_u0(ctx.u0.to(S.device))
                dnu, drho, _ = S.adjoint(U, gT=gT, du0=du0)
            dev, dt = ctx.u0.device, torch.float64
            return (None, torch.tensor(dnu, dtype=dt, device=dev), torch.tensor(drho, dtype=dt, device=dev),
                    du0.reshape(ctx.u0.shape).to(dev))

    _STSOLVE = _STSolve
    return _STSOLVE


class STSolve:
    """u(T) = STSolve.apply(solver, nu, rho, u0): the final node plane of the
    all-at-once collocation solution (Eq. 3.4) as a differentiable function of
    the diffusion coefficient, the reaction rate and the initial value.  The
    backward pass is the discrete adjoint (transposed all-at-once system,
    solved by the same multigrid) with the incoming gradient as the terminal
    data, returning (dnu, drho, du0).  nu and rho are 0-d float64 tensors, u0
    a float64 tensor of the grid's shape; the solver's own problem sizes,
    boundary and reaction kind are used."""

    @staticmethod
    def apply(solver, nu, rho, u0):
        return _stsolve_function().apply(solver, nu, rho, u0)


class CheckpointSolver:
    """Slab recomputation checkpointing (st_ckpt_*): the Nt-slab problem solved
    in blocks of `block_slabs` slabs on one block-sized handle, keeping only
    each block's initial plane; the adjoint recomputes each block's U from
    it.  forward() -> u(T); adjoint(gT) -> (dnu, drho, du0).  Usable with
    STSolve.apply in place of a Solver."""

    def __init__(self, grid_shape, bc, nu, Nt, M, u0, block_slabs, T=1.0, X=1.0, reaction=NONE, rho=0.0,
                 opts: StSolverOpts | None = None, stream=None):
        torch = _torch()
        self.grid_shape = tuple(grid_shape)
        self.Nt, self.M, self.block_slabs = Nt, M, block_slabs
        self.Ns = 1
        for n in self.grid_shape:
            self.Ns *= n
        self.opts = opts if opts is not None else st_default_opts()
        self.opts.recompute_slabs = int(block_slabs)
        u0t = torch.as_tensor(u0, dtype=torch.float64).reshape(-1).contiguous()
        self._u0 = u0t
        self.problem = make_problem(self.grid_shape[::-1], bc, nu, Nt, M, T, X, reaction, rho, u0t.data_ptr())
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        rt = StRuntime()
        rt.stream = self.stream.cuda_stream
        rt.ctx = None
        dev = self.device.index

        def _alloc(nbytes, st, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev, st or 0)
            except Exception:
                return None

        def _free(ptr, nbytes, st, ctx):
            torch.cuda.caching_allocator_delete(ptr)

        rt.alloc = ALLOC_FN(_alloc)
        rt.free = FREE_FN(_free)
        self._rt = rt
        h = c_void_p()
        check(lib().st_ckpt_create(ctypes.byref(self.problem), ctypes.byref(self.opts), ctypes.byref(rt),
                                   ctypes.byref(h)), "st_ckpt_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().st_ckpt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, nu, rho):
        check(lib().st_ckpt_set_params(self.h, float(nu), float(rho)), "st_ckpt_set_params")

    def set_u0(self, u0):
        torch = _torch()
        u0t = torch.as_tensor(u0, dtype=torch.float64).reshape(-1).contiguous()
        check(lib().st_ckpt_set_u0(self.h, u0t.data_ptr()), "st_ckpt_set_u0")

    def forward(self, uT=None, raise_on_error=True):
        torch = _torch()
        if uT is None:
            uT = torch.empty(self.grid_shape, dtype=torch.float64, device=self.device)
        info = StSolveInfo()
        s = lib().st_ckpt_forward(self.h, uT.data_ptr(), ctypes.byref(info))
        if raise_on_error:
            check(s, "st_ckpt_forward")
        return uT, info.as_dict()

    def adjoint(self, gT, du0=None, raise_on_error=True):
        dnu, drho = c_double(), c_double()
        info = StSolveInfo()
        assert gT.is_contiguous() and (du0 is None or du0.is_contiguous())
        s = lib().st_ckpt_adjoint(self.h, gT.data_ptr(), ctypes.byref(dnu), ctypes.byref(drho),
                                  None if du0 is None else du0.data_ptr(), ctypes.byref(info))
        if raise_on_error:
            check(s, "st_ckpt_adjoint")
        return dnu.value, drho.value, info.as_dict()
