"""The allocation-free residual norm entry point (for callers that cannot
allocate device memory where they need a residual norm: code under another
framework's fixed-budget pool, inside an allocator callback, or in a loop
that must not synchronise on cudaMalloc).  Its output must match the handle
based st_residual on two calls in a row - the scratch array it shares
between calls keeps the previous call's contents, which must not leak into
the next result.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

import stgen
from tests.gpu_cases import LOG2D, residual_scale

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _call_noalloc(stlib, case, u0_dev, U, R):
    prob = stlib.make_problem(case.shape[::-1], case.bc, case.nu, case.Nt, case.M, T=case.T, X=case.X,
                              reaction=case.reaction, rho=case.rho, u0_ptr=u0_dev.data_ptr())
    nrm = ctypes.c_double()
    stream = torch.cuda.current_stream().cuda_stream
    s = stlib.lib().st_residual_noalloc(ctypes.byref(prob), U.data_ptr(), R.data_ptr(), ctypes.byref(nrm),
                                        ctypes.c_void_p(stream))
    stlib.check(s, "st_residual_noalloc")
    return nrm.value


def test_noalloc_matches_handle_residual_twice():
    from paper_2006_12883_gb300 import build, stlib
    build()
    case = LOG2D
    p = case.problem()
    u0_dev = torch.tensor(case.u0(), device="cuda")
    S = case.solver(precision=stlib.FP64)
    # two different inputs, back to back: the second result must not depend on the first
    for seed, scale in ((71, 0.3), (72, 2.0)):
        U = torch.tensor(stgen.random_field((p.Nt, p.M, p.Ns), seed, scale) + 0.5, device="cuda")
        R_ref = torch.empty_like(U)
        n_ref = S.residual(U.reshape(S.field_shape), R_ref.reshape(S.field_shape), fp64=True)
        R = torch.full_like(U, float("nan"))
        n = _call_noalloc(stlib, case, u0_dev, U, R)
        tol = 1e-13 * residual_scale(p, U.cpu().numpy())
        assert np.abs((R - R_ref).cpu().numpy()).max() <= tol
        assert abs(n - n_ref) <= 1e-12 * n_ref
    S.close()


def test_noalloc_rejects_host_pointers_and_oversize():
    from paper_2006_12883_gb300 import build, stlib
    build()
    case = LOG2D
    u0_host = torch.tensor(case.u0())
    U = torch.zeros((case.Nt, case.M) + case.shape, dtype=torch.float64, device="cuda")
    prob = stlib.make_problem(case.shape[::-1], case.bc, case.nu, case.Nt, case.M, reaction=case.reaction,
                              rho=case.rho, u0_ptr=u0_host.data_ptr())
    s = stlib.lib().st_residual_noalloc(ctypes.byref(prob), U.data_ptr(), None, None, None)
    assert s == stlib.ST_ERR_INVALID_ARG
    u0_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    big = stlib.make_problem((1 << 14, 1 << 13), stlib.PERIODIC, 1.0, 1, 1, u0_ptr=u0_dev.data_ptr())
    s = stlib.lib().st_residual_noalloc(ctypes.byref(big), U.data_ptr(), None, None, None)
    assert s == stlib.ST_ERR_UNSUPPORTED
