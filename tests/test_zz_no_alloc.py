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
from oracle import system
from tests.gpu_cases import LOG2D, residual_scale

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _call_noalloc(stlib, case, u0_dev, U, R, want_norm=True):
    prob = stlib.make_problem(case.shape[::-1], case.bc, case.nu, case.Nt, case.M, T=case.T, X=case.X,
                              reaction=case.reaction, rho=case.rho, u0_ptr=u0_dev.data_ptr())
    nrm = ctypes.c_double()
    stream = torch.cuda.current_stream().cuda_stream
    s = stlib.lib().st_residual_noalloc(ctypes.byref(prob), U.data_ptr(), None if R is None else R.data_ptr(),
                                        ctypes.byref(nrm) if want_norm else None, ctypes.c_void_p(stream))
    stlib.check(s, "st_residual_noalloc")
    return nrm.value if want_norm else None


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
        # and directly against the oracle's G(U) (Eq. 2.3 with the slab coupling)
        G = system.residual(p, U.cpu().numpy(), case.u0())
        assert np.abs(R.cpu().numpy().reshape(G.shape) - G).max() <= tol
        assert abs(n - np.linalg.norm(G)) <= 1e-12 * np.linalg.norm(G) + 1e-13 * residual_scale(p, U.cpu().numpy())
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


def test_noalloc_long_slab_runs_and_optional_outputs():
    """256^2 points x 1100 slabs at M = 1: Ns*Nt > 2^26, so the call lengthens
    its slab runs until the partial sums fit the shared array.  R and the norm
    must still match the handle residual; each output may be left out; and the
    second call must leave the device's free memory unchanged."""
    from paper_2006_12883_gb300 import build, stlib
    from tests.gpu_cases import Case
    from oracle import space
    build()
    case = Case("long_runs", (256, 256), space.PERIODIC, 1e-2, 1100, 1, T=1.0, reaction=space.LOGISTIC, rho=1.0,
                u0_kind="noise", seed=5)
    p = case.problem()
    assert p.Ns * p.Nt > (1 << 26)
    u0_dev = torch.tensor(case.u0(), device="cuda")
    U = torch.tensor(stgen.random_field((p.Nt, p.M, p.Ns), 73, 0.2) + 0.5, device="cuda")
    S = case.solver(precision=stlib.FP64)
    R_ref = torch.empty_like(U)
    n_ref = S.residual(U.reshape(S.field_shape), R_ref.reshape(S.field_shape), fp64=True)
    S.close()
    tol = 1e-13 * residual_scale(p, U.cpu().numpy())
    R = torch.full_like(U, float("nan"))
    n1 = _call_noalloc(stlib, case, u0_dev, U, R)
    assert np.abs((R - R_ref).cpu().numpy()).max() <= tol
    assert abs(n1 - n_ref) <= 1e-12 * n_ref
    G = system.residual(p, U.cpu().numpy(), case.u0())
    assert np.abs(R.cpu().numpy().reshape(G.shape) - G).max() <= tol
    del G
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    n2 = _call_noalloc(stlib, case, u0_dev, U, None)  # norm only
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert n2 == n1
    R2 = torch.full_like(U, float("nan"))
    assert _call_noalloc(stlib, case, u0_dev, U, R2, want_norm=False) is None  # R only
    torch.cuda.synchronize()
    assert torch.equal(R2, R)
