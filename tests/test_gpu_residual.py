"""Fine FP64 residual G(U) (Eq. 2.3 with the slab coupling of Eq. 3.4), its
norm and the node-averaged reaction derivative: CUDA path through the C ABI
against the oracle, element by element."""
import numpy as np
import pytest

import stgen
from oracle import system
from tests.gpu_cases import RESIDUAL_CASES, residual_scale

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("case", RESIDUAL_CASES, ids=lambda c: c.name)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_residual_parity(case, prec):
    from paper_2006_12883_gb300 import stlib
    p = case.problem()
    u0 = case.u0()
    U = stgen.random_field((p.Nt, p.M, p.Ns), 7, 0.4) + 0.5
    G = system.residual(p, U, u0)
    S = case.solver(precision=stlib.FP64 if prec == "fp64" else stlib.FP32_REFINE)
    Ut = torch.tensor(U, device="cuda").reshape(S.field_shape)
    R = torch.empty_like(Ut)
    nrm = S.residual(Ut, R, fp64=True)
    Rg = R.cpu().numpy().reshape(G.shape)
    scale = residual_scale(p, U)
    # FP64 arithmetic in a different order: a few ulps of the largest term
    assert np.abs(Rg - G).max() <= 1e-13 * scale, (np.abs(Rg - G).max(), scale)
    assert abs(nrm - np.linalg.norm(G)) <= 1e-12 * np.linalg.norm(G) + 1e-13 * scale
    # the cycle-precision copy
    R32 = torch.empty(S.field_shape, dtype=S.cycle_dtype, device="cuda")
    S.residual(Ut, R32, fp64=False)
    tol = 1e-13 * scale if prec == "fp64" else 2e-7 * np.abs(G).max() + 1e-13 * scale
    assert np.abs(R32.double().cpu().numpy().reshape(G.shape) - G).max() <= tol
    # host pointers: same numbers through the staging path
    Rh = torch.empty(S.field_shape, dtype=torch.float64)
    nrm_h = S.residual(Ut.cpu(), Rh, fp64=True)
    assert np.array_equal(Rh.numpy().reshape(G.shape), Rg)
    assert nrm_h == nrm
    # cbar = mean_m R'(U_{n,m})
    S.linearize(Ut)
    cb = S.level_cbar(0).double().cpu().numpy().reshape(p.Nt, p.Ns)
    ref = system.cbar(p, U)
    ctol = 1e-14 if prec == "fp64" else 1e-6
    assert np.abs(cb - ref).max() <= ctol * max(1.0, np.abs(ref).max())
    S.close()


def test_residual_norm_deterministic():
    from paper_2006_12883_gb300 import stlib
    case = RESIDUAL_CASES[-2]
    p = case.problem()
    U = stgen.random_field((p.Nt, p.M, p.Ns), 9)
    S = case.solver(precision=stlib.FP32_REFINE)
    Ut = torch.tensor(U, device="cuda").reshape(S.field_shape)
    norms = {S.residual(Ut) for _ in range(5)}
    assert len(norms) == 1
    S.close()


def test_zero_guess_reference_norm():
    """||G(0)|| = sqrt(M) ||u0|| (the zero initial guess of Section 5.2)."""
    case = RESIDUAL_CASES[3]
    p = case.problem()
    S = case.solver()
    Z = torch.zeros(S.field_shape, dtype=torch.float64, device="cuda")
    nrm = S.residual(Z)
    assert abs(nrm - system.reference_norm(p, case.u0())) <= 1e-13 * nrm
    S.close()
