"""PFASST through the C ABI (paper Section 4.1) against the oracle's PFASST
iterates (exact spatial solves there; converged inner multigrid here) and,
converged, against the collocation solution."""
import numpy as np
import pytest

import stgen
from oracle import pfasst as opf
from oracle import space, system
from tests.gpu_cases import Case

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HEAT_PF = Case("heat_pfasst", (33,), space.NEUMANN, 1.0, 6, 3, T=0.3, u0_kind="cosine")
LOG_PF = Case("logistic_pfasst", (16, 16), space.PERIODIC, 1e-2, 4, 3, T=0.2, reaction=space.LOGISTIC, rho=1.0,
              u0_kind="noise", seed=12884)


def _spread(case, S):
    u0 = torch.tensor(case.u0(), dtype=torch.float64, device="cuda").reshape(case.shape)
    return u0.expand(S.field_shape).contiguous()


@pytest.mark.parametrize("case,hier", [
    (HEAT_PF, [((33,), 3), ((17,), 1), ((9,), 1)]),
    (LOG_PF, [((16, 16), 3), ((8, 8), 1)]),
])
@pytest.mark.parametrize("iters", [1, 3])
def test_pfasst_iterates_match_oracle(case, hier, iters):
    from paper_2006_12883_gb300 import stlib
    S = case.solver(precision=stlib.FP64, coarsening=stlib.COARSEN_SPACE, pfasst_levels=len(hier),
                    pfasst_coarse_M=1, sdc_inner_cycles=40, inner_coarse_iters=60, tol=0.0, max_iters=iters)
    U = _spread(case, S)
    info = S.pfasst(U, raise_on_error=False)
    assert info["status"] == stlib.ST_ERR_NOT_CONVERGED and info["iterations"] == iters, info
    p = case.problem()
    ref = opf.pfasst(p, case.u0(), hier, iters)[-1]
    got = U.cpu().numpy().reshape(ref.shape)
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()
    S.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_pfasst_converges_to_collocation_solution(prec):
    from paper_2006_12883_gb300 import stlib
    case = Case("logistic2d_pfasst", (32, 32), space.PERIODIC, 1e-2, 8, 3, reaction=space.LOGISTIC, rho=1.0,
                u0_kind="noise", seed=12884)
    S = case.solver(precision=stlib.FP64 if prec == "fp64" else stlib.FP32_REFINE, coarsening=stlib.COARSEN_SPACE,
                    pfasst_levels=3, tol=1e-10, max_iters=200)
    U = _spread(case, S)
    info = S.pfasst(U)
    assert info["status"] == 0, info
    ref = system.solve_sequential(case.problem(), case.u0())
    got = U.cpu().numpy().reshape(ref.shape)
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()
    S.close()


def test_pfasst_needs_space_only_levels():
    from paper_2006_12883_gb300 import stlib
    case = Case("mixed", (32, 32), space.PERIODIC, 2e-3, 16, 3, reaction=space.LOGISTIC, rho=1.0)
    S = case.solver(coarsening=stlib.COARSEN_AUTO_MU, pfasst_levels=3)
    U = S.zeros()
    with pytest.raises(stlib.StError):
        S.pfasst(U)
    S.close()
