"""Discrete adjoint through the C ABI (transposed V-cycle, FP64 refinement):
gradients against the oracle's adjoint, central finite differences of the
GPU forward solve and the linear closed form."""
import numpy as np
import pytest

import stgen
from oracle import adjoint as oadj
from oracle import space, system
from tests.gpu_cases import Case

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ADJ = Case("adjoint2d", (32, 32), space.PERIODIC, 1e-2, 8, 3, T=0.5, reaction=space.LOGISTIC, rho=1.0,
           u0_kind="noise", seed=12887)


def _target(case):
    q = case.problem().with_params(nu=1.3e-2, rho=0.8)
    return system.solve_sequential(q, case.u0())[-1, -1]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_adjoint_matches_oracle(prec):
    from paper_2006_12883_gb300 import stlib
    case = ADJ
    p = case.problem()
    target = _target(case)
    S = case.solver(precision=stlib.FP64 if prec == "fp64" else stlib.FP32_REFINE, tol=1e-12)
    U = S.zeros()
    S.solve(U)
    du0 = torch.empty(p.Ns, dtype=torch.float64, device="cuda")
    dnu, drho, info = S.adjoint(U, target=torch.tensor(target, device="cuda"), du0=du0)
    assert info["status"] == 0
    _, _, (rnu, rrho, rdu0) = oadj.solve_and_gradients(p, case.u0(), target)
    assert abs(dnu - rnu) <= 1e-6 * abs(rnu)
    assert abs(drho - rrho) <= 1e-6 * abs(rrho)
    assert np.linalg.norm(du0.cpu().numpy() - rdu0) <= 1e-6 * np.linalg.norm(rdu0)
    S.close()


def test_adjoint_central_fd_on_gpu():
    """dPhi/dnu, dPhi/drho against central differences of GPU forward solves."""
    from paper_2006_12883_gb300 import stlib
    case = ADJ
    p = case.problem()
    target = _target(case)
    S = case.solver(precision=stlib.FP64, tol=1e-13)
    U = S.zeros()
    S.solve(U)
    dnu, drho, _ = S.adjoint(U, target=torch.tensor(target, device="cuda"))

    def phi(nu, rho):
        S.set_params(nu, rho)
        V = S.zeros()
        S.solve(V)
        return oadj.objective(p, V.cpu().numpy().reshape(p.Nt, p.M, -1), target)

    for name, th, g in (("nu", case.nu, dnu), ("rho", case.rho, drho)):
        d = 1e-6 * th
        args = [case.nu, case.rho]
        i = 0 if name == "nu" else 1
        a1 = list(args); a1[i] += d
        a2 = list(args); a2[i] -= d
        fd = (phi(*a1) - phi(*a2)) / (2 * d)
        assert abs(g - fd) <= 1e-6 * abs(fd), (name, g, fd)
    S.close()


def test_adjoint_terminal_gradient_and_host_pointers():
    from paper_2006_12883_gb300 import stlib
    case = ADJ
    p = case.problem()
    S = case.solver(precision=stlib.FP64, tol=1e-12)
    U = S.zeros()
    S.solve(U)
    gT = stgen.random_field((p.Ns,), 77)
    du0 = torch.empty(p.Ns, dtype=torch.float64)  # host
    dnu, drho, info = S.adjoint(U.cpu(), gT=torch.tensor(gT), du0=du0)
    lam = oadj.adjoint_solve(p, U.cpu().numpy().reshape(p.Nt, p.M, -1), gT)
    rnu, rrho, rdu0 = oadj.gradients(p, U.cpu().numpy().reshape(p.Nt, p.M, -1), lam)
    assert abs(dnu - rnu) <= 1e-8 * abs(rnu)
    assert np.linalg.norm(du0.numpy() - rdu0) <= 1e-8 * np.linalg.norm(rdu0)
    # the adjoint state itself, read back to host memory, after a host FP64
    # residual (which must not disturb it)
    S.residual(U.cpu(), torch.empty(U.shape, dtype=torch.float64), fp64=True)
    lam_h = S.adjoint_lambda(torch.empty(U.shape, dtype=torch.float64))
    assert np.linalg.norm(lam_h.numpy().reshape(lam.shape) - lam) <= 1e-8 * np.linalg.norm(lam)
    S.close()


NEU_CASES = [
    # the paper's heat example (Section 5.3: Neumann, cosine data) at 64 cells
    Case("heat_neumann", (65,), space.NEUMANN, 1.0, 8, 3, u0_kind="cosine"),
    # the paper's monodomain example (Section 5.4) at small size
    Case("monodomain", (129,), space.NEUMANN, 1.0, 16, 2, T=0.5, X=10.0, reaction=space.CUBIC, rho=5.0,
         u0_kind="stimulus"),
    # a 2D Neumann grid with the logistic reaction
    Case("neumann2d", (17, 33), space.NEUMANN, 0.05, 6, 3, T=0.3, reaction=space.LOGISTIC, rho=1.0),
]


@pytest.mark.parametrize("case", NEU_CASES, ids=lambda c: c.name)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_adjoint_neumann_matches_oracle(case, prec):
    """Neumann boundaries (the paper's own examples): the mirrored-ghost
    Laplacian is not symmetric, so the adjoint uses L^T = W L W^-1 (W the
    lumped mass weights); gradients and the adjoint state against the
    oracle's backward solve with the transposed slab Jacobians."""
    from paper_2006_12883_gb300 import stlib
    p = case.problem()
    S = case.solver(precision=stlib.FP64 if prec == "fp64" else stlib.FP32_REFINE, tol=1e-12, max_iters=200)
    U = S.zeros()
    assert S.solve(U)["status"] == 0
    Uh = U.cpu().numpy().reshape(p.Nt, p.M, -1)
    gT = stgen.random_field((p.Ns,), 78)
    du0 = torch.empty(p.Ns, dtype=torch.float64, device="cuda")
    dnu, drho, info = S.adjoint(U, gT=torch.tensor(gT, device="cuda"), du0=du0)
    assert info["status"] == 0, info
    lam = oadj.adjoint_solve(p, Uh, gT)
    rnu, rrho, rdu0 = oadj.gradients(p, Uh, lam)
    # the gradients to the adjoint's 1e-6 (dPhi/dnu of the decayed heat
    # solution is a sum with heavy cancellation: it is 1e-5 of its terms)
    assert abs(dnu - rnu) <= 1e-6 * abs(rnu), (dnu, rnu)
    if case.reaction != space.NONE:
        assert abs(drho - rrho) <= 1e-6 * abs(rrho), (drho, rrho)
    assert np.linalg.norm(du0.cpu().numpy() - rdu0) <= 1e-8 * np.linalg.norm(rdu0)
    lam_g = S.adjoint_lambda(torch.empty(U.shape, dtype=torch.float64)).numpy().reshape(lam.shape)
    assert np.linalg.norm(lam_g - lam) <= 1e-8 * np.linalg.norm(lam)
    S.close()


def test_stsolve_autograd_matches_oracle_gradients():
    from paper_2006_12883_gb300 import stlib
    case = ADJ
    p = case.problem()
    S = case.solver(precision=stlib.FP64, tol=1e-12)
    target = torch.tensor(_target(case), device="cuda")
    nu = torch.tensor(case.nu, dtype=torch.float64, requires_grad=True)
    rho = torch.tensor(case.rho, dtype=torch.float64, requires_grad=True)
    u0 = torch.tensor(case.u0(), device="cuda").reshape(case.shape).requires_grad_(True)
    uT = stlib.STSolve.apply(S, nu, rho, u0)
    h2 = float(np.prod([space.spacing(case.bc, n, case.X) for n in case.shape]))
    loss = 0.5 * h2 * ((uT.reshape(-1) - target) ** 2).sum()
    loss.backward()
    U = S.zeros()
    S.solve(U)
    Uh = U.cpu().numpy().reshape(p.Nt, p.M, -1)
    gT = h2 * (Uh[-1, -1] - target.cpu().numpy())
    lam = oadj.adjoint_solve(p, Uh, gT)
    rnu, rrho, rdu0 = oadj.gradients(p, Uh, lam)
    assert abs(nu.grad.item() - rnu) <= 1e-8 * abs(rnu)
    assert abs(rho.grad.item() - rrho) <= 1e-8 * abs(rrho)
    assert np.linalg.norm(u0.grad.cpu().numpy().ravel() - rdu0) <= 1e-8 * np.linalg.norm(rdu0)
    S.close()


@pytest.mark.parametrize("K", [1, 2, 4])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_checkpointed_adjoint_matches_stored(K, prec):
    """Slab recomputation checkpointing: blocks of K slabs solved one after
    another (exact by causality of Eq. 3.4), the adjoint recomputing each
    block's U; u(T) and the gradients equal the stored-U path's to the solve
    tolerance, and the oracle's."""
    from paper_2006_12883_gb300 import stlib
    case = ADJ
    p = case.problem()
    pr = stlib.FP64 if prec == "fp64" else stlib.FP32_REFINE
    S = case.solver(precision=pr, tol=1e-12)
    U = S.zeros()
    assert S.solve(U)["status"] == 0
    gT = torch.tensor(stgen.random_field((p.Ns,), 79), device="cuda")
    du0 = torch.empty(p.Ns, dtype=torch.float64, device="cuda")
    dnu, drho, _ = S.adjoint(U, gT=gT, du0=du0)
    C = stlib.CheckpointSolver(case.shape, case.bc, case.nu, case.Nt, case.M, case.u0(), K, T=case.T,
                               reaction=case.reaction, rho=case.rho, opts=stlib.make_opts(precision=pr, tol=1e-12))
    uT, finfo = C.forward()
    assert finfo["status"] == 0
    assert torch.allclose(uT.reshape(-1), U[-1, -1].reshape(-1), rtol=0, atol=1e-10 * float(U.abs().max()))
    cdu0 = torch.empty_like(du0)
    cnu, crho, ainfo = C.adjoint(gT, du0=cdu0)
    assert ainfo["status"] == 0
    assert abs(cnu - dnu) <= 1e-9 * abs(dnu) and abs(crho - drho) <= 1e-9 * abs(drho), (cnu, dnu, crho, drho)
    assert float((cdu0 - du0).norm()) <= 1e-9 * float(du0.norm())
    Uh = U.cpu().numpy().reshape(p.Nt, p.M, -1)
    rnu, rrho, rdu0 = oadj.gradients(p, Uh, oadj.adjoint_solve(p, Uh, gT.cpu().numpy()))
    assert abs(cnu - rnu) <= 1e-8 * abs(rnu)
    # a parameter change invalidates the stored planes: the adjoint refuses
    # until the next forward pass
    C.set_params(case.nu * 1.01, case.rho)
    s = stlib.lib().st_ckpt_adjoint(C.h, gT.data_ptr(), None, None, None, None)
    assert s == stlib.ST_ERR_INVALID_ARG
    C.close()
    S.close()


def test_checkpointed_stsolve_autograd():
    """STSolve.apply on a CheckpointSolver: the forward keeps only the blocks'
    initial planes, the backward recomputes; gradients equal the oracle's."""
    from paper_2006_12883_gb300 import stlib
    case = ADJ
    p = case.problem()
    C = stlib.CheckpointSolver(case.shape, case.bc, case.nu, case.Nt, case.M, case.u0(), 2, T=case.T,
                               reaction=case.reaction, rho=case.rho,
                               opts=stlib.make_opts(precision=stlib.FP64, tol=1e-12))
    target = torch.tensor(_target(case), device="cuda")
    nu = torch.tensor(case.nu, dtype=torch.float64, requires_grad=True)
    rho = torch.tensor(case.rho, dtype=torch.float64, requires_grad=True)
    u0 = torch.tensor(case.u0(), device="cuda").reshape(case.shape).requires_grad_(True)
    uT = stlib.STSolve.apply(C, nu, rho, u0)
    h2 = float(np.prod([space.spacing(case.bc, n, case.X) for n in case.shape]))
    loss = 0.5 * h2 * ((uT.reshape(-1) - target) ** 2).sum()
    loss.backward()
    _, _, (rnu, rrho, rdu0) = oadj.solve_and_gradients(p, case.u0(), target.cpu().numpy())
    assert abs(nu.grad.item() - rnu) <= 1e-8 * abs(rnu)
    assert abs(rho.grad.item() - rrho) <= 1e-8 * abs(rrho)
    assert np.linalg.norm(u0.grad.cpu().numpy().ravel() - rdu0) <= 1e-8 * np.linalg.norm(rdu0)
    C.close()
