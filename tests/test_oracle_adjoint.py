"""Pins of oracle.adjoint: transposition identity, closed form for the linear
heat equation, central finite differences.  CPU only."""
import numpy as np
import pytest

import stgen
from oracle import adjoint, space, system

D, P = space.DIRICHLET, space.PERIODIC


def test_adjoint_dot_product_identity():
    """lambda solves J^T lambda = -g, so <lambda, J v> = -<g, v> for every v,
    with J v from the forward directional derivative."""
    p = system.Problem(shape=(6, 6), bc=P, nu=0.03, Nt=4, M=3, T=0.5, reaction=space.LOGISTIC, rho=1.0)
    u0 = stgen.smoothed_noise((6, 6), 41).ravel()
    U = system.solve_sequential(p, u0)
    gT = stgen.random_field((36,), 42)
    lam = adjoint.adjoint_solve(p, U, gT)
    for seed in (43, 44):
        v = stgen.random_field((4, 3, 36), seed)
        lhs = float(np.sum(lam * system.jacobian_apply(p, U, v)))
        rhs = -float(gT @ v[-1, -1])
        assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(rhs))


def test_adjoint_linear_closed_form():
    """1D heat with sine-mode data: u(T) = sum_k c_k R(z_k)^Nt s_k, so
    Phi = 1/4 sum_k c_k^2 R_k^{2Nt} (target 0) has closed-form derivatives."""
    n, Nt, nu, M = 31, 8, 0.5, 2
    p = system.Problem(shape=(n,), bc=D, nu=nu, Nt=Nt, M=M, T=0.5)
    u0 = stgen.sine_modes(n)
    U, lam, (dnu, drho, du0) = adjoint.solve_and_gradients(p, u0, np.zeros(n))
    x = stgen.coords1d(D, n)
    h = 1.0 / (n + 1)

    def R(z):
        return (1 + z / 3) / (1 - 2 * z / 3 + z * z / 6)

    def dR(z):
        N, Dn = 1 + z / 3, 1 - 2 * z / 3 + z * z / 6
        return (Dn / 3 - N * (-2 / 3 + z / 3)) / Dn ** 2

    phi, dphi_dnu, grad_u0 = 0.0, 0.0, np.zeros(n)
    for k, c in ((1, 1.0), (3, 0.5)):
        lh = (2 * np.cos(k * np.pi * h) - 2) / h ** 2
        z = p.dt * nu * lh
        phi += 0.25 * c * c * R(z) ** (2 * Nt)
        dphi_dnu += 0.25 * c * c * 2 * Nt * R(z) ** (2 * Nt - 1) * dR(z) * p.dt * lh
        grad_u0 += h * c * R(z) ** (2 * Nt) * np.sin(k * np.pi * x)
    assert abs(adjoint.objective(p, U, np.zeros(n)) - phi) < 1e-13
    assert abs(dnu - dphi_dnu) < 1e-11 * abs(dphi_dnu)
    assert drho == 0.0
    assert np.abs(du0 - grad_u0).max() < 1e-12 * np.abs(grad_u0).max()


@pytest.mark.parametrize("kind", [space.LOGISTIC, space.CUBIC])
def test_adjoint_central_fd(kind):
    p = system.Problem(shape=(8, 8), bc=P, nu=0.02, Nt=4, M=3, T=0.4, reaction=kind, rho=1.0)
    u0 = stgen.smoothed_noise((8, 8), 45).ravel()
    target = system.solve_sequential(p.with_params(nu=0.026, rho=0.8), u0)[-1, -1]
    U, lam, (dnu, drho, du0) = adjoint.solve_and_gradients(p, u0, target)
    fd_nu = adjoint.fd_gradient_param(p, u0, target, "nu")
    fd_rho = adjoint.fd_gradient_param(p, u0, target, "rho")
    assert abs(dnu - fd_nu) < 1e-6 * abs(fd_nu)
    assert abs(drho - fd_rho) < 1e-6 * abs(fd_rho)
    direction = stgen.random_field((64,), 46)
    fd_u0 = adjoint.fd_gradient_u0(p, u0, target, direction)
    assert abs(float(du0 @ direction) - fd_u0) < 1e-6 * abs(fd_u0)


def test_large_periodic_transposed_solves_match_direct(monkeypatch):
    """The adjoint's Krylov path for large periodic slabs (matrix-free J^T,
    preconditioned by the exact transposed constant-coefficient inverse)
    gives the sparse-LU adjoint, forced here on a small grid."""
    p = system.Problem(shape=(12, 16), bc=space.PERIODIC, nu=0.05, Nt=3, M=3, T=0.3, reaction=space.LOGISTIC,
                       rho=1.2)
    u0 = stgen.random_field(p.shape, 31, 0.3).ravel() + 0.5
    U = system.solve_sequential(p, u0)
    gT = stgen.random_field((p.Ns,), 32)
    direct = adjoint.adjoint_solve(p, U, gT)
    monkeypatch.setattr(system, "_DIRECT_MAX", 0)
    krylov = adjoint.adjoint_solve(p, U, gT)
    assert np.abs(krylov - direct).max() <= 1e-12 * np.abs(direct).max()
