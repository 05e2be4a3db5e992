"""Pins of oracle.system / multilevel / sdc: the collocation residual, the
direct and sequential solves, closed forms and invariants.  CPU only."""
import math

import numpy as np
import pytest

import stgen
from oracle import collocation as col
from oracle import multilevel as ml
from oracle import sdc, space, system

D, P, N = space.DIRICHLET, space.PERIODIC, space.NEUMANN


def pade2(z):
    return (1 + z / 3) / (1 - 2 * z / 3 + z * z / 6)


def test_residual_brute_force_loops():
    """G(U) of Eq. (2.3)+(2.11) written with explicit index loops (1D
    Dirichlet, logistic) against the vectorised oracle."""
    n, Nt, M = 5, 3, 2
    p = system.Problem(shape=(n,), bc=D, nu=0.7, Nt=Nt, M=M, T=0.6, reaction=space.LOGISTIC, rho=1.3)
    U = stgen.random_field((Nt, M, n), 1)
    u0 = stgen.random_field((n,), 2)
    h = 1.0 / (n + 1)
    dt = 0.6 / Nt
    q = [[5 / 12, -1 / 12], [3 / 4, 1 / 4]]
    G = np.zeros((Nt, M, n))
    for s in range(Nt):
        for m in range(M):
            for i in range(n):
                prev = u0[i] if s == 0 else U[s - 1, M - 1, i]
                acc = 0.0
                for j in range(M):
                    left = U[s, j, i - 1] if i > 0 else 0.0
                    right = U[s, j, i + 1] if i < n - 1 else 0.0
                    lap = (left - 2 * U[s, j, i] + right) / (h * h)
                    f = 0.7 * lap + 1.3 * U[s, j, i] * (1 - U[s, j, i])
                    acc += q[m][j] * f
                G[s, m, i] = prev + dt * acc - U[s, m, i]
    assert np.abs(system.residual(p, U, u0) - G).max() < 1e-12


def test_residual_zero_guess_and_linearity():
    p = system.Problem(shape=(4, 8), bc=P, nu=0.1, Nt=4, M=3)
    u0 = stgen.random_field((4, 8), 3).ravel()
    G0 = system.residual(p, np.zeros((4, 3, 32)), u0)
    assert np.abs(G0[0] - u0[None, :]).max() == 0 and np.abs(G0[1:]).max() == 0
    assert abs(system.reference_norm(p, u0) - math.sqrt(3) * np.linalg.norm(u0)) < 1e-12
    U = stgen.random_field((4, 3, 32), 4)
    V = stgen.random_field((4, 3, 32), 5)
    # affine in U for a linear problem: G(U+V) - G(U) = J V, and J V = G(V) - G(0)
    lhs = system.residual(p, U + V, u0) - system.residual(p, U, u0)
    assert np.abs(lhs - system.jacobian_apply(p, U, V)).max() < 1e-12


def test_jacobian_apply_matches_finite_differences():
    p = system.Problem(shape=(6, 6), bc=P, nu=0.05, Nt=3, M=3, reaction=space.CUBIC, rho=2.0)
    U = stgen.random_field((3, 3, 36), 6, 0.5)
    V = stgen.random_field((3, 3, 36), 7)
    u0 = stgen.random_field((36,), 8)
    eps = 1e-6
    fd = (system.residual(p, U + eps * V, u0) - system.residual(p, U - eps * V, u0)) / (2 * eps)
    assert np.abs(fd - system.jacobian_apply(p, U, V)).max() < 1e-7
    Jd = system.full_jacobian_dense(p, U)
    assert np.abs(Jd @ V.ravel() - system.jacobian_apply(p, U, V).ravel()).max() < 1e-12


@pytest.mark.parametrize("M", [1, 2, 3])
def test_heat_sine_mode_closed_form(M):
    """1D heat, Dirichlet: slab-end amplitude of mode k is R(dt*lam_k)^n with R
    the Pade(M-1, M) function (closed form) - exact to rounding."""
    n, Nt, nu = 63, 16, 1.0
    p = system.Problem(shape=(n,), bc=D, nu=nu, Nt=Nt, M=M)
    u0 = stgen.sine_modes(n)
    U = system.solve_sequential(p, u0)
    x = stgen.coords1d(D, n)
    num = {1: lambda z: 1.0, 2: lambda z: 1 + z / 3, 3: lambda z: 1 + 2 * z / 5 + z * z / 20}[M]
    den = {1: lambda z: 1 - z, 2: lambda z: 1 - 2 * z / 3 + z * z / 6,
           3: lambda z: 1 - 3 * z / 5 + 3 * z * z / 20 - z ** 3 / 60}[M]
    for nslab in (0, 7, Nt - 1):
        exact = np.zeros(n)
        for k, a in ((1, 1.0), (3, 0.5)):
            z = p.dt * system.sine_mode_eigenvalue(k, n, nu)
            exact += a * (num(z) / den(z)) ** (nslab + 1) * np.sin(k * np.pi * x)
        assert np.abs(U[nslab, -1] - exact).max() < 1e-12 * np.abs(u0).max()
    if M == 2:
        # stage values at node 1 with the textbook M=2 Q: (I - zQ)^{-1} 1
        Qt = np.array([[5 / 12, -1 / 12], [3 / 4, 1 / 4]])
        z = p.dt * system.sine_mode_eigenvalue(1, n, nu)
        st = np.linalg.solve(np.eye(2) - z * Qt, np.ones(2))
        z3 = p.dt * system.sine_mode_eigenvalue(3, n, nu)
        st3 = np.linalg.solve(np.eye(2) - z3 * Qt, np.ones(2))
        exact0 = st[0] * np.sin(np.pi * x) + 0.5 * st3[0] * np.sin(3 * np.pi * x)
        assert np.abs(U[0, 0] - exact0).max() < 1e-12


@pytest.mark.parametrize("M", [1, 2, 3])
def test_heat_order_against_semidiscrete(M):
    """Error w.r.t. the semi-discrete solution (Eq. 5.3 analogue, sine mode)
    decays at order 2M-1 (Fig. 5.1, right)."""
    n, nu = 15, 1.0
    x = stgen.coords1d(D, n)
    lam = system.sine_mode_eigenvalue(1, n, nu)
    errs = []
    Nts = [16, 32, 64] if M > 1 else [64, 128, 256]
    for Nt in Nts:
        p = system.Problem(shape=(n,), bc=D, nu=nu, Nt=Nt, M=M, T=0.1)
        U = system.solve_sequential(p, np.sin(np.pi * x))
        errs.append(np.abs(U[-1, -1] - math.exp(lam * 0.1) * np.sin(np.pi * x)).max())
    slope = math.log2(errs[-2] / errs[-1])
    assert abs(slope - (2 * M - 1)) < 0.3, (errs, slope)


def test_dense_equals_sequential_and_dg():
    """All-at-once dense Newton == slab-by-slab Newton == DG solve (the paper's
    'same solution up to machine precision', Section 5.1)."""
    p = system.Problem(shape=(5, 4), bc=P, nu=0.02, Nt=4, M=3, T=0.5, reaction=space.LOGISTIC, rho=1.0)
    u0 = stgen.smoothed_noise((5, 4), 11).ravel()
    Us = system.solve_sequential(p, u0)
    Ud = system.solve_dense(p, u0)
    Ug = system.dg_solve(p, u0)
    assert np.abs(Us - Ud).max() < 1e-13
    assert np.abs(Us - Ug).max() < 1e-13
    assert system.residual_norm(p, Us, u0) < 1e-13


def test_neumann_dg_equals_collocation():
    p = system.Problem(shape=(9,), bc=N, nu=1.0, Nt=3, M=2, T=0.2, X=10.0, reaction=space.CUBIC, rho=5.0)
    u0 = stgen.stimulus(9, X=10.0)
    assert np.abs(system.solve_sequential(p, u0) - system.dg_solve(p, u0)).max() < 1e-12


@pytest.mark.parametrize("M", [2, 3])
def test_logistic_constant_state_is_radau_ode(M):
    """A spatially constant u0 reduces to the scalar logistic ODE; its Radau
    IIA solution converges at order 2M-1 to the closed form
    u(t) = 1/(1 + (1/u0 - 1) e^{-rho t})."""
    errs = []
    for Nt in (8, 16, 32):
        p = system.Problem(shape=(4,), bc=P, nu=0.3, Nt=Nt, M=M, T=2.0, reaction=space.LOGISTIC, rho=1.5)
        U = system.solve_sequential(p, np.full(4, 0.2))
        exact = 1.0 / (1.0 + (1 / 0.2 - 1) * math.exp(-1.5 * 2.0))
        assert np.abs(U[-1, -1] - U[-1, -1, 0]).max() < 1e-14  # stays constant in space
        errs.append(abs(U[-1, -1, 0] - exact))
    slope = math.log2(errs[-2] / errs[-1])
    assert abs(slope - (2 * M - 1)) < 0.35, (errs, slope)


def test_fixed_points_and_mean_conservation():
    for kind, vals in [(space.LOGISTIC, [0.0, 1.0]), (space.CUBIC, [-1.0, 0.0, 1.0])]:
        p = system.Problem(shape=(6, 6), bc=P, nu=0.1, Nt=3, M=3, reaction=kind, rho=2.0)
        for v in vals:
            U = np.full((3, 3, 36), v)
            assert np.abs(system.residual(p, U, np.full(36, v))).max() < 1e-15
    # rho = 0, periodic: the spatial mean is conserved exactly by every slab
    p = system.Problem(shape=(8, 8), bc=P, nu=0.05, Nt=5, M=3)
    u0 = stgen.smoothed_noise((8, 8), 12).ravel()
    U = system.solve_sequential(p, u0)
    assert np.abs(U.mean(axis=2) - u0.mean()).max() < 1e-14


def test_time_truncation_causality():
    p = system.Problem(shape=(8, 8), bc=P, nu=0.01, Nt=8, M=3, reaction=space.LOGISTIC, rho=1.0)
    u0 = stgen.smoothed_noise((8, 8), 13).ravel()
    full = system.solve_sequential(p, u0)
    part = system.solve_sequential(p, u0, nslabs=3)
    assert np.abs(full[:3] - part).max() == 0
    p3 = p.with_params(Nt=3, T=3 * p.dt)
    assert np.abs(system.solve_sequential(p3, u0) - part).max() < 1e-15


# ------------------------------------------------------------- multilevel

def _level(p, U):
    return ml.Level(shape=p.shape, bc=p.bc, Nt=p.Nt, M=p.M, dt=p.dt, nu=p.nu, X=p.X,
                    cbar=system.cbar(p, U))


def test_level_operator_is_minus_jacobian_linear():
    p = system.Problem(shape=(8,), bc=P, nu=0.1, Nt=4, M=3)
    U = np.zeros((4, 3, 8))
    lev = _level(p, U)
    e = stgen.random_field((4, 3, 8), 21)
    assert np.abs(ml.apply_A(lev, e) - ml.coupling(lev, e) + system.jacobian_apply(p, U, e)).max() < 1e-13


def test_level_operator_is_minus_jacobian_when_cbar_exact():
    """With R' equal on all nodes of a slab (U constant in m), cbar is exact."""
    p = system.Problem(shape=(6,), bc=D, nu=0.1, Nt=3, M=2, reaction=space.LOGISTIC, rho=1.0)
    base = stgen.random_field((3, 1, 6), 22)
    U = np.repeat(base, 2, axis=1)
    lev = _level(p, U)
    e = stgen.random_field((3, 2, 6), 23)
    assert np.abs(ml.apply_A(lev, e) - ml.coupling(lev, e) + system.jacobian_apply(p, U, e)).max() < 1e-13


def test_coarse_solve_exact():
    lev = ml.Level(shape=(4,), bc=P, Nt=5, M=3, dt=0.1, nu=0.3, X=1.0,
                   cbar=stgen.random_field((5, 4), 24, 0.2))
    r = stgen.random_field((5, 3, 4), 25)
    e = ml.coarse_solve_exact(lev, r)
    assert np.abs(ml.linear_residual(lev, e, r)).max() < 1e-13


@pytest.mark.parametrize("M", [1, 3, 5])
def test_time_transfer_roundtrip(M):
    """Through the level operators: with a reaction coefficient constant in
    space and time, restricting the fine level's operator (A - C, slab
    coupling included) applied to a prolonged coarse correction gives the
    coarse level's operator on that correction,
        R_t (A_f - C_f) P_t v = (A_c - C_c) v,
    because slab bisection is a Galerkin coarsening of the DG form (Eq. 2.9,
    3.4) and rediscretisation with 2 dt is its exact coarse operator."""
    shape, Nc = (6,), 4
    v = stgen.random_field((Nc, M, 6), 26)
    mk = lambda Nt, dt: ml.Level(shape=shape, bc=P, Nt=Nt, M=M, dt=dt, nu=0.3, X=1.0,
                                 cbar=np.full((Nt, 6), -0.7))
    fine, coarse = mk(2 * Nc, 0.05), mk(Nc, 0.1)
    pv = ml.prolong_time(M, v)
    assert pv.shape == (2 * Nc, M, 6)
    lhs = ml.restrict_time(M, ml.apply_A(fine, pv) - ml.coupling(fine, pv))
    rhs = ml.apply_A(coarse, v) - ml.coupling(coarse, v)
    assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(rhs).max()
    # R_t P_t is not the identity (nor 2 x identity): the restriction is the
    # Galerkin one, not a left inverse of P_t
    if M > 1:
        assert np.abs(ml.restrict_time(M, pv) - v).max() > 1e-3


def test_space_time_transfers_commute_and_keep_constants():
    """The STMG transfers are tensor products of the space and the slab
    transfers: either order gives the same values; a field constant in space
    restricts as its slab restriction alone (full weighting keeps spatial
    constants); the prolongation keeps constants (linear interpolation,
    nodal polynomial evaluation)."""
    shape, M = (8, 8), 3
    v = stgen.random_field((4, M, 64), 31)
    a = ml.restrict_space_time(P, shape, M, v)
    b = ml.restrict_space(P, shape, ml.restrict_time(M, v))
    assert a.shape == (2, M, 16)
    assert np.abs(a - b).max() < 1e-15
    t = stgen.random_field((4, M, 1), 33)
    flat = np.broadcast_to(t, (4, M, 64))
    assert np.abs(ml.restrict_space_time(P, shape, M, flat) - ml.restrict_time(M, t)).max() < 1e-14
    assert np.abs(ml.prolong_space_time(P, shape, M, np.full((2, M, 16), -1.3)) + 1.3).max() < 1e-14
    w = stgen.random_field((2, M, 16), 32)
    c = ml.prolong_space_time(P, shape, M, w)
    d = ml.prolong_time(M, ml.prolong_space(P, shape, w))
    assert c.shape == (4, M, 64)
    assert np.abs(c - d).max() < 1e-15


def test_exact_block_jacobi_with_omega1_is_nilpotent():
    """Undamped block Jacobi in time with exact slab solves solves slab k
    exactly after k sweeps (the system is block lower bidiagonal)."""
    lev = ml.Level(shape=(4,), bc=P, Nt=4, M=2, dt=0.2, nu=0.5, X=1.0, cbar=np.zeros((4, 4)))
    r = stgen.random_field((4, 2, 4), 27)
    e = np.zeros_like(r)
    for _ in range(4):
        e = ml.smoothing_step_exact(lev, e, r, 1.0)
    assert np.abs(e - ml.coarse_solve_exact(lev, r)).max() < 1e-13


@pytest.mark.parametrize("reaction", [space.LOGISTIC, space.CUBIC])
def test_level_with_node_derivatives_is_exact_jacobian(reaction):
    """A level carrying R'(U) per node is minus the exact Jacobian of G:
    r - A e + C e = r + dG(U)[e], and dG(U)[e] matches a central difference
    of G (exact up to rounding for the quadratic logistic term; O(eps^2)
    for the cubic)."""
    p = system.Problem(shape=(6, 5), bc=P, nu=0.1, Nt=3, M=3, T=0.3, reaction=reaction, rho=2.0)
    U = stgen.random_field((3, 3, 30), 34, 0.4) + 0.3
    u0 = stgen.random_field((30,), 35)
    lev = ml.Level(shape=p.shape, bc=P, Nt=3, M=3, dt=p.dt, nu=p.nu, X=1.0,
                   cbar=system.cbar(p, U), cnode=p.dR(U))
    e = stgen.random_field((3, 3, 30), 36)
    r = stgen.random_field((3, 3, 30), 37)
    got = ml.linear_residual(lev, e, r)
    Je = system.jacobian_apply(p, U, e)
    assert np.abs(got - (r + Je)).max() < 1e-13
    h = 1e-5
    fd = (system.residual(p, U + h * e, u0) - system.residual(p, U - h * e, u0)) / (2 * h)
    assert np.abs(fd.reshape(Je.shape) - Je).max() < 1e-8


@pytest.mark.parametrize("M", [2, 3, 5])
def test_jacobi_smoothing_step_tends_to_exact(M):
    """Many Jacobi sweeps on the eigen-decoupled slab systems (complex shifts
    for M >= 2) reproduce the exact slab solve of the assembled matrix."""
    lev = ml.Level(shape=(6, 5), bc=P, Nt=3, M=M, dt=0.05, nu=0.1, X=1.0,
                   cbar=stgen.random_field((3, 30), 28, 0.3))
    r = stgen.random_field((3, M, 30), 29)
    e = stgen.random_field((3, M, 30), 30)
    ref = ml.smoothing_step_exact(lev, e, r, 0.8)
    got = ml.smoothing_step_jacobi(lev, e, r, 0.8, 200, 0.8)
    assert np.abs(got - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


def test_jacobi_smoothing_step_without_spatial_operator():
    """With L + diag cbar = 0 every slab system is the identity, so a single
    undamped sweep is already the exact slab solve."""
    lev = ml.Level(shape=(5,), bc=P, Nt=4, M=3, dt=0.1, nu=0.0, X=1.0, cbar=np.zeros((4, 5)))
    r = stgen.random_field((4, 3, 5), 32)
    e = stgen.random_field((4, 3, 5), 33)
    ref = ml.smoothing_step_exact(lev, e, r, 0.7)
    got = ml.smoothing_step_jacobi(lev, e, r, 0.7, 1, 1.0)
    assert np.abs(got - ref).max() < 1e-13


def test_jacobi_smoothing_step_damps_oscillatory_error():
    """A few sweeps remove most of a checkerboard slab error (the part the
    smoother is responsible for) but leave most of a spatially constant one
    (which Jacobi reduces only through the shift's diagonal, 1 + 4 dt lambda nu / h^2)."""
    n = 16
    lev = ml.Level(shape=(n, n), bc=P, Nt=1, M=3, dt=0.1, nu=0.05, X=1.0, cbar=np.zeros((1, n * n)))
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    r = np.zeros((1, 3, n * n))
    checker = ((-1.0) ** (ii + jj)).ravel()
    for u, expect_small in ((checker, True), (np.ones(n * n), False)):
        e_true = np.tile(u, (1, 3, 1))
        r = ml.apply_A(lev, e_true)          # A e_true = r with a single slab
        e = ml.smoothing_step_jacobi(lev, np.zeros_like(r), r, 1.0, 5, 0.8)
        rel = np.abs(e - e_true).max() / np.abs(e_true).max()
        assert (rel < 0.05) if expect_small else (rel > 0.5), rel


# -------------------------------------------------------------------- sdc

def test_sdc_m1_is_implicit_euler():
    """M = 1 with implicit-Euler QI: one sweep of the linear heat equation is
    an implicit Euler step from the previous iterate's slab-end value."""
    p = system.Problem(shape=(7,), bc=D, nu=1.0, Nt=3, M=1, T=0.3)
    u0 = stgen.sine_modes(7)
    U = stgen.random_field((3, 1, 7), 31)
    Un = sdc.sdc_sweep(p, U, u0)
    A = np.eye(7) - p.dt * p.L.toarray()
    prev = [u0, U[0, 0], U[1, 0]]
    for n in range(3):
        assert np.abs(Un[n, 0] - np.linalg.solve(A, prev[n])).max() < 1e-13


@pytest.mark.parametrize("kind", ["IE", "LU"])
def test_sdc_fixed_point_and_convergence(kind):
    p = system.Problem(shape=(8, 8), bc=P, nu=0.01, Nt=4, M=3, T=0.2, reaction=space.LOGISTIC, rho=1.0)
    u0 = stgen.smoothed_noise((8, 8), 32).ravel()
    Ustar = system.solve_sequential(p, u0)
    assert np.abs(sdc.sdc_sweep(p, Ustar, u0, kind) - Ustar).max() < 1e-14
    U = np.tile(u0, (p.Nt, p.M, 1))
    for _ in range(30):
        U = sdc.sdc_sweep(p, U, u0, kind)
    assert np.abs(U - Ustar).max() < 1e-12


def test_transposed_level_operator_dot_product():
    """<(A - C) e, v> = <e, (A^T - C^T) v> for the level operators."""
    lev = ml.Level(shape=(6,), bc=P, Nt=4, M=3, dt=0.1, nu=0.3, X=1.0,
                   cbar=stgen.random_field((4, 6), 28, 0.3))
    e = stgen.random_field((4, 3, 6), 29)
    v = stgen.random_field((4, 3, 6), 30)
    z = np.zeros_like(e)
    lhs = float(np.sum(-ml.linear_residual(lev, e, z) * v))
    rhs = float(np.sum(e * -ml.linear_residual_T(lev, v, z)))
    assert abs(lhs - rhs) < 1e-12 * max(1, abs(lhs))
    r = stgen.random_field((4, 3, 6), 31)
    x = ml.coarse_solve_exact_T(lev, r)
    assert np.abs(ml.linear_residual_T(lev, x, r)).max() < 1e-13


def test_residual_points_matches_full_residual():
    for bc, shape in [(P, (6, 8)), (D, (5, 3, 7)), (N, (9,))]:
        p = system.Problem(shape=shape, bc=bc, nu=0.2, Nt=3, M=3, reaction=space.CUBIC, rho=1.5)
        Ns = int(np.prod(shape))
        U = stgen.random_field((3, 3, Ns), 50)
        u0 = stgen.random_field((Ns,), 51)
        G = system.residual(p, U, u0)
        slabs = [0, 1, 2, 2, 0]
        pts = [0, Ns - 1, Ns // 2, 1, Ns // 3]
        Gp = system.residual_points(p, U, u0, slabs, pts)
        for t, (n, s) in enumerate(zip(slabs, pts)):
            assert np.abs(Gp[t] - G[n, :, s]).max() < 1e-11


@pytest.mark.parametrize("shape,bc,M,rx", [((24, 20), space.PERIODIC, 3, space.LOGISTIC),
                                           ((6, 8, 4), space.PERIODIC, 2, space.CUBIC),
                                           ((17, 9), space.DIRICHLET, 3, space.LOGISTIC),
                                           ((33,), space.NEUMANN, 5, space.CUBIC)])
def test_krylov_slab_solves_match_direct(monkeypatch, shape, bc, M, rx):
    """The large-slab path of the sequential solve (matrix-free GMRES, with the
    exact constant-coefficient inverse as preconditioner on periodic grids)
    gives the solution of the sparse-LU path, forced here on small sizes."""
    p = system.Problem(shape=shape, bc=bc, nu=0.05, Nt=3, M=M, T=0.3, reaction=rx, rho=1.5)
    u0 = stgen.random_field(shape, 77, 0.4).ravel() + 0.5
    direct = system.solve_sequential(p, u0)
    monkeypatch.setattr(system, "_DIRECT_MAX", 0)
    krylov = system.solve_sequential(p, u0)
    assert np.abs(krylov - direct).max() <= 1e-13 * np.abs(direct).max()
    assert np.abs(system.residual(p, krylov, u0)).max() < 1e-13


@pytest.mark.parametrize("shape", [(8, 6, 10), (12, 16), (20,), (2, 5)])
def test_periodic_slab_inverse_is_exact_for_constant_coefficient(shape):
    """periodic_slab_inverse(c) inverts the assembled slab Jacobian when
    R'(U) = c everywhere (logistic at U = (1 - c/rho)/2), on 1D-3D grids,
    including the two-point periodic Laplacian."""
    p = system.Problem(shape=shape, bc=space.PERIODIC, nu=0.2, Nt=4, M=3, T=0.4, reaction=space.LOGISTIC, rho=2.0)
    c = -0.7
    Un = np.full((p.M, p.Ns), (1.0 - c / p.rho) / 2.0)
    assert np.allclose(p.dR(Un), c)
    A = system.slab_jacobian(p, Un).toarray()
    Pinv = system.periodic_slab_inverse(p, c)
    v = stgen.random_field((p.M * p.Ns,), 5)
    assert np.abs(Pinv.matvec(A @ v) - v).max() < 1e-12
