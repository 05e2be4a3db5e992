"""End-to-end solves through the C ABI (V-cycles inside FP64 defect
correction / Newton) and SDC sweeps, against the oracle's direct solution of
the collocation system; closed forms; error handling."""
import math

import numpy as np
import pytest

import stgen
from oracle import sdc as osdc
from oracle import space, system
from tests.gpu_cases import HEAT1D, LOG2D, MONO, SOLVE_CASES, TILED_HEAT3, TILED_LOG5, TILED_M5, Case

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


_REF = {}


def _oracle_solution(case):
    if case.name not in _REF:
        _REF[case.name] = system.solve_sequential(case.problem(), case.u0())
    return _REF[case.name]


@pytest.mark.parametrize("case", SOLVE_CASES, ids=lambda c: c.name)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_solve_matches_oracle(case, prec):
    from paper_2006_12883_gb300 import stlib
    tol = 1e-12
    if prec == "fp32" and case in (TILED_LOG5, TILED_HEAT3):
        # the double-float residual carries a few 1e-14 of its largest term,
        # here dt nu / h^2 = 27 times |u|: the FP32 path's relative residual
        # stops near 3e-12 on these grids (the all-FP64 path goes on)
        tol = 1e-10
    S = case.solver(precision=stlib.FP64 if prec == "fp64" else stlib.FP32_REFINE, tol=tol, max_iters=200)
    U = S.zeros()
    info = S.solve(U)
    assert info["status"] == 0 and info["rel_residual"] <= tol
    ref = _oracle_solution(case)
    err = _rel(U.cpu().numpy().reshape(ref.shape), ref)
    print(f"\n[oracle] {case.name} {prec}: rel 2-norm error {err:.3e}, rel residual {info['rel_residual']:.3e}, "
          f"cycles {info['cycles']}")
    # all-FP64 path within 1e-10, FP32 cycle + FP64 refinement within 1e-8
    assert err <= (1e-10 if prec == "fp64" else 1e-8), err
    h = info["history"]
    assert all(b < a for a, b in zip(h[1:], h[2:])), h  # monotone after the first cycle
    S.close()


@pytest.mark.parametrize("case", [TILED_LOG5, TILED_HEAT3], ids=lambda c: c.name)
def test_vcycle_iteration_matches_oracle(case):
    """st_vcycle repeated from zero (on these grids every step runs the fine
    residual with the first smoothing step, the two-sweep kernel that also
    updates U and the level residual with its restriction) converges to the
    oracle's collocation solution."""
    from paper_2006_12883_gb300 import stlib
    S = case.solver(precision=stlib.FP32_REFINE)
    U = S.zeros()
    norms = [S.vcycle(U) for _ in range(25)]
    assert S.stats()["update_in_cycle"] == 1
    assert norms[-1] <= 1e-10 * norms[0], norms
    ref = _oracle_solution(case)
    err = _rel(U.cpu().numpy().reshape(ref.shape), ref)
    print(f"\n[oracle] {case.name} st_vcycle x 25: rel 2-norm error {err:.3e}")
    assert err <= 1e-8, err
    S.close()


def test_heat_closed_form_and_vcycle_api():
    from paper_2006_12883_gb300 import stlib
    case = HEAT1D
    S = case.solver(precision=stlib.FP64, tol=1e-13)
    U = S.zeros()
    norms = [S.vcycle(U) for _ in range(30)]
    assert norms[-1] < 1e-11 * norms[0]
    x = stgen.coords1d(space.DIRICHLET, 63)
    p = case.problem()

    def R(z):
        return (1 + z / 3) / (1 - 2 * z / 3 + z * z / 6)

    exact = sum(a * R(p.dt * system.sine_mode_eigenvalue(k, 63, 1.0)) ** 16 * np.sin(k * np.pi * x)
                for k, a in ((1, 1.0), (3, 0.5)))
    assert np.abs(U.cpu().numpy()[-1, -1] - exact).max() < 1e-11
    S.close()


@pytest.mark.parametrize("coarsening", [0, 1])
def test_space_only_and_auto_mu(coarsening):
    from paper_2006_12883_gb300 import stlib
    S = LOG2D.solver(coarsening=coarsening, tol=1e-10, max_iters=100)
    U = S.zeros()
    info = S.solve(U)
    assert info["status"] == 0
    ref = _oracle_solution(LOG2D)
    assert _rel(U.cpu().numpy().reshape(ref.shape), ref) < 1e-8
    S.close()


def test_host_pointer_solve():
    case = LOG2D
    S = case.solver(tol=1e-10)
    U = torch.zeros(S.field_shape, dtype=torch.float64)  # host memory
    info = S.solve(U)
    assert info["status"] == 0
    ref = _oracle_solution(case)
    assert _rel(U.numpy().reshape(ref.shape), ref) < 1e-8
    S.close()


def test_full_size_sampled_residual_and_truncation():
    """2D logistic at 256^2 x 256 slabs x M=3 (50M space-time dofs): the GPU
    solution's collocation residual, evaluated point by point by the oracle at
    sampled points, is at the solver tolerance; the whole solution matches the
    oracle's slab-by-slab solve of all 256 slabs."""
    from paper_2006_12883_gb300 import stlib
    case = Case("logistic2d_256", (256, 256), space.PERIODIC, 1e-2, 256, 3, reaction=space.LOGISTIC, rho=1.0,
                u0_kind="noise", seed=12884)
    S = case.solver(tol=1e-10, max_iters=60)
    U = S.zeros()
    info = S.solve(U)
    assert info["status"] == 0, info
    Uh = U.cpu().numpy().reshape(case.Nt, case.M, -1)
    p = case.problem()
    u0 = case.u0()
    rng = np.random.default_rng(0)
    slabs = list(rng.integers(0, case.Nt, 64))
    pts = list(rng.integers(0, p.Ns, 64))
    Gs = system.residual_points(p, Uh, u0, slabs, pts)
    from tests.gpu_cases import residual_scale
    bound = 1e-10 * system.reference_norm(p, u0) + 1e-13 * residual_scale(p, Uh[:2])
    assert np.abs(Gs).max() <= bound, (np.abs(Gs).max(), bound)
    ref = system.solve_sequential(p, u0)
    err = _rel(Uh, ref)
    print(f"\n[oracle] logistic2d_256: all {case.Nt} slabs, rel 2-norm error {err:.3e}, GPU rel residual "
          f"{info['rel_residual']:.3e}, cycles {info['cycles']}")
    assert err < 1e-8
    S.close()


# ------------------------------------------------------------------ SDC

@pytest.mark.parametrize("case", [HEAT1D, LOG2D, MONO], ids=lambda c: c.name)
@pytest.mark.parametrize("kind", [0, 1])
def test_sdc_one_sweep_matches_oracle(case, kind):
    """One IMEX sweep (correction form, converged inner solves) equals the
    oracle's standard-form sweep with exact spatial solves."""
    from paper_2006_12883_gb300 import stlib
    p = case.problem()
    S = case.solver(precision=stlib.FP64, sdc_qdelta=kind, sdc_inner_cycles=40, inner_coarse_iters=60)
    U0 = stgen.random_field((p.Nt, p.M, p.Ns), 21, 0.2) + np.tile(case.u0(), (p.Nt, p.M, 1))
    U = torch.tensor(U0, device="cuda").reshape(S.field_shape)
    S.sdc_sweep(U, 1)
    ref = osdc.sdc_sweep(p, U0, case.u0(), "IE" if kind == 0 else "LU")
    assert _rel(U.cpu().numpy().reshape(ref.shape), ref) < 1e-9
    S.close()


@pytest.mark.parametrize("case", [LOG2D, TILED_M5], ids=lambda c: c.name)
def test_sdc_fp32_sweep_matches_oracle(case):
    """The same sweep with the FP32 node solves (one-plane float4 spatial
    multigrid on periodic 2D grids) inside the FP64 sweep: equal to the
    oracle's exact-solve sweep to FP32 accuracy."""
    from paper_2006_12883_gb300 import stlib
    p = case.problem()
    S = case.solver(precision=stlib.FP32_REFINE, sdc_inner_cycles=30, inner_coarse_iters=60)
    U0 = stgen.random_field((p.Nt, p.M, p.Ns), 23, 0.2) + np.tile(case.u0(), (p.Nt, p.M, 1))
    U = torch.tensor(U0, device="cuda").reshape(S.field_shape)
    S.sdc_sweep(U, 1)
    ref = osdc.sdc_sweep(p, U0, case.u0(), "IE")
    assert _rel(U.cpu().numpy().reshape(ref.shape), ref) < 2e-6
    S.close()


def test_sdc_converges_to_collocation():
    """Config-1 heat problem: SDC sweeps from the spread initial value reach a
    1e-10 residual and the collocation solution."""
    from paper_2006_12883_gb300 import stlib
    case = HEAT1D
    p = case.problem()
    S = case.solver(precision=stlib.FP32_REFINE, sdc_inner_cycles=3)
    U = torch.tensor(np.tile(case.u0(), (p.Nt, p.M, 1)), device="cuda").reshape(S.field_shape)
    r0 = system.reference_norm(p, case.u0())
    rel = 1.0
    for _ in range(200):
        S.sdc_sweep(U, 1)
        rel = S.residual(U) / r0
        if rel < 1e-10:
            break
    assert rel < 1e-10
    ref = _oracle_solution(case)
    assert _rel(U.cpu().numpy().reshape(ref.shape), ref) < 1e-8
    S.close()


# ------------------------------------------------------------- failures

def test_error_statuses():
    from paper_2006_12883_gb300 import stlib
    p = stlib.make_problem((8,), stlib.PERIODIC, -1.0, 4, 2)  # nu <= 0
    with pytest.raises(stlib.StError) as ei:
        stlib.st_plan(p)
    assert ei.value.status == stlib.ST_ERR_INVALID_ARG
    p = stlib.make_problem((100, 100), stlib.PERIODIC, 1.0, 4, 2)  # 100 -> 50 -> 25: coarsest too big
    with pytest.raises(stlib.StError) as ei:
        stlib.st_plan(p)
    assert ei.value.status == stlib.ST_ERR_UNSUPPORTED
    # max_iters = 1: not converged, info filled
    S = LOG2D.solver(max_iters=1, tol=1e-14)
    U = S.zeros()
    info = S.solve(U, raise_on_error=False)
    assert info["status"] == stlib.ST_ERR_NOT_CONVERGED and info["iterations"] == 1
    S.close()
    # NaN in u0: diverged, no abort
    bad = Case("nan", (16, 16), space.PERIODIC, 0.01, 4, 2, reaction=space.LOGISTIC, rho=1.0)
    u0 = bad.u0()
    u0[5] = np.nan
    S = stlib.Solver(bad.shape, bad.bc, bad.nu, bad.Nt, bad.M, u0, reaction=bad.reaction, rho=1.0)
    info = S.solve(S.zeros(), raise_on_error=False)
    assert info["status"] == stlib.ST_ERR_DIVERGED
    S.close()


def test_bounded_wait_expiry_is_reported_once_and_handle_survives():
    """Failure detection on the GPU without a fault: one block waits on an
    mbarrier that nothing completes, with the bounded wait of the TMA-staged
    kernels.  The wait expires, the block counts it and returns; the host
    reports ST_ERR_TIMEOUT once, and the handle keeps working (residuals and
    asynchronous V-cycles give the same numbers as before, no stale report)."""
    from paper_2006_12883_gb300 import stlib
    p = LOG2D.problem()
    S = LOG2D.solver(precision=stlib.FP32_REFINE)
    U = torch.tensor(stgen.random_field((p.Nt, p.M, p.Ns), 5, 0.3) + 0.4, device="cuda").reshape(S.field_shape)
    n0 = S.residual(U)
    assert S.wait_selftest() == stlib.ST_ERR_TIMEOUT
    assert S.residual(U) == n0
    V = U.clone()
    a = [S.vcycle(V) for _ in range(3)]
    assert S.residual(V) < a[0]
    S.close()


def test_allocator_failure_is_oom():
    from paper_2006_12883_gb300 import stlib
    import ctypes
    case = LOG2D
    u0 = torch.tensor(case.u0())
    prob = stlib.make_problem(case.shape[::-1], case.bc, case.nu, case.Nt, case.M, reaction=case.reaction,
                              rho=case.rho, u0_ptr=u0.data_ptr())
    rt = stlib.StRuntime()
    rt.stream = None
    rt.alloc = stlib.ALLOC_FN(lambda n, s, c: None)
    rt.free = stlib.FREE_FN(lambda p, n, s, c: None)
    h = ctypes.c_void_p()
    s = stlib.lib().st_create(ctypes.byref(prob), None, ctypes.byref(rt), ctypes.byref(h))
    assert s == stlib.ST_ERR_OOM and not h.value


# The paper's monodomain problem (Section 5.4: X = 10, T = 2, gamma = 5, a
# narrow stimulus) on a coarser grid.  From the zero initial guess the first
# Newton correction follows the linearisation at u = 0, which grows like
# e^{5t}; only a damped step keeps the iteration in range.
MONO_LS = Case("monodomain_ls", (257,), space.NEUMANN, 1.0, 256, 3, T=2.0, X=10.0, reaction=space.CUBIC,
               rho=5.0, u0_kind="stimulus")


@pytest.mark.parametrize("ej", [0, 1], ids=["cbar", "exactJ"])
def test_monodomain_with_line_search(ej):
    from paper_2006_12883_gb300 import stlib
    case = MONO_LS
    S = case.solver(precision=stlib.FP64, tol=1e-11, max_iters=200, exact_jacobian=ej)
    U = S.zeros()
    info = S.solve(U)
    assert info["status"] == 0, info
    ref = _oracle_solution(case)
    got = U.cpu().numpy().reshape(ref.shape)
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()
    # without the line search the first full step leaves the basin
    S2 = case.solver(precision=stlib.FP64, tol=1e-11, max_iters=200, exact_jacobian=ej, line_search=0)
    U2 = S2.zeros()
    info2 = S2.solve(U2, raise_on_error=False)
    assert info2["status"] != 0 or info2["iterations"] >= info["iterations"]
    S.close()
    S2.close()


# The paper's monodomain configurations of Section 5.4 (N_x = 1024, X = 10,
# T = 2, gamma = 5) at the (M, N_t) pairs of its SMG table.  At these time
# steps the cycle's quasi-Newton correction from the zero guess is no descent
# direction; the solver continues with FGMRES on the exact Jacobian.
@pytest.mark.parametrize("M,Nt", [(3, 32), (5, 8)])
def test_monodomain_paper_configs(M, Nt):
    from paper_2006_12883_gb300 import stlib
    case = Case(f"monodomain_paper_m{M}", (1025,), space.NEUMANN, 1.0, Nt, M, T=2.0, X=10.0,
                reaction=space.CUBIC, rho=5.0, u0_kind="stimulus")
    S = case.solver(precision=stlib.FP64, tol=1e-11, max_iters=300)
    U = S.zeros()
    info = S.solve(U)
    assert info["status"] == 0, info
    assert info["cycles"] > info["iterations"]  # the Krylov steps took over
    ref = _oracle_solution(case)
    got = U.cpu().numpy().reshape(ref.shape)
    assert np.abs(got - ref).max() <= 1e-8 * np.abs(ref).max()
    # the same with the Krylov steps requested from the start
    S2 = case.solver(precision=stlib.FP64, tol=1e-11, max_iters=300, krylov=10, exact_jacobian=1)
    U2 = S2.zeros()
    assert S2.solve(U2)["status"] == 0
    assert np.abs(U2.cpu().numpy().reshape(ref.shape) - ref).max() <= 1e-8 * np.abs(ref).max()
    S.close()
    S2.close()


def test_krylov_step_on_linear_problem():
    """For a linear problem FGMRES with the V-cycle preconditioner solves the
    all-at-once system in one outer iteration to the Krylov tolerance."""
    from paper_2006_12883_gb300 import stlib
    case = HEAT1D
    S = case.solver(precision=stlib.FP64, tol=1e-6, krylov=20, krylov_rtol=1e-8)
    U = S.zeros()
    info = S.solve(U)
    assert info["status"] == 0 and info["iterations"] == 1, info
    assert info["rel_residual"] <= 1e-7
    S.close()


@pytest.mark.parametrize("M,Nt", [(1, 1024), (2, 256), (3, 32), (4, 16), (5, 8)])
def test_heat_paper_configs_closed_form(M, Nt):
    """The paper's heat example (Section 5.3, Eq. 5.1 data, N_x = 1024,
    Neumann) at its (M, N_t) pairs: the cosine modes are exact eigenvectors of
    the mirrored-ghost Laplacian with eigenvalues rho_k (Eq. 5.3), so the
    fully discrete end value is sum_k c_k R(dt rho_k)^Nt cos(k pi x) with R the
    Radau IIA stability function, up to rounding."""
    from oracle import collocation as col
    from paper_2006_12883_gb300 import stlib
    n = 1025
    case = Case(f"heat_paper_m{M}", (n,), space.NEUMANN, 1.0, Nt, M, u0_kind="cosine")
    # the FP64 residual's rounding floor relative to ||G(0)|| grows like
    # eps * dt * nu * ||Delta_h|| (about 2e-11 at Nt = 32, 1e-10 at Nt = 8), so
    # the large steps stop at 1e-10; the error is still at rounding level
    tol = 1e-12 if Nt >= 256 else 1e-10
    S = case.solver(precision=stlib.FP64, tol=tol, max_iters=400, coarsening=stlib.COARSEN_SPACE, max_levels=7)
    U = S.zeros()
    info = S.solve(U)
    assert info["status"] == 0, info
    Q = col.collocation_matrix(col.radau_right_nodes(M))
    x = stgen.coords1d(space.NEUMANN, n)
    h = 1.0 / (n - 1)
    dt = 1.0 / Nt
    exact = sum(a * col.stability_function(dt * (2 * np.cos(k * np.pi * h) - 2) / h ** 2, Q).real ** Nt
                * np.cos(k * np.pi * x) for k, a in ((1, 1.0), (3, 2.0), (4, 3.0)))
    # exact up to rounding: within 1e-12 of the data's size; u(T) has
    # decayed to about 5e-5 (e^{-pi^2}) of u0, so also within 1e-7 of itself
    u0 = case.u0()
    err = np.abs(U[-1, -1].cpu().numpy() - exact).max()
    print(f"\n[closed form] heat M={M} Nt={Nt}: max error {err:.3e} (max|u0| {np.abs(u0).max():.2f}, "
          f"max|u(T)| {np.abs(exact).max():.3e})")
    assert err <= 1e-12 * np.abs(u0).max()
    assert err <= 1e-7 * np.abs(exact).max()
    S.close()
