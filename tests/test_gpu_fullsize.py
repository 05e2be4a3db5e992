"""The remaining workloads at full size, solved through the C ABI in the
configuration bench.py uses (FP32 cycle + FP64-accurate residual):

  2D logistic 1024^2 periodic, Nt=1024, M=3 (3.2e9 space-time dofs) and M=5
  3D cubic 128^3 periodic, Nt=128, M=3 (8e8 dofs)
  adjoint: 2D logistic 512^2, Nt=512, M=3 (4e8 dofs)

The oracle cannot solve them whole, so each is checked on what it can compute:
the error against the oracle's solution of the first K slabs at full spatial
resolution (the system of Eq. 3.4 is block lower bidiagonal, so by causality
the first K slabs of the full solution are the K-slab problem's solution);
the collocation residual (Eq. 2.3 + slab coupling) evaluated point by point at
sampled (slab, point) pairs of the GPU solution; and the complete residual of
the first and the last slab.  The adjoint gradients are checked by the
transposition identity and by exact directional derivatives of the FP64
residual."""
import numpy as np
import pytest

import stgen
from oracle import adjoint as oadj
from oracle import space, system
from tests.gpu_cases import Case, residual_scale

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _sampled_residual(case, p, U, u0, nsamples=48, seed=0):
    """max |G| over sampled (slab, point) pairs, from two slabs copied to the host."""
    rng = np.random.default_rng(seed)
    worst = 0.0
    Ns = p.Ns
    p2 = p.with_params(Nt=2, T=2 * p.dt)
    scale = 0.0
    for _ in range(nsamples):
        n = int(rng.integers(0, case.Nt))
        s = int(rng.integers(0, Ns))
        cur = U[n].reshape(p.M, Ns).double().cpu().numpy()
        if n == 0:
            g = system.residual_points(p.with_params(Nt=1, T=p.dt), cur[None], u0, [0], [s])
        else:
            prv = U[n - 1].reshape(p.M, Ns).double().cpu().numpy()
            sub = np.stack([prv, cur])
            g = system.residual_points(p2, sub, u0, [1], [s])
        worst = max(worst, float(np.abs(g).max()))
        scale = max(scale, residual_scale(p, cur))
    return worst, scale


def _truncation_error(p, U, u0, K):
    """Relative 2-norm error of the GPU's first K slabs against the oracle's
    solve of the K-slab problem (same dt, full spatial resolution)."""
    pk = p.with_params(Nt=K, T=K * p.dt)
    ref = system.solve_sequential(pk, u0)
    got = U[:K].reshape(K, p.M, -1).double().cpu().numpy()
    assert np.abs(system.residual(pk, ref, u0)).max() < 1e-13
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref)), float(np.abs(got[-1, -1] - ref[-1, -1]).max())


def _check_solution(case, tol=1e-10, K=2):
    from paper_2006_12883_gb300 import stlib
    p = case.problem()
    u0 = case.u0()
    S = case.solver(precision=stlib.FP32_REFINE, tol=tol, max_iters=80)
    U = S.zeros()
    info = S.solve(U)
    assert info["status"] == 0 and info["rel_residual"] <= tol, info
    # error against the oracle by time truncation (FP32 cycle + FP64
    # refinement: within 1e-8 relative)
    rel, mx = _truncation_error(p, U, u0, K)
    print(f"\n[truncation] {case.name}: first {K} slabs, rel 2-norm error {rel:.3e}, max error at the "
          f"last node {mx:.3e}, GPU rel residual {info['rel_residual']:.3e}, cycles {info['cycles']}")
    assert rel <= 1e-8, rel
    worst, scale = _sampled_residual(case, p, U, u0)
    ref = system.reference_norm(p, u0)
    assert worst <= tol * ref + 1e-13 * scale, (worst, tol * ref, scale)
    # complete residuals of the first and the last slab
    first = U[0].reshape(1, p.M, -1).double().cpu().numpy()
    g0 = system.residual(p.with_params(Nt=1, T=p.dt), first, u0)
    last2 = U[-2:].reshape(2, p.M, -1).double().cpu().numpy()
    prev = U[-3, -1].reshape(-1).double().cpu().numpy()
    gl = system.residual(p.with_params(Nt=2, T=2 * p.dt), last2, prev)
    bound = tol * ref + 1e-13 * max(residual_scale(p, first), residual_scale(p, last2))
    assert float(np.linalg.norm(g0)) <= bound, (float(np.linalg.norm(g0)), bound)
    assert float(np.linalg.norm(gl)) <= bound, (float(np.linalg.norm(gl)), bound)
    S.close()
    del U
    torch.cuda.empty_cache()
    return info


def test_logistic2d_1024_m3():
    _check_solution(Case("logistic2d_1024_m3", (1024, 1024), space.PERIODIC, 1e-2, 1024, 3,
                         reaction=space.LOGISTIC, rho=1.0, u0_kind="noise", seed=12885))


def test_logistic2d_1024_m5():
    _check_solution(Case("logistic2d_1024_m5", (1024, 1024), space.PERIODIC, 1e-2, 1024, 5,
                         reaction=space.LOGISTIC, rho=1.0, u0_kind="noise", seed=12885))


def test_cubic3d_128():
    _check_solution(Case("cubic3d_128", (128, 128, 128), space.PERIODIC, 5e-3, 128, 3,
                         reaction=space.CUBIC, rho=2.0, u0_kind="bumps", seed=12886))


def test_adjoint_512_exact_identities():
    """Adjoint at 512^2 x 512 slabs x M = 3 (gradient of 1/2 h^2 |u(T) - u_target|^2
    at (nu, rho) = (1e-2, 1), target from (1.3e-2, 0.8)), checked by identities
    that hold at any size.  G is quadratic in U and linear in nu, rho and u0, so
    central differences of the FP64 residual are exact up to rounding:
      J v       = (G(U + e v) - G(U - e v)) / 2e,
      dG/dtheta = (G(theta + e) - G(theta - e)) / 2e.
    Then <lambda, J v> = -<g, v> (lambda solves J^T lambda = -g) and
    dPhi/dtheta = <lambda, dG/dtheta>."""
    from paper_2006_12883_gb300 import stlib
    case = Case("adjoint_512", (512, 512), space.PERIODIC, 1e-2, 512, 3, reaction=space.LOGISTIC, rho=1.0,
                u0_kind="noise", seed=12887)
    p = case.problem()
    h2 = (1.0 / 512) ** 2
    S = case.solver(precision=stlib.FP32_REFINE, tol=1e-11, max_iters=80)
    S.set_params(1.3e-2, 0.8)
    V = S.zeros()
    assert S.solve(V)["status"] == 0
    target = V[-1, -1].reshape(-1).clone()
    S.set_params(case.nu, case.rho)
    U = S.zeros()
    assert S.solve(U)["status"] == 0
    du0 = torch.empty(p.Ns, dtype=torch.float64, device="cuda")
    dnu, drho, info = S.adjoint(U, target=target, du0=du0)
    assert info["status"] == 0, info
    lam = S.adjoint_lambda()
    gT = h2 * (U[-1, -1].reshape(-1) - target)
    # the last K slabs of lambda against the oracle's backward solve of those
    # slabs: J^T is block upper bidiagonal, so the window needs only the
    # terminal data and the window's U
    K = 2
    pk = p.with_params(Nt=K, T=K * p.dt)
    lam_ref = oadj.adjoint_solve(pk, U[-K:].reshape(K, p.M, -1).double().cpu().numpy(), gT.cpu().numpy())
    lam_w = lam[-K:].reshape(K, p.M, -1).double().cpu().numpy()
    err = float(np.linalg.norm(lam_w - lam_ref) / np.linalg.norm(lam_ref))
    print(f"\n[adjoint window] adjoint_512: last {K} slabs, rel 2-norm error of lambda {err:.3e}, "
          f"adjoint rel residual {info['rel_residual']:.3e}")
    assert err <= 1e-6, err

    def G(Uv, nu=case.nu, rho=case.rho, u0=None):
        S.set_params(nu, rho)
        if u0 is not None:
            S.set_u0(u0)
        R = torch.empty_like(Uv)
        S.residual(Uv, R, fp64=True)
        return R

    def dot(a, b):
        return float((a.double() * b.double()).sum())

    v = torch.tensor(stgen.random_field((p.Nt, p.M, p.Ns), 101), device="cuda").reshape(U.shape)
    e = 1e-3
    Jv = (G(U + e * v) - G(U - e * v)) / (2 * e)
    lhs, rhs = dot(lam, Jv), -dot(gT, v[-1, -1].reshape(-1))
    assert abs(lhs - rhs) <= 1e-7 * abs(rhs), (lhs, rhs)
    for name, g, kw in (("nu", dnu, "nu"), ("rho", drho, "rho")):
        th = getattr(case, name)
        d = 1e-3 * th
        dG = (G(U, **{kw: th + d}) - G(U, **{kw: th - d})) / (2 * d)
        ref = dot(lam, dG)
        assert abs(g - ref) <= 1e-8 * abs(ref), (name, g, ref)
    u0 = torch.tensor(case.u0(), device="cuda")
    w = torch.tensor(stgen.random_field((p.Ns,), 99), device="cuda")
    dG = (G(U, u0=u0 + e * w) - G(U, u0=u0 - e * w)) / (2 * e)
    assert abs(dot(du0, w) - dot(lam, dG)) <= 1e-8 * abs(dot(lam, dG))
    S.close()


def test_adjoint_512_checkpointed_matches_stored_and_saves_memory():
    """The adjoint workload (512^2 x 512 slabs x M = 3, gradient of
    1/2 h^2 |u(T) - u_target|^2) with slab recomputation checkpointing in
    blocks of 64 slabs: the gradients equal the stored-U path's, with a
    fraction of its device memory."""
    from paper_2006_12883_gb300 import stlib
    case = Case("adjoint_512", (512, 512), space.PERIODIC, 1e-2, 512, 3, reaction=space.LOGISTIC, rho=1.0,
                u0_kind="noise", seed=12887)
    p = case.problem()
    h2 = (1.0 / 512) ** 2
    gT = torch.tensor(stgen.random_field((p.Ns,), 81, h2), device="cuda")
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    torch.cuda.reset_peak_memory_stats()
    base = torch.cuda.memory_allocated()
    S = case.solver(precision=stlib.FP32_REFINE, tol=1e-11, max_iters=80)
    U = S.zeros()
    assert S.solve(U)["status"] == 0
    du0 = torch.empty(p.Ns, dtype=torch.float64, device="cuda")
    dnu, drho, info = S.adjoint(U, gT=gT, du0=du0)
    assert info["status"] == 0
    uT = U[-1, -1].clone()
    peak_stored = torch.cuda.max_memory_allocated() - base
    S.close()
    del U
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    torch.cuda.reset_peak_memory_stats()
    base = torch.cuda.memory_allocated()
    C = stlib.CheckpointSolver(case.shape, case.bc, case.nu, case.Nt, case.M, case.u0(), 64, T=case.T,
                               reaction=case.reaction, rho=case.rho,
                               opts=stlib.make_opts(precision=stlib.FP32_REFINE, tol=1e-11, max_iters=80))
    cuT, finfo = C.forward()
    assert finfo["status"] == 0
    cdu0 = torch.empty_like(du0)
    cnu, crho, ainfo = C.adjoint(gT, du0=cdu0)
    assert ainfo["status"] == 0
    peak_ckpt = torch.cuda.max_memory_allocated() - base
    C.close()
    print(f"\n[checkpointing] adjoint_512: blocks of 64 slabs, peak device memory {peak_ckpt / 1e9:.2f} GB "
          f"vs {peak_stored / 1e9:.2f} GB stored; dnu {cnu:.9e} vs {dnu:.9e}, drho {crho:.9e} vs {drho:.9e}")
    assert float((cuT - uT).abs().max()) <= 1e-9 * float(uT.abs().max())
    assert abs(cnu - dnu) <= 1e-8 * abs(dnu) and abs(crho - drho) <= 1e-8 * abs(drho)
    assert float((cdu0 - du0).norm()) <= 1e-8 * float(du0.norm())
    assert peak_ckpt < 0.3 * peak_stored
