"""Level-wise steps of the space-time V-cycle (Eq. 4.1 hierarchy): level
operator residuals (forward and transposed), cbar restriction, space / slab
transfers, the exact coarsest solve and the smoothing step, through the C ABI
against the oracle."""
import numpy as np
import pytest

import stgen
from oracle import multilevel as ml
from oracle import space, system
from tests.gpu_cases import (CUB3D, DIR2D_M5, HEAT1D, LOG2D, PER2D_M5, PER3D_M5, RAGGED, SMMG1D, SMMG2D, STMG1D, STMG2D,
                             TILED_HEAT3, TILED_M5, TILED_SQ3, TILED_SQ5,
                             Case)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

P_ = space.PERIODIC
# a case whose hierarchy mixes space and slab bisection (AUTO_MU) and one
# with space bisection only (SPACE)
MIXED = Case("mixed2d", (32, 32), P_, 2e-3, 16, 3, reaction=space.LOGISTIC, rho=1.0, u0_kind="noise", seed=5)
LEVEL_CASES = [HEAT1D, LOG2D, MIXED, CUB3D, DIR2D_M5, PER2D_M5, PER3D_M5, SMMG2D, SMMG1D, RAGGED, TILED_M5,
               STMG2D, STMG1D]


def _oracle_level(S, case, l, cbar, U=None):
    """The oracle's level l; with U (the linearisation point) level 0 carries
    R'(U) per node, as the library's finest level does with exact_jacobian."""
    li = S.level_info(l)
    d = len(case.shape)
    shape = tuple(li["n"][:d][::-1])
    cnode = None
    if U is not None and l == 0 and case.reaction != space.NONE:
        p = case.problem()
        cnode = p.dR(np.asarray(U).reshape(p.Nt, p.M, p.Ns))
    return ml.Level(shape=shape, bc=case.bc, Nt=li["Nt"], M=li["M"], dt=li["dt"], nu=case.nu, X=case.X,
                    cbar=cbar, cnode=cnode)


def _setup(case, prec, **opts):
    from paper_2006_12883_gb300 import stlib
    p = case.problem()
    S = case.solver(precision=stlib.FP64 if prec == "fp64" else stlib.FP32_REFINE, **opts)
    U = stgen.random_field((p.Nt, p.M, p.Ns), 11, 0.3) + 0.4
    Ut = torch.tensor(U, device="cuda").reshape(S.field_shape)
    S.linearize(Ut)
    return p, S, U


def _tol(prec):
    return 1e-12 if prec == "fp64" else 3e-6


@pytest.mark.parametrize("case", LEVEL_CASES, ids=lambda c: c.name)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cbar_hierarchy(case, prec):
    p, S, U = _setup(case, prec)
    cb = system.cbar(p, U)
    for l in range(S.num_levels()):
        got = S.level_cbar(l).double().cpu().numpy()
        got = got.reshape(got.shape[0], -1)
        assert np.abs(got - cb).max() <= _tol(prec) * max(1, np.abs(cb).max()), l
        if l + 1 < S.num_levels():
            li = S.level_info(l)
            lev = _oracle_level(S, case, l, cb)
            if li["next_kind"] in (1, 3):
                cb = ml.restrict_space(case.bc, lev.shape, cb)
            elif li["next_kind"] == 4:
                cb = ml.restrict_cbar_time(ml.restrict_space(case.bc, lev.shape, cb))
            else:
                cb = ml.restrict_cbar_time(cb)
    S.close()


@pytest.mark.parametrize("case", LEVEL_CASES, ids=lambda c: c.name)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("ej", [0, 1], ids=["cbar", "exactJ"])
def test_level_residual_and_transfers(case, prec, ej):
    p, S, U = _setup(case, prec, exact_jacobian=ej)
    dt = S.cycle_dtype
    for l in range(S.num_levels()):
        cb = S.level_cbar(l).double().cpu().numpy()
        cb = cb.reshape(cb.shape[0], -1)
        lev = _oracle_level(S, case, l, cb)
        lev_fwd = _oracle_level(S, case, l, cb, U if ej else None)
        shp = S.level_shape(l)
        e = stgen.random_field(shp, 100 + l)
        r = stgen.random_field(shp, 200 + l)
        et = torch.tensor(e, dtype=dt, device="cuda")
        rt = torch.tensor(r, dtype=dt, device="cuda")
        e_, r_ = et.double().cpu().numpy(), rt.double().cpu().numpy()
        M = lev.M
        for tr in (False, True):
            if tr and case.bc == space.NEUMANN:
                continue
            got = S.level_residual(l, et, rt, transpose=tr).double().cpu().numpy().reshape(lev.Nt, M, -1)
            ref = ml.linear_residual_T(lev, e_, r_) if tr else ml.linear_residual(lev_fwd, e_, r_)
            if l == 0 and not tr and ej:
                # the finest level's operator is minus the exact Jacobian of G
                ref2 = r_.reshape(ref.shape) + system.jacobian_apply(p, U, e_).reshape(ref.shape)
                assert np.abs(ref - ref2).max() <= 1e-12 * (np.abs(ref).max() + 1)
            scale = np.abs(e_).max() * (1 + lev.dt * case.nu * 4 * len(case.shape) / min(S.level_info(l)["h"][:len(case.shape)]) ** 2) + np.abs(r_).max()
            assert np.abs(got - ref).max() <= _tol(prec) * scale, (l, tr)
        if l + 1 < S.num_levels():
            from oracle import collocation as col
            li = S.level_info(l)
            Mc = S.level_info(l + 1)["M"]
            kind = li["next_kind"]
            tf, tc = col.radau_right_nodes(M), col.radau_right_nodes(Mc)
            for tr in (False, True):
                c = S.level_restrict(l, rt, transpose=tr).double().cpu().numpy()
                rr = r_.reshape(lev.Nt, M, -1)
                if kind == 1:
                    ref = ml.restrict_space(case.bc, lev.shape, rr)
                elif kind == 3:
                    X = col.node_prolongation(tf, tc).T if tr else col.node_restriction(tf, tc)
                    ref = np.einsum("cf,nfs->ncs", X, ml.restrict_space(case.bc, lev.shape, rr))
                elif kind == 4 and tr:
                    Pt = col.time_prolongation(tf)
                    rs = ml.restrict_space(case.bc, lev.shape, rr)
                    ref = np.einsum("km,nks->nms", Pt, rs.reshape(lev.Nt // 2, 2 * M, -1))
                elif kind == 4:
                    ref = ml.restrict_space_time(case.bc, lev.shape, M, rr)
                elif tr:
                    Pt = col.time_prolongation(tf)
                    ref = np.einsum("km,nks->nms", Pt, r_.reshape(lev.Nt // 2, 2 * M, -1))
                else:
                    ref = ml.restrict_time(M, rr)
                assert np.abs(c.reshape(ref.shape) - ref).max() <= _tol(prec) * 4 * np.abs(r_).max(), (l, tr)
                cshape = S.level_shape(l + 1)
                cv = stgen.random_field(cshape, 300 + l)
                ct = torch.tensor(cv, dtype=dt, device="cuda")
                cv_ = ct.double().cpu().numpy().reshape(cshape[0], Mc, -1)
                fine = et.clone()
                S.level_prolong(l, ct, fine, transpose=tr)
                if kind == 1:
                    add = ml.prolong_space(case.bc, lev.shape, cv_)
                elif kind == 3:
                    X = col.node_restriction(tf, tc).T if tr else col.node_prolongation(tf, tc)
                    add = ml.prolong_space(case.bc, lev.shape, np.einsum("fc,ncs->nfs", X, cv_))
                elif kind == 4 and tr:
                    Rt = col.time_restriction(tf)
                    add = ml.prolong_space(case.bc, lev.shape, np.einsum("mk,nms->nks", Rt, cv_).reshape(lev.Nt, M, -1))
                elif kind == 4:
                    add = ml.prolong_space_time(case.bc, lev.shape, M, cv_)
                elif tr:
                    Rt = col.time_restriction(tf)
                    add = np.einsum("mk,nms->nks", Rt, cv_).reshape(lev.Nt, M, -1)
                else:
                    add = ml.prolong_time(M, cv_)
                ref = e_.reshape(add.shape) + add
                assert np.abs(fine.double().cpu().numpy().reshape(ref.shape) - ref).max() <= \
                    _tol(prec) * 8 * (np.abs(e_).max() + np.abs(cv_).max()), (l, tr)
    S.close()


@pytest.mark.parametrize("case", LEVEL_CASES, ids=lambda c: c.name)
@pytest.mark.parametrize("transpose", [False, True])
def test_coarse_solve_exact(case, transpose):
    p, S, U = _setup(case, "fp64")
    L = S.num_levels() - 1
    cb = S.level_cbar(L).double().cpu().numpy()
    lev = _oracle_level(S, case, L, cb.reshape(cb.shape[0], -1))
    shp = S.level_shape(L)
    r = stgen.random_field(shp, 400)
    e = S.coarse_solve(torch.tensor(r, device="cuda"), transpose=transpose).cpu().numpy().reshape(lev.Nt, lev.M, -1)
    ref = (ml.coarse_solve_exact_T if transpose else ml.coarse_solve_exact)(lev, r.reshape(lev.Nt, lev.M, -1))
    assert np.abs(e - ref).max() <= 1e-10 * max(1, np.abs(ref).max())
    S.close()


@pytest.mark.parametrize("case", [HEAT1D, LOG2D, CUB3D, PER2D_M5, PER3D_M5], ids=lambda c: c.name)
@pytest.mark.parametrize("ej", [0, 1], ids=["cbar", "exactJ"])
def test_smoothing_step_converged_inner(case, ej):
    """With many inner cycles the Q-diagonalised slab solve is exact, so one
    smoothing step equals damped block Jacobi with exact slab solves (of the
    node-averaged slab matrices; with the exact Jacobian only the residual
    uses R' per node)."""
    p, S, U = _setup(case, "fp64", inner_cycles=40, inner_coarse_iters=60, smooth_inner_levels=0,
                     exact_jacobian=ej)
    l = 0
    cb = S.level_cbar(l).cpu().numpy()
    lev = _oracle_level(S, case, l, cb.reshape(cb.shape[0], -1), U if ej else None)
    shp = S.level_shape(l)
    e = stgen.random_field(shp, 500)
    r = stgen.random_field(shp, 501)
    et = torch.tensor(e, device="cuda")
    S.level_smooth(l, et, torch.tensor(r, device="cuda"))
    ref = ml.smoothing_step_exact(lev, e.reshape(lev.Nt, p.M, -1), r.reshape(lev.Nt, p.M, -1),
                                  S.level_info(l)["omega"])
    err = np.abs(et.cpu().numpy().reshape(ref.shape) - ref).max() / np.abs(ref).max()
    assert err < 1e-9, err
    S.close()


@pytest.mark.parametrize("case", [HEAT1D, LOG2D, DIR2D_M5, PER2D_M5, RAGGED, TILED_M5], ids=lambda c: c.name)
@pytest.mark.parametrize("sweeps", [2, 3, 5])
@pytest.mark.parametrize("tma", [0, 1], ids=["direct", "tma"])
def test_smoothing_step_jacobi_slab_solves(case, sweeps, tma):
    """On a level that coarsens in space next, the default smoother replaces
    each slab solve by a few weighted-Jacobi sweeps on the eigen-decoupled
    shifted systems (no inner multigrid): compared with the oracle's
    complex-arithmetic version of exactly that step."""
    if tma and case not in (RAGGED, TILED_M5):
        pytest.skip("the TMA-staged sweep takes 2D periodic grids in whole 64 x 16 tiles")
    p, S, U = _setup(case, "fp32" if tma else "fp64", smooth_inner_levels=1, smooth_sweeps=sweeps,
                     exact_jacobian=sweeps % 2, use_tma=tma)
    info = S.level_info(0)
    assert info["next_kind"] == 1
    cb = S.level_cbar(0).cpu().numpy()
    lev = _oracle_level(S, case, 0, cb.reshape(cb.shape[0], -1), U if sweeps % 2 else None)
    shp = S.level_shape(0)
    et = torch.tensor(stgen.random_field(shp, 510), dtype=S.cycle_dtype, device="cuda")
    rt = torch.tensor(stgen.random_field(shp, 511), dtype=S.cycle_dtype, device="cuda")
    e, r = et.double().cpu().numpy(), rt.double().cpu().numpy()
    S.level_smooth(0, et, rt)
    omega_j = {1: 2.0 / 3.0, 2: 0.8, 3: 6.0 / 7.0}[len(case.shape)]
    ref = ml.smoothing_step_jacobi(lev, e.reshape(lev.Nt, p.M, -1), r.reshape(lev.Nt, p.M, -1), info["omega"],
                                   sweeps, omega_j)
    err = np.abs(et.double().cpu().numpy().reshape(ref.shape) - ref).max() / np.abs(ref).max()
    # FP32: a few ulps times the conditioning of the eigenbasis (M = 5) and the sweeps
    assert err < (5e-5 if tma else 1e-12), err
    S.close()


@pytest.mark.parametrize("case", [HEAT1D, LOG2D, MIXED, CUB3D, DIR2D_M5, PER2D_M5, PER3D_M5], ids=lambda c: c.name)
@pytest.mark.parametrize("transpose", [False, True])
def test_level_vcycle_contracts(case, transpose):
    """One V-cycle on A e - C e = r (zero start) reduces the residual.  Levels
    with mu_l < 1 smooth with damping 0.5, which bounds the per-cycle
    contraction of slab-local error near 1/2, hence the 0.6 bound."""
    p, S, U = _setup(case, "fp64")
    shp = S.level_shape(0)
    r = torch.tensor(stgen.random_field(shp, 600), device="cuda")
    e = S.level_vcycle(r, transpose=transpose)
    res = S.level_residual(0, e, r, transpose=transpose)
    ratio = float(res.norm() / r.norm())
    assert ratio < 0.6, ratio
    S.close()


@pytest.mark.parametrize("case", [RAGGED, TILED_M5], ids=lambda c: c.name)
@pytest.mark.parametrize("prec", ["fp32"])
def test_tma_staged_sweeps_equal_direct_loads(case, prec):
    """With use_tma, Jacobi sweeps on 2D periodic grids in whole 64 x 16 tiles
    stage their operands through TMA copies; the arithmetic is the same as
    the direct-load kernel's, so a V-cycle gives identical results either way."""
    outs = []
    for tma in (1, 0):
        p, S, U = _setup(case, prec, use_tma=tma)
        r = torch.tensor(stgen.random_field(S.level_shape(0), 700), dtype=S.cycle_dtype, device="cuda")
        outs.append(S.level_vcycle(r).cpu())
        S.close()
    assert torch.equal(outs[0], outs[1])


@pytest.mark.parametrize("case", [RAGGED, TILED_M5], ids=lambda c: c.name)
def test_staged_whole_cycles_same_bits(case):
    """Whole FP32 V-cycles (graph replay, with the FP64-accurate residual and
    the update of U) with and without the TMA-staged kernels give the same
    iterate to the bit."""
    from paper_2006_12883_gb300 import stlib
    outs = []
    for tma in (1, 0):
        p = case.problem()
        S = case.solver(precision=stlib.FP32_REFINE, use_tma=tma)
        U = torch.tensor(stgen.random_field((p.Nt, p.M, p.Ns), 11, 0.3) + 0.4, device="cuda")
        U = U.reshape(S.field_shape)
        S.vcycle(U)
        S.vcycle(U)
        outs.append(U.cpu())
        S.close()
    assert torch.equal(outs[0], outs[1])


@pytest.mark.parametrize("case", [RAGGED, TILED_M5, TILED_SQ3, TILED_SQ5], ids=lambda c: c.name)
@pytest.mark.parametrize("adjoint", [False, True])
def test_two_sweep_kernel_same_bits(case, adjoint):
    """The last two Jacobi sweeps of a slab solve as one kernel (the middle
    iterate in shared memory) against the two separate launches: whole FP32
    V-cycles, forward and transposed, give the same bits (the Jacobi update's
    roundings are spelt out in one shared helper)."""
    from paper_2006_12883_gb300 import stlib
    outs = []
    for fuse in (1, 0):
        p, S, U = _setup(case, "fp32", fuse_sweeps=fuse)
        r = torch.tensor(stgen.random_field(S.level_shape(0), 701), dtype=S.cycle_dtype, device="cuda")
        e1 = S.level_vcycle(r, transpose=adjoint)
        e2 = S.level_vcycle(r - 0.5 * e1, transpose=adjoint)
        outs.append(torch.cat([e1.reshape(-1), e2.reshape(-1)]).cpu())
        S.close()
    assert torch.equal(outs[0], outs[1])


# a 2D periodic case in whole 64 x 16 tiles whose level 0 has inner levels
# (the fine residual's smoothing start applies), beside the two square ones
TILED_START = Case("tiled_start_m5", (128, 64), P_, 1e-2, 6, 5, reaction=space.LOGISTIC, rho=1.0, u0_kind="noise",
                   seed=23)


@pytest.mark.parametrize("case", [TILED_SQ3, TILED_SQ5, TILED_START, TILED_HEAT3], ids=lambda c: c.name)
def test_fine_residual_smoothing_start_same_bits(case):
    """The fine residual doing the first step of the cycle's first level-0
    smoothing (y = F r and the zero-start iterate, from e = 0) against the
    cycle doing it: two whole outer steps (residual, relinearisation, FP32
    V-cycle, update of U) give the same bits, and the started cycle has one
    launch fewer."""
    from paper_2006_12883_gb300 import stlib
    p = case.problem()
    U0 = stgen.random_field((p.Nt, p.M, p.Ns), 11, 0.3) + 0.4
    outs, norms, launches = [], [], []
    for fuse in (1, 0):
        S = case.solver(precision=stlib.FP32_REFINE, fuse_start=fuse)
        U = torch.tensor(U0, device="cuda").reshape(S.field_shape)
        n1 = S.vcycle(U)
        n2 = S.vcycle(U)
        torch.cuda.synchronize()
        outs.append(U.reshape(-1).cpu())
        norms.append((n1, n2))
        launches.append(S.stats()["launches_per_vcycle"])
        S.close()
    assert torch.equal(outs[0], outs[1])
    assert norms[0] == norms[1]
    # one launch fewer at level 0, and one per level below whose smoothing
    # start the residual-restriction kernel wrote
    assert launches[0] <= launches[1] - 1, launches


@pytest.mark.parametrize("case", [TILED_SQ3, TILED_SQ5, TILED_START, TILED_HEAT3], ids=lambda c: c.name)
def test_residual_restriction_kernel_same_bits(case):
    """The level residual of the coarse-grid correction fused with its full
    weighting onto the next grid (the fine residual kept in shared memory)
    against the two launches: two outer steps and a level V-cycle give the
    same bits, and the fused cycle has fewer launches."""
    from paper_2006_12883_gb300 import stlib
    p = case.problem()
    U0 = stgen.random_field((p.Nt, p.M, p.Ns), 12, 0.3) + 0.4
    outs, launches = [], []
    for fuse in (1, 0):
        S = case.solver(precision=stlib.FP32_REFINE, fuse_restrict=fuse)
        U = torch.tensor(U0, device="cuda").reshape(S.field_shape)
        S.vcycle(U)
        S.vcycle(U)
        r = torch.tensor(stgen.random_field(S.level_shape(0), 702), dtype=S.cycle_dtype, device="cuda")
        e = S.level_vcycle(r)
        torch.cuda.synchronize()
        outs.append((U.reshape(-1).cpu(), e.reshape(-1).cpu()))
        launches.append(S.stats()["launches_per_vcycle"])
        S.close()
    assert torch.equal(outs[0][0], outs[1][0])
    assert torch.equal(outs[0][1], outs[1][1])
    assert launches[0] < launches[1], launches


@pytest.mark.parametrize("case", [TILED_SQ3, TILED_SQ5, TILED_START, TILED_HEAT3], ids=lambda c: c.name)
def test_update_in_cycle_same_bits(case):
    """The defect-correction update U += e done by the cycle's last level-0
    two-sweep kernel (its epilogue adds e' to U) against the update's own
    launch: three st_vcycle steps give the same bits and norms."""
    from paper_2006_12883_gb300 import stlib
    p = case.problem()
    U0 = stgen.random_field((p.Nt, p.M, p.Ns), 13, 0.3) + 0.4
    outs, norms, where = [], [], []
    for fuse in (1, 0):
        S = case.solver(precision=stlib.FP32_REFINE, fuse_update=fuse)
        U = torch.tensor(U0, device="cuda").reshape(S.field_shape)
        norms.append([S.vcycle(U) for _ in range(3)])
        torch.cuda.synchronize()
        outs.append(U.reshape(-1).cpu())
        where.append(S.stats()["update_in_cycle"])
        S.close()
    assert torch.equal(outs[0], outs[1])
    assert norms[0] == norms[1]
    assert where == [1, 0], where
