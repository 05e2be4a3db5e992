"""Fine FP64 residual G(U) (Eq. 2.3 with the slab coupling of Eq. 3.4), its
norm and the node-averaged reaction derivative: CUDA path through the C ABI
against the oracle, element by element."""
import numpy as np
import pytest

import stgen
from oracle import space, system
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
    from tests.gpu_cases import PER3D_M5
    case = PER3D_M5
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


def _tile_scales(p, U, tw=64, th=16):
    """Per point: the largest |U| over its 64 x 16 tile and the tile's
    one-point halo, over every node of every slab (an upper bound of the
    magnitude the tiled residual's split is relative to)."""
    ny, nx = p.shape
    A = np.abs(U.reshape(-1, ny, nx)).max(axis=0)
    out = np.empty((ny, nx))
    for j0 in range(0, ny, th):
        for i0 in range(0, nx, tw):
            rows = [(j0 - 1) % ny] + list(range(j0, j0 + th)) + [(j0 + th) % ny]
            cols = [(i0 - 1) % nx] + list(range(i0, i0 + tw)) + [(i0 + tw) % nx]
            out[j0:j0 + th, i0:i0 + tw] = A[np.ix_(rows, cols)].max()
    return out.ravel()


@pytest.mark.parametrize("which", ["ragged", "square"])
def test_tiled_residual_dynamic_range_and_nonfinite(which):
    """The residual for the FP32 cycle on 2D periodic grids in whole 64 x 16
    tiles holds every value as a high part on a grid set by its tile's
    largest exponent plus a float low part.  With tiles whose magnitudes
    differ by up to 1e9, each tile keeps an absolute error of about 1e-13 of
    its own terms; a non-finite value gives a non-finite norm and leaves the
    tiles away from it exact as before."""
    from paper_2006_12883_gb300 import stlib
    from tests.gpu_cases import RAGGED, Case
    if which == "square":
        RAGGED = Case("square_dyn", (128, 128), space.PERIODIC, 1e-2, 6, 3, reaction=space.LOGISTIC, rho=1.0,
                      u0_kind="noise", seed=4)
    p = RAGGED.problem()
    ny, nx = p.shape
    U = stgen.random_field((p.Nt, p.M, p.Ns), 11, 0.4) + 0.5
    mag = np.ones((ny, nx))
    for j0 in range(0, ny, 16):
        for i0 in range(0, nx, 64):
            mag[j0:j0 + 16, i0:i0 + 64] = 10.0 ** ((3 * (j0 // 16) + 5 * (i0 // 64)) % 10 - 6)
    U = U * mag.ravel()
    u0 = RAGGED.u0()
    G = system.residual(p, U, u0)
    S = RAGGED.solver(precision=stlib.FP32_REFINE)
    Ut = torch.tensor(U, device="cuda").reshape(S.field_shape)
    R32 = torch.empty(S.field_shape, dtype=torch.float32, device="cuda")
    nrm = S.residual(Ut, R32, fp64=False)
    got = R32.double().cpu().numpy().reshape(G.shape)
    ut = np.maximum(_tile_scales(p, U), np.abs(u0).max())
    ih2 = max(1.0 / space.spacing(p.bc, n, p.X) ** 2 for n in p.shape)
    qsum = float(np.abs(p.Q).sum(axis=1).max())
    tile_scale = ut + p.dt * qsum * (p.nu * 8 * ih2 * ut + np.abs(p.rho) * (ut + ut ** 2))
    err = np.abs(got - G)
    assert (err <= 2e-7 * np.abs(G) + 1e-13 * tile_scale[None, None, :]).all(), \
        (err / (2e-7 * np.abs(G) + 1e-13 * tile_scale)).max()
    assert abs(nrm - np.linalg.norm(G)) <= 1e-6 * np.linalg.norm(G)
    # one infinite value in slab 3, node 1, the first tile of the grid
    U2 = U.copy()
    U2[3, 1, 5 * nx + 7] = np.inf
    Ut2 = torch.tensor(U2, device="cuda").reshape(S.field_shape)
    nrm2 = S.residual(Ut2, R32, fp64=False)
    assert not np.isfinite(nrm2)
    got2 = R32.double().cpu().numpy().reshape(G.shape)
    far = np.ones(G.shape, bool)
    far[3] = False  # the slab with the infinite value; slab 4 only couples to node M
    far[4] = False
    assert np.array_equal(got2[far], got[far])
    S.close()
