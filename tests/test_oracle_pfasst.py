"""Pins of the PFASST oracle (paper Section 4.1; multilevel SDC with FAS and
a serial coarsest level)."""
import numpy as np
import pytest

import stgen
from oracle import pfasst as opf
from oracle import sdc, space, system

P, N = space.PERIODIC, space.NEUMANN


def _heat(n=33, Nt=6, M=3):
    return system.Problem(shape=(n,), bc=N, nu=1.0, Nt=Nt, M=M, T=0.3), stgen.cosine_modes(n)


def test_single_level_is_sdc():
    """One level and one sweep per iteration: the SDC sweep of all slabs."""
    p, u0 = _heat()
    U0 = np.broadcast_to(u0, (p.Nt, p.M, p.Ns)).copy()
    it = opf.pfasst(p, u0, [(p.shape, p.M)], 2)
    ref = sdc.sdc_sweep(p, sdc.sdc_sweep(p, U0, u0), u0)
    assert np.abs(it[-1] - ref).max() < 1e-13


def test_two_identical_implicit_euler_levels_solve_in_one_iteration():
    """Two copies of the M = 1 level: tau = 0, and the coarse sweep, slab after
    slab, is the sequential implicit Euler solve (for M = 1 and a linear
    problem one sweep is exact)."""
    p, u0 = _heat(M=1)
    it = opf.pfasst(p, u0, [(p.shape, 1), (p.shape, 1)], 1)
    ref = system.solve_sequential(p, u0)
    assert np.abs(it[0] - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("hier", [
    [((33,), 3), ((17,), 1)],
    [((33,), 3), ((17,), 2), ((9,), 1)],
    [((33,), 3), ((33,), 1)],
])
def test_collocation_solution_is_a_fixed_point(hier):
    p, u0 = _heat()
    ref = system.solve_sequential(p, u0)
    out = opf.pfasst(p, u0, hier, 1, U=ref)
    assert np.abs(out[0] - ref).max() < 1e-11 * np.abs(ref).max()


def test_converges_to_collocation_solution():
    """Three levels (M = 3, 1, 1; space bisected twice), one sweep each: the
    fine iterate converges to the collocation solution."""
    p, u0 = _heat()
    ref = system.solve_sequential(p, u0)
    its = opf.pfasst(p, u0, [((33,), 3), ((17,), 1), ((9,), 1)], 40)
    errs = [np.abs(U - ref).max() / np.abs(ref).max() for U in its]
    assert errs[-1] < 1e-12, errs
    assert all(b < a for a, b in zip(errs[:20], errs[1:20]))


def test_nonlinear_fixed_point_and_convergence():
    """Logistic reaction (explicit in the sweeps): the collocation solution is
    a fixed point and the iteration converges to it."""
    p = system.Problem(shape=(16, 16), bc=P, nu=1e-2, Nt=4, M=3, T=0.2, reaction=space.LOGISTIC, rho=1.0)
    u0 = stgen.smoothed_noise((16, 16), 12884).ravel()
    ref = system.solve_sequential(p, u0)
    hier = [((16, 16), 3), ((8, 8), 1)]
    assert np.abs(opf.pfasst(p, u0, hier, 1, U=ref)[0] - ref).max() < 1e-12
    its = opf.pfasst(p, u0, hier, 20)
    assert np.abs(its[-1] - ref).max() < 1e-10
