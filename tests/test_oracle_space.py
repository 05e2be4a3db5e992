"""Pins of oracle.space: Laplacian eigenpairs, lumped FEM == FD, reaction
terms and spatial transfers.  CPU only."""
import numpy as np
import pytest

import stgen
from oracle import space

D, P, N = space.DIRICHLET, space.PERIODIC, space.NEUMANN


@pytest.mark.parametrize("n", [7, 31, 63])
def test_dirichlet_sine_eigenpairs(n):
    """sin(k pi x) is an eigenvector of the 3-point Laplacian with eigenvalue
    (2cos(k pi h) - 2)/h^2 (the rho_k of the paper's Eq. 5.3)."""
    L = space.laplacian_1d(D, n)
    x = stgen.coords1d(D, n)
    h = 1.0 / (n + 1)
    for k in (1, 2, n // 2, n):
        v = np.sin(k * np.pi * x)
        lam = (2 * np.cos(k * np.pi * h) - 2) / h ** 2
        assert np.abs(L @ v - lam * v).max() < 1e-9 * abs(lam)


@pytest.mark.parametrize("n", [8, 32])
def test_periodic_fourier_eigenpairs(n):
    L = space.laplacian_1d(P, n)
    x = stgen.coords1d(P, n)
    h = 1.0 / n
    for k in range(n // 2 + 1):
        lam = (2 * np.cos(2 * np.pi * k * h) - 2) / h ** 2
        for v in (np.cos(2 * np.pi * k * x), np.sin(2 * np.pi * k * x)):
            assert np.abs(L @ v - lam * v).max() < 1e-9 * max(1, abs(lam))


@pytest.mark.parametrize("nv", [9, 33, 1025])
def test_neumann_lumped_fem_is_mirror_fd(nv):
    """-M_lumped^{-1} K_h (Eq. 3.2 with the lumped mass of Section 3) equals the
    3-point FD Laplacian with a mirrored ghost point, and cos(k pi x/X) are its
    eigenvectors with the paper's rho_k = (2cos(k pi h)-2)/h^2 (Eq. 5.3)."""
    X = 1.0
    L = space.laplacian_1d(N, nv, X).toarray()
    h = X / (nv - 1)
    ref = np.zeros((nv, nv))
    for i in range(nv):
        for di in (-1, 1):
            j = i + di
            if j < 0:
                j = 1
            if j >= nv:
                j = nv - 2
            ref[i, j] += 1.0 / h ** 2
        ref[i, i] -= 2.0 / h ** 2
    assert np.abs(L - ref).max() < 1e-9 / h ** 2
    x = stgen.coords1d(N, nv, X)
    for k in (1, 3, 4):
        v = np.cos(k * np.pi * x / X)
        lam = (2 * np.cos(k * np.pi * h) - 2) / h ** 2
        assert np.abs(L @ v - lam * v).max() < 1e-8 * abs(lam)


def test_kronecker_sum_2d_3d():
    # product modes: eigenvalue is the sum of the 1D eigenvalues
    for shape in [(8, 16), (4, 8, 8)]:
        L = space.laplacian(P, shape)
        xs = stgen.mesh(P, shape)
        ks = [1, 2, 3][:len(shape)]
        v = np.ones(shape)
        lam = 0.0
        for k, xk, n in zip(ks, xs, shape[::-1]):
            v = v * np.cos(2 * np.pi * k * xk)
            lam += (2 * np.cos(2 * np.pi * k / n) - 2) * n * n
        assert np.abs(L @ v.ravel() - lam * v.ravel()).max() < 1e-9 * abs(lam)
    # Dirichlet 2D with different mode per axis (x fastest)
    shape = (7, 15)
    L = space.laplacian(D, shape)
    x, y = stgen.mesh(D, shape)
    v = np.sin(2 * np.pi * x) * np.sin(np.pi * y)
    lam = (2 * np.cos(2 * np.pi / 16) - 2) * 256 + (2 * np.cos(np.pi / 8) - 2) * 64
    assert np.abs(L @ v.ravel() - lam * v.ravel()).max() < 1e-9 * abs(lam)


def test_reaction_terms_and_fixed_points():
    u = np.linspace(-2, 2, 41)
    for kind, zeros in [(space.LOGISTIC, [0.0, 1.0]), (space.CUBIC, [-1.0, 0.0, 1.0])]:
        for z in zeros:
            assert space.reaction(kind, 1.7, np.array([z]))[0] == 0.0
        eps = 1e-6
        fd = (space.reaction(kind, 1.7, u + eps) - space.reaction(kind, 1.7, u - eps)) / (2 * eps)
        assert np.abs(fd - space.reaction_deriv(kind, 1.7, u)).max() < 1e-8
        assert np.allclose(space.reaction(kind, 1.7, u), 1.7 * space.reaction_shape(kind, u))
    # CUBIC is the paper's -gamma (u^3 - u) (Eq. 3.1, 3.7)
    assert np.allclose(space.reaction(space.CUBIC, 5.0, u), -5.0 * (u ** 3 - u))


@pytest.mark.parametrize("bc,n", [(D, 15), (P, 16), (N, 17)])
def test_transfers_1d(bc, n):
    Pm = space.prolongation_1d(bc, n).toarray()
    R = space.restriction_1d(bc, n).toarray()
    nc = space.coarse_size(bc, n)
    assert Pm.shape == (n, nc) and R.shape == (nc, n)
    xf = stgen.coords1d(bc, n)
    xc = stgen.coords1d(bc, nc)
    if bc == D:
        # linear interpolation reproduces linear functions vanishing at both ends
        f = lambda x: x * (1 - x) * 0 + np.minimum(x, 1 - x)  # piecewise linear, kink at 1/2
        assert np.abs(Pm @ f(xc) - f(xf)).max() < 1e-14
        assert np.abs(Pm - 2 * R.T).max() == 0
    if bc == P:
        assert np.abs(R @ np.ones(n) - 1).max() < 1e-15
        assert np.abs(Pm @ np.ones(nc) - 1).max() < 1e-15
        assert np.abs(Pm - 2 * R.T).max() == 0
    if bc == N:
        assert np.abs(R @ np.ones(n) - 1).max() < 1e-15
        assert np.abs(Pm @ xc - xf).max() < 1e-14  # linear functions exact
    # full weighting is [1 2 1]/4 around an interior coarse point
    I = nc // 2
    i = 2 * I + 1 if bc == D else 2 * I
    row = np.zeros(n)
    row[i - 1:i + 2] = [0.25, 0.5, 0.25]
    assert np.abs(R[I] - row).max() == 0


def test_transfers_tensor():
    shape = (8, 16)
    R = space.restriction(P, shape)
    Pm = space.prolongation(P, shape)
    assert R.shape == (4 * 8, 8 * 16)
    assert abs(Pm - 4 * R.T).max() == 0
    assert space.coarse_shape(D, (15, 31, 7)) == (7, 15, 3)
