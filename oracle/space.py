"""Spatial discretisation (paper Section 3).  Oracle: test infrastructure only.

Fields are numpy arrays with x fastest: shape (nx,), (ny, nx) or (nz, ny, nx),
flattened in C order.  Grid conventions match ``stgen`` (DIRICHLET interior
points, PERIODIC unique points, NEUMANN vertices).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

DIRICHLET, PERIODIC, NEUMANN = 0, 1, 2
NONE, LOGISTIC, CUBIC = 0, 1, 2


def spacing(bc: int, n: int, X: float = 1.0) -> float:
    if bc == DIRICHLET:
        return X / (n + 1)
    if bc == PERIODIC:
        return X / n
    if bc == NEUMANN:
        return X / (n - 1)
    raise ValueError(bc)


def fem_matrices_1d(n_vertices: int, X: float):
    """Linear-FEM stiffness K_h and lumped mass M_h on n_vertices uniform
    vertices of [0, X] (Eq. 3.2, with the lumped mass of Section 3)."""
    N = n_vertices - 1
    h = X / N
    K = sp.lil_matrix((n_vertices, n_vertices))
    Mc = sp.lil_matrix((n_vertices, n_vertices))
    for e in range(N):
        idx = [e, e + 1]
        Ke = np.array([[1.0, -1.0], [-1.0, 1.0]]) / h
        Me = np.array([[2.0, 1.0], [1.0, 2.0]]) * h / 6.0
        for a in range(2):
            for b in range(2):
                K[idx[a], idx[b]] += Ke[a, b]
                Mc[idx[a], idx[b]] += Me[a, b]
    Ml = sp.diags(np.asarray(Mc.sum(axis=1)).ravel())
    return K.tocsr(), Ml.tocsr()


def laplacian_1d(bc: int, n: int, X: float = 1.0) -> sp.csr_matrix:
    """Second-order 1D Laplacian Delta_h (x fastest, n unknowns).

    DIRICHLET: 3-point FD on interior points with zero boundary values.
    PERIODIC : 3-point FD, circulant.
    NEUMANN  : -M_h^{-1} K_h of the lumped linear FEM (paper Section 3)."""
    h = spacing(bc, n, X)
    if bc == NEUMANN:
        K, Ml = fem_matrices_1d(n, X)
        return (-sp.diags(1.0 / Ml.diagonal()) @ K).tocsr()
    main = -2.0 * np.ones(n)
    off = np.ones(n - 1)
    L = sp.diags([off, main, off], [-1, 0, 1], shape=(n, n)).tolil()
    if bc == PERIODIC:
        if n == 1:
            L[0, 0] = 0.0
        elif n == 2:
            L[0, 1] = 2.0
            L[1, 0] = 2.0
        else:
            L[0, n - 1] = 1.0
            L[n - 1, 0] = 1.0
    return (L.tocsr() / (h * h)).tocsr()


def laplacian(bc: int, shape, X: float = 1.0) -> sp.csr_matrix:
    """d-dimensional Laplacian as the Kronecker sum of 1D ones (shape in numpy
    order, slowest axis first)."""
    shape = tuple(shape)
    N = int(np.prod(shape))
    L = sp.csr_matrix((N, N))
    for a, na in enumerate(shape):
        before = int(np.prod(shape[:a]))
        after = int(np.prod(shape[a + 1:]))
        La = laplacian_1d(bc, na, X)
        L = L + sp.kron(sp.identity(before), sp.kron(La, sp.identity(after)))
    return L.tocsr()


def reaction(kind: int, rho: float, u):
    """R(u): NONE 0; LOGISTIC rho*u*(1-u); CUBIC rho*u*(1-u^2).

    CUBIC is the paper's monodomain term moved to the right-hand side:
    -gamma*(u^3 - u) of Eq. (3.1)/(3.7) with gamma = rho."""
    if kind == NONE:
        return np.zeros_like(u)
    if kind == LOGISTIC:
        return rho * u * (1.0 - u)
    if kind == CUBIC:
        return rho * u * (1.0 - u * u)
    raise ValueError(kind)


def reaction_shape(kind: int, u):
    """r(u) = R(u)/rho, the derivative of R with respect to rho."""
    return reaction(kind, 1.0, u)


def reaction_deriv(kind: int, rho: float, u):
    """R'(u) = dR/du."""
    if kind == NONE:
        return np.zeros_like(u)
    if kind == LOGISTIC:
        return rho * (1.0 - 2.0 * u)
    if kind == CUBIC:
        return rho * (1.0 - 3.0 * u * u)
    raise ValueError(kind)


# --------------------------------------------------------- spatial coarsening

def coarse_size(bc: int, n: int) -> int:
    """Bisection of a 1D grid (Section 5.2, SMG): DIRICHLET 2^k-1 -> 2^(k-1)-1,
    PERIODIC 2^k -> 2^(k-1), NEUMANN 2^k+1 vertices -> 2^(k-1)+1."""
    if bc == DIRICHLET:
        if n % 2 == 0 or n < 3:
            raise ValueError("Dirichlet bisection needs odd n >= 3")
        return (n - 1) // 2
    if bc == PERIODIC:
        if n % 2 or n < 2:
            raise ValueError("periodic bisection needs even n >= 2")
        return n // 2
    if bc == NEUMANN:
        if (n - 1) % 2 or n < 3:
            raise ValueError("Neumann bisection needs n = 2^k + 1 >= 3")
        return (n - 1) // 2 + 1
    raise ValueError(bc)


def _fine_index(bc: int, I: int) -> int:
    """Fine index of coarse point I (coarse points sit on even fine points)."""
    return 2 * I + 1 if bc == DIRICHLET else 2 * I


def prolongation_1d(bc: int, nf: int) -> sp.csr_matrix:
    """Linear interpolation, coarse -> fine (nf x nc).  Coarse point I coincides
    with its fine point; fine points between two coarse points take their mean
    (zero boundary values for DIRICHLET, wrap-around for PERIODIC)."""
    nc = coarse_size(bc, nf)
    P = sp.lil_matrix((nf, nc))
    for I in range(nc):
        i = _fine_index(bc, I)
        P[i, I] += 1.0
        for di in (-1, 1):
            j = i + di
            if bc == PERIODIC:
                j %= nf
            if 0 <= j < nf:
                P[j, I] += 0.5
    return P.tocsr()


def restriction_1d(bc: int, nf: int) -> sp.csr_matrix:
    """Full weighting [1 2 1]/4, fine -> coarse (Section 5.2, SMG stencil).

    Interior and periodic rows are P^T/2; at a NEUMANN end the stencil reads a
    mirrored ghost value f[-1] = f[1]."""
    nc = coarse_size(bc, nf)
    R = sp.lil_matrix((nc, nf))
    for I in range(nc):
        i = _fine_index(bc, I)
        R[I, i] += 0.5
        for di in (-1, 1):
            j = i + di
            if bc == PERIODIC:
                j %= nf
            if bc == NEUMANN:
                if j < 0:
                    j = 1
                if j >= nf:
                    j = nf - 2
            if 0 <= j < nf:
                R[I, j] += 0.25
    return R.tocsr()


def _kron_all(mats):
    out = mats[0]
    for m in mats[1:]:
        out = sp.kron(out, m)
    return out.tocsr()


def prolongation(bc: int, shape) -> sp.csr_matrix:
    """Tensor-product linear interpolation (numpy-order shape of the fine grid)."""
    return _kron_all([prolongation_1d(bc, n) for n in shape])


def restriction(bc: int, shape) -> sp.csr_matrix:
    """Tensor-product full weighting."""
    return _kron_all([restriction_1d(bc, n) for n in shape])


def coarse_shape(bc: int, shape):
    return tuple(coarse_size(bc, n) for n in shape)
