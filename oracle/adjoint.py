"""Adjoint of the all-at-once system and parameter gradients.  Oracle: test
infrastructure only.

The paper has no adjoint; this is the discrete adjoint of the system it
defines (Eq. 2.3 with 2.11 / 3.4).  For an objective Phi(u_{Nt,M}) the
gradient with respect to a parameter theta of G(U; theta) = 0 is
lambda^T dG/dtheta, where J^T lambda = -dPhi/dU and J = dG/dU.  J is block
lower bidiagonal, so J^T is block upper bidiagonal and is solved backward:

    J_nn^T lambda_n = -g_n - e_M (x) sum_m lambda_{n+1,m},   n = Nt..1,

g_n being dPhi/dU_n (nonzero on the last node of the last slab only).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import space
from . import system
from .system import Problem, slab_jacobian, solve_sequential


def _transposed_slab_solve(p: Problem, Un: np.ndarray, rhs: np.ndarray) -> np.ndarray:
    """x with J_nn^T x = rhs, J_nn = dG_n/dU_n at U_n.  Sparse LU up to the
    oracle's direct-solve size; beyond it (periodic grids) matrix-free GMRES
    on J_nn^T v = dt (L^T + D)(Q^T v) - v with the exact inverse of the
    constant-coefficient transposed slab matrix as preconditioner, to a
    1e-13 relative residual."""
    M, Ns = p.M, p.Ns
    if M * Ns <= system._DIRECT_MAX or p.bc != space.PERIODIC:
        return spla.spsolve(slab_jacobian(p, Un).T.tocsc(), rhs.ravel()).reshape(M, Ns)
    dR = p.dR(Un.reshape(M, Ns))
    LT = p.L.T.tocsr()

    def apply(v):
        W = p.Q.T @ np.asarray(v).reshape(M, Ns)
        return (p.dt * ((LT @ W.T).T + dR * W) - np.asarray(v).reshape(M, Ns)).reshape(-1)

    A = spla.LinearOperator((M * Ns, M * Ns), matvec=apply, dtype=np.float64)
    pre = system.periodic_slab_inverse(p, float(np.mean(dR)), transpose=True)
    x, info = spla.gmres(A, rhs.ravel(), rtol=1e-13, atol=0.0, restart=50, maxiter=200, M=pre)
    if info != 0:
        raise RuntimeError(f"transposed slab solve did not converge ({info})")
    return x.reshape(M, Ns)


def cell_volume(p: Problem) -> float:
    return float(np.prod([space.spacing(p.bc, n, p.X) for n in p.shape]))


def objective(p: Problem, U: np.ndarray, target: np.ndarray) -> float:
    """Phi = 1/2 h^d sum_x (u_{Nt,M} - target)^2."""
    d = U.reshape(p.Nt, p.M, p.Ns)[-1, -1] - target.reshape(-1)
    return 0.5 * cell_volume(p) * float(d @ d)


def objective_gradient(p: Problem, U: np.ndarray, target: np.ndarray) -> np.ndarray:
    """dPhi/du_{Nt,M} = h^d (u_{Nt,M} - target)."""
    return cell_volume(p) * (U.reshape(p.Nt, p.M, p.Ns)[-1, -1] - target.reshape(-1))


def adjoint_solve(p: Problem, U: np.ndarray, gT: np.ndarray) -> np.ndarray:
    """lambda solving J^T lambda = -g with g = gT on node M of slab Nt."""
    U = U.reshape(p.Nt, p.M, p.Ns)
    lam = np.zeros_like(U)
    carry = np.zeros(p.Ns)          # sum_m lambda_{n+1,m}
    for n in range(p.Nt - 1, -1, -1):
        rhs = np.zeros((p.M, p.Ns))
        if n == p.Nt - 1:
            rhs[-1] -= gT.reshape(-1)
        rhs[-1] -= carry
        lam[n] = _transposed_slab_solve(p, U[n], rhs)
        carry = lam[n].sum(axis=0)
    return lam


def gradients(p: Problem, U: np.ndarray, lam: np.ndarray):
    """(dPhi/dnu, dPhi/drho, dPhi/du0) = lambda^T dG/dtheta with
    dG_n/dnu = dt (Q (x) I) Delta_h U_n, dG_n/drho = dt (Q (x) I) r(U_n) and
    dG_1/du0 = 1 (x) I."""
    U = U.reshape(p.Nt, p.M, p.Ns)
    lam = lam.reshape(U.shape)
    lap = space.laplacian(p.bc, p.shape, p.X)
    QtL = np.einsum("mj,nms->njs", p.Q, lam)   # (Q^T lambda_n)_j
    DU = (lap @ U.reshape(-1, p.Ns).T).T.reshape(U.shape)
    dnu = p.dt * float(np.sum(QtL * DU))
    drho = p.dt * float(np.sum(QtL * space.reaction_shape(p.reaction, U)))
    du0 = lam[0].sum(axis=0)
    return dnu, drho, du0


def solve_and_gradients(p: Problem, u0: np.ndarray, target: np.ndarray):
    U = solve_sequential(p, u0)
    lam = adjoint_solve(p, U, objective_gradient(p, U, target))
    return U, lam, gradients(p, U, lam)


def fd_gradient_param(p: Problem, u0, target, name: str, rel: float = 1e-6) -> float:
    """Central finite difference of Phi with respect to nu or rho."""
    th = getattr(p, name)
    dth = rel * abs(th) if th != 0 else rel
    vals = []
    for s in (+1, -1):
        q = p.with_params(**{name: th + s * dth})
        vals.append(objective(q, solve_sequential(q, u0), target))
    return (vals[0] - vals[1]) / (2 * dth)


def fd_gradient_u0(p: Problem, u0, target, direction, eps: float = 1e-6) -> float:
    """Central finite difference of Phi along ``direction`` in u0."""
    vals = []
    for s in (+1, -1):
        v = u0 + s * eps * direction
        vals.append(objective(p, solve_sequential(p, v), target))
    return (vals[0] - vals[1]) / (2 * eps)
