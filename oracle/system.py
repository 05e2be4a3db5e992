"""The all-at-once space-time system (paper Sections 2-3).  Oracle: test
infrastructure only.

Unknowns U have shape (Nt, M, Ns): slab n, Radau node m, spatial point s
(x fastest) - the node-major slab vector of Eq. (3.6).  The system is the
collocation form (2.3) on every slab, chained through the slab coupling of
Eq. (2.11)/(3.4):

    G_n(U) = 1 (x) u_{n-1,M} + dt (Q (x) I) F(U_n) - U_n,
    F(u)   = nu * Delta_h u + R(u),        u_{0,M} := u0.

The paper's DG form (3.4) is this system premultiplied by the DG mass
matrices (see ``dg_solve`` and the DG == collocation pins in the tests).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import collocation as col
from . import space


@dataclass
class Problem:
    """Reaction-diffusion problem u_t = nu*Delta u + R(u) (Eq. 3.1 generalised)."""
    shape: tuple            # numpy order, slowest first
    bc: int
    nu: float
    Nt: int
    M: int
    T: float = 1.0
    X: float = 1.0
    reaction: int = space.NONE
    rho: float = 0.0
    _cache: dict = field(default_factory=dict, repr=False, compare=False)

    @property
    def Ns(self) -> int:
        return int(np.prod(self.shape))

    @property
    def dt(self) -> float:
        return self.T / self.Nt

    @property
    def tau(self):
        if "tau" not in self._cache:
            self._cache["tau"] = col.radau_right_nodes(self.M)
        return self._cache["tau"]

    @property
    def Q(self):
        if "Q" not in self._cache:
            self._cache["Q"] = col.collocation_matrix(self.tau)
        return self._cache["Q"]

    @property
    def L(self) -> sp.csr_matrix:
        """nu * Delta_h."""
        if "L" not in self._cache:
            self._cache["L"] = (self.nu * space.laplacian(self.bc, self.shape, self.X)).tocsr()
        return self._cache["L"]

    def R(self, u):
        return space.reaction(self.reaction, self.rho, u)

    def dR(self, u):
        return space.reaction_deriv(self.reaction, self.rho, u)

    def with_params(self, **kw) -> "Problem":
        d = dict(shape=self.shape, bc=self.bc, nu=self.nu, Nt=self.Nt, M=self.M, T=self.T,
                 X=self.X, reaction=self.reaction, rho=self.rho)
        d.update(kw)
        return Problem(**d)


def F(p: Problem, u: np.ndarray) -> np.ndarray:
    """F(u) = nu*Delta_h u + R(u) applied to the last axis (points)."""
    Lu = (p.L @ u.reshape(-1, p.Ns).T).T.reshape(u.shape)
    return Lu + p.R(u)


def previous_node(p: Problem, U: np.ndarray, u0: np.ndarray) -> np.ndarray:
    """u_{n-1,M} for every slab n (u0 for the first): the coupling of Eq. (2.11)."""
    prev = np.empty((p.Nt, p.Ns))
    prev[0] = u0.reshape(-1)
    prev[1:] = U[:-1, -1, :]
    return prev


def residual(p: Problem, U: np.ndarray, u0: np.ndarray) -> np.ndarray:
    """G(U) of the collocation form (2.3) on all slabs (shape (Nt, M, Ns))."""
    U = U.reshape(p.Nt, p.M, p.Ns)
    FU = F(p, U)
    QF = np.einsum("mj,njs->nms", p.Q, FU)
    return previous_node(p, U, u0)[:, None, :] + p.dt * QF - U


def residual_points(p: Problem, U: np.ndarray, u0: np.ndarray, slabs, points) -> np.ndarray:
    """G_{n,m}(s) for the listed (slab n, point s) pairs and every node m,
    evaluated one point at a time from the stencil definition (any problem
    size; no global operator is formed).  Returns shape (len(slabs), M)."""
    U = U.reshape(p.Nt, p.M, p.Ns)
    shape = p.shape
    d = len(shape)
    hs = [space.spacing(p.bc, n, p.X) for n in shape]
    strides = [int(np.prod(shape[a + 1:])) for a in range(d)]
    out = np.zeros((len(slabs), p.M))
    for t, (n, s) in enumerate(zip(slabs, points)):
        idx = np.unravel_index(int(s), shape)
        Fv = np.zeros(p.M)
        for j in range(p.M):
            plane = U[n, j]
            c = plane[s]
            lap = 0.0
            for a in range(d):
                vals = []
                for di in (-1, 1):
                    q = idx[a] + di
                    if 0 <= q < shape[a]:
                        vals.append(plane[s + di * strides[a]])
                    elif p.bc == space.PERIODIC:
                        q %= shape[a]
                        vals.append(plane[s + (q - idx[a]) * strides[a]])
                    elif p.bc == space.NEUMANN:
                        q = 1 if q < 0 else shape[a] - 2
                        vals.append(plane[s + (q - idx[a]) * strides[a]])
                    else:
                        vals.append(0.0)
                lap += (vals[0] + vals[1] - 2 * c) / hs[a] ** 2
            Fv[j] = p.nu * lap + float(p.R(np.array([c]))[0])
        prev = u0.reshape(-1)[s] if n == 0 else U[n - 1, -1, s]
        out[t] = prev + p.dt * (p.Q @ Fv) - U[n, :, s]
    return out


def residual_norm(p: Problem, U, u0) -> float:
    return float(np.linalg.norm(residual(p, U, u0).ravel()))


def reference_norm(p: Problem, u0) -> float:
    """||G(0)||_2: the zero initial guess's residual (Section 5.2 stopping rule);
    G(0) is u0 on every node of the first slab when R(0) = 0."""
    return float(np.linalg.norm(residual(p, np.zeros((p.Nt, p.M, p.Ns)), u0).ravel()))


def cbar(p: Problem, U: np.ndarray) -> np.ndarray:
    """Node-averaged reaction derivative cbar_n(x) = mean_m R'(U_{n,m}(x))."""
    U = U.reshape(p.Nt, p.M, p.Ns)
    return p.dR(U).mean(axis=1)


def jacobian_apply(p: Problem, U: np.ndarray, V: np.ndarray) -> np.ndarray:
    """Directional derivative dG(U)[V] (exact Jacobian of G)."""
    U = U.reshape(p.Nt, p.M, p.Ns)
    V = V.reshape(p.Nt, p.M, p.Ns)
    LV = (p.L @ V.reshape(-1, p.Ns).T).T.reshape(V.shape)
    FV = LV + p.dR(U) * V
    QF = np.einsum("mj,njs->nms", p.Q, FV)
    prev = np.zeros((p.Nt, p.Ns))
    prev[1:] = V[:-1, -1, :]
    return prev[:, None, :] + p.dt * QF - V


# ------------------------------------------------------------ slab matrices

def slab_jacobian(p: Problem, Un: np.ndarray, dt: float | None = None) -> sp.csr_matrix:
    """dG_n/dU_n = dt (Q (x) I)(I_M (x) L + diag R'(U_n)) - I for one slab."""
    dt = p.dt if dt is None else dt
    M, Ns = p.M, p.Ns
    QI = sp.kron(sp.csr_matrix(p.Q), sp.identity(Ns))
    LL = sp.kron(sp.identity(M), p.L)
    D = sp.diags(p.dR(Un.reshape(M, Ns)).ravel())
    return (dt * (QI @ (LL + D)) - sp.identity(M * Ns)).tocsc()


def full_jacobian_dense(p: Problem, U: np.ndarray) -> np.ndarray:
    """The assembled all-at-once Jacobian (block lower bidiagonal, Eq. 3.4) as a
    dense matrix - for tiny problems only."""
    U = U.reshape(p.Nt, p.M, p.Ns)
    n1 = p.M * p.Ns
    D = p.Nt * n1
    Jd = np.zeros((D, D))
    for n in range(p.Nt):
        Jd[n * n1:(n + 1) * n1, n * n1:(n + 1) * n1] = slab_jacobian(p, U[n]).toarray()
        if n > 0:
            for m in range(p.M):
                r0 = n * n1 + m * p.Ns
                c0 = (n - 1) * n1 + (p.M - 1) * p.Ns
                Jd[r0:r0 + p.Ns, c0:c0 + p.Ns] += np.eye(p.Ns)
    return Jd


# ------------------------------------------------------------------ solves

_DIRECT_MAX = 20000  # slab systems up to this size use sparse LU, larger ones GMRES


def periodic_slab_inverse(p: Problem, c: float, dt: float | None = None,
                          transpose: bool = False) -> spla.LinearOperator:
    """Exact inverse of the constant-coefficient slab matrix
    dt (Q (x) (L + c I)) - I on a periodic grid (the slab Jacobian of Eq. 2.3
    with R'(u) replaced by the constant c).  Q = V diag(mu) V^-1 decouples
    the nodes and the discrete Fourier transform diagonalises the periodic
    FD Laplacian (eigenvalue sum_a (2 cos(2 pi k_a / n_a) - 2) / h_a^2 for
    mode k), so the inverse divides mode k of node q by
    dt mu_q (nu lambda_k + c) - 1.  Used as the preconditioner of the
    Newton steps' Krylov solves on large periodic slabs.  ``transpose``: the
    inverse of the transposed matrix (Q^T in place of Q; the periodic FD
    Laplacian is symmetric), for the adjoint's backward slab solves."""
    dt = p.dt if dt is None else dt
    M, Ns, shape = p.M, p.Ns, p.shape
    mu, V = np.linalg.eig(p.Q.T if transpose else p.Q)
    Vinv = np.linalg.inv(V)
    lam = np.zeros(shape)
    for a, n in enumerate(shape):
        h = space.spacing(space.PERIODIC, n, p.X)
        k = np.arange(n)
        ev = (2.0 * np.cos(2.0 * np.pi * k / n) - 2.0) / (h * h)
        lam = lam + ev.reshape([n if b == a else 1 for b in range(len(shape))])
    denom = dt * mu.reshape((M,) + (1,) * len(shape)) * (p.nu * lam[None] + c) - 1.0
    axes = tuple(range(1, len(shape) + 1))

    def apply(b):
        B = np.asarray(b).reshape((M,) + shape)
        Y = np.fft.fftn(np.tensordot(Vinv, B, axes=1), axes=axes) / denom
        return np.tensordot(V, np.fft.ifftn(Y, axes=axes), axes=1).real.reshape(-1)

    return spla.LinearOperator((M * Ns, M * Ns), matvec=apply, dtype=np.float64)


def slab_jacobian_operator(p: Problem, Un: np.ndarray) -> spla.LinearOperator:
    """dG_n/dU_n (``slab_jacobian``) applied without assembling it:
    v -> dt Q (L v_j + R'(U_{n,j}) v_j)_j - v."""
    M, Ns = p.M, p.Ns
    dR = p.dR(Un.reshape(M, Ns))

    def apply(v):
        V = np.asarray(v).reshape(M, Ns)
        LV = (p.L @ V.T).T
        return (p.dt * (p.Q @ (LV + dR * V)) - V).reshape(-1)

    return spla.LinearOperator((M * Ns, M * Ns), matvec=apply, dtype=np.float64)


class _SlabSolver:
    """Linear solves with one slab Jacobian: sparse LU for small systems;
    restarted GMRES(50) to a 1e-14 relative residual for large ones (the slab
    matrix I - dt Q (x) (L + D) is well conditioned for these step sizes),
    matrix-free, preconditioned on periodic grids by the exact inverse of the
    constant-coefficient slab matrix (``periodic_slab_inverse``)."""

    def __init__(self, p: Problem, Un: np.ndarray):
        self.p, self.Un = p, Un
        n = p.M * p.Ns
        self.lu = spla.splu(slab_jacobian(p, Un)) if n <= _DIRECT_MAX else None
        self.precond = None
        if self.lu is None and p.bc == space.PERIODIC:
            self.precond = periodic_slab_inverse(p, float(np.mean(p.dR(Un))))

    def solve(self, b):
        if self.lu is not None:
            return self.lu.solve(b)
        A = slab_jacobian_operator(self.p, self.Un)
        # preconditioned, the relative residual stalls at its rounding floor
        # (a few 1e-14); the Newton iteration around the solve takes G itself
        # to 1e-14, so a 1e-12 linear solve costs no accuracy
        rtol = 1e-14 if self.precond is None else 1e-12
        x, info = spla.gmres(A, b, rtol=rtol, atol=0.0, restart=50, maxiter=200, M=self.precond)
        if info != 0:
            x = spla.spsolve(slab_jacobian(self.p, self.Un), b)
        return x


def _slab_solver(p: Problem, Un: np.ndarray) -> _SlabSolver:
    return _SlabSolver(p, Un.copy())


def _newton_slab(p: Problem, prev: np.ndarray, guess: np.ndarray, lu_cache: dict | None,
                 tol: float = 1e-14, maxit: int = 40) -> np.ndarray:
    """Newton's method on G_n(U_n) = 0 for one slab given u_{n-1,M} = prev
    (the nonlinear solve of Section 4.2), with backtracking when ||G_n|| grows.
    A linear problem takes one step plus one refinement step."""
    M, Ns = p.M, p.Ns
    Q, dt = p.Q, p.dt
    Un = guess.copy()

    def Gn(V):
        return (prev[None, :] + dt * (Q @ F(p, V)) - V)

    g = Gn(Un)
    scale = max(1.0, float(np.abs(prev).max()), float(np.abs(Un).max()))
    linear = p.reaction == space.NONE
    for it in range(maxit):
        gnorm = float(np.abs(g).max())
        if gnorm <= tol * scale:
            break
        if linear and lu_cache is not None:
            if "lu" not in lu_cache:
                lu_cache["lu"] = _slab_solver(p, Un)
            lu = lu_cache["lu"]
        else:
            lu = _slab_solver(p, Un)
        delta = lu.solve(-g.ravel()).reshape(M, Ns)
        if linear:
            Un = Un + delta
            g = Gn(Un)
            if it >= 1:
                break
            continue
        step = 1.0
        while True:
            trial = Un + step * delta
            gt = Gn(trial)
            if float(np.abs(gt).max()) < gnorm or step < 1e-3:
                break
            step *= 0.5
        if float(np.abs(gt).max()) >= gnorm:
            break  # rounding floor reached
        Un, g = trial, gt
    return Un


def solve_sequential(p: Problem, u0: np.ndarray, nslabs: int | None = None) -> np.ndarray:
    """Solve G(U) = 0 slab by slab, n = 1..Nt (forward substitution in time,
    exact because the system (3.4) is block lower bidiagonal).

    ``nslabs`` < Nt solves only the first slabs; by causality they equal the
    first slabs of the full solution."""
    ns = p.Nt if nslabs is None else nslabs
    U = np.zeros((ns, p.M, p.Ns))
    prev = u0.reshape(-1).astype(np.float64).copy()
    cache: dict = {}
    for n in range(ns):
        U[n] = _newton_slab(p, prev, np.tile(prev, (p.M, 1)), cache)
        prev = U[n, -1].copy()
    return U


def solve_dense(p: Problem, u0: np.ndarray, tol: float = 1e-14, maxit: int = 40) -> np.ndarray:
    """Newton on the assembled all-at-once system with dense LU (tiny sizes)."""
    U = np.zeros((p.Nt, p.M, p.Ns))
    g = residual(p, U, u0)
    scale = max(1.0, float(np.abs(u0).max()))
    for _ in range(maxit):
        if float(np.abs(g).max()) <= tol * scale:
            break
        Jd = full_jacobian_dense(p, U)
        delta = np.linalg.solve(Jd, -g.ravel()).reshape(U.shape)
        step = 1.0
        gn = float(np.abs(g).max())
        while True:
            trial = U + step * delta
            gt = residual(p, trial, u0)
            if float(np.abs(gt).max()) < gn or step < 1e-3:
                break
            step *= 0.5
        if float(np.abs(gt).max()) >= gn:
            break
        U, g = trial, gt
    return U


def dg_solve(p: Problem, u0: np.ndarray) -> np.ndarray:
    """Slab-by-slab Newton solve of the DG form (2.11),
    K U_n = J U_{n-1} + dt Mq F(U_n), with the matrices of ``dg_matrices``."""
    K, Mq, Jm = col.dg_matrices(p.tau)
    M, Ns = p.M, p.Ns
    U = np.zeros((p.Nt, M, Ns))
    prev_block = np.zeros((M, Ns))
    prev_block[-1] = u0.reshape(-1)
    Kk = sp.kron(sp.csr_matrix(K), sp.identity(Ns))
    Mk = sp.kron(sp.csr_matrix(Mq), sp.identity(Ns))
    LL = sp.kron(sp.identity(M), p.L)
    for n in range(p.Nt):
        rhs0 = Jm @ prev_block
        Un = np.tile(prev_block[-1], (M, 1))
        for _ in range(40):
            res = rhs0 + p.dt * (Mq @ F(p, Un)) - K @ Un
            if float(np.abs(res).max()) <= 1e-14 * max(1.0, float(np.abs(Un).max())):
                break
            Jac = (Kk - p.dt * (Mk @ (LL + sp.diags(p.dR(Un).ravel())))).tocsc()
            Un = Un + spla.spsolve(Jac, res.ravel()).reshape(M, Ns)
        U[n] = Un
        prev_block = Un
    return U


# --------------------------------------------------- closed forms (1D heat)

def sine_mode_eigenvalue(k: int, n: int, nu: float, X: float = 1.0) -> float:
    """nu*(2cos(k pi h) - 2)/h^2, eigenvalue of nu*Delta_h on sin(k pi x) with
    Dirichlet interior points (the rho_k of Eq. 5.3 for X = 1)."""
    h = X / (n + 1)
    return nu * (2.0 * np.cos(k * np.pi * h / X) - 2.0) / (h * h)
