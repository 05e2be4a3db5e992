"""Level operators, transfers and the exact coarse solve of the space-time
multigrid (paper Section 4.2, Eq. 4.1).  Oracle: test infrastructure only.

A level l carries its own grid (shape, Nt_l, dt_l) and a per-slab, per-point
reaction coefficient cbar_l (Nt_l, Ns_l).  Its linear operator is the slab
Jacobian with the reaction derivative averaged over the nodes:

    (A_l e)_n = e_n - dt_l (Q (x) (nu*Delta_{h_l} + diag cbar_{l,n})) e_n,
    (C e)_n   = 1 (x) e_{n-1,M}    (e_{-1} = 0),

and a correction e at level l solves  A_l e - C e = r.  On the finest level
with cbar = mean_m R'(U_{n,m}) this is -dG/dU up to the node averaging; for a
linear problem it is exactly -dG/dU.

Transfers are Eq. (4.1) with the mass-coarsening factor fixed to the
identity: either S (x) I_t (spatial full weighting / linear interpolation) or
I_s (x) T (slab bisection, ``collocation.time_restriction``).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import collocation as col
from . import space


@dataclass
class Level:
    shape: tuple     # numpy order
    bc: int
    Nt: int
    M: int
    dt: float
    nu: float
    X: float
    cbar: np.ndarray  # (Nt, Ns)
    # optional R'(U) at every node, (Nt, M, Ns): the finest level's operator
    # is then the exact Jacobian, A e - C e = -dG/dU e; slab solves keep cbar
    cnode: np.ndarray | None = None

    @property
    def Ns(self):
        return int(np.prod(self.shape))

    @property
    def Q(self):
        return col.collocation_matrix(col.radau_right_nodes(self.M))

    @property
    def L(self):
        return (self.nu * space.laplacian(self.bc, self.shape, self.X)).tocsr()


def _apply_L(L, E):
    return (L @ E.reshape(-1, L.shape[0]).T).T.reshape(E.shape)


def apply_A(lev: Level, e: np.ndarray) -> np.ndarray:
    """A_l e (block diagonal part, no slab coupling); with cnode the reaction
    term of node j is R'(U_{n,j}) e_j instead of cbar_n e_j."""
    e = e.reshape(lev.Nt, lev.M, lev.Ns)
    c = lev.cbar[:, None, :] if lev.cnode is None else lev.cnode.reshape(e.shape)
    Fe = _apply_L(lev.L, e) + c * e
    return e - lev.dt * np.einsum("mj,njs->nms", lev.Q, Fe)


def coupling(lev: Level, e: np.ndarray) -> np.ndarray:
    """(C e)_n = 1 (x) e_{n-1,M}."""
    e = e.reshape(lev.Nt, lev.M, lev.Ns)
    out = np.zeros_like(e)
    out[1:] = e[:-1, -1:, :]
    return out


def linear_residual(lev: Level, e: np.ndarray, r: np.ndarray) -> np.ndarray:
    """r - A_l e + C e."""
    return r.reshape(lev.Nt, lev.M, lev.Ns) - apply_A(lev, e) + coupling(lev, e)


def apply_AT(lev: Level, e: np.ndarray) -> np.ndarray:
    """A_l^T e: (A^T e)_j = e_j - dt_l sum_m Q_mj (L_l + diag cbar_n) e_m
    (L_l symmetric for DIRICHLET and PERIODIC)."""
    e = e.reshape(lev.Nt, lev.M, lev.Ns)
    Fe = _apply_L(lev.L.T.tocsr(), e) + lev.cbar[:, None, :] * e
    return e - lev.dt * np.einsum("mj,nms->njs", lev.Q, Fe)


def coupling_T(lev: Level, e: np.ndarray) -> np.ndarray:
    """(C^T e)_n: the last node of slab n receives sum_m e_{n+1,m}."""
    e = e.reshape(lev.Nt, lev.M, lev.Ns)
    out = np.zeros_like(e)
    out[:-1, -1, :] = e[1:].sum(axis=1)
    return out


def linear_residual_T(lev: Level, e: np.ndarray, r: np.ndarray) -> np.ndarray:
    """r - A_l^T e + C^T e (the transposed level system of the adjoint)."""
    return r.reshape(lev.Nt, lev.M, lev.Ns) - apply_AT(lev, e) + coupling_T(lev, e)


def coarse_solve_exact_T(lev: Level, r: np.ndarray) -> np.ndarray:
    """Exact solution of A_l^T e - C^T e = r by backward substitution."""
    r = r.reshape(lev.Nt, lev.M, lev.Ns)
    e = np.zeros_like(r)
    nxt = np.zeros(lev.Ns)
    for n in range(lev.Nt - 1, -1, -1):
        rhs = r[n].copy()
        rhs[-1] += nxt
        e[n] = spla.spsolve(slab_matrix(lev, n).T.tocsc(), rhs.ravel()).reshape(lev.M, lev.Ns)
        nxt = e[n].sum(axis=0)
    return e


def slab_matrix(lev: Level, n: int) -> sp.csc_matrix:
    """A_{l,n} = I - dt_l Q (x) (L_l + diag cbar_{l,n}) as a sparse matrix."""
    Ln = lev.L + sp.diags(lev.cbar[n])
    return (sp.identity(lev.M * lev.Ns) - lev.dt * sp.kron(sp.csr_matrix(lev.Q), Ln)).tocsc()


def coarse_solve_exact(lev: Level, r: np.ndarray) -> np.ndarray:
    """Exact solution of A_l e - C e = r by forward substitution over slabs."""
    r = r.reshape(lev.Nt, lev.M, lev.Ns)
    e = np.zeros_like(r)
    prev = np.zeros(lev.Ns)
    for n in range(lev.Nt):
        rhs = r[n] + prev[None, :]
        e[n] = spla.spsolve(slab_matrix(lev, n), rhs.ravel()).reshape(lev.M, lev.Ns)
        prev = e[n, -1]
    return e


def smoothing_step_exact(lev: Level, e: np.ndarray, r: np.ndarray, omega: float) -> np.ndarray:
    """Damped block Jacobi in time with exact slab solves (one block per slab,
    the Cores = Nt case of Section 4.2): e + omega * A_n^{-1}(r - A e + C e).
    Parity unpinned: the weight omega is a solver parameter, not paper content."""
    res = linear_residual(lev, e, r)
    out = e.reshape(res.shape).copy()
    for n in range(lev.Nt):
        out[n] += omega * spla.spsolve(slab_matrix(lev, n), res[n].ravel()).reshape(lev.M, lev.Ns)
    return out


def smoothing_step_jacobi(lev: Level, e: np.ndarray, r: np.ndarray, omega: float, sweeps: int,
                          omega_j: float) -> np.ndarray:
    """Damped block Jacobi in time whose slab solves are replaced by ``sweeps``
    weighted-Jacobi sweeps (weight omega_j, zero start) on the M systems that
    the eigen-decomposition Q = V diag(lambda) V^{-1} decouples:

        (I - dt lambda_q (L + diag cbar_n)) z_q = (V^{-1} res_n)_q,

    then e_n += omega * Re(V z).  Complex arithmetic throughout.
    Parity unpinned: the sweep count and weights are solver parameters.  It
    tends to ``smoothing_step_exact`` as sweeps grows, and equals it after one
    sweep with omega_j = 1 when L + diag cbar vanishes."""
    res = linear_residual(lev, e, r)
    lam, V = np.linalg.eig(lev.Q)
    Vinv = np.linalg.inv(V)
    out = e.reshape(res.shape).copy()
    Ldiag = lev.L.diagonal()
    I = sp.identity(lev.Ns, format="csr")
    for n in range(lev.Nt):
        Ln = (lev.L + sp.diags(lev.cbar[n])).tocsr()
        Y = Vinv @ res[n]
        Z = np.zeros_like(Y, dtype=complex)
        for q in range(lev.M):
            s = lev.dt * lam[q]
            Aq = I - s * Ln
            d = 1.0 - s * (Ldiag + lev.cbar[n])
            for _ in range(sweeps):
                Z[q] = Z[q] + omega_j * (Y[q] - Aq @ Z[q]) / d
        out[n] += omega * (V @ Z).real
    return out


# -------------------------------------------------------------- transfers

def restrict_space(bc: int, shape, v: np.ndarray) -> np.ndarray:
    """Full weighting of every (slab, node) plane; v has shape (..., Ns)."""
    R = space.restriction(bc, shape)
    lead = v.shape[:-1]
    return (R @ v.reshape(-1, v.shape[-1]).T).T.reshape(*lead, R.shape[0])


def prolong_space(bc: int, shape, v: np.ndarray) -> np.ndarray:
    """Linear interpolation of every plane to the fine grid ``shape``."""
    P = space.prolongation(bc, shape)
    lead = v.shape[:-1]
    return (P @ v.reshape(-1, v.shape[-1]).T).T.reshape(*lead, P.shape[0])


def restrict_nodes(Mf: int, Mc: int, v: np.ndarray) -> np.ndarray:
    """M-coarsening restriction of every (slab, point): (Nt, Mf, Ns) -> (Nt, Mc, Ns)."""
    R = col.node_restriction(col.radau_right_nodes(Mf), col.radau_right_nodes(Mc))
    return np.einsum("cf,nfs->ncs", R, v)


def prolong_nodes(Mf: int, Mc: int, v: np.ndarray) -> np.ndarray:
    """(Nt, Mc, Ns) -> (Nt, Mf, Ns) with P_M."""
    P = col.node_prolongation(col.radau_right_nodes(Mf), col.radau_right_nodes(Mc))
    return np.einsum("fc,ncs->nfs", P, v)


def restrict_time(M: int, v: np.ndarray) -> np.ndarray:
    """Slab bisection restriction: (Nt, M, Ns) -> (Nt/2, M, Ns) with R_t."""
    Nt, _, Ns = v.shape
    Rt = col.time_restriction(col.radau_right_nodes(M))
    pairs = v.reshape(Nt // 2, 2 * M, Ns)
    return np.einsum("mk,nks->nms", Rt, pairs)


def prolong_time(M: int, v: np.ndarray) -> np.ndarray:
    """(Nt/2, M, Ns) -> (Nt, M, Ns) with P_t."""
    Nc, _, Ns = v.shape
    Pt = col.time_prolongation(col.radau_right_nodes(M))
    return np.einsum("km,nms->nks", Pt, v).reshape(2 * Nc, M, Ns)


def restrict_space_time(bc: int, shape, M: int, v: np.ndarray) -> np.ndarray:
    """Space and slab bisection on one level (the STMG hierarchy of Section
    5.2): full weighting of every plane, then the slab restriction.  The two
    act on different indices, so their order does not matter.
    (Nt, M, Ns) -> (Nt/2, M, Ns_coarse)."""
    return restrict_time(M, restrict_space(bc, shape, v))


def prolong_space_time(bc: int, shape, M: int, v: np.ndarray) -> np.ndarray:
    """(Nt/2, M, Ns_coarse) -> (Nt, M, Ns): P_t on the coarse grid, then
    linear interpolation to the fine grid ``shape``."""
    return prolong_space(bc, shape, prolong_time(M, v))


def restrict_cbar_space(bc: int, shape, cb: np.ndarray) -> np.ndarray:
    return restrict_space(bc, shape, cb)


def restrict_cbar_time(cb: np.ndarray) -> np.ndarray:
    """Average of the two fine slabs' coefficients.  Parity unpinned: how the
    coarse levels' reaction coefficient is formed is solver design (any
    choice leaves the converged solution unchanged)."""
    return 0.5 * (cb[0::2] + cb[1::2])
