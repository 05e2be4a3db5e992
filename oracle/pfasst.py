"""PFASST on the collocation problem (paper Section 4.1: SDC iterations on a
hierarchy of levels with FAS corrections, new initial values passed forward
between time slabs, serial only on the coarsest level; Emmett and Minion
2012).  Oracle: test infrastructure only.  Exact spatial solves, FP64.

Levels l = 0 (finest) .. L-1 share N_t and dt; level l has its own spatial
grid and node count M_l.  One iteration:

  1. on every level from the finest down except the coarsest: IMEX SDC
     sweeps on all slabs at once (each slab starts from the last node of the
     previous slab of the current iterate; u0 for the first), then the
     restriction of the iterate to the next level and the FAS correction
         tau_{l+1} = R(dt Q_l F(U_l) + tau_l) - dt Q_{l+1} F(R U_l),
     which makes R U_l a solution of the coarse equations whenever U_l solves
     the fine ones;
  2. on the coarsest level: the sweeps slab after slab, each slab starting
     from the new last node of the slab before (the serial part);
  3. back up: every level adds the interpolated coarse correction
     P(U_{l+1} - R U_l) and, except the finest, sweeps again.

The level-l equations are U_n = 1 (x) U_{n-1,M} + dt Q_l F(U_n) + tau_{l,n}.
Transfers: full weighting / linear interpolation in space; between node
sets, values and node integrals are restricted by evaluating the fine nodal
polynomial at the coarse nodes and corrections interpolated by evaluating
the coarse nodal polynomial at the fine nodes.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import collocation as col
from . import space
from .system import F, Problem


def node_values(tau_from: np.ndarray, tau_to: np.ndarray) -> np.ndarray:
    """(len(tau_to) x len(tau_from)): the nodal polynomial on tau_from
    evaluated at tau_to."""
    return np.array([[col.lagrange_eval(tau_from, j, t) for j in range(len(tau_from))] for t in tau_to])


class _Level:
    def __init__(self, p: Problem, kind: str):
        self.p = p
        self.QI, self.QE = col.sdc_qdelta(p.tau, kind)
        self.solvers = {}

    def solve(self, a: float, rhs: np.ndarray) -> np.ndarray:
        """(I - a L) x = rhs for every row of rhs (points last)."""
        if a not in self.solvers:
            self.solvers[a] = spla.splu((sp.identity(self.p.Ns) - a * self.p.L).tocsc())
        return self.solvers[a].solve(rhs.T).T

    def integrals(self, U: np.ndarray, tau: np.ndarray | None) -> np.ndarray:
        """dt Q F(U_n) + tau_n for every slab."""
        out = self.p.dt * np.einsum("mj,njs->nms", self.p.Q, F(self.p, U))
        return out if tau is None else out + tau


def sweep_slab(lev: _Level, Un: np.ndarray, U0: np.ndarray, tau_n: np.ndarray | None) -> np.ndarray:
    """One IMEX SDC sweep of one slab (node-to-node standard form, exact
    spatial solves) on U_n = 1 (x) U0 + dt Q F(U_n) + tau_n."""
    p = lev.p
    dt, L = p.dt, p.L
    FU = F(p, Un[None])[0]
    LU = (L @ Un.T).T
    RU = p.R(Un)
    QF = dt * (p.Q @ FU)
    if tau_n is not None:
        QF = QF + tau_n
    new = np.zeros_like(Un)
    for m in range(p.M):
        rhs = U0 + QF[m] - dt * lev.QI[m, m] * LU[m]
        for j in range(m):
            rhs = rhs + dt * lev.QI[m, j] * ((L @ new[j]) - LU[j])
            rhs = rhs + dt * lev.QE[m, j] * (p.R(new[j]) - RU[j])
        new[m] = lev.solve(dt * lev.QI[m, m], rhs[None])[0]
    return new


def sweep_all(lev: _Level, U: np.ndarray, u0: np.ndarray, tau: np.ndarray | None) -> np.ndarray:
    """One sweep on every slab at once (initial values from the iterate)."""
    prev = np.empty((lev.p.Nt, lev.p.Ns))
    prev[0] = u0
    prev[1:] = U[:-1, -1]
    return np.stack([sweep_slab(lev, U[n], prev[n], None if tau is None else tau[n]) for n in range(lev.p.Nt)])


def pfasst(p: Problem, u0: np.ndarray, hierarchy, iters: int, nsweeps=None, kind: str = "IE", U=None):
    """Fine iterates of PFASST.  hierarchy: [(shape, M), ...] finest first
    (the finest entry must match p); nsweeps: sweeps per level (default 1).
    The start iterate (default) spreads u0 over every node and slab.
    Returns the list of fine iterates after each iteration."""
    nl = len(hierarchy)
    nsweeps = nsweeps or [1] * nl
    levs = [_Level(p.with_params(shape=tuple(s), M=M), kind) for s, M in hierarchy]
    same = [levs[l].p.shape == levs[l + 1].p.shape for l in range(nl - 1)]
    Rs = [sp.identity(levs[l].p.Ns, format="csr") if same[l] else space.restriction(p.bc, levs[l].p.shape)
          for l in range(nl - 1)]
    Ps = [sp.identity(levs[l].p.Ns, format="csr") if same[l] else space.prolongation(p.bc, levs[l].p.shape)
          for l in range(nl - 1)]
    Rn = [node_values(levs[l].p.tau, levs[l + 1].p.tau) for l in range(nl - 1)]
    Pn = [node_values(levs[l + 1].p.tau, levs[l].p.tau) for l in range(nl - 1)]

    def restrict(l, V):  # (Nt, M_l, Ns_l) -> (Nt, M_{l+1}, Ns_{l+1})
        Vs = (Rs[l] @ V.reshape(-1, V.shape[-1]).T).T.reshape(V.shape[0], V.shape[1], -1)
        return np.einsum("cf,nfs->ncs", Rn[l], Vs)

    def prolong(l, V):  # (Nt, M_{l+1}, Ns_{l+1}) -> (Nt, M_l, Ns_l)
        Vn = np.einsum("fc,ncs->nfs", Pn[l], V)
        return (Ps[l] @ Vn.reshape(-1, Vn.shape[-1]).T).T.reshape(Vn.shape[0], Vn.shape[1], -1)

    u0s = [np.asarray(u0, dtype=float).reshape(-1)]
    for l in range(nl - 1):
        u0s.append(Rs[l] @ u0s[l])
    Us = [None] * nl
    Us[0] = (np.broadcast_to(u0s[0], (p.Nt, p.M, p.Ns)).copy() if U is None
             else np.asarray(U, dtype=float).reshape(p.Nt, p.M, p.Ns).copy())
    taus = [None] * nl
    out = []
    for _ in range(iters):
        bars = [None] * nl
        for l in range(nl - 1):
            for _s in range(nsweeps[l]):
                Us[l] = sweep_all(levs[l], Us[l], u0s[l], taus[l])
            Uc = restrict(l, Us[l])
            taus[l + 1] = restrict(l, levs[l].integrals(Us[l], taus[l])) - levs[l + 1].integrals(Uc, None)
            Us[l + 1] = Uc
            bars[l + 1] = Uc.copy()
        c = nl - 1
        if c == 0:
            for _s in range(nsweeps[0]):
                Us[0] = sweep_all(levs[0], Us[0], u0s[0], None)
        else:
            Uc = Us[c]
            for n in range(p.Nt):
                U0 = u0s[c] if n == 0 else Uc[n - 1, -1]
                for _s in range(nsweeps[c]):
                    Uc[n] = sweep_slab(levs[c], Uc[n], U0, taus[c][n])
            for l in range(nl - 2, -1, -1):
                Us[l] = Us[l] + prolong(l, Us[l + 1] - bars[l + 1])
                if l > 0:
                    for _s in range(nsweeps[l]):
                        Us[l] = sweep_all(levs[l], Us[l], u0s[l], taus[l])
        out.append(Us[0].copy())
    return out
