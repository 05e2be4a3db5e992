"""IMEX spectral deferred correction sweep on the collocation problem (paper
Section 4.1; Eq. 2.3).  Oracle: test infrastructure only.

One sweep updates every slab at once; slab n takes its initial value from the
previous iterate's last node of slab n-1 (u0 for the first slab).  Diffusion
is implicit (QI, lower triangular), the reaction explicit (QE, strictly
lower), as in the semi-implicit sweeps of Section 5.4.  The sweep is written
in its node-to-node standard form with exact spatial solves:

  U^{k+1}_m = U_0 + dt sum_{j<=m} QI_mj L (U^{k+1}_j - U^k_j)
                  + dt sum_{j<m}  QE_mj (R(U^{k+1}_j) - R(U^k_j))
                  + dt sum_j      Q_mj  F(U^k_j).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import collocation as col
from .system import Problem, F


def sdc_sweep(p: Problem, U: np.ndarray, u0: np.ndarray, kind: str = "IE") -> np.ndarray:
    QI, QE = col.sdc_qdelta(p.tau, kind)
    Q, dt, L = p.Q, p.dt, p.L
    U = U.reshape(p.Nt, p.M, p.Ns)
    Unew = np.zeros_like(U)
    prev = np.empty((p.Nt, p.Ns))
    prev[0] = u0.reshape(-1)
    prev[1:] = U[:-1, -1]
    FU = F(p, U)
    LU = (L @ U.reshape(-1, p.Ns).T).T.reshape(U.shape)
    RU = p.R(U)
    QF = np.einsum("mj,njs->nms", Q, FU)
    solvers = {}
    for m in range(p.M):
        key = QI[m, m]
        if key not in solvers:
            solvers[key] = spla.splu((sp.identity(p.Ns) - dt * key * L).tocsc())
        rhs = prev + dt * QF[:, m] - dt * QI[m, m] * LU[:, m]
        for j in range(m):
            LUj_new = (L @ Unew[:, j].T).T
            rhs += dt * QI[m, j] * (LUj_new - LU[:, j])
            rhs += dt * QE[m, j] * (p.R(Unew[:, j]) - RU[:, j])
        Unew[:, m] = solvers[key].solve(rhs.T).T
    return Unew
