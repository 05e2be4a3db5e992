"""Collocation in time (paper Section 2).  Oracle: test infrastructure only.

Everything here works on the reference interval [0, 1]; a slab of length dt
scales Q and the DG mass matrix by dt.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import Polynomial
from numpy.polynomial import legendre as leg


def radau_right_nodes(M: int) -> np.ndarray:
    """The M right Gauss-Radau nodes 0 < tau_1 < ... < tau_M = 1 of Section 2.1.

    They are the roots of P_{M-1}(x) - P_M(x) on [-1, 1] (P_k Legendre),
    mapped by tau = (x + 1)/2.  Roots come from the Legendre companion matrix
    and are polished by Newton's method; tau_M is set to 1 exactly."""
    if M < 1:
        raise ValueError("M >= 1")
    c = np.zeros(M + 1)
    c[M - 1] = 1.0
    c[M] = -1.0
    x = np.sort(np.real(leg.legroots(c)))
    dc = leg.legder(c)
    for _ in range(8):
        x = x - leg.legval(x, c) / leg.legval(x, dc)
    x[-1] = 1.0
    return (x + 1.0) / 2.0


def lagrange_basis(tau: np.ndarray):
    """Lagrange polynomials l_j with l_j(tau_i) = delta_ij (Section 2.1)."""
    polys = []
    for j, tj in enumerate(tau):
        others = np.delete(tau, j)
        p = Polynomial.fromroots(others) if len(others) else Polynomial([1.0])
        polys.append(p / p(tj))
    return polys


def lagrange_eval(tau: np.ndarray, j: int, s):
    """l_j(s) in product form prod_{k != j} (s - tau_k)/(tau_j - tau_k)."""
    s = np.asarray(s, dtype=np.float64)
    out = np.ones_like(s)
    for k, tk in enumerate(tau):
        if k != j:
            out = out * (s - tk) / (tau[j] - tk)
    return out


def _gauss01(npts: int):
    x, w = leg.leggauss(npts)
    return (x + 1) / 2, w / 2


def collocation_matrix(tau: np.ndarray) -> np.ndarray:
    """Q with q_mj = int_0^{tau_m} l_j(s) ds (Eq. 2.3-2.4 on the unit interval).

    Each integral of the degree M-1 polynomial l_j is taken exactly by an
    (M+1)-point Gauss-Legendre rule on [0, tau_m]."""
    M = len(tau)
    x, w = _gauss01(M + 1)
    Q = np.zeros((M, M))
    for m in range(M):
        for j in range(M):
            Q[m, j] = tau[m] * float(w @ lagrange_eval(tau, j, tau[m] * x))
    return Q


def quadrature_weights(tau: np.ndarray) -> np.ndarray:
    """b_j = int_0^1 l_j: the last row of Q for right Radau nodes (Section 2.1)."""
    x, w = _gauss01(len(tau) + 1)
    return np.array([float(w @ lagrange_eval(tau, j, x)) for j in range(len(tau))])


def q_eig(Q: np.ndarray):
    """Eigen-decomposition Q = V diag(lam) V^{-1} (a library routine).

    Ordered: real eigenvalues first (ascending), then each complex eigenvalue
    with Im > 0 (ascending real part) immediately followed by its conjugate."""
    lam, V = np.linalg.eig(Q.astype(complex))
    tol = 1e-12
    real = [i for i in range(len(lam)) if abs(lam[i].imag) <= tol]
    upper = [i for i in range(len(lam)) if lam[i].imag > tol]
    real.sort(key=lambda i: lam[i].real)
    upper.sort(key=lambda i: lam[i].real)
    order = list(real)
    for i in upper:
        j = min((k for k in range(len(lam)) if lam[k].imag < -tol),
                key=lambda k: abs(lam[k] - np.conj(lam[i])))
        order += [i, j]
    lam = lam[order]
    lam[:len(real)] = lam[:len(real)].real
    return lam, V[:, order]


def stability_function(z, Q: np.ndarray) -> complex:
    """R(z) = 1 + z b^T (I - zQ)^{-1} 1: the slab-end amplification of the
    collocation step (2.3) for u' = lambda u, z = dt*lambda (the Runge-Kutta
    stability function of the equivalent Radau IIA method)."""
    M = Q.shape[0]
    b = Q[-1]
    one = np.ones(M)
    return 1.0 + z * (b @ np.linalg.solve(np.eye(M) - z * Q, one))


def stage_amplification(z, Q: np.ndarray) -> np.ndarray:
    """(I - zQ)^{-1} 1: stage values of one collocation step from U_0 = 1."""
    M = Q.shape[0]
    return np.linalg.solve(np.eye(M) - z * Q, np.ones(M))


def dg_matrices(tau: np.ndarray):
    """DG-in-time matrices of Eq. (2.9)-(2.10) on the unit interval.

    K(i,j) = -int l_i' l_j + l_i(1) l_j(1),   Mq(i,j) = int l_i l_j,
    J(i,j) = l_i(0) * delta_{jM}.
    J follows from the upwind flux v(T_n) U_0 of Eq. (2.6) with U_0 the
    previous slab's value at its last node (the previous basis evaluated at
    its right end is delta_{jM}); the integrals are exact Gauss quadratures."""
    M = len(tau)
    ls = lagrange_basis(tau)
    dls = [l.deriv() for l in ls]
    s, w = _gauss01(M + 2)
    Lv = np.array([l(s) for l in ls])
    dLv = np.array([dl(s) for dl in dls])
    K = -(dLv * w) @ Lv.T + np.outer([l(1.0) for l in ls], [l(1.0) for l in ls])
    Mq = (Lv * w) @ Lv.T
    J = np.zeros((M, M))
    J[:, M - 1] = [l(0.0) for l in ls]
    return K, Mq, J


def time_prolongation(tau: np.ndarray) -> np.ndarray:
    """P_t (2M x M): values at the two fine slabs' nodes of the coarse slab's
    nodal polynomial (reading of the time bisection of Section 5.2, STMG).

    Row a*M + j (a = 0 first half, 1 second half) evaluates the coarse
    Lagrange basis at s = (a + tau_j)/2."""
    M = len(tau)
    ls = lagrange_basis(tau)
    P = np.zeros((2 * M, M))
    for a in range(2):
        s = (a + tau) / 2.0
        for m, l in enumerate(ls):
            P[a * M:(a + 1) * M, m] = l(s)
    return P


def time_restriction(tau: np.ndarray) -> np.ndarray:
    """R_t (M x 2M) for residuals of the collocation form.

    The paper restricts the DG system (3.4) with the transpose of the time
    prolongation (Eq. 4.1, time bisection of Section 5.2).  A DG residual is K
    times the collocation residual of the same slab (K of Eq. 2.9 on the
    unit interval), so the same restriction acting on collocation residuals
    is  R_t = K^{-1} P_t^T blockdiag(K, K).  Constants in time are mapped to
    constants on the last node (row M sums to 2, the other rows do not)."""
    K, _, _ = dg_matrices(tau)
    Pt = time_prolongation(tau)
    return np.linalg.solve(K, Pt.T @ np.kron(np.eye(2), K))


def node_prolongation(tau_f: np.ndarray, tau_c: np.ndarray) -> np.ndarray:
    """P_M (M_f x M_c): the coarse slab's nodal polynomial (Lagrange basis on
    the M_c coarse nodes) evaluated at the M_f fine nodes -- the interpolation
    between node sets of the M-coarsening of Section 5.2 (SMMG), same slab."""
    ls = lagrange_basis(tau_c)
    return np.array([[l(t) for l in ls] for t in tau_f])


def node_restriction(tau_f: np.ndarray, tau_c: np.ndarray) -> np.ndarray:
    """R_M (M_c x M_f) for collocation-form residuals: the DG system restricted
    with P_M^T (Eq. 4.1), written for collocation residuals exactly as the
    slab-bisection restriction is, R_M = K_c^{-1} P_M^T K_f."""
    Kf, _, _ = dg_matrices(tau_f)
    Kc, _, _ = dg_matrices(tau_c)
    return np.linalg.solve(Kc, node_prolongation(tau_f, tau_c).T @ Kf)


def sdc_qdelta(tau: np.ndarray, kind: str = "IE"):
    """Lower-triangular SDC preconditioners (Section 4.1).

    Returns (QI, QE): QI implicit (lower triangular incl. diagonal), QE
    explicit (strictly lower), both on the unit interval.
      IE: implicit Euler node to node, QI[m, j] = tau_j - tau_{j-1} (j <= m)
      LU: QI = U^T from the LU factorisation Q^T = L U (no pivoting)
      QE: explicit Euler node to node, QE[m, j] = tau_{j+1} - tau_j (j < m)
    (The explicit term at the slab's left end cancels in correction form.)"""
    M = len(tau)
    dtau = np.diff(np.concatenate([[0.0], tau]))
    QE = np.zeros((M, M))
    for m in range(M):
        for j in range(m):
            QE[m, j] = dtau[j + 1]
    if kind == "IE":
        QI = np.zeros((M, M))
        for m in range(M):
            QI[m, :m + 1] = dtau[:m + 1]
    elif kind == "LU":
        Q = collocation_matrix(tau)
        A = Q.T.copy()
        U = np.zeros((M, M))
        L = np.eye(M)
        for k in range(M):
            U[k, k:] = A[k, k:] - L[k, :k] @ U[:k, k:]
            for i in range(k + 1, M):
                L[i, k] = (A[i, k] - L[i, :k] @ U[:k, k]) / U[k, k]
        QI = U.T
    else:
        raise ValueError(kind)
    return QI, QE
