"""Pins of oracle.collocation against closed forms (paper Section 2, textbook
Radau IIA facts).  CPU only."""
import math
import os

import numpy as np
import pytest

from oracle import collocation as col

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_radau3():
    vals = {}
    with open(os.path.join(GOLDEN, "radau_iia_m3.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, _, val = line.split()
            vals[key] = float(val)
    return vals


def test_nodes_closed_forms():
    assert np.allclose(col.radau_right_nodes(1), [1.0], atol=0)
    assert np.allclose(col.radau_right_nodes(2), [1 / 3, 1.0], atol=1e-15)
    s6 = math.sqrt(6.0)
    assert np.allclose(col.radau_right_nodes(3), [(4 - s6) / 10, (4 + s6) / 10, 1.0], atol=1e-15)


@pytest.mark.parametrize("M", [1, 2, 3, 4, 5])
def test_radau_quadrature_degree(M):
    """Right Radau quadrature is exact for degree 2M-2 and not for 2M-1."""
    tau = col.radau_right_nodes(M)
    b = col.quadrature_weights(tau)
    for k in range(2 * M - 1):
        assert abs(b @ tau ** k - 1.0 / (k + 1)) < 1e-14
    assert abs(b @ tau ** (2 * M - 1) - 1.0 / (2 * M)) > 1e-6
    assert tau[-1] == 1.0 and np.all(np.diff(tau) > 0) and tau[0] > 0


def test_q_m2_exact():
    Q = col.collocation_matrix(col.radau_right_nodes(2))
    assert np.allclose(Q, [[5 / 12, -1 / 12], [3 / 4, 1 / 4]], atol=1e-15)


def test_q_m3_golden():
    g = _golden_radau3()
    Q = col.collocation_matrix(col.radau_right_nodes(3))
    for i in range(3):
        for j in range(3):
            assert abs(Q[i, j] - g[f"a{i + 1}{j + 1}"]) < 2e-15


@pytest.mark.parametrize("M", [1, 2, 3, 4, 5])
def test_q_simplifying_assumption(M):
    """Collocation integrates polynomials of degree < M exactly on every
    sub-interval: Q tau^{k-1} = tau^k / k for k = 1..M; the last row is b."""
    tau = col.radau_right_nodes(M)
    Q = col.collocation_matrix(tau)
    for k in range(1, M + 1):
        assert np.abs(Q @ tau ** (k - 1) - tau ** k / k).max() < 1e-14
    assert np.abs(Q[-1] - col.quadrature_weights(tau)).max() < 1e-15
    assert np.abs(Q.sum(axis=1) - tau).max() < 1e-15


# Pade (M-1, M) approximants of exp: the stability functions of Radau IIA
PADE = {
    1: (lambda z: 1.0, lambda z: 1 - z),
    2: (lambda z: 1 + z / 3, lambda z: 1 - 2 * z / 3 + z * z / 6),
    3: (lambda z: 1 + 2 * z / 5 + z * z / 20, lambda z: 1 - 3 * z / 5 + 3 * z * z / 20 - z ** 3 / 60),
}
PADE_DEN_COEFFS = {  # numpy.roots order, highest power first
    1: [-1.0, 1.0],
    2: [1 / 6, -2 / 3, 1.0],
    3: [-1 / 60, 3 / 20, -3 / 5, 1.0],
}


@pytest.mark.parametrize("M", [1, 2, 3])
def test_stability_function_is_pade(M):
    Q = col.collocation_matrix(col.radau_right_nodes(M))
    num, den = PADE[M]
    for z in [-0.3, -2.0, -50.0, 0.7j - 1.0, -1e3 + 5j]:
        assert abs(col.stability_function(z, Q) - num(z) / den(z)) < 1e-13 * max(1, abs(num(z) / den(z)))


@pytest.mark.parametrize("M", [1, 2, 3])
def test_q_eigenvalues_pade_roots(M):
    Q = col.collocation_matrix(col.radau_right_nodes(M))
    lam, V = col.q_eig(Q)
    roots = np.roots(PADE_DEN_COEFFS[M])
    expect = 1.0 / roots
    for e in expect:  # every Pade-denominator root's reciprocal is an eigenvalue
        assert np.abs(lam - e).min() < 1e-13
    assert len(lam) == len(expect)
    assert np.abs(Q @ V - V @ np.diag(lam)).max() < 1e-14
    if M == 3:
        real = lam[np.abs(lam.imag) < 1e-12].real
        assert abs(real[0] - 1 / 3.6378342527444957) < 1e-12


@pytest.mark.parametrize("M", [1, 2, 3, 4, 5])
def test_dg_equals_collocation_matrices(M):
    """DG in time (Eq. 2.8-2.10) and collocation (Eq. 2.3) define the same
    step: Mq^{-1} K = Q^{-1} and K 1 = l(0) (the J column)."""
    tau = col.radau_right_nodes(M)
    K, Mq, J = col.dg_matrices(tau)
    Q = col.collocation_matrix(tau)
    rel = np.abs(np.linalg.solve(Mq, K) - np.linalg.inv(Q)).max() / np.abs(np.linalg.inv(Q)).max()
    assert rel < 1e-12
    assert np.abs(K @ np.ones(M) - J[:, M - 1]).max() < 1e-13
    if M == 2:
        assert np.allclose(J[:, 1], [1.5, -0.5], atol=1e-14)


@pytest.mark.parametrize("M", [1, 2, 3])
def test_order_2m_minus_1(M):
    """|R(dt*lam)^Nt - e^{lam T}| falls at order 2M-1 (Section 2.1; Fig. 5.1)."""
    Q = col.collocation_matrix(col.radau_right_nodes(M))
    lam, T = -1.0, 1.0
    errs = []
    Nts = [4, 8, 16, 32]
    for Nt in Nts:
        R = col.stability_function(lam * T / Nt, Q)
        errs.append(abs(R ** Nt - math.exp(lam * T)))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert abs(slopes[-1] - (2 * M - 1)) < 0.15


@pytest.mark.parametrize("M", [1, 2, 3, 4])
def test_time_transfers(M):
    tau = col.radau_right_nodes(M)
    P = col.time_prolongation(tau)
    R = col.time_restriction(tau)
    # the coarse slab's polynomial of degree < M is reproduced at the fine nodes
    for k in range(M):
        coarse = tau ** k
        fine_t = np.concatenate([tau / 2, (1 + tau) / 2])
        assert np.abs(P @ coarse - fine_t ** k).max() < 1e-13
    # R_t is P_t^T acting on DG residuals K r (Eq. 2.9): K R = P^T blockdiag(K, K)
    K, _, _ = col.dg_matrices(tau)
    assert np.abs(K @ R - P.T @ np.kron(np.eye(2), K)).max() < 1e-12
    # a DG residual supported on one fine slab's node keeps its total weight
    # against the coarse constant test function (Galerkin restriction property)
    one = np.ones(M)
    for k in range(2 * M):
        v = np.zeros(2 * M)
        v[k] = 1.0
        assert abs(one @ (K @ (R @ v)) - np.ones(2 * M) @ (np.kron(np.eye(2), K) @ v)) < 1e-12


def _two_slab_operator(M, Q, dt, lam):
    """-dG/dU of the scalar problem u' = lam u over two slabs of length dt/2
    (the collocation form of Eq. 2.3 on each, chained by the slab coupling
    of Eq. 3.4): [[I - (dt/2) lam Q, 0], [-1 e_M^T, I - (dt/2) lam Q]]."""
    I = np.eye(M)
    eM = np.eye(M)[-1]
    B = I - 0.5 * dt * lam * Q
    return np.block([[B, np.zeros((M, M))], [-np.outer(np.ones(M), eM), B]])


LAMBDAS = (-3.7, 0.8, -50.0, 2.0 + 1.5j, -1.0e3, -0.25 - 4.0j)


@pytest.mark.parametrize("M", [1, 2, 3, 4, 5])
def test_time_restriction_galerkin_identity(M):
    """Slab bisection is a Galerkin coarsening (the DG spaces of Eq. 2.9 on
    the coarse slab are a subspace of those on its two halves, and the DG
    form integrates polynomials exactly), so for the scalar problem
    u' = lam u the restricted two-half-slab operator is the coarse slab's
    collocation operator:  R_t A_f P_t = A_c = I - dt lam Q, for real
    negative, positive and complex lam.  The data entering a coarse slab
    from its predecessor (1 (x) u_prev on the first half) restricts to the
    coarse slab's own coupling (1 (x) u_prev)."""
    tau = col.radau_right_nodes(M)
    Q = col.collocation_matrix(tau)
    P = col.time_prolongation(tau)
    R = col.time_restriction(tau)
    dt = 0.37
    for lam in LAMBDAS:
        Ac = np.eye(M) - dt * lam * Q
        got = R @ _two_slab_operator(M, Q, dt, lam) @ P
        assert np.abs(got - Ac).max() <= 1e-12 * np.abs(Ac).max(), lam
    inflow = R @ np.concatenate([np.ones(M), np.zeros(M)])
    assert np.abs(inflow - 1.0).max() < 1e-12


@pytest.mark.parametrize("M", [2, 3, 5])
def test_time_restriction_galerkin_identity_rejects_wrong_forms(M):
    """Plausible mistakes in R_t = K^-1 P_t^T blockdiag(K, K) break the
    Galerkin identity: P_t^T alone (rows rescaled to keep constants), K
    applied on the wrong side, and the two fine slabs' blocks swapped."""
    tau = col.radau_right_nodes(M)
    Q = col.collocation_matrix(tau)
    P = col.time_prolongation(tau)
    K, _, _ = col.dg_matrices(tau)
    dt, lam = 0.37, -3.7
    Af = _two_slab_operator(M, Q, dt, lam)
    Ac = np.eye(M) - dt * lam * Q
    swap = np.block([[np.zeros((M, M)), np.eye(M)], [np.eye(M), np.zeros((M, M))]])
    wrong = {
        "P^T row-normalised": P.T / P.T.sum(axis=1, keepdims=True),
        "K on the wrong side": K @ P.T @ np.kron(np.eye(2), np.linalg.inv(K)),
        "halves swapped": col.time_restriction(tau) @ swap,
    }
    for name, Rw in wrong.items():
        assert np.abs(Rw @ Af @ P - Ac).max() > 1e-6, name


@pytest.mark.parametrize("kind", ["IE", "LU"])
@pytest.mark.parametrize("M", [1, 2, 3, 5])
def test_sdc_qdelta(kind, M):
    tau = col.radau_right_nodes(M)
    QI, QE = col.sdc_qdelta(tau, kind)
    assert np.allclose(np.triu(QI, 1), 0) and np.allclose(np.triu(QE), 0)
    if kind == "IE":
        # implicit Euler node to node integrates constants exactly: row sums = tau
        assert np.abs(QI.sum(axis=1) - tau).max() < 1e-15
    else:
        # Q^T = L U with unit-lower L: Q^T - QI^T is strictly lower (U = QI^T)
        Q = col.collocation_matrix(tau)
        Lm = np.linalg.solve(QI, Q).T  # L = Q^T U^{-1} = (QI^{-1} Q)^T
        assert np.allclose(np.diag(Lm), 1.0)
        assert np.allclose(np.triu(Lm, 1), 0, atol=1e-13)
    # explicit Euler from node j to node j+1 (strictly lower; row sums tau - tau_1)
    assert np.abs(QE.sum(axis=1) - (tau - tau[0])).max() < 1e-15


# ---------------------------------------------------------------- M-coarsening

@pytest.mark.parametrize("Mf,Mc", [(2, 1), (3, 2), (4, 3), (5, 4), (5, 2), (3, 1)])
def test_node_prolongation_interpolates_polynomials(Mf, Mc):
    """P_M reproduces every polynomial of degree < M_c from its coarse node
    values, and keeps the slab-end node (tau = 1 is a node of both sets)."""
    tf, tc = col.radau_right_nodes(Mf), col.radau_right_nodes(Mc)
    P = col.node_prolongation(tf, tc)
    for deg in range(Mc):
        assert np.abs(P @ tc ** deg - tf ** deg).max() < 1e-13
    assert np.abs(P[-1] - np.eye(Mc)[-1]).max() < 1e-14


@pytest.mark.parametrize("Mf,Mc", [(2, 1), (3, 2), (4, 3), (5, 4), (5, 2), (3, 1)])
def test_node_restriction_is_left_inverse(Mf, Mc):
    """The coarse polynomials are a subspace of the fine ones and the DG form
    is integrated exactly, so P^T K_f P = K_c and R_M P_M = I."""
    tf, tc = col.radau_right_nodes(Mf), col.radau_right_nodes(Mc)
    P = col.node_prolongation(tf, tc)
    Kf, _, _ = col.dg_matrices(tf)
    Kc, _, _ = col.dg_matrices(tc)
    assert np.abs(P.T @ Kf @ P - Kc).max() < 1e-12
    assert np.abs(col.node_restriction(tf, tc) @ P - np.eye(Mc)).max() < 1e-12


@pytest.mark.parametrize("Mf", [2, 3, 5])
def test_node_restriction_to_one_node_takes_the_last_residual(Mf):
    """M_c = 1: K_c = 1 and the column sums of K_f are l_j(1) = delta_{jM}
    (sum_i l_i = 1), so R_M = e_M^T."""
    R = col.node_restriction(col.radau_right_nodes(Mf), col.radau_right_nodes(1))
    assert np.abs(R - np.eye(Mf)[-1:]).max() < 1e-12
