"""Radau IIA collocation nodes and the collocation matrix Q (oracle; test
infrastructure only).

Paper, Sec. 2.1 eq. (collocation): q_{mi} = int_0^{t_m} c_i(s) ds with c_i the
Lagrange polynomials on the nodes t_1 < ... < t_M.  Sec. 2.3 (discussion after
Lemma 2): the Radau nodes are the roots of R_M = P_{M-1} + P_M (Legendre
polynomials) on [-1, 1], mapped to [0, 1] with x(t) = -2t + 1, so that the
right end point t_M = 1 is a node.
"""
import numpy as np
from numpy.polynomial import Polynomial, legendre


def radau_iia_nodes(M):
    """Nodes 0 < t_1 < ... < t_M = 1 of Radau IIA collocation (Sec. 2.3).

    Roots of P_{M-1} + P_M in x, then t = (1 - x) / 2.  Each root is polished
    with a few Newton steps on the Legendre series itself.
    """
    if M < 1:
        raise ValueError("M >= 1")
    coef = np.zeros(M + 1)
    coef[M] = 1.0
    coef[M - 1] += 1.0
    x = legendre.legroots(coef)
    dcoef = legendre.legder(coef)
    for _ in range(3):
        x = x - legendre.legval(x, coef) / legendre.legval(x, dcoef)
    t = np.sort((1.0 - np.real(x)) / 2.0)
    t[-1] = 1.0  # x = -1 is an exact root of P_{M-1} + P_M
    return t


def lagrange_basis(t, i):
    """The i-th Lagrange polynomial c_i on nodes t, as a numpy Polynomial."""
    p = Polynomial([1.0])
    for j, tj in enumerate(t):
        if j != i:
            p = p * Polynomial([-tj, 1.0]) / (t[i] - tj)
    return p


def collocation_matrix(t):
    """Q with q_{mi} = int_0^{t_m} c_i(s) ds (eq. (collocation)), by exact
    integration of each Lagrange polynomial."""
    t = np.asarray(t, dtype=np.float64)
    M = len(t)
    Q = np.empty((M, M))
    for i in range(M):
        ci = lagrange_basis(t, i).integ()   # antiderivative with value 0 at 0
        Q[:, i] = ci(t)
    return Q


def H_matrix(M):
    """H_M of eq. (Hm): ones in the last column, zeros elsewhere."""
    H = np.zeros((M, M))
    H[:, -1] = 1.0
    return H
