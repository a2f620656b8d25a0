"""The alpha-circulant preconditioner and the Richardson iteration, written
out step by step from the paper (oracle; test infrastructure only).

* Lemma 1: E_alpha = V D V^{-1} with V = (1/L) J F, V^{-1} = F^* J^{-1},
  d_l = -alpha^{1/L} exp(-2 pi i (l-1)/L), J = diag(alpha^{-(l-1)/L}),
  [F]_{jk} = exp(2 pi i (j-1)(k-1)/L).
* Eqs. (s1)-(s3): x = (V^{-1} (x) I) r;  block-diagonal solve;  y -> (V (x) I) y.
* Eq. (inner1): block l is ((d_l H_M + I_M) (x) I_N - dT Q (x) A) y_l = x_l,
  solved here directly with a sparse LU (no node diagonalisation, so this
  path shares nothing with the eigenbasis route of eqs. (d1)-(d3)).
* Eq. (Riteration): C_alpha u^{k+1} = (C_alpha - C) u^k + w, or the
  algebraically identical correction form u^{k+1} = u^k + C_alpha^{-1}(w - C u^k).
* Lemma 2 / eq. (QGL): Q G_l^{-1} = Q - r_l D_t H_M with r_l = d_l / (1 + d_l).
  The lemma's printed coefficients correspond to the eigen-equation with
  +r_l t_m h(t_M); eq. (QGL) gives -r_l.  ``lemma2_char_poly`` follows eq.
  (QGL), i.e. the printed coefficients with r -> -r.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from math import factorial

from .collocation import H_matrix
from .operators import apply_C, rhs_w
from .sequential import ordering


def lemma1(L, alpha):
    """Dense (V, Vinv, d) of Lemma 1."""
    j = np.arange(L)
    F = np.exp(2j * np.pi * np.outer(j, j) / L)
    J = np.diag(alpha ** (-j / L))
    Jinv = np.diag(alpha ** (j / L))
    V = J @ F / L
    Vinv = F.conj().T @ Jinv
    d = -alpha ** (1.0 / L) * np.exp(-2j * np.pi * j / L)
    return V, Vinv, d


def eigenvalues_d(L, alpha):
    """d_l = -alpha^{1/L} exp(-2 pi i (l-1)/L), l = 1..L (Lemma 1)."""
    j = np.arange(L)
    return -alpha ** (1.0 / L) * np.exp(-2j * np.pi * j / L)


def time_forward(r, alpha):
    """x = (V^{-1} (x) I) r = F^* J^{-1} r along axis 0 (eq. (s1)).
    F^* applied to a vector is numpy's forward FFT."""
    L = r.shape[0]
    s = alpha ** (np.arange(L) / L)
    return np.fft.fft(s.reshape((L,) + (1,) * (r.ndim - 1)) * r, axis=0)


def time_inverse(y, alpha):
    """u = (V (x) I) y = (1/L) J F y along axis 0 (eq. (s3)).
    (1/L) F applied to a vector is numpy's inverse FFT."""
    L = y.shape[0]
    s = alpha ** (-np.arange(L) / L)
    return s.reshape((L,) + (1,) * (y.ndim - 1)) * np.fft.ifft(y, axis=0)


def block_matrix(A, Q, dT, d):
    """(d H_M + I_M) (x) I_N - dT Q (x) A of eq. (inner1)."""
    M, N = Q.shape[0], A.shape[0]
    G = d * H_matrix(M) + np.eye(M)
    return (sp.kron(sp.csr_matrix(G), sp.identity(N)) - dT * sp.kron(Q, A)).tocsc()


def precond_solve(A, Q, dT, alpha, r):
    """e = C_alpha^{-1} r for r of shape (L, M, N), by eqs. (s1)-(s3) with
    eq. (inner1) solved per block.  Returns complex128 (real up to rounding
    for real r)."""
    L, M, N = r.shape
    x = time_forward(r.astype(np.complex128), alpha)
    d = eigenvalues_d(L, alpha)
    y = np.empty_like(x)
    for l in range(L):
        # the block has the sparsity pattern of C_coll: the same ordering
        lu = spla.splu(block_matrix(A, Q, dT, d[l]).astype(np.complex128), permc_spec=ordering(A))
        y[l] = lu.solve(x[l].reshape(-1)).reshape(M, N)
    return time_inverse(y, alpha)


def richardson(A, Q, dT, L, u0, alphas, form="correction", u_init=None, b=None):
    """Iterates of eq. (Riteration) for the given alpha_k sequence.

    form = "paper":      u^{k+1} = C_alpha^{-1} ((C_alpha - C) u^k + w), where
                         (C_alpha - C) u^k is -alpha H u^k_L in block 1 only.
    form = "correction": u^{k+1} = u^k + C_alpha^{-1} (w - C u^k).
    Initial iterate u^{(0)} = (u_0, ..., u_0) (Sec. 5) unless u_init given.
    Returns the list [u^{(0)}, u^{(1)}, ...] (real parts)."""
    M, N = Q.shape[0], A.shape[0]
    w = rhs_w(u0, L, M, b)
    u = np.broadcast_to(np.asarray(u0, np.float64), (L, M, N)).copy() if u_init is None \
        else np.array(u_init, dtype=np.float64)
    out = [u.copy()]
    for alpha in alphas:
        if form == "paper":
            rhs = w.copy()
            rhs[0] += -alpha * u[L - 1, M - 1][None, :]
            u = precond_solve(A, Q, dT, alpha, rhs).real
        else:
            r = w - apply_C(u, A, Q, dT)
            u = u + precond_solve(A, Q, dT, alpha, r).real
        out.append(u.copy())
    return out


def QGinv(Q, t, d):
    """Q G_l^{-1} = Q - r D_t H_M with r = d / (1 + d) (eq. (QGL))."""
    r = d / (1.0 + d)
    return Q - r * np.diag(t) @ H_matrix(len(t))


def lemma2_char_poly(t, r):
    """Coefficients [c_0, ..., c_M] (c_M = M!) of the scaled characteristic
    polynomial of Q - r D_t H_M (Lemma 2 with the sign of eq. (QGL)):
        c_0 = (1 - r) b_0,
        c_m = m! b_m + r sum_{j=1}^{M-m} (m+j)!/j! b_{m+j},  1 <= m <= M-1,
    where w_M(t) = prod (t - t_m) = sum_m b_m t^m, b_M = 1."""
    M = len(t)
    b = np.poly(t)[::-1]          # b[m] = coefficient of t^m, b[M] = 1
    c = np.zeros(M + 1, dtype=np.result_type(r, np.float64))
    c[0] = (1 - r) * b[0]
    for m in range(1, M):
        c[m] = factorial(m) * b[m] + r * sum(
            factorial(m + j) / factorial(j) * b[m + j] for j in range(1, M - m + 1))
    c[M] = factorial(M)
    return c
